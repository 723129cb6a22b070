"""The network's product on tcgen05 (tensor-memory accumulators; loader
warps and an MMA-issuing thread linked by mbarriers) against the mma.sync
kernel and an FP64 reference of the same BF16 operands, on one tile, K loops
that wrap the stage ring, several tiles in M and N, each tile width, and the
network's widest K; then the whole network's gradients on the tcgen05 path
against the FP64 oracle."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1312_3039_gb300 import build, scs
    build.build()
    return torch, scs


# tiles of 64 (N = 64, 192, 4416), 128 (N = 384) and 256 columns (N = 512, 768,
# 2048); K from one k-block to 70 (the stage ring wraps many times); the last
# two shapes have more tiles than SMs, so CTAs walk several tiles and
# alternate their two tensor-memory accumulators
@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (128, 64, 512), (384, 192, 256), (128, 384, 1024),
                                   (256, 512, 4480), (384, 768, 192), (6144, 2048, 128), (2560, 4416, 64)])
def test_tcgen05_product(env, M, N, K):
    torch, scs = env
    rng = np.random.default_rng(M + N + K)
    A = torch.tensor(rng.standard_normal((M, K)), dtype=torch.bfloat16, device="cuda")
    B = torch.tensor(rng.standard_normal((N, K)), dtype=torch.bfloat16, device="cuda")
    ref = A.double().cpu().numpy() @ B.double().cpu().numpy().T
    out = {}
    for tc in (0, 1):
        C = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        rc = scs.lib().scs_bf16_gemm(A.data_ptr(), K, B.data_ptr(), K, M, N, K, C.data_ptr(), N, tc, None)
        assert rc == 0, (tc, rc, scs.last_error())
        out[tc] = C.cpu().numpy().astype(np.float64)
    scale = np.abs(ref).max()
    np.testing.assert_allclose(out[1], ref, rtol=0, atol=1e-5 * scale * np.sqrt(K / 64))
    np.testing.assert_allclose(out[1], out[0], rtol=0, atol=1e-5 * scale * np.sqrt(K / 64))


def test_network_gradients_on_tcgen05(env):
    torch, scs = env
    rng = np.random.default_rng(7)
    sizes = [64, 512, 512, 512, 4406]
    B = 128
    params = omlp.init_params(rng, sizes)
    params = [(W, rng.standard_normal(b.shape) * 0.05) for W, b in params]
    X = rng.standard_normal((B, 64))
    T = rng.standard_normal((B, 4406))
    pr = [(omlp.bf16_round(W), b.astype(np.float32).astype(np.float64)) for W, b in params]
    loss_ref, g_ref = omlp.loss_and_grads(pr, omlp.bf16_round(X.astype(np.float32)), T.astype(np.float32))
    with scs.MLP(64, 512, 3, 4406, B) as net:
        net.set_params(scs.pack_params(params))
        assert scs.lib().scs_mlp_set_tensor_path(net._w, 1) == 0
        dx = torch.tensor(X, dtype=torch.float32, device="cuda")
        dt = torch.tensor(T, dtype=torch.float32, device="cuda")
        loss, g = net.gradients(dx.data_ptr(), dt.data_ptr())
        assert scs.lib().scs_mlp_error(net._w) == 0
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    for li, ((gW, gb), (rW, rb)) in enumerate(zip(scs.unpack_params(g.astype(np.float64), sizes), g_ref)):
        e = np.linalg.norm(gW - rW) / np.linalg.norm(rW)
        assert e < 5e-2, (li, e)


def test_enqueue_only_product(env):
    """scs_bf16_gemm_async (enqueue only, caller's status word) gives the
    synchronising call's result, bit for bit, and leaves the status at 0."""
    torch, scs = env
    rng = np.random.default_rng(11)
    M, N, K = 256, 512, 1024
    A = torch.tensor(rng.standard_normal((M, K)), dtype=torch.bfloat16, device="cuda")
    B = torch.tensor(rng.standard_normal((N, K)), dtype=torch.bfloat16, device="cuda")
    C1 = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    C2 = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    assert scs.lib().scs_bf16_gemm(A.data_ptr(), K, B.data_ptr(), K, M, N, K, C1.data_ptr(), N, 1, None) == 0
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    for _ in range(3):
        assert scs.lib().scs_bf16_gemm_async(A.data_ptr(), K, B.data_ptr(), K, M, N, K, C2.data_ptr(), N, 1,
                                             err.data_ptr(), s.cuda_stream) == 0
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert torch.equal(C1, C2)
    # shapes outside the tiling are refused on the host
    assert scs.lib().scs_bf16_gemm_async(A.data_ptr(), K, B.data_ptr(), K, M, N - 8, K, C2.data_ptr(), N, 1,
                                         err.data_ptr(), s.cuda_stream) == scs.INVALID_INPUT
