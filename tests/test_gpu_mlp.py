"""Warm-start network kernels (BF16 tensor-core products, FP32 master
weights) against the FP64 oracle network on the same BF16-rounded inputs and
weights: outputs, loss and every layer's gradients; a training run lowers the
loss; the data helpers (column statistics, standardisation, gather, the
prediction-to-warm-start map) against numpy."""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

SIZES = [64, 512, 512, 512, 4406]


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1312_3039_gb300 import build, scs
    build.build()
    return torch, scs


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def test_forward_and_gradients_match_oracle(env):
    """Batch 512 (four row tiles) through the full 64-512-512-512-4406
    network, the oracle rounding to BF16 where the kernels do (inputs,
    weights, hidden activations, dZ before the products): every entry of the
    output and of every gradient within one BF16 ulp (2^-8) of each summed
    term, |g - g_ref| <= 2^-8 (|dZ|^T |A|) (weights) and 2^-8 sum |dZ|
    (biases), plus FP32 accumulation; the loss to 1e-4 relative."""
    torch, scs = env
    rng = np.random.default_rng(0)
    B = 512
    params = omlp.init_params(rng, SIZES)
    params = [(W, rng.standard_normal(b.shape) * 0.05) for W, b in params]
    X = rng.standard_normal((B, SIZES[0]))
    T = rng.standard_normal((B, SIZES[-1]))
    flat = scs.pack_params(params)
    # the GPU reads X and W in BF16: the oracle gets the same rounded values
    pr = [(omlp.bf16_round(W), b.astype(np.float32).astype(np.float64)) for W, b in params]
    Xr = omlp.bf16_round(X.astype(np.float32))
    Tr = T.astype(np.float32).astype(np.float64)
    Y_ref, cache = omlp.forward(pr, Xr, bf16_points=True)
    loss_ref, g_ref = omlp.loss_and_grads(pr, Xr, Tr, bf16_points=True)
    with scs.MLP(SIZES[0], SIZES[1], 3, SIZES[-1], B) as net:
        net.set_params(flat)
        np.testing.assert_array_equal(net.get_params(), flat)
        dx = torch.tensor(X, dtype=torch.float32, device="cuda")
        dt = torch.tensor(T, dtype=torch.float32, device="cuda")
        dy = torch.empty((B, SIZES[-1]), dtype=torch.float32, device="cuda")
        net.forward(dx.data_ptr(), dy.data_ptr())
        Y = dy.cpu().numpy().astype(np.float64)
        loss, g = net.gradients(dx.data_ptr(), dt.data_ptr())
    u = 2.0 ** -8
    A_last = cache[-1][0]
    W_last = pr[-1][0]
    ybound = u * (np.abs(A_last) @ np.abs(W_last).T) + 1e-6 * np.abs(Y_ref).max()
    assert np.all(np.abs(Y - Y_ref) <= ybound), float((np.abs(Y - Y_ref) / ybound).max())
    assert abs(loss - loss_ref) <= 1e-4 * loss_ref, (loss, loss_ref)
    got = scs.unpack_params(g.astype(np.float64), SIZES)
    # dZ of each layer from the oracle's chain rule (for the magnitude bound)
    R = (Y_ref - Tr) * 2.0 / Y_ref.size
    dZs = [None] * len(pr)
    dA = R
    for li in range(len(pr) - 1, -1, -1):
        dZ = dA if li == len(pr) - 1 else dA * omlp.gelu_grad(cache[li][1])
        dZs[li] = dZ
        dA = omlp.bf16_round(dZ) @ pr[li][0]
    for li, ((gW, gb), (rW, rb)) in enumerate(zip(got, g_ref)):
        A_in = cache[li][0]
        wbound = u * (np.abs(dZs[li]).T @ np.abs(A_in)) + 1e-6 * np.abs(rW).max()
        bbound = u * np.abs(dZs[li]).sum(axis=0) + 1e-6 * np.abs(rb).max()
        assert np.all(np.abs(gW - rW) <= wbound), (li, float((np.abs(gW - rW) / wbound).max()))
        assert np.all(np.abs(gb - rb) <= bbound), (li, float((np.abs(gb - rb) / bbound).max()))
        assert rel(gW, rW) < 5e-3 and rel(gb, rb) < 5e-3, (li, rel(gW, rW), rel(gb, rb))


def test_training_lowers_loss(env):
    """Targets that are a fixed smooth function of the input: 300 Adam steps
    take the loss down by more than 5x."""
    torch, scs = env
    rng = np.random.default_rng(1)
    B, din, dout = 256, 64, 300
    sizes = [din, 128, 128, 128, dout]
    params = omlp.init_params(rng, sizes)
    Mix = rng.standard_normal((din, dout)) / 8
    X = rng.standard_normal((4 * B, din)).astype(np.float32)
    T = np.tanh(X @ Mix).astype(np.float32)
    with scs.MLP(din, 128, 3, dout, B) as net:
        net.set_params(scs.pack_params(params))
        dX = torch.tensor(X, device="cuda")
        dT = torch.tensor(T, device="cuda")
        first = None
        for step in range(300):
            k = step % 4
            loss = net.train_step(dX[k * B:(k + 1) * B].data_ptr(), dT[k * B:(k + 1) * B].data_ptr(), 1e-3,
                                  want_loss=(step == 0 or step == 299))
            if step == 0:
                first = loss
        last = loss
    assert last < first / 5, (first, last)


def test_data_helpers(env):
    torch, scs = env
    rng = np.random.default_rng(2)
    D = (rng.standard_normal((500, 37)) * rng.uniform(0.1, 5, 37) + rng.uniform(-3, 3, 37)).astype(np.float32)
    dD = torch.tensor(D, device="cuda")
    mean = torch.empty(37, device="cuda")
    sd = torch.empty(37, device="cuda")
    scs.column_stats(dD.data_ptr(), 500, 37, mean.data_ptr(), sd.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_allclose(mean.cpu().numpy(), D.astype(np.float64).mean(0), rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(sd.cpu().numpy(), D.astype(np.float64).std(0), rtol=1e-4)
    scs.standardize(dD.data_ptr(), 500, 37, mean.data_ptr(), sd.data_ptr())
    torch.cuda.synchronize()
    Z = dD.cpu().numpy()
    np.testing.assert_allclose(Z.mean(0), 0, atol=1e-4)
    idx = torch.tensor(rng.permutation(500)[:100], dtype=torch.int64, device="cuda")
    out = torch.empty((100, 37), device="cuda")
    scs.gather_rows(dD.data_ptr(), 37, idx.data_ptr(), 100, out.data_ptr())
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), Z[idx.cpu().numpy()])
    # prediction -> warm start: x^ = (p sd + mean) / max(tau, tau_min)
    n, m, cnt = 3, 4, 5
    w = n + 2 * m + 1
    P = rng.standard_normal((cnt, w + 2)).astype(np.float32)
    mu = rng.standard_normal(w).astype(np.float32)
    s_ = rng.uniform(0.5, 2, w).astype(np.float32)
    xs = torch.empty((cnt, n), dtype=torch.float64, device="cuda")
    ys = torch.empty((cnt, m), dtype=torch.float64, device="cuda")
    ss = torch.empty((cnt, m), dtype=torch.float64, device="cuda")
    dP = torch.tensor(P, device="cuda")
    dmu = torch.tensor(mu, device="cuda")       # kept alive until the kernel has run
    dsd = torch.tensor(s_, device="cuda")
    scs.warm_from_prediction(dP.data_ptr(), w + 2, dmu.data_ptr(), dsd.data_ptr(), n, m, cnt, 1e-3,
                             xs.data_ptr(), ys.data_ptr(), ss.data_ptr())
    torch.cuda.synchronize()
    U = P[:, :w].astype(np.float64) * s_ + mu
    tau = np.maximum(U[:, -1], 1e-3)[:, None]
    np.testing.assert_allclose(xs.cpu().numpy(), U[:, :n] / tau, rtol=1e-6)
    np.testing.assert_allclose(ys.cpu().numpy(), U[:, n:n + m] / tau, rtol=1e-6)
    np.testing.assert_allclose(ss.cpu().numpy(), U[:, n + m:n + 2 * m] / tau, rtol=1e-6)
