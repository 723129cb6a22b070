"""The family solver's dense product (scs_dense_gemm, CUDA cores) against an
FP64 product of the same operands, through the C ABI.

C = alpha A B + beta C, column-major.  The kernel sums the K products of each
entry in k order with fused multiply-adds, so the classical bound for a
recursively summed dot product holds entrywise:
    |C_gpu - C_exact| <= gamma_K (|alpha| |A| |B| + |beta| |C0|) + u |C_exact|,
gamma_K = K u / (1 - K u), u the unit roundoff (2^-24 FP32, 2^-53 FP64; the
last term is the rounding of the stored result).  Precision 2 (the FP32
family solver's tensor-core path: three-way BF16 split, six products, FP32
accumulation in two products) is held to the same bound for 6K terms plus
the split's truncation, 8 u |A||B|, and its mean error to within 4x of the
FP32 kernel's.  Shapes cover one tile, many
tiles with ragged edges in M, N and K, the family solver's own shapes (with
few member columns: 64 x 64 tiles; with many: FP32 128 x 128 tiles), K = 0,
leading dimensions above the row count, and beta = 0 with NaN in C.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1312_3039_gb300 import build, scs
    build.build()
    return torch, scs


def run(env, precision, M, N, K, alpha, beta, lda_pad=0, ldb_pad=0, ldc_pad=0, nan_c=False, seed=0):
    torch, scs = env
    rng = np.random.default_rng(seed)
    dt = np.float64 if precision == 0 else np.float32
    tdt = torch.float64 if precision == 0 else torch.float32
    lda, ldb, ldc = max(M, 1) + lda_pad, max(K, 1) + ldb_pad, max(M, 1) + ldc_pad
    A = rng.standard_normal((K, lda)).astype(dt)          # column k of A is row k here (column-major storage)
    B = rng.standard_normal((N, ldb)).astype(dt)
    C0 = rng.standard_normal((N, ldc)).astype(dt)
    if nan_c:
        C0[:] = np.nan
    dA, dB = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    dC = torch.tensor(C0, device="cuda")
    scs.dense_gemm(precision, M, N, K, alpha, dA.data_ptr(), lda, dB.data_ptr(), ldb, beta, dC.data_ptr(), ldc)
    torch.cuda.synchronize()
    got = dC.cpu().numpy().astype(np.float64)
    Am = A[:, :M].T.astype(np.float64)                   # M x K
    Bm = B[:, :K].T.astype(np.float64)                   # K x N
    Cm = C0[:, :M].T.astype(np.float64)                  # M x N
    a32 = float(dt(alpha))
    b32 = float(dt(beta))
    exact = a32 * (Am @ Bm) + (b32 * Cm if beta != 0 else 0.0)
    u = 2.0 ** -53 if precision == 0 else 2.0 ** -24
    if precision == 2:
        # split path: six BF16 products per term, FP32 accumulation over 6K
        # terms in an unspecified order, the split's truncation below 8 u |a||b|
        gam = 6 * K * u / (1 - 6 * K * u) + 8 * u
    else:
        gam = K * u / (1 - K * u)
    bound = gam * (abs(a32) * (np.abs(Am) @ np.abs(Bm)) + (abs(b32) * np.abs(Cm) if beta != 0 else 0.0)) \
        + 2 * u * np.abs(exact) + 1e-300
    err = np.abs(got[:, :M].T - exact)
    assert np.all(err <= bound), (precision, M, N, K, float((err / bound).max()))
    # entries outside the M x N block (ldc padding) are untouched
    if ldc_pad:
        np.testing.assert_array_equal(got[:, M:], C0[:, M:].astype(np.float64))
    return float((err / bound).max())


@pytest.mark.parametrize("precision", [0, 1, 2])
@pytest.mark.parametrize("shape", [(1, 1, 1), (128, 128, 8), (64, 64, 8), (129, 257, 9), (7, 3, 1000),
                                   (801, 700, 1802), (1802, 333, 801), (801, 513, 801), (1802, 4100, 801)])
def test_gemm_matches_fp64_bound(env, precision, shape):
    M, N, K = shape
    run(env, precision, M, N, K, -1.0, 1.0, seed=M + N + K)
    run(env, precision, M, N, K, 1.0, 0.0, seed=M * N + K)


@pytest.mark.parametrize("precision", [0, 1, 2])
def test_gemm_edges(env, precision):
    run(env, precision, 100, 37, 0, 1.0, 0.5)                     # K = 0: C = beta C
    run(env, precision, 130, 65, 70, 0.75, -2.0, lda_pad=3, ldb_pad=5, ldc_pad=7)
    run(env, precision, 200, 40, 33, 1.0, 0.0, nan_c=True)        # beta = 0 never reads C


def test_gemm_rejects_bad_arguments(env):
    torch, scs = env
    with pytest.raises(scs.ScsError) as ei:
        scs.dense_gemm(1, 10, 10, 10, 1.0, 0, 5, 0, 10, 0.0, 0, 10)   # lda < M
    assert ei.value.code == scs.INVALID_INPUT


def test_split_product_is_as_accurate_as_fp32(env):
    """The tensor-core split product's error against the FP64 product is of
    the FP32 product's order (within 4x of the CUDA-core FP32 kernel's, in the
    mean over the entries), far below a single BF16 product's."""
    torch, scs = env
    M, N, K = 801, 700, 1802
    rng = np.random.default_rng(5)
    A = rng.standard_normal((K, M)).astype(np.float32)
    B = rng.standard_normal((N, K)).astype(np.float32)
    exact = A.T.astype(np.float64) @ B.T.astype(np.float64)
    errs = {}
    for prec in (1, 2):
        dC = torch.zeros((N, M), dtype=torch.float32, device="cuda")
        dA, dB = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
        scs.dense_gemm(prec, M, N, K, 1.0, dA.data_ptr(), M, dB.data_ptr(), K, 0.0, dC.data_ptr(), M)
        torch.cuda.synchronize()
        errs[prec] = float(np.abs(dC.cpu().numpy().T.astype(np.float64) - exact).mean())
    from oracle.mlp import bf16_round
    bf16_one = float(np.abs(bf16_round(A).T @ bf16_round(B).T - exact).mean())   # one plain BF16 product
    assert errs[2] <= 4 * errs[1], errs
    assert errs[2] <= 1e-2 * bf16_one, (errs, bf16_one)
