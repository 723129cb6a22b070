"""PSD cone on the GPU (Sec. 6.1: eigendecomposition per block, negative
eigenvalues set to zero) against the FP64 oracle.

* scs_project (cold FP64 Jacobi) on single blocks of many orders -- on chip
  up to order 96, in global scratch above -- and on special matrices with a
  known projection (PSD: unchanged, negative definite: zero, repeated
  eigenvalues, eigenvalues over 1e-7..1);
* the FP64 engine (warm-started Jacobi every iteration) follows the
  oracle's exact-solve trajectory to 1e-9 for 50 iterations, with blocks on
  chip and in global scratch;
* the mixed FP32/FP64 engine solves small SDPs to the Sec. 3.5 tests, and
  its ill-conditioned blocks take the FP64 reconstruction.
"""
import numpy as np
import pytest

from oracle import admm, cones
from paper_1312_3039_gb300 import synth

from test_gpu_parity import TIGHT, assert_objective_parity, check_solution, same_settings, trajectory_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_1312_3039_gb300 import build, scs
    build.build()
    return torch, scs


def sym_svec(M):
    return cones.svec(0.5 * (M + M.T))


def project_batch(env, cone, V, dual=1):
    torch, scs = env
    dv = torch.tensor(np.atleast_2d(V), dtype=torch.float64, device="cuda")
    out = torch.full_like(dv, float("nan"))
    d2 = scs.project(cone, dual, dv.data_ptr(), out.data_ptr(), dv.shape[0])
    return out.cpu().numpy(), d2


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5, 8, 17, 40, 48, 49, 64, 96, 97, 128, 200])
def test_project_orders(env, order):
    rng = np.random.default_rng(order)
    cone = synth.Cone(s=(order,))
    V = rng.standard_normal((3, cone.m)) * np.array([[0.1], [1.0], [30.0]])
    got, d2 = project_batch(env, cone, V)
    ref = np.stack([cones.proj_psd(v, order) for v in V])
    for g, r, v in zip(got, ref, V):
        np.testing.assert_allclose(g, r, rtol=0, atol=1e-12 * np.linalg.norm(v))
    want = float(np.sum((ref - V) ** 2))
    assert abs(d2 - want) <= 1e-10 * max(1.0, want)


@pytest.mark.parametrize("k", [12, 64])          # scalar and blocked Jacobi
def test_project_special_matrices(env, k):
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    lam_pos = rng.uniform(0.5, 2.0, k)
    h = k // 2
    cases = {
        "psd": (Q * lam_pos) @ Q.T,                                   # unchanged
        "negdef": -(Q * lam_pos) @ Q.T,                               # -> 0
        "repeated": (Q * np.r_[[1.0] * h, [-1.0] * h]) @ Q.T,         # -> Q1 Q1^T
        "spread": (Q * (10.0 ** np.linspace(-7, 0, k) * np.r_[[1, -1] * h])) @ Q.T,
        "zero": np.zeros((k, k)),
    }
    cone = synth.Cone(s=(k,))
    V = np.stack([sym_svec(M) for M in cases.values()])
    got, _ = project_batch(env, cone, V)
    want = {
        "psd": sym_svec(cases["psd"]),
        "negdef": np.zeros(cone.m),
        "repeated": sym_svec(Q[:, :h] @ Q[:, :h].T),
    }
    for (name, M), g, v in zip(cases.items(), got, V):
        ref = want.get(name, cones.proj_psd(v, k))
        np.testing.assert_allclose(g, ref, rtol=0, atol=1e-12 * max(1.0, np.linalg.norm(v)), err_msg=name)


def test_project_mixed_cone_batch(env):
    """PSD blocks among the other cones; K and K* agree on the PSD rows."""
    cone = synth.Cone(z=3, l=20, q=(4, 9), s=(3, 7, 1, 20), ep=5)
    rng = np.random.default_rng(5)
    V = rng.standard_normal((6, cone.m)) * 2.0
    for dual in (0, 1):
        got, d2 = project_batch(env, cone, V, dual)
        ref = np.stack([(cones.proj_Kdual if dual else cones.proj_K)(v, cone) for v in V])
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-11 * np.abs(V).max())
        assert abs(d2 - np.sum((ref - V) ** 2)) <= 1e-9 * np.sum((ref - V) ** 2)


def test_noalloc_rejects_psd(env):
    torch, scs = env
    cone = synth.Cone(l=2, s=(3,))
    dv = torch.zeros(cone.m, dtype=torch.float64, device="cuda")
    with pytest.raises(scs.ScsError) as ei:
        scs.project_noalloc(cone, 0, dv.data_ptr(), dv.data_ptr(), 1)
    assert ei.value.code == scs.UNSUPPORTED


def small_sdp(seed, order=6, n_psd=3, n_ill=1, n=60, n_nonneg=20, density=0.2):
    return synth.sdp(seed=seed, n=n, n_psd=n_psd, order=order, n_nonneg=n_nonneg, density=density, n_ill=n_ill)


def test_sdp_trajectory_fp64(env):
    torch, scs = env
    trajectory_parity(scs, small_sdp(0, order=7, n_psd=3))


def test_sdp_trajectory_fp64_mixed_cones(env):
    torch, scs = env
    cone = synth.Cone(z=4, l=10, q=(3, 5), s=(2, 4, 9), ep=3)
    trajectory_parity(scs, synth.random_cone(21, n=30, cone=cone))


def test_sdp_trajectory_fp64_blocked(env):
    """Order 56 (padded to 64): the blocked Jacobi with X, V, W on chip."""
    torch, scs = env
    trajectory_parity(scs, small_sdp(4, order=56, n_psd=2, n_ill=1, n=60, n_nonneg=10, density=0.05), iters=30)


def test_sdp_trajectory_fp64_global_scratch(env):
    """Order 100 in FP64 does not fit on chip: X, W in global scratch and V in
    its persistent storage."""
    torch, scs = env
    trajectory_parity(scs, small_sdp(1, order=100, n_psd=1, n_ill=0, n=40, n_nonneg=10, density=0.05), iters=20)


@pytest.mark.parametrize("precision", [0, 1])
# scalar Jacobi; blocked; blocked with V a round late; order 150: the
# matrices in global scratch, the blocked sweeps' subproblems on chip
@pytest.mark.parametrize("order,n_psd", [(10, 4), (60, 2), (100, 1), (150, 1)])
def test_sdp_solve(env, precision, order, n_psd):
    torch, scs = env
    P = small_sdp(2, order=order, n_psd=n_psd, n_ill=1, n=120, n_nonneg=40, density=0.1)
    ref = admm.solve(P.A, P.b, P.c, P.cone, same_settings())
    with scs.Solver(P.A, P.b, P.c, P.cone, precision=precision) as g:
        st, x, y, s, info = g.solve()
        calls, sweeps, fp64 = g.psd_counters()
    assert st == 1, st
    # FP32: the sweeps stop at ||off(X)||_F <= 1e-6 ||X||_F <= 1e-6 sqrt(order)
    # ||X||_2, and the FP32 rounding of the eigenvector products adds about
    # as much to the dual iterate s
    check_solution(P, x, y, s, cone_tol=1e-7 if precision == 0 else max(1e-5, 3e-6 * np.sqrt(order)))
    assert_objective_parity(P, precision, info, x, y, s, ref)
    assert calls == n_psd * info["iters"]
    assert 0 < sweeps < 10 * calls     # warm-started blocks often need no sweep at all
    if precision == 0:
        assert fp64 == 0         # the FP64 engine has nothing to promote


@pytest.mark.parametrize("cond,expect", [(1.0, "all"), (float("inf"), "none")])
def test_sdp_fp64_reconstruction_switch(env, cond, expect):
    """FP32 engine: psd_fp64_cond = 1 sums every block's reconstruction in
    FP64, infinity none; both reach the Sec. 3.5 tests."""
    torch, scs = env
    P = small_sdp(5, order=9, n_psd=3, n_ill=2, n=100, n_nonneg=30, density=0.1)
    with scs.Solver(P.A, P.b, P.c, P.cone, precision=1, psd_fp64_cond=cond) as g:
        st, x, y, s, info = g.solve()
        calls, sweeps, fp64 = g.psd_counters()
    assert st == 1, st
    check_solution(P, x, y, s, cone_tol=1e-5)
    assert calls == 3 * info["iters"]
    # every call with a positive eigenvalue counts when cond = 1
    assert (fp64 >= calls // 2) if expect == "all" else (fp64 == 0)


def test_plain_launch_path_matches_graph_psd(env):
    torch, scs = env
    P = small_sdp(3, order=5, n_psd=2)
    with scs.Solver(P.A, P.b, P.c, P.cone, **TIGHT) as g1, \
            scs.Solver(P.A, P.b, P.c, P.cone, use_graph=0, **TIGHT) as g2:
        g1.iterate(25)
        g2.iterate(25)
        u1, _ = g1.iterates()
        u2, _ = g2.iterates()
        np.testing.assert_allclose(u1, u2, rtol=0, atol=1e-12 * np.linalg.norm(u1))
