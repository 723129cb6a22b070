"""GPU path (through the C ABI) against the FP64 oracle on the same seeded inputs.

* FP64 mode with a tight CG (cg_rate 0, cg_tol_rel 1e-13) follows the
  oracle's exact-solve trajectory: ||u_gpu - u_orc|| / ||u_orc|| <= 1e-9 and
  the same for v, at every one of the first 50 iterations (the iteration is
  nonexpansive, Eq. "e-nonexpansive", so per-step solve errors of ~1e-13
  cannot grow).
* Full solves (FP64 and mixed FP32/FP64, the paper's CG schedule) reach the
  Sec. 3.5 tests; the returned point is checked on the CPU against the
  original data and against the oracle run with the same method and
  settings (indirect CG, same schedule):
    - FP64: the same iteration count and the objective within 1e-4
      relative (the two follow one trajectory);
    - FP32: the objective difference within the bound weak duality puts on
      two points with their residuals (two_point_bound), which at eps = 1e-4
      can exceed 1e-4 relative (the oracle's own 1e-4 point of the 1/500
      mixed program lies 8e-4 from p*);
    - both: at eps = 1e-6 the objective within 1e-4 relative of the
      oracle's at the same eps.
* Infeasible / unbounded problems return valid certificates (Sec. 2.2).
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import admm, cones
from paper_1312_3039_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scs():
    from paper_1312_3039_gb300 import build, scs as _scs
    build.build()
    return _scs


TIGHT = dict(precision=0, cg_rate=0.0, cg_adapt=0.0, cg_tol_rel=1e-13, cg_max_iters=500)


def same_settings(eps=1e-4, **kw):
    """The oracle with the GPU's default method and settings: indirect CG,
    zeta^k = (1/k)^1.5 capped at 0.3 x the last step, at most 50 CG steps."""
    return admm.Settings(linsys="indirect", cg_max_iters=50, eps_pri=eps, eps_dual=eps, eps_gap=eps, **kw)


def rel(a, b):
    return abs(a - b) / (1 + abs(b))


def two_point_bound(P, x1, y1, s1, x2, y2, s2):
    """Weak duality (Sec. 2) bounds how far the objectives of two points can
    be apart given their residuals: with r_p = A x + s - b, r_d = A^T y + c,
    g = c^T x + b^T y, s1, s2 in K and y1, y2 in K*,
        c^T x1 - c^T x2 in [-g2 - e12, g1 + e21],
        e12 = ||y2|| ||r_p1|| + ||x1|| ||r_d2||
    (c^T x1 + b^T y2 = y2^T s1 - y2^T r_p1 + x1^T r_d2 and y2^T s1 >= 0)."""
    def parts(x, y, s):
        return (np.linalg.norm(P.A @ x + s - P.b), np.linalg.norm(P.A.T @ y + P.c), P.c @ x + P.b @ y,
                np.linalg.norm(x), np.linalg.norm(y))
    rp1, rd1, g1, nx1, ny1 = parts(x1, y1, s1)
    rp2, rd2, g2, nx2, ny2 = parts(x2, y2, s2)
    return max(g2 + ny2 * rp1 + nx1 * rd2, g1 + ny1 * rp2 + nx2 * rd1)


def assert_objective_parity(P, precision, info, x, y, s, ref):
    """FP64: one trajectory with the oracle; FP32: within two_point_bound."""
    d = abs(info["pobj"] - ref.pobj)
    if precision == 0:
        assert info["iters"] == ref.iters, (info["iters"], ref.iters)
        assert d <= 1e-4 * (1 + abs(ref.pobj)), (info["pobj"], ref.pobj)
    else:
        bound = two_point_bound(P, x, y, s, ref.x, ref.y, ref.s)
        assert d <= bound * 1.01 + 1e-9 * (1 + abs(ref.pobj)), (info["pobj"], ref.pobj, bound)


def trajectory_parity(scs, P, iters=50, tol=1e-9, **gpu_kw):
    orc = admm.HSDSolver(P.A, P.b, P.c, P.cone, admm.Settings())
    kw = dict(TIGHT)
    kw.update(gpu_kw)
    with scs.Solver(P.A, P.b, P.c, P.cone, **kw) as g:
        D, E, sigma, rho = g.scaling()
        np.testing.assert_allclose(D, orc.D, rtol=1e-12)
        np.testing.assert_allclose(E, orc.E, rtol=1e-12)
        assert abs(sigma - orc.sigma) <= 1e-12 * orc.sigma
        assert abs(rho - orc.rho) <= 1e-12 * orc.rho
        worst = 0.0
        for k in range(iters):
            g.iterate(1)
            orc.step()
            u, v = g.iterates()
            eu = np.linalg.norm(u - orc.u) / np.linalg.norm(orc.u)
            ev = np.linalg.norm(v - orc.v) / max(np.linalg.norm(orc.v), 1e-300)
            worst = max(worst, eu, ev)
            assert eu <= tol and ev <= tol, (k + 1, eu, ev)
    return worst


def test_lp_trajectory_fp64(scs):
    trajectory_parity(scs, synth.lp(0))


def test_lp_trajectory_fp64_alpha1_no_scaling(scs):
    P = synth.lp(1)
    orc_settings = admm.Settings(alpha=1.0, normalize=False)
    orc = admm.HSDSolver(P.A, P.b, P.c, P.cone, orc_settings)
    with scs.Solver(P.A, P.b, P.c, P.cone, alpha=1.0, normalize=0, **TIGHT) as g:
        for k in range(50):
            g.iterate(1)
            orc.step()
            u, v = g.iterates()
            assert np.linalg.norm(u - orc.u) <= 1e-9 * np.linalg.norm(orc.u)
            assert np.linalg.norm(v - orc.v) <= 1e-9 * max(np.linalg.norm(orc.v), 1e-300)


def test_soc_exp_trajectory_fp64(scs):
    P = synth.random_cone(11, n=40, cone=synth.Cone(z=5, l=20, q=(3, 7, 1, 2, 40), ep=8))
    trajectory_parity(scs, P)


def test_every_cone_type_trajectory_fp64(scs):
    """Power cones and their duals, dual exponential triples, among every
    other cone type (Sec. 6.1): the FP64 engine follows the oracle for 50
    iterations."""
    cone = synth.Cone(z=4, l=15, q=(3, 5), s=(3,), ep=4, ed=3, p=(0.3, -0.7, 0.5, -0.2, 0.9))
    trajectory_parity(scs, synth.random_cone(31, n=45, cone=cone))


@pytest.mark.parametrize("precision", [0, 1])
def test_power_cone_solve(scs, precision):
    """A program with power, dual power and dual exponential cones among the
    others reaches the Sec. 3.5 tests; objective parity with the oracle as in
    test_lp_solve."""
    cone = synth.Cone(z=3, l=12, q=(4,), ep=3, ed=3, p=(0.25, -0.6, 0.5, 0.8, -0.35, 0.1))
    P = synth.random_cone(32, n=40, cone=cone)
    st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, precision=precision)
    assert st == scs.SOLVED, info
    check_solution(P, x, y, s, cone_tol=1e-5 if precision else 1e-7)
    ref = admm.solve(P.A, P.b, P.c, P.cone, same_settings())
    assert_objective_parity(P, precision, info, x, y, s, ref)


def test_mixed_small_trajectory_fp64(scs):
    trajectory_parity(scs, synth.mixed_small(0, scale=500))


@pytest.mark.parametrize("mode,name", [(0, "mean"), (1, "rms"), (2, "max")])
def test_block_scale_variants(scs, mode, name):
    """The three per-block values of the Sec. 5 equilibration give the
    oracle's D, E, sigma, rho, and the first iterations follow it."""
    P = synth.mixed_small(3, scale=500)
    orc = admm.HSDSolver(P.A, P.b, P.c, P.cone, admm.Settings(block_scale=name))
    with scs.Solver(P.A, P.b, P.c, P.cone, block_scale=mode, **TIGHT) as g:
        D, E, sigma, rho = g.scaling()
        np.testing.assert_allclose(D, orc.D, rtol=1e-12)
        np.testing.assert_allclose(E, orc.E, rtol=1e-12)
        assert abs(sigma - orc.sigma) <= 1e-12 * orc.sigma
        assert abs(rho - orc.rho) <= 1e-12 * orc.rho
        g.iterate(20)
        for _ in range(20):
            orc.step()
        u, _ = g.iterates()
        assert np.linalg.norm(u - orc.u) <= 1e-9 * np.linalg.norm(orc.u)


def test_plain_launch_path_matches_graph(scs):
    """The un-graphed launch sequence gives the same iterates as the graph."""
    P = synth.random_cone(12, n=30, cone=synth.Cone(z=3, l=15, q=(4, 5), ep=3))
    with scs.Solver(P.A, P.b, P.c, P.cone, **TIGHT) as g1, \
            scs.Solver(P.A, P.b, P.c, P.cone, use_graph=0, **TIGHT) as g2:
        g1.iterate(30)
        g2.iterate(30)
        u1, v1 = g1.iterates()
        u2, v2 = g2.iterates()
        np.testing.assert_allclose(u1, u2, rtol=0, atol=1e-12 * np.linalg.norm(u1))


def check_solution(P, x, y, s, eps=1e-4, cone_tol=1e-7, slack=1.0001):
    """Sec. 3.5 tests on the returned point against the original data, and
    the objective inside the band weak duality gives around the known optimum
    (cone membership to cone_tol: FP32 iterates round at ~1e-7 relative):
    with r_p = A x + s - b and r_d = A^T y + c, the generator's x*, y* give
    p* - c^T x <= ||y*|| ||r_p||  and  c^T x - p* <= |gap| + ||x*|| ||r_d||."""
    nb, nc = np.linalg.norm(P.b), np.linalg.norm(P.c)
    rp = np.linalg.norm(P.A @ x + s - P.b)
    rd = np.linalg.norm(P.A.T @ y + P.c)
    assert rp <= eps * (1 + nb) * slack
    assert rd <= eps * (1 + nc) * slack
    cx, by = P.c @ x, P.b @ y
    assert abs(cx + by) <= eps * (1 + abs(cx) + abs(by)) * slack
    assert cones.in_K(s, P.cone, cone_tol)
    assert cones.in_Kdual(y, P.cone, cone_tol)
    if P.p_star is not None:
        slack = 1e-9 * (1 + abs(P.p_star))
        assert P.p_star - cx <= np.linalg.norm(P.y_star) * rp + slack
        assert cx - P.p_star <= abs(cx + by) + np.linalg.norm(P.x_star) * rd + slack


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("seed", [0, 1])
def test_lp_solve(scs, precision, seed):
    P = synth.lp(seed)
    ref = admm.solve(P.A, P.b, P.c, P.cone, same_settings())
    st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, precision=precision)
    assert st == scs.SOLVED, info
    check_solution(P, x, y, s, cone_tol=1e-5 if precision else 1e-7)
    assert_objective_parity(P, precision, info, x, y, s, ref)
    # one A^T product per iteration, the warm-start A product every 20th
    # iteration (A z carried in between), two per CG step
    assert info["matvecs"] == info["iters"] + (info["iters"] + 19) // 20 + 2 * info["cg_iters"]
    assert info["iters"] % 20 == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_mixed_small_solve(scs, precision):
    P = synth.mixed_small(1, scale=500)
    st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, precision=precision)
    assert st == scs.SOLVED, info
    check_solution(P, x, y, s, cone_tol=1e-5 if precision else 1e-7)
    ref = admm.solve(P.A, P.b, P.c, P.cone, same_settings())
    assert_objective_parity(P, precision, info, x, y, s, ref)


_TIGHT_REF = {}


def tight_problems():
    return {"lp0": synth.lp(0), "lp1": synth.lp(1),
            "soc_exp": synth.random_cone(11, n=40, cone=synth.Cone(z=5, l=20, q=(3, 7, 1, 2, 40), ep=8)),
            "all_cones": synth.random_cone(3, n=60),
            "sdp": synth.sdp(seed=4, n=60, n_psd=3, order=6, n_nonneg=20, density=0.2, n_ill=1),
            "mixed_500": synth.mixed_small(1, scale=500)}


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("name", ["lp0", "lp1", "soc_exp", "all_cones", "sdp", "mixed_500"])
def test_objective_within_1e4_of_oracle_at_eps_1e6(scs, precision, name):
    """At eps = 1e-6 the Sec. 3.5 tests leave the objective far less room
    than 1e-4: both precisions land within 1e-4 relative of the FP64
    oracle's objective at the same eps (and of the generator's p*)."""
    P = tight_problems()[name]
    st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, precision=precision, eps_pri=1e-6, eps_dual=1e-6,
                                  eps_gap=1e-6, max_iters=100000)
    assert st == scs.SOLVED, info
    if name not in _TIGHT_REF:
        _TIGHT_REF[name] = admm.solve(P.A, P.b, P.c, P.cone, same_settings(1e-6, max_iters=100000))
    ref = _TIGHT_REF[name]
    assert ref.status == 1
    assert rel(info["pobj"], ref.pobj) <= 1e-4, (info["pobj"], ref.pobj)
    assert rel(info["pobj"], P.p_star) <= 1e-4, (info["pobj"], P.p_star)
    check_solution(P, x, y, s, eps=1e-6, cone_tol=1e-5 if precision else 1e-7, slack=1.01)


@pytest.mark.parametrize("precision", [0, 1])
def test_infeasible_certificate(scs, precision):
    P = synth.lp(0, variant="infeasible")
    st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, precision=precision)
    assert st == scs.INFEASIBLE, info
    assert abs(P.b @ y + 1.0) < 1e-9
    assert np.linalg.norm(P.A.T @ y) <= 1e-3
    assert cones.in_Kdual(y, P.cone, 1e-5 if precision else 1e-6)
    assert np.all(np.isnan(x)) and np.all(np.isnan(s))


@pytest.mark.parametrize("precision", [0, 1])
def test_unbounded_certificate(scs, precision):
    P = synth.lp(0, variant="unbounded")
    st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, precision=precision)
    assert st == scs.UNBOUNDED, info
    assert abs(P.c @ x + 1.0) < 1e-9
    np.testing.assert_allclose(s, -(P.A @ x), atol=1e-9)
    assert cones.in_K(s, P.cone, 1e-5)
    assert np.all(np.isnan(y))


def test_warm_start_from_solution(scs):
    P = synth.lp(3)
    with scs.Solver(P.A, P.b, P.c, P.cone, precision=0) as g:
        st, x, y, s, info = g.solve()
        assert st == scs.SOLVED
        g.warm_start(x, y, s)
        st2, x2, y2, s2, info2 = g.solve()
        assert st2 == scs.SOLVED
        assert info2["iters"] <= 20 < info["iters"]
        # a third call starts cold again
        st3, *_rest, info3 = g.solve()
        assert info3["iters"] == info["iters"]


def test_long_rows_and_empty_rows(scs):
    """Every SpMV path: rows longer than 2048 nonzeros (one CTA each), rows of
    257..2048 (one warp each), short rows of every length class packed into
    warp tasks; empty rows and columns go through every kernel."""
    rng = np.random.default_rng(5)
    n, m = 3000, 3200
    A = sp.lil_matrix((m, n))
    A[7, :] = rng.standard_normal(n)            # one dense row of 3000 entries
    A[40, :2500] = rng.standard_normal(2500)
    A[60, 500:1500] = rng.standard_normal(1000)  # one warp
    A[61, 100:400] = rng.standard_normal(300)
    B = synth.bernoulli_sparse(rng, m, n, 0.002).tolil()
    B[7, :] = 0
    B[40, :] = 0
    B[60:62, :] = 0
    B[100:120, :] = 0                           # empty rows
    A = sp.csc_matrix(A + B)
    cone = synth.Cone(z=50, l=m - 50 - 12, q=(5, 4), ep=1)
    P = synth.from_pair(A, cone, rng)
    trajectory_parity(scs, P, iters=25)


def test_noncanonical_csc_input(scs):
    """A CSC with rows out of order inside columns and every entry split into
    two exact halves (v/2 + v/2 = v) builds the same CSR layouts as the
    canonical CSC: the FP64 iterates agree to rounding."""
    rng = np.random.default_rng(17)
    P = synth.random_cone(23, n=40, cone=synth.Cone(z=5, l=30, q=(4, 6), ep=2), density=0.2)
    A = sp.csc_matrix(P.A)
    A.sum_duplicates()
    ptr, idx, val = [0], [], []
    for j in range(A.shape[1]):
        rows = np.repeat(A.indices[A.indptr[j]:A.indptr[j + 1]], 2)
        vals = np.repeat(A.data[A.indptr[j]:A.indptr[j + 1]] * 0.5, 2)
        order = rng.permutation(len(rows))
        idx.extend(rows[order])
        val.extend(vals[order])
        ptr.append(len(idx))
    A2 = sp.csc_matrix((np.array(val), np.array(idx, dtype=np.int32), np.array(ptr)), shape=A.shape)
    assert not A2.has_canonical_format and A2.nnz == 2 * A.nnz
    kw = dict(TIGHT)
    with scs.Solver(A, P.b, P.c, P.cone, **kw) as g1, scs.Solver(A2, P.b, P.c, P.cone, **kw) as g2:
        for _ in range(3):
            g1.iterate(10)
            g2.iterate(10)
            u1, v1 = g1.iterates()
            u2, v2 = g2.iterates()
            np.testing.assert_allclose(u2, u1, rtol=0, atol=1e-13 * np.abs(u1).max())
            np.testing.assert_allclose(v2, v1, rtol=0, atol=1e-13 * max(np.abs(v1).max(), 1e-300))


def test_tiny_and_ragged(scs):
    """n = 1 and odd sizes that leave ragged tails in every kernel."""
    for seed, (n, cone) in enumerate([(1, synth.Cone(z=1, l=2)),
                                      (3, synth.Cone(l=5, q=(2,))),
                                      (7, synth.Cone(z=2, l=3, q=(1, 3), ep=2)),
                                      (257, synth.Cone(z=13, l=300, q=(33,), ep=5))]):
        P = synth.random_cone(20 + seed, n=n, cone=cone, density=0.5 if n < 10 else 0.05)
        trajectory_parity(scs, P, iters=20)


@pytest.mark.parametrize("linsys", [0, 1])
def test_update_bc_equals_a_fresh_solver(scs, linsys):
    """Sec. 4.2 repeated solves: new b, c on the same A (scs_update_bc) give
    the FP64 solve a fresh scs_init on the new data gives (same iterations,
    same objective); the cached scaling D, E and, with the direct step, the
    cached inverse are reused."""
    P1 = synth.lp(3)
    P2 = synth.from_pair(P1.A, P1.cone, np.random.default_rng(77))
    with scs.Solver(P1.A, P1.b, P1.c, P1.cone, precision=0, linsys=linsys) as g:
        st1, *_r, info1 = g.solve()
        assert st1 == scs.SOLVED
        D1, E1, _s1, _r1 = g.scaling()
        g.update_bc(P2.b, P2.c)
        st2, x2, y2, s2, info2 = g.solve()
        D2, E2, sg2, rh2 = g.scaling()
    st3, x3, y3, s3, info3 = scs.solve(P2.A, P2.b, P2.c, P2.cone, precision=0, linsys=linsys)
    assert st2 == st3 == scs.SOLVED
    np.testing.assert_array_equal(D1, D2)
    np.testing.assert_array_equal(E1, E2)
    assert info2["iters"] == info3["iters"], (info2["iters"], info3["iters"])
    assert rel(info2["pobj"], info3["pobj"]) <= 1e-9, (info2["pobj"], info3["pobj"])
    check_solution(P2, x2, y2, s2)


def test_solve_writes_device_outputs(scs):
    """scs_solve accepts device pointers for x, y, s (unified addressing)."""
    import torch
    P = synth.lp(2)
    with scs.Solver(P.A, P.b, P.c, P.cone, precision=0) as g:
        st, x, y, s, info = g.solve()
        dx = torch.full((P.n,), float("nan"), dtype=torch.float64, device="cuda")
        dy = torch.full((P.m,), float("nan"), dtype=torch.float64, device="cuda")
        ds = torch.full((P.m,), float("nan"), dtype=torch.float64, device="cuda")
        st2, info2 = g.solve_to(dx.data_ptr(), dy.data_ptr(), ds.data_ptr())
    assert st == st2 == scs.SOLVED and info["iters"] == info2["iters"]
    np.testing.assert_array_equal(dx.cpu().numpy(), x)
    np.testing.assert_array_equal(dy.cpu().numpy(), y)
    np.testing.assert_array_equal(ds.cpu().numpy(), s)
