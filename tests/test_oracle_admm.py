"""Pins of the oracle's ADMM against facts the paper and the mathematics fix.

* Linear step: the SMW route of Sec. 4.1 equals a dense solve of (I + Q) u = w.
* Sec. 3.2.1: the naive ADMM of Eq. "e-SCS-naive" started with
  lambda0 = v0, mu0 = u0 has the same (u, v) iterates as Eq. "e-SCS".
* Eq. "e-iter-guarantees": u^k in C, v^k in C*, u^k . v^k = 0 for k >= 1.
* Eq. "e-nonexpansive": one iteration is nonexpansive.
* Sec. 3.2.3: the algorithm is homogeneous in (u0, v0).
* Sec. 6.6: the generated problem's optimal value is c^T x*.
* Brute-force vertex enumeration gives the exact optimum of tiny LPs.
* Sec. 2.2 / 2.3: infeasible and unbounded problems return certificates.
"""
import itertools
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import admm, cones, naive
from paper_1312_3039_gb300 import synth


def exact_settings(**kw):
    st = admm.Settings(eps_pri=1e-9, eps_dual=1e-9, eps_gap=1e-9, eps_infeas=1e-9,
                       eps_unbdd=1e-9, max_iters=20000)
    for k, v in kw.items():
        setattr(st, k, v)
    return st


def test_smw_equals_dense_solve():
    P = synth.random_cone(3, n=12)
    for linsys in ("direct", "indirect"):
        S = admm.HSDSolver(P.A, P.b, P.c, P.cone,
                           exact_settings(linsys=linsys, cg_rate=0.0, cg_adapt=0.0, cg_tol_rel=1e-14))
        Q = naive.hsd_Q(S.A, S.b, S.c)
        rng = np.random.default_rng(0)
        for _ in range(5):
            w = rng.standard_normal(Q.shape[0])
            S._wnorm = float(np.linalg.norm(w))
            got = S.solve_IQ(w, k=1)
            want = np.linalg.solve(np.eye(Q.shape[0]) + Q, w)
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-11 * np.linalg.norm(w))


def test_naive_equals_simplified():
    P = synth.random_cone(4, n=10)
    S = admm.HSDSolver(P.A, P.b, P.c, P.cone, exact_settings(alpha=1.0))
    ref = naive.run(S.A, S.b, S.c, P.cone, 40)
    for k in range(40):
        S.step()
        u_ref, v_ref = ref[k]
        scale = max(1.0, np.linalg.norm(u_ref))
        np.testing.assert_allclose(S.u, u_ref, atol=1e-9 * scale)
        np.testing.assert_allclose(S.v, v_ref, atol=1e-9 * scale)


@pytest.mark.parametrize("alpha", [1.0, 1.5])
def test_iterate_guarantees(alpha):
    P = synth.random_cone(5, n=20)
    S = admm.HSDSolver(P.A, P.b, P.c, P.cone, exact_settings(alpha=alpha))
    n, m = S.n, S.m
    for _ in range(60):
        S.step()
        u, v = S.u, S.v
        assert cones.in_Kdual(u[n:n + m], P.cone, 1e-9) and u[-1] >= 0
        assert np.all(v[:n] == 0.0)
        assert cones.in_K(v[n:n + m], P.cone, 1e-9) and v[-1] >= 0
        assert abs(u @ v) <= 1e-9 * max(1.0, np.linalg.norm(u) * np.linalg.norm(v))


def test_nonexpansive():
    P = synth.random_cone(6, n=15)
    S = admm.HSDSolver(P.A, P.b, P.c, P.cone, exact_settings(alpha=1.0))
    rng = np.random.default_rng(1)
    N = S.n + S.m + 1
    for _ in range(100):
        a_u, a_v = rng.standard_normal(N), rng.standard_normal(N)
        b_u, b_v = rng.standard_normal(N), rng.standard_normal(N)
        a_v[:S.n] = 0
        b_v[:S.n] = 0
        S.u, S.v = a_u.copy(), a_v.copy(); S.step(); pa = np.concatenate([S.u, S.v])
        S.u, S.v = b_u.copy(), b_v.copy(); S.step(); pb = np.concatenate([S.u, S.v])
        before = np.linalg.norm(np.concatenate([a_u - b_u, a_v - b_v]))
        assert np.linalg.norm(pa - pb) <= before * (1 + 1e-12)


def test_homogeneous():
    P = synth.random_cone(7, n=15)
    S1 = admm.HSDSolver(P.A, P.b, P.c, P.cone, exact_settings())
    S2 = admm.HSDSolver(P.A, P.b, P.c, P.cone, exact_settings())
    gamma = 3.7
    S2.u *= gamma
    S2.v *= gamma
    for _ in range(30):
        S1.step(); S2.step()
        np.testing.assert_allclose(S2.u, gamma * S1.u, atol=1e-10 * gamma * np.linalg.norm(S1.u))


@pytest.mark.parametrize("seed", [0, 1])
def test_lp_known_optimum(seed):
    P = synth.lp(seed)
    r = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings())
    assert r.status == admm.SOLVED
    assert abs(r.pobj - P.p_star) <= 1e-3 * (1 + abs(P.p_star))
    r = admm.solve(P.A, P.b, P.c, P.cone, exact_settings(eps_pri=1e-8, eps_dual=1e-8, eps_gap=1e-8))
    assert r.status == admm.SOLVED
    assert abs(r.pobj - P.p_star) <= 1e-6 * (1 + abs(P.p_star))
    assert abs(r.dobj - P.p_star) <= 1e-6 * (1 + abs(P.p_star))
    # primal and dual feasibility of the returned point
    assert np.linalg.norm(P.A @ r.x + r.s - P.b) <= 1e-7 * (1 + np.linalg.norm(P.b))
    assert np.linalg.norm(P.A.T @ r.y + P.c) <= 1e-7 * (1 + np.linalg.norm(P.c))
    assert cones.in_K(r.s, P.cone, 1e-9) and cones.in_Kdual(r.y, P.cone, 1e-9)


def vertex_optimum(P):
    A = np.asarray(P.A.todense())
    z = P.cone.z
    n = A.shape[1]
    best = math.inf
    for rows in itertools.combinations(range(z, A.shape[0]), n - z):
        act = list(range(z)) + list(rows)
        M = A[act]
        if abs(np.linalg.det(M)) < 1e-10:
            continue
        x = np.linalg.solve(M, P.b[act])
        s = P.b - A @ x
        if np.all(s[z:] >= -1e-9):
            best = min(best, float(P.c @ x))
    return best


@pytest.mark.parametrize("seed", range(6))
def test_tiny_lp_vertex_enumeration(seed):
    P = synth.tiny_lp(seed, n=3 + seed % 2, m=9 + seed % 3)
    want = vertex_optimum(P)
    assert abs(want - P.p_star) <= 1e-9 * (1 + abs(want))
    r = admm.solve(P.A, P.b, P.c, P.cone, exact_settings(eps_pri=1e-8, eps_dual=1e-8, eps_gap=1e-8))
    assert r.status == admm.SOLVED
    assert abs(r.pobj - want) <= 1e-6 * (1 + abs(want))


def test_infeasible_certificate():
    P = synth.lp(0, variant="infeasible")
    r = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings())
    assert r.status == admm.INFEASIBLE
    y = r.y
    assert abs(P.b @ y + 1.0) < 1e-12
    assert np.linalg.norm(P.A.T @ y) <= 1e-4 * 10
    assert cones.in_Kdual(y, P.cone, 1e-6)


def test_unbounded_certificate():
    P = synth.lp(0, variant="unbounded")
    r = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings())
    assert r.status == admm.UNBOUNDED
    x = r.x
    assert abs(P.c @ x + 1.0) < 1e-12
    assert cones.in_K(-(P.A @ x), P.cone, 1e-5)


@pytest.mark.parametrize("seed", [1, 2])
def test_mixed_cones_known_optimum(seed):
    P = synth.random_cone(seed, n=30)
    r = admm.solve(P.A, P.b, P.c, P.cone, exact_settings(eps_pri=1e-7, eps_dual=1e-7, eps_gap=1e-7))
    assert r.status == admm.SOLVED
    assert abs(r.pobj - P.p_star) <= 1e-5 * (1 + abs(P.p_star))
    assert cones.in_K(r.s, P.cone, 1e-8) and cones.in_Kdual(r.y, P.cone, 1e-8)


def test_direct_and_tight_indirect_agree():
    P = synth.lp(2)
    Sd = admm.HSDSolver(P.A, P.b, P.c, P.cone, admm.Settings())
    Si = admm.HSDSolver(P.A, P.b, P.c, P.cone, admm.Settings(linsys="indirect", cg_rate=0.0,
                                                             cg_adapt=0.0, cg_tol_rel=1e-13))
    for _ in range(50):
        Sd.step(); Si.step()
    np.testing.assert_allclose(Si.u, Sd.u, atol=1e-9 * np.linalg.norm(Sd.u))


def test_scaling_preserves_solution():
    P = synth.random_cone(8, n=25)
    st = exact_settings(eps_pri=1e-8, eps_dual=1e-8, eps_gap=1e-8)
    r1 = admm.solve(P.A, P.b, P.c, P.cone, st)
    st.normalize = False
    r2 = admm.solve(P.A, P.b, P.c, P.cone, st)
    assert r1.status == r2.status == admm.SOLVED
    assert abs(r1.pobj - r2.pobj) <= 1e-6 * (1 + abs(r1.pobj))


def test_equilibration_targets():
    """Sec. 5: D is one scalar per SOC / PSD / exp block, and the scaled
    columns have norms near one."""
    from oracle.scaling import equilibrate
    P = synth.random_cone(9, n=40)
    Ah, bh, ch, D, E, sigma, rho = equilibrate(P.A, P.b, P.c, P.cone)
    for kind, off, size, _ in P.cone.blocks():
        if kind in ("soc", "psd", "exp"):
            assert np.ptp(D[off:off + size]) == 0.0
    cn = np.sqrt(np.asarray(Ah.multiply(Ah).sum(axis=0)).ravel())
    assert np.all(np.abs(cn - 1.0) < 0.2)
    assert abs(np.linalg.norm(bh) - 1.0) < 1e-12
    np.testing.assert_allclose((sp.diags(D) @ P.A @ sp.diags(E) - Ah).toarray(), 0, atol=1e-12)


@pytest.mark.parametrize("block", ["rms", "mean", "max"])
def test_equilibration_one_pass_by_hand(block):
    """One Ruiz pass (Sec. 5 reading) on a 4x2 matrix with known norms: the
    SOC block's rows (norms 4, 12, 5) share one value -- their RMS, mean or
    maximum -- the free row keeps its norm 3, and the columns have norms 13
    and 5."""
    from oracle.scaling import equilibrate
    A = np.array([[0.0, 3.0],        # free row, norm 3
                  [4.0, 0.0],        # SOC rows: norms 4, 12, 5
                  [12.0, 0.0],
                  [3.0, 4.0]])
    cone = synth.Cone(z=1, q=(3,))
    Ah, bh, ch, D, E, sigma, rho = equilibrate(sp.csr_matrix(A), np.zeros(4), np.zeros(2),
                                               cone, passes=1, block=block)
    seg = np.array([4.0, 12.0, 5.0])
    want_r = {"rms": np.sqrt(np.mean(seg ** 2)), "mean": seg.mean(), "max": seg.max()}[block]
    np.testing.assert_allclose(D, [1 / np.sqrt(3.0)] + [1 / np.sqrt(want_r)] * 3, rtol=1e-15)
    np.testing.assert_allclose(E, [1 / np.sqrt(13.0), 1 / np.sqrt(5.0)], rtol=1e-15)
    np.testing.assert_allclose(Ah.toarray(), np.diag(D) @ A @ np.diag(E), rtol=1e-15)
    # b = 0 and c = 0: sigma and rho fall back to the 1e-4 floor
    assert sigma == 1e4
    assert bh.tolist() == [0.0] * 4 and ch.tolist() == [0.0] * 2


def test_warm_start_from_solution():
    """Sec. 4.2: restarting from the solution (u0 = (x, y, 1), v0 = (0, s, 0))
    stops at the first check."""
    P = synth.lp(3)
    st = exact_settings(eps_pri=1e-6, eps_dual=1e-6, eps_gap=1e-6)
    r = admm.solve(P.A, P.b, P.c, P.cone, st)
    r2 = admm.solve(P.A, P.b, P.c, P.cone, st, warm=(r.x, r.y, r.s))
    assert r2.status == admm.SOLVED
    assert r2.iters <= st.check_interval < r.iters


@pytest.mark.parametrize("variant", ["infeasible", "unbounded"])
def test_indirect_certificates(variant):
    """The indirect method with the capped CG schedule certifies as fast as
    the exact solve (the absolute schedule alone does not within 3000)."""
    P = synth.lp(0, variant=variant)
    r = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings(linsys="indirect", max_iters=2000))
    assert r.status == (admm.INFEASIBLE if variant == "infeasible" else admm.UNBOUNDED)
    assert r.iters <= 600


def test_indirect_warm_start():
    P = synth.lp(3)
    st = admm.Settings(linsys="indirect")
    r = admm.solve(P.A, P.b, P.c, P.cone, st)
    r2 = admm.solve(P.A, P.b, P.c, P.cone, st, warm=(r.x, r.y, r.s))
    assert r2.status == admm.SOLVED and r2.iters <= 40 < r.iters


@pytest.mark.parametrize("seed", [0, 1])
def test_weak_duality_band(seed):
    """At the 1e-4 tolerances the objective need not be within 1e-4 of p*,
    but weak duality bounds it by the residuals: with the generator's x*, y*,
    p* - c^T x <= ||y*|| ||A x + s - b|| and c^T x - p* <= |gap| + ||x*|| ||A^T y + c||."""
    P = synth.mixed_small(seed, scale=500)
    r = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings())
    assert r.status == admm.SOLVED
    rp = np.linalg.norm(P.A @ r.x + r.s - P.b)
    rd = np.linalg.norm(P.A.T @ r.y + P.c)
    gap = abs(P.c @ r.x + P.b @ r.y)
    assert P.p_star - P.c @ r.x <= np.linalg.norm(P.y_star) * rp + 1e-9
    assert P.c @ r.x - P.p_star <= gap + np.linalg.norm(P.x_star) * rd + 1e-9


def test_sdp_solve_known_optimum():
    """Sec. 6.1 PSD cone in the whole iteration: a small SDP built from a
    complementary PSD pair (one block with eigenvalues over 1e-7..1) solves
    to the generator's optimum, with s in K and y in K*."""
    P = synth.sdp(seed=4, n=60, n_psd=3, order=6, n_nonneg=20, density=0.2, n_ill=1)
    st = exact_settings(eps_pri=1e-7, eps_dual=1e-7, eps_gap=1e-7)
    r = admm.solve(P.A, P.b, P.c, P.cone, st)
    assert r.status == admm.SOLVED
    assert abs(r.pobj - P.p_star) <= 1e-5 * (1 + abs(P.p_star))
    assert cones.in_K(r.s, P.cone, 1e-7) and cones.in_Kdual(r.y, P.cone, 1e-7)


@pytest.mark.parametrize("case", ["lp", "mixed", "soc_exp"])
def test_returned_point_passes_tests_on_original_data(case):
    """Sec. 3.5 / Sec. 5: the oracle tests its residuals in scaled coordinates
    (D, E, sigma, rho); the point it returns must pass the same tests written
    directly on the original data: ||A x + s - b|| <= eps (1 + ||b||),
    ||A^T y + c|| <= eps (1 + ||c||), |c^T x + b^T y| <= eps (1 + |c^T x| + |b^T y|)."""
    if case == "lp":
        P = synth.lp(2)
    elif case == "mixed":
        P = synth.mixed_small(2, scale=500)
    else:
        P = synth.random_cone(13, n=30, cone=synth.Cone(z=4, l=20, q=(5, 3, 8), ep=4))
    st = admm.Settings()
    r = admm.solve(P.A, P.b, P.c, P.cone, st)
    assert r.status == admm.SOLVED
    nb, nc = np.linalg.norm(P.b), np.linalg.norm(P.c)
    cx, by = P.c @ r.x, P.b @ r.y
    tol = 1 + 1e-9
    assert np.linalg.norm(P.A @ r.x + r.s - P.b) <= st.eps_pri * (1 + nb) * tol
    assert np.linalg.norm(P.A.T @ r.y + P.c) <= st.eps_dual * (1 + nc) * tol
    assert abs(cx + by) <= st.eps_gap * (1 + abs(cx) + abs(by)) * tol
