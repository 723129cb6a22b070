"""Pins of the oracle's cone projections against facts the mathematics fixes.

* Projection characterisation for a closed convex cone K:
  p = Pi_K(v)  iff  p in K,  p - v in K*,  p.(p - v) = 0.
* Moreau decomposition (Eq. "e-moreau"): v = Pi_K(v) - Pi_K*(-v), the two
  parts orthogonal.
* Complementary pairs built by explicit parametrisation (no projection):
  s in K, y in K*, s.y = 0  =>  Pi_K(s - y) = s and Pi_K*(y - s) = y.
* Closed forms: SOC(2) is the nonnegative orthant rotated by 45 degrees,
  PSD(1) is R+, a 2x2 PSD projection from its explicit eigen-pair formula.
* Brute force: no point of the exponential (or power) cone's boundary is
  closer to v than the computed projection.
* Power cone (Sec. 6.1): the printed dual is the dual (y.s >= 0 over the two
  sets, complementary boundary rays reach y.s = 0); projections of points in
  K, in the polar cone and with z = 0 have their closed forms.
"""
import math

import numpy as np
import pytest
import scipy.optimize as so

from oracle import cones
from paper_1312_3039_gb300 import synth


def kkt_triple(p, v, in_K, in_Kd, tol):
    d = p - v
    scale = max(1.0, np.linalg.norm(v))
    assert in_K(p, tol), (p, v)
    assert in_Kd(d, tol), (p, v, d)
    assert abs(p @ d) <= tol * scale * scale, (p @ d, p, v)


def test_soc_kkt_random():
    rng = np.random.default_rng(1)
    soc_in = lambda x, t: np.linalg.norm(x[1:]) <= x[0] + t * max(1.0, abs(x[0]))
    for _ in range(500):
        k = int(rng.integers(2, 12))
        v = rng.standard_normal(k) * rng.uniform(0.1, 10)
        p = cones.proj_soc(v)
        kkt_triple(p, v, soc_in, soc_in, 1e-12)


def test_soc2_is_rotated_orthant():
    """SOC(2) = {(t, x): |x| <= t} = R (R+ x R+) with the 45-degree rotation."""
    rng = np.random.default_rng(2)
    R = np.array([[1.0, 1.0], [1.0, -1.0]]) / math.sqrt(2.0)
    for _ in range(200):
        v = rng.standard_normal(2) * 3
        want = R @ np.maximum(R.T @ v, 0.0)
        np.testing.assert_allclose(cones.proj_soc(v), want, atol=1e-14)


def test_psd_order1_and_order2_closed_form():
    rng = np.random.default_rng(3)
    for _ in range(100):
        a = rng.standard_normal()
        np.testing.assert_allclose(cones.proj_psd(np.array([a]), 1), [max(a, 0.0)])
    for _ in range(200):
        a, b, c = rng.standard_normal(3) * 2
        # eigenpairs of [[a, b], [b, c]] written out
        mean, rad = 0.5 * (a + c), math.hypot(0.5 * (a - c), b)
        l1, l2 = mean + rad, mean - rad
        theta = 0.5 * math.atan2(2 * b, a - c)
        q1 = np.array([math.cos(theta), math.sin(theta)])
        q2 = np.array([-math.sin(theta), math.cos(theta)])
        P = max(l1, 0) * np.outer(q1, q1) + max(l2, 0) * np.outer(q2, q2)
        want = np.array([P[0, 0], math.sqrt(2) * P[1, 0], P[1, 1]])
        v = np.array([a, math.sqrt(2) * b, c])
        np.testing.assert_allclose(cones.proj_psd(v, 2), want, atol=1e-12)


def test_svec_is_isometry():
    rng = np.random.default_rng(4)
    for k in (1, 2, 5, 9):
        M = rng.standard_normal((k, k))
        M = M + M.T
        assert abs(np.linalg.norm(cones.svec(M)) - np.linalg.norm(M)) < 1e-12
        np.testing.assert_allclose(cones.smat(cones.svec(M), k), M, atol=1e-14)


def test_psd_kkt_random():
    rng = np.random.default_rng(5)
    for _ in range(100):
        k = int(rng.integers(1, 8))
        v = rng.standard_normal(k * (k + 1) // 2)
        p = cones.proj_psd(v, k)
        cone = synth.Cone(s=(k,))
        kkt_triple(p, v, lambda x, t: cones.in_K(x, cone, t), lambda x, t: cones.in_Kdual(x, cone, t), 1e-12)


def _exp_points(rng, count):
    pts = []
    for _ in range(count):
        u = rng.random()
        if u < 0.7:
            pts.append(rng.standard_normal(3) * rng.uniform(0.1, 5))
        elif u < 0.8:      # inside K
            y = rng.uniform(0.1, 2); x = rng.standard_normal()
            pts.append(np.array([x, y, y * math.exp(x / y) + rng.uniform(0, 1)]))
        elif u < 0.9:      # inside the polar cone (-v in K*)
            uu = -rng.uniform(0.1, 2); vv = rng.standard_normal()
            pts.append(-np.array([uu, vv, -uu * math.exp(vv / uu) / math.e + rng.uniform(0, 1)]))
        else:              # x < 0 and y < 0
            pts.append(np.array([-rng.uniform(0, 3), -rng.uniform(0, 3), rng.standard_normal()]))
    return pts


def test_exp_kkt_random():
    rng = np.random.default_rng(6)
    for v in _exp_points(rng, 1000):
        p = cones.proj_exp(v)
        kkt_triple(p, v, cones.in_exp, cones.in_exp_dual, 1e-10)


def test_exp_dual_kkt_random():
    rng = np.random.default_rng(7)
    for v in _exp_points(rng, 500):
        p = cones.proj_exp_dual(v)
        kkt_triple(p, v, cones.in_exp_dual, cones.in_exp, 1e-10)


def test_exp_dual_reading():
    """Sec. 6.1 prints Kexp* with a factor e; read as Euler's number the printed
    set is exactly the dual of Kexp: (1) y.s >= 0 for y in the printed set and
    s in Kexp; (2) for every boundary ray s = t(rho, 1, e^rho) the printed set
    holds the ray y = mu(-1, rho - 1, e^-rho) with y.s = 0 (so it is not a
    strict subset of the dual).  Without the factor e the smallest admissible
    third entry for the same (u, v) is e times larger and y.s > 0 for every
    rho, so that reading would give a strictly smaller set (not the dual)."""
    rng = np.random.default_rng(8)
    for _ in range(5000):
        y0 = rng.uniform(0.05, 3); x0 = rng.uniform(-4, 4)
        s = np.array([x0, y0, y0 * math.exp(x0 / y0)])
        u = -rng.uniform(0.05, 3); v = rng.uniform(-4, 4)
        y = np.array([u, v, -u * math.exp(v / u) / math.e])
        assert cones.in_exp_dual(y, 1e-12)
        assert (y @ s) >= -1e-12 * np.linalg.norm(y) * np.linalg.norm(s)
    for rho in np.linspace(-5, 5, 41):
        s = np.array([rho, 1.0, math.exp(rho)])
        y = np.array([-1.0, rho - 1.0, math.exp(-rho)])
        assert cones.in_exp_dual(y, 1e-12)
        assert abs(y @ s) <= 1e-12 * np.linalg.norm(y) * np.linalg.norm(s)
        u, v = y[0], y[1]
        w_alt = -u * math.exp(v / u)          # boundary without the factor e
        y_alt = np.array([u, v, w_alt])
        assert y_alt @ s > 0.5 * np.linalg.norm(y_alt) * 1e-3


def test_exp_brute_force():
    """No boundary point (y e^(x/y) = z, y > 0) nor point of the face
    {x <= 0, y = 0, z >= 0} is closer to v than Pi(v)."""
    rng = np.random.default_rng(9)
    for v in [rng.standard_normal(3) * 2 for _ in range(60)]:
        p = cones.proj_exp(v)
        dist = np.linalg.norm(p - v)

        def f(t):
            x, ly = t
            y = math.exp(ly)
            z = y * math.exp(min(x / y, 600))
            return np.linalg.norm(np.array([x, y, z]) - v)

        best = math.inf
        for x0 in (-3, -1, 0, 1, 3):
            for ly0 in (-4, -1, 0, 1):
                r = so.minimize(f, [x0, ly0], method="Nelder-Mead",
                                options=dict(xatol=1e-12, fatol=1e-14, maxiter=4000))
                best = min(best, r.fun)
        face = np.array([min(v[0], 0.0), 0.0, max(v[2], 0.0)])
        best = min(best, np.linalg.norm(face - v))
        if cones.in_exp(v):
            best = 0.0
        assert dist <= best + 1e-7, (v, dist, best)


POW_A = (0.03, 0.2, 0.5, 0.71, 0.97)


def _pow_points(rng, count, a):
    pts = []
    for _ in range(count):
        u = rng.random()
        if u < 0.6:
            pts.append(rng.standard_normal(3) * rng.uniform(0.1, 5))
        elif u < 0.7:      # inside K
            x, y = rng.uniform(0.1, 3, size=2)
            pts.append(np.array([x, y, rng.uniform(-1, 1) * x ** a * y ** (1 - a)]))
        elif u < 0.8:      # inside the polar cone (-v in K*)
            uu, vv = rng.uniform(0.1, 3, size=2)
            r = (uu / a) ** a * (vv / (1 - a)) ** (1 - a)
            pts.append(-np.array([uu, vv, rng.uniform(-1, 1) * r]))
        elif u < 0.9:      # extreme scales
            pts.append(rng.standard_normal(3) * 10.0 ** rng.uniform(-6, 6))
        else:              # one of x, y negative
            v = rng.standard_normal(3) * 2
            v[int(rng.integers(0, 2))] = -abs(v[0]) - 0.1
            pts.append(v)
    return pts


@pytest.mark.parametrize("a", POW_A)
def test_pow_kkt_random(a):
    rng = np.random.default_rng(int(a * 1000) + 11)
    for v in _pow_points(rng, 600, a):
        p = cones.proj_pow(v, a)
        kkt_triple(p, v, lambda x, t: cones.in_pow(x, a, t), lambda x, t: cones.in_pow_dual(x, a, t), 1e-12)


@pytest.mark.parametrize("a", POW_A)
def test_pow_dual_kkt_random(a):
    rng = np.random.default_rng(int(a * 1000) + 12)
    for v in _pow_points(rng, 400, a):
        p = cones.proj_pow_dual(v, a)
        kkt_triple(p, v, lambda x, t: cones.in_pow_dual(x, a, t), lambda x, t: cones.in_pow(x, a, t), 1e-12)


def test_pow_dual_reading():
    """The dual printed in Sec. 6.1 is the dual of Kpow^a: (1) y.s >= 0 for
    s on the boundary of Kpow^a and y on the printed dual's boundary (by the
    weighted AM-GM inequality); (2) every boundary ray s = (x, y, sigma r),
    r = x^a y^(1-a), has the printed-dual ray (a r/x, (1-a) r/y, -sigma)
    with y.s = 0, so the printed set is not a strict subset of the dual."""
    rng = np.random.default_rng(13)
    for _ in range(4000):
        a = rng.uniform(0.02, 0.98)
        x, y = rng.uniform(0.01, 5, size=2)
        sig = rng.choice([-1.0, 1.0])
        s = np.array([x, y, sig * x ** a * y ** (1 - a)])
        u, vv = rng.uniform(0.01, 5, size=2)
        w = rng.choice([-1.0, 1.0]) * (u / a) ** a * (vv / (1 - a)) ** (1 - a)
        d = np.array([u, vv, w])
        assert cones.in_pow(s, a, 1e-12) and cones.in_pow_dual(d, a, 1e-12)
        assert s @ d >= -1e-12 * np.linalg.norm(s) * np.linalg.norm(d)
        r = x ** a * y ** (1 - a)
        ray = np.array([a * r / x, (1 - a) * r / y, -sig])
        assert cones.in_pow_dual(ray, a, 1e-12)
        assert abs(ray @ s) <= 1e-12 * np.linalg.norm(ray) * np.linalg.norm(s)


@pytest.mark.parametrize("a", (0.2, 0.5, 0.83))
def test_pow_brute_force(a):
    """No point of the curved boundary (x^a y^(1-a) = |z|, z of either sign)
    nor of the face {x, y >= 0, z = 0} is closer to v than Pi(v)."""
    rng = np.random.default_rng(int(a * 100) + 14)
    for v in [rng.standard_normal(3) * 2 for _ in range(40)]:
        p = cones.proj_pow(v, a)
        dist = np.linalg.norm(p - v)
        best = 0.0 if cones.in_pow(v, a) else np.linalg.norm(np.array([max(v[0], 0), max(v[1], 0), 0.0]) - v)
        for sig in (-1.0, 1.0):
            def f(t):
                x, y = math.exp(t[0]), math.exp(t[1])
                return np.linalg.norm(np.array([x, y, sig * x ** a * y ** (1 - a)]) - v)
            for lx in (-3, -1, 0, 1):
                for ly in (-3, -1, 0, 1):
                    r = so.minimize(f, [lx, ly], method="Nelder-Mead",
                                    options=dict(xatol=1e-12, fatol=1e-14, maxiter=4000))
                    best = min(best, r.fun)
        assert dist <= best + 1e-7, (v, dist, best)


def test_pow_special_cases():
    a = 0.3
    v = np.array([2.0, 1.5, 0.7 * 2.0 ** a * 1.5 ** (1 - a)])        # in K: unchanged
    np.testing.assert_array_equal(cones.proj_pow(v, a), v)
    w = -np.array([1.0, 2.0, 0.5 * (1 / a) ** a * (2 / (1 - a)) ** (1 - a)])   # -w in K*: projection 0
    np.testing.assert_array_equal(cones.proj_pow(w, a), np.zeros(3))
    np.testing.assert_array_equal(cones.proj_pow(np.array([-1.0, 3.0, 0.0]), a), [0.0, 3.0, 0.0])


@pytest.mark.parametrize("seed", range(5))
def test_complementary_pairs_fix_projection(seed):
    rng = np.random.default_rng(100 + seed)
    cone = synth.Cone(z=3, l=7, q=(3, 6, 2), s=(1, 3, 4), ep=6, ed=3, p=(0.3, -0.6, 0.5, -0.1))
    s, y = synth.complementary_pair(cone, rng, ill_psd_blocks=1)
    assert abs(s @ y) < 1e-10
    np.testing.assert_allclose(cones.proj_K(s - y, cone), s, atol=1e-9)
    np.testing.assert_allclose(cones.proj_Kdual(y - s, cone), y, atol=1e-9)


@pytest.mark.parametrize("seed", range(5))
def test_moreau_mixed(seed):
    rng = np.random.default_rng(200 + seed)
    cone = synth.Cone(z=3, l=7, q=(3, 6, 2), s=(1, 3, 4), ep=6, ed=3, p=(0.3, -0.6, 0.5, -0.1))
    v = rng.standard_normal(cone.m) * 2
    pk = cones.proj_K(v, cone)
    pd = cones.proj_Kdual(-v, cone)
    np.testing.assert_allclose(pk - pd, v, atol=1e-9)
    assert abs(pk @ pd) < 1e-8
    assert cones.in_K(pk, cone, 1e-9)
    assert cones.in_Kdual(pd, cone, 1e-9)
