"""The parametric lasso family (Sec. 6.2 SOCP form) solved by the FP64
oracle agrees with scikit-learn's coordinate-descent lasso (an independent
textbook solver of the unconstrained problem (1/2)||F z - g||^2 + mu ||z||_1)."""
import numpy as np
import pytest

from oracle import admm, cones
from paper_1312_3039_gb300 import synth


def test_family_shapes_and_data():
    fam = synth.lasso_family(0, p=40, q=100, d=8)
    assert fam.A.shape == (2 * 40 + 100 + 2, 2 * 40 + 1)
    assert fam.cone.l == 80 and fam.cone.q == (102,)
    th = fam.thetas(1, 3)
    b0, c0 = fam.bc(th[0])
    b1, c1 = fam.bc(th[1])
    assert np.all(c0[40:80] > 0) and c0[80] == 0.5 and np.all(c0[:40] == 0)
    assert b0[80] == b0[81] == 1.0 and not np.allclose(b0, b1)


def test_family_member_matches_sklearn_lasso():
    sk = pytest.importorskip("sklearn.linear_model")
    fam = synth.lasso_family(2, p=40, q=100, d=8)
    for th in fam.thetas(3, 2):
        P = fam.problem(th)
        st = admm.Settings(eps_pri=1e-8, eps_dual=1e-8, eps_gap=1e-8, max_iters=50000)
        r = admm.solve(P.A, P.b, P.c, P.cone, st)
        assert r.status == admm.SOLVED
        z = r.x[:fam.p]
        g = fam.G @ th
        mu = fam.mu(th)
        ref = sk.Lasso(alpha=mu / fam.q, fit_intercept=False, tol=1e-12, max_iter=200000).fit(fam.F, g).coef_
        np.testing.assert_allclose(z, ref, atol=1e-5 * max(1.0, np.abs(ref).max()))
        obj = 0.5 * np.sum((fam.F @ ref - g) ** 2) + mu * np.abs(ref).sum()
        assert abs(r.pobj - obj) <= 1e-6 * (1 + abs(obj))
        assert cones.in_K(r.s, P.cone, 1e-7)
