"""The paper's application workloads (Sec. 6.2 - 6.5) encode the problems
they are built from: on small instances the FP64 oracle's solution of each
generated cone program is optimal for the original problem, checked against
an independent solve of that problem (scikit-learn's lasso, scipy's SLSQP and
L-BFGS-B) or against the problem's own optimality facts (RPCA: the SDP's
objective equals the nuclear norm of the returned L, and L + S = M)."""
import numpy as np
import pytest
import scipy.optimize as so

from oracle import admm
from paper_1312_3039_gb300 import synth

TIGHT = dict(eps_pri=1e-8, eps_dual=1e-8, eps_gap=1e-8, max_iters=200000)


def test_lasso_paper_encodes_the_lasso():
    sk = pytest.importorskip("sklearn.linear_model")
    P = synth.lasso_paper(seed=3, p=40, q=25)
    m = P.meta
    r = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings(**TIGHT))
    assert r.status == 1
    z = r.x[:m["p"]]
    obj = 0.5 * np.sum((m["F"] @ z - m["g"]) ** 2) + m["mu"] * np.abs(z).sum()
    assert abs(r.pobj - obj) <= 1e-6 * (1 + abs(obj))          # the SOCP's epigraph variables are tight
    ref = sk.Lasso(alpha=m["mu"] / m["q"], fit_intercept=False, tol=1e-14, max_iter=1_000_000).fit(m["F"], m["g"])
    zr = ref.coef_
    obj_ref = 0.5 * np.sum((m["F"] @ zr - m["g"]) ** 2) + m["mu"] * np.abs(zr).sum()
    assert abs(obj - obj_ref) <= 1e-6 * (1 + abs(obj_ref)), (obj, obj_ref)


def test_portfolio_paper_encodes_the_portfolio_problem():
    P = synth.portfolio_paper(seed=4, p=30, q=4)
    m = P.meta
    r = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings(**TIGHT))
    assert r.status == 1
    p = m["p"]
    Sig = m["F"] @ m["F"].T + np.diag(m["D"])
    f = lambda z: -(m["mu"] @ z - m["gamma"] * z @ Sig @ z)
    z = r.x[:p]
    res = so.minimize(f, np.full(p, 1.0 / p), jac=lambda z: -(m["mu"] - 2 * m["gamma"] * Sig @ z),
                      method="SLSQP", bounds=[(0, None)] * p,
                      constraints=[dict(type="eq", fun=lambda z: z.sum() - 1.0)],
                      options=dict(ftol=1e-15, maxiter=2000))
    assert abs(-r.pobj - (-f(z))) <= 1e-6 * (1 + abs(r.pobj))    # t = u^2, s = v^2 at the optimum
    assert abs(f(z) - res.fun) <= 1e-6 * (1 + abs(res.fun)), (f(z), res.fun)


def test_rpca_paper_encodes_the_nuclear_norm_problem():
    P = synth.rpca_paper(seed=5, p=8, r=2)
    m = P.meta
    r = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings(**TIGHT))
    assert r.status == 1
    p, q = m["p"], m["q"]
    L = r.x[:p * q].reshape((p, q), order="F")
    S = r.x[p * q:2 * p * q].reshape((p, q), order="F")
    np.testing.assert_allclose(L + S, m["M"], atol=1e-6)
    assert np.abs(S).sum() <= m["mu"] * (1 + 1e-6)
    nuc = np.linalg.svd(L, compute_uv=False).sum()
    assert abs(r.pobj - nuc) <= 1e-6 * (1 + nuc), (r.pobj, nuc)     # min (TrW1 + TrW2)/2 = ||L||_*
    # (L^, S^) is feasible, so the optimum is at most its nuclear norm
    assert nuc <= np.linalg.svd(m["L_hat"], compute_uv=False).sum() * (1 + 1e-6)


def test_logreg_paper_encodes_l1_logistic_regression():
    P = synth.logreg_paper(seed=6, p=6, q=80)
    m = P.meta
    r = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings(**TIGHT))
    assert r.status == 1
    p = m["p"]
    Zy = m["y"][:, None] * m["Z"]

    def f(w):
        return np.logaddexp(0.0, Zy @ w).sum() + m["mu"] * np.abs(w).sum()

    def f_split(ab):                      # w = a - b, a, b >= 0: smooth
        w = ab[:p] - ab[p:]
        s = 1.0 / (1.0 + np.exp(-(Zy @ w)))
        g = Zy.T @ s
        return np.logaddexp(0.0, Zy @ w).sum() + m["mu"] * ab.sum(), np.concatenate([g + m["mu"], -g + m["mu"]])

    res = so.minimize(f_split, np.zeros(2 * p), jac=True, method="L-BFGS-B", bounds=[(0, None)] * (2 * p),
                      options=dict(ftol=1e-15, gtol=1e-12, maxiter=10000))
    w = r.x[:p]
    assert abs(r.pobj - f(w)) <= 1e-6 * (1 + abs(f(w)))       # the epigraph variables are tight
    assert abs(f(w) - res.fun) <= 1e-6 * (1 + abs(res.fun)), (f(w), res.fun)
