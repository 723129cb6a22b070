"""Seeded synthetic cone programs shaped like the paper's workloads.

This module is shared by the FP64 oracle (``oracle/``) and by the GPU path's
tests and benchmark.  It holds *no* arithmetic of the solver: no cone
projection, no scaling, no ADMM step.  Complementary primal/dual pairs are
built directly from explicit parametrisations of each cone's boundary instead
of projecting a random vector, so a projection routine can be checked against
them (if ``s in K``, ``y in K*`` and ``s.y = 0`` then ``Pi_K(s - y) = s``).

Recipe (Sec. 6.6, "Random Cone Programs"): draw a complementary pair
``(s*, y*)``, a sparse ``A`` with N(0,1) values, ``x* ~ N(0,1)``, then set
``b = A x* + s*`` and ``c = -A^T y*``; the optimal value is ``c^T x*``.
Infeasible and unbounded variants embed a certificate (Sec. 2.2).

Row order of every cone: zero rows, nonnegative rows, second-order blocks
(head first), PSD blocks in svec form (lower triangle, column-major,
off-diagonal entries times sqrt 2), exponential triples (x, y, z).
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np
import scipy.sparse as sp

SQRT2 = math.sqrt(2.0)


@dataclass(frozen=True)
class Cone:
    """Cone ``K = {0}^z x R+^l x SOC(q_1) x ... x PSD(s_1) x ... x Kexp^ep
    x (Kexp*)^ed x Kpow(p_1) x ...`` (Sec. 6.1).  ``p`` holds one parameter
    per power triple: a in (0, 1) is the power cone Kpow^a, -a the dual
    power cone (Kpow^a)*."""

    z: int = 0
    l: int = 0
    q: tuple = ()
    s: tuple = ()
    ep: int = 0
    ed: int = 0
    p: tuple = ()

    @property
    def m(self) -> int:
        return (self.z + self.l + int(sum(self.q))
                + int(sum(k * (k + 1) // 2 for k in self.s)) + 3 * (self.ep + self.ed + len(self.p)))

    def blocks(self):
        """Yield ``(kind, start, size, order)`` for every block, in row order."""
        off = 0
        if self.z:
            yield ("zero", off, self.z, 0)
            off += self.z
        if self.l:
            yield ("nonneg", off, self.l, 0)
            off += self.l
        for k in self.q:
            yield ("soc", off, int(k), 0)
            off += int(k)
        for k in self.s:
            d = int(k) * (int(k) + 1) // 2
            yield ("psd", off, d, int(k))
            off += d
        for _ in range(self.ep):
            yield ("exp", off, 3, 0)
            off += 3
        for _ in range(self.ed):
            yield ("exp_dual", off, 3, 0)
            off += 3
        for a in self.p:
            if a > 0:
                yield ("pow", off, 3, float(a))
            else:
                yield ("pow_dual", off, 3, float(-a))
            off += 3


@dataclass
class Problem:
    """``min c^T x  s.t.  A x + s = b, s in K`` with its known solution or certificate."""

    A: sp.csc_matrix
    b: np.ndarray
    c: np.ndarray
    cone: Cone
    kind: str = "feasible"          # "feasible" | "infeasible" | "unbounded"
    x_star: np.ndarray | None = None
    s_star: np.ndarray | None = None
    y_star: np.ndarray | None = None
    p_star: float | None = None
    cert: np.ndarray | None = None  # y (infeasible) or x (unbounded)
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.A.shape[0]

    @property
    def n(self) -> int:
        return self.A.shape[1]


# ---------------------------------------------------------------------------
# complementary pairs, one cone type at a time (no projections involved)
# ---------------------------------------------------------------------------

def _svec(M: np.ndarray) -> np.ndarray:
    k = M.shape[0]
    out = np.empty(k * (k + 1) // 2)
    pos = 0
    for j in range(k):
        col = M[j:, j].copy()
        col[1:] *= SQRT2
        out[pos:pos + k - j] = col
        pos += k - j
    return out


def _pair_soc(rng, k):
    if k == 1:                      # SOC(1) = {t >= 0}: one side takes the mass
        g = abs(rng.standard_normal()) + 0.1
        return (np.array([g]), np.zeros(1)) if rng.random() < 0.5 else (np.zeros(1), np.array([g]))
    d = rng.standard_normal(k - 1)
    nd = np.linalg.norm(d)
    d = d / nd if nd > 0 else np.eye(k - 1)[0]
    a = abs(rng.standard_normal()) + 0.1
    u = rng.random()
    s = np.zeros(k)
    y = np.zeros(k)
    if u < 0.15:            # s strictly inside, y = 0
        s[0] = a * (1.0 + rng.uniform(0.1, 1.0))
        s[1:] = a * d
    elif u < 0.30:          # y strictly inside, s = 0
        y[0] = a * (1.0 + rng.uniform(0.1, 1.0))
        y[1:] = a * d
    else:                   # both on the boundary, opposite rays
        beta = abs(rng.standard_normal()) + 0.1
        s[0], s[1:] = a, a * d
        y[0], y[1:] = beta, -beta * d
    return s, y


def _pair_exp(rng):
    """Boundary of Kexp: s = t(rho, 1, e^rho); its complementary ray in
    Kexp*: y = mu(-1, rho - 1, e^-rho) (orthogonal to s, on the boundary of
    the dual cone as printed in Sec. 6.1)."""
    rho = rng.uniform(-2.0, 2.0)
    t = rng.uniform(0.5, 1.5)
    mu = rng.uniform(0.5, 1.5)
    u = rng.random()
    s = np.zeros(3)
    y = np.zeros(3)
    if u < 0.15:
        s[:] = (t * rho, t, t * math.exp(rho) * (1.0 + rng.uniform(0.1, 1.0)))
    elif u < 0.30:
        y[:] = (-mu, mu * (rho - 1.0), mu * math.exp(-rho) * (1.0 + rng.uniform(0.1, 1.0)))
    else:
        s[:] = (t * rho, t, t * math.exp(rho))
        y[:] = (-mu, mu * (rho - 1.0), mu * math.exp(-rho))
    return s, y


def _pair_pow(rng, a):
    """Boundary of Kpow^a = {x^a y^(1-a) >= |z|, x, y >= 0} (Sec. 6.1):
    s = (x, y, sigma x^a y^(1-a)); its complementary ray in the dual cone
    (Kpow^a)* = {(u/a)^a (v/(1-a))^(1-a) >= |w|, u, v >= 0}:
    y = mu (a r / x, (1 - a) r / y, -sigma) with r = x^a y^(1-a), which is
    orthogonal to s (a r + (1 - a) r - r = 0) and on the dual boundary
    ((r/x)^a (r/y)^(1-a) = 1).  Or one side strictly inside, the other 0."""
    x, y = rng.uniform(0.3, 2.0, size=2)
    sig = 1.0 if rng.random() < 0.5 else -1.0
    r = x ** a * y ** (1.0 - a)
    mu = rng.uniform(0.5, 1.5)
    u = rng.random()
    s = np.zeros(3)
    d = np.zeros(3)
    if u < 0.15:
        s[:] = (x, y, sig * r * rng.uniform(0.0, 0.9))
    elif u < 0.30:
        d[:] = (mu * a * r / x, mu * (1.0 - a) * r / y, -sig * mu * rng.uniform(0.0, 0.9))
    else:
        s[:] = (x, y, sig * r)
        d[:] = (mu * a * r / x, mu * (1.0 - a) * r / y, -sig * mu)
    return s, d


def _pair_psd(rng, k, ill=False):
    Q, _ = np.linalg.qr(rng.standard_normal((k, k)))
    if ill:
        lam = 10.0 ** rng.uniform(-7.0, 0.0, size=k)
    else:
        lam = np.abs(rng.standard_normal(k))
    mask = np.zeros(k, dtype=bool)
    mask[rng.permutation(k)[: k // 2]] = True
    S = (Q * np.where(mask, lam, 0.0)) @ Q.T
    Y = (Q * np.where(mask, 0.0, lam)) @ Q.T
    return _svec(0.5 * (S + S.T)), _svec(0.5 * (Y + Y.T))


def complementary_pair(cone: Cone, rng, ill_psd_blocks: int = 0):
    """Return ``(s*, y*)`` with ``s* in K``, ``y* in K*`` and ``s*.y* = 0``."""
    m = cone.m
    s = np.zeros(m)
    y = np.zeros(m)
    n_psd = 0
    for kind, off, size, order in cone.blocks():
        if kind == "zero":
            y[off:off + size] = rng.standard_normal(size)
        elif kind == "nonneg":
            g = np.abs(rng.standard_normal(size))
            on_s = rng.random(size) < 0.5
            s[off:off + size] = np.where(on_s, g, 0.0)
            y[off:off + size] = np.where(on_s, 0.0, g)
        elif kind == "soc":
            s[off:off + size], y[off:off + size] = _pair_soc(rng, size)
        elif kind == "psd":
            s[off:off + size], y[off:off + size] = _pair_psd(rng, order, n_psd < ill_psd_blocks)
            n_psd += 1
        elif kind == "exp":
            s[off:off + 3], y[off:off + 3] = _pair_exp(rng)
        elif kind == "exp_dual":        # K = Kexp*, K* = Kexp: the roles swap
            y[off:off + 3], s[off:off + 3] = _pair_exp(rng)
        elif kind == "pow":
            s[off:off + 3], y[off:off + 3] = _pair_pow(rng, order)
        elif kind == "pow_dual":        # K = (Kpow^a)*, K* = Kpow^a
            y[off:off + 3], s[off:off + 3] = _pair_pow(rng, order)
    return s, y


# ---------------------------------------------------------------------------
# sparse matrices
# ---------------------------------------------------------------------------

def bernoulli_sparse(rng, m, n, density) -> sp.csc_matrix:
    mask = rng.random((m, n)) < density
    vals = rng.standard_normal((m, n)) * mask
    return sp.csc_matrix(vals)


def powerlaw_rows(rng, m, n, nnz, exponent=2.0, max_len=10_000) -> sp.csc_matrix:
    """Rows with power-law lengths (p(L) ~ L^-exponent on [1, max_len],
    rescaled to ``nnz`` in total), uniform random columns, N(0,1) values."""
    u = rng.random(m)
    a = exponent - 1.0
    top = (max_len + 1.0) ** (-a)
    x = (1.0 - u * (1.0 - top)) ** (-1.0 / a)
    L = np.floor(x)
    L = np.maximum(1, np.round(L * (nnz / L.sum()))).astype(np.int64)
    L = np.minimum(L, min(max_len, n))
    diff = int(nnz - L.sum())
    while diff != 0:
        idx = rng.integers(0, m, size=abs(diff))
        if diff > 0:
            np.add.at(L, idx, 1)
            L = np.minimum(L, min(max_len, n))
        else:
            np.subtract.at(L, idx, 1)
            L = np.maximum(L, 1)
        diff = int(nnz - L.sum())
    rows = np.repeat(np.arange(m, dtype=np.int64), L)
    cols = rng.integers(0, n, size=rows.size, dtype=np.int64)
    keys = np.unique(rows * n + cols)
    rows = keys // n
    cols = keys - rows * n
    vals = rng.standard_normal(keys.size)
    return sp.csc_matrix((vals, (rows, cols)), shape=(m, n))


def uniform_sparse(rng, m, n, nnz) -> sp.csc_matrix:
    rows = rng.integers(0, m, size=nnz, dtype=np.int64)
    cols = rng.integers(0, n, size=nnz, dtype=np.int64)
    keys = np.unique(rows * n + cols)
    rows = keys // n
    cols = keys - rows * n
    vals = rng.standard_normal(keys.size)
    return sp.csc_matrix((vals, (rows, cols)), shape=(m, n))


# ---------------------------------------------------------------------------
# Sec. 6.6 construction and its infeasible / unbounded variants
# ---------------------------------------------------------------------------

def from_pair(A, cone, rng, ill_psd_blocks=0, meta=None) -> Problem:
    A = sp.csc_matrix(A)
    s, y = complementary_pair(cone, rng, ill_psd_blocks)
    x = rng.standard_normal(A.shape[1])
    b = A @ x + s
    c = -(A.T @ y)
    return Problem(A=A, b=b, c=c, cone=cone, kind="feasible", x_star=x, s_star=s,
                   y_star=y, p_star=float(c @ x), meta=dict(meta or {}))


def make_infeasible(prob: Problem, rng, delta=1.0) -> Problem:
    """Pick nonnegative rows i != j, set row_j(A) = -row_i(A) and
    b_i + b_j = -delta; then y = (e_i + e_j)/delta has A^T y = 0, y >= 0 and
    b^T y = -1 (the set D of Sec. 2.2 is nonempty)."""
    cone = prob.cone
    assert cone.l >= 2
    i, j = cone.z + rng.choice(cone.l, size=2, replace=False)
    A = sp.lil_matrix(prob.A.tocsr())
    A[j, :] = -A[i, :]
    A = sp.csc_matrix(A)
    b = prob.b.copy()
    b[j] = -delta - b[i]
    cert = np.zeros(prob.m)
    cert[i] = cert[j] = 1.0 / delta
    return Problem(A=A, b=b, c=prob.c.copy(), cone=cone, kind="infeasible", cert=cert,
                   meta=dict(prob.meta, rows=(int(i), int(j))))


def make_unbounded(prob: Problem, rng) -> Problem:
    """Pick a column l; zero it on every row outside the nonnegative block,
    make it nonpositive on the nonnegative rows and set c_l = -1.  Then
    x = e_l has -A x in K and c^T x = -1 (the set P~ of Sec. 2.2 is nonempty),
    while b = A x* + s* keeps the primal feasible."""
    cone = prob.cone
    col = int(rng.integers(0, prob.n))
    A = prob.A.tolil()
    for r in range(prob.m):
        v = A[r, col]
        if v != 0.0:
            if cone.z <= r < cone.z + cone.l:
                A[r, col] = -abs(v)
            else:
                A[r, col] = 0.0
    A = sp.csc_matrix(A)
    A.eliminate_zeros()
    s = prob.s_star
    x = prob.x_star
    b = A @ x + s
    c = prob.c.copy()
    c[col] = -1.0
    cert = np.zeros(prob.n)
    cert[col] = 1.0
    return Problem(A=A, b=b, c=c, cone=cone, kind="unbounded", cert=cert,
                   meta=dict(prob.meta, col=col))


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def lp(seed=0, n=200, m=400, n_zero=100, density=0.05, variant="feasible") -> Problem:
    """Random sparse LP: zero rows then nonnegative rows, Bernoulli(density)
    pattern with N(0,1) values (n=200, m=400, 5% is the small LP workload)."""
    rng = np.random.default_rng(seed)
    cone = Cone(z=n_zero, l=m - n_zero)
    A = bernoulli_sparse(rng, m, n, density)
    prob = from_pair(A, cone, rng, meta=dict(workload="lp", seed=seed))
    if variant == "infeasible":
        return make_infeasible(prob, rng)
    if variant == "unbounded":
        return make_unbounded(prob, rng)
    return prob


def mixed(seed=0, n=1_000_000, m=2_000_000, nnz=20_000_000, n_zero=100_000,
          n_soc=20_000, soc_range=(3, 50), n_exp=10_000, max_row=10_000) -> Problem:
    """Large mixed-cone program: power-law row lengths (exponent 2, rescaled to
    ``nnz``), zero / nonnegative / SOC (sizes uniform in ``soc_range``) / exp
    cones; rows not used by the other cones are nonnegative."""
    rng = np.random.default_rng(seed)
    q = tuple(int(v) for v in rng.integers(soc_range[0], soc_range[1] + 1, size=n_soc))
    n_l = m - n_zero - sum(q) - 3 * n_exp
    if n_l < 0:
        raise ValueError("cone rows exceed m")
    cone = Cone(z=n_zero, l=n_l, q=q, ep=n_exp)
    A = powerlaw_rows(rng, m, n, nnz, max_len=max_row)
    return from_pair(A, cone, rng, meta=dict(workload="mixed", seed=seed))


def mixed_small(seed=0, scale=500) -> Problem:
    """The large mixed-cone program shrunk by ``scale`` with the same recipe."""
    return mixed(seed, n=1_000_000 // scale, m=2_000_000 // scale,
                 nnz=20_000_000 // scale, n_zero=100_000 // scale,
                 n_soc=max(1, 20_000 // scale), n_exp=max(1, 10_000 // scale),
                 max_row=max(10, 10_000 // scale))


def sdp(seed=0, n=200_000, n_psd=64, order=128, n_nonneg=50_000, density=1e-3,
        n_ill=8) -> Problem:
    """SDP-heavy program: ``n_psd`` PSD blocks (svec) plus nonnegative rows;
    uniform sparse A; the first ``n_ill`` PSD pairs have eigenvalues spread
    over 1e-7..1."""
    rng = np.random.default_rng(seed)
    cone = Cone(l=n_nonneg, s=tuple([order] * n_psd))
    m = cone.m
    A = uniform_sparse(rng, m, n, int(round(density * m * n)))
    return from_pair(A, cone, rng, ill_psd_blocks=n_ill, meta=dict(workload="sdp", seed=seed))


def portfolio(rng, n_assets, gamma=1.0) -> Problem:
    """Long-only factor-model portfolio (Sec. 6.3 form with one risk SOC):
    variables (z, t); minimise -mu^T z + gamma t subject to 1^T z = 1, z >= 0,
    ||(1 - t, 2 F^T z)|| <= 1 + t (i.e. ||F^T z||^2 <= t), k = n/10 factors."""
    p = int(n_assets)
    k = max(1, p // 10)
    F = rng.standard_normal((p, k))
    mu = rng.uniform(0.0, 1.0, size=p)
    n = p + 1
    rows = []
    rows.append(np.concatenate([np.ones(p), [0.0]])[None, :])       # zero row
    rows.append(np.hstack([-np.eye(p), np.zeros((p, 1))]))           # z >= 0
    rows.append(np.concatenate([np.zeros(p), [-1.0]])[None, :])      # 1 + t
    rows.append(np.concatenate([np.zeros(p), [1.0]])[None, :])       # 1 - t
    rows.append(np.hstack([-2.0 * F.T, np.zeros((k, 1))]))           # 2 F^T z
    A = sp.csc_matrix(np.vstack(rows))
    b = np.zeros(A.shape[0])
    b[0] = 1.0
    b[p + 1] = 1.0
    b[p + 2] = 1.0
    c = np.concatenate([-mu, [gamma]])
    cone = Cone(z=1, l=p, q=(k + 2,))
    assert A.shape == (cone.m, n)
    return Problem(A=A, b=b, c=c, cone=cone, kind="feasible",
                   meta=dict(workload="portfolio", assets=p, factors=k))


def portfolio_batch(seed=0, count=4096, lo=20, hi=500):
    rng = np.random.default_rng(seed)
    sizes = rng.integers(lo, hi + 1, size=count)
    return [portfolio(rng, int(p)) for p in sizes]


def tiny_lp(seed=0, n=3, m=9, n_zero=1) -> Problem:
    """Small dense LP for brute-force vertex enumeration."""
    rng = np.random.default_rng(seed)
    cone = Cone(z=n_zero, l=m - n_zero)
    A = sp.csc_matrix(rng.standard_normal((m, n)))
    return from_pair(A, cone, rng, meta=dict(workload="tiny_lp", seed=seed))


def random_cone(seed=0, n=30, m=None, cone=None, density=0.3) -> Problem:
    """Small mixed-cone program with every cone type present (parity cases)."""
    rng = np.random.default_rng(seed)
    if cone is None:
        cone = Cone(z=4, l=12, q=(3, 5, 4), s=(2, 3), ep=3)
    m = cone.m
    A = bernoulli_sparse(rng, m, n, density)
    # keep every column nonempty
    for j in np.flatnonzero(np.diff(A.indptr) == 0):
        A[int(rng.integers(0, m)), j] = rng.standard_normal()
    A = sp.csc_matrix(A)
    return from_pair(A, cone, rng, meta=dict(workload="random_cone", seed=seed))


# ---------------------------------------------------------------------------
# Parametric lasso family (Sec. 6.2 SOCP form) for the learned warm start
# ---------------------------------------------------------------------------

@dataclass
class LassoFamily:
    """minimize (1/2)||F z - g||^2 + mu ||z||_1 over z in R^p, as the SOCP of
    Sec. 6.2 with variables x = (z, t, w) in R^(2p+1):

        minimize (1/2) w + mu 1^T t
        s.t.  -t <= z <= t,   ||(1 - w, 2 (F z - g))|| <= 1 + w,

    standard form A x + s = b, s in K = R+^(2p) x SOC(q + 2):
        rows 0..p-1    (z - t <= 0):  A = [ I, -I, 0],  b = 0
        rows p..2p-1   (-z - t <= 0): A = [-I, -I, 0],  b = 0
        SOC head       1 + w:         A = [0, 0, -1],   b = 1
        SOC            1 - w:         A = [0, 0,  1],   b = 1
        SOC tail       2 (F z - g):   A = [-2F, 0, 0],  b = -2 g
    c = (0, mu 1, 1/2).  A is the same for every member; theta in R^d moves
    only b (through g = G theta) and c (through mu = mu0 (1 + tanh(a.theta/8)/2),
    which stays positive; mu0 is 0.1 times the median of ||F^T g||_inf over
    1000 draws of theta, the paper's mu = 0.1 mu_max rule)."""

    F: np.ndarray
    G: np.ndarray
    a: np.ndarray
    mu0: float
    A: sp.csc_matrix
    cone: Cone

    @property
    def p(self):
        return self.F.shape[1]

    @property
    def q(self):
        return self.F.shape[0]

    @property
    def d(self):
        return self.G.shape[1]

    def mu(self, theta):
        return self.mu0 * (1.0 + 0.5 * np.tanh(self.a @ theta / 8.0))

    def bc(self, theta):
        """(b, c) of the member theta."""
        p, q = self.p, self.q
        g = self.G @ theta
        b = np.zeros(2 * p + q + 2)
        b[2 * p] = 1.0
        b[2 * p + 1] = 1.0
        b[2 * p + 2:] = -2.0 * g
        c = np.zeros(2 * p + 1)
        c[p:2 * p] = self.mu(theta)
        c[2 * p] = 0.5
        return b, c

    def problem(self, theta) -> Problem:
        b, c = self.bc(theta)
        return Problem(A=self.A, b=b, c=c, cone=self.cone, kind="feasible",
                       meta=dict(workload="lasso", theta=np.asarray(theta)))

    def thetas(self, seed, count):
        return np.random.default_rng(seed).standard_normal((count, self.d))


def lasso_family(seed=0, p=400, q=1000, d=64) -> LassoFamily:
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((q, p)) / math.sqrt(q)
    G = rng.standard_normal((q, d)) / 8.0
    a = rng.standard_normal(d)
    th = rng.standard_normal((1000, d))
    mu0 = 0.1 * float(np.median(np.abs((G @ th.T).T @ F).max(axis=1)))
    A, cone = lasso_socp_matrix(F)
    return LassoFamily(F=F, G=G, a=a, mu0=mu0, A=A, cone=cone)


def lasso_socp_matrix(F):
    """A and K of the Sec. 6.2 lasso SOCP for the design F (q x p): variables
    (z, t, w), rows z - t <= 0, -z - t <= 0 (R+^(2p)) and the SOC(q + 2)
    (1 + w, 1 - w, 2 (F z - g)) (the b part carries g)."""
    q, p = F.shape
    Ip = sp.identity(p, format="csc")
    top = sp.hstack([Ip, -Ip, sp.csc_matrix((p, 1))])
    mid = sp.hstack([-Ip, -Ip, sp.csc_matrix((p, 1))])
    head = sp.csc_matrix(np.concatenate([np.zeros(2 * p), [-1.0]])[None, :])
    head2 = sp.csc_matrix(np.concatenate([np.zeros(2 * p), [1.0]])[None, :])
    tail = sp.hstack([sp.csc_matrix(-2.0 * F), sp.csc_matrix((q, p)), sp.csc_matrix((q, 1))])
    A = sp.csc_matrix(sp.vstack([top, mid, head, head2, tail]))
    cone = Cone(l=2 * p, q=(q + 2,))
    assert A.shape == (cone.m, 2 * p + 1)
    return A, cone


# ---------------------------------------------------------------------------
# The paper's application workloads (Sec. 6.2 - 6.5), built as printed there.
# None has a known optimum; meta keeps the original problem's data so that
# tests can check the cone program against the problem it encodes.
# ---------------------------------------------------------------------------

def lasso_paper(seed=0, p=10_000, q=2_000) -> Problem:
    """Sec. 6.2 instance: F (q x p) ~ N(0, 1); z^ with p/10 nonzero N(0, 1)
    entries; g = F z^ + e, e ~ N(0, 0.1) (read as variance 0.1);
    mu = 0.1 ||F^T g||_inf; the SOCP of Sec. 6.2 (n = 2p + 1, m = 2p + q + 2)."""
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((q, p))
    zh = np.zeros(p)
    nz = rng.choice(p, size=max(1, p // 10), replace=False)
    zh[nz] = rng.standard_normal(nz.size)
    g = F @ zh + math.sqrt(0.1) * rng.standard_normal(q)
    mu = 0.1 * float(np.abs(F.T @ g).max())
    A, cone = lasso_socp_matrix(F)
    b = np.zeros(cone.m)
    b[2 * p] = 1.0
    b[2 * p + 1] = 1.0
    b[2 * p + 2:] = -2.0 * g
    c = np.zeros(2 * p + 1)
    c[p:2 * p] = mu
    c[2 * p] = 0.5
    return Problem(A=A, b=b, c=c, cone=cone, kind="feasible",
                   meta=dict(workload="lasso_paper", p=p, q=q, F=F, g=g, mu=mu))


def portfolio_paper(seed=0, p=100_000, q=100, gamma=1.0) -> Problem:
    """Sec. 6.3 instance, both risk terms: maximize mu^T z - gamma (t + s)
    s.t. 1^T z = 1, z >= 0, ||D^(1/2) z|| <= u, ||F^T z|| <= v,
    ||(1 - t, 2u)|| <= 1 + t, ||(1 - s, 2v)|| <= 1 + s, posed as the
    minimisation of -mu^T z + gamma (t + s).  log(mu) ~ N(0, 1);
    F (p x q) ~ N(0, 0.1) (variance 0.1); D_ii ~ U[0, 0.1]; gamma = 1.
    Variables (z, t, s, u, v): n = p + 4; rows: zero 1, nonneg p,
    SOC(p + 1) (u, D^(1/2) z), SOC(q + 1) (v, F^T z), SOC(3) twice."""
    rng = np.random.default_rng(seed)
    mu = np.exp(rng.standard_normal(p))
    F = math.sqrt(0.1) * rng.standard_normal((p, q))
    Dg = rng.uniform(0.0, 0.1, size=p)
    n = p + 4
    it, is_, iu, iv = p, p + 1, p + 2, p + 3
    Ip = sp.identity(p, format="csc")
    zc = lambda r: sp.csc_matrix((r, 4))
    one_row = lambda col, val: sp.csc_matrix(([val], ([0], [col])), shape=(1, n))
    blocks = [
        sp.hstack([sp.csc_matrix(np.ones((1, p))), zc(1)]),             # 1^T z = 1
        sp.hstack([-Ip, zc(p)]),                                         # z >= 0
        one_row(iu, -1.0),                                               # SOC(p + 1) head u
        sp.hstack([-sp.diags(np.sqrt(Dg)).tocsc(), zc(p)]),              # D^(1/2) z
        one_row(iv, -1.0),                                               # SOC(q + 1) head v
        sp.hstack([sp.csc_matrix(-F.T), zc(q)]),                         # F^T z
        one_row(it, -1.0), one_row(it, 1.0), one_row(iu, -2.0),          # (1 + t, 1 - t, 2u)
        one_row(is_, -1.0), one_row(is_, 1.0), one_row(iv, -2.0),        # (1 + s, 1 - s, 2v)
    ]
    A = sp.csc_matrix(sp.vstack(blocks))
    cone = Cone(z=1, l=p, q=(p + 1, q + 1, 3, 3))
    b = np.zeros(cone.m)
    b[0] = 1.0
    o = 1 + p + (p + 1) + (q + 1)
    b[o] = 1.0
    b[o + 1] = 1.0
    b[o + 3] = 1.0
    b[o + 4] = 1.0
    c = np.concatenate([-mu, [gamma, gamma, 0.0, 0.0]])
    assert A.shape == (cone.m, n)
    return Problem(A=A, b=b, c=c, cone=cone, kind="feasible",
                   meta=dict(workload="portfolio_paper", p=p, q=q, mu=mu, F=F, D=Dg, gamma=gamma))


def _svec_index(r, c, k):
    """Position of entry (r, c), r >= c, of an order-k block in svec order
    (lower triangle column by column)."""
    return c * k - c * (c - 1) // 2 + (r - c)


def rpca_paper(seed=0, p=100, r=10, frac=0.1) -> Problem:
    """Sec. 6.4 instance (square, p = q): M = L^ + S^ with L^ = U V^T of rank
    r (U, V ~ N(0, 1)) and S^ with about frac of its entries N(0, 1);
    mu = sum |S^|.  The SDP as printed, with the objective read as a
    minimisation (the nuclear norm is the minimum of (Tr W1 + Tr W2) / 2 over
    [W1 L; L^T W2] >= 0; the paper prints "maximize"): variables
    (vec L, vec S, t, svec W1, svec W2), rows: zero pq (L + S = M),
    nonneg 2pq + 1 (t -+ vec S >= 0, mu - 1^T t >= 0), PSD of order 2p
    (svec [W1 L; L^T W2], off-diagonal entries times sqrt 2)."""
    rng = np.random.default_rng(seed)
    q = p
    Lh = rng.standard_normal((p, r)) @ rng.standard_normal((r, q))
    Sh = np.where(rng.random((p, q)) < frac, rng.standard_normal((p, q)), 0.0)
    M = Lh + Sh
    mu = float(np.abs(Sh).sum())
    pq = p * q
    d1, d2 = p * (p + 1) // 2, q * (q + 1) // 2
    oL, oS, oT, oW1, oW2 = 0, pq, 2 * pq, 3 * pq, 3 * pq + d1
    n = 3 * pq + d1 + d2
    Ipq = sp.identity(pq, format="csc")
    Z = lambda r_, c_: sp.csc_matrix((r_, c_))
    rows_eq = sp.hstack([Ipq, Ipq, Z(pq, pq), Z(pq, d1 + d2)])
    rows_t1 = sp.hstack([Z(pq, pq), Ipq, -Ipq, Z(pq, d1 + d2)])       # t - S >= 0
    rows_t2 = sp.hstack([Z(pq, pq), -Ipq, -Ipq, Z(pq, d1 + d2)])      # t + S >= 0
    rows_mu = sp.hstack([Z(1, 2 * pq), sp.csc_matrix(np.ones((1, pq))), Z(1, d1 + d2)])
    # PSD block of order N = p + q: s = svec(block), A = -(map to the variables)
    N = p + q
    ri, ci, vv = [], [], []
    for col in range(N):
        for row in range(col, N):
            k = _svec_index(row, col, N)
            if col < p and row < p:
                ri.append(k); ci.append(oW1 + _svec_index(row, col, p)); vv.append(-1.0)
            elif col < p:                           # L^T (row - p, col) = L(col, row - p)
                ri.append(k); ci.append(oL + col + (row - p) * p); vv.append(-SQRT2)
            else:
                ri.append(k); ci.append(oW2 + _svec_index(row - p, col - p, q)); vv.append(-1.0)
    dN = N * (N + 1) // 2
    rows_psd = sp.csc_matrix((vv, (ri, ci)), shape=(dN, n))
    A = sp.csc_matrix(sp.vstack([rows_eq, rows_t1, rows_t2, rows_mu, rows_psd]))
    cone = Cone(z=pq, l=2 * pq + 1, s=(N,))
    b = np.zeros(cone.m)
    b[:pq] = M.reshape(-1, order="F")
    b[3 * pq] = mu
    c = np.zeros(n)
    for j in range(p):
        c[oW1 + _svec_index(j, j, p)] = 0.5
    for j in range(q):
        c[oW2 + _svec_index(j, j, q)] = 0.5
    assert A.shape == (cone.m, n)
    return Problem(A=A, b=b, c=c, cone=cone, kind="feasible",
                   meta=dict(workload="rpca_paper", p=p, q=q, M=M, L_hat=Lh, S_hat=Sh, mu=mu))


def logreg_paper(seed=0, p=100, q=10_000) -> Problem:
    """Sec. 6.5 instance: w_true with p/5 nonzero N(0, 1) entries, z_i ~ N(0, I),
    label y_i = +1 with probability 1/(1 + exp(-w_true^T z_i)), else -1;
    mu = 0.1 mu_max, mu_max = (1/2) ||sum_i y_i z_i||_inf.  The exponential
    cone program as printed: minimize 1^T t + mu 1^T s s.t. -s <= w <= s,
    u + v <= 1, (y_i w^T z_i - t_i, 1, u_i) in Kexp, (-t_i, 1, v_i) in Kexp;
    variables (w, s, t, u, v): n = 2p + 3q, m = 2p + 7q."""
    rng = np.random.default_rng(seed)
    wt = np.zeros(p)
    nz = rng.choice(p, size=max(1, p // 5), replace=False)
    wt[nz] = rng.standard_normal(nz.size)
    Zd = rng.standard_normal((q, p))
    prob = 1.0 / (1.0 + np.exp(-(Zd @ wt)))
    y = np.where(rng.random(q) < prob, 1.0, -1.0)
    mu = 0.1 * 0.5 * float(np.abs(y @ Zd).max())
    n = 2 * p + 3 * q
    ow, os_, ot, ou, ov = 0, p, 2 * p, 2 * p + q, 2 * p + 2 * q
    Ip, Iq = sp.identity(p, format="csc"), sp.identity(q, format="csc")
    Z = lambda r_, c_: sp.csc_matrix((r_, c_))
    r1 = sp.hstack([Ip, -Ip, Z(p, 3 * q)])                       # s - w >= 0
    r2 = sp.hstack([-Ip, -Ip, Z(p, 3 * q)])                      # s + w >= 0
    r3 = sp.hstack([Z(q, 2 * p + q), Iq, Iq])                    # 1 - u - v >= 0
    # exponential triples, three rows each, interleaved per sample
    YZ = sp.csr_matrix(-(y[:, None] * Zd))
    tri1 = sp.vstack([sp.hstack([YZ, Z(q, p), Iq, Z(q, 2 * q)]),                  # y_i z_i^T w - t_i
                      Z(q, n),                                                   # 1
                      sp.hstack([Z(q, 2 * p + q), -Iq, Z(q, q)])]).tocsr()       # u_i
    tri2 = sp.vstack([sp.hstack([Z(q, 2 * p), Iq, Z(q, 2 * q)]),                  # -t_i
                      Z(q, n),
                      sp.hstack([Z(q, 2 * p + 2 * q), -Iq])]).tocsr()            # v_i
    perm = np.arange(3 * q).reshape(3, q).T.reshape(-1)          # rows (k, i) -> triple i, entry k
    E1 = tri1[perm]
    E2 = tri2[perm]
    A = sp.csc_matrix(sp.vstack([r1, r2, r3, E1, E2]))
    cone = Cone(l=2 * p + q, ep=2 * q)
    b = np.zeros(cone.m)
    b[2 * p:2 * p + q] = 1.0
    base = 2 * p + q
    b[base + 1:base + 6 * q:3] = 1.0                             # the middle entry of every triple
    c = np.zeros(n)
    c[os_:os_ + p] = mu
    c[ot:ot + q] = 1.0
    assert A.shape == (cone.m, n)
    return Problem(A=A, b=b, c=c, cone=cone, kind="feasible",
                   meta=dict(workload="logreg_paper", p=p, q=q, Z=Zd, y=y, mu=mu, w_true=wt))
