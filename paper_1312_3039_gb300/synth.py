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
    Ip = sp.identity(p, format="csc")
    Z = sp.csc_matrix((p, p))
    top = sp.hstack([Ip, -Ip, sp.csc_matrix((p, 1))])
    mid = sp.hstack([-Ip, -Ip, sp.csc_matrix((p, 1))])
    head = sp.csc_matrix(np.concatenate([np.zeros(2 * p), [-1.0]])[None, :])
    head2 = sp.csc_matrix(np.concatenate([np.zeros(2 * p), [1.0]])[None, :])
    tail = sp.hstack([sp.csc_matrix(-2.0 * F), sp.csc_matrix((q, p)), sp.csc_matrix((q, 1))])
    A = sp.csc_matrix(sp.vstack([top, mid, head, head2, tail]))
    del Z
    cone = Cone(l=2 * p, q=(q + 2,))
    assert A.shape == (cone.m, 2 * p + 1)
    return LassoFamily(F=F, G=G, a=a, mu0=mu0, A=A, cone=cone)
