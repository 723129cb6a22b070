"""FP64 cone projections and membership tests (oracle; test infrastructure).

The cone of the primal slack is ``K = {0}^z x R+^l x SOC... x PSD... x Kexp...``
(Sec. 2, Sec. 6.1).  The ADMM iteration projects the y-part of ``u`` onto the
dual cone ``K*`` (Eq. "e-hsdnice": ``C = R^n x K* x R+``), so both
``proj_K`` and ``proj_Kdual`` are provided.

Conventions (the paper does not fix them):
  * SOC(k) = {(t, x) in R x R^(k-1) : ||x||_2 <= t}, head first.
  * PSD blocks are stored in svec form: the lower triangle, column by
    column, with off-diagonal entries multiplied by sqrt 2, so svec is an
    isometry and the Euclidean projection in svec space is the Frobenius
    projection of the matrix.
  * Exponential triples are ordered (x, y, z) as in the definition of Kexp
    (Sec. 6.1).
  * Power triples (x, y, z) with parameter a in (0, 1):
    Kpow^a = {x^a y^(1-a) >= |z|, x >= 0, y >= 0} and its dual
    (Kpow^a)* = {(u/a)^a (v/(1-a))^(1-a) >= |w|, u >= 0, v >= 0} (Sec. 6.1).
    A cone may also hold Kexp* or (Kpow^a)* itself ("exp_dual", "pow_dual").
"""
from __future__ import annotations

import math

import numpy as np

SQRT2 = math.sqrt(2.0)
E = math.e


# ---------------------------------------------------------------------------
# svec / smat
# ---------------------------------------------------------------------------

def svec(M: np.ndarray) -> np.ndarray:
    k = M.shape[0]
    parts = []
    for j in range(k):
        col = np.array(M[j:, j], dtype=float)
        col[1:] *= SQRT2
        parts.append(col)
    return np.concatenate(parts)


def smat(v: np.ndarray, k: int) -> np.ndarray:
    M = np.zeros((k, k))
    pos = 0
    for j in range(k):
        col = np.array(v[pos:pos + k - j], dtype=float)
        col[1:] /= SQRT2
        M[j:, j] = col
        M[j, j:] = col
        pos += k - j
    return M


# ---------------------------------------------------------------------------
# single-block projections
# ---------------------------------------------------------------------------

def proj_nonneg(v):
    return np.maximum(v, 0.0)


def proj_soc(v):
    """Euclidean projection onto SOC (the textbook three-case formula)."""
    v = np.asarray(v, dtype=float)
    t, x = v[0], v[1:]
    nx = float(np.linalg.norm(x))
    if nx <= t:
        return v.copy()
    if nx <= -t:
        return np.zeros_like(v)
    a = 0.5 * (t + nx)
    out = np.empty_like(v)
    out[0] = a
    out[1:] = (a / nx) * x
    return out


def proj_psd(v, k):
    """Sec. 6.1: eigendecompose the symmetric matrix and clip negative
    eigenvalues to zero; returned in svec form."""
    M = smat(v, k)
    lam, Q = np.linalg.eigh(M)
    P = (Q * np.maximum(lam, 0.0)) @ Q.T
    return svec(0.5 * (P + P.T))


def in_exp(v, tol=0.0):
    """Membership in Kexp = {y > 0, y e^(x/y) <= z} U {x <= 0, y = 0, z >= 0},
    up to a distance ``tol * max(1, ||v||)``: accepted when a point of Kexp
    that close is exhibited (v with x moved down to the boundary value
    y ln(z/y); v with z moved up to y e^(x/y); or v moved onto the face
    {x <= 0, y = 0, z >= 0})."""
    x, y, z = (float(t) for t in v)
    slack = tol * max(1.0, math.sqrt(x * x + y * y + z * z))
    if y > 0.0 and z > 0.0 and x <= y * math.log(z / y) + slack:
        return True
    if y > 0.0 and x / y < 700.0 and y * math.exp(x / y) <= z + slack:
        return True
    face = math.sqrt(max(x, 0.0) ** 2 + y * y + min(z, 0.0) ** 2)
    return face <= slack


def in_exp_dual(v, tol=0.0):
    """Membership in Kexp* = {u < 0, -u e^(v/u) <= e w} U {(0, v, w): v, w >= 0}
    (Sec. 6.1, the factor ``e`` read as Euler's number), up to a distance
    ``tol * max(1, ||v||)``: v with its second entry moved up to the boundary
    value u (1 + ln(w/(-u))); v with w moved up to -u e^(v/u) / e; or v moved
    onto the face {u = 0, v >= 0, w >= 0}."""
    u, vv, w = (float(t) for t in v)
    slack = tol * max(1.0, math.sqrt(u * u + vv * vv + w * w))
    if u < 0.0 and w > 0.0 and vv >= u * (1.0 + math.log(w / -u)) - slack:
        return True
    if u < 0.0 and vv / u < 700.0 and -u * math.exp(vv / u) <= math.e * (w + slack):
        return True
    face = math.sqrt(u * u + min(vv, 0.0) ** 2 + min(w, 0.0) ** 2)
    return face <= slack


def _exp_h(rho, r0, s0, t0):
    """Residual of the third coordinate of ``p - d`` on the one-parameter
    family where the first two coordinates of ``v`` are matched.

    With p = y (rho, 1, e^rho) on the boundary of Kexp and its complementary
    ray d = mu (-1, rho - 1, e^-rho) on the boundary of Kexp*, the equations
    r0 = y rho + mu and s0 = y - mu (rho - 1) give
        y  = ((rho - 1) r0 + s0) / (rho^2 - rho + 1),
        mu = (r0 - rho s0)       / (rho^2 - rho + 1),
    and the projection is found where y e^rho - mu e^-rho = t0."""
    den = rho * rho - rho + 1.0
    y = ((rho - 1.0) * r0 + s0) / den
    mu = (r0 - rho * s0) / den
    with np.errstate(over="ignore", invalid="ignore"):
        return y * np.exp(rho) - mu * np.exp(-rho) - t0, y


def proj_exp(v):
    """Euclidean projection onto Kexp.

    The paper only cites the method (Sec. 6.1); this follows the projection's
    optimality conditions directly: p = Pi(v) iff p in K, p - v in K* and
    p.(p - v) = 0.  Cases: v already in K; -v in K* (v in the polar cone,
    projection 0); x <= 0 and y <= 0 (projection onto the face
    {x <= 0, y = 0, z >= 0}); otherwise p lies on the curved boundary and the
    one-dimensional root of ``_exp_h`` is found by bisection on the interval
    where y > 0 and mu > 0 (h < 0 at the end where y -> 0 because -v is not
    in K*, h > 0 at the end where mu -> 0 because v is not in K)."""
    r0, s0, t0 = (float(t) for t in v)
    if in_exp((r0, s0, t0)):
        return np.array([r0, s0, t0])
    if in_exp_dual((-r0, -s0, -t0)):
        return np.zeros(3)
    if r0 <= 0.0 and s0 <= 0.0:
        return np.array([r0, 0.0, max(t0, 0.0)])
    # interval of rho on which y > 0 and mu > 0
    lo, hi = -math.inf, math.inf
    if r0 > 0.0:
        lo = 1.0 - s0 / r0          # y -> 0 here
    if s0 > 0.0:
        hi = r0 / s0                # mu -> 0 here
    if not math.isfinite(lo):
        step = 1.0
        lo = hi - step
        while _exp_h(lo, r0, s0, t0)[0] >= 0.0:
            step *= 2.0
            lo = hi - step
    if not math.isfinite(hi):
        step = 1.0
        hi = lo + step
        while _exp_h(hi, r0, s0, t0)[0] <= 0.0:
            step *= 2.0
            hi = lo + step
    for _ in range(400):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        h, _y = _exp_h(mid, r0, s0, t0)
        if h < 0.0:
            lo = mid
        else:
            hi = mid
    rho = 0.5 * (lo + hi)
    # p = y (rho, 1, e^rho) and p = v + mu (-1, rho - 1, e^-rho) are equal at
    # the root; return the one whose rounding error bound is smaller (y
    # cancels near the end where y -> 0, mu near the end where mu -> 0).
    den = rho * rho - rho + 1.0
    y = ((rho - 1.0) * r0 + s0) / den
    mu = (r0 - rho * s0) / den
    with np.errstate(over="ignore"):
        ray_p = np.array([rho, 1.0, np.exp(rho)])
        ray_d = np.array([-1.0, rho - 1.0, np.exp(-rho)])
    with np.errstate(over="ignore", invalid="ignore"):
        err_p = (abs(rho - 1.0) * abs(r0) + abs(s0)) / den * np.sqrt(ray_p @ ray_p)
        err_d = ((abs(r0) + abs(rho) * abs(s0)) / den * np.sqrt(ray_d @ ray_d)
                 + math.sqrt(r0 * r0 + s0 * s0 + t0 * t0))
    if err_p <= err_d:
        return y * ray_p
    return np.array([r0, s0, t0]) + mu * ray_d


def proj_exp_dual(v):
    """Moreau (Eq. "e-moreau" applied to K*): Pi_{K*}(w) = w + Pi_K(-w)."""
    v = np.asarray(v, dtype=float)
    return v + proj_exp(-v)


def _pow_dist(v1, v2, w, a, s1, s2):
    """Upper bound on the distance from (v1, v2, w) to the cone
    {(v1/s1)^a (v2/s2)^(1-a) >= |w|, v1 >= 0, v2 >= 0}: the smallest of three
    moves onto it -- negative v1, v2 raised to 0 and |w| lowered to the
    boundary value; or v1 raised (or v2 raised) until the boundary reaches
    |w|, with the other entry raised to 0 if negative."""
    p1, p2 = max(v1, 0.0), max(v2, 0.0)
    aw = abs(w)
    r = (p1 / s1) ** a * (p2 / s2) ** (1.0 - a)
    best = math.sqrt((p1 - v1) ** 2 + (p2 - v2) ** 2 + max(aw - r, 0.0) ** 2)
    try:
        if p2 > 0.0:
            need1 = s1 * (aw / (p2 / s2) ** (1.0 - a)) ** (1.0 / a)
            best = min(best, math.sqrt(max(need1 - v1, 0.0) ** 2 + (p2 - v2) ** 2))
        if p1 > 0.0:
            need2 = s2 * (aw / (p1 / s1) ** a) ** (1.0 / (1.0 - a))
            best = min(best, math.sqrt((p1 - v1) ** 2 + max(need2 - v2, 0.0) ** 2))
    except OverflowError:
        pass
    return best


def in_pow(v, a, tol=0.0):
    """Membership in Kpow^a = {x^a y^(1-a) >= |z|, x >= 0, y >= 0} up to a
    distance ``tol * max(1, ||v||)`` (accepted when one of the moves of
    ``_pow_dist`` reaches the cone within it)."""
    x, y, z = (float(t) for t in v)
    slack = tol * max(1.0, math.sqrt(x * x + y * y + z * z))
    return _pow_dist(x, y, z, a, 1.0, 1.0) <= slack


def in_pow_dual(v, a, tol=0.0):
    """Membership in (Kpow^a)* = {(u/a)^a (v/(1-a))^(1-a) >= |w|, u, v >= 0}
    (Sec. 6.1), with the same distance test as ``in_pow``."""
    u, vv, w = (float(t) for t in v)
    slack = tol * max(1.0, math.sqrt(u * u + vv * vv + w * w))
    return _pow_dist(u, vv, w, a, a, 1.0 - a) <= slack


def _pow_branch(c0, k, r, r0):
    """The positive root t of t^2 - c0 t - k r (r0 - r) = 0 (k r (r0 - r) >= 0),
    written without cancellation for c0 < 0."""
    q = k * r * (r0 - r)
    d = math.sqrt(c0 * c0 + 4.0 * q)
    return 0.5 * (c0 + d) if c0 >= 0.0 else 2.0 * q / (d - c0) if d - c0 > 0.0 else 0.0


def proj_pow(v, a):
    """Euclidean projection onto Kpow^a (Sec. 6.1 gives only the cone).

    From the projection's optimality conditions: p = Pi(v) iff p in K,
    p - v in K* and p.(p - v) = 0.  Cases: v in K; -v in K* (projection 0);
    z0 = 0 (projection (x0+, y0+, 0)).  Otherwise p lies on the curved
    boundary x^a y^(1-a) = |z| with z of the sign of z0.  With r = |z| and
    the multiplier mu of the constraint g = x^a y^(1-a) - |z| >= 0, the
    stationarity p - v = mu grad g reads
        x - x0 = mu a r / x,   y - y0 = mu (1 - a) r / y,   r - |z0| = -mu,
    so mu = |z0| - r and x, y are the positive roots of
        x^2 - x0 x - a r (|z0| - r) = 0,   y^2 - y0 y - (1-a) r (|z0| - r) = 0;
    r is the root in (0, |z0|) of phi(r) = x(r)^a y(r)^(1-a) - r, where phi
    changes sign from >= 0 at r = 0 to < 0 at r = |z0| (v not in K), found
    by bisection."""
    x0, y0, z0 = (float(t) for t in v)
    if in_pow((x0, y0, z0), a):
        return np.array([x0, y0, z0])
    if in_pow_dual((-x0, -y0, -z0), a):
        return np.zeros(3)
    if z0 == 0.0:
        return np.array([max(x0, 0.0), max(y0, 0.0), 0.0])
    r0 = abs(z0)

    def phi(r):
        x = _pow_branch(x0, a, r, r0)
        y = _pow_branch(y0, 1.0 - a, r, r0)
        return x ** a * y ** (1.0 - a) - r, x, y

    lo, hi = 0.0, r0
    for _ in range(300):
        mid = 0.5 * (lo + hi)
        if mid <= lo or mid >= hi:
            break
        if phi(mid)[0] > 0.0:
            lo = mid
        else:
            hi = mid
    r = 0.5 * (lo + hi)
    _, x, y = phi(r)
    return np.array([x, y, math.copysign(r, z0)])


def proj_pow_dual(v, a):
    """Moreau (Eq. "e-moreau" applied to K*): Pi_{K*}(w) = w + Pi_K(-w)."""
    v = np.asarray(v, dtype=float)
    return v + proj_pow(-v, a)


# ---------------------------------------------------------------------------
# whole-cone projections and membership
# ---------------------------------------------------------------------------

def proj_K(v, cone):
    """Euclidean projection onto K (block by block)."""
    v = np.asarray(v, dtype=float)
    out = np.empty_like(v)
    for kind, off, size, order in cone.blocks():
        seg = v[off:off + size]
        if kind == "zero":
            out[off:off + size] = 0.0
        elif kind == "nonneg":
            out[off:off + size] = proj_nonneg(seg)
        elif kind == "soc":
            out[off:off + size] = proj_soc(seg)
        elif kind == "psd":
            out[off:off + size] = proj_psd(seg, order)
        elif kind == "exp":
            out[off:off + size] = proj_exp(seg)
        elif kind == "exp_dual":
            out[off:off + size] = proj_exp_dual(seg)
        elif kind == "pow":
            out[off:off + size] = proj_pow(seg, order)
        elif kind == "pow_dual":
            out[off:off + size] = proj_pow_dual(seg, order)
    return out


def proj_Kdual(v, cone):
    """Euclidean projection onto K*: the dual of {0} is R (free), the
    nonnegative, second-order and PSD cones are self-dual, Kexp* and
    (Kpow^a)* via Moreau; the dual of Kexp* is Kexp, of (Kpow^a)* Kpow^a."""
    v = np.asarray(v, dtype=float)
    out = np.empty_like(v)
    for kind, off, size, order in cone.blocks():
        seg = v[off:off + size]
        if kind == "zero":
            out[off:off + size] = seg
        elif kind == "nonneg":
            out[off:off + size] = proj_nonneg(seg)
        elif kind == "soc":
            out[off:off + size] = proj_soc(seg)
        elif kind == "psd":
            out[off:off + size] = proj_psd(seg, order)
        elif kind == "exp":
            out[off:off + size] = proj_exp_dual(seg)
        elif kind == "exp_dual":
            out[off:off + size] = proj_exp(seg)
        elif kind == "pow":
            out[off:off + size] = proj_pow_dual(seg, order)
        elif kind == "pow_dual":
            out[off:off + size] = proj_pow(seg, order)
    return out


def _in_soc(seg, tol):
    return np.linalg.norm(seg[1:]) <= seg[0] + tol * max(1.0, abs(seg[0]))


def _in_psd(seg, order, tol):
    lam = np.linalg.eigvalsh(smat(seg, order))
    return lam.min() >= -tol * max(1.0, np.abs(lam).max())


def in_K(v, cone, tol=1e-9):
    for kind, off, size, order in cone.blocks():
        seg = np.asarray(v[off:off + size], dtype=float)
        if kind == "zero" and np.abs(seg).max() > tol:
            return False
        if kind == "nonneg" and seg.min() < -tol:
            return False
        if kind == "soc" and not _in_soc(seg, tol):
            return False
        if kind == "psd" and not _in_psd(seg, order, tol):
            return False
        if kind == "exp" and not in_exp(seg, tol):
            return False
        if kind == "exp_dual" and not in_exp_dual(seg, tol):
            return False
        if kind == "pow" and not in_pow(seg, order, tol):
            return False
        if kind == "pow_dual" and not in_pow_dual(seg, order, tol):
            return False
    return True


def in_Kdual(v, cone, tol=1e-9):
    for kind, off, size, order in cone.blocks():
        seg = np.asarray(v[off:off + size], dtype=float)
        if kind == "nonneg" and seg.min() < -tol:
            return False
        if kind == "soc" and not _in_soc(seg, tol):
            return False
        if kind == "psd" and not _in_psd(seg, order, tol):
            return False
        if kind == "exp" and not in_exp_dual(seg, tol):
            return False
        if kind == "exp_dual" and not in_exp(seg, tol):
            return False
        if kind == "pow" and not in_pow_dual(seg, order, tol):
            return False
        if kind == "pow_dual" and not in_pow(seg, order, tol):
            return False
    return True
