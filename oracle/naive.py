"""Un-simplified ADMM on the embedding, Eq. "e-SCS-naive" (oracle; test infrastructure).

Sec. 3.1 applies ADMM to Eq. "e-consensus" directly:
    (u~, v~) = Pi_{Qu=v}(u^k + lambda^k, v^k + mu^k)
    u+       = Pi_C(u~ - lambda^k)
    v+       = Pi_C*(v~ - mu^k)
    lambda+  = lambda^k - u~ + u+
    mu+      = mu^k - v~ + v+
Sec. 3.2.1 shows that with lambda^0 = v^0 and mu^0 = u^0 its (u, v) iterates
equal those of the simplified method.  Dense and small by design: the
projection onto {(u, v) : v = Q u} solves the normal equations of
min ||u - a||^2 + ||Q u - b||^2, i.e. (I + Q^T Q) u = a + Q^T b, v = Q u.
"""
from __future__ import annotations

import numpy as np

from . import cones as _cones


def hsd_Q(A, b, c):
    """The skew-symmetric matrix Q of Sec. 2.3 (dense)."""
    A = np.asarray(A.todense() if hasattr(A, "todense") else A, dtype=float)
    m, n = A.shape
    N = n + m + 1
    Q = np.zeros((N, N))
    Q[:n, n:n + m] = A.T
    Q[:n, -1] = c
    Q[n:n + m, :n] = -A
    Q[n:n + m, -1] = b
    Q[-1, :n] = -c
    Q[-1, n:n + m] = -b
    return Q


def run(A, b, c, cone, iters, u0=None, v0=None):
    """Return the list of (u^k, v^k), k = 1..iters, of Eq. "e-SCS-naive"."""
    Q = hsd_Q(A, b, c)
    N = Q.shape[0]
    m = cone.m
    n = N - m - 1
    if u0 is None:
        u0 = np.zeros(N)
        u0[-1] = 1.0
    if v0 is None:
        v0 = np.zeros(N)
        v0[-1] = 1.0
    u, v = u0.copy(), v0.copy()
    lam, mu = v.copy(), u.copy()
    G = np.eye(N) + Q.T @ Q

    def proj_C(x):
        out = x.copy()
        out[n:n + m] = _cones.proj_Kdual(x[n:n + m], cone)
        out[-1] = max(x[-1], 0.0)
        return out

    def proj_Cdual(x):
        out = np.zeros_like(x)               # {0}^n
        out[n:n + m] = _cones.proj_K(x[n:n + m], cone)
        out[-1] = max(x[-1], 0.0)
        return out

    out = []
    for _ in range(iters):
        a, bb = u + lam, v + mu
        ut = np.linalg.solve(G, a + Q.T @ bb)
        vt = Q @ ut
        u = proj_C(ut - lam)
        v = proj_Cdual(vt - mu)
        lam = lam - ut + u
        mu = mu - vt + v
        out.append((u.copy(), v.copy()))
    return out
