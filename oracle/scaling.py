"""Data equilibration of Sec. 5 (oracle; test infrastructure).

Sec. 5 scales the data to  A^ = D A E,  b^ = sigma D b,  c^ = rho E c  with
positive diagonal D (which must preserve K, so it is one scalar per cone block
for the SOC, PSD and exponential blocks) and E, and positive scalars sigma and
rho.  It names the goal -- columns of A and b with Euclidean norm near one,
rows of A and c with similar norms -- and cites Ruiz, but gives no algorithm.
The reading implemented here (identically, but independently, on the GPU):

  repeat ``passes`` times:
    r_i = ||row_i(A^)||_2 and c_j = ||col_j(A^)||_2, both from the current A^;
    over every SOC, PSD and exponential block, replace r_i by one value for
    the block (``block``: the root mean square of the block's norms -- the
    Frobenius norm of the block over the square root of its row count, the
    block form of a 2-norm row equilibration -- or their mean, or maximum);
    a norm below ``lo`` is replaced by 1 (nothing to scale), a norm above
    ``hi`` is clamped to ``hi``;
    d_i = 1/sqrt(r_i), e_j = 1/sqrt(c_j);  A^ <- diag(d) A^ diag(e);
    D <- D d, E <- E e.
  then  sigma = 1 / max(||D b||_2, lo)  (so ||b^|| = 1, b joins the columns)
  and   rho = mean_i ||row_i(A^)||_2 / max(||E c||_2, lo)
        (so ||c^|| equals the mean row norm, c joins the rows).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _clamp(nrm, lo, hi):
    nrm = np.where(nrm < lo, 1.0, nrm)
    return np.minimum(nrm, hi)


def _block_value(seg, block):
    if block == "rms":
        return float(np.sqrt(np.mean(seg * seg)))
    if block == "max":
        return float(seg.max())
    return float(seg.mean())


def equilibrate(A, b, c, cone, passes=10, lo=1e-4, hi=1e4, block="rms"):
    """Return ``(A_hat (csr), b_hat, c_hat, D, E, sigma, rho)``."""
    A = sp.csr_matrix(A, dtype=np.float64, copy=True)
    m, n = A.shape
    D = np.ones(m)
    E = np.ones(n)
    for _ in range(passes):
        sq = A.multiply(A)
        rn = np.sqrt(np.asarray(sq.sum(axis=1)).ravel())
        cn = np.sqrt(np.asarray(sq.sum(axis=0)).ravel())
        for kind, off, size, _order in cone.blocks():
            if kind in ("soc", "psd", "exp", "exp_dual", "pow", "pow_dual"):
                rn[off:off + size] = _block_value(rn[off:off + size], block)
        d = 1.0 / np.sqrt(_clamp(rn, lo, hi))
        e = 1.0 / np.sqrt(_clamp(cn, lo, hi))
        A = sp.csr_matrix(sp.diags(d) @ A @ sp.diags(e))
        D *= d
        E *= e
    sq = A.multiply(A)
    mean_row = float(np.sqrt(np.asarray(sq.sum(axis=1)).ravel()).mean()) if m else 1.0
    if not mean_row > 0.0:
        mean_row = 1.0
    sigma = 1.0 / max(float(np.linalg.norm(D * b)), lo)
    rho = mean_row / max(float(np.linalg.norm(E * c)), lo)
    b_hat = sigma * D * b
    c_hat = rho * E * c
    return A, b_hat, c_hat, D, E, sigma, rho


def identity_scaling(A, b, c):
    m, n = A.shape
    return (sp.csr_matrix(A, dtype=np.float64, copy=True), np.array(b, float),
            np.array(c, float), np.ones(m), np.ones(n), 1.0, 1.0)
