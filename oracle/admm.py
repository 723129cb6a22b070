"""ADMM on the homogeneous self-dual embedding, FP64 (oracle; test infrastructure).

Follows, in order:
  * Eq. "e-hsd" / "e-hsdnice" (Sec. 2.3): u = (x, y, tau), v = (r, s, kappa),
    v = Q u, (u, v) in C x C*, C = R^n x K* x R+.
  * Eq. "e-SCS" (Sec. 3.2.3) with over-relaxation (Sec. 3.3):
        u~    = (I + Q)^-1 (u^k + v^k)
        u_bar = alpha u~ + (1 - alpha) u^k
        u+    = Pi_C(u_bar - v^k)
        v+    = v^k - u_bar + u+
  * Initial point (Sec. 3.4): u0 = (0, 0, 1), v0 = (0, 0, 1); warm start
    (Sec. 4.2): u0 = (x, y, 1), v0 = (0, s, 0), in scaled coordinates.
  * Linear system (Sec. 4.1, Eq. "e-lin-sys"): M = [I A^T; -A I], h = (c, b),
    p = M^-1 h cached; (u~_x, u~_y) = z - p (h^T z)/(1 + h^T p) with
    z = M^-1 (w_xy - w_tau h); u~_tau = w_tau + c^T u~_x + b^T u~_y.
    M^-1 is applied either
      - "direct": a sparse factorisation of the quasi-definite matrix of
        Eq. "e-linsys", [I -A^T; -A -I] (z_x, -z_y) = (w_x, w_y), computed
        once and cached (factorisation caching), or
      - "indirect": z_x = (I + A^T A)^-1 (w_x - A^T w_y) by Jacobi-
        preconditioned CG warm-started from the previous z_x, stopped when
        the residual is below zeta^k = (1/k)^cg_rate (Sec. 3.3 Eq.
        "e-approx-proj-resid", Sec. 6.1), then z_y = w_y + A z_x.
        Reading: the tolerance is also capped at cg_adapt times the length
        ||(u^k - u^(k-1), v^k - v^(k-1))|| of the previous ADMM step (after a
        warm start: max(eps) * ||(u0, v0)||).  A cap below zeta^k keeps the
        tolerances summable, as Sec. 3.3 requires, while tracking the
        accuracy the iteration has reached: with the absolute schedule alone
        a certificate test that needs ~1e-6 relative accuracy is not met
        before k ~ 1e4, and a warm start is undone by the loose first solves.
  * Termination (Sec. 3.5) on the scaled data (Sec. 5, "Scaled termination
    criteria"), every ``check_interval`` iterations, tested in the order
    optimality, primal infeasibility, dual infeasibility.
  * Certificates (Sec. 2.3 cases): y/(-b^T y) and x/(-c^T x).

The whole vector v is kept, including v_x (= r), which the iteration keeps at
exactly zero because the x-part of C is all of R^n.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math
import time

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import cones as _cones
from .scaling import equilibrate, identity_scaling

SOLVED = 1
SOLVED_INACCURATE = 2
INFEASIBLE = -1
UNBOUNDED = -2
INFEASIBLE_INACCURATE = -3
UNBOUNDED_INACCURATE = -4
UNFINISHED = 0


@dataclass
class Settings:
    eps_pri: float = 1e-4
    eps_dual: float = 1e-4
    eps_gap: float = 1e-4
    eps_infeas: float = 1e-4
    eps_unbdd: float = 1e-4
    alpha: float = 1.5
    max_iters: int = 10000
    check_interval: int = 20
    normalize: bool = True
    scale_passes: int = 10
    block_scale: str = "rms"        # one D value per cone block: "mean", "rms" or "max" of its row norms
    linsys: str = "direct"          # "direct" | "indirect"
    cg_rate: float = 1.5            # zeta^k = (1/k)^cg_rate; <= 0 disables it
    cg_adapt: float = 0.3           # also at most cg_adapt * (last ADMM step length); 0 disables
    cg_tol_rel: float = 0.0         # floor: cg_tol_rel * ||w||
    cg_max_iters: int = 1000


@dataclass
class Result:
    status: int
    x: np.ndarray
    y: np.ndarray
    s: np.ndarray
    iters: int
    pobj: float
    dobj: float
    res_pri: float
    res_dual: float
    gap: float
    tau: float
    kappa: float
    cg_iters: int = 0
    matvecs: int = 0
    solve_s: float = 0.0
    trajectory: list = field(default_factory=list)


class HSDSolver:
    """Holds the scaled data and the iterates (u, v) of one problem."""

    def __init__(self, A, b, c, cone, settings: Settings | None = None):
        self.st = settings or Settings()
        self.cone = cone
        A = sp.csc_matrix(A, dtype=np.float64)
        self.m, self.n = A.shape
        self.b_orig = np.asarray(b, float)
        self.c_orig = np.asarray(c, float)
        if self.st.normalize:
            Ah, bh, ch, D, E, sigma, rho = equilibrate(A, b, c, cone, self.st.scale_passes,
                                                       block=self.st.block_scale)
        else:
            Ah, bh, ch, D, E, sigma, rho = identity_scaling(A, b, c)
        self.A = sp.csr_matrix(Ah)
        self.At = sp.csr_matrix(Ah.T)
        self.b, self.c = bh, ch
        self.D, self.E, self.sigma, self.rho = D, E, sigma, rho
        self.h = np.concatenate([ch, bh])
        self.matvecs = 0
        self.cg_iters = 0
        n, m = self.n, self.m
        if self.st.linsys == "direct":
            K = sp.bmat([[sp.identity(n), -self.At], [-self.A, -sp.identity(m)]], format="csc")
            self._lu = spla.splu(K)
        else:
            self.pre = 1.0 + np.asarray(self.A.multiply(self.A).sum(axis=0)).ravel()
            self.z_prev = np.zeros(n)
        # cached p = M^-1 h and 1 + h^T p (Sec. 4.1)
        self.p = self._solve_M(self.h, k=None)
        self.hp1 = 1.0 + float(self.h @ self.p)
        if self.st.linsys == "indirect":
            self.z_prev = np.zeros(n)
        self.reset()

    # -- iterates ---------------------------------------------------------
    def reset(self):
        n, m = self.n, self.m
        self.u = np.zeros(n + m + 1)
        self.v = np.zeros(n + m + 1)
        self.u[-1] = 1.0
        self.v[-1] = 1.0
        self.k = 0
        self.dstep = math.inf

    def warm_start(self, x, y, s):
        """Sec. 4.2: u0 = (x, y, 1), v0 = (0, s, 0), mapped into the scaled
        problem (x^ = sigma E^-1 x, y^ = rho D^-1 y, s^ = sigma D s)."""
        n = self.n
        self.u = np.concatenate([self.sigma * np.asarray(x) / self.E,
                                 self.rho * np.asarray(y) / self.D, [1.0]])
        self.v = np.concatenate([np.zeros(n), self.sigma * self.D * np.asarray(s), [0.0]])
        self.k = 0
        st = self.st
        self.dstep = max(st.eps_pri, st.eps_dual, st.eps_gap) * float(
            np.linalg.norm(np.concatenate([self.u, self.v])))

    # -- linear system ----------------------------------------------------
    def _solve_M(self, r, k):
        """z = M^-1 r with M = [I A^T; -A I]."""
        n = self.n
        if self.st.linsys == "direct":
            sol = self._lu.solve(r)
            return np.concatenate([sol[:n], -sol[n:]])
        rx, ry = r[:n], r[n:]
        t = rx - self.At @ ry
        self.matvecs += 1
        if k is None:       # setup solve of p: as tight as FP64 allows
            tol = 1e-14 * max(np.linalg.norm(t), 1e-300)
            zx = self._pcg(t, np.zeros(n), tol, max(self.st.cg_max_iters, 10 * n))
        else:
            tol = math.inf
            if self.st.cg_rate > 0:
                tol = (1.0 / k) ** self.st.cg_rate
            if self.st.cg_adapt > 0:
                tol = min(tol, self.st.cg_adapt * self.dstep)
            if not math.isfinite(tol):
                tol = 0.0
            tol = max(tol, self.st.cg_tol_rel * self._wnorm)
            zx = self._pcg(t, self.z_prev, tol, self.st.cg_max_iters)
            self.z_prev = zx.copy()
        zy = ry + self.A @ zx
        self.matvecs += 1
        return np.concatenate([zx, zy])

    def _G(self, x):
        self.matvecs += 2
        return x + self.At @ (self.A @ x)

    def _pcg(self, t, x0, tol, max_iters):
        """Jacobi-preconditioned CG on (I + A^T A) x = t from x0, stopped
        when ||t - (I + A^T A) x||_2 <= tol."""
        x = x0.copy()
        r = t - self._G(x)
        if np.linalg.norm(r) <= tol:
            return x
        zr = r / self.pre
        p = zr.copy()
        rz = float(r @ zr)
        for _ in range(max_iters):
            Gp = self._G(p)
            a = rz / float(p @ Gp)
            x += a * p
            r -= a * Gp
            self.cg_iters += 1
            if np.linalg.norm(r) <= tol:
                break
            zr = r / self.pre
            rz_new = float(r @ zr)
            p = zr + (rz_new / rz) * p
            rz = rz_new
        return x

    def solve_IQ(self, w, k=None):
        """u~ = (I + Q)^-1 w via Sherman-Morrison-Woodbury (Sec. 4.1)."""
        n, m = self.n, self.m
        wxy, wt = w[:n + m], w[-1]
        z = self._solve_M(wxy - wt * self.h, k)
        ut_xy = z - self.p * (float(self.h @ z) / self.hp1)
        ut_t = wt + float(self.c @ ut_xy[:n]) + float(self.b @ ut_xy[n:])
        return np.concatenate([ut_xy, [ut_t]])

    # -- one iteration of Eq. "e-SCS" with relaxation -----------------------
    def proj_C(self, x):
        """Pi_C with C = R^n x K* x R+ (Eq. "e-hsdnice")."""
        n, m = self.n, self.m
        out = np.empty_like(x)
        out[:n] = x[:n]
        out[n:n + m] = _cones.proj_Kdual(x[n:n + m], self.cone)
        out[-1] = max(x[-1], 0.0)
        return out

    def step(self):
        self.k += 1
        w = self.u + self.v
        if self.st.linsys == "indirect":
            self._wnorm = float(np.linalg.norm(w))
        ut = self.solve_IQ(w, self.k)
        a = self.st.alpha
        ubar = a * ut + (1.0 - a) * self.u
        u_new = self.proj_C(ubar - self.v)
        v_new = self.v - ubar + u_new
        self.dstep = float(np.sqrt(np.sum((u_new - self.u) ** 2) + np.sum((v_new - self.v) ** 2)))
        self.u, self.v = u_new, v_new

    # -- termination (Sec. 3.5 and Sec. 5) -----------------------------------
    def residuals(self):
        n, m = self.n, self.m
        ux, uy, tau = self.u[:n], self.u[n:n + m], self.u[-1]
        vs, kappa = self.v[n:n + m], self.v[-1]
        Ax = self.A @ ux
        Aty = self.At @ uy
        D, E, sg, rh = self.D, self.E, self.sigma, self.rho
        out = dict(tau=tau, kappa=kappa)
        cx = float(self.c @ ux)
        by = float(self.b @ uy)
        out["ctx"], out["bty"] = cx, by
        if tau > 0:
            out["pri"] = np.linalg.norm((Ax + vs - tau * self.b) / D) / (tau * sg)
            out["dual"] = np.linalg.norm((Aty + tau * self.c) / E) / (tau * rh)
            out["cx"] = cx / (tau * rh * sg)
            out["by"] = by / (tau * rh * sg)
            out["gap"] = abs(out["cx"] + out["by"])
        else:
            out["pri"] = out["dual"] = out["gap"] = math.inf
            out["cx"] = out["by"] = math.nan
        out["infeas_res"] = np.linalg.norm(Aty / E)
        out["unbdd_res"] = np.linalg.norm((Ax + vs) / D)
        return out

    def check(self):
        st = self.st
        r = self.residuals()
        nb = float(np.linalg.norm(self.b_orig))
        nc = float(np.linalg.norm(self.c_orig))
        if r["tau"] > 0:
            if (r["pri"] <= st.eps_pri * (1 + nb) and r["dual"] <= st.eps_dual * (1 + nc)
                    and r["gap"] <= st.eps_gap * (1 + abs(r["cx"]) + abs(r["by"]))):
                return SOLVED, r
        if nb > 0 and r["bty"] < 0:
            if r["infeas_res"] <= (-r["bty"] / (self.sigma * nb)) * st.eps_infeas:
                return INFEASIBLE, r
        if nc > 0 and r["ctx"] < 0:
            if r["unbdd_res"] <= (-r["ctx"] / (self.rho * nc)) * st.eps_unbdd:
                return UNBOUNDED, r
        return UNFINISHED, r

    # -- output --------------------------------------------------------------
    def result(self, status, r, t0, trajectory):
        n, m = self.n, self.m
        ux, uy, tau = self.u[:n], self.u[n:n + m], self.u[-1]
        vs = self.v[n:n + m]
        nan_n, nan_m = np.full(n, np.nan), np.full(m, np.nan)
        if status in (SOLVED, SOLVED_INACCURATE):
            x = self.E * ux / (tau * self.sigma)
            y = self.D * uy / (tau * self.rho)
            s = vs / (self.D * tau * self.sigma)
        elif status in (INFEASIBLE, INFEASIBLE_INACCURATE):
            y = self.D * uy
            y = y / (-float(self.b_orig @ y))
            x, s = nan_n, nan_m
        elif status in (UNBOUNDED, UNBOUNDED_INACCURATE):
            x = self.E * ux
            x = x / (-float(self.c_orig @ x))
            s = -(sp.csc_matrix(self._A_orig) @ x) if hasattr(self, "_A_orig") else nan_m
            y = nan_m
        else:
            x, y, s = nan_n, nan_m, nan_m
        pobj = float(self.c_orig @ x) if np.all(np.isfinite(x)) else math.nan
        dobj = -float(self.b_orig @ y) if np.all(np.isfinite(y)) else math.nan
        return Result(status=status, x=x, y=y, s=s, iters=self.k, pobj=pobj, dobj=dobj,
                      res_pri=r.get("pri", math.nan), res_dual=r.get("dual", math.nan),
                      gap=r.get("gap", math.nan), tau=float(tau), kappa=float(self.v[-1]),
                      cg_iters=self.cg_iters, matvecs=self.matvecs,
                      solve_s=time.perf_counter() - t0, trajectory=trajectory)

    def solve(self, record=0):
        """Iterate until a check passes or ``max_iters``; ``record`` keeps the
        first ``record`` iterates (u, v) for trajectory comparisons."""
        st = self.st
        t0 = time.perf_counter()
        traj = []
        status, r = UNFINISHED, {}
        while self.k < st.max_iters:
            self.step()
            if len(traj) < record:
                traj.append((self.u.copy(), self.v.copy()))
            if self.k % st.check_interval == 0 or self.k == st.max_iters:
                status, r = self.check()
                if status != UNFINISHED:
                    break
        if status == UNFINISHED:
            status = self._inaccurate_status(r)
        return self.result(status, r, t0, traj)

    def _inaccurate_status(self, r):
        if r.get("tau", 0.0) > 0 and r["tau"] >= r["kappa"]:
            return SOLVED_INACCURATE
        if r.get("bty", 0.0) < 0 and r["bty"] <= r.get("ctx", 0.0):
            return INFEASIBLE_INACCURATE
        if r.get("ctx", 0.0) < 0:
            return UNBOUNDED_INACCURATE
        return SOLVED_INACCURATE if r.get("tau", 0.0) > 0 else INFEASIBLE_INACCURATE


def solve(A, b, c, cone, settings: Settings | None = None, warm=None, record=0) -> Result:
    """Solve ``min c^T x s.t. A x + s = b, s in K`` (Eq. "e-coneprob")."""
    S = HSDSolver(A, b, c, cone, settings)
    S._A_orig = sp.csc_matrix(A, dtype=np.float64)
    if warm is not None:
        S.warm_start(*warm)
    return S.solve(record=record)
