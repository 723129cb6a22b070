"""The oracle's pins catch plausible mistakes: each case plants one mistake
in the oracle (a flipped sign, a dropped term or factor, swapped weights, a
missing clip or scaling) and runs the pin that guards that step; the pin must
fail.  (Mistakes that only make the method stop later, such as an
over-reported residual, do not change a correct result and are out of reach
of result pins.)

Planted only in the oracle, on the CPU (monkeypatch, undone after each case).
"""
import numpy as np
import pytest

from oracle import admm, cones
from oracle import mlp as omlp

import test_oracle_admm as pins_admm
import test_oracle_cones as pins_cones
import test_oracle_mlp as pins_mlp


# ---- subspace step (Sec. 4.1) ------------------------------------------------

def iq_gamma_sign(self, w, k=None):
    n, m = self.n, self.m
    wxy, wt = w[:n + m], w[-1]
    z = self._solve_M(wxy - wt * self.h, k)
    ut_xy = z + self.p * (float(self.h @ z) / self.hp1)          # planted: + instead of -
    ut_t = wt + float(self.c @ ut_xy[:n]) + float(self.b @ ut_xy[n:])
    return np.concatenate([ut_xy, [ut_t]])


def iq_tau_drops_b(self, w, k=None):
    n, m = self.n, self.m
    wxy, wt = w[:n + m], w[-1]
    z = self._solve_M(wxy - wt * self.h, k)
    ut_xy = z - self.p * (float(self.h @ z) / self.hp1)
    ut_t = wt + float(self.c @ ut_xy[:n])                       # planted: b^T u~_y dropped
    return np.concatenate([ut_xy, [ut_t]])


_solve_M = admm.HSDSolver._solve_M


def solve_M_zy_sign(self, r, k):
    z = _solve_M(self, r, k).copy()
    z[self.n:] = -z[self.n:]                                    # planted: sign of z_y
    return z


def pcg_residual_sign(self, t, x0, tol, max_iters):
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
        r += a * Gp                                             # planted: residual updated with + a G p
        self.cg_iters += 1
        if np.linalg.norm(r) <= tol:
            break
        zr = r / self.pre
        rz_new = float(r @ zr)
        p = zr + (rz_new / rz) * p
        rz = rz_new
    return x


# ---- the iteration (Eq. "e-SCS" with relaxation) -------------------------------

def step_relax_swapped(self):
    self.k += 1
    w = self.u + self.v
    if self.st.linsys == "indirect":
        self._wnorm = float(np.linalg.norm(w))
    ut = self.solve_IQ(w, self.k)
    a = self.st.alpha
    ubar = (1.0 - a) * ut + a * self.u                          # planted: weights swapped
    u_new = self.proj_C(ubar - self.v)
    v_new = self.v - ubar + u_new
    self.u, self.v = u_new, v_new


def step_dual_sign(self):
    self.k += 1
    w = self.u + self.v
    if self.st.linsys == "indirect":
        self._wnorm = float(np.linalg.norm(w))
    ut = self.solve_IQ(w, self.k)
    a = self.st.alpha
    ubar = a * ut + (1.0 - a) * self.u
    u_new = self.proj_C(ubar - self.v)
    v_new = self.v + ubar - u_new                               # planted: signs of the dual update
    self.u, self.v = u_new, v_new


def proj_C_tau_unclipped(self, x):
    n, m = self.n, self.m
    out = np.empty_like(x)
    out[:n] = x[:n]
    out[n:n + m] = cones.proj_Kdual(x[n:n + m], self.cone)
    out[-1] = x[-1]                                             # planted: tau not kept >= 0
    return out


# ---- cone projections -------------------------------------------------------

_proj_soc, _proj_exp = cones.proj_soc, cones.proj_exp


def exp_curve_mu_sign(rho, r0, s0, t0):
    den = rho * rho - rho + 1.0
    y = ((rho - 1.0) * r0 + s0) / den
    mu = (r0 - rho * s0) / den
    with np.errstate(over="ignore", invalid="ignore"):
        return y * np.exp(rho) + mu * np.exp(-rho) - t0, y       # planted: + mu e^-rho


def soc_half_dropped(v):
    p = _proj_soc(v)
    t, x = v[0], v[1:]
    if abs(t) < np.linalg.norm(x):
        return 2.0 * p                                          # planted: the 1/2 of (t + ||x||)/2 dropped
    return p


def psd_abs_eigenvalues(v, k):
    lam, Q = np.linalg.eigh(cones.smat(v, k))
    return cones.svec((Q * np.abs(lam)) @ Q.T)                  # planted: |lambda| instead of max(lambda, 0)


def exp_dual_moreau_sign(v):
    return np.asarray(v, dtype=float) - _proj_exp(-np.asarray(v, dtype=float))   # planted: w - Pi(-w)


# ---- termination (Sec. 3.5, Sec. 5) -----------------------------------------------

_residuals = admm.HSDSolver.residuals


def residuals_pri_without_sigma(self):
    out = _residuals(self)
    n, m = self.n, self.m
    tau = self.u[-1]
    if tau > 0:
        r = self.A @ self.u[:n] + self.v[n:n + m] - tau * self.b
        out["pri"] = np.linalg.norm(r / self.D) / tau              # planted: 1/sigma dropped
    return out


def residuals_dual_without_rho(self):
    out = _residuals(self)
    n, m = self.n, self.m
    tau = self.u[-1]
    if tau > 0:
        r = self.At @ self.u[n:n + m] + tau * self.c
        out["dual"] = np.linalg.norm(r / self.E) / tau             # planted: 1/rho dropped
    return out


# ---- equilibration (Sec. 5) ---------------------------------------------------

_equilibrate = admm.equilibrate


def equilibrate_b_unscaled(*args, **kw):
    Ah, bh, ch, D, E, sigma, rho = _equilibrate(*args, **kw)
    return Ah, bh / D, ch, D, E, sigma, rho                     # planted: b^ misses the row scaling D


# ---- power cone (Sec. 6.1) -------------------------------------------------------

def pow_branch_weights_swapped(v, a):
    x0, y0, z0 = (float(t) for t in v)
    return _proj_pow(np.array([x0, y0, z0]), 1.0 - a)              # planted: a and 1 - a swapped


_proj_pow = cones.proj_pow


def pow_sign_of_z(v, a):
    p = _proj_pow(v, a).copy()
    if not cones.in_pow(v, a):
        p[2] = -p[2]                                               # planted: z takes the wrong sign
    return p


# ---- warm-start network ---------------------------------------------------------

_gelu_grad = omlp.gelu_grad


def gelu_grad_drops_density_term(z):
    return 0.5 * (1.0 + omlp.erf(z / omlp.SQRT2))                # planted: z phi(z) dropped


_adam = omlp.adam


def adam_without_bias_correction(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    # planted: the moments used as they are (no division by 1 - beta^t)
    if not state:
        state["t"] = 0
        state["m"] = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
        state["v"] = [[np.zeros_like(W), np.zeros_like(b)] for W, b in params]
    state["t"] += 1
    new = []
    for li, (layer, grad) in enumerate(zip(params, grads)):
        pair = []
        for k in range(2):
            g = grad[k]
            m = beta1 * state["m"][li][k] + (1.0 - beta1) * g
            v = beta2 * state["v"][li][k] + (1.0 - beta2) * g * g
            state["m"][li][k], state["v"][li][k] = m, v
            pair.append(layer[k] - lr * m / (np.sqrt(v) + eps))
        new.append(tuple(pair))
    return new


MUTANTS = [
    ("SMW correction sign", admm.HSDSolver, "solve_IQ", iq_gamma_sign, pins_admm.test_smw_equals_dense_solve),
    ("tau drops b^T u_y", admm.HSDSolver, "solve_IQ", iq_tau_drops_b, pins_admm.test_smw_equals_dense_solve),
    ("z_y sign", admm.HSDSolver, "_solve_M", solve_M_zy_sign, pins_admm.test_smw_equals_dense_solve),
    ("relaxation weights swapped", admm.HSDSolver, "step", step_relax_swapped,
     pins_admm.test_naive_equals_simplified),
    ("dual update signs", admm.HSDSolver, "step", step_dual_sign, pins_admm.test_naive_equals_simplified),
    ("tau not clipped", admm.HSDSolver, "proj_C", proj_C_tau_unclipped, pins_admm.test_infeasible_certificate),
    ("SOC factor 1/2 dropped", cones, "proj_soc", soc_half_dropped, pins_cones.test_soc_kkt_random),
    ("PSD keeps |lambda|", cones, "proj_psd", psd_abs_eigenvalues, pins_cones.test_psd_kkt_random),
    ("exp dual Moreau sign", cones, "proj_exp_dual", exp_dual_moreau_sign, pins_cones.test_exp_dual_kkt_random),
    ("b^ without D", admm, "equilibrate", equilibrate_b_unscaled, pins_admm.test_scaling_preserves_solution),
    ("primal residual without 1/sigma", admm.HSDSolver, "residuals", residuals_pri_without_sigma,
     lambda: pins_admm.test_returned_point_passes_tests_on_original_data("mixed")),
    ("dual residual without 1/rho", admm.HSDSolver, "residuals", residuals_dual_without_rho,
     lambda: pins_admm.test_returned_point_passes_tests_on_original_data("lp")),
    ("exp curve: sign of mu e^-rho", cones, "_exp_h", exp_curve_mu_sign, pins_cones.test_exp_kkt_random),
    ("power cone: weights a, 1 - a swapped", cones, "proj_pow", pow_branch_weights_swapped,
     lambda: pins_cones.test_pow_kkt_random(0.2)),
    ("power cone: sign of z", cones, "proj_pow", pow_sign_of_z, lambda: pins_cones.test_pow_kkt_random(0.71)),
    ("CG residual update sign", admm.HSDSolver, "_pcg", pcg_residual_sign,
     pins_admm.test_direct_and_tight_indirect_agree),
    ("GELU derivative without z phi(z)", omlp, "gelu_grad", gelu_grad_drops_density_term,
     pins_mlp.test_backward_matches_finite_differences),
    ("Adam without bias correction", omlp, "adam", adam_without_bias_correction, pins_mlp.test_adam_scalar_quadratic),
]


@pytest.mark.parametrize("name,target,attr,mutant,pin", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pin_catches_mutant(monkeypatch, name, target, attr, mutant, pin):
    pin()                                   # the pin holds on the oracle as written
    monkeypatch.setattr(target, attr, mutant)
    with pytest.raises(AssertionError):
        pin()
