// Device cone projections, FP64.  The iteration projects the y-part of u onto
// the dual cone K* (Eq. "e-hsdnice": C = R^n x K* x R+): the dual of the zero
// cone is R (identity), the nonnegative and second-order cones are
// self-dual, and the dual exponential cone is reached through Moreau
// (Eq. "e-moreau"): Pi_{K*}(w) = w + Pi_K(-w).
#pragma once

#include <math.h>

namespace scs {

// ---------------------------------------------------------------------------
// exponential cone (Sec. 6.1):
//   Kexp  = closure{(x, y, z): y > 0, y e^(x/y) <= z}
//   Kexp* = closure{(u, v, w): u < 0, -u e^(v/u) <= e w}
// ---------------------------------------------------------------------------

__device__ __forceinline__ bool exp_member(double x, double y, double z) {
    if (y > 0.0) {
        const double q = x / y;
        return q < 700.0 && y * exp(q) <= z;
    }
    return y == 0.0 && x <= 0.0 && z >= 0.0;
}

__device__ __forceinline__ bool exp_dual_member(double u, double v, double w) {
    if (u < 0.0) {
        const double q = v / u;
        return q < 700.0 && -u * exp(q) <= M_E * w;
    }
    return u == 0.0 && v >= 0.0 && w >= 0.0;
}

// On the curve p = y (rho, 1, e^rho) (boundary of Kexp) paired with
// d = mu (-1, rho - 1, e^-rho) (boundary of Kexp*, orthogonal to p), the
// first two entries of v = p - d fix y and mu for each rho:
//   y  = ((rho - 1) r0 + s0) / (rho^2 - rho + 1)
//   mu = (r0 - rho s0)       / (rho^2 - rho + 1)
// and the projection is the rho where y e^rho - mu e^-rho = t0.
struct ExpCurve {
    double r0, s0, t0;
    __device__ __forceinline__ void eval(double rho, double &h, double &dh) const {
        const double den = rho * rho - rho + 1.0;
        const double ep = exp(rho), em = exp(-rho);
        const double a = (rho - 1.0) * r0 + s0;        // y * den
        const double c = r0 - rho * s0;                // mu * den
        const double num = a * ep - c * em;
        const double dnum = ep * (rho * r0 + s0) + em * (r0 - rho * s0 + s0);
        h = num / den - t0;
        dh = (dnum * den - num * (2.0 * rho - 1.0)) / (den * den);
    }
};

// Euclidean projection of (r0, s0, t0) onto Kexp.
__device__ inline void proj_exp(double r0, double s0, double t0, double &px, double &py, double &pz) {
    if (exp_member(r0, s0, t0)) { px = r0; py = s0; pz = t0; return; }
    if (exp_dual_member(-r0, -s0, -t0)) { px = 0.0; py = 0.0; pz = 0.0; return; }
    if (r0 <= 0.0 && s0 <= 0.0) { px = r0; py = 0.0; pz = fmax(t0, 0.0); return; }
    const ExpCurve f{r0, s0, t0};
    // bracket: h < 0 where y -> 0 (rho = 1 - s0/r0 when r0 > 0, else -inf),
    //          h > 0 where mu -> 0 (rho = r0/s0 when s0 > 0, else +inf)
    double lo = 0.0, hi = 0.0, h, dh;
    const bool lo_open = !(r0 > 0.0), hi_open = !(s0 > 0.0);
    if (!lo_open) lo = 1.0 - s0 / r0;
    if (!hi_open) hi = r0 / s0;
    if (lo_open) {
        double step = 1.0;
        lo = hi - step;
        for (int it = 0; it < 80; ++it) {
            f.eval(lo, h, dh);
            if (h < 0.0) break;
            step *= 2.0;
            lo = hi - step;
        }
    }
    if (hi_open) {
        double step = 1.0;
        hi = lo + step;
        for (int it = 0; it < 80; ++it) {
            f.eval(hi, h, dh);
            if (h > 0.0) break;
            step *= 2.0;
            hi = lo + step;
        }
    }
    // safeguarded Newton: keep the sign bracket, bisect when a Newton step
    // leaves it
    double rho = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        f.eval(rho, h, dh);
        if (h == 0.0) break;
        if (h < 0.0) lo = rho; else hi = rho;
        double nr = rho - h / dh;
        if (!(nr > lo && nr < hi)) nr = 0.5 * (lo + hi);
        const double tol = 1e-15 * fmax(1.0, fabs(nr));
        if (fabs(nr - rho) <= tol || hi - lo <= tol) { rho = nr; break; }
        rho = nr;
    }
    // return whichever of the two equal expressions rounds better: the
    // primal ray y (rho, 1, e^rho) or v + mu (-1, rho - 1, e^-rho)
    const double den = rho * rho - rho + 1.0;
    const double y = ((rho - 1.0) * r0 + s0) / den;
    const double mu = (r0 - rho * s0) / den;
    const double ep = exp(rho), em = exp(-rho);
    const double err_p = (fabs(rho - 1.0) * fabs(r0) + fabs(s0)) / den * sqrt(rho * rho + 1.0 + ep * ep);
    const double err_d = (fabs(r0) + fabs(rho) * fabs(s0)) / den *
                             sqrt(1.0 + (rho - 1.0) * (rho - 1.0) + em * em) +
                         sqrt(r0 * r0 + s0 * s0 + t0 * t0);
    if (err_p <= err_d) {
        px = y * rho; py = y; pz = y * ep;
    } else {
        px = r0 - mu; py = s0 + mu * (rho - 1.0); pz = t0 + mu * em;
    }
}

// Pi_{Kexp*}(w) = w + Pi_{Kexp}(-w)
__device__ inline void proj_exp_dual(double u, double v, double w, double &pu, double &pv, double &pw) {
    double a, b, c;
    proj_exp(-u, -v, -w, a, b, c);
    pu = u + a; pv = v + b; pw = w + c;
}

}  // namespace scs
