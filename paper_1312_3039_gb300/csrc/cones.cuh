// Device cone projections, FP64 (and FP32 exponential- and power-cone
// projections for the mixed-precision iteration).  The iteration projects the y-part of u onto
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

__host__ __device__ __forceinline__ bool exp_member(double x, double y, double z) {
    if (y > 0.0) {
        const double q = x / y;
        return q < 700.0 && y * exp(q) <= z;
    }
    return y == 0.0 && x <= 0.0 && z >= 0.0;
}

__host__ __device__ __forceinline__ bool exp_dual_member(double u, double v, double w) {
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
    __host__ __device__ __forceinline__ void eval(double rho, double &h, double &dh) const {
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

// The same curve in FP32 for the first, coarse root search.
struct ExpCurveF {
    float r0, s0, t0;
    __host__ __device__ __forceinline__ void eval(float rho, float &h, float &dh) const {
        const float den = rho * rho - rho + 1.0f;
        const float ep = expf(rho), em = expf(-rho);
        const float a = (rho - 1.0f) * r0 + s0;
        const float c = r0 - rho * s0;
        const float num = a * ep - c * em;
        const float dnum = ep * (rho * r0 + s0) + em * (r0 - rho * s0 + s0);
        h = num / den - t0;
        dh = (dnum * den - num * (2.0f * rho - 1.0f)) / (den * den);
        // inside the bracket y > 0 and mu > 0, so an overflowed h has the sign of rho
        if (!isfinite(h)) h = rho > 0.0f ? INFINITY : -INFINITY;
    }
};

// Euclidean projection of (r0, s0, t0) onto Kexp.
__host__ __device__ inline void proj_exp(double r0, double s0, double t0, double &px, double &py, double &pz) {
    if (exp_member(r0, s0, t0)) { px = r0; py = s0; pz = t0; return; }
    if (exp_dual_member(-r0, -s0, -t0)) { px = 0.0; py = 0.0; pz = 0.0; return; }
    if (r0 <= 0.0 && s0 <= 0.0) { px = r0; py = 0.0; pz = fmax(t0, 0.0); return; }
    // the projection is positively homogeneous: solve for v / ||v||_inf
    const double nrm = fmax(fabs(r0), fmax(fabs(s0), fabs(t0)));
    const double r = r0 / nrm, s = s0 / nrm, t = t0 / nrm;
    // bracket: h < 0 where y -> 0 (rho = 1 - s/r when r > 0, else -inf),
    //          h > 0 where mu -> 0 (rho = r/s when s > 0, else +inf)
    const bool lo_open = !(r > 0.0), hi_open = !(s > 0.0);
    double lo = lo_open ? 0.0 : 1.0 - s / r;
    double hi = hi_open ? 0.0 : r / s;
    // 1. coarse search in FP32: close the open end by doubling steps, bisect
    //    while the bracket is wide (h grows like e^|rho|), then Newton
    const ExpCurveF ff{(float)r, (float)s, (float)t};
    float h, dh;
    if (lo_open) {
        float step = 1.0f;
        for (int it = 0; it < 60; ++it) {
            ff.eval((float)hi - step, h, dh);
            if (h < 0.0f) break;
            step *= 2.0f;
        }
        lo = (double)((float)hi - step);
    }
    if (hi_open) {
        float step = 1.0f;
        for (int it = 0; it < 60; ++it) {
            ff.eval((float)lo + step, h, dh);
            if (h > 0.0f) break;
            step *= 2.0f;
        }
        hi = (double)((float)lo + step);
    }
    float flo = (float)lo, fhi = (float)hi, frho = 0.5f * (flo + fhi);
    for (int it = 0; it < 120; ++it) {
        ff.eval(frho, h, dh);
        if (h == 0.0f) break;
        if (h < 0.0f) flo = frho; else fhi = frho;
        const float tol = 2e-7f * fmaxf(1.0f, fabsf(frho));
        if (fhi - flo <= 1.0f && isfinite(dh) && dh > 0.0f) {
            const float step = h / dh;
            if (fabsf(step) <= tol) { frho -= step; break; }      // converged
            const float c = frho - step;
            if (c > flo && c < fhi) { frho = c; continue; }
        }
        frho = 0.5f * (flo + fhi);
        if (fhi - flo <= tol) break;
    }
    // 2. FP64 Newton from the FP32 root, kept inside the (FP64) sign bracket
    const ExpCurve f{r, s, t};
    double rho = (double)frho, hd, dhd;
    if (!(rho > lo && rho < hi)) rho = 0.5 * (lo + hi);
    for (int it = 0; it < 80; ++it) {
        f.eval(rho, hd, dhd);
        if (hd == 0.0) break;
        if (hd < 0.0) lo = rho; else hi = rho;
        const double tol = 1e-15 * fmax(1.0, fabs(rho));
        if (isfinite(hd) && isfinite(dhd) && dhd > 0.0) {
            const double step = hd / dhd;
            if (fabs(step) <= tol) { rho -= step; break; }        // converged
            const double c = rho - step;
            if (c > lo && c < hi) { rho = c; continue; }
        }
        rho = 0.5 * (lo + hi);
        if (hi - lo <= tol) break;
    }
    // return whichever of the two equal expressions rounds better: the
    // primal ray y (rho, 1, e^rho) or v + mu (-1, rho - 1, e^-rho)
    const double den = rho * rho - rho + 1.0;
    const double y = ((rho - 1.0) * r + s) / den;
    const double mu = (r - rho * s) / den;
    const double ep = exp(rho), em = exp(-rho);
    const double err_p = (fabs(rho - 1.0) * fabs(r) + fabs(s)) / den * sqrt(rho * rho + 1.0 + ep * ep);
    const double err_d = (fabs(r) + fabs(rho) * fabs(s)) / den * sqrt(1.0 + (rho - 1.0) * (rho - 1.0) + em * em) +
                         sqrt(r * r + s * s + t * t);
    if (err_p <= err_d) {
        px = nrm * (y * rho); py = nrm * y; pz = nrm * (y * ep);
    } else {
        px = nrm * (r - mu); py = nrm * (s + mu * (rho - 1.0)); pz = nrm * (t + mu * em);
    }
}

// Pi_{Kexp*}(w) = w + Pi_{Kexp}(-w)
__host__ __device__ inline void proj_exp_dual(double u, double v, double w, double &pu, double &pv, double &pw) {
    double a, b, c;
    proj_exp(-u, -v, -w, a, b, c);
    pu = u + a; pv = v + b; pw = w + c;
}

// ---------------------------------------------------------------------------
// FP32 version for the mixed-precision iteration (its iterates are FP32):
// the same special cases, bracket, bisection and Newton steps, all in FP32
// (GB300's FP64 rate is a small fraction of its FP32 rate), converged to
// |step| <= 2e-7 max(1, |rho|); the better-conditioned of the two
// expressions of the projection is returned.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ bool exp_member_f(float x, float y, float z) {
    if (y > 0.0f) {
        const float q = x / y;
        return q < 80.0f && y * expf(q) <= z;
    }
    return y == 0.0f && x <= 0.0f && z >= 0.0f;
}

__host__ __device__ __forceinline__ bool exp_dual_member_f(float u, float v, float w) {
    if (u < 0.0f) {
        const float q = v / u;
        return q < 80.0f && -u * expf(q) <= 2.718281828459045f * w;
    }
    return u == 0.0f && v >= 0.0f && w >= 0.0f;
}

__host__ __device__ inline void proj_exp_f(float r0, float s0, float t0, float &px, float &py, float &pz) {
    if (exp_member_f(r0, s0, t0)) { px = r0; py = s0; pz = t0; return; }
    if (exp_dual_member_f(-r0, -s0, -t0)) { px = 0.0f; py = 0.0f; pz = 0.0f; return; }
    if (r0 <= 0.0f && s0 <= 0.0f) { px = r0; py = 0.0f; pz = fmaxf(t0, 0.0f); return; }
    const float nrm = fmaxf(fabsf(r0), fmaxf(fabsf(s0), fabsf(t0)));
    const float r = r0 / nrm, s = s0 / nrm, t = t0 / nrm;
    const bool lo_open = !(r > 0.0f), hi_open = !(s > 0.0f);
    float lo = lo_open ? 0.0f : 1.0f - s / r;
    float hi = hi_open ? 0.0f : r / s;
    const ExpCurveF ff{r, s, t};
    float h, dh;
    if (lo_open) {
        float step = 1.0f;
        for (int it = 0; it < 60; ++it) {
            ff.eval(hi - step, h, dh);
            if (h < 0.0f) break;
            step *= 2.0f;
        }
        lo = hi - step;
    }
    if (hi_open) {
        float step = 1.0f;
        for (int it = 0; it < 60; ++it) {
            ff.eval(lo + step, h, dh);
            if (h > 0.0f) break;
            step *= 2.0f;
        }
        hi = lo + step;
    }
    float rho = 0.5f * (lo + hi);
    for (int it = 0; it < 120; ++it) {
        ff.eval(rho, h, dh);
        if (h == 0.0f) break;
        if (h < 0.0f) lo = rho; else hi = rho;
        const float tol = 2e-7f * fmaxf(1.0f, fabsf(rho));
        if (hi - lo <= 1.0f && isfinite(dh) && dh > 0.0f) {
            const float step = h / dh;
            if (fabsf(step) <= tol) { rho -= step; break; }
            const float c = rho - step;
            if (c > lo && c < hi) { rho = c; continue; }
        }
        rho = 0.5f * (lo + hi);
        if (hi - lo <= tol) break;
    }
    const float den = rho * rho - rho + 1.0f;
    const float y = ((rho - 1.0f) * r + s) / den;
    const float mu = (r - rho * s) / den;
    const float ep = expf(rho), em = expf(-rho);
    const float err_p = (fabsf(rho - 1.0f) * fabsf(r) + fabsf(s)) / den * sqrtf(rho * rho + 1.0f + ep * ep);
    const float err_d = (fabsf(r) + fabsf(rho) * fabsf(s)) / den * sqrtf(1.0f + (rho - 1.0f) * (rho - 1.0f) + em * em) +
                        sqrtf(r * r + s * s + t * t);
    if (err_p <= err_d) {
        px = nrm * (y * rho); py = nrm * y; pz = nrm * (y * ep);
    } else {
        px = nrm * (r - mu); py = nrm * (s + mu * (rho - 1.0f)); pz = nrm * (t + mu * em);
    }
}

__host__ __device__ inline void proj_exp_dual_f(float u, float v, float w, float &pu, float &pv, float &pw) {
    float a, b, c;
    proj_exp_f(-u, -v, -w, a, b, c);
    pu = u + a; pv = v + b; pw = w + c;
}

// ---------------------------------------------------------------------------
// power cone (Sec. 6.1), a in (0, 1):
//   Kpow^a    = {(x, y, z): x^a y^(1-a) >= |z|, x >= 0, y >= 0}
//   (Kpow^a)* = {(u, v, w): (u/a)^a (v/(1-a))^(1-a) >= |w|, u >= 0, v >= 0}
// Outside K and the polar cone, and with z0 != 0, the projection of
// v = (x0, y0, z0) lies on the curved boundary with z of the sign of z0 and
// |z| = r, the root in (0, |z0|) of phi(r) = x(r)^a y(r)^(1-a) - r: the
// stationarity of the distance with the multiplier |z0| - r makes x(r), y(r)
// the positive roots of x^2 - x0 x - a r (|z0| - r) = 0 and
// y^2 - y0 y - (1 - a) r (|z0| - r) = 0.  phi >= 0 at 0 and < 0 at |z0|;
// the root is found by bisection in the iterate's precision T.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ float pw_sqrt(float x) { return sqrtf(x); }
__host__ __device__ __forceinline__ double pw_sqrt(double x) { return sqrt(x); }
__host__ __device__ __forceinline__ float pw_exp(float x) { return expf(x); }
__host__ __device__ __forceinline__ double pw_exp(double x) { return exp(x); }
__host__ __device__ __forceinline__ float pw_log(float x) { return logf(x); }
__host__ __device__ __forceinline__ double pw_log(double x) { return log(x); }

// x^a y^(1-a) for x, y >= 0 (0 when either is 0)
template <typename T>
__host__ __device__ __forceinline__ T pow_mean(T x, T y, T a) {
    if (!(x > T(0)) || !(y > T(0))) return T(0);
    return pw_exp(a * pw_log(x) + (T(1) - a) * pw_log(y));
}

// positive root t of t^2 - c0 t - k r (r0 - r) = 0, without cancellation for c0 < 0
template <typename T>
__host__ __device__ __forceinline__ T pow_branch(T c0, T k, T r, T r0) {
    const T q = k * r * (r0 - r);
    const T d = pw_sqrt(c0 * c0 + T(4) * q);
    if (c0 >= T(0)) return T(0.5) * (c0 + d);
    const T den = d - c0;
    return den > T(0) ? T(2) * q / den : T(0);
}

template <typename T>
__host__ __device__ inline void proj_pow(T x0, T y0, T z0, T a, T &px, T &py, T &pz) {
    const T az = fabs(z0);
    if (x0 >= T(0) && y0 >= T(0) && pow_mean(x0, y0, a) >= az) { px = x0; py = y0; pz = z0; return; }   // v in K
    if (x0 <= T(0) && y0 <= T(0) && pow_mean(-x0 / a, -y0 / (T(1) - a), a) >= az) {                   // -v in K*
        px = T(0); py = T(0); pz = T(0);
        return;
    }
    if (az == T(0)) { px = fmax(x0, T(0)); py = fmax(y0, T(0)); pz = T(0); return; }
    T lo = T(0), hi = az;
    for (int it = 0; it < 200; ++it) {
        const T mid = T(0.5) * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        const T phi = pow_mean(pow_branch(x0, a, mid, az), pow_branch(y0, T(1) - a, mid, az), a) - mid;
        if (phi > T(0)) lo = mid; else hi = mid;
    }
    const T r = T(0.5) * (lo + hi);
    px = pow_branch(x0, a, r, az);
    py = pow_branch(y0, T(1) - a, r, az);
    pz = z0 < T(0) ? -r : r;
}

// Moreau (Eq. "e-moreau"): Pi_{K*}(w) = w + Pi_K(-w)
template <typename T>
__host__ __device__ inline void proj_pow_dual(T u, T v, T w, T a, T &pu, T &pv, T &pw) {
    T p0, p1, p2;
    proj_pow(-u, -v, -w, a, p0, p1, p2);
    pu = u + p0; pv = v + p1; pw = w + p2;
}

}  // namespace scs
