// Family solver: many programs that share A (and the cone) and differ in b
// and c -- the repeated-solve setting of Sec. 4.2, where only b and c
// change -- solved together with a dense direct subspace step.
//
// Sec. 4.1's linear system has the same matrix M = [I A^T; -A I] for every
// member (the equilibration D, E depends on A only; sigma and rho, which
// depend on b and c, are per member).  So (I + A^T A)^-1 is formed once (FP64
// Gauss-Jordan on the device, kept in T), and one iteration of every member
// at once is three dense products over the member columns:
//     t  = r_x - A^T r_y            (n x m) (m x B)
//     z_x = (I + A^T A)^-1 t        (n x n) (n x B)
//     z_y = r_y + A z_x             (m x n) (n x B)
// (the CUDA-core GEMM of dense.cuh, in T; A^ is kept in both orientations
// so that every product is a plain column-major one), then per member the
// SMW correction, relaxation,
// projection and dual update of Eq. "e-SCS" (one CTA per member).  The
// Sec. 3.5 tests run every check_interval iterations on the active members
// (two more products); a member that passes is recorded (status, iterations,
// solution and its scaled HSD state).  Once a few percent of the active
// columns have finished, finished columns are swapped behind the active ones
// and the products run over the active prefix only; the swaps are undone in
// reverse order when the solve ends.
//
// Layout: member vectors are the columns of column-major matrices (n x B,
// m x B); A^ is dense m x n.  Cones: zero, nonnegative, SOC.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/scs_gpu.h"
#include "common.cuh"
#include "dense.cuh"
#include "engine_base.h"
#include "kernels.cuh"
#include "tc_split.h"

namespace scs {
namespace family {

constexpr int kFamThreads = 256;


template <typename T>
struct Dev {
    int n, m, B, z, l, nq;
    const int32_t *soc_off, *soc_len;   // SOC blocks (rows within y)
    const double *D, *E;                // shared equilibration
    // per member (column b)
    T *ch, *bh;                         // c^ (n x B), b^ (m x B)
    double *c64, *b64;                  // the same in FP64 (tests)
    T *px, *py;                         // p = M^-1 h
    double *hp1, *sigma, *rho, *nb, *nc;
    // state
    T *ux, *uy, *vs;                    // u_x (n x B), u_y, v_s (m x B)
    double *tau, *kappa;                // per member
    // work
    T *rx, *ry;                         // r_x -> t, r_y -> z_y
    T *zx;
    T *ax, *aty;                        // A^ u_x, A^T u_y (tests)
    // results
    int32_t *status, *iters;            // per member (indexed by member id)
    int32_t *done;                      // per column
    int32_t *perm;                      // member id held by each column
    double *x, *y, *s;                  // caller's units (n x B, m x B, m x B)
    float *snap;                        // (u_x, u_y, v_s, u_tau) / u_tau at the first passing test, (n + 2m + 1) x B
    double *pobj, *dobj, *res_pri, *res_dual, *gap;   // per member
    int *ndone;
    double alpha, eps_pri, eps_dual, eps_gap, eps_infeas, eps_unbdd;
};

template <typename T>
__device__ __forceinline__ double cta_sum(double v, double *red) {
    // kFamThreads threads; valid in every thread
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int k = 0; k < kFamThreads / 32; ++k) t += red[k];
    return t;
}

// r_x = u_x - w_tau c^,  r_y = u_y + v_s - w_tau b^   (w_tau = tau + kappa)
template <typename T>
__global__ void __launch_bounds__(kFamThreads) rhs_kernel(Dev<T> F) {
    const int64_t nx = (int64_t)F.n * F.B, ny = (int64_t)F.m * F.B;
    for (int64_t e = (int64_t)blockIdx.x * kFamThreads + threadIdx.x; e < nx + ny;
         e += (int64_t)gridDim.x * kFamThreads) {
        if (e < nx) {
            const int b = static_cast<int>(e / F.n);
            const T wt = static_cast<T>(F.tau[b] + F.kappa[b]);
            F.rx[e] = F.ux[e] - wt * F.ch[e];
        } else {
            const int64_t f = e - nx;
            const int b = static_cast<int>(f / F.m);
            const T wt = static_cast<T>(F.tau[b] + F.kappa[b]);
            F.ry[f] = F.uy[f] + F.vs[f] - wt * F.bh[f];
        }
    }
}

// one CTA per member: gamma, relaxation, projection onto R^n x K* x R+,
// dual update (Eq. "e-SCS"; SMW correction of Sec. 4.1)
template <typename T>
__global__ void __launch_bounds__(kFamThreads) update_kernel(Dev<T> F) {
    __shared__ double red[kFamThreads / 32];
    const int b = blockIdx.x;
    const int n = F.n, m = F.m;
    const size_t cx = (size_t)b * n, cy = (size_t)b * m;
    const T *zx = F.zx + cx, *zy = F.ry + cy, *ch = F.ch + cx, *bh = F.bh + cy;
    double g = 0.0;
    for (int j = threadIdx.x; j < n; j += kFamThreads) g += static_cast<double>(ch[j] * zx[j]);
    for (int i = threadIdx.x; i < m; i += kFamThreads) g += static_cast<double>(bh[i] * zy[i]);
    g = cta_sum<T>(g, red);
    const double gamma = g / F.hp1[b];
    const T gm = static_cast<T>(gamma), al = static_cast<T>(F.alpha);
    T *ux = F.ux + cx, *uy = F.uy + cy, *vs = F.vs + cy;
    const T *px = F.px + cx, *py = F.py + cy;
    for (int j = threadIdx.x; j < n; j += kFamThreads) ux[j] = al * (zx[j] - px[j] * gm) + (T(1) - al) * ux[j];
    const int nlin = F.z + F.l;
    for (int i = threadIdx.x; i < nlin; i += kFamThreads) {
        const T ub = al * (zy[i] - py[i] * gm) + (T(1) - al) * uy[i];
        const T t = ub - vs[i];
        const T up = i < F.z ? t : (t > T(0) ? t : T(0));
        uy[i] = up;
        vs[i] = up - t;
    }
    for (int q = 0; q < F.nq; ++q) {
        const int off = F.soc_off[q], len = F.soc_len[q];
        double xx = 0.0;
        for (int e = 1 + threadIdx.x; e < len; e += kFamThreads) {
            const int i = off + e;
            const T t = al * (zy[i] - py[i] * gm) + (T(1) - al) * uy[i] - vs[i];
            xx += static_cast<double>(t * t);
        }
        xx = cta_sum<T>(xx, red);
        const int i0 = off;
        const T t0 = al * (zy[i0] - py[i0] * gm) + (T(1) - al) * uy[i0] - vs[i0];
        const T nx = static_cast<T>(sqrt(xx));
        T head, tail;
        if (nx <= t0) { head = t0; tail = T(1); }
        else if (nx <= -t0) { head = T(0); tail = T(0); }
        else { head = T(0.5) * (t0 + nx); tail = head / nx; }
        __syncthreads();   // every thread has read row i0 before it changes
        for (int e = threadIdx.x; e < len; e += kFamThreads) {
            const int i = off + e;
            const T t = al * (zy[i] - py[i] * gm) + (T(1) - al) * uy[i] - vs[i];
            const T up = e == 0 ? head : tail * t;
            uy[i] = up;
            vs[i] = up - t;
        }
    }
    if (threadIdx.x == 0) {
        const double wt = F.tau[b] + F.kappa[b];
        const double ub = F.alpha * (wt + gamma) + (1.0 - F.alpha) * F.tau[b];
        const double t = ub - F.kappa[b];
        const double up = fmax(t, 0.0);
        F.tau[b] = up;
        F.kappa[b] = up - t;
    }
}

// Sec. 3.5 tests of every member (FP64 sums; ax = A^ u_x, aty = A^T u_y in T);
// a member that passes for the first time records its results
template <typename T>
__global__ void __launch_bounds__(kFamThreads) check_kernel(Dev<T> F, int k, int final_pass) {
    __shared__ double red[kFamThreads / 32];
    const int b = blockIdx.x;
    if (F.done[b]) return;
    const int n = F.n, m = F.m;
    const size_t cx = (size_t)b * n, cy = (size_t)b * m;
    const double tau = F.tau[b], kappa = F.kappa[b];
    double s[6] = {0, 0, 0, 0, 0, 0};
    for (int i = threadIdx.x; i < m; i += kFamThreads) {
        const double a = static_cast<double>(F.ax[cy + i]) + static_cast<double>(F.vs[cy + i]);
        const double bb = F.b64[cy + i], d = F.D[i];
        const double pr = (a - tau * bb) / d, ub = a / d;
        s[0] += pr * pr;
        s[1] += ub * ub;
        s[2] += bb * static_cast<double>(F.uy[cy + i]);
    }
    for (int j = threadIdx.x; j < n; j += kFamThreads) {
        const double a = static_cast<double>(F.aty[cx + j]);
        const double cc = F.c64[cx + j], e = F.E[j];
        const double du = (a + tau * cc) / e, inf = a / e;
        s[3] += du * du;
        s[4] += inf * inf;
        s[5] += cc * static_cast<double>(F.ux[cx + j]);
    }
#pragma unroll
    for (int e = 0; e < 6; ++e) s[e] = cta_sum<T>(s[e], red);
    const double sg = F.sigma[b], rh = F.rho[b], nbv = F.nb[b], ncv = F.nc[b];
    int st = 0;
    double pri = INFINITY, dual = INFINITY, gap = INFINITY, cxv = NAN, by = NAN;
    if (tau > 0.0) {
        pri = sqrt(s[0]) / (tau * sg);
        dual = sqrt(s[3]) / (tau * rh);
        cxv = s[5] / (tau * rh * sg);
        by = s[2] / (tau * rh * sg);
        gap = fabs(cxv + by);
        if (pri <= F.eps_pri * (1.0 + nbv) && dual <= F.eps_dual * (1.0 + ncv) &&
            gap <= F.eps_gap * (1.0 + fabs(cxv) + fabs(by)))
            st = 1;
    }
    if (!st && nbv > 0.0 && s[2] < 0.0 && sqrt(s[4]) <= (-s[2] / (sg * nbv)) * F.eps_infeas) st = -1;
    if (!st && ncv > 0.0 && s[5] < 0.0 && sqrt(s[1]) <= (-s[5] / (rh * ncv)) * F.eps_unbdd) st = -2;
    if (!isfinite(tau) || !isfinite(kappa) || !isfinite(s[0]) || !isfinite(s[3])) st = -13;
    if (!st && final_pass) {
        if (tau > 0 && tau >= kappa) st = SCS_SOLVED_INACCURATE;
        else if (s[2] < 0 && s[2] <= s[5]) st = SCS_INFEASIBLE_INACCURATE;
        else if (s[5] < 0) st = SCS_UNBOUNDED_INACCURATE;
        else st = tau > 0 ? SCS_SOLVED_INACCURATE : SCS_INFEASIBLE_INACCURATE;
    }
    if (!st) return;
    // record (at the member's own index): outputs in the caller's units,
    // the scaled state, the tests
    const int mid = F.perm[b];
    const size_t ox = (size_t)mid * n, oy = (size_t)mid * m;
    for (int e = threadIdx.x; e < n + 2 * m; e += kFamThreads) {
        double val;
        if (st == 1 || st == 2) {
            if (e < n) val = F.E[e] * static_cast<double>(F.ux[cx + e]) / (tau * sg);
            else if (e < n + m) val = F.D[e - n] * static_cast<double>(F.uy[cy + e - n]) / (tau * rh);
            else val = static_cast<double>(F.vs[cy + e - n - m]) / (F.D[e - n - m] * tau * sg);
        } else if (st == -1 || st == -3) {
            val = (e >= n && e < n + m) ? F.D[e - n] * static_cast<double>(F.uy[cy + e - n]) * (sg / (-s[2])) : NAN;
        } else if (st == -2 || st == -4) {
            const double f = rh / (-s[5]);
            if (e < n) val = F.E[e] * static_cast<double>(F.ux[cx + e]) * f;
            else if (e < n + m) val = NAN;
            else val = -static_cast<double>(F.ax[cy + e - n - m]) * f / F.D[e - n - m];
        } else {
            val = NAN;
        }
        if (e < n) F.x[ox + e] = val;
        else if (e < n + m) F.y[oy + e - n] = val;
        else F.s[oy + e - n - m] = val;
    }
    // the state on the ray through it with u_tau = 1 (the HSD iteration is
    // positively homogeneous, so only the direction carries the solution)
    const size_t so = (size_t)mid * (n + 2 * m + 1);
    const double inv = tau > 0.0 ? 1.0 / tau : 1.0;
    for (int e = threadIdx.x; e < n + 2 * m + 1; e += kFamThreads) {
        double val;
        if (e < n) val = static_cast<double>(F.ux[cx + e]);
        else if (e < n + m) val = static_cast<double>(F.uy[cy + e - n]);
        else if (e < n + 2 * m) val = static_cast<double>(F.vs[cy + e - n - m]);
        else val = tau;
        F.snap[so + e] = static_cast<float>(val * inv);
    }
    if (threadIdx.x == 0) {
        F.status[mid] = st;
        F.iters[mid] = k;
        F.done[b] = 1;
        F.res_pri[mid] = pri;
        F.res_dual[mid] = dual;
        F.gap[mid] = gap;
        if (st == 1 || st == 2) {
            F.pobj[mid] = cxv;
            F.dobj[mid] = -by;
        } else if (st == -1 || st == -3) {
            F.pobj[mid] = NAN;
            F.dobj[mid] = 1.0;
        } else if (st == -2 || st == -4) {
            F.pobj[mid] = -1.0;
            F.dobj[mid] = NAN;
        } else {
            F.pobj[mid] = F.dobj[mid] = NAN;
        }
        atomicAdd(F.ndone, 1);
    }
}

// swap columns pairs[2p], pairs[2p + 1] of every per-member array (member
// data, state, the column's flags and member id); one CTA per pair
template <typename T>
__global__ void __launch_bounds__(kFamThreads) swap_kernel(Dev<T> F, const int32_t *__restrict__ pairs) {
    const int c1 = pairs[2 * blockIdx.x], c2 = pairs[2 * blockIdx.x + 1];
    const int n = F.n, m = F.m;
    auto sw = [](auto *a, size_t i, size_t j) {
        const auto t = a[i];
        a[i] = a[j];
        a[j] = t;
    };
    for (int j = threadIdx.x; j < n; j += kFamThreads) {
        const size_t a = (size_t)c1 * n + j, b = (size_t)c2 * n + j;
        sw(F.ch, a, b);
        sw(F.c64, a, b);
        sw(F.px, a, b);
        sw(F.ux, a, b);
    }
    for (int i = threadIdx.x; i < m; i += kFamThreads) {
        const size_t a = (size_t)c1 * m + i, b = (size_t)c2 * m + i;
        sw(F.bh, a, b);
        sw(F.b64, a, b);
        sw(F.py, a, b);
        sw(F.uy, a, b);
        sw(F.vs, a, b);
    }
    if (threadIdx.x == 0) {
        sw(F.hp1, c1, c2);
        sw(F.sigma, c1, c2);
        sw(F.rho, c1, c2);
        sw(F.nb, c1, c2);
        sw(F.nc, c1, c2);
        sw(F.tau, c1, c2);
        sw(F.kappa, c1, c2);
        sw(F.done, c1, c2);
        sw(F.perm, c1, c2);
    }
}

// per member: sigma, rho, b^, c^ (Sec. 5 with the shared D, E)
template <typename T>
__global__ void __launch_bounds__(kFamThreads) member_scale_kernel(Dev<T> F, const double *__restrict__ b,
                                                                    const double *__restrict__ c, double mean_row,
                                                                    int normalize) {
    __shared__ double red[kFamThreads / 32];
    const int k = blockIdx.x;
    const int n = F.n, m = F.m;
    const size_t cx = (size_t)k * n, cy = (size_t)k * m;
    double s[4] = {0, 0, 0, 0};
    for (int i = threadIdx.x; i < m; i += kFamThreads) {
        const double t = F.D[i] * b[cy + i];
        s[0] += t * t;
        s[2] += b[cy + i] * b[cy + i];
    }
    for (int j = threadIdx.x; j < n; j += kFamThreads) {
        const double t = F.E[j] * c[cx + j];
        s[1] += t * t;
        s[3] += c[cx + j] * c[cx + j];
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) s[e] = cta_sum<T>(s[e], red);
    const double sg = normalize ? 1.0 / fmax(sqrt(s[0]), 1e-4) : 1.0;
    const double rh = normalize ? mean_row / fmax(sqrt(s[1]), 1e-4) : 1.0;
    for (int i = threadIdx.x; i < m; i += kFamThreads) {
        const double t = sg * F.D[i] * b[cy + i];
        F.b64[cy + i] = t;
        F.bh[cy + i] = static_cast<T>(t);
    }
    for (int j = threadIdx.x; j < n; j += kFamThreads) {
        const double t = rh * F.E[j] * c[cx + j];
        F.c64[cx + j] = t;
        F.ch[cx + j] = static_cast<T>(t);
    }
    if (threadIdx.x == 0) {
        F.sigma[k] = sg;
        F.rho[k] = rh;
        F.nb[k] = sqrt(s[2]);
        F.nc[k] = sqrt(s[3]);
    }
}

// hp1 = 1 + c^.p_x + b^.p_y per member
template <typename T>
__global__ void __launch_bounds__(kFamThreads) hp1_kernel(Dev<T> F) {
    __shared__ double red[kFamThreads / 32];
    const int k = blockIdx.x;
    const size_t cx = (size_t)k * F.n, cy = (size_t)k * F.m;
    double s = 0.0;
    for (int j = threadIdx.x; j < F.n; j += kFamThreads) s += F.c64[cx + j] * static_cast<double>(F.px[cx + j]);
    for (int i = threadIdx.x; i < F.m; i += kFamThreads) s += F.b64[cy + i] * static_cast<double>(F.py[cy + i]);
    s = cta_sum<T>(s, red);
    if (threadIdx.x == 0) F.hp1[k] = 1.0 + s;
}

// dense A^ (column-major m x n) and A^T (column-major n x m) from CSR scaled values
static __global__ void densify_kernel(const int32_t *__restrict__ rp, const int32_t *__restrict__ col,
                                      const double *__restrict__ val, int m, int n, double *__restrict__ A64,
                                      double *__restrict__ At64) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        for (int k = rp[i]; k < rp[i + 1]; ++k) {
            A64[(size_t)col[k] * m + i] = val[k];
            At64[(size_t)i * n + col[k]] = val[k];
        }
}

template <typename T>
static __global__ void cast_kernel(const double *__restrict__ a, T *__restrict__ b, int64_t len) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = static_cast<T>(a[e]);
}

// cold start u = (0, 0, 1), v = (0, 0, 1)
template <typename T>
__global__ void cold_kernel(Dev<T> F) {
    const int64_t nx = (int64_t)F.n * F.B, ny = (int64_t)F.m * F.B;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nx + ny + F.B;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nx) F.ux[e] = T(0);
        else if (e < nx + ny) {
            F.uy[e - nx] = T(0);
            F.vs[e - nx] = T(0);
        } else {
            const int b = static_cast<int>(e - nx - ny);
            F.tau[b] = 1.0;
            F.kappa[b] = 1.0;
            F.done[b] = 0;
            F.status[b] = 0;
            F.iters[b] = 0;
        }
    }
}

// warm start u = (x^, y^, 1), v = (0, s^, 0) from scaled device arrays
template <typename T>
__global__ void warm_kernel(Dev<T> F, const double *__restrict__ xh, const double *__restrict__ yh,
                            const double *__restrict__ sh) {
    const int64_t nx = (int64_t)F.n * F.B, ny = (int64_t)F.m * F.B;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nx + ny + F.B;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nx) F.ux[e] = xh ? static_cast<T>(xh[e]) : T(0);
        else if (e < nx + ny) {
            F.uy[e - nx] = yh ? static_cast<T>(yh[e - nx]) : T(0);
            F.vs[e - nx] = sh ? static_cast<T>(sh[e - nx]) : T(0);
        } else {
            const int b = static_cast<int>(e - nx - ny);
            F.tau[b] = 1.0;
            F.kappa[b] = 0.0;
            F.done[b] = 0;
            F.status[b] = 0;
            F.iters[b] = 0;
        }
    }
}

// caller's units -> scaled: x^ = sigma E^-1 x, y^ = rho D^-1 y, s^ = sigma D s
template <typename T>
__global__ void to_scaled_kernel(Dev<T> F, double *x, double *y, double *s) {
    const int64_t nx = (int64_t)F.n * F.B, ny = (int64_t)F.m * F.B;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nx + ny;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nx) {
            const int b = static_cast<int>(e / F.n), j = static_cast<int>(e % F.n);
            if (x) x[e] = F.sigma[b] * x[e] / F.E[j];
        } else {
            const int64_t f = e - nx;
            const int b = static_cast<int>(f / F.m), i = static_cast<int>(f % F.m);
            if (y) y[f] = F.rho[b] * y[f] / F.D[i];
            if (s) s[f] = F.sigma[b] * F.D[i] * s[f];
        }
    }
}

// the inverse map: a scaled point (x^, y^, s^) of each member to the
// caller's units, x = E x^ / sigma, y = D y^ / rho, s = s^ / (sigma D)
// (Sec. 5 scaling; the warm start of Sec. 4.2 takes these units)
template <typename T>
__global__ void from_scaled_kernel(Dev<T> F, const double *xh, const double *yh, const double *sh, double *x,
                                   double *y, double *s) {
    const int64_t nx = (int64_t)F.n * F.B, ny = (int64_t)F.m * F.B;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nx + ny;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nx) {
            const int b = static_cast<int>(e / F.n), j = static_cast<int>(e % F.n);
            if (x) x[e] = F.E[j] * xh[e] / F.sigma[b];
        } else {
            const int64_t f = e - nx;
            const int b = static_cast<int>(f / F.m), i = static_cast<int>(f % F.m);
            if (y) y[f] = F.D[i] * yh[f] / F.rho[b];
            if (s) s[f] = sh[f] / (F.sigma[b] * F.D[i]);
        }
    }
}

// ---------------------------------------------------------------------------
class FamilyBase {
   public:
    virtual ~FamilyBase() {}
    virtual int set_data(const double *b, const double *c) = 0;
    virtual int warm_start(const double *x, const double *y, const double *s, int device_scaled) = 0;
    virtual int solve(double *x, double *y, double *s, scs_info *info, int device_out) = 0;
    virtual int iterate(int iters) = 0;
    virtual int get_iterates(int idx, double *u, double *v) = 0;
    virtual int snapshots(float *dst) = 0;
    virtual int unscale(const double *xh, const double *yh, const double *sh, double *x, double *y, double *s) = 0;
    virtual void dims(int32_t *n, int32_t *m, int32_t *count) = 0;
};

template <typename T>
class FamilyEngine : public FamilyBase {
   public:
    FamilyEngine(const HostProblem &P, int count, const double *b, const double *c, const scs_settings &st)
        : st_(st) {
        device_ = st.device;
        SCS_CUDA(cudaSetDevice(device_));
        SCS_CUDA(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, device_));
        if (st.cuda_stream) {
            stream_ = static_cast<cudaStream_t>(st.cuda_stream);
        } else {
            SCS_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
            own_stream_ = true;
        }
        n_ = P.n;
        m_ = P.m;
        B_ = count;
        setup(P, b, c);
    }

    ~FamilyEngine() override {
        cudaSetDevice(device_);
        if (exec_) cudaGraphExecDestroy(exec_);
        if (graph_) cudaGraphDestroy(graph_);
        for (void *p : allocs_) cudaFree(p);
        if (own_stream_ && stream_) cudaStreamDestroy(stream_);
    }

    template <typename U>
    U *dalloc(size_t cnt) {
        void *p = nullptr;
        SCS_CUDA(cudaMalloc(&p, sizeof(U) * (cnt ? cnt : 1)));
        allocs_.push_back(p);
        return static_cast<U *>(p);
    }
    template <typename U>
    U *upload(const U *h, size_t cnt) {
        U *d = dalloc<U>(cnt);
        if (cnt) SCS_CUDA(cudaMemcpyAsync(d, h, sizeof(U) * cnt, cudaMemcpyHostToDevice, stream_));
        return d;
    }
    int grid(int64_t len) const {
        int64_t g = (len + kBlock - 1) / kBlock;
        return static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)sms_ * 8)));
    }

    void setup(const HostProblem &P, const double *b, const double *c) {
        const int m = m_, n = n_;
        // ---- shared equilibration (Sec. 5; same passes as the single solver)
        std::vector<int32_t> rid_m(m), rid_n(n);
        for (int i = 0; i < m; ++i) rid_m[i] = i;
        for (int j = 0; j < n; ++j) rid_n[j] = j;
        int32_t *a_rp = upload(P.a_rowptr.data(), P.a_rowptr.size()), *a_col = upload(P.a_col.data(), P.a_col.size());
        int32_t *at_rp = upload(P.at_rowptr.data(), P.at_rowptr.size());
        int32_t *at_col = upload(P.at_col.data(), P.at_col.size());
        int32_t *rm = upload(rid_m.data(), m), *rn = upload(rid_n.data(), n);
        double *av = upload(P.a_val.data(), P.a_val.size()), *atv = upload(P.at_val.data(), P.at_val.size());
        double *D = dalloc<double>(m), *E = dalloc<double>(n), *tm = dalloc<double>(m), *tn = dalloc<double>(n);
        std::vector<int32_t> bo, bl, soc_off, soc_len;
        int off = P.z + P.l;
        for (int32_t qs : P.q) {
            bo.push_back(off);
            bl.push_back(qs);
            soc_off.push_back(off);
            soc_len.push_back(qs);
            off += qs;
        }
        int32_t *d_bo = upload(bo.data(), bo.size()), *d_bl = upload(bl.data(), bl.size());
        {
            std::vector<double> ones(std::max(m, n), 1.0);
            SCS_CUDA(cudaMemcpyAsync(D, ones.data(), sizeof(double) * m, cudaMemcpyHostToDevice, stream_));
            SCS_CUDA(cudaMemcpyAsync(E, ones.data(), sizeof(double) * n, cudaMemcpyHostToDevice, stream_));
            SCS_CUDA(cudaStreamSynchronize(stream_));
        }
        if (st_.normalize) {
            for (int pass = 0; pass < st_.scale_passes; ++pass) {
                row_sumsq_kernel<<<grid((int64_t)m * 32), kBlock, 0, stream_>>>(a_rp, av, rm, m, tm);
                row_sumsq_kernel<<<grid((int64_t)n * 32), kBlock, 0, stream_>>>(at_rp, atv, rn, n, tn);
                sqrt_kernel<<<grid(m), kBlock, 0, stream_>>>(tm, m);
                sqrt_kernel<<<grid(n), kBlock, 0, stream_>>>(tn, n);
                if (!bo.empty())
                    block_mean_kernel<<<grid((int64_t)bo.size() * 32), kBlock, 0, stream_>>>(
                        tm, d_bo, d_bl, (int)bo.size(), st_.block_scale);
                inv_sqrt_clamp_kernel<<<grid(m), kBlock, 0, stream_>>>(tm, m, 1e-4, 1e4, tm, D);
                inv_sqrt_clamp_kernel<<<grid(n), kBlock, 0, stream_>>>(tn, n, 1e-4, 1e4, tn, E);
                scale_vals_kernel<<<grid((int64_t)m * 32), kBlock, 0, stream_>>>(a_rp, a_col, av, rm, m, tm, tn);
                scale_vals_kernel<<<grid((int64_t)n * 32), kBlock, 0, stream_>>>(at_rp, at_col, atv, rn, n, tn, tm);
                SCS_CUDA(cudaGetLastError());
            }
        }
        row_sumsq_kernel<<<grid((int64_t)m * 32), kBlock, 0, stream_>>>(a_rp, av, rm, m, tm);
        sqrt_kernel<<<grid(m), kBlock, 0, stream_>>>(tm, m);
        std::vector<double> rown(m);
        SCS_CUDA(cudaMemcpyAsync(rown.data(), tm, sizeof(double) * m, cudaMemcpyDeviceToHost, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        double mean_row = 0.0;
        for (double t : rown) mean_row += t;
        mean_row = m ? mean_row / m : 1.0;
        if (!(mean_row > 0.0)) mean_row = 1.0;
        mean_row_ = mean_row;
        // ---- dense A^ (FP64, then T) and (I + A^T A)^-1
        double *A64 = dalloc<double>((size_t)m * n), *At64 = dalloc<double>((size_t)m * n);
        SCS_CUDA(cudaMemsetAsync(A64, 0, sizeof(double) * m * n, stream_));
        SCS_CUDA(cudaMemsetAsync(At64, 0, sizeof(double) * m * n, stream_));
        densify_kernel<<<grid(m), kBlock, 0, stream_>>>(a_rp, a_col, av, m, n, A64, At64);
        double *G = dalloc<double>((size_t)n * n), *colk = dalloc<double>(2 * (size_t)n);
        {
            std::vector<double> I((size_t)n * n, 0.0);
            for (int j = 0; j < n; ++j) I[(size_t)j * n + j] = 1.0;
            SCS_CUDA(cudaMemcpyAsync(G, I.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, stream_));
            SCS_CUDA(dense::gemm_nn<double>(stream_, n, n, m, 1.0, At64, n, A64, m, 1.0, G, n));   // I + A^T A
            SCS_CUDA(dense::invert_spd_gj<double>(stream_, G, n, colk, grid((int64_t)n * n)));
            SCS_CUDA(cudaStreamSynchronize(stream_));
        }
        Ah_ = dalloc<T>((size_t)m * n);
        Aht_ = dalloc<T>((size_t)m * n);
        Minv_ = dalloc<T>((size_t)n * n);
        cast_kernel<T><<<grid((int64_t)m * n), kBlock, 0, stream_>>>(A64, Ah_, (int64_t)m * n);
        cast_kernel<T><<<grid((int64_t)m * n), kBlock, 0, stream_>>>(At64, Aht_, (int64_t)m * n);
        cast_kernel<T><<<grid((int64_t)n * n), kBlock, 0, stream_>>>(G, Minv_, (int64_t)n * n);
        if constexpr (std::is_same<T, float>::value) {
            // FP32 family: the three fixed matrices split once for the tensor-core products
            Kpn_ = (n + 63) / 64 * 64;
            Kpm_ = (m + 63) / 64 * 64;
            S_At_ = dalloc<__nv_bfloat16>((size_t)n * 3 * Kpm_);   // A^T x: rows n, K = m (A^ column-major)
            S_A_ = dalloc<__nv_bfloat16>((size_t)m * 3 * Kpn_);    // A^ x: rows m, K = n (A^T column-major)
            S_M_ = dalloc<__nv_bfloat16>((size_t)n * 3 * Kpn_);    // (I + A^T A)^-1, symmetric
            mlp::split3_bf16(Ah_, n, m, m, 0, Kpm_, S_At_, stream_);
            mlp::split3_bf16(Aht_, m, n, n, 0, Kpn_, S_A_, stream_);
            mlp::split3_bf16(Minv_, n, n, n, 0, Kpn_, S_M_, stream_);
            S_mem_ = dalloc<__nv_bfloat16>((size_t)B_ * 3 * std::max(Kpn_, Kpm_));
            tc_err_ = dalloc<int>(1);
            SCS_CUDA(cudaMemsetAsync(tc_err_, 0, sizeof(int), stream_));
        }
        // ---- member arrays
        const size_t nx = (size_t)n * B_, ny = (size_t)m * B_;
        F_.n = n;
        F_.m = m;
        F_.B = B_;
        F_.z = P.z;
        F_.l = P.l;
        F_.nq = static_cast<int>(P.q.size());
        F_.soc_off = upload(soc_off.data(), soc_off.size());
        F_.soc_len = upload(soc_len.data(), soc_len.size());
        F_.D = D;
        F_.E = E;
        F_.ch = dalloc<T>(nx);
        F_.bh = dalloc<T>(ny);
        F_.c64 = dalloc<double>(nx);
        F_.b64 = dalloc<double>(ny);
        F_.px = dalloc<T>(nx);
        F_.py = dalloc<T>(ny);
        F_.hp1 = dalloc<double>(B_);
        F_.sigma = dalloc<double>(B_);
        F_.rho = dalloc<double>(B_);
        F_.nb = dalloc<double>(B_);
        F_.nc = dalloc<double>(B_);
        F_.ux = dalloc<T>(nx);
        F_.uy = dalloc<T>(ny);
        F_.vs = dalloc<T>(ny);
        F_.tau = dalloc<double>(B_);
        F_.kappa = dalloc<double>(B_);
        F_.rx = dalloc<T>(nx);
        F_.ry = dalloc<T>(ny);
        F_.zx = dalloc<T>(nx);
        F_.ax = dalloc<T>(ny);
        F_.aty = dalloc<T>(nx);
        F_.status = dalloc<int32_t>(B_);
        F_.iters = dalloc<int32_t>(B_);
        F_.done = dalloc<int32_t>(B_);
        F_.perm = dalloc<int32_t>(B_);
        {
            std::vector<int32_t> id(B_);
            for (int b = 0; b < B_; ++b) id[b] = b;
            SCS_CUDA(cudaMemcpyAsync(F_.perm, id.data(), sizeof(int32_t) * B_, cudaMemcpyHostToDevice, stream_));
        }
        pairs_ = dalloc<int32_t>(2 * (size_t)B_);
        F_.x = dalloc<double>(nx);
        F_.y = dalloc<double>(ny);
        F_.s = dalloc<double>(ny);
        F_.snap = dalloc<float>((size_t)(n + 2 * m + 1) * B_);
        F_.pobj = dalloc<double>(B_);
        F_.dobj = dalloc<double>(B_);
        F_.res_pri = dalloc<double>(B_);
        F_.res_dual = dalloc<double>(B_);
        F_.gap = dalloc<double>(B_);
        F_.ndone = dalloc<int>(1);
        F_.alpha = st_.alpha;
        F_.eps_pri = st_.eps_pri;
        F_.eps_dual = st_.eps_dual;
        F_.eps_gap = st_.eps_gap;
        F_.eps_infeas = st_.eps_infeas;
        F_.eps_unbdd = st_.eps_unbdd;
        bdev_ = dalloc<double>(ny);
        cdev_ = dalloc<double>(nx);
        SCS_CUDA(cudaStreamSynchronize(stream_));
        set_data(b, c);
        cold();
        build_graph();
    }

    // new b, c for every member (the cached inverse is kept, Sec. 4.2)
    int set_data(const double *b, const double *c) override {
        SCS_CUDA(cudaSetDevice(device_));
        const size_t nx = (size_t)n_ * B_, ny = (size_t)m_ * B_;
        SCS_CUDA(cudaMemcpyAsync(bdev_, b, sizeof(double) * ny, cudaMemcpyHostToDevice, stream_));
        SCS_CUDA(cudaMemcpyAsync(cdev_, c, sizeof(double) * nx, cudaMemcpyHostToDevice, stream_));
        member_scale_kernel<T><<<B_, kFamThreads, 0, stream_>>>(F_, bdev_, cdev_, mean_row_, st_.normalize);
        // p = M^-1 h, h = (c^, b^):  p_x = Minv (c^ - A^T b^),  p_y = b^ + A^ p_x
        SCS_CUDA(cudaMemcpyAsync(F_.rx, F_.ch, sizeof(T) * nx, cudaMemcpyDeviceToDevice, stream_));
        SCS_CUDA(cudaMemcpyAsync(F_.py, F_.bh, sizeof(T) * ny, cudaMemcpyDeviceToDevice, stream_));
        prod_At(B_, F_.bh, F_.rx, T(-1), T(1));
        prod_M(B_, F_.rx, F_.px);
        prod_A(B_, F_.px, F_.py, T(1), T(1));
        hp1_kernel<T><<<B_, kFamThreads, 0, stream_>>>(F_);
        SCS_CUDA(cudaGetLastError());
        SCS_CUDA(cudaStreamSynchronize(stream_));
        warm_pending_ = false;
        return 0;
    }

    void cold() {
        cold_kernel<T><<<grid((int64_t)(n_ + m_) * B_ + B_), kBlock, 0, stream_>>>(F_);
        SCS_CUDA(cudaGetLastError());
    }

    int warm_start(const double *x, const double *y, const double *s, int device_scaled) override {
        SCS_CUDA(cudaSetDevice(device_));
        const size_t nx = (size_t)n_ * B_, ny = (size_t)m_ * B_;
        if (device_scaled) {
            warm_kernel<T><<<grid((int64_t)(n_ + m_) * B_ + B_), kBlock, 0, stream_>>>(F_, x, y, s);
        } else {
            double *xs = x ? upload(x, nx) : nullptr, *ys = y ? upload(y, ny) : nullptr;
            double *ss = s ? upload(s, ny) : nullptr;
            to_scaled_kernel<T><<<grid((int64_t)(n_ + m_) * B_), kBlock, 0, stream_>>>(F_, xs, ys, ss);
            warm_kernel<T><<<grid((int64_t)(n_ + m_) * B_ + B_), kBlock, 0, stream_>>>(F_, xs, ys, ss);
            SCS_CUDA(cudaStreamSynchronize(stream_));
            for (double *p : {xs, ys, ss})
                if (p) release(p);
        }
        SCS_CUDA(cudaGetLastError());
        SCS_CUDA(cudaStreamSynchronize(stream_));
        warm_pending_ = true;
        return 0;
    }

    void release(void *p) {
        for (size_t i = 0; i < allocs_.size(); ++i)
            if (allocs_[i] == p) {
                cudaFree(p);
                allocs_.erase(allocs_.begin() + i);
                return;
            }
    }

    // The member products (Sec. 4.1 direct step in dense form) over the first
    // `cols` member columns, all column-major:
    //   prod_At: C (n x cols) = alpha A^T X (m x cols) + beta C
    //   prod_M:  C (n x cols) = (I + A^T A)^-1 X (n x cols)
    //   prod_A:  C (m x cols) = alpha A^ X (n x cols) + beta C
    // FP32: three-way BF16 split of X, then one tcgen05 product against the
    // matrix's split (FP32-accurate); FP64: the CUDA-core GEMM.
    void prod_At(int cols, const T *X, T *C, T alpha, T beta) {
        if constexpr (std::is_same<T, float>::value)
            prod_tc(S_At_, n_, m_, Kpm_, X, cols, C, alpha, beta);
        else
            SCS_CUDA(dense::gemm_nn<T>(stream_, n_, cols, m_, alpha, Aht_, n_, X, m_, beta, C, n_));
    }
    void prod_M(int cols, const T *X, T *C) {
        if constexpr (std::is_same<T, float>::value)
            prod_tc(S_M_, n_, n_, Kpn_, X, cols, C, T(1), T(0));
        else
            SCS_CUDA(dense::gemm_nn<T>(stream_, n_, cols, n_, T(1), Minv_, n_, X, n_, T(0), C, n_));
    }
    void prod_A(int cols, const T *X, T *C, T alpha, T beta) {
        if constexpr (std::is_same<T, float>::value)
            prod_tc(S_A_, m_, n_, Kpn_, X, cols, C, alpha, beta);
        else
            SCS_CUDA(dense::gemm_nn<T>(stream_, m_, cols, n_, alpha, Ah_, m_, X, n_, beta, C, m_));
    }
    void prod_tc(const __nv_bfloat16 *B3, int rows, int K, int Kp, const T *X, int cols, T *C, T alpha, T beta) {
        if (cols <= 0) return;
        const float *Xf = reinterpret_cast<const float *>(X);
        mlp::split3_bf16(Xf, cols, K, K, 0, Kp, S_mem_, stream_);
        mlp::gemm_fp32x3(S_mem_, cols, B3, rows, Kp, reinterpret_cast<float *>(C), rows, static_cast<float>(alpha),
                         static_cast<float>(beta), tc_err_, stream_);
    }

    // one iteration of the first A columns (the active members)
    void launch_iteration(int A) {
        Dev<T> F = F_;
        F.B = A;
        rhs_kernel<T><<<grid((int64_t)(n_ + m_) * A), kFamThreads, 0, stream_>>>(F);
        prod_At(A, F_.ry, F_.rx, T(-1), T(1));
        prod_M(A, F_.rx, F_.zx);
        prod_A(A, F_.zx, F_.ry, T(1), T(1));
        update_kernel<T><<<A, kFamThreads, 0, stream_>>>(F);
    }
    void launch_iteration() { launch_iteration(B_); }

    void launch_check(int A, int k, int final_pass) {
        Dev<T> F = F_;
        F.B = A;
        prod_A(A, F_.ux, F_.ax, T(1), T(0));
        prod_At(A, F_.uy, F_.aty, T(1), T(0));
        check_kernel<T><<<A, kFamThreads, 0, stream_>>>(F, k, final_pass);
    }

    // CUDA graph of check_interval iterations of the first A columns
    void build_graph(int A) {
        if (exec_) cudaGraphExecDestroy(exec_);
        if (graph_) cudaGraphDestroy(graph_);
        exec_ = nullptr;
        graph_ = nullptr;
        SCS_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
        const int ci = st_.check_interval > 0 ? st_.check_interval : 1;
        for (int i = 0; i < ci; ++i) launch_iteration(A);
        SCS_CUDA(cudaStreamEndCapture(stream_, &graph_));
        SCS_CUDA(cudaGraphInstantiate(&exec_, graph_, 0));
        graph_cols_ = A;
    }
    void build_graph() {
        // one iteration outside the capture first: the products' one-time
        // per-device set-up (the tensor-core kernel's shared-memory
        // attribute, the SM count) runs there
        launch_iteration();
        SCS_CUDA(cudaStreamSynchronize(stream_));
        cold();
        build_graph(B_);
    }

    // move the active columns of [0, A) to the front by swapping pairs
    // (done column in front, active column behind); returns the new A and
    // records the swaps so that they can be undone in reverse order
    int compact(int A) {
        std::vector<int32_t> done(A);
        SCS_CUDA(cudaMemcpyAsync(done.data(), F_.done, sizeof(int32_t) * A, cudaMemcpyDeviceToHost, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        int active = 0;
        for (int c = 0; c < A; ++c) active += done[c] ? 0 : 1;
        std::vector<int32_t> pr;
        int lo = 0, hi = A - 1;
        while (true) {
            while (lo < active && !done[lo]) ++lo;
            while (hi >= active && done[hi]) --hi;
            if (lo >= active || hi < active) break;
            pr.push_back(lo++);
            pr.push_back(hi--);
        }
        if (!pr.empty()) {
            const size_t off = swap_log_.size();
            swap_log_.insert(swap_log_.end(), pr.begin(), pr.end());
            swap_batches_.push_back({off, pr.size() / 2});
            SCS_CUDA(cudaMemcpyAsync(pairs_ + 0, pr.data(), sizeof(int32_t) * pr.size(), cudaMemcpyHostToDevice,
                                     stream_));
            swap_kernel<T><<<(int)(pr.size() / 2), kFamThreads, 0, stream_>>>(F_, pairs_);
            SCS_CUDA(cudaGetLastError());
            SCS_CUDA(cudaStreamSynchronize(stream_));
        }
        return active;
    }
    // undo every recorded swap (reverse order): columns hold members 0..B-1 again
    void restore_order() {
        for (size_t k = swap_batches_.size(); k-- > 0;) {
            const auto &bt = swap_batches_[k];
            SCS_CUDA(cudaMemcpyAsync(pairs_, swap_log_.data() + bt.first, sizeof(int32_t) * 2 * bt.second,
                                     cudaMemcpyHostToDevice, stream_));
            swap_kernel<T><<<(int)bt.second, kFamThreads, 0, stream_>>>(F_, pairs_);
            SCS_CUDA(cudaStreamSynchronize(stream_));
        }
        swap_log_.clear();
        swap_batches_.clear();
        SCS_CUDA(cudaGetLastError());
    }

    int solve(double *x, double *y, double *s, scs_info *info, int device_out) override {
        SCS_CUDA(cudaSetDevice(device_));
        const auto t0 = std::chrono::steady_clock::now();
        if (!warm_pending_) cold();
        warm_pending_ = false;
        SCS_CUDA(cudaMemsetAsync(F_.ndone, 0, sizeof(int), stream_));
        const int ci = st_.check_interval > 0 ? st_.check_interval : 1;
        int k = 0, ndone = 0, A = B_, ndone_at_compact = 0;
        if (graph_cols_ != A) build_graph(A);
        while (k < st_.max_iters && A > 0) {
            if (ci <= st_.max_iters - k) {
                SCS_CUDA(cudaGraphLaunch(exec_, stream_));
                k += ci;
            } else {
                while (k < st_.max_iters) {
                    launch_iteration(A);
                    ++k;
                }
            }
            launch_check(A, k, k >= st_.max_iters);
            SCS_CUDA(cudaMemcpyAsync(&ndone, F_.ndone, sizeof(int), cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaStreamSynchronize(stream_));
            if (ndone >= B_) break;
            // drop finished members from the products once a few percent of
            // the active columns have finished
            if (ndone - ndone_at_compact >= std::max(1, A / 32)) {
                A = compact(A);
                ndone_at_compact = ndone;
                if (A > 0) build_graph(A);
            }
        }
        restore_order();
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        const size_t nx = (size_t)n_ * B_, ny = (size_t)m_ * B_;
        const cudaMemcpyKind kind = device_out ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (x) SCS_CUDA(cudaMemcpyAsync(x, F_.x, sizeof(double) * nx, kind, stream_));
        if (y) SCS_CUDA(cudaMemcpyAsync(y, F_.y, sizeof(double) * ny, kind, stream_));
        if (s) SCS_CUDA(cudaMemcpyAsync(s, F_.s, sizeof(double) * ny, kind, stream_));
        if (info) {
            std::vector<int32_t> st(B_), it(B_);
            std::vector<double> po(B_), dob(B_), rp(B_), rd(B_), gp(B_), ta(B_), ka(B_);
            SCS_CUDA(cudaMemcpyAsync(st.data(), F_.status, 4 * B_, cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaMemcpyAsync(it.data(), F_.iters, 4 * B_, cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaMemcpyAsync(po.data(), F_.pobj, 8 * B_, cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaMemcpyAsync(dob.data(), F_.dobj, 8 * B_, cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaMemcpyAsync(rp.data(), F_.res_pri, 8 * B_, cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaMemcpyAsync(rd.data(), F_.res_dual, 8 * B_, cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaMemcpyAsync(gp.data(), F_.gap, 8 * B_, cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaMemcpyAsync(ta.data(), F_.tau, 8 * B_, cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaMemcpyAsync(ka.data(), F_.kappa, 8 * B_, cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaStreamSynchronize(stream_));
            for (int b = 0; b < B_; ++b) {
                scs_info f{};
                f.status = st[b];
                f.iters = it[b];
                f.cg_iters = 0;
                f.matvecs = 3 * it[b];
                f.pobj = po[b];
                f.dobj = dob[b];
                f.res_pri = rp[b];
                f.res_dual = rd[b];
                f.gap = gp[b];
                f.tau = ta[b];
                f.kappa = ka[b];
                f.solve_s = el;
                info[b] = f;
            }
        }
        SCS_CUDA(cudaStreamSynchronize(stream_));
        check_tc();
        return 0;
    }

    int iterate(int iters) override {
        SCS_CUDA(cudaSetDevice(device_));
        for (int i = 0; i < iters; ++i) launch_iteration();
        SCS_CUDA(cudaGetLastError());
        SCS_CUDA(cudaStreamSynchronize(stream_));
        check_tc();
        return 0;
    }

    // a bounded wait of a tensor-core product timed out: its output is not written
    void check_tc() {
        if (!tc_err_) return;
        int e = 0;
        SCS_CUDA(cudaMemcpy(&e, tc_err_, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) throw CudaError("a tensor-core product's bounded wait timed out", SCS_DEVICE_ERROR);
    }

    int get_iterates(int idx, double *u, double *v) override {
        if (idx < 0 || idx >= B_) return SCS_INVALID_INPUT;
        SCS_CUDA(cudaSetDevice(device_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        const int n = n_, m = m_, N = n + m + 1;
        std::vector<T> hx(n), hy(m), hs(m);
        double tau = 0.0, kappa = 0.0;
        SCS_CUDA(cudaMemcpy(hx.data(), F_.ux + (size_t)idx * n, sizeof(T) * n, cudaMemcpyDeviceToHost));
        SCS_CUDA(cudaMemcpy(hy.data(), F_.uy + (size_t)idx * m, sizeof(T) * m, cudaMemcpyDeviceToHost));
        SCS_CUDA(cudaMemcpy(hs.data(), F_.vs + (size_t)idx * m, sizeof(T) * m, cudaMemcpyDeviceToHost));
        SCS_CUDA(cudaMemcpy(&tau, F_.tau + idx, sizeof(double), cudaMemcpyDeviceToHost));
        SCS_CUDA(cudaMemcpy(&kappa, F_.kappa + idx, sizeof(double), cudaMemcpyDeviceToHost));
        for (int j = 0; j < n; ++j) {
            if (u) u[j] = static_cast<double>(hx[j]);
            if (v) v[j] = 0.0;
        }
        for (int i = 0; i < m; ++i) {
            if (u) u[n + i] = static_cast<double>(hy[i]);
            if (v) v[n + i] = static_cast<double>(hs[i]);
        }
        if (u) u[N - 1] = tau;
        if (v) v[N - 1] = kappa;
        return 0;
    }

    int unscale(const double *xh, const double *yh, const double *sh, double *x, double *y, double *s) override {
        SCS_CUDA(cudaSetDevice(device_));
        from_scaled_kernel<T><<<grid((int64_t)(n_ + m_) * B_), kBlock, 0, stream_>>>(F_, xh, yh, sh, x, y, s);
        SCS_CUDA(cudaGetLastError());
        SCS_CUDA(cudaStreamSynchronize(stream_));
        return 0;
    }

    int snapshots(float *dst) override {
        SCS_CUDA(cudaSetDevice(device_));
        SCS_CUDA(cudaMemcpyAsync(dst, F_.snap, sizeof(float) * (size_t)(n_ + 2 * m_ + 1) * B_,
                                 cudaMemcpyDefault, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        return 0;
    }

    void dims(int32_t *n, int32_t *m, int32_t *count) override {
        if (n) *n = n_;
        if (m) *m = m_;
        if (count) *count = B_;
    }

    scs_settings st_;
    int device_ = 0, sms_ = 1, n_ = 0, m_ = 0, B_ = 0;
    double mean_row_ = 1.0;
    bool own_stream_ = false, warm_pending_ = false;
    cudaStream_t stream_ = nullptr;
    std::vector<void *> allocs_;
    T *Ah_ = nullptr, *Aht_ = nullptr, *Minv_ = nullptr;   // A^ (m x n), A^T (n x m), (I + A^T A)^-1
    // FP32 family: BF16 three-way splits of A^T, A^, (I + A^T A)^-1 and of the
    // member operand of the product in progress; the products' error flag
    __nv_bfloat16 *S_At_ = nullptr, *S_A_ = nullptr, *S_M_ = nullptr, *S_mem_ = nullptr;
    int *tc_err_ = nullptr;
    int Kpn_ = 0, Kpm_ = 0;
    double *bdev_ = nullptr, *cdev_ = nullptr;
    int32_t *pairs_ = nullptr;
    std::vector<int32_t> swap_log_;
    std::vector<std::pair<size_t, size_t>> swap_batches_;
    int graph_cols_ = -1;
    Dev<T> F_{};
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
};

}  // namespace family
}  // namespace scs

struct scs_family {
    scs::family::FamilyBase *eng = nullptr;
};

namespace {
template <typename F>
int32_t family_guarded(F f) {
    try {
        return f();
    } catch (const scs::CudaError &e) {
        scs::set_last_error(e.what());
        return e.code;
    } catch (const std::exception &e) {
        scs::set_last_error(e.what());
        return SCS_DEVICE_ERROR;
    }
}
}  // namespace

extern "C" {

scs_family *scs_family_init(const scs_csc *A, const scs_cone *k, int32_t count, const double *b, const double *c,
                            const scs_settings *st, int32_t *err) {
    int32_t e = 0;
    scs_family *w = nullptr;
    scs::HostProblem P;
    if (count <= 0 || !A || !k || !b || !c) {
        scs::set_last_error("bad family arguments");
        e = SCS_INVALID_INPUT;
    } else if (k->ns > 0 || k->ep > 0 || k->ed > 0 || k->np > 0) {
        scs::set_last_error("family programs take zero, nonnegative and second-order cones only");
        e = SCS_UNSUPPORTED;
    } else {
        e = scs::validate_and_build(A, b, c, k, P);
    }
    scs_settings s{};
    if (!e) {
        if (st) s = *st;
        else scs_default_settings(&s);
        if ((int64_t)A->m * A->n > ((int64_t)1 << 31)) {
            scs::set_last_error("dense A^ too large for the family solver");
            e = SCS_UNSUPPORTED;
        }
    }
    if (!e) {
        e = family_guarded([&]() -> int32_t {
            w = new scs_family;
            if (s.precision == 0)
                w->eng = new scs::family::FamilyEngine<double>(P, count, b, c, s);
            else
                w->eng = new scs::family::FamilyEngine<float>(P, count, b, c, s);
            return 0;
        });
        if (e && w) {
            delete w->eng;
            delete w;
            w = nullptr;
        }
    }
    if (err) *err = e;
    return e ? nullptr : w;
}

int32_t scs_family_set_data(scs_family *w, const double *b, const double *c) {
    if (!w || !w->eng || !b || !c) return SCS_INVALID_INPUT;
    return family_guarded([&] { return w->eng->set_data(b, c); });
}

int32_t scs_family_warm_start(scs_family *w, const double *x, const double *y, const double *s,
                              int32_t device_scaled) {
    if (!w || !w->eng) return SCS_INVALID_INPUT;
    return family_guarded([&] { return w->eng->warm_start(x, y, s, device_scaled); });
}

int32_t scs_family_solve(scs_family *w, double *x, double *y, double *s, scs_info *info, int32_t device_out) {
    if (!w || !w->eng) return SCS_INVALID_INPUT;
    return family_guarded([&] { return w->eng->solve(x, y, s, info, device_out); });
}

int32_t scs_family_iterate(scs_family *w, int32_t iters) {
    if (!w || !w->eng || iters < 0) return SCS_INVALID_INPUT;
    return family_guarded([&] { return w->eng->iterate(iters); });
}

int32_t scs_family_get_iterates(scs_family *w, int32_t index, double *u, double *v) {
    if (!w || !w->eng) return SCS_INVALID_INPUT;
    return family_guarded([&] { return w->eng->get_iterates(index, u, v); });
}

int32_t scs_family_snapshots(scs_family *w, float *dst) {
    if (!w || !w->eng || !dst) return SCS_INVALID_INPUT;
    return family_guarded([&] { return w->eng->snapshots(dst); });
}

int32_t scs_family_unscale(scs_family *w, const double *xh, const double *yh, const double *sh, double *x, double *y,
                           double *s) {
    if (!w || !w->eng || !xh || !yh || !sh || !x || !y || !s) return SCS_INVALID_INPUT;
    return family_guarded([&] { return w->eng->unscale(xh, yh, sh, x, y, s); });
}

int32_t scs_family_dims(scs_family *w, int32_t *n, int32_t *m, int32_t *count) {
    if (!w || !w->eng) return SCS_INVALID_INPUT;
    w->eng->dims(n, m, count);
    return 0;
}

void scs_family_finish(scs_family *w) {
    if (!w) return;
    delete w->eng;
    delete w;
}

int32_t scs_dense_gemm(int32_t precision, int32_t M, int32_t N, int32_t K, double alpha, const void *A, int64_t lda,
                       const void *B, int64_t ldb, double beta, void *C, int64_t ldc, void *stream) {
    using namespace scs;
    if (M < 0 || N < 0 || K < 0 || precision < 0 || precision > 2 || lda < std::max(1, M) ||
        ldb < std::max(1, K) || ldc < std::max(1, M) || (M && N && (!C || (K && (!A || !B))))) {
        set_last_error("scs_dense_gemm: bad sizes, leading dimensions or pointers");
        return SCS_INVALID_INPUT;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (precision == 2) {
        // FP32 through the three-way BF16 split on the tensor cores: C^T
        // (N x M) = B^T A^T, B's columns and A's rows K-contiguous after the split
        if (!M || !N) return 0;
        const int Kp = std::max(64, (K + 63) / 64 * 64);
        __nv_bfloat16 *a3 = nullptr, *b3 = nullptr;
        int *err = nullptr;
        int rc = 0;
        if (cudaMalloc(&a3, sizeof(__nv_bfloat16) * 3 * (size_t)Kp * N) != cudaSuccess ||
            cudaMalloc(&b3, sizeof(__nv_bfloat16) * 3 * (size_t)Kp * M) != cudaSuccess ||
            cudaMalloc(&err, sizeof(int)) != cudaSuccess || cudaMemsetAsync(err, 0, sizeof(int), s) != cudaSuccess) {
            rc = SCS_DEVICE_ERROR;
        } else {
            try {
                mlp::split3_bf16(static_cast<const float *>(B), N, K, ldb, 0, Kp, a3, s);
                mlp::split3_bf16(static_cast<const float *>(A), M, K, lda, 1, Kp, b3, s);
                mlp::gemm_fp32x3(a3, N, b3, M, Kp, static_cast<float *>(C), ldc, static_cast<float>(alpha),
                                 static_cast<float>(beta), err, s);
                int h = 0;
                if (cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess || h)
                    rc = SCS_DEVICE_ERROR;
            } catch (const CudaError &ex) {
                set_last_error(std::string("scs_dense_gemm: ") + ex.what());
                rc = ex.code;
            }
        }
        cudaFree(a3);
        cudaFree(b3);
        cudaFree(err);
        if (rc == SCS_DEVICE_ERROR) set_last_error("scs_dense_gemm: the tensor-core product failed");
        return rc;
    }
    const cudaError_t e =
        precision == 0 ? dense::gemm_nn<double>(s, M, N, K, alpha, static_cast<const double *>(A), lda,
                                                static_cast<const double *>(B), ldb, beta, static_cast<double *>(C),
                                                ldc)
                       : dense::gemm_nn<float>(s, M, N, K, static_cast<float>(alpha), static_cast<const float *>(A),
                                               lda, static_cast<const float *>(B), ldb, static_cast<float>(beta),
                                               static_cast<float *>(C), ldc);
    if (e != cudaSuccess) {
        set_last_error(std::string("scs_dense_gemm: ") + cudaGetErrorString(e));
        return SCS_DEVICE_ERROR;
    }
    return 0;
}

}  // extern "C"
