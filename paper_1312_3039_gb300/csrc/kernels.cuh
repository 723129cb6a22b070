// Kernels of one ADMM iteration on the homogeneous self-dual embedding.
//
// Notation (Sec. 2.3, Sec. 4.1): u = (u_x, u_y, u_tau) in R^(n+m+1),
// v = (0, v_s, v_kappa) (v_x stays 0 and is never touched), A^ = D A E is the
// equilibrated data with b^, c^ (Sec. 5).  One iteration of Eq. "e-SCS" with
// over-relaxation (Sec. 3.3):
//   w      = u + v
//   r      = w_xy - w_tau h,  h = (c^, b^)
//   z      = M^-1 r, M = [I A^T; -A I]  via  z_x = (I + A^T A)^-1 (r_x - A^T r_y)
//            (Jacobi PCG warm-started from the previous z_x, Sec. 4.1) and
//            z_y = r_y + A z_x
//   u~_xy  = z - p gamma,  gamma = h^T z / (1 + h^T p),  u~_tau = w_tau + gamma
//   u_bar  = alpha u~ + (1 - alpha) u
//   u+     = Pi_C(u_bar - v),  v+ = v - u_bar + u+
//
// Arrangement on the device (2 + 2K sparse products per iteration for K CG
// steps, the count of Table 5, on every kAzEvery-th iteration; 1 + 2K on the
// others):
//   K1  SpMV A   : y_acc = r_y + A z_prev, az = A z_prev     (r_y formed per row)
//                  on iterations k = 0 mod kAzEvery; on the others
//   K1' elementwise: y_acc = r_y + az, where az = A z_prev is carried from the
//                  previous iteration (K5 adds alpha q to it whenever z moves
//                  by alpha p, so az = A z holds in exact arithmetic; the
//                  product every kAzEvery iterations bounds the drift of the
//                  carried sum to a few rounding errors)
//   K2  SpMV A^T : r0 = r_x - z_prev - A^T y_acc  (= t - (I + A^T A) z_prev),
//                  p0 = r0 / diag, CG dots, CG tolerance zeta^k
//   CG step (while not converged):
//   K3  SpMV A   : q = A p,  alpha = r.s / (p.p + q.q)   (p^T (I + A^T A) p)
//   K4  SpMV A^T : z += alpha p,  r -= alpha (p + A^T q),  new r.s, ||r||;
//                  its CTAs also run y_acc += alpha q (keeps y_acc = r_y + A z)
//                  and az += alpha q over the m rows
//   K5  update   : p = s + beta p
//   K6  SMW      : gamma = (c^.z_x + b^.y_acc) / (1 + h^T p)
//   KP  relax + project + dual update of the PSD blocks (one CTA per block,
//       Jacobi eigensolver; psd.cuh), when the cone has PSD blocks
//   K7  relax + project onto C + dual update (fused, per cone type) of the
//       other rows; its last CTA adds the PSD blocks' step lengths
// Each reduction is a deterministic grid sum whose last CTA updates the
// scalars (and, inside a CUDA graph, the CG loop's conditional handle).
//
// Precision: T is the type of A, the CG vectors and the working copies of the
// iterates u, v and of p = M^-1 h (float in the mixed-precision engine,
// double in the FP64 engine).  Threads accumulate their reduction values in
// T and the grid sums add them in FP64; the scaling, the termination tests,
// tau / kappa and the exponential-cone root polish are FP64 (GB300's FP64
// rate is a small fraction of its FP32 rate, so FP64 stays off the
// per-element paths of the mixed-precision engine).
#pragma once

#include <math.h>

#include <type_traits>

#include "common.cuh"
#include "cones.cuh"
#include "psd.cuh"
#include "spmv.cuh"

namespace scs {

struct CondHandle {
    cudaGraphConditionalHandle h;
    int valid;
    __device__ __forceinline__ void set(unsigned v) const {
        if (valid) cudaGraphSetConditional(h, v);
    }
};

// iterations whose K1 recomputes A z_prev by the sparse product
__device__ __forceinline__ bool az_product(const Scalars *S) { return S->k % kAzEvery == 0; }

// ---------------------------------------------------------------------------
// K1: rows of A.  y_acc_i = (u_y + v_s - w_tau b^)_i + (A^ z)_i, az_i = (A^ z)_i
// ---------------------------------------------------------------------------
template <typename T>
struct EpiAInit {
    static constexpr int NV = 1;
    static constexpr int kSite = kSiteAInit;
    const T *u, *v, *b;
    T *yacc, *az;
    Scalars *S;
    int n, N;
    double wtau;
    struct In { T w, b; };
    __device__ bool skip() const { return !az_product(S); }
    __device__ void begin() { wtau = static_cast<double>(u[N - 1]) + static_cast<double>(v[N - 1]); }
    __device__ In load(int i) const { return In{u[n + i] + v[n + i], b[i]}; }
    __device__ void row(int i, T s, const In &in, T (&red)[NV]) {
        yacc[i] = in.w - static_cast<T>(wtau) * in.b + s;
        az[i] = s;
        red[0] += in.w * in.w;
    }
    __device__ void finish(const double (&t)[NV]) { S->ww_y = t[0]; }
};

// ---------------------------------------------------------------------------
// K1': the same y_acc from the carried az = A^ z (iterations k != 0 mod kAzEvery)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock) yacc_init_kernel(int n, int m, int N, const T *__restrict__ u,
                                                           const T *__restrict__ v, const T *__restrict__ b,
                                                           const T *__restrict__ az, T *__restrict__ yacc,
                                                           Scalars *S, ReduceBuf rb) {
    if (az_product(S)) return;
    const T wtau = static_cast<T>(static_cast<double>(u[N - 1]) + static_cast<double>(v[N - 1]));
    T acc = 0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < m; i += gridDim.x * kBlock) {
        const T w = u[n + i] + v[n + i];
        yacc[i] = w - wtau * b[i] + az[i];
        acc += w * w;
    }
    double red[1] = {static_cast<double>(acc)}, tot[1];
    if (grid_sum<1>(red, rb, kSiteAz, tot)) {
        if (threadIdx.x == 0) S->ww_y = tot[0];
    }
}

// ---------------------------------------------------------------------------
// K2: rows of A^T.  r0_j = (u_x - w_tau c^)_j - z_j - (A^T y_acc)_j
// ---------------------------------------------------------------------------
template <typename T>
struct EpiAtInit {
    static constexpr int NV = 4;
    static constexpr int kSite = kSiteAtInit;
    const T *u, *v, *c;
    const T *diag;
    T *z, *r, *p;
    Scalars *S;
    CondHandle cond;
    int N;
    double wtau;
    struct In { T ux, c, z, d; };
    __device__ bool skip() const { return false; }
    __device__ void begin() { wtau = static_cast<double>(u[N - 1]) + static_cast<double>(v[N - 1]); }
    __device__ In load(int j) const { return In{u[j], c[j], z[j], diag[j]}; }
    __device__ void row(int j, T s, const In &in, T (&red)[NV]) {
        const T rj = in.ux - static_cast<T>(wtau) * in.c - in.z - s;
        const T sj = rj / in.d;
        r[j] = rj;
        p[j] = sj;
        red[0] += rj * sj;
        red[1] += rj * rj;
        red[2] += sj * sj;
        red[3] += in.ux * in.ux;
    }
    __device__ void finish(const double (&t)[NV]) {
        const double ww = t[3] + S->ww_y + wtau * wtau;
        // zeta^k = (1/k)^cg_rate (Sec. 6.1), capped at cg_adapt times the last
        // ADMM step length, floored at cg_tol_rel ||w||
        double tol = INFINITY;
        if (S->cg_rate > 0.0) tol = pow(1.0 / (double)(S->k + 1), S->cg_rate);
        if (S->cg_adapt > 0.0) tol = fmin(tol, S->cg_adapt * S->dstep);
        if (!isfinite(tol)) tol = 0.0;
        tol = fmax(tol, S->cg_tol_rel * sqrt(ww));
        S->tol = tol;
        S->wtau = wtau;
        S->rz = t[0];
        S->rr = t[1];
        S->pp = t[2];
        S->cg_it = 0;
        const int done = !(sqrt(t[1]) > tol) || S->cg_max <= 0;
        S->done = done;
        S->active = !done;
        cond.set(!done);
    }
};

// ---------------------------------------------------------------------------
// K3: rows of A.  q = A^ p
// ---------------------------------------------------------------------------
template <typename T>
struct EpiACG {
    static constexpr int NV = 1;
    static constexpr int kSite = kSiteACG;
    T *q;
    Scalars *S;
    struct In {};
    __device__ bool skip() const { return !S->active; }
    __device__ void begin() {}
    __device__ In load(int) const { return In{}; }
    __device__ void row(int i, T s, const In &, T (&red)[NV]) {
        q[i] = s;
        red[0] += s * s;
    }
    __device__ void finish(const double (&t)[NV]) {
        S->qq = t[0];
        S->alpha = S->rz / (S->pp + t[0]);
    }
};

// ---------------------------------------------------------------------------
// K4: rows of A^T.  (I + A^T A) p = p + A^T q; z += alpha p; r -= alpha G p;
// side task over the m rows of A: y_acc += alpha q (keeps y_acc = r_y + A z)
// and az += alpha q (the carried A z), while the product's gathers wait
// ---------------------------------------------------------------------------
template <typename T>
struct EpiAtCG {
    static constexpr int NV = 2;
    static constexpr int kSite = kSiteAtCG;
    const T *diag;
    T *z, *r, *p;
    Scalars *S;
    T alpha;
    const T *q;
    T *yacc, *az;
    int m;
    __device__ void side(int b, int nb) {
        for (int i = b * kBlock + threadIdx.x; i < m; i += nb * kBlock) {
            const T qi = q[i];
            yacc[i] = yacc[i] + alpha * qi;
            az[i] = az[i] + alpha * qi;
        }
    }
    struct In { T p, z, r, d; };
    __device__ bool skip() const { return !S->active; }
    __device__ void begin() { alpha = static_cast<T>(S->alpha); }
    __device__ In load(int j) const { return In{p[j], z[j], r[j], diag[j]}; }
    __device__ void row(int j, T s, const In &in, T (&red)[NV]) {
        const T pj = in.p;
        const T gp = pj + s;
        z[j] = in.z + alpha * pj;
        const T rj = in.r - alpha * gp;
        r[j] = rj;
        const T sj = rj / in.d;
        red[0] += rj * sj;
        red[1] += rj * rj;
    }
    __device__ void finish(const double (&t)[NV]) {
        S->cg_it += 1;
        S->cg_total += 1;
        S->rr = t[1];
        const int done = !(sqrt(t[1]) > S->tol) || S->cg_it >= S->cg_max;
        S->done = done;
        S->beta = t[0] / S->rz;
        S->rz = t[0];
    }
};

// ---------------------------------------------------------------------------
// K5: p = r / diag + beta p (K4's side task has updated y_acc and az)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock) cg_update_kernel(int n, int m, const T *__restrict__ q,
                                                           T *__restrict__ yacc, T *__restrict__ az,
                                                           const T *__restrict__ r, const T *__restrict__ diag,
                                                           T *__restrict__ p, Scalars *S, CondHandle cond,
                                                           ReduceBuf rb) {
    if (!S->active) return;
    const T beta = static_cast<T>(S->beta);
    const int done = S->done;
    T acc = 0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n && !done; i += gridDim.x * kBlock) {
        const T pj = r[i] / diag[i] + beta * p[i];
        p[i] = pj;
        acc += pj * pj;
    }
    double red[1] = {static_cast<double>(acc)}, tot[1];
    if (grid_sum<1>(red, rb, kSiteCGUpd, tot)) {
        if (threadIdx.x == 0) {
            if (!done) S->pp = tot[0];
            S->active = !done;
            cond.set(!done);
        }
    }
}

// ---------------------------------------------------------------------------
// Direct subspace step (settings.linsys = 1, Sec. 4.1 "direct method" with
// the factorization cached, Sec. 4.2): after K2 has formed
// r0 = t - (I + A^T A) z_prev, one exact correction d = (I + A^T A)^-1 r0
// replaces the CG loop:
//   KD1 dense   : d = Minv r0 (Minv symmetric, n x n, column j read as row j;
//                 one warp per row, lanes striding over the row, a fixed
//                 shuffle tree: deterministic); z += d; p = d
//   KD2 SpMV A  : q = A^ d; y_acc += q (keeps y_acc = r_y + A^ z);
//                 az += q (keeps the carried az = A^ z)
// so that z = Minv t and y_acc = r_y + A^ z up to rounding.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock) direct_gemv_kernel(int n, const T *__restrict__ Minv,
                                                             const T *__restrict__ r, T *__restrict__ z,
                                                             T *__restrict__ p) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * kWarps;
    for (int j = blockIdx.x * kWarps + (threadIdx.x >> 5); j < n; j += warps) {
        const T *row = Minv + (size_t)j * n;
        T acc = 0;
        for (int i = lane; i < n; i += 32) acc += row[i] * r[i];
        acc = warp_sum(acc);
        if (lane == 0) {
            z[j] = z[j] + acc;
            p[j] = acc;
        }
    }
}

template <typename T>
struct EpiADirect {
    static constexpr int NV = 1;
    static constexpr int kSite = kSiteACG;     // K3 does not run in the direct step
    T *q, *yacc, *az;
    Scalars *S;
    struct In { T y, a; };
    __device__ bool skip() const { return false; }
    __device__ void begin() {}
    __device__ In load(int i) const { return In{yacc[i], az[i]}; }
    __device__ void row(int i, T s, const In &in, T (&red)[NV]) {
        q[i] = s;
        yacc[i] = in.y + s;
        az[i] = in.a + s;
        red[0] += s * s;
    }
    __device__ void finish(const double (&t)[NV]) { S->qq = t[0]; }
};

// ---------------------------------------------------------------------------
// K6: gamma = h^T z / (1 + h^T p)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kBlock) smw_kernel(int n, int m, const T *__restrict__ c,
                                                     const T *__restrict__ b, const T *__restrict__ z,
                                                     const T *__restrict__ yacc, Scalars *S, ReduceBuf rb) {
    T acc = 0;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n + m; i += gridDim.x * kBlock) {
        acc += i < n ? c[i] * z[i] : b[i - n] * yacc[i - n];
    }
    double red[1] = {static_cast<double>(acc)}, tot[1];
    if (grid_sum<1>(red, rb, kSiteSmw, tot)) {
        if (threadIdx.x == 0) S->gamma = tot[0] / S->hp1;
    }
}

// ---------------------------------------------------------------------------
// K7: relax, project onto C = R^n x K* x R+, update v  (one launch)
//   block ranges: [0, nb_exp)       exponential, dual exponential and power
//                                   triples, kExpPerCta per CTA
//                                   (long dependent chains: started first,
//                                   spread over many SMs)
//                 [.., + nb_soc)    second-order blocks, one warp per block,
//                                   warps striding over the blocks
//                 [.., + nb_elem)   x-part, zero rows, nonnegative rows, tau:
//                                   threads striding over the rows, four rows'
//                                   loads issued before their stores
//   nb_soc and nb_elem are capped at one wave of resident CTAs: one CTA per
//   256 rows made ~1e4 CTAs whose partial sums, arrival atomics and final
//   reduction cost more than the streaming itself.
// ---------------------------------------------------------------------------
constexpr int kExpPerCta = 64;

struct ConeDev {
    int z, l;              // zero and nonnegative row counts
    int nq;                // second-order blocks
    const int32_t *q_off;  // row offset (within y) of each SOC block
    const int32_t *q_len;
    int ep;                // exponential triples, then
    int ed;                // dual exponential triples (K holds Kexp*), then
    int np;                // power triples, parameter pow_a[i] (< 0: dual power cone)
    const double *pow_a;
    int exp_off;           // row offset of the first triple
    int nb_elem, nb_soc, nb_exp;
    int npsd;              // PSD blocks (projected by psd_project_kernel)
    const double *psd_dd;  // squared step length of each PSD block's rows
};

template <typename T>
struct ProjArgs {
    int n, m, N;
    T *u, *v;
    const T *p;            // cached M^-1 h (n + m)
    const T *z;            // z_x
    const T *yacc;         // z_y
    Scalars *S;
};

template <typename T>
__device__ __forceinline__ T relaxed(const ProjArgs<T> &a, int idx, T gamma, T alpha) {
    // u~ = z - p gamma; u_bar = alpha u~ + (1 - alpha) u
    const T zi = idx < a.n ? a.z[idx] : a.yacc[idx - a.n];
    const T ut = zi - a.p[idx] * gamma;
    return alpha * ut + (T(1) - alpha) * a.u[idx];
}

template <typename T>
__global__ void __launch_bounds__(kBlock) relax_project_kernel(ProjArgs<T> a, ConeDev K, ReduceBuf rb) {
    const double gamma_d = a.S->gamma;
    const T gamma = static_cast<T>(gamma_d);
    const T alpha = static_cast<T>(a.S->relax);
    const int bid = blockIdx.x;
    T dd = 0;               // squared length of this thread's part of the step
    if (bid < K.nb_exp) {
        const int tri = bid * kExpPerCta + threadIdx.x;
        if (threadIdx.x < kExpPerCta && tri < K.ep + K.ed + K.np) {
            const int off = a.n + K.exp_off + 3 * tri;
            T t[3], up[3];
            T uo[3], vo[3];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                uo[e] = a.u[off + e];
                vo[e] = a.v[off + e];
                t[e] = relaxed(a, off + e, gamma, alpha) - vo[e];
            }
            // in the precision of the iterates (FP32: no FP64 in this kernel).
            // The y-part goes to K*: Kexp* for an exponential triple, Kexp for
            // a dual one, (Kpow^a)* for a power triple, Kpow^a for a dual one.
            if (tri < K.ep + K.ed) {
                const bool dual_cone = tri >= K.ep;
                if constexpr (std::is_same<T, float>::value) {
                    if (dual_cone) proj_exp_f(t[0], t[1], t[2], up[0], up[1], up[2]);
                    else proj_exp_dual_f(t[0], t[1], t[2], up[0], up[1], up[2]);
                } else {
                    if (dual_cone) proj_exp(t[0], t[1], t[2], up[0], up[1], up[2]);
                    else proj_exp_dual(t[0], t[1], t[2], up[0], up[1], up[2]);
                }
            } else {
                const double pa = K.pow_a[tri - K.ep - K.ed];
                if (pa > 0.0) proj_pow_dual<T>(t[0], t[1], t[2], static_cast<T>(pa), up[0], up[1], up[2]);
                else proj_pow<T>(t[0], t[1], t[2], static_cast<T>(-pa), up[0], up[1], up[2]);
            }
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                const T un = up[e], vn = up[e] - t[e];
                a.u[off + e] = un;
                a.v[off + e] = vn;
                dd += (un - uo[e]) * (un - uo[e]) + (vn - vo[e]) * (vn - vo[e]);
            }
        }
    } else if (bid - K.nb_exp < K.nb_soc) {
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int blk = (bid - K.nb_exp) * kWarps + warp; blk < K.nq; blk += K.nb_soc * kWarps) {
            const int off = a.n + K.q_off[blk];
            const int len = K.q_len[blk];
            // t = u_bar - v over the block; projection onto SOC (self-dual)
            T t0 = 0, xx = 0;
            for (int e = lane; e < len; e += 32) {
                const T t = relaxed(a, off + e, gamma, alpha) - a.v[off + e];
                if (e == 0) t0 = t; else xx += t * t;
            }
            xx = warp_sum(xx);
            t0 = __shfl_sync(0xffffffffu, t0, 0);
            const T nx = sqrt(xx);
            T head, tail;                       // projection = (head, tail * x)
            if (nx <= t0) { head = t0; tail = T(1); }
            else if (nx <= -t0) { head = T(0); tail = T(0); }
            else {
                head = T(0.5) * (t0 + nx);
                tail = head / nx;
            }
            for (int e = lane; e < len; e += 32) {
                const T uo = a.u[off + e], vo = a.v[off + e];
                const T t = relaxed(a, off + e, gamma, alpha) - vo;
                const T up = e == 0 ? head : tail * t;
                a.u[off + e] = up;
                a.v[off + e] = up - t;
                dd += (up - uo) * (up - uo) + (up - t - vo) * (up - t - vo);
            }
        }
    } else {
        const int ebid = bid - K.nb_exp - K.nb_soc;
        const int nlin = a.n + K.z + K.l;
        const int stride = K.nb_elem * kBlock;
        constexpr int kU = 4;
        for (int64_t base = ebid * kBlock + threadIdx.x; base < nlin; base += static_cast<int64_t>(kU) * stride) {
            T ub[kU], uo[kU], vo[kU];
#pragma unroll
            for (int j = 0; j < kU; ++j) {
                const int64_t i64 = base + static_cast<int64_t>(j) * stride;
                if (i64 < nlin) {
                    const int idx = static_cast<int>(i64);
                    ub[j] = relaxed(a, idx, gamma, alpha);
                    uo[j] = a.u[idx];
                    vo[j] = idx < a.n ? T(0) : a.v[idx];
                }
            }
#pragma unroll
            for (int j = 0; j < kU; ++j) {
                const int64_t i64 = base + static_cast<int64_t>(j) * stride;
                if (i64 >= nlin) break;
                const int idx = static_cast<int>(i64);
                if (idx < a.n) {
                    a.u[idx] = ub[j];                    // R^n: identity, v_x stays 0
                    dd += (ub[j] - uo[j]) * (ub[j] - uo[j]);
                } else {
                    const T t = ub[j] - vo[j];
                    const T up = (idx < a.n + K.z) ? t : (t > T(0) ? t : T(0));   // K* of {0} is R
                    a.u[idx] = up;
                    a.v[idx] = up - t;
                    dd += (up - uo[j]) * (up - uo[j]) + (up - t - vo[j]) * (up - t - vo[j]);
                }
            }
        }
        if (ebid == 0 && threadIdx.x == 0) {
            // tau (FP64): u~_tau = w_tau + gamma
            const int it = a.N - 1;
            const double ut = a.S->wtau + gamma_d;
            const double uo = static_cast<double>(a.u[it]), vo = static_cast<double>(a.v[it]);
            const double ub = a.S->relax * ut + (1.0 - a.S->relax) * uo;
            const double t = ub - vo;
            const double up = fmax(t, 0.0);
            a.u[it] = static_cast<T>(up);
            a.v[it] = static_cast<T>(up - t);
            dd += static_cast<T>((up - uo) * (up - uo) + (up - t - vo) * (up - t - vo));
        }
    }
    double red[1] = {static_cast<double>(dd)}, tot[1];
    if (grid_sum<1>(red, rb, kSiteProj, tot)) {
        if (threadIdx.x < 32) {
            double extra = 0.0;
            for (int b = threadIdx.x; b < K.npsd; b += 32) extra += K.psd_dd[b];
            extra = warp_sum(extra);
            if (threadIdx.x == 0) {
                a.S->dstep = sqrt(tot[0] + extra);
                a.S->k += 1;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// KP: relax + project + dual update of the PSD blocks, one CTA per block.
// The rows of block b start at y-row P.off[b]; the block's eigenvectors
// persist in P.V between iterations (warm start of the Jacobi sweeps).
// ---------------------------------------------------------------------------
template <typename T>
struct PsdDev {
    int npsd;
    const int32_t *ord;    // order of each block
    const int32_t *off;    // y-row offset of each block's svec
    const int64_t *voff;   // offset of each block's eigenvector matrix in V
    T *V;                  // eigenvectors (psd_ne x psd_ld per block)
    T *work;               // 2 matrices per block when they do not fit on chip
    int64_t work_stride;   // elements of one matrix in `work`
    double *dd;            // squared step length of each block
    int ne_max;            // psd_ne of the largest order
    int smem;              // X, V, W in shared memory
    int small_bytes;       // bytes of the small tables at the start of shared memory
    double fp64_cond;      // FP64 reconstruction above this spread of the positive eigenvalues
};

template <typename T>
struct PsdEngineIO {
    const ProjArgs<T> *a;
    T gamma, alpha;
    int base;              // global index of the block's first row
    T dd;
    __device__ T in(int64_t s) const {
        const int idx = base + static_cast<int>(s);
        return relaxed(*a, idx, gamma, alpha) - a->v[idx];
    }
    __device__ void out(int64_t s, T up) {
        const int idx = base + static_cast<int>(s);
        const T uo = a->u[idx], vo = a->v[idx];
        const T t = relaxed(*a, idx, gamma, alpha) - vo;
        const T vn = up - t;
        a->u[idx] = up;
        a->v[idx] = vn;
        dd += (up - uo) * (up - uo) + (vn - vo) * (vn - vo);
    }
};

// kSm: X, V, W in shared memory (else X, W in P.work and V in place in P.V,
// with the blocked sweeps' subproblems in shared memory when they fit)
template <typename T, bool kSm>
__global__ void __launch_bounds__(kPsdThreads, 1) psd_project_kernel(ProjArgs<T> a, PsdDev<T> P, PsdStats st) {
    extern __shared__ __align__(16) unsigned char psd_smem[];
    const int b = blockIdx.x;
    const int n = P.ord[b];
    const int ne = psd_ne(n), ld = ne + 1;
    const PsdSmall<T> sm = psd_small_tables<T>(psd_smem, P.ne_max);
    T *keep = P.V + P.voff[b];
    T *X, *V, *W, *Wsub = nullptr;
    if constexpr (kSm) {
        X = reinterpret_cast<T *>(psd_smem + P.small_bytes);
        V = X + ne * ld;
        W = V + ne * ld;
    } else {
        X = P.work + (size_t)b * 2 * P.work_stride;
        W = X + P.work_stride;
        V = keep;
        // the blocked sweeps' subproblems on chip when they fit
        if (psd_sub_on_chip<T>(P.ne_max)) Wsub = reinterpret_cast<T *>(psd_smem + P.small_bytes);
    }
    PsdEngineIO<T> io{&a, static_cast<T>(a.S->gamma), static_cast<T>(a.S->relax), a.n + P.off[b], T(0)};
    psd_project_block<T>(io, n, X, V, W, keep, sm, st, P.fp64_cond, Wsub);
    const double dd = psd_block_sum(static_cast<double>(io.dd), sm.red);
    if (threadIdx.x == 0) P.dd[b] = dd;
}

// V <- I for every PSD block (cold start of the eigenvector warm start)
template <typename T>
__global__ void psd_identity_kernel(T *V, const int32_t *ord, const int64_t *voff, int npsd) {
    for (int b = blockIdx.x; b < npsd; b += gridDim.x) {
        const int ne = psd_ne(ord[b]), ld = ne + 1;
        T *M = V + voff[b];
        for (int e = threadIdx.x; e < ne * ld; e += blockDim.x) {
            const int i = e / ld, j = e - i * ld;
            M[e] = (i == j) ? T(1) : T(0);
        }
    }
}

// ---------------------------------------------------------------------------
// Termination (Sec. 3.5 with Sec. 5's scaled residuals), FP64 throughout.
//   KC1 rows of A  : a = A^ u_x + v_s;  ||D^-1 (a - tau b^)||, ||D^-1 a||, b^.u_y
//   KC2 rows of A^T: d = A^T u_y;  ||E^-1 (d + tau c^)||, ||E^-1 d||, c^.u_x
// The last CTA of KC2 evaluates the tests in the order optimality, primal
// infeasibility, dual infeasibility and writes S->status.
// ---------------------------------------------------------------------------
template <typename T>
struct EpiChkA {
    static constexpr int NV = 3;
    static constexpr int kSite = kSiteChkA;
    const T *u, *v;
    const double *b, *Dinv;     // 1 / D: no FP64 division per row
    double *ax;
    Scalars *S;
    int n, N;
    double tau;
    struct In { double vs, b, dinv, uy; };
    __device__ bool skip() const { return false; }
    __device__ void begin() { tau = static_cast<double>(u[N - 1]); }
    __device__ In load(int i) const {
        return In{static_cast<double>(v[n + i]), b[i], Dinv[i], static_cast<double>(u[n + i])};
    }
    __device__ void row(int i, double s, const In &in, double (&red)[NV]) {
        ax[i] = s;
        const double a = s + in.vs;
        const double pr = (a - tau * in.b) * in.dinv;
        const double ub = a * in.dinv;
        red[0] += pr * pr;
        red[1] += ub * ub;
        red[2] += in.b * in.uy;
    }
    __device__ void finish(const double (&t)[NV]) {
        S->pri2 = t[0];
        S->unb2 = t[1];
        S->bty = t[2];
    }
};

template <typename T>
struct EpiChkAt {
    static constexpr int NV = 3;
    static constexpr int kSite = kSiteChkAt;
    const T *u, *v;
    const double *c, *Einv;     // 1 / E
    Scalars *S;
    int N;
    double tau;
    struct In { double c, einv, ux; };
    __device__ bool skip() const { return false; }
    __device__ void begin() { tau = static_cast<double>(u[N - 1]); }
    __device__ In load(int j) const { return In{c[j], Einv[j], static_cast<double>(u[j])}; }
    __device__ void row(int j, double s, const In &in, double (&red)[NV]) {
        const double du = (s + tau * in.c) * in.einv;
        const double inf = s * in.einv;
        red[0] += du * du;
        red[1] += inf * inf;
        red[2] += in.c * in.ux;
    }
    __device__ void finish(const double (&t)[NV]) {
        S->dual2 = t[0];
        S->inf2 = t[1];
        S->ctx = t[2];
        const double tau_ = static_cast<double>(u[N - 1]), kappa = static_cast<double>(v[N - 1]);
        const double sg = S->sigma, rh = S->rho;
        S->tau = tau_;
        S->kappa = kappa;
        int status = 0;
        if (tau_ > 0.0) {
            const double pri = sqrt(S->pri2) / (tau_ * sg);
            const double dual = sqrt(t[0]) / (tau_ * rh);
            const double cx = t[2] / (tau_ * rh * sg);
            const double by = S->bty / (tau_ * rh * sg);
            const double gap = fabs(cx + by);
            S->res_pri = pri;
            S->res_dual = dual;
            S->gap = gap;
            S->pobj = cx;
            S->dobj = -by;
            if (pri <= S->eps_pri * (1.0 + S->nb) && dual <= S->eps_dual * (1.0 + S->nc) &&
                gap <= S->eps_gap * (1.0 + fabs(cx) + fabs(by)))
                status = 1;
        } else {
            S->res_pri = S->res_dual = S->gap = INFINITY;
            S->pobj = S->dobj = NAN;
        }
        if (!status && S->nb > 0.0 && S->bty < 0.0 &&
            sqrt(t[1]) <= (-S->bty / (sg * S->nb)) * S->eps_infeas)
            status = -1;
        if (!status && S->nc > 0.0 && t[2] < 0.0 &&
            sqrt(S->unb2) <= (-t[2] / (rh * S->nc)) * S->eps_unbdd)
            status = -2;
        if (!isfinite(tau_) || !isfinite(kappa) || !isfinite(S->pri2) || !isfinite(t[0]) ||
            !isfinite(S->unb2) || !isfinite(t[1]))
            status = -13;
        S->status = status;
    }
};

// Solution or certificate in the caller's units (Sec. 5 unscaling, Sec. 2.3 cases).
template <typename T>
__global__ void __launch_bounds__(kBlock) output_kernel(int n, int m, int status, const T *__restrict__ u,
                                                        const T *__restrict__ v, const double *__restrict__ D,
                                                        const double *__restrict__ E, const double *__restrict__ ax,
                                                        const Scalars *S, double *__restrict__ x,
                                                        double *__restrict__ y, double *__restrict__ s) {
    const int N = n + m + 1;
    const double tau = static_cast<double>(u[N - 1]);
    const double sg = S->sigma, rh = S->rho;
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < n + 2 * m; i += gridDim.x * kBlock) {
        if (status == 1 || status == 2) {
            if (i < n) x[i] = E[i] * u[i] / (tau * sg);
            else if (i < n + m) y[i - n] = D[i - n] * u[i] / (tau * rh);
            else s[i - n - m] = v[i - m] / (D[i - n - m] * tau * sg);
        } else if (status == -1 || status == -3) {
            const double f = sg / (-S->bty);       // b^T (D u_y) = b^.u_y / sigma
            if (i < n) x[i] = NAN;
            else if (i < n + m) y[i - n] = D[i - n] * u[i] * f;
            else s[i - n - m] = NAN;
        } else if (status == -2 || status == -4) {
            const double f = rh / (-S->ctx);       // c^T (E u_x) = c^.u_x / rho
            if (i < n) x[i] = E[i] * u[i] * f;
            else if (i < n + m) y[i - n] = NAN;
            else s[i - n - m] = -ax[i - n - m] * f / D[i - n - m];   // s = -A x
        } else {
            if (i < n) x[i] = NAN;
            else if (i < n + m) y[i - n] = NAN;
            else s[i - n - m] = NAN;
        }
    }
}

// ---------------------------------------------------------------------------
// setup kernels (FP64): equilibration (Sec. 5) and conversions
// ---------------------------------------------------------------------------
// Rows of a CSR matrix gathered into its stored layout: stored row w is
// source row rowid[w] (one warp per row, lanes stride the row).
static __global__ void gather_rows_kernel(int rows, const int32_t *__restrict__ rowid,
                                          const int32_t *__restrict__ src_rp, const int32_t *__restrict__ src_col,
                                          const double *__restrict__ src_val, const int32_t *__restrict__ dst_rp,
                                          int32_t *__restrict__ dst_col, double *__restrict__ dst_val) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
    for (int64_t w = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; w < rows; w += warps) {
        const int r = rowid[w];
        const int s0 = src_rp[r], len = src_rp[r + 1] - s0, d0 = dst_rp[w];
        for (int k = lane; k < len; k += 32) {
            dst_col[d0 + k] = src_col[s0 + k];
            dst_val[d0 + k] = src_val[s0 + k];
        }
    }
}

static __global__ void row_sumsq_kernel(const int32_t *__restrict__ rowptr, const double *__restrict__ val,
                                        const int32_t *__restrict__ rowid, int rows, double *__restrict__ out) {
    const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * kBlock) >> 5;
    for (int r = warp; r < rows; r += nw) {
        double s = 0.0;
        for (int k = rowptr[r] + lane; k < rowptr[r + 1]; k += 32) s += val[k] * val[k];
        s = warp_sum(s);
        if (lane == 0) out[rowid[r]] = s;
    }
}

static __global__ void scale_vals_kernel(const int32_t *__restrict__ rowptr, const int32_t *__restrict__ col,
                                         double *__restrict__ val, const int32_t *__restrict__ rowid, int rows,
                                         const double *__restrict__ drow, const double *__restrict__ ecol) {
    const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * kBlock) >> 5;
    for (int r = warp; r < rows; r += nw) {
        const double d = drow[rowid[r]];
        for (int k = rowptr[r] + lane; k < rowptr[r + 1]; k += 32) val[k] *= d * ecol[col[k]];
    }
}

static __global__ void sqrt_kernel(double *__restrict__ nrm, int len) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < len; i += gridDim.x * kBlock) nrm[i] = sqrt(nrm[i]);
}

// over each cone block that D must keep scalar: replace the norms by one
// value for the block (mode 0: mean, 1: root mean square, 2: maximum)
static __global__ void block_mean_kernel(double *__restrict__ nrm, const int32_t *__restrict__ bo,
                                         const int32_t *__restrict__ bl, int nblocks, int mode) {
    const int warp = (blockIdx.x * kBlock + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int nw = (gridDim.x * kBlock) >> 5;
    for (int b = warp; b < nblocks; b += nw) {
        double s = 0.0, mx = 0.0;
        for (int i = lane; i < bl[b]; i += 32) {
            const double t = nrm[bo[b] + i];
            s += mode == 1 ? t * t : t;
            mx = fmax(mx, t);
        }
        s = warp_sum(s);
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        const double val = mode == 2 ? mx : mode == 1 ? sqrt(s / bl[b]) : s / bl[b];
        for (int i = lane; i < bl[b]; i += 32) nrm[bo[b] + i] = val;
    }
}

// d = 1 / sqrt(clamp(norm)); acc *= d
static __global__ void inv_sqrt_clamp_kernel(const double *__restrict__ nrm, int len, double lo, double hi,
                                      double *__restrict__ d, double *__restrict__ acc) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < len; i += gridDim.x * kBlock) {
        double t = nrm[i];
        if (t < lo) t = 1.0;
        if (t > hi) t = hi;
        const double s = 1.0 / sqrt(t);
        d[i] = s;
        acc[i] *= s;
    }
}

template <typename F>
__global__ void __launch_bounds__(kBlock) reduce_kernel(F f, int len, ReduceBuf rb, double *out) {
    double red[1] = {0.0};
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < len; i += gridDim.x * kBlock) red[0] += f(i);
    double tot[1];
    if (grid_sum<1>(red, rb, kSiteMisc, tot)) {
        if (threadIdx.x == 0) *out = tot[0];
    }
}

template <typename F>
__global__ void __launch_bounds__(kBlock) foreach_kernel(F f, int len) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < len; i += gridDim.x * kBlock) f(i);
}

}  // namespace scs
