// Batched persistent solver: many independent small cone programs (zero,
// nonnegative and second-order cones) solved by the same iteration as the
// single-problem engine (Eq. "e-SCS" with relaxation, indirect subspace
// projection by warm-started Jacobi PCG, Sec. 4.1; equilibration, Sec. 5;
// termination, Sec. 3.5) inside ONE persistent kernel launch.
//
// Work split: a CTA is a team that owns one program at a time; it takes the
// next program from an atomic queue ordered by decreasing size (largest
// first), keeps the program's iterates u, v and all CG vectors in shared
// memory for the whole solve, and reads the program's scaled CSR of A and
// of A^T from global memory (a few hundred KB at most, so it stays in L1/L2
// while the team works on it).  Inside a team, the rows of each product are
// split by length: rows longer than `row_split` nonzeros are summed by a
// warp each (lanes stride the row), the others by one thread each; rows are
// stored longest first so the split is a prefix.  A team reduction is a
// warp shuffle, one shared-memory exchange and one barrier.
//
// The host autotuner (BatchEngine::tune) times the team size (64, 128, 256
// or 512 threads) and the row split on a sample of programs that keeps every
// resident team busy and keeps the fastest.  Setup (equilibration in FP64, Jacobi diagonal, cached
// p = M^-1 h) is a second persistent launch run once by scs_batch_init; each
// solve is a CUDA graph of a queue reset and the solve launch.
//
// Precision: T (float or double) holds A^, the iterates and CG vectors;
// per-thread sums are in T, team sums in FP64; the termination tests
// accumulate in FP64 with the T copy of A^; the scaling is FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/scs_gpu.h"
#include "common.cuh"
#include "engine_base.h"
#include "host_par.h"

namespace scs {
namespace batch {

constexpr int kMaxNV = 8;   // values per team reduction

// Per-program layout (offsets into the concatenated device arrays).
struct Meta {
    int n, m, z, l, nq;
    int soc0;              // first entry of the program in the SOC tables
    int a_row0, a_nlong;   // rows of A^ at [a_row0, a_row0 + m) of the row arrays; the first a_nlong are long
    int at_row0, at_nlong; // rows of A^T likewise (n rows)
    int xo, yo, uo;        // offsets of its n-, m- and (n + m + 1)-vectors
};

template <typename T>
struct Dev {
    int count;
    const Meta *meta;
    const int32_t *order;         // programs in queue order
    int norder;
    const int32_t *soc_off, *soc_len;   // SOC block row offsets (within y) and sizes
    // A^ and A^T (rows longest first; rowid maps a stored row to its index)
    const int32_t *a_rp, *a_rid, *a_col;
    const int32_t *at_rp, *at_rid, *at_col;
    T *a_val, *at_val;            // scaled values (written by the setup)
    const double *a_v64, *at_v64; // the caller's values
    // data, scaling, cached quantities
    const double *b, *c;          // the caller's b (sum m), c (sum n)
    double *D, *E;                // equilibration
    double *b64, *c64;            // b^, c^ in FP64 (checks)
    T *bh, *ch;                   // b^, c^ in T
    T *dg;                        // 1 + ||col_j(A^)||^2
    T *pM;                        // p = M^-1 h (n + m per program)
    double *sigma, *rho, *hp1, *nb, *nc;
    // iteration state
    T *u, *v, *zcg;               // iterates and the CG warm-start vector
    int32_t *k, *warm;
    double *dstep;
    // outputs
    double *ax;                   // A^ u_x of the last check (certificates)
    double *x, *y, *s;
    scs_info *info;
    int *queue;                   // [0]: next queue position
    // settings
    double alpha, eps_pri, eps_dual, eps_gap, eps_infeas, eps_unbdd, cg_rate, cg_adapt, cg_tol_rel;
    int max_iters, check_interval, cg_max, normalize, passes, block_scale;
};

// ---------------------------------------------------------------------------
// team utilities
// ---------------------------------------------------------------------------
template <int NT>
struct Team {
    double *red;   // 2 x kMaxNV x NT/32 doubles
    int parity;
    // sum NV values over the team; the totals are valid in every thread.
    // Two alternating exchange buffers make one barrier per call enough.
    template <int NV>
    __device__ __forceinline__ void sum(double (&v)[NV]) {
        constexpr int NW = NT / 32;
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
        double *buf = red + parity * (kMaxNV * NW);
        parity ^= 1;
        if (lane == 0) {
#pragma unroll
            for (int i = 0; i < NV; ++i) buf[i * NW + w] = v[i];
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            double t = 0.0;
#pragma unroll
            for (int k = 0; k < NW; ++k) t += buf[i * NW + k];
            v[i] = t;
        }
    }
};

// rows [row0, row0 + rows) of a stored CSR, the first nlong by warps:
// epi(original row, sum).  The values are read with plain loads (the setup
// launch reads values it wrote itself; the structure arrays never change).
template <int NT, typename Acc, typename TV, typename TX, typename Epi>
__device__ __forceinline__ void team_spmv(const int32_t *__restrict__ rp, const int32_t *__restrict__ rid,
                                          const int32_t *__restrict__ col, const TV *val, int row0,
                                          int rows, int nlong, const TX *x, Epi epi) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int r = w; r < nlong; r += NW) {
        const int k0 = __ldg(rp + row0 + r), k1 = __ldg(rp + row0 + r + 1);
        Acc s = Acc(0);
        for (int k = k0 + lane; k < k1; k += 32) s += static_cast<Acc>(val[k]) * static_cast<Acc>(x[__ldg(col + k)]);
        s = warp_sum(s);
        if (lane == 0) epi(__ldg(rid + row0 + r), s);
    }
    for (int r = nlong + threadIdx.x; r < rows; r += NT) {
        const int k0 = __ldg(rp + row0 + r), k1 = __ldg(rp + row0 + r + 1);
        Acc s = Acc(0);
        for (int k = k0; k < k1; ++k) s += static_cast<Acc>(val[k]) * static_cast<Acc>(x[__ldg(col + k)]);
        epi(__ldg(rid + row0 + r), s);
    }
}

// same rows, sum of (val * f(col))^2 over the row with FP64 values (setup)
template <int NT, typename F, typename Epi>
__device__ __forceinline__ void team_rownorm(const int32_t *__restrict__ rp, const int32_t *__restrict__ rid,
                                             const int32_t *__restrict__ col, const double *__restrict__ val,
                                             int row0, int rows, int nlong, F f, Epi epi) {
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int r = w; r < nlong; r += NW) {
        const int k0 = rp[row0 + r], k1 = rp[row0 + r + 1];
        double s = 0.0;
        for (int k = k0 + lane; k < k1; k += 32) {
            const double t = val[k] * f(col[k]);
            s += t * t;
        }
        s = warp_sum(s);
        if (lane == 0) epi(rid[row0 + r], s);
    }
    for (int r = nlong + threadIdx.x; r < rows; r += NT) {
        const int k0 = rp[row0 + r], k1 = rp[row0 + r + 1];
        double s = 0.0;
        for (int k = k0; k < k1; ++k) {
            const double t = val[k] * f(col[k]);
            s += t * t;
        }
        epi(rid[row0 + r], s);
    }
}

// shared-memory bytes of one team: T vectors of the solve, or FP64 scaling
// vectors plus T vectors of the setup, whichever is larger, and the
// exchange buffers
template <typename T>
__host__ __device__ inline size_t team_bytes(int n, int m) {
    const size_t N = (size_t)n + m + 1;
    const size_t solve = sizeof(T) * (2 * N + 6 * (size_t)n + 5 * (size_t)m);
    const size_t setup = sizeof(double) * 2 * ((size_t)n + m) + sizeof(T) * (5 * (size_t)n + 3 * (size_t)m);
    size_t b = solve > setup ? solve : setup;
    return (b + 15) & ~size_t(15);
}

// take the next queue position (one atomic per team, broadcast)
__device__ __forceinline__ int next_job(int *queue, int *slot) {
    __syncthreads();
    if (threadIdx.x == 0) *slot = atomicAdd(queue, 1);
    __syncthreads();
    return *slot;
}

// ---------------------------------------------------------------------------
// one program's CG on (I + A^T A) z = r_x - A^T r_y, warm-started from z,
// the subspace step of Sec. 4.1.  On entry ya = r_y + A z and r, p, rz, rr,
// pp are those of the starting point; ya is kept equal to r_y + A z, and az
// (when given) equal to A z.
// ---------------------------------------------------------------------------
template <typename T, int NT>
__device__ __forceinline__ int team_cg(const Dev<T> &B, const Meta &M, Team<NT> &tm, T *z, T *r, T *p, T *q, T *ya,
                                       T *az, const T *dg, double rz, double rr, double pp, double tol, int cg_max) {
    const int n = M.n, m = M.m;
    int it = 0;
    bool done = !(sqrt(rr) > tol) || cg_max <= 0;
    while (!done) {
        double r3[1] = {0.0};
        team_spmv<NT, T>(B.a_rp, B.a_rid, B.a_col, B.a_val, M.a_row0, m, M.a_nlong, p, [&](int i, T s) {
            q[i] = s;
            r3[0] += static_cast<double>(s * s);
        });
        tm.sum(r3);
        const T a = static_cast<T>(rz / (pp + r3[0]));
        double r4[2] = {0.0, 0.0};
        T acc0 = T(0), acc1 = T(0);
        team_spmv<NT, T>(B.at_rp, B.at_rid, B.at_col, B.at_val, M.at_row0, n, M.at_nlong, q, [&](int j, T s) {
            const T pj = p[j];
            z[j] += a * pj;
            const T rj = r[j] - a * (pj + s);
            r[j] = rj;
            acc0 += rj * (rj / dg[j]);
            acc1 += rj * rj;
        });
        for (int i = threadIdx.x; i < m; i += NT) ya[i] += a * q[i];
        if (az)
            for (int i = threadIdx.x; i < m; i += NT) az[i] += a * q[i];
        r4[0] = static_cast<double>(acc0);
        r4[1] = static_cast<double>(acc1);
        tm.sum(r4);
        ++it;
        done = !(sqrt(r4[1]) > tol) || it >= cg_max;
        const T beta = static_cast<T>(r4[0] / rz);
        rz = r4[0];
        if (!done) {
            T acc = T(0);
            for (int j = threadIdx.x; j < n; j += NT) {
                const T pj = r[j] / dg[j] + beta * p[j];
                p[j] = pj;
                acc += pj * pj;
            }
            double r5[1] = {static_cast<double>(acc)};
            tm.sum(r5);
            pp = r5[0];
        }
    }
    return it;
}

// ---------------------------------------------------------------------------
// setup of one program: Sec. 5 equilibration (FP64), b^, c^, A^ in T, the
// Jacobi diagonal, and p = M^-1 h by a tight CG
// ---------------------------------------------------------------------------
template <typename T, int NT>
__device__ __forceinline__ void setup_program(const Dev<T> &B, int id, unsigned char *smem, Team<NT> &tm) {
    const Meta M = B.meta[id];
    const int n = M.n, m = M.m;
    double *Dd = reinterpret_cast<double *>(smem);
    double *Ee = Dd + m;
    T *tz = reinterpret_cast<T *>(Ee + n);
    T *tr = tz + n, *tp = tr + n, *tdg = tp + n, *tq = tdg + n, *tya = tq + m, *tbh = tya + m;
    T *tch = tbh + m;
    for (int i = threadIdx.x; i < m; i += NT) Dd[i] = 1.0;
    for (int j = threadIdx.x; j < n; j += NT) Ee[j] = 1.0;
    __syncthreads();
    // row and column norms of a pass: the program's m (n) doubles of the
    // global ax (x) output arrays serve as scratch until the solve
    double *rn = B.ax + M.yo;
    double *cn = B.x + M.xo;
    if (B.normalize) {
        for (int pass = 0; pass < B.passes; ++pass) {
            team_rownorm<NT>(B.a_rp, B.a_rid, B.a_col, B.a_v64, M.a_row0, m, M.a_nlong,
                             [&](int j) { return Ee[j]; }, [&](int i, double s) { rn[i] = Dd[i] * sqrt(s); });
            team_rownorm<NT>(B.at_rp, B.at_rid, B.at_col, B.at_v64, M.at_row0, n, M.at_nlong,
                             [&](int i) { return Dd[i]; }, [&](int j, double s) { cn[j] = Ee[j] * sqrt(s); });
            __syncthreads();
            // one value per SOC block (mean, RMS or max of its row norms)
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            for (int bq = w; bq < M.nq; bq += NT / 32) {
                const int off = B.soc_off[M.soc0 + bq], len = B.soc_len[M.soc0 + bq];
                double sm_ = 0.0, mx = 0.0;
                for (int e = lane; e < len; e += 32) {
                    const double t = rn[off + e];
                    sm_ += B.block_scale == 1 ? t * t : t;
                    mx = fmax(mx, t);
                }
                sm_ = warp_sum(sm_);
                for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                const double val = B.block_scale == 2 ? mx : B.block_scale == 1 ? sqrt(sm_ / len) : sm_ / len;
                __syncwarp();
                for (int e = lane; e < len; e += 32) rn[off + e] = val;
            }
            __syncthreads();
            for (int i = threadIdx.x; i < m; i += NT) {
                double t = rn[i];
                if (t < 1e-4) t = 1.0;
                if (t > 1e4) t = 1e4;
                Dd[i] *= 1.0 / sqrt(t);
            }
            for (int j = threadIdx.x; j < n; j += NT) {
                double t = cn[j];
                if (t < 1e-4) t = 1.0;
                if (t > 1e4) t = 1e4;
                Ee[j] *= 1.0 / sqrt(t);
            }
            __syncthreads();
        }
    }
    // sigma = 1 / max(||D b||, 1e-4); rho = mean_i ||row_i(A^)|| / max(||E c||, 1e-4)
    double r0[3] = {0.0, 0.0, 0.0};
    double racc = 0.0;
    team_rownorm<NT>(B.a_rp, B.a_rid, B.a_col, B.a_v64, M.a_row0, m, M.a_nlong, [&](int j) { return Ee[j]; },
                     [&](int i, double s) { racc += Dd[i] * sqrt(s); });
    r0[0] = racc;
    for (int i = threadIdx.x; i < m; i += NT) {
        const double t = Dd[i] * B.b[M.yo + i];
        r0[1] += t * t;
    }
    for (int j = threadIdx.x; j < n; j += NT) {
        const double t = Ee[j] * B.c[M.xo + j];
        r0[2] += t * t;
    }
    tm.sum(r0);
    double sg = 1.0, rh = 1.0;
    if (B.normalize) {
        double mean_row = m ? r0[0] / m : 1.0;
        if (!(mean_row > 0.0)) mean_row = 1.0;
        sg = 1.0 / fmax(sqrt(r0[1]), 1e-4);
        rh = mean_row / fmax(sqrt(r0[2]), 1e-4);
    }
    double nbc[2] = {0.0, 0.0};
    for (int i = threadIdx.x; i < m; i += NT) {
        const double bi = B.b[M.yo + i];
        nbc[0] += bi * bi;
        const double bs = sg * Dd[i] * bi;
        B.D[M.yo + i] = Dd[i];
        B.b64[M.yo + i] = bs;
        B.bh[M.yo + i] = static_cast<T>(bs);
        tbh[i] = static_cast<T>(bs);
    }
    for (int j = threadIdx.x; j < n; j += NT) {
        const double cj = B.c[M.xo + j];
        nbc[1] += cj * cj;
        const double cs = rh * Ee[j] * cj;
        B.E[M.xo + j] = Ee[j];
        B.c64[M.xo + j] = cs;
        B.ch[M.xo + j] = static_cast<T>(cs);
        tch[j] = static_cast<T>(cs);
    }
    tm.sum(nbc);
    if (threadIdx.x == 0) {
        B.sigma[id] = sg;
        B.rho[id] = rh;
        B.nb[id] = sqrt(nbc[0]);
        B.nc[id] = sqrt(nbc[1]);
    }
    // A^ = D A E in T, both layouts; diag = 1 + ||col_j(A^)||^2
    {
        // threads stride the program's nonzeros; the stored row of nonzero kk
        // comes from a binary search in the program's row pointers
        const int k0 = B.a_rp[M.a_row0], k1 = B.a_rp[M.a_row0 + m];
        for (int kk = k0 + threadIdx.x; kk < k1; kk += NT) {
            int lo = 0, hi = m;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (B.a_rp[M.a_row0 + mid] <= kk) lo = mid; else hi = mid;
            }
            const int i = B.a_rid[M.a_row0 + lo];
            B.a_val[kk] = static_cast<T>(Dd[i] * B.a_v64[kk] * Ee[B.a_col[kk]]);
        }
        const int t0 = B.at_rp[M.at_row0], t1 = B.at_rp[M.at_row0 + n];
        for (int kk = t0 + threadIdx.x; kk < t1; kk += NT) {
            int lo = 0, hi = n;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (B.at_rp[M.at_row0 + mid] <= kk) lo = mid; else hi = mid;
            }
            const int j = B.at_rid[M.at_row0 + lo];
            B.at_val[kk] = static_cast<T>(Ee[j] * B.at_v64[kk] * Dd[B.at_col[kk]]);
        }
    }
    team_rownorm<NT>(B.at_rp, B.at_rid, B.at_col, B.at_v64, M.at_row0, n, M.at_nlong, [&](int i) { return Dd[i]; },
                     [&](int j, double s) {
                         const T d = static_cast<T>(1.0 + Ee[j] * Ee[j] * s);
                         B.dg[M.xo + j] = d;
                         tdg[j] = d;
                     });
    __threadfence_block();
    __syncthreads();     // A^ values (global) and the T copies written by the whole team
    // p = M^-1 h: u = (c^, b^, 0), v = 0, z = 0:  ya = b^,  r = c^ - A^T b^
    for (int j = threadIdx.x; j < n; j += NT) tz[j] = T(0);
    for (int i = threadIdx.x; i < m; i += NT) tya[i] = tbh[i];
    __syncthreads();
    double r2[4] = {0.0, 0.0, 0.0, 0.0};
    {
        T a0 = T(0), a1 = T(0), a2 = T(0);
        team_spmv<NT, T>(B.at_rp, B.at_rid, B.at_col, B.at_val, M.at_row0, n, M.at_nlong, tya, [&](int j, T s) {
            const T rj = tch[j] - s;
            const T sj = rj / tdg[j];
            tr[j] = rj;
            tp[j] = sj;
            a0 += rj * sj;
            a1 += rj * rj;
            a2 += sj * sj;
        });
        T ww = T(0);
        for (int j = threadIdx.x; j < n; j += NT) ww += tch[j] * tch[j];
        for (int i = threadIdx.x; i < m; i += NT) ww += tbh[i] * tbh[i];
        r2[0] = a0;
        r2[1] = a1;
        r2[2] = a2;
        r2[3] = ww;
    }
    tm.sum(r2);
    const double tol = (sizeof(T) == 8 ? 1e-14 : 1e-7) * sqrt(r2[3]);
    const int cap = B.cg_max * 10 > 500 ? B.cg_max * 10 : 500;
    team_cg<T, NT>(B, M, tm, tz, tr, tp, tq, tya, nullptr, tdg, r2[0], r2[1], r2[2], tol, cap);
    double hp[1] = {0.0};
    for (int j = threadIdx.x; j < n; j += NT) {
        B.pM[M.xo + M.yo + j] = tz[j];
        hp[0] += B.c64[M.xo + j] * static_cast<double>(tz[j]);
    }
    for (int i = threadIdx.x; i < m; i += NT) {
        B.pM[M.xo + M.yo + n + i] = tya[i];
        hp[0] += B.b64[M.yo + i] * static_cast<double>(tya[i]);
    }
    tm.sum(hp);
    if (threadIdx.x == 0) B.hp1[id] = 1.0 + hp[0];
}

template <typename T, int NT>
__global__ void __launch_bounds__(NT) setup_kernel(Dev<T> B) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[2 * kMaxNV * (NT / 32)];
    __shared__ int slot;
    Team<NT> tm{red, 0};
    for (;;) {
        const int pos = next_job(B.queue, &slot);
        if (pos >= B.norder) break;
        setup_program<T, NT>(B, B.order[pos], smem, tm);
    }
}

// ---------------------------------------------------------------------------
// solve of one program: iterations from the stored state (cold or warm),
// termination tests every check_interval iterations (mode 0), or exactly
// `iters` iterations without tests (mode 1)
// ---------------------------------------------------------------------------
// last[]: the latest test's values (team-wide; written by thread 0)
//   0 pri2  1 unb2  2 b^.u_y  3 dual2  4 inf2  5 c^.u_x  6 tau  7 kappa
//   8 res_pri  9 res_dual  10 gap  11 pobj  12 dobj
template <typename T, int NT>
__device__ __forceinline__ void solve_program(const Dev<T> &B, int id, unsigned char *smem, Team<NT> &tm, int mode, int iters,
                              double *last) {
    const Meta M = B.meta[id];
    const int n = M.n, m = M.m, N = n + m + 1;
    T *u = reinterpret_cast<T *>(smem);
    T *v = u + N, *z = v + N, *r = z + n, *p = r + n, *dg = p + n, *ch = dg + n, *px = ch + n;
    T *q = px + n, *ya = q + m, *bh = ya + m, *py = bh + m, *az = py + m;
    const T *pMg = B.pM + M.xo + M.yo;
    // state
    const bool cold = mode == 0 && !B.warm[id];
    for (int i = threadIdx.x; i < N; i += NT) {
        if (cold) {
            u[i] = i == N - 1 ? T(1) : T(0);
            v[i] = i == N - 1 ? T(1) : T(0);
        } else {
            u[i] = B.u[M.uo + i];
            v[i] = B.v[M.uo + i];
        }
    }
    for (int j = threadIdx.x; j < n; j += NT) {
        z[j] = cold ? T(0) : B.zcg[M.xo + j];
        dg[j] = B.dg[M.xo + j];
        ch[j] = B.ch[M.xo + j];
        px[j] = pMg[j];
    }
    for (int i = threadIdx.x; i < m; i += NT) {
        bh[i] = B.bh[M.yo + i];
        py[i] = pMg[n + i];
    }
    int k = cold ? 0 : B.k[id];
    double dstep = cold ? INFINITY : B.dstep[id];
    const double hp1 = B.hp1[id], sg = B.sigma[id], rh = B.rho[id], nbv = B.nb[id], ncv = B.nc[id];
    const T al = static_cast<T>(B.alpha);
    int status = 0, it = 0;
    int cg_total = 0;
    if (threadIdx.x < 13) last[threadIdx.x] = NAN;
    __syncthreads();
    const int cap = mode == 1 ? iters : B.max_iters;
    while (it < cap) {
        // ---- K1: ya = r_y + A^ z  (r_y = u_y + v_s - w_tau b^); the product
        //      A^ z on iterations k = 0 mod kAzEvery and on the first of the
        //      call (az is not kept between calls), the carried az = A^ z on
        //      the others
        const double wtau = static_cast<double>(u[N - 1]) + static_cast<double>(v[N - 1]);
        const T wt = static_cast<T>(wtau);
        T acc_wy = T(0);
        if (it == 0 || k % kAzEvery == 0) {
            team_spmv<NT, T>(B.a_rp, B.a_rid, B.a_col, B.a_val, M.a_row0, m, M.a_nlong, z, [&](int i, T s) {
                const T w = u[n + i] + v[n + i];
                ya[i] = w - wt * bh[i] + s;
                az[i] = s;
                acc_wy += w * w;
            });
        } else {
            for (int i = threadIdx.x; i < m; i += NT) {
                const T w = u[n + i] + v[n + i];
                ya[i] = w - wt * bh[i] + az[i];
                acc_wy += w * w;
            }
        }
        __syncthreads();
        // ---- K2: r = r_x - z - A^T ya, p = r / diag
        T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
        team_spmv<NT, T>(B.at_rp, B.at_rid, B.at_col, B.at_val, M.at_row0, n, M.at_nlong, ya, [&](int j, T s) {
            const T ux = u[j];
            const T rj = ux - wt * ch[j] - z[j] - s;
            const T sj = rj / dg[j];
            r[j] = rj;
            p[j] = sj;
            a0 += rj * sj;
            a1 += rj * rj;
            a2 += sj * sj;
            a3 += ux * ux;
        });
        double r2[5] = {static_cast<double>(a0), static_cast<double>(a1), static_cast<double>(a2),
                        static_cast<double>(a3), static_cast<double>(acc_wy)};
        tm.sum(r2);
        const double ww = r2[3] + r2[4] + wtau * wtau;
        double tol = INFINITY;
        if (B.cg_rate > 0.0) tol = pow(1.0 / (double)(k + 1), B.cg_rate);
        if (B.cg_adapt > 0.0) tol = fmin(tol, B.cg_adapt * dstep);
        if (!isfinite(tol)) tol = 0.0;
        tol = fmax(tol, B.cg_tol_rel * sqrt(ww));
        cg_total += team_cg<T, NT>(B, M, tm, z, r, p, q, ya, az, dg, r2[0], r2[1], r2[2], tol, B.cg_max);
        // ---- K6: gamma = h^T z / (1 + h^T p)
        T ag = T(0);
        for (int j = threadIdx.x; j < n; j += NT) ag += ch[j] * z[j];
        for (int i = threadIdx.x; i < m; i += NT) ag += bh[i] * ya[i];
        double r6[1] = {static_cast<double>(ag)};
        tm.sum(r6);
        const double gamma = r6[0] / hp1;
        const T g = static_cast<T>(gamma);
        // ---- K7: relax, project onto C = R^n x K* x R+, dual update
        T dd = T(0);
        const int nlin = n + M.z + M.l;
        for (int i = threadIdx.x; i < nlin; i += NT) {
            const T zi = i < n ? z[i] : ya[i - n];
            const T pi = i < n ? px[i] : py[i - n];
            const T uo = u[i];
            const T ub = al * (zi - pi * g) + (T(1) - al) * uo;
            if (i < n) {
                u[i] = ub;
                dd += (ub - uo) * (ub - uo);
            } else {
                const T vo = v[i];
                const T t = ub - vo;
                const T up = (i < n + M.z) ? t : (t > T(0) ? t : T(0));
                u[i] = up;
                v[i] = up - t;
                dd += (up - uo) * (up - uo) + (up - t - vo) * (up - t - vo);
            }
        }
        {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            for (int bq = w; bq < M.nq; bq += NT / 32) {
                const int off = n + B.soc_off[M.soc0 + bq], len = B.soc_len[M.soc0 + bq];
                T t0 = T(0), xx = T(0);
                for (int e = lane; e < len; e += 32) {
                    const int i = off + e;
                    const T t = al * (ya[i - n] - py[i - n] * g) + (T(1) - al) * u[i] - v[i];
                    if (e == 0) t0 = t; else xx += t * t;
                }
                xx = warp_sum(xx);
                t0 = __shfl_sync(0xffffffffu, t0, 0);
                const T nx = sqrt(xx);
                T head, tail;
                if (nx <= t0) { head = t0; tail = T(1); }
                else if (nx <= -t0) { head = T(0); tail = T(0); }
                else { head = T(0.5) * (t0 + nx); tail = head / nx; }
                for (int e = lane; e < len; e += 32) {
                    const int i = off + e;
                    const T uo = u[i], vo = v[i];
                    const T t = al * (ya[i - n] - py[i - n] * g) + (T(1) - al) * uo - vo;
                    const T up = e == 0 ? head : tail * t;
                    u[i] = up;
                    v[i] = up - t;
                    dd += (up - uo) * (up - uo) + (up - t - vo) * (up - t - vo);
                }
            }
        }
        double r7[2] = {static_cast<double>(dd), 0.0};
        if (threadIdx.x == 0) {
            // tau (FP64): u~_tau = w_tau + gamma
            const double uo = static_cast<double>(u[N - 1]), vo = static_cast<double>(v[N - 1]);
            const double ub = B.alpha * (wtau + gamma) + (1.0 - B.alpha) * uo;
            const double t = ub - vo;
            const double up = fmax(t, 0.0);
            u[N - 1] = static_cast<T>(up);
            v[N - 1] = static_cast<T>(up - t);
            r7[1] = (up - uo) * (up - uo) + (up - t - vo) * (up - t - vo);
        }
        tm.sum(r7);
        dstep = sqrt(r7[0] + r7[1]);
        ++k;
        ++it;
        // ---- Sec. 3.5 tests (FP64 accumulation) every check_interval
        if (mode == 0 && (it % (B.check_interval > 0 ? B.check_interval : 1) == 0 || it >= cap)) {
            const double tau = static_cast<double>(u[N - 1]);
            double c8[6] = {0, 0, 0, 0, 0, 0};
            team_spmv<NT, double>(B.a_rp, B.a_rid, B.a_col, B.a_val, M.a_row0, m, M.a_nlong, u, [&](int i, double s) {
                B.ax[M.yo + i] = s;
                const double a = s + static_cast<double>(v[n + i]);
                const double bb = B.b64[M.yo + i], dd_ = B.D[M.yo + i];
                const double pr = (a - tau * bb) / dd_;
                const double ub = a / dd_;
                c8[0] += pr * pr;
                c8[1] += ub * ub;
                c8[2] += bb * static_cast<double>(u[n + i]);
            });
            team_spmv<NT, double>(B.at_rp, B.at_rid, B.at_col, B.at_val, M.at_row0, n, M.at_nlong, u + n,
                                  [&](int j, double s) {
                                      const double cc = B.c64[M.xo + j], ee = B.E[M.xo + j];
                                      const double du = (s + tau * cc) / ee;
                                      const double inf = s / ee;
                                      c8[3] += du * du;
                                      c8[4] += inf * inf;
                                      c8[5] += cc * static_cast<double>(u[j]);
                                  });
            tm.sum(c8);
            const double kappa = static_cast<double>(v[N - 1]);
            int st = 0;
            double pri = INFINITY, dual = INFINITY, gap = INFINITY, cx = NAN, by = NAN;
            if (tau > 0.0) {
                pri = sqrt(c8[0]) / (tau * sg);
                dual = sqrt(c8[3]) / (tau * rh);
                cx = c8[5] / (tau * rh * sg);
                by = c8[2] / (tau * rh * sg);
                gap = fabs(cx + by);
                if (pri <= B.eps_pri * (1.0 + nbv) && dual <= B.eps_dual * (1.0 + ncv) &&
                    gap <= B.eps_gap * (1.0 + fabs(cx) + fabs(by)))
                    st = 1;
            }
            if (threadIdx.x == 0) {
#pragma unroll
                for (int e = 0; e < 6; ++e) last[e] = c8[e];
                last[6] = tau;
                last[7] = kappa;
                last[8] = pri;
                last[9] = dual;
                last[10] = gap;
                last[11] = cx;
                last[12] = -by;
            }
            if (!st && nbv > 0.0 && c8[2] < 0.0 && sqrt(c8[4]) <= (-c8[2] / (sg * nbv)) * B.eps_infeas) st = -1;
            if (!st && ncv > 0.0 && c8[5] < 0.0 && sqrt(c8[1]) <= (-c8[5] / (rh * ncv)) * B.eps_unbdd) st = -2;
            if (!isfinite(tau) || !isfinite(kappa) || !isfinite(c8[0]) || !isfinite(c8[3]) || !isfinite(c8[1]) ||
                !isfinite(c8[4]))
                st = -13;
            status = st;
            if (status != 0) break;
        }
    }
    __syncthreads();
    // ---- store the state
    for (int i = threadIdx.x; i < N; i += NT) {
        B.u[M.uo + i] = u[i];
        B.v[M.uo + i] = v[i];
    }
    for (int j = threadIdx.x; j < n; j += NT) B.zcg[M.xo + j] = z[j];
    if (threadIdx.x == 0) {
        B.k[id] = k;
        B.dstep[id] = dstep;
        B.warm[id] = 0;
    }
    if (mode == 1) return;
    // ---- inaccurate status at the iteration limit (from the last test)
    if (status == 0) {
        const double tau = last[6], kappa = last[7], bty = last[2], ctx = last[5];
        if (!isfinite(tau) || !isfinite(kappa)) status = SCS_NUMERICAL;
        else if (tau > 0 && tau >= kappa) status = SCS_SOLVED_INACCURATE;
        else if (bty < 0 && bty <= ctx) status = SCS_INFEASIBLE_INACCURATE;
        else if (ctx < 0) status = SCS_UNBOUNDED_INACCURATE;
        else status = tau > 0 ? SCS_SOLVED_INACCURATE : SCS_INFEASIBLE_INACCURATE;
    }
    // ---- outputs in the caller's units (Sec. 5 unscaling, Sec. 2.3 cases)
    const double tau = static_cast<double>(u[N - 1]);
    for (int e = threadIdx.x; e < n + 2 * m; e += NT) {
        if (status == 1 || status == 2) {
            if (e < n) B.x[M.xo + e] = B.E[M.xo + e] * static_cast<double>(u[e]) / (tau * sg);
            else if (e < n + m) B.y[M.yo + e - n] = B.D[M.yo + e - n] * static_cast<double>(u[e]) / (tau * rh);
            else B.s[M.yo + e - n - m] = static_cast<double>(v[e - m]) / (B.D[M.yo + e - n - m] * tau * sg);
        } else if (status == -1 || status == -3) {
            const double f = sg / (-last[2]);
            if (e < n) B.x[M.xo + e] = NAN;
            else if (e < n + m) B.y[M.yo + e - n] = B.D[M.yo + e - n] * static_cast<double>(u[e]) * f;
            else B.s[M.yo + e - n - m] = NAN;
        } else if (status == -2 || status == -4) {
            const double f = rh / (-last[5]);
            if (e < n) B.x[M.xo + e] = B.E[M.xo + e] * static_cast<double>(u[e]) * f;
            else if (e < n + m) B.y[M.yo + e - n] = NAN;
            else B.s[M.yo + e - n - m] = -B.ax[M.yo + e - n - m] * f / B.D[M.yo + e - n - m];
        } else {
            if (e < n) B.x[M.xo + e] = NAN;
            else if (e < n + m) B.y[M.yo + e - n] = NAN;
            else B.s[M.yo + e - n - m] = NAN;
        }
    }
    if (threadIdx.x == 0) {
        scs_info f{};
        f.status = status;
        f.iters = k;
        f.cg_iters = cg_total;
        f.matvecs = k + (k + kAzEvery - 1) / kAzEvery + 2 * cg_total;
        f.tau = last[6];
        f.kappa = last[7];
        f.res_pri = last[8];
        f.res_dual = last[9];
        f.gap = last[10];
        if (status == 1 || status == 2) {
            f.pobj = last[11];
            f.dobj = last[12];
        } else if (status == -1 || status == -3) {
            f.pobj = NAN;
            f.dobj = 1.0;
        } else if (status == -2 || status == -4) {
            f.pobj = -1.0;
            f.dobj = NAN;
        } else {
            f.pobj = f.dobj = NAN;
        }
        B.info[id] = f;
    }
}

// at least 640 threads' worth of CTAs per SM: about 100 registers a thread
// (the team code keeps several row sums and reduction values live)
template <int NT>
constexpr int min_blocks() { return 640 / NT > 1 ? 640 / NT : 1; }

template <typename T, int NT>
__global__ void __launch_bounds__(NT, min_blocks<NT>()) solve_kernel(Dev<T> B, int mode, int iters) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ double red[2 * kMaxNV * (NT / 32)];
    __shared__ double last[13];
    __shared__ int slot;
    Team<NT> tm{red, 0};
    for (;;) {
        const int pos = next_job(B.queue, &slot);
        if (pos >= B.norder) break;
        solve_program<T, NT>(B, B.order[pos], smem, tm, mode, iters, last);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
class BatchBase {
   public:
    virtual ~BatchBase() {}
    virtual int solve(double *x, double *y, double *s, scs_info *info) = 0;
    virtual int warm_start(const double *x, const double *y, const double *s) = 0;
    virtual int iterate(int iters) = 0;
    virtual int get_iterates(int idx, double *u, double *v) = 0;
    virtual void config(int32_t *threads, int32_t *split, double *tune_ms, double *setup_ms) = 0;
    int device = 0;
};

template <typename T>
using SolveFn = void (*)(Dev<T>, int, int);

template <typename T>
SolveFn<T> solve_fn(int nt) {
    switch (nt) {
        case 64: return solve_kernel<T, 64>;
        case 128: return solve_kernel<T, 128>;
        case 256: return solve_kernel<T, 256>;
        default: return solve_kernel<T, 512>;
    }
}

template <typename T>
class BatchEngine : public BatchBase {
   public:
    BatchEngine(const std::vector<HostProblem> &P, const scs_settings &st) : st_(st) {
        const auto t0 = std::chrono::steady_clock::now();
        device = st.device;
        SCS_CUDA(cudaSetDevice(device));
        SCS_CUDA(cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, device));
        if (st.cuda_stream) {
            stream_ = static_cast<cudaStream_t>(st.cuda_stream);
        } else {
            SCS_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
            own_stream_ = true;
        }
        layout(P);
        // setup: one persistent launch of 256-thread teams
        D_.norder = count_;
        D_.order = order_d_;
        SCS_CUDA(cudaMemsetAsync(queue_, 0, sizeof(int), stream_));
        {
            auto kern = setup_kernel<T, 256>;
            SCS_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_));
            int per_sm = 0;
            SCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem_));
            if (per_sm < 1) throw CudaError("a program needs more shared memory than a CTA has", SCS_UNSUPPORTED);
            kern<<<std::min(count_, sms_ * per_sm), 256, smem_, stream_>>>(D_);
            SCS_CUDA(cudaGetLastError());
        }
        SCS_CUDA(cudaStreamSynchronize(stream_));
        setup_ms_ = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        // host copies of the scaling (warm starts)
        Dh_.resize(ym_);
        Eh_.resize(xn_);
        sgh_.resize(count_);
        rhh_.resize(count_);
        SCS_CUDA(cudaMemcpy(Dh_.data(), D_.D, sizeof(double) * ym_, cudaMemcpyDeviceToHost));
        SCS_CUDA(cudaMemcpy(Eh_.data(), D_.E, sizeof(double) * xn_, cudaMemcpyDeviceToHost));
        SCS_CUDA(cudaMemcpy(sgh_.data(), D_.sigma, sizeof(double) * count_, cudaMemcpyDeviceToHost));
        SCS_CUDA(cudaMemcpy(rhh_.data(), D_.rho, sizeof(double) * count_, cudaMemcpyDeviceToHost));
        tune();
        reset_state();
        build_graph();
    }

    ~BatchEngine() override {
        cudaSetDevice(device);
        if (exec_) cudaGraphExecDestroy(exec_);
        if (graph_) cudaGraphDestroy(graph_);
        for (void *p : allocs_) cudaFree(p);
        if (own_stream_ && stream_) cudaStreamDestroy(stream_);
    }

    int solve(double *x, double *y, double *s, scs_info *info) override {
        SCS_CUDA(cudaSetDevice(device));
        const auto t0 = std::chrono::steady_clock::now();
        SCS_CUDA(cudaGraphLaunch(exec_, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (x) SCS_CUDA(cudaMemcpy(x, D_.x, sizeof(double) * xn_, cudaMemcpyDeviceToHost));
        if (y) SCS_CUDA(cudaMemcpy(y, D_.y, sizeof(double) * ym_, cudaMemcpyDeviceToHost));
        if (s) SCS_CUDA(cudaMemcpy(s, D_.s, sizeof(double) * ym_, cudaMemcpyDeviceToHost));
        if (info) {
            SCS_CUDA(cudaMemcpy(info, D_.info, sizeof(scs_info) * count_, cudaMemcpyDeviceToHost));
            for (int i = 0; i < count_; ++i) {
                info[i].setup_s = setup_ms_ * 1e-3;
                info[i].solve_s = el;
            }
        }
        return 0;
    }

    int warm_start(const double *x, const double *y, const double *s) override {
        SCS_CUDA(cudaSetDevice(device));
        std::vector<T> u(un_), v(un_);
        std::vector<double> dstep(count_);
        const double e = std::max(st_.eps_pri, std::max(st_.eps_dual, st_.eps_gap));
        for (int i = 0; i < count_; ++i) {
            const Meta &M = meta_[i];
            double nrm = 0.0;
            for (int j = 0; j < M.n; ++j) {
                const double t = x ? sgh_[i] * x[M.xo + j] / Eh_[M.xo + j] : 0.0;
                u[M.uo + j] = static_cast<T>(t);
                nrm += t * t;
            }
            for (int r = 0; r < M.m; ++r) {
                const double ty = y ? rhh_[i] * y[M.yo + r] / Dh_[M.yo + r] : 0.0;
                const double ts = s ? sgh_[i] * Dh_[M.yo + r] * s[M.yo + r] : 0.0;
                u[M.uo + M.n + r] = static_cast<T>(ty);
                v[M.uo + M.n + r] = static_cast<T>(ts);
                nrm += ty * ty + ts * ts;
            }
            u[M.uo + M.n + M.m] = T(1);
            v[M.uo + M.n + M.m] = T(0);
            for (int j = 0; j < M.n; ++j) v[M.uo + j] = T(0);
            dstep[i] = e * std::sqrt(nrm + 1.0);
        }
        SCS_CUDA(cudaMemcpy(D_.u, u.data(), sizeof(T) * un_, cudaMemcpyHostToDevice));
        SCS_CUDA(cudaMemcpy(D_.v, v.data(), sizeof(T) * un_, cudaMemcpyHostToDevice));
        SCS_CUDA(cudaMemcpy(D_.dstep, dstep.data(), sizeof(double) * count_, cudaMemcpyHostToDevice));
        SCS_CUDA(cudaMemset(D_.k, 0, sizeof(int32_t) * count_));
        std::vector<int32_t> ones(count_, 1);
        SCS_CUDA(cudaMemcpy(D_.warm, ones.data(), sizeof(int32_t) * count_, cudaMemcpyHostToDevice));
        return 0;
    }

    int iterate(int iters) override {
        SCS_CUDA(cudaSetDevice(device));
        run(D_, nt_, 1, iters);
        SCS_CUDA(cudaStreamSynchronize(stream_));
        return 0;
    }

    int get_iterates(int idx, double *u, double *v) override {
        if (idx < 0 || idx >= count_) return SCS_INVALID_INPUT;
        SCS_CUDA(cudaSetDevice(device));
        const Meta &M = meta_[idx];
        const int N = M.n + M.m + 1;
        std::vector<T> h(N);
        if (u) {
            SCS_CUDA(cudaMemcpy(h.data(), D_.u + M.uo, sizeof(T) * N, cudaMemcpyDeviceToHost));
            for (int i = 0; i < N; ++i) u[i] = static_cast<double>(h[i]);
        }
        if (v) {
            SCS_CUDA(cudaMemcpy(h.data(), D_.v + M.uo, sizeof(T) * N, cudaMemcpyDeviceToHost));
            for (int i = 0; i < N; ++i) v[i] = static_cast<double>(h[i]);
        }
        return 0;
    }

    void config(int32_t *threads, int32_t *split, double *tune_ms, double *setup_ms) override {
        if (threads) *threads = nt_;
        if (split) *split = split_;
        if (tune_ms) *tune_ms = tune_ms_;
        if (setup_ms) *setup_ms = setup_ms_;
    }

    // ---------------------------------------------------------------- layout
    template <typename U>
    U *dalloc(size_t count) {
        void *p = nullptr;
        SCS_CUDA(cudaMalloc(&p, sizeof(U) * (count ? count : 1)));
        allocs_.push_back(p);
        return static_cast<U *>(p);
    }
    template <typename U>
    U *upload(const std::vector<U> &h) {
        U *d = dalloc<U>(h.size());
        if (!h.empty()) SCS_CUDA(cudaMemcpy(d, h.data(), sizeof(U) * h.size(), cudaMemcpyHostToDevice));
        return d;
    }

    // rows of one program's stored CSR, longest first (stable), written at
    // row0 / nz0 of the concatenated arrays (rp[row0] already holds nz0)
    static void place_rows(const std::vector<int32_t> &rp, const std::vector<int32_t> &col,
                           const std::vector<double> &val, int rows, int64_t row0, int64_t nz0,
                           std::vector<int32_t> &grp, std::vector<int32_t> &grid, std::vector<int32_t> &gcol,
                           std::vector<double> &gval, std::vector<int32_t> &lens) {
        std::vector<int32_t> idx(rows);
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(),
                         [&](int a, int b) { return rp[a + 1] - rp[a] > rp[b + 1] - rp[b]; });
        int64_t w = nz0;
        for (int r = 0; r < rows; ++r) {
            const int i = idx[r];
            const int len = rp[i + 1] - rp[i];
            grid[row0 + r] = i;
            lens[row0 + r] = len;
            std::copy(col.begin() + rp[i], col.begin() + rp[i + 1], gcol.begin() + w);
            std::copy(val.begin() + rp[i], val.begin() + rp[i + 1], gval.begin() + w);
            w += len;
            grp[row0 + r + 1] = static_cast<int32_t>(w);
        }
    }

    void layout(const std::vector<HostProblem> &P) {
        count_ = static_cast<int>(P.size());
        // offsets of every program in the concatenated arrays (one pass),
        // then the programs' rows copied on threads
        std::vector<int64_t> a_r0(count_ + 1, 0), at_r0(count_ + 1, 0), a_nz0(count_ + 1, 0), at_nz0(count_ + 1, 0);
        std::vector<int64_t> q0(count_ + 1, 0), wpre(count_ + 1, 0);
        int64_t xn = 0, ym = 0, un = 0;
        size_t smem = 0;
        meta_.resize(count_);
        for (int i = 0; i < count_; ++i) {
            const HostProblem &H = P[i];
            Meta &M = meta_[i];
            M.n = H.n;
            M.m = H.m;
            M.z = H.z;
            M.l = H.l;
            M.nq = static_cast<int>(H.q.size());
            M.soc0 = static_cast<int>(q0[i]);
            M.a_row0 = static_cast<int>(a_r0[i]);
            M.at_row0 = static_cast<int>(at_r0[i]);
            M.xo = static_cast<int>(xn);
            M.yo = static_cast<int>(ym);
            M.uo = static_cast<int>(un);
            q0[i + 1] = q0[i] + static_cast<int64_t>(H.q.size());
            a_r0[i + 1] = a_r0[i] + H.m;
            at_r0[i + 1] = at_r0[i] + H.n;
            a_nz0[i + 1] = a_nz0[i] + static_cast<int64_t>(H.a_col.size());
            at_nz0[i + 1] = at_nz0[i] + static_cast<int64_t>(H.at_col.size());
            wpre[i + 1] = wpre[i] + static_cast<int64_t>(H.a_col.size()) + H.m + H.n;
            xn += H.n;
            ym += H.m;
            un += H.n + H.m + 1;
            smem = std::max(smem, team_bytes<T>(H.n, H.m));
            work_.push_back(static_cast<double>(H.nnz) + H.n + H.m);
        }
        if (a_nz0[count_] >= ((int64_t)1 << 31) || un >= ((int64_t)1 << 31) || a_r0[count_] >= ((int64_t)1 << 31))
            throw CudaError("batch too large for 32-bit offsets", SCS_UNSUPPORTED);
        std::vector<int32_t> a_rp(a_r0[count_] + 1, 0), a_rid(a_r0[count_]), a_col(a_nz0[count_]);
        std::vector<int32_t> at_rp(at_r0[count_] + 1, 0), at_rid(at_r0[count_]), at_col(at_nz0[count_]);
        std::vector<int32_t> soc_off(q0[count_]), soc_len(q0[count_]);
        std::vector<double> a_val(a_nz0[count_]), at_val(at_nz0[count_]), b(ym), c(xn);
        a_len_.assign(a_r0[count_], 0);
        at_len_.assign(at_r0[count_], 0);
        const int nth = std::max(1, std::min(host_threads(wpre[count_]), count_));
        const std::vector<int32_t> cut = weight_cuts(wpre.data(), count_, nth);
        std::vector<char> failed(nth, 0);
        run_parts(nth, [&](int t) {
            try {
                for (int i = cut[t]; i < cut[t + 1]; ++i) {
                    const HostProblem &H = P[i];
                    const Meta &M = meta_[i];
                    int off = H.z + H.l;
                    for (size_t j = 0; j < H.q.size(); ++j) {
                        soc_off[q0[i] + j] = off;
                        soc_len[q0[i] + j] = H.q[j];
                        off += H.q[j];
                    }
                    place_rows(H.a_rowptr, H.a_col, H.a_val, H.m, a_r0[i], a_nz0[i], a_rp, a_rid, a_col, a_val, a_len_);
                    place_rows(H.at_rowptr, H.at_col, H.at_val, H.n, at_r0[i], at_nz0[i], at_rp, at_rid, at_col,
                               at_val, at_len_);
                    std::copy(H.b.begin(), H.b.end(), b.begin() + M.yo);
                    std::copy(H.c.begin(), H.c.end(), c.begin() + M.xo);
                }
            } catch (...) {
                failed[t] = 1;
            }
        });
        for (char f : failed)
            if (f) throw std::bad_alloc();
        xn_ = xn;
        ym_ = ym;
        un_ = un;
        smem_ = smem;
        // queue order: largest programs first
        order_.resize(count_);
        std::iota(order_.begin(), order_.end(), 0);
        std::stable_sort(order_.begin(), order_.end(), [&](int a, int b) { return work_[a] > work_[b]; });
        set_split(16);
        D_.count = count_;
        D_.meta = meta_d_ = upload(meta_);
        order_d_ = upload(order_);
        D_.soc_off = upload(soc_off);
        D_.soc_len = upload(soc_len);
        D_.a_rp = upload(a_rp);
        D_.a_rid = upload(a_rid);
        D_.a_col = upload(a_col);
        D_.at_rp = upload(at_rp);
        D_.at_rid = upload(at_rid);
        D_.at_col = upload(at_col);
        D_.a_v64 = upload(a_val);
        D_.at_v64 = upload(at_val);
        D_.a_val = dalloc<T>(a_val.size());
        D_.at_val = dalloc<T>(at_val.size());
        D_.b = upload(b);
        D_.c = upload(c);
        D_.D = dalloc<double>(ym);
        D_.E = dalloc<double>(xn);
        D_.b64 = dalloc<double>(ym);
        D_.c64 = dalloc<double>(xn);
        D_.bh = dalloc<T>(ym);
        D_.ch = dalloc<T>(xn);
        D_.dg = dalloc<T>(xn);
        D_.pM = dalloc<T>(xn + ym);
        D_.sigma = dalloc<double>(count_);
        D_.rho = dalloc<double>(count_);
        D_.hp1 = dalloc<double>(count_);
        D_.nb = dalloc<double>(count_);
        D_.nc = dalloc<double>(count_);
        D_.u = dalloc<T>(un);
        D_.v = dalloc<T>(un);
        D_.zcg = dalloc<T>(xn);
        D_.k = dalloc<int32_t>(count_);
        D_.warm = dalloc<int32_t>(count_);
        D_.dstep = dalloc<double>(count_);
        D_.ax = dalloc<double>(ym);
        D_.x = dalloc<double>(xn);
        D_.y = dalloc<double>(ym);
        D_.s = dalloc<double>(ym);
        D_.info = dalloc<scs_info>(count_);
        D_.queue = queue_ = dalloc<int>(1);
        D_.alpha = st_.alpha;
        D_.eps_pri = st_.eps_pri;
        D_.eps_dual = st_.eps_dual;
        D_.eps_gap = st_.eps_gap;
        D_.eps_infeas = st_.eps_infeas;
        D_.eps_unbdd = st_.eps_unbdd;
        D_.cg_rate = st_.cg_rate;
        D_.cg_adapt = st_.cg_adapt;
        D_.cg_tol_rel = st_.cg_tol_rel;
        D_.max_iters = st_.max_iters;
        D_.check_interval = st_.check_interval;
        D_.cg_max = st_.cg_max_iters;
        D_.normalize = st_.normalize;
        D_.passes = st_.scale_passes;
        D_.block_scale = st_.block_scale;
        upload_meta();
    }

    // long rows: more than `split` nonzeros (rows are stored longest first)
    void set_split(int split) {
        split_ = split;
        for (int i = 0; i < count_; ++i) {
            Meta &M = meta_[i];
            int c = 0;
            while (c < M.m && a_len_[M.a_row0 + c] > split) ++c;
            M.a_nlong = c;
            c = 0;
            while (c < M.n && at_len_[M.at_row0 + c] > split) ++c;
            M.at_nlong = c;
        }
    }
    void upload_meta() {
        SCS_CUDA(cudaMemcpy(meta_d_, meta_.data(), sizeof(Meta) * count_, cudaMemcpyHostToDevice));
    }

    // cold state u = (0, 0, 1), v = (0, 0, 1), z = 0, k = 0 for every program
    void reset_state() {
        std::vector<T> u(un_, T(0));
        for (int i = 0; i < count_; ++i) u[meta_[i].uo + meta_[i].n + meta_[i].m] = T(1);
        SCS_CUDA(cudaMemcpy(D_.u, u.data(), sizeof(T) * un_, cudaMemcpyHostToDevice));
        SCS_CUDA(cudaMemcpy(D_.v, u.data(), sizeof(T) * un_, cudaMemcpyHostToDevice));
        SCS_CUDA(cudaMemset(D_.zcg, 0, sizeof(T) * xn_));
        SCS_CUDA(cudaMemset(D_.k, 0, sizeof(int32_t) * count_));
        SCS_CUDA(cudaMemset(D_.warm, 0, sizeof(int32_t) * count_));
        std::vector<double> inf(count_, INFINITY);
        SCS_CUDA(cudaMemcpy(D_.dstep, inf.data(), sizeof(double) * count_, cudaMemcpyHostToDevice));
    }

    int grid_for(int nt) {
        SolveFn<T> f = solve_fn<T>(nt);
        SCS_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_));
        int per_sm = 0;
        SCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, nt, smem_));
        if (per_sm < 1) throw CudaError("a program needs more shared memory than a CTA has", SCS_UNSUPPORTED);
        return sms_ * per_sm;
    }

    // queue reset + one persistent launch over D.order[0, D.norder)
    void run(const Dev<T> &D, int nt, int mode, int iters) {
        SCS_CUDA(cudaMemsetAsync(queue_, 0, sizeof(int), stream_));
        const int grid = std::min(D.norder, grid_for(nt));
        solve_fn<T>(nt)<<<grid, nt, smem_, stream_>>>(D, mode, iters);
        SCS_CUDA(cudaGetLastError());
    }

    // Autotuner: team size x row split, timed over `kTuneIters` iterations of
    // a sample of programs spread over the size order (kept largest first, as
    // the solve's queue is); keeps the fastest.  The sample holds at least
    // four programs per resident team of every candidate, so each candidate
    // is timed with all of its teams busy, as in the solve: a sample that
    // fills only part of the resident teams favours large teams.
    void tune() {
        const auto t0 = std::chrono::steady_clock::now();
        static const int kThreads[] = {64, 128, 256, 512};
        static const int kSplits[] = {4, 16, 64};
        const int kTuneIters = 10;
        int teams = 1;
        for (int nt : kThreads) teams = std::max(teams, grid_for(nt));
        const int ns = static_cast<int>(std::min<int64_t>(count_, 4 * static_cast<int64_t>(teams)));
        std::vector<int32_t> sample;
        for (int i = 0; i < ns; ++i) sample.push_back(order_[(int64_t)i * count_ / ns]);
        int32_t *sample_d = upload(sample);
        Dev<T> Ds = D_;
        Ds.order = sample_d;
        Ds.norder = ns;
        cudaEvent_t e0, e1;
        SCS_CUDA(cudaEventCreate(&e0));
        SCS_CUDA(cudaEventCreate(&e1));
        float best = INFINITY;
        int best_nt = 256, best_split = 16;
        set_split(kSplits[0]);     // one untimed launch first (module load, cold caches)
        upload_meta();
        reset_state();
        run(Ds, kThreads[0], 1, 1);
        for (int sp : kSplits) {
            set_split(sp);
            upload_meta();
            for (int nt : kThreads) {
                reset_state();
                SCS_CUDA(cudaEventRecord(e0, stream_));
                run(Ds, nt, 1, kTuneIters);
                SCS_CUDA(cudaEventRecord(e1, stream_));
                SCS_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                SCS_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    best_nt = nt;
                    best_split = sp;
                }
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        nt_ = best_nt;
        set_split(best_split);
        upload_meta();
        tune_ms_ = 1e3 * std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    // the solve as a CUDA graph: queue reset, persistent launch
    void build_graph() {
        D_.order = order_d_;
        D_.norder = count_;
        const int grid = std::min(count_, grid_for(nt_));
        SCS_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
        SCS_CUDA(cudaMemsetAsync(queue_, 0, sizeof(int), stream_));
        solve_fn<T>(nt_)<<<grid, nt_, smem_, stream_>>>(D_, 0, 0);
        SCS_CUDA(cudaStreamEndCapture(stream_, &graph_));
        SCS_CUDA(cudaGraphInstantiate(&exec_, graph_, 0));
    }

    scs_settings st_;
    int sms_ = 1, count_ = 0, nt_ = 256, split_ = 16;
    int64_t xn_ = 0, ym_ = 0, un_ = 0;
    size_t smem_ = 0;
    double setup_ms_ = 0.0, tune_ms_ = 0.0;
    cudaStream_t stream_ = nullptr;
    bool own_stream_ = false;
    std::vector<void *> allocs_;
    std::vector<Meta> meta_;
    std::vector<int32_t> order_, a_len_, at_len_;
    std::vector<double> work_, Dh_, Eh_, sgh_, rhh_;
    Meta *meta_d_ = nullptr;
    int32_t *order_d_ = nullptr;
    int *queue_ = nullptr;
    Dev<T> D_{};
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
};

}  // namespace batch
}  // namespace scs

struct scs_batch {
    scs::batch::BatchBase *eng = nullptr;
};

namespace {

template <typename F>
int32_t batch_guarded(F f) {
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

scs_batch *scs_batch_init(int32_t count, const scs_csc *A, const double *b, const double *c, const scs_cone *k,
                          const scs_settings *st, int32_t *err) {
    int32_t e = 0;
    scs_batch *w = nullptr;
    if (count <= 0 || !A || !b || !c || !k) {
        scs::set_last_error("bad batch arguments");
        e = SCS_INVALID_INPUT;
    }
    scs_settings s{};
    if (!e) {
        if (st) s = *st;
        else scs_default_settings(&s);
        if (s.linsys != 0) {
            scs::set_last_error("batched programs take the indirect subspace step only (linsys 0)");
            e = SCS_UNSUPPORTED;
        }
    }
    std::vector<scs::HostProblem> P;
    if (!e) {
        P.resize(count);
        // offsets of each program's b and c; from the first program with a
        // non-positive size on they mean nothing, so only the programs before
        // it are validated on threads (parts of about equal nonzeros)
        std::vector<int64_t> yo(count + 1, 0), xo(count + 1, 0), pre(count + 1, 0);
        int32_t nvalid = count;
        for (int32_t i = 0; i < count; ++i) {
            if (A[i].m <= 0 || A[i].n <= 0) {
                nvalid = i;
                break;
            }
            yo[i + 1] = yo[i] + A[i].m;
            xo[i + 1] = xo[i] + A[i].n;
            pre[i + 1] = pre[i] + 1 + (A[i].colptr ? std::max<int64_t>(0, A[i].colptr[A[i].n]) : 0);
        }
        std::vector<int32_t> rc(count, 0);
        std::vector<std::string> msg(count);
        auto check = [&](int32_t i) {
            try {
                if (k[i].ns > 0 || k[i].ep > 0 || k[i].ed > 0 || k[i].np > 0) {
                    rc[i] = SCS_UNSUPPORTED;
                    msg[i] = "batched programs take zero, nonnegative and second-order cones only";
                    return;
                }
                rc[i] = scs::validate_and_build(&A[i], b + yo[i], c + xo[i], &k[i], P[i]);
                if (rc[i]) msg[i] = scs_last_error();
            } catch (...) {
                rc[i] = SCS_DEVICE_ERROR;
            }
        };
        const int T = std::max(1, std::min(scs::host_threads(pre[nvalid]), static_cast<int>(nvalid)));
        const std::vector<int32_t> cut = scs::weight_cuts(pre.data(), nvalid, T);
        scs::run_parts(T, [&](int t) {
            for (int32_t i = cut[t]; i < cut[t + 1]; ++i) check(i);
        });
        if (nvalid < count) check(nvalid);         // fails: a non-positive size (or its cone)
        // the error of the first failing program, as a program-by-program
        // check would report it
        for (int32_t i = 0; i <= std::min(nvalid, count - 1) && !e; ++i)
            if (rc[i]) {
                e = rc[i];
                scs::set_last_error("program " + std::to_string(i) + ": " +
                                    (msg[i].empty() ? std::string("host allocation failed") : msg[i]));
            }
    }
    if (!e) {
        e = batch_guarded([&]() -> int32_t {
            w = new scs_batch;
            if (s.precision == 0)
                w->eng = new scs::batch::BatchEngine<double>(P, s);
            else
                w->eng = new scs::batch::BatchEngine<float>(P, s);
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

int32_t scs_batch_solve(scs_batch *w, double *x, double *y, double *s, scs_info *info) {
    if (!w || !w->eng) return SCS_INVALID_INPUT;
    return batch_guarded([&] { return w->eng->solve(x, y, s, info); });
}

int32_t scs_batch_warm_start(scs_batch *w, const double *x, const double *y, const double *s) {
    if (!w || !w->eng) return SCS_INVALID_INPUT;
    return batch_guarded([&] { return w->eng->warm_start(x, y, s); });
}

int32_t scs_batch_iterate(scs_batch *w, int32_t iters) {
    if (!w || !w->eng || iters < 0) return SCS_INVALID_INPUT;
    return batch_guarded([&] { return w->eng->iterate(iters); });
}

int32_t scs_batch_get_iterates(scs_batch *w, int32_t index, double *u, double *v) {
    if (!w || !w->eng) return SCS_INVALID_INPUT;
    return batch_guarded([&] { return w->eng->get_iterates(index, u, v); });
}

int32_t scs_batch_config(scs_batch *w, int32_t *threads, int32_t *row_split, double *tune_ms, double *setup_ms) {
    if (!w || !w->eng) return SCS_INVALID_INPUT;
    w->eng->config(threads, row_split, tune_ms, setup_ms);
    return 0;
}

void scs_batch_finish(scs_batch *w) {
    if (!w) return;
    delete w->eng;
    delete w;
}

}  // extern "C"
