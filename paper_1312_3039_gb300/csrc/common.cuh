// Device-side helpers shared by the solver kernels: error handling, the
// scalar state of one solve, warp/block sums and a deterministic grid sum.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace scs {

constexpr int kBlock = 256;          // threads per CTA for every kernel
constexpr int kWarps = kBlock / 32;
constexpr int kMaxRed = 6;           // most values one grid sum carries

// Scalars of one solve.  Written by the "last block" finishers of the grid
// sums and read by later kernels; the host reads a copy at check time.
struct Scalars {
    // current ADMM iteration
    double wtau;        // w_tau = u_tau + v_kappa
    double ww_y;        // ||u_y + v_y||^2 (for ||w||)
    double tol;         // CG stopping tolerance of this iteration
    double rz, pp, qq, rr;
    double alpha, beta;
    double gamma;       // h^T z / (1 + h^T p)
    double hp1;         // 1 + h^T p   (Sec. 4.1, cached)
    // settings mirrored on the device
    double cg_rate, cg_adapt, cg_tol_rel, relax;
    double dstep;       // ||(u, v) - (u, v)_previous|| of the last ADMM step
    // termination quantities (scaled problem, Sec. 5)
    double pri2, unb2, bty, dual2, inf2, ctx;
    double res_pri, res_dual, gap, pobj, dobj, tau, kappa;
    double eps_pri, eps_dual, eps_gap, eps_infeas, eps_unbdd;
    double nb, nc;      // ||b||, ||c|| of the unscaled data
    double sigma, rho;
    int32_t k;          // completed ADMM iterations
    int32_t cg_it;      // CG steps in the current ADMM iteration
    int32_t cg_max;
    int32_t done;       // CG residual test passed (or cap reached)
    int32_t active;     // CG loop still running
    int32_t status;     // termination status written by the check
    int32_t dev_error;  // set by a kernel whose bounded wait timed out
    int64_t cg_total;   // CG steps since the last reset
    unsigned long long psd_calls;    // PSD block projections since setup
    unsigned long long psd_sweeps;   // their Jacobi sweeps
    unsigned long long psd_fp64;     // of them reconstructed in FP64
};

struct ReduceBuf {
    double *partials;   // [kMaxRed][cap]: value i of block b at i * cap + b
    unsigned *counter;  // one counter per call site
    int cap;            // blocks the buffer holds
};

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV values over the block; the result is valid in every thread.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
    __shared__ double sm[kMaxRed][kWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    __syncthreads();
    if (lane == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) sm[i][warp] = v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        double t = lane < kWarps ? sm[i][lane] : 0.0;
        v[i] = warp_sum(t);
    }
    __syncthreads();
}

// Deterministic grid-wide sum of NV values: every block writes its partial
// sums, the last block to arrive adds them in block order.  Returns true (in
// all threads of that last block only) with the totals in `tot`.
template <int NV>
__device__ __forceinline__ bool grid_sum(double (&v)[NV], ReduceBuf rb, int site, double (&tot)[NV]) {
    __shared__ bool last;
    block_sum<NV>(v);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) rb.partials[(size_t)i * rb.cap + blockIdx.x] = v[i];
        __threadfence();
        unsigned t = atomicAdd(rb.counter + site, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) {
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += __ldcg(rb.partials + (size_t)i * rb.cap + b);
    }
    block_sum<NV>(acc);
#pragma unroll
    for (int i = 0; i < NV; ++i) tot[i] = acc[i];
    if (threadIdx.x == 0) rb.counter[site] = 0u;
    return true;
}

// The warm-start product A^ z_prev of the CG runs on every kAzEvery-th ADMM
// iteration; the iterations between carry A^ z_x forward from the CG's own
// A^ p products (kernels.cuh header).
constexpr int kAzEvery = 20;

// grid-sum call sites (each has its own arrival counter)
enum Site : int {
    kSiteAInit = 0, kSiteAtInit, kSiteACG, kSiteAtCG, kSiteCGUpd, kSiteSmw,
    kSiteChkA, kSiteChkAt, kSiteProj, kSiteMisc, kSiteMisc2, kSiteAz, kSiteCount
};

}  // namespace scs
