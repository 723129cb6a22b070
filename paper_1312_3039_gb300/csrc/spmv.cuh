// CSR sparse matrix-vector product with a fused per-row epilogue and a fused
// deterministic grid reduction.
//
// Rows are grouped at setup into "stream blocks" of consecutive rows holding
// at most kStreamCap nonzeros (or one longer row).  One CTA per stream block:
//   1. the CTA streams its contiguous slice of (col, val) with coalesced,
//      unrolled loads, multiplies by the gathered x entries and stages the
//      products in shared memory;
//   2. each row is summed from shared memory by a group of 1..32 lanes sized
//      to the block's row count, and the epilogue consumes the row sum
//      (writes outputs and adds to the block's reduction values);
//   3. the reduction values go through grid_sum; the last CTA runs the
//      epilogue's finisher (scalar updates of CG, termination tests).
// A row longer than kStreamCap is summed by its CTA directly from global
// memory.  Keeping the original row order keeps output writes coalesced.
#pragma once

#include <vector>

#include "common.cuh"

namespace scs {

template <typename TA>
struct Csr {
    const int32_t *rowptr;   // rows + 1
    const int32_t *col;      // nnz
    const TA *val;           // nnz
    const int32_t *blk;      // nblk + 1 first rows of the stream blocks
    int32_t nblk;
    int32_t rows;
};

template <typename Acc, typename TA, typename TX>
__device__ __forceinline__ Acc fmul(TA a, TX x) {
    return static_cast<Acc>(a) * static_cast<Acc>(x);
}

// The matrix arrays are read once per product: load them with the streaming
// (evict-first) policy so that they do not push the gathered vector out of L2.
template <typename U>
__device__ __forceinline__ U ld_stream(const U *p) { return __ldcs(p); }

template <typename TA, typename TX, typename Acc, typename Epi>
__global__ void __launch_bounds__(kBlock) spmv_stream_kernel(Csr<TA> A, const TX *__restrict__ x,
                                                             Epi epi, ReduceBuf rb) {
    constexpr int NV = Epi::NV;
    if (epi.skip()) return;
    __shared__ Acc prod[kStreamCap];
    epi.begin();
    static_assert(NV >= 1 && NV <= kMaxRed, "epilogue reduction width");
    double red[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i] = 0.0;

    const int b = blockIdx.x;
    const int r0 = A.blk[b], r1 = A.blk[b + 1];
    const int k0 = A.rowptr[r0], k1 = A.rowptr[r1];
    const int nz = k1 - k0;
    const int tid = threadIdx.x;

    if (nz > kStreamCap) {
        // one long row: the whole CTA sums it
        Acc s = 0;
        const int32_t *__restrict__ col = A.col;
        const TA *__restrict__ val = A.val;
#pragma unroll 4
        for (int k = k0 + tid; k < k1; k += kBlock) s += fmul<Acc>(ld_stream(val + k), __ldg(x + ld_stream(col + k)));
        double t[1] = {static_cast<double>(s)};
        // sum in Acc precision order-independent of warps: use block_sum in double
        block_sum<1>(t);
        if (tid == 0) epi.row(r0, static_cast<Acc>(t[0]), red);
    } else {
        const int32_t *__restrict__ col = A.col + k0;
        const TA *__restrict__ val = A.val + k0;
#pragma unroll 8
        for (int k = tid; k < nz; k += kBlock) prod[k] = fmul<Acc>(ld_stream(val + k), __ldg(x + ld_stream(col + k)));
        __syncthreads();
        const int nr = r1 - r0;
        int L = 1;
        while (L < 32 && 2 * L * nr <= kBlock) L *= 2;
        const int groups = kBlock / L;
        const int g = tid / L, lane = tid % L;
        for (int base = 0; base < nr; base += groups) {
            const int rr = base + g;
            const bool valid = rr < nr;
            Acc s = 0;
            if (valid) {
                const int rs = A.rowptr[r0 + rr] - k0, re = A.rowptr[r0 + rr + 1] - k0;
                for (int k = rs + lane; k < re; k += L) s += prod[k];
            }
            for (int o = L >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            if (valid && lane == 0) epi.row(r0 + rr, s, red);
        }
    }
    double tot[NV];
    if (grid_sum<NV>(red, rb, Epi::kSite, tot)) {
        if (tid == 0) epi.finish(tot);
    }
}

// Host-side partition of rows into stream blocks.
inline void stream_blocks(const int32_t *rowptr, int32_t rows, std::vector<int32_t> &blk) {
    blk.clear();
    blk.push_back(0);
    int32_t r = 0;
    while (r < rows) {
        int32_t start = rowptr[r];
        int32_t e = r + 1;
        if (rowptr[e] - start <= kStreamCap) {
            while (e < rows && rowptr[e + 1] - start <= kStreamCap) ++e;
        }
        blk.push_back(e);
        r = e;
    }
    if (rows == 0) blk.push_back(0);
}

}  // namespace scs
