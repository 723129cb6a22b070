// CSR sparse matrix-vector product with a fused per-row epilogue and a fused
// deterministic grid reduction, built for rows of power-law lengths.
//
// Layout (setup, host): rows are stored grouped by length class (1, 2, 3-4,
// 5-8, ...; original order kept inside a class; `rowid` maps a stored row
// back to its matrix row, which is where the epilogue writes).  The stored
// rows are cut into chunks of at most kChunkNnz nonzeros:
//   * runs of same-class rows (at most kChunkRows rows), so the rows summed
//     together have similar lengths;
//   * pieces of a row longer than kChunkNnz, in order; the pieces of one
//     row carry a running sum and the last one completes the row.
// The chunk list is cut into one contiguous, nnz-balanced range per CTA of a
// persistent grid (never inside the pieces of one row).
//
// Kernel: each CTA keeps kStages shared-memory stages.  One thread fills a
// stage with TMA bulk copies (cp.async.bulk, completion on an mbarrier) of
// the chunk's column indices and values (and, for a run of rows, its row
// pointers and row ids), and puts the chunk descriptor in the stage header.
// For each chunk the threads wait on the stage's barrier (bounded: on
// timeout an error flag is set), form the products val * x[col] (the only
// global loads left on the threads' path are the gathers of x, served from
// L2), stage them in shared memory, and either sum each row with a group of
// L lanes sized to the chunk's row count, or (a piece) sum the whole chunk
// into the row's running sum; completed row sums go to the epilogue.  Every thread accumulates the epilogue's
// reduction values over all its rows; each CTA joins one grid_sum at the end,
// whose last CTA runs the epilogue's finisher.
#pragma once

#include <stdint.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace scs {

constexpr int kChunkNnz = 1024;      // nonzeros of one chunk (and the long-row threshold)
constexpr int kChunkRows = 512;      // rows of one chunk
constexpr int kStages = 2;           // TMA stages per CTA
constexpr int kPad = 4;              // elements of zero padding after every array a copy may touch

// chunk kinds
constexpr int kRun = 0;          // whole rows [r0, r1)
constexpr int kPiece = 1;        // nonzeros [k0, k1) of the single row r0
constexpr int kLastPiece = 3;    // ... and the row ends here

template <typename TA>
struct Csr {
    const int32_t *rowptr;   // rows + 1 (+kPad) (stored order)
    const int32_t *col;      // nnz (+kPad)
    const TA *val;           // nnz (+kPad)
    const int32_t *rowid;    // rows (+kPad): matrix row of each stored row
    const int4 *chunk;       // nchunk: (r0, r1, k0, k1)
    const int32_t *kind;     // nchunk: kRun, kPiece or kLastPiece
    const int32_t *cta_item; // grid + 1: chunk range of each CTA
    int32_t *err;            // set to 1 by a CTA whose copy wait timed out
    int32_t nchunk, rows, grid;
};

template <typename TA, typename Acc>
struct SpmvSmem {
    // one stage; each array starts on a 16-byte boundary
    static constexpr int kColWords = kChunkNnz + 2 * kPad;
    static constexpr int kValElems = kChunkNnz + 2 * kPad;
    static constexpr int kRowWords = kChunkRows + 2 * kPad;
    static constexpr size_t kColOff = 0;
    static constexpr size_t kValOff = kColOff + sizeof(int32_t) * kColWords;
    static constexpr size_t kRpOff = kValOff + ((sizeof(TA) * kValElems + 15) / 16) * 16;
    static constexpr size_t kRidOff = kRpOff + sizeof(int32_t) * kRowWords;
    static constexpr size_t kStageBytes = kRidOff + sizeof(int32_t) * kRowWords;
    static constexpr size_t kProdOff = kStages * kStageBytes;
    static constexpr size_t kBarOff = kProdOff + ((sizeof(Acc) * kChunkNnz + 15) / 16) * 16;
    static constexpr size_t kHdrOff = kBarOff + 8 * kStages;          // int4 descriptor + kind per stage
    static constexpr size_t kBytes = kHdrOff + 32 * kStages;
};

// ---------------------------------------------------------------------------
// TMA / mbarrier helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait: false if the phase did not complete within the limit
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    for (int i = 0; i < (1 << 20); ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <typename Acc, typename TA, typename TX>
__device__ __forceinline__ Acc fmul(TA a, TX x) {
    return static_cast<Acc>(a) * static_cast<Acc>(x);
}

// first element of the 16-byte block holding element k of an array of U,
// and the end of the 16-byte block holding element k - 1
template <typename U>
__device__ __host__ __forceinline__ int64_t align_down16(int64_t k) {
    constexpr int per = 16 / (int)sizeof(U);
    return k & ~(int64_t)(per - 1);
}
template <typename U>
__device__ __host__ __forceinline__ int64_t align_up16(int64_t k) {
    constexpr int per = 16 / (int)sizeof(U);
    return (k + per - 1) & ~(int64_t)(per - 1);
}

// Issue the copies of chunk c into stage s (one thread); the descriptor goes
// to the stage header (written before the arrive, which releases it).
template <typename TA, typename Acc>
__device__ __forceinline__ void issue_chunk(const Csr<TA> &A, int c, unsigned char *smem, int s) {
    using L = SpmvSmem<TA, Acc>;
    unsigned char *st = smem + s * L::kStageBytes;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::kBarOff) + s;
    int4 *hdr = reinterpret_cast<int4 *>(smem + L::kHdrOff);
    int *hkind = reinterpret_cast<int *>(smem + L::kHdrOff + 16 * kStages);
    const int4 d = A.chunk[c];
    const int kind = A.kind[c];
    hdr[s] = d;
    hkind[s] = kind;
    const int r0 = d.x, r1 = d.y, k0 = d.z, k1 = d.w;
    const int64_t ca = align_down16<int32_t>(k0), cb = align_up16<int32_t>(k1);
    const int64_t va = align_down16<TA>(k0), vb = align_up16<TA>(k1);
    const uint32_t bc = (uint32_t)(4 * (cb - ca)), bv = (uint32_t)(sizeof(TA) * (vb - va));
    uint32_t bp = 0, bi = 0;
    int64_t pa = 0, ia = 0;
    if (kind == kRun) {
        pa = align_down16<int32_t>(r0);
        ia = pa;
        bp = (uint32_t)(4 * (align_up16<int32_t>(r1 + 1) - pa));
        bi = (uint32_t)(4 * (align_up16<int32_t>(r1) - ia));
    }
    mbar_expect_tx(bar, bc + bv + bp + bi);
    if (bc) bulk_g2s(st + L::kColOff, A.col + ca, bc, bar);
    if (bv) bulk_g2s(st + L::kValOff, A.val + va, bv, bar);
    if (bp) bulk_g2s(st + L::kRpOff, A.rowptr + pa, bp, bar);
    if (bi) bulk_g2s(st + L::kRidOff, A.rowid + ia, bi, bar);
}

template <typename TA, typename TX, typename Acc, typename Epi>
__global__ void __launch_bounds__(kBlock) spmv_kernel(Csr<TA> A, const TX *__restrict__ x, Epi epi, ReduceBuf rb) {
    using L = SpmvSmem<TA, Acc>;
    constexpr int NV = Epi::NV;
    static_assert(NV >= 1 && NV <= kMaxRed, "epilogue reduction width");
    if (epi.skip()) return;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + L::kBarOff);
    const int4 *hdr = reinterpret_cast<const int4 *>(smem + L::kHdrOff);
    const int *hkind = reinterpret_cast<const int *>(smem + L::kHdrOff + 16 * kStages);
    Acc *prod = reinterpret_cast<Acc *>(smem + L::kProdOff);
    epi.begin();
    double red[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i] = 0.0;
    const int tid = threadIdx.x;
    const int c0 = A.cta_item[blockIdx.x], c1 = A.cta_item[blockIdx.x + 1];
    const int nch = c1 - c0;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&bar[s], 1);
        mbar_init_fence();
        for (int j = 0; j < nch && j < kStages; ++j) issue_chunk<TA, Acc>(A, c0 + j, smem, j);
    }
    __syncthreads();

    double piece_sum = 0.0;          // running sum of a row split into pieces (thread 0)
    bool ok = true;
    for (int j = 0; j < nch; ++j) {
        const int s = j % kStages;
        const uint32_t parity = (uint32_t)((j / kStages) & 1);
        unsigned char *st = smem + s * L::kStageBytes;
        // every thread observes the stage's phase; the CTA leaves together if
        // any wait timed out
        const bool got = mbar_wait(&bar[s], parity);
        if (!__syncthreads_and(got)) { ok = false; break; }
        const int32_t *col_s = reinterpret_cast<const int32_t *>(st + L::kColOff);
        const TA *val_s = reinterpret_cast<const TA *>(st + L::kValOff);
        const int4 d = hdr[s];
        const int kind = hkind[s];
        const int r0 = d.x, r1 = d.y, k0 = d.z, k1 = d.w;
        const int cofs = k0 - (int)align_down16<int32_t>(k0), vofs = k0 - (int)align_down16<TA>(k0);
        const int nz = k1 - k0;
#pragma unroll 8
        for (int e = tid; e < nz; e += kBlock) prod[e] = fmul<Acc>(val_s[vofs + e], __ldg(x + col_s[cofs + e]));
        __syncthreads();
        if (kind == kRun) {
            const int32_t *rp_s = reinterpret_cast<const int32_t *>(st + L::kRpOff);
            const int32_t *rid_s = reinterpret_cast<const int32_t *>(st + L::kRidOff);
            const int pa = (int)align_down16<int32_t>(r0);
            const int nr = r1 - r0;
            int Ln = 1;
            while (Ln < 32 && 2 * Ln * nr <= kBlock) Ln *= 2;
            const int groups = kBlock / Ln, g = tid / Ln, gl = tid % Ln;
            for (int base = 0; base < nr; base += groups) {
                const int rr = base + g;
                Acc sacc = 0;
                if (rr < nr) {
                    const int rs = rp_s[r0 + rr - pa] - k0, re = rp_s[r0 + rr + 1 - pa] - k0;
                    for (int e = rs + gl; e < re; e += Ln) sacc += prod[e];
                }
                for (int o = Ln >> 1; o > 0; o >>= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                if (rr < nr && gl == 0) epi.row(rid_s[r0 + rr - pa], sacc, red);
            }
        } else {
            Acc sacc = 0;
            for (int e = tid; e < nz; e += kBlock) sacc += prod[e];
            double t[1] = {static_cast<double>(sacc)};
            block_sum<1>(t);
            if (tid == 0) {
                piece_sum += t[0];
                if (kind == kLastPiece) {
                    epi.row(A.rowid[r0], static_cast<Acc>(piece_sum), red);
                    piece_sum = 0.0;
                }
            }
        }
        __syncthreads();      // stage s and prod are free again
        if (tid == 0 && j + kStages < nch) {
            fence_proxy_async_smem();
            issue_chunk<TA, Acc>(A, c0 + j + kStages, smem, s);
        }
    }
    if (!ok) {
        // a copy did not complete: flag it, let the outstanding copies land
        // (bounded) and leave without joining the grid sum
        if (tid == 0) {
            atomicExch(A.err, 1);
            for (int s = 0; s < kStages; ++s) mbar_wait(&bar[s], 0);
        }
        return;
    }
    double tot[NV];
    if (grid_sum<NV>(red, rb, Epi::kSite, tot)) {
        if (tid == 0) epi.finish(tot);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------

// length class of a row (0 for <= 1, else ceil(log2(len)))
inline int length_class(int32_t len) {
    int c = 0;
    while ((1 << c) < len) ++c;
    return c;
}

// Stored layout and chunks of one CSR matrix for a grid of `grid` CTAs.
template <typename V>
struct SpmvLayout {
    std::vector<int32_t> rowptr, col, rowid, kind, cta_item;
    std::vector<int32_t> chunk;       // 4 ints per chunk: r0, r1, k0, k1
    std::vector<V> val;
    int32_t nchunk = 0, grid = 1;
};

template <typename V>
inline SpmvLayout<V> spmv_layout(const std::vector<int32_t> &rp, const std::vector<int32_t> &cl,
                                 const std::vector<V> &vl, int grid) {
    SpmvLayout<V> L;
    const int32_t rows = (int32_t)rp.size() - 1;
    std::vector<int> cls(rows);
    int maxc = 0;
    for (int32_t r = 0; r < rows; ++r) {
        cls[r] = length_class(rp[r + 1] - rp[r]);
        maxc = std::max(maxc, cls[r]);
    }
    std::vector<int32_t> start(maxc + 2, 0);
    for (int32_t r = 0; r < rows; ++r) start[cls[r] + 1]++;
    for (int c = 0; c <= maxc; ++c) start[c + 1] += start[c];
    L.rowid.assign(rows + kPad, 0);
    std::vector<int32_t> pos(start.begin(), start.end() - 1);
    for (int32_t r = 0; r < rows; ++r) L.rowid[pos[cls[r]]++] = r;
    const size_t nnz = cl.size();
    L.rowptr.assign(rows + 1 + kPad, 0);
    L.col.assign(nnz + kPad, 0);
    L.val.assign(nnz + kPad, V(0));
    for (int32_t i = 0; i < rows; ++i) {
        const int32_t r = L.rowid[i], len = rp[r + 1] - rp[r];
        L.rowptr[i + 1] = L.rowptr[i] + len;
        std::copy(cl.begin() + rp[r], cl.begin() + rp[r + 1], L.col.begin() + L.rowptr[i]);
        std::copy(vl.begin() + rp[r], vl.begin() + rp[r + 1], L.val.begin() + L.rowptr[i]);
    }
    for (int k = 0; k < kPad; ++k) L.rowptr[rows + 1 + k] = L.rowptr[rows];
    // chunks; `cut_ok[c]`: a CTA range may start at chunk c
    std::vector<char> cut_ok;
    auto add = [&](int32_t r0, int32_t r1, int32_t k0, int32_t k1, int32_t kind, bool ok) {
        L.chunk.insert(L.chunk.end(), {r0, r1, k0, k1});
        L.kind.push_back(kind);
        cut_ok.push_back(ok ? 1 : 0);
    };
    int32_t i = 0;
    while (i < rows) {
        const int32_t k0 = L.rowptr[i], len = L.rowptr[i + 1] - k0;
        if (len > kChunkNnz) {
            for (int32_t k = k0; k < k0 + len; k += kChunkNnz) {
                const int32_t ke = std::min(k + kChunkNnz, k0 + len);
                add(i, i + 1, k, ke, ke == k0 + len ? kLastPiece : kPiece, k == k0);
            }
            ++i;
            continue;
        }
        const int c = cls[L.rowid[i]];
        int32_t e = i + 1;
        while (e < rows && cls[L.rowid[e]] == c && L.rowptr[e + 1] - k0 <= kChunkNnz && e - i < kChunkRows) ++e;
        add(i, e, k0, L.rowptr[e], kRun, true);
        i = e;
    }
    L.nchunk = (int32_t)L.kind.size();
    // contiguous chunk ranges per CTA, balanced by nonzeros (+ a per-chunk
    // cost), cut only where a row starts
    std::vector<int64_t> work(L.nchunk);
    for (int32_t c = 0; c < L.nchunk; ++c) work[c] = L.chunk[4 * c + 3] - L.chunk[4 * c + 2] + 64;
    const int64_t total = std::accumulate(work.begin(), work.end(), (int64_t)0);
    grid = std::max(1, std::min(grid, std::max(L.nchunk, 1)));
    L.cta_item.assign(grid + 1, L.nchunk);
    L.cta_item[0] = 0;
    int64_t acc = 0;
    int b = 1;
    for (int32_t c = 0; c < L.nchunk && b < grid; ++c) {
        acc += work[c];
        while (b < grid && acc * grid >= total * b) {
            int32_t cut = c + 1;
            while (cut < L.nchunk && !cut_ok[cut]) ++cut;
            L.cta_item[b++] = cut;
        }
    }
    for (int k = 1; k <= grid; ++k) L.cta_item[k] = std::max(L.cta_item[k], L.cta_item[k - 1]);
    L.grid = grid;
    return L;
}

}  // namespace scs
