// CSR sparse matrix-vector product with a fused per-row epilogue and a fused
// deterministic grid reduction, built for rows of power-law lengths.
//
// With uniformly random columns every product gathers one 4- or 8-byte
// entry of x from its own 32-byte L2 sector; on GB300 those gathers (not the
// HBM stream of the matrix) bound the product.  The kernel is therefore a
// flat, barrier-free launch that keeps as many independent gathers in
// flight as possible:
//
// Layout (setup, host): rows are stored grouped by length class (1, 2, 3-4,
// 5-8, ...; original order kept inside a class; `rowid` maps a stored row
// back to its matrix row, which is where the epilogue writes).  Each run of
// classes forms a region:
//   rows of up to 8 nonzeros: groups of L lanes per row (L = 1 up to 4
//     nonzeros, 2 up to 8), every lane holding a few nonzeros of one row;
//   rows of 9..256 nonzeros: tiles of whole rows with at most kTileNnz
//     nonzeros; a CTA gathers a tile's products into shared memory with
//     coalesced index loads (kTileNnz / kBlock independent gathers per
//     thread, one dependent chain per tile), then one thread per row sums
//     its products in order;
//   longer rows: a warp per row up to kWarpRow nonzeros, a CTA beyond.
// One launch covers all regions (grid-stride loops whose trip counts are
// uniform per warp or per CTA; region grids sized by their work).  Every
// thread accumulates the epilogue's reduction values over all its rows;
// each CTA joins one grid_sum at the end, whose last CTA runs the
// epilogue's finisher.
#pragma once

#include <type_traits>
#include <utility>

#include <stdint.h>

#include <algorithm>
#include <thread>
#include <vector>

#include "common.cuh"

namespace scs {

constexpr int kWarpRow = 4096;       // rows up to this length: one warp (longer: one CTA)
constexpr int kMaxRegions = 10;
constexpr int kWarpLoop = 33;        // region tag: one warp per row, looping over the row
constexpr int kCtaLanes = kBlock;    // region tag: one CTA per row
constexpr int kRowsPerLane = 2;      // rows a lane of a small group serves per step
constexpr int kTileLanes = 64;       // region tag: tiles of whole rows
constexpr int kTileNnz = 2048;       // nonzeros of a tile (at most)
constexpr int kTileMinRow = 9, kTileMaxRow = 256;   // row lengths served by tiles

// lanes per row for a row length: groups of 1..32 lanes give every lane at
// most 4 nonzeros; rows of 9..256 nonzeros go to tiles; longer rows loop with
// a warp, the longest with a CTA
inline int lanes_for(int32_t len) {
    if (len >= kTileMinRow && len <= kTileMaxRow) return kTileLanes;
    if (len <= 4) return 1;
    if (len <= 8) return 2;
    if (len <= 16) return 4;
    if (len <= 32) return 8;
    if (len <= 64) return 16;
    if (len <= 128) return 32;
    if (len <= kWarpRow) return kWarpLoop;
    return kCtaLanes;
}

struct SpmvRegions {
    int32_t n;                        // regions in use
    int32_t row0[kMaxRegions];        // stored rows [row0, row1)
    int32_t row1[kMaxRegions];
    int32_t lanes[kMaxRegions];       // 1, 2, 4, 8, 16, 32, kWarpLoop or kCtaLanes
    int32_t cta0[kMaxRegions + 1];    // CTAs [cta0[i], cta0[i+1]) serve region i
};

template <typename TA>
struct Csr {
    const int32_t *rowptr;   // rows + 1 (stored order)
    const int32_t *col;      // nnz
    const TA *val;           // nnz
    const int32_t *rowid;    // rows: matrix row of each stored row
    int32_t rows;
    SpmvRegions reg;
    const int32_t *tile_row; // ntiles + 1: first stored row of each tile
    int32_t ntiles;
    int32_t grid() const { return reg.cta0[reg.n]; }
};

// Epilogues may carry an elementwise task unrelated to the product's rows
// (side(cta, nctas)); the kernel runs it in every CTA after its rows.
template <typename E, typename = void>
struct HasSide : std::false_type {};
template <typename E>
struct HasSide<E, std::void_t<decltype(std::declval<E &>().side(0, 0))>> : std::true_type {};

template <typename Acc, typename TA, typename TX>
__device__ __forceinline__ Acc fmul(TA a, TX x) {
    return static_cast<Acc>(a) * static_cast<Acc>(x);
}

// Groups of L <= 32 lanes: a row of such a group has at most 4 L nonzeros,
// so each lane holds at most 4 of them and the loop is unrolled and
// predicated.  Each lane serves kRowsPerLane rows per step, and the
// epilogue's inputs are loaded (Epi::load) as soon as the row id is known, so
// the row pointers, matrix entries, epilogue inputs and gathers of several
// rows are in flight together.
template <int L, typename TA, typename TX, typename Acc, typename Epi>
__device__ __forceinline__ void spmv_small_groups(const Csr<TA> &A, const TX *__restrict__ x, Epi &epi,
                                                  Acc (&red)[Epi::NV], int r0, int r1, int cta, int nctas) {
    constexpr int G = 32 / L;                 // groups per warp
    constexpr int R = kRowsPerLane;
    const int lane = threadIdx.x & 31, g = lane / L, gl = lane % L;
    const int warp = cta * kWarps + (threadIdx.x >> 5), nwarps = nctas * kWarps;
    const int32_t *__restrict__ rowptr = A.rowptr;
    const int32_t *__restrict__ col = A.col;
    const TA *__restrict__ val = A.val;
    // the loop runs while any row of the warp's step exists, so the shuffles
    // below always see the whole warp
    for (int base = r0 + warp * G * R; base < r1; base += nwarps * G * R) {
        int k0[R], k1[R], rid[R];
        bool ok[R];
        typename Epi::In in[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            const int r = base + q * G + g;
            ok[q] = r < r1;
            k0[q] = ok[q] ? rowptr[r] : 0;
            k1[q] = ok[q] ? rowptr[r + 1] : 0;
            rid[q] = ok[q] ? A.rowid[r] : 0;
        }
#pragma unroll
        for (int q = 0; q < R; ++q)
            if (ok[q] && gl == 0) in[q] = epi.load(rid[q]);
        int c[R][4];
        TA v[R][4];
#pragma unroll
        for (int q = 0; q < R; ++q) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int k = k0[q] + gl + j * L;
                const bool has = k < k1[q];
                c[q][j] = has ? __ldcs(col + k) : 0;
                v[q][j] = has ? __ldcs(val + k) : TA(0);
            }
        }
        Acc acc[R];
#pragma unroll
        for (int q = 0; q < R; ++q) {
            acc[q] = 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (k0[q] + gl + j * L < k1[q]) acc[q] += fmul<Acc>(v[q][j], __ldg(x + c[q][j]));
        }
#pragma unroll
        for (int q = 0; q < R; ++q) {
#pragma unroll
            for (int o = L >> 1; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
            if (ok[q] && gl == 0) epi.row(rid[q], acc[q], in[q], red);
        }
    }
}

// a warp per row (rows of up to kWarpRow nonzeros)
template <typename TA, typename TX, typename Acc, typename Epi>
__device__ __forceinline__ void spmv_warp_rows(const Csr<TA> &A, const TX *__restrict__ x, Epi &epi,
                                               Acc (&red)[Epi::NV], int r0, int r1, int cta, int nctas) {
    const int lane = threadIdx.x & 31;
    const int warp = cta * kWarps + (threadIdx.x >> 5), nwarps = nctas * kWarps;
    const int32_t *__restrict__ col = A.col;
    const TA *__restrict__ val = A.val;
    for (int r = r0 + warp; r < r1; r += nwarps) {
        const int k0 = A.rowptr[r], k1 = A.rowptr[r + 1];
        const int rid = A.rowid[r];
        typename Epi::In in;
        if (lane == 0) in = epi.load(rid);
        Acc sacc = 0;
#pragma unroll 4
        for (int k = k0 + lane; k < k1; k += 32) sacc += fmul<Acc>(__ldcs(val + k), __ldg(x + __ldcs(col + k)));
        sacc = warp_sum(sacc);
        if (lane == 0) epi.row(rid, sacc, in, red);
    }
}

// tiles of whole rows (each of at most kTileNnz nonzeros, rows of at most
// kTileMaxRow): phase 1 gathers the tile's products into shared memory,
// phase 2 sums each row's products in order (one thread per row); the first
// row of each thread has its pointers and epilogue inputs loaded before the
// gathers
template <typename TA, typename TX, typename Acc, typename Epi>
__device__ __forceinline__ void spmv_tiles(const Csr<TA> &A, const TX *__restrict__ x, Epi &epi,
                                           Acc (&red)[Epi::NV], Acc *prod, int cta, int nctas) {
    const int32_t *__restrict__ rowptr = A.rowptr;
    const int32_t *__restrict__ col = A.col;
    const TA *__restrict__ val = A.val;
    const int tid = threadIdx.x;
    for (int t = cta; t < A.ntiles; t += nctas) {
        const int r0 = A.tile_row[t], r1 = A.tile_row[t + 1];
        const int nz0 = rowptr[r0], nz1 = rowptr[r1];
        const int rf = r0 + tid;
        int fa = 0, fb = 0, fid = 0;
        typename Epi::In fin{};
        if (rf < r1) {
            fa = rowptr[rf];
            fb = rowptr[rf + 1];
            fid = A.rowid[rf];
            fin = epi.load(fid);
        }
#pragma unroll
        for (int j = 0; j < kTileNnz / kBlock; ++j) {
            const int k = nz0 + tid + j * kBlock;
            if (k < nz1) prod[k - nz0] = fmul<Acc>(__ldcs(val + k), __ldg(x + __ldcs(col + k)));
        }
        __syncthreads();
        for (int r = rf; r < r1; r += kBlock) {
            int a = fa, b = fb, id = fid;
            typename Epi::In in = fin;
            if (r != rf) {
                a = rowptr[r];
                b = rowptr[r + 1];
                id = A.rowid[r];
                in = epi.load(id);
            }
            Acc sacc = 0;
            for (int k = a - nz0; k < b - nz0; ++k) sacc += prod[k];
            epi.row(id, sacc, in, red);
        }
        __syncthreads();
    }
}

template <typename TA, typename TX, typename Acc, typename Epi>
__global__ void __launch_bounds__(kBlock) spmv_kernel(Csr<TA> A, const TX *__restrict__ x, Epi epi, ReduceBuf rb) {
    __shared__ Acc tile_prod[kTileNnz];
    constexpr int NV = Epi::NV;
    static_assert(NV >= 1 && NV <= kMaxRed, "epilogue reduction width");
    if (epi.skip()) return;
    epi.begin();
    Acc red[NV];                  // per-thread reduction values, in the product's precision
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i] = Acc(0);
    const int b = blockIdx.x;
    int ri = 0;
    while (ri + 1 < A.reg.n && b >= A.reg.cta0[ri + 1]) ++ri;
    const int r0 = A.reg.row0[ri], r1 = A.reg.row1[ri];
    const int cta = b - A.reg.cta0[ri], nctas = A.reg.cta0[ri + 1] - A.reg.cta0[ri];
    switch (A.reg.lanes[ri]) {
        case 1: spmv_small_groups<1, TA, TX, Acc>(A, x, epi, red, r0, r1, cta, nctas); break;
        case 2: spmv_small_groups<2, TA, TX, Acc>(A, x, epi, red, r0, r1, cta, nctas); break;
        case 4: spmv_small_groups<4, TA, TX, Acc>(A, x, epi, red, r0, r1, cta, nctas); break;
        case 8: spmv_small_groups<8, TA, TX, Acc>(A, x, epi, red, r0, r1, cta, nctas); break;
        case 16: spmv_small_groups<16, TA, TX, Acc>(A, x, epi, red, r0, r1, cta, nctas); break;
        case 32: spmv_small_groups<32, TA, TX, Acc>(A, x, epi, red, r0, r1, cta, nctas); break;
        case kWarpLoop: spmv_warp_rows<TA, TX, Acc>(A, x, epi, red, r0, r1, cta, nctas); break;
        case kTileLanes: spmv_tiles<TA, TX, Acc>(A, x, epi, red, tile_prod, cta, nctas); break;
        default: {
            // one CTA per row
            const int tid = threadIdx.x;
            for (int r = r0 + cta; r < r1; r += nctas) {
                const int k0 = A.rowptr[r], k1 = A.rowptr[r + 1];
                const int rid = A.rowid[r];
                typename Epi::In in;
                if (tid == 0) in = epi.load(rid);
                Acc sacc = 0;
#pragma unroll 4
                for (int k = k0 + tid; k < k1; k += kBlock)
                    sacc += fmul<Acc>(__ldcs(A.val + k), __ldg(x + __ldcs(A.col + k)));
                double t[1] = {static_cast<double>(sacc)};
                block_sum<1>(t);
                if (tid == 0) epi.row(rid, static_cast<Acc>(t[0]), in, red);
            }
        }
    }
    // an epilogue's elementwise side task (if it has one), spread over the CTAs
    if constexpr (HasSide<Epi>::value) epi.side(b, gridDim.x);
    double redd[NV], tot[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) redd[i] = static_cast<double>(red[i]);
    if (grid_sum<NV>(redd, rb, Epi::kSite, tot)) {
        if (threadIdx.x == 0) epi.finish(tot);
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

// Stored layout of one CSR matrix and its regions for a grid of about `ctas` CTAs.
template <typename V>
struct SpmvLayout {
    std::vector<int32_t> rowptr, col, rowid;
    std::vector<V> val;
    SpmvRegions reg{};
    std::vector<int32_t> tile_row;   // tiles of the kTileLanes region (ntiles + 1 entries, or empty)
};

// threads: host threads for the copy into stored order (0: up to 16, one for
// matrices under 2^20 nonzeros); the layout is the same for any count.
// copy = false plans the layout only (rowid, rowptr, regions, tiles) and
// leaves col and val empty, for a gather of the rows on the device.
template <typename V>
inline SpmvLayout<V> spmv_layout(const std::vector<int32_t> &rp, const std::vector<int32_t> &cl,
                                 const std::vector<V> &vl, int ctas, int threads = 0, bool copy = true) {
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
    L.rowid.assign(rows, 0);
    std::vector<int32_t> pos(start.begin(), start.end() - 1);
    for (int32_t r = 0; r < rows; ++r) L.rowid[pos[cls[r]]++] = r;
    const size_t nnz = cl.size();
    L.rowptr.assign(rows + 1, 0);
    for (int32_t i = 0; i < rows; ++i) {
        const int32_t r = L.rowid[i];
        L.rowptr[i + 1] = L.rowptr[i] + (rp[r + 1] - rp[r]);
    }
    if (copy) {
        L.col.resize(nnz);
        L.val.resize(nnz);
        // the copies (one random jump per row into the source arrays) over ranges
        // of stored rows with about equal nonzeros
        auto copy_rows = [&](int32_t a, int32_t b) {
            for (int32_t i = a; i < b; ++i) {
                const int32_t r = L.rowid[i];
                std::copy(cl.begin() + rp[r], cl.begin() + rp[r + 1], L.col.begin() + L.rowptr[i]);
                std::copy(vl.begin() + rp[r], vl.begin() + rp[r + 1], L.val.begin() + L.rowptr[i]);
            }
        };
        int T = threads;
        if (T <= 0) {
            const unsigned hc = std::thread::hardware_concurrency();
            T = nnz < (size_t(1) << 20) ? 1 : (int)std::min<unsigned>(16, hc > 0 ? hc : 1);
        }
        std::vector<int32_t> cut(1, 0);
        for (int k = 1; k < T; ++k) {
            const int64_t target = (int64_t)nnz * k / T;
            const int32_t b = (int32_t)(std::lower_bound(L.rowptr.begin() + cut.back(), L.rowptr.end() - 1, target) -
                                        L.rowptr.begin());
            cut.push_back(std::max(cut.back(), std::min(b, rows)));
        }
        cut.push_back(rows);
        std::vector<std::thread> pool;
        size_t started = 1;                   // range 0 runs on this thread
        try {
            for (; started + 1 < cut.size(); ++started) pool.emplace_back(copy_rows, cut[started], cut[started + 1]);
        } catch (...) {
            // no more threads: the remaining ranges run here
        }
        copy_rows(cut[0], cut[1]);
        for (size_t k = started; k + 1 < cut.size(); ++k) copy_rows(cut[k], cut[k + 1]);
        for (auto &t : pool) t.join();
    }
    // regions: maximal runs of stored rows with the same lanes per row
    SpmvRegions &R = L.reg;
    R.n = 0;
    std::vector<int64_t> work;
    int32_t i = 0;
    while (i < rows && R.n < kMaxRegions) {
        const int lanes = lanes_for(L.rowptr[i + 1] - L.rowptr[i]);
        int32_t e = i + 1;
        while (e < rows && lanes_for(L.rowptr[e + 1] - L.rowptr[e]) == lanes) ++e;
        R.row0[R.n] = i;
        R.row1[R.n] = e;
        R.lanes[R.n] = lanes;
        // cost in warp steps (each step is one chain of dependent loads):
        // small groups serve 32 / lanes * kRowsPerLane rows per step, a
        // looping warp 128 nonzeros per step, a CTA 1024 per step of 8 warps
        int64_t steps = 0;
        if (lanes == kTileLanes) {
            // tiles: whole rows, at most kTileNnz nonzeros each; a tile costs
            // about as many warp steps as its nonzeros take in a looping warp
            L.tile_row.assign(1, i);
            int64_t acc = 0;
            for (int32_t r = i; r < e; ++r) {
                const int64_t len = L.rowptr[r + 1] - L.rowptr[r];
                if (acc + len > kTileNnz) {
                    L.tile_row.push_back(r);
                    acc = 0;
                }
                acc += len;
            }
            L.tile_row.push_back(e);
            steps = (int64_t)(L.tile_row.size() - 1) * (kTileNnz / 128);
        } else if (lanes <= 32) {
            steps = (e - i + (32 / lanes) * kRowsPerLane - 1) / ((32 / lanes) * kRowsPerLane);
        } else if (lanes == kWarpLoop) {
            for (int32_t r = i; r < e; ++r) steps += (L.rowptr[r + 1] - L.rowptr[r] + 127) / 128;
        } else {
            for (int32_t r = i; r < e; ++r) steps += kWarps * ((L.rowptr[r + 1] - L.rowptr[r] + 1023) / 1024);
        }
        work.push_back(steps);
        ++R.n;
        i = e;
    }
    if (R.n == 0) {                   // no rows: one empty region
        R.n = 1;
        R.row0[0] = R.row1[0] = 0;
        R.lanes[0] = 1;
        work.push_back(0);
    }
    // CTAs in proportion to the work, at least one per region and no more
    // than the region can use
    ctas = std::max(ctas, R.n);
    int64_t total = 0;
    for (int64_t wv : work) total += wv;
    R.cta0[0] = 0;
    for (int k = 0; k < R.n; ++k) {
        const int64_t nrows = R.row1[k] - R.row0[k];
        const int64_t rows_per_cta = R.lanes[k] == kCtaLanes ? 1 : R.lanes[k] == kWarpLoop ? kWarps : (int64_t)kBlock / R.lanes[k] * kRowsPerLane;
        const int64_t useful = R.lanes[k] == kTileLanes ? std::max<int64_t>(1, (int64_t)L.tile_row.size() - 1)
                                                        : std::max<int64_t>(1, (nrows + rows_per_cta - 1) / rows_per_cta);
        int64_t g = total > 0 ? (int64_t)((double)ctas * work[k] / total) : 1;
        g = std::max<int64_t>(1, std::min(g, useful));
        R.cta0[k + 1] = R.cta0[k] + (int32_t)g;
    }
    return L;
}

}  // namespace scs
