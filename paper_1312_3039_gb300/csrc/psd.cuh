// Projection of one PSD block onto the positive semidefinite cone, one CTA
// per block (Sec. 6.1: eigendecompose the symmetric matrix and zero its
// negative eigenvalues; the PSD cone is self-dual, so the same map serves
// K and K*).
//
// Storage: a block of order n is held in svec form, the lower triangle
// column by column with the off-diagonal entries times sqrt 2 (svec is then
// an isometry and the Euclidean projection in svec space is the Frobenius
// projection of the matrix).
//
// On the CTA the block is a dense ne x ne matrix, ne = n rounded up to a
// multiple of 4, or of 16 above order 48 (the padding rows and columns are
// zero and never rotated),
// row-major with leading dimension ld = ne + 1 (odd, so a column walk hits
// 32 different shared-memory banks).  Three such matrices X, V, W live in
// shared memory when they fit, else in a global scratch area of the CTA.
//
// Eigensolver: parallel cyclic Jacobi.  A sweep is ne - 1 rounds of the
// round-robin tournament; each round rotates ne/2 disjoint index pairs at
// once.  The rotation of pair (p, q) zeroes X[p][q] (the two-by-two
// symmetric Schur decomposition: tau = (x_qq - x_pp) / (2 x_pq),
// t = sign(tau) / (|tau| + sqrt(1 + tau^2)), c = 1 / sqrt(1 + t^2), s = t c).
// One thread applies both sides of the round's rotations to one 2 x 2 block
// of the lower triangle and mirrors it, so X stays exactly symmetric.  V
// accumulates the rotations (its columns become the eigenvectors).  A
// rotation is skipped when |x_pq| <= eps max(sqrt|x_pp x_qq|, ||X||_F / ne).
// The sweeps stop once ||off(X)||_F <= tol ||X||_F (tol 1e-6 in FP32, 1e-14
// in FP64): the projection onto the PSD cone is 1-Lipschitz, so taking the
// diagonal for the eigenvalues then moves the result by at most that much.
// The round's pairs and rotations sit in shared-memory tables, and each
// thread walks its 2 x 2 blocks (the lower triangle folded into an
// h/2 x (h + 1) rectangle) and its rows of V by increments, without integer
// division in the sweep.
//
// Above order 48 the same cyclic Jacobi runs blocked, so that most of its
// work is dense panel products instead of two CTA barriers per round: the
// ne indices are split into nb = ne / 8 blocks, and a block round pairs
// the blocks by the round-robin tournament (nb - 1 block rounds a sweep).
// For each block pair one warp rotates, in rounds of 8 disjoint pairs with
// the same rotation and skip rules, the index pairs of the 16 x 16
// subproblem S = X[R, R] (R: the pair's 16 indices) that the sweep has not
// rotated yet: all 120 in the first block round of a sweep (every block is
// in one of its pairs), the 64 pairs across the two blocks in the others,
// so a sweep rotates every index pair once.  The rotations accumulate in Q
// (S <- Q^T S Q); S is scaled exactly by a power of two to entries <= 1.
// The pairs of a block round are disjoint, so the round's transformation
// is J = Q_1 (+) Q_2 (+) ... on disjoint index sets: X <- J^T X J and
// V <- V J.  X stays symmetric: its diagonal block X[R_k, R_k] is the
// rotated S of pair k, and the block of two pairs k > l is
// Q_k^T X[R_k, R_l] Q_l (one warp, written with its mirror);
// V[:, R] <- V[:, R] Q is a column panel product, run one block round late
// by the warps without a subproblem where W has room for a second Q.  The
// stopping test is the same.
//
// Warm start (the iteration's blocks change little from one ADMM step to
// the next): V from the previous projection is first made orthogonal again
// by one Newton-Schulz step V <- V (3 I - V^T V) / 2, the input is rotated
// to X <- V^T X V, and Jacobi continues from that nearly diagonal matrix.
//
// Reconstruction P = V diag(max(lambda, 0)) V^T sums over the positive
// eigenvalues only.  With FP32 storage a block whose positive eigenvalues
// spread wider than `fp64_cond` (max >= fp64_cond min; 1e6 by default) is
// summed in FP64: in FP32 the terms of the small eigenvalues would drown in
// the rounding of the large ones.
#pragma once

#include <cuda_runtime.h>

#include <cfloat>
#include <cstdint>

#include "common.cuh"

namespace scs {

constexpr int kPsdThreads = 512;
constexpr int kPsdMaxSweeps = 40;
constexpr int kPsdMaxOrder = 1024;
constexpr int kPsdSmemCap = 232448;       // bytes of dynamic shared memory per CTA (opt-in maximum)

template <typename T> struct PsdEps;
template <> struct PsdEps<float> {
    static constexpr float v = FLT_EPSILON;
    static constexpr float off_tol = 1e-6f;
};
template <> struct PsdEps<double> {
    static constexpr double v = DBL_EPSILON;
    static constexpr double off_tol = 1e-14;
};

// Blocks of order above kPsdBlockedMin run the blocked eigensolver, which
// needs ne to be a multiple of 16 (pairs of 8-index blocks).
constexpr int kPsdBlockedMin = 48;
// ---- blocked Jacobi layout (orders above kPsdBlockedMin)
constexpr int kPsdB = 8;                    // indices per block
constexpr int kPsdR = 2 * kPsdB;            // order of a block pair's subproblem
constexpr int kPsdSld = kPsdR + 1;          // leading dimension of S
// per block pair in W: S (16 x 17); Q while the rounds run (16 x 17: a
// column of 16 rows hits 16 banks); Q for the panel products (16 x 16, rows
// 16-byte aligned for vector loads); the 8 rotation records of a round
constexpr int kPsdOffQi = kPsdR * kPsdSld;
constexpr int kPsdOffQ = 2 * kPsdR * kPsdSld;
constexpr int kPsdOffRot = kPsdOffQ + kPsdR * kPsdR;
constexpr int kPsdSlice = kPsdOffRot + 4 * kPsdB;

// Padded order: a multiple of 4, or of 16 above kPsdBlockedMin.
__host__ __device__ inline int psd_ne(int n) {
    return n < 4 ? 4 : n <= kPsdBlockedMin ? (n + 3) & ~3 : (n + 15) & ~15;
}
__host__ __device__ inline int psd_ld(int n) { return psd_ne(n) + 1; }
__host__ __device__ inline int64_t psd_svec_len(int n) { return (int64_t)n * (n + 1) / 2; }
__host__ __device__ inline int64_t psd_mat_elems(int n) { return (int64_t)psd_ne(n) * psd_ld(n); }

// Small per-CTA tables (shared memory in every mode), sized for order ne.
// Rotation of one index pair of the current round: J = [[c, s], [-s, c]] on
// columns (p, q), t = s / c; pq = p | q << 16.  One 16-byte (FP32) or 32-byte
// (FP64) record, read with one wide shared-memory load.
template <typename T>
struct alignas(16) PsdRot {
    T c, s, t;
    int pq;
};

template <typename T>
__host__ __device__ inline size_t psd_small_bytes(int ne) {
    const size_t h = ne / 2;
    size_t b = 32 * sizeof(double) + h * sizeof(PsdRot<T>) + ne * sizeof(T) + ne * sizeof(int) + 16 * sizeof(int);
    return (b + 15) & ~size_t(15);
}
template <typename T>
__host__ __device__ inline size_t psd_mats_bytes(int ne) {
    return 3 * (size_t)ne * (ne + 1) * sizeof(T);
}
// Entries the blocked sweeps of an order-ne block need for its block pairs'
// subproblems (slices with the second Q) and the warps' scratch tiles.
__host__ __device__ inline int64_t psd_sub_elems(int ne) {
    if (ne <= kPsdBlockedMin) return 0;
    const int64_t npairs = ne / (2 * kPsdB), nblk = npairs * (npairs - 1) / 2;
    const int64_t tiles = nblk < kPsdThreads / 32 ? nblk : kPsdThreads / 32;
    return npairs * (kPsdSlice + kPsdR * kPsdR) + tiles * kPsdR * kPsdSld;
}
// Whether, with X, V, W in global scratch, the subproblem area of the
// largest block (ne) fits in shared memory after the small tables.
template <typename T>
__host__ __device__ inline bool psd_sub_on_chip(int ne) {
    return ne > kPsdBlockedMin && psd_small_bytes<T>(ne) + psd_sub_elems(ne) * sizeof(T) <= (size_t)kPsdSmemCap;
}

// Dynamic shared memory of a launch whose largest block has order n_max;
// `smem_mats` tells whether the three matrices fit on chip (else the
// blocked sweeps' subproblem area does when it fits).
template <typename T>
inline size_t psd_smem_bytes(int n_max, bool &smem_mats) {
    const int ne = psd_ne(n_max);
    const size_t small = psd_small_bytes<T>(ne), mats = psd_mats_bytes<T>(ne);
    smem_mats = small + mats <= (size_t)kPsdSmemCap;
    if (smem_mats) return small + mats;
    return small + (psd_sub_on_chip<T>(ne) ? psd_sub_elems(ne) * sizeof(T) : 0);
}

// Pair k of round r of the round-robin tournament on ne players (ne even):
// player ne-1 stays, the others turn; every pair meets once in ne-1 rounds.
__device__ __forceinline__ void psd_pair(int r, int k, int ne, int &p, int &q) {
    const int m = ne - 1;
    if (k == 0) {
        p = r;
        q = m;
    } else {
        p = (r + k) % m;
        q = (r - k + m) % m;
    }
}

// Column j and row i of svec index s of an order-n block
// (column j starts at j n - j (j - 1) / 2).
__device__ __forceinline__ void psd_svec_ij(int64_t s, int n, int &i, int &j) {
    const double b = 2.0 * n + 1.0;
    int jj = static_cast<int>((b - sqrt(fmax(b * b - 8.0 * (double)s, 0.0))) * 0.5);
    if (jj < 0) jj = 0;
    if (jj > n - 1) jj = n - 1;
    auto start = [n](int c) { return (int64_t)c * n - (int64_t)c * (c - 1) / 2; };
    while (jj > 0 && start(jj) > s) --jj;
    while (jj < n - 1 && start(jj + 1) <= s) ++jj;
    j = jj;
    i = jj + static_cast<int>(s - start(jj));
}

template <typename T>
__device__ __forceinline__ T psd_block_sum(T v, double *red) {
    // red: at least blockDim.x / 32 slots; result valid in every thread
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[warp] = static_cast<double>(v);
    __syncthreads();
    T t = lane < nw ? static_cast<T>(red[lane]) : T(0);
    t = warp_sum(t);
    __syncthreads();
    return t;
}

// C = A^T B over the ne x ne output, inner index j in [0, kdim); rows of A
// and B are contiguous (leading dimension ld).  Each thread owns a TS x TS
// tile with rows ti + r ne/TS and columns tk + c ne/TS, so the lanes of a
// warp read consecutive words of B and broadcast words of A.  The products
// are bound by shared-memory loads (2 TS FMAs per 2 TS loads), so FP32
// takes 8 x 8 tiles where ne allows; FP64 keeps 4 x 4 (registers).
// epi(i, k, acc).
template <typename Acc, int TS, typename T, typename Epi>
__device__ __forceinline__ void psd_gemm_atb_tiles(const T *A, const T *B, int ne, int ld, int kdim, Epi epi) {
    const int q = ne / TS;
    const int tiles = q * q;
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
        const int ti = t / q, tk = t - ti * q;
        Acc acc[TS][TS];
#pragma unroll
        for (int r = 0; r < TS; ++r)
#pragma unroll
            for (int c = 0; c < TS; ++c) acc[r][c] = Acc(0);
        for (int j = 0; j < kdim; ++j) {
            const T *a = A + (size_t)j * ld, *b = B + (size_t)j * ld;
            Acc ar[TS], bc[TS];
#pragma unroll
            for (int r = 0; r < TS; ++r) ar[r] = static_cast<Acc>(a[ti + r * q]);
#pragma unroll
            for (int c = 0; c < TS; ++c) bc[c] = static_cast<Acc>(b[tk + c * q]);
#pragma unroll
            for (int r = 0; r < TS; ++r)
#pragma unroll
                for (int c = 0; c < TS; ++c) acc[r][c] = fma(ar[r], bc[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < TS; ++r)
#pragma unroll
            for (int c = 0; c < TS; ++c) epi(ti + r * q, tk + c * q, acc[r][c]);
    }
}
template <typename Acc, typename T, typename Epi>
__device__ __forceinline__ void psd_gemm_atb(const T *A, const T *B, int ne, int ld, int kdim, Epi epi) {
    if (sizeof(Acc) == 4 && ne % 8 == 0)
        psd_gemm_atb_tiles<Acc, 8>(A, B, ne, ld, kdim, epi);
    else
        psd_gemm_atb_tiles<Acc, 4>(A, B, ne, ld, kdim, epi);
}

// P[i][k] = sum over the positive eigenvalues j of lam_j Vt[j][i] Vt[j][k]
// (Vt = V^T, rows are eigenvectors), written into P (full square); tiles as
// in psd_gemm_atb.
template <typename Acc, int TS, typename T>
__device__ __forceinline__ void psd_reconstruct_tiles(const T *Vt, const T *lam, const int *pos, int npos, T *P,
                                                      int ne, int ld) {
    const int q = ne / TS;
    const int tiles = q * q;
    for (int t = threadIdx.x; t < tiles; t += blockDim.x) {
        const int ti = t / q, tk = t - ti * q;
        Acc acc[TS][TS];
#pragma unroll
        for (int r = 0; r < TS; ++r)
#pragma unroll
            for (int c = 0; c < TS; ++c) acc[r][c] = Acc(0);
        for (int jj = 0; jj < npos; ++jj) {
            const int j = pos[jj];
            const T *row = Vt + (size_t)j * ld;
            const Acc w = static_cast<Acc>(lam[j]);
            Acc ar[TS], bc[TS];
#pragma unroll
            for (int r = 0; r < TS; ++r) ar[r] = w * static_cast<Acc>(row[ti + r * q]);
#pragma unroll
            for (int c = 0; c < TS; ++c) bc[c] = static_cast<Acc>(row[tk + c * q]);
#pragma unroll
            for (int r = 0; r < TS; ++r)
#pragma unroll
                for (int c = 0; c < TS; ++c) acc[r][c] = fma(ar[r], bc[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < TS; ++r)
#pragma unroll
            for (int c = 0; c < TS; ++c) P[(size_t)(ti + r * q) * ld + tk + c * q] = static_cast<T>(acc[r][c]);
    }
}
template <typename Acc, typename T>
__device__ __forceinline__ void psd_reconstruct(const T *Vt, const T *lam, const int *pos, int npos, T *P, int ne,
                                                int ld) {
    if (sizeof(Acc) == 4 && ne % 8 == 0)
        psd_reconstruct_tiles<Acc, 8>(Vt, lam, pos, npos, P, ne, ld);
    else
        psd_reconstruct_tiles<Acc, 4>(Vt, lam, pos, npos, P, ne, ld);
}

// dst = src^T (ne x ne)
template <typename T>
__device__ __forceinline__ void psd_transpose(const T *src, T *dst, int ne, int ld) {
    for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) {
        const int i = e / ne, j = e - i * ne;
        dst[(size_t)j * ld + i] = src[(size_t)i * ld + j];
    }
}

template <typename T>
__device__ __forceinline__ void psd_identity(T *M, int ne, int ld) {
    for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) {
        const int i = e / ne, j = e - i * ne;
        M[(size_t)i * ld + j] = i == j ? T(1) : T(0);
    }
}

template <typename T>
struct PsdSmall {
    PsdRot<T> *rot;    // rotation of each pair of the current round
    T *lam;            // eigenvalues
    int *pos;          // indices of the positive eigenvalues
    int *flags;        // [0..1] rotation flags of alternate rounds, [2] count, [3] ill
    double *red;       // 32 block-reduction slots
};

template <typename T>
__device__ __forceinline__ PsdSmall<T> psd_small_tables(unsigned char *base, int ne) {
    PsdSmall<T> s;
    const int h = ne / 2;
    s.red = reinterpret_cast<double *>(base);
    s.rot = reinterpret_cast<PsdRot<T> *>(s.red + 32);
    s.lam = reinterpret_cast<T *>(s.rot + h);
    s.pos = reinterpret_cast<int *>(s.lam + ne);
    s.flags = s.pos + ne;
    return s;
}

// ||off(X)||_F^2 (valid in every thread)
template <typename T>
__device__ __forceinline__ T psd_off2(const T *X, int ne, int ld, double *red) {
    T o = T(0);
    int i = threadIdx.x / ne, j = threadIdx.x - (threadIdx.x / ne) * ne;
    const int di = blockDim.x / ne, dj = blockDim.x - di * ne;
    for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) {
        if (i != j) {
            const T x = X[(size_t)i * ld + j];
            o += x * x;
        }
        i += di;
        j += dj;
        if (j >= ne) {
            j -= ne;
            ++i;
        }
    }
    return psd_block_sum(o, red);
}

// Both sides of the round's rotations on the 2 x 2 block (i, j), i > j, of
// the lower triangle, mirrored into the upper one.
template <typename T>
__device__ __forceinline__ void psd_rotate_block(T *X, int ld, const PsdRot<T> &ri, const PsdRot<T> &rj) {
    const int pi = ri.pq & 0xffff, qi = ri.pq >> 16, pj = rj.pq & 0xffff, qj = rj.pq >> 16;
    const int o_pp = pi * ld + pj, o_pq = pi * ld + qj, o_qp = qi * ld + pj, o_qq = qi * ld + qj;
    const T a = X[o_pp], b = X[o_pq], c = X[o_qp], d = X[o_qq];
    // rows: J_i^T from the left
    const T a1 = ri.c * a - ri.s * c, b1 = ri.c * b - ri.s * d;
    const T c1 = ri.s * a + ri.c * c, d1 = ri.s * b + ri.c * d;
    // columns: J_j from the right
    const T a2 = rj.c * a1 - rj.s * b1, b2 = rj.s * a1 + rj.c * b1;
    const T c2 = rj.c * c1 - rj.s * d1, d2 = rj.s * c1 + rj.c * d1;
    X[o_pp] = a2;
    X[o_pq] = b2;
    X[o_qp] = c2;
    X[o_qq] = d2;
    X[pj * ld + pi] = a2;
    X[qj * ld + pi] = b2;
    X[pj * ld + qi] = c2;
    X[qj * ld + qi] = d2;
}

// Rotation of pair (p, q) that zeroes a_pq of the 2 x 2 block
// [[a_pp, a_pq], [a_pq, a_qq]]; the identity (s = 0) when
// |a_pq| <= max(eps sqrt|a_pp a_qq|, floor_abs).
template <typename T>
__device__ __forceinline__ PsdRot<T> psd_rotation(T app, T aqq, T apq, int p, int q, T eps, T floor_abs) {
    PsdRot<T> rt;
    rt.c = T(1);
    rt.s = T(0);
    rt.t = T(0);
    rt.pq = p | (q << 16);
    const T thr = fmax(eps * sqrt(fabs(app * aqq)), floor_abs);
    if (fabs(apq) > thr) {
        const T tau = (aqq - app) / (T(2) * apq);
        const T at = fabs(tau);
        const T root = at > T(1) ? at * sqrt(T(1) + (T(1) / at) / at) : sqrt(T(1) + at * at);
        T t = T(1) / (at + root);
        if (tau < T(0)) t = -t;
        rt.c = T(1) / sqrt(T(1) + t * t);
        rt.s = t * rt.c;
        rt.t = t;
    }
    return rt;
}

// The same rotation with a shorter FP32 dependency chain, for the blocked
// sweeps' subproblems, whose entries are scaled to magnitude <= 1 (exactly,
// by a power of two): the skip test compares squares; with d = a_qq - a_pp,
// t = 2 a_pq sgn(d) / (|d| + sqrt(d^2 + 4 a_pq^2)) is the root of the
// IEEE formula's t = sgn(tau) / (|tau| + sqrt(1 + tau^2)), from rsqrtf and
// a fast reciprocal (an inexact t still gives an exact rotation, and only
// perturbs the zeroed a_pq by about eps |a_pq|); c = 1 / sqrt(1 + t^2) from
// rsqrtf refined by one Newton-Raphson step (y <- y (3 - x y^2) / 2), so
// c^2 + s^2 = 1 to about an ulp.  FP64 keeps the IEEE path.
template <typename T>
__device__ __forceinline__ PsdRot<T> psd_rotation_fast(T app, T aqq, T apq, int p, int q, T eps, T floor_abs) {
    return psd_rotation(app, aqq, apq, p, q, eps, floor_abs);
}
template <>
__device__ __forceinline__ PsdRot<float> psd_rotation_fast<float>(float app, float aqq, float apq, int p, int q,
                                                                  float eps, float floor_abs) {
    PsdRot<float> rt;
    rt.c = 1.f;
    rt.s = 0.f;
    rt.t = 0.f;
    rt.pq = p | (q << 16);
    const float apq2 = apq * apq;
    if (apq2 > fmaxf(eps * eps * fabsf(app * aqq), floor_abs * floor_abs)) {
        const float d = aqq - app, ad = fabsf(d);
        const float r2 = fmaf(4.f * apq, apq, d * d);
        float t = __fdividef(2.f * apq, ad + r2 * rsqrtf(r2));
        if (d < 0.f) t = -t;
        const float x = fmaf(t, t, 1.f);
        float c = rsqrtf(x);
        c = c * (1.5f - 0.5f * x * c * c);
        rt.c = c;
        rt.s = t * c;
        rt.t = t;
    }
    return rt;
}

// Cyclic Jacobi on the symmetric X (ne x ne), accumulating V <- V J on the
// first nrows_v rows of V.  Returns the number of sweeps run.
//
// Work split (fixed for the whole call, so the sweep has no integer
// division): the lower 2 x 2 blocks (i >= j) are folded into h/2 rows of
// h + 1 blocks (fold row r holds triangle rows r and h - 1 - r); `tpr`
// threads share a fold row, taking every tpr-th block of it.  Each V row is
// owned by threads that take every ks-th pair.
template <typename T>
__device__ __forceinline__ int psd_jacobi(T *X, T *V, int ne, int ld, int nrows_v, const PsdSmall<T> &sm, T fro) {
    const int h = ne >> 1;
    const int nt = blockDim.x, tid = threadIdx.x;
    const T eps = PsdEps<T>::v;
    const T floor_abs = eps * fro / static_cast<T>(ne);
    const T stop2 = (PsdEps<T>::off_tol * fro) * (PsdEps<T>::off_tol * fro);
    const int nfold = h >> 1, rw = h + 1;
    const int tpr = nt / nfold < 1 ? 1 : nt / nfold;
    const int frow = tid / tpr, fcol0 = tid - frow * tpr;
    const bool has_fold = frow < nfold;
    const int ia = frow, ib = h - 1 - frow;          // the two triangle rows of this fold row
    // V: rows [0, nrows_v) x pairs [0, h)
    const bool v_small = nrows_v <= nt;
    const int ks = v_small ? nt / nrows_v : 1;
    const int vrow = v_small ? tid % nrows_v : tid, vk0 = v_small ? tid / nrows_v : 0;
    if (psd_off2(X, ne, ld, sm.red) <= stop2) return 0;
    if (tid == 0) {
        sm.flags[0] = 0;
        sm.flags[1] = 0;
    }
    __syncthreads();
    int sweeps = 0, round = 0;
    while (sweeps < kPsdMaxSweeps) {
        ++sweeps;
        bool any = false;
        for (int r = 0; r < ne - 1; ++r, ++round) {
            int *fl = sm.flags + (round & 1);
            for (int k = tid; k < h; k += nt) {
                int p, q;
                psd_pair(r, k, ne, p, q);
                const PsdRot<T> rt = psd_rotation(X[p * ld + p], X[q * ld + q], X[p * ld + q], p, q, eps, floor_abs);
                if (rt.s != T(0)) *fl = 1;
                sm.rot[k] = rt;
            }
            if (tid == 0) sm.flags[(round + 1) & 1] = 0;
            __syncthreads();
            const bool rot = *fl != 0;
            any = any || rot;
            if (rot) {
                if (has_fold) {
                    const PsdRot<T> ra = sm.rot[ia], rb = sm.rot[ib];
                    for (int cc = fcol0; cc < rw; cc += tpr) {
                        const bool lo = cc <= frow;
                        const PsdRot<T> &ri = lo ? ra : rb;
                        const int j = lo ? cc : cc - frow - 1;
                        const int i = lo ? ia : ib;
                        const PsdRot<T> rj = sm.rot[j];
                        if (ri.s == T(0) && rj.s == T(0)) continue;
                        if (i == j) {
                            const int p = ri.pq & 0xffff, q = ri.pq >> 16;
                            const T apq = X[p * ld + q];
                            X[p * ld + p] -= ri.t * apq;
                            X[q * ld + q] += ri.t * apq;
                            X[p * ld + q] = T(0);
                            X[q * ld + p] = T(0);
                        } else {
                            psd_rotate_block(X, ld, ri, rj);
                        }
                    }
                }
                // V <- V J (columns p, q of every row)
                if (v_small) {
                    if (vk0 < ks) {
                        T *vr = V + vrow * ld;
                        for (int k = vk0; k < h; k += ks) {
                            const PsdRot<T> rk = sm.rot[k];
                            if (rk.s == T(0)) continue;
                            const int p = rk.pq & 0xffff, q = rk.pq >> 16;
                            const T vp = vr[p], vq = vr[q];
                            vr[p] = rk.c * vp - rk.s * vq;
                            vr[q] = rk.s * vp + rk.c * vq;
                        }
                    }
                } else {
                    for (int row = tid; row < nrows_v; row += nt) {
                        T *vr = V + (size_t)row * ld;
                        for (int k = 0; k < h; ++k) {
                            const PsdRot<T> rk = sm.rot[k];
                            if (rk.s == T(0)) continue;
                            const int p = rk.pq & 0xffff, q = rk.pq >> 16;
                            const T vp = vr[p], vq = vr[q];
                            vr[p] = rk.c * vp - rk.s * vq;
                            vr[q] = rk.s * vp + rk.c * vq;
                        }
                    }
                }
            }
            __syncthreads();
        }
        if (!any || psd_off2(X, ne, ld, sm.red) <= stop2) break;
    }
    return sweeps;
}

// ---- blocked Jacobi (orders above kPsdBlockedMin)

// Index of the subproblem's local index a (0..15) in the block pair (bI, bJ).
__device__ __forceinline__ int psd_sub_index(int a, int bI, int bJ) {
    return a < kPsdB ? bI * kPsdB + a : bJ * kPsdB + (a - kPsdB);
}

// Four consecutive entries from a 16-byte aligned shared or global address.
__device__ __forceinline__ void psd_load4(const float *p, float (&v)[4]) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
__device__ __forceinline__ void psd_load4(const double *p, double (&v)[4]) {
    const double2 a = *reinterpret_cast<const double2 *>(p), b = *reinterpret_cast<const double2 *>(p + 2);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

// Rounds of cyclic Jacobi, by one warp, on the 16 x 16 symmetric S
// (leading dimension kPsdSld), accumulating Q <- Q J (leading dimension
// kPsdSld).  full: one sweep over
// all 120 index pairs (15 round-robin rounds); else the 64 pairs across the
// two blocks (8 rounds, pairs (a, 8 + (a + m) mod 8) in round m).  Returns
// (in every lane) whether any rotation was applied.
template <typename T>
__device__ __forceinline__ bool psd_sub_sweep(T *S, T *Q, PsdRot<T> *rot, int lane, bool full, T eps, T floor_abs) {
    constexpr int h = kPsdB;
    bool any = false;
    const int nrounds = full ? kPsdR - 1 : kPsdB;
    // this lane's 2 x 2 block (i, j), i > j, of the round's 8 pairs
    // (lanes 0..27; lane = i (i - 1) / 2 + j); the pairs' own blocks are
    // updated by the lanes that compute their rotations
    const int bi = lane < h * (h - 1) / 2 ? static_cast<int>((1.f + sqrtf(8.f * lane + 1.f)) * 0.5f) : 0;
    const int bj = lane - bi * (bi - 1) / 2;
    for (int ir = 0; ir < nrounds; ++ir) {
        bool mine = false;
        if (lane < h) {
            int p, q;
            if (full) {
                psd_pair(ir, lane, kPsdR, p, q);
            } else {
                p = lane;
                q = kPsdB + ((lane + ir) & (kPsdB - 1));
            }
            const T app = S[p * kPsdSld + p], aqq = S[q * kPsdSld + q], apq = S[p * kPsdSld + q];
            const PsdRot<T> rt = psd_rotation_fast(app, aqq, apq, p, q, eps, floor_abs);
            mine = rt.s != T(0);
            rot[lane] = rt;
            if (mine) {
                // the pair's own block: zero s_pq exactly
                S[p * kPsdSld + p] = app - rt.t * apq;
                S[q * kPsdSld + q] = aqq + rt.t * apq;
                S[p * kPsdSld + q] = T(0);
                S[q * kPsdSld + p] = T(0);
            }
        }
        const bool round_any = __any_sync(0xffffffffu, mine);
        __syncwarp();
        if (!round_any) continue;
        any = true;
        // both sides on the lower 2 x 2 blocks of two different pairs, mirrored
        if (lane < h * (h - 1) / 2) {
            const PsdRot<T> ri = rot[bi], rj = rot[bj];
            if (ri.s != T(0) || rj.s != T(0)) {
                const int pi = ri.pq & 0xffff, qi = ri.pq >> 16, pj = rj.pq & 0xffff, qj = rj.pq >> 16;
                const T a = S[pi * kPsdSld + pj], b = S[pi * kPsdSld + qj];
                const T c = S[qi * kPsdSld + pj], d = S[qi * kPsdSld + qj];
                const T a1 = ri.c * a - ri.s * c, b1 = ri.c * b - ri.s * d;
                const T c1 = ri.s * a + ri.c * c, d1 = ri.s * b + ri.c * d;
                const T a2 = rj.c * a1 - rj.s * b1, b2 = rj.s * a1 + rj.c * b1;
                const T c2 = rj.c * c1 - rj.s * d1, d2 = rj.s * c1 + rj.c * d1;
                S[pi * kPsdSld + pj] = a2;
                S[pi * kPsdSld + qj] = b2;
                S[qi * kPsdSld + pj] = c2;
                S[qi * kPsdSld + qj] = d2;
                S[pj * kPsdSld + pi] = a2;
                S[qj * kPsdSld + pi] = b2;
                S[pj * kPsdSld + qi] = c2;
                S[qj * kPsdSld + qi] = d2;
            }
        }
        // Q <- Q J: lane owns row lane % 16 and every other pair (disjoint
        // columns: all loads first)
        {
            T *qr = Q + (lane & (kPsdR - 1)) * kPsdSld;
            PsdRot<T> rk[h / 2];
            T vp[h / 2], vq[h / 2];
#pragma unroll
            for (int m = 0; m < h / 2; ++m) {
                rk[m] = rot[(lane >> 4) + 2 * m];
                vp[m] = qr[rk[m].pq & 0xffff];
                vq[m] = qr[rk[m].pq >> 16];
            }
#pragma unroll
            for (int m = 0; m < h / 2; ++m) {
                qr[rk[m].pq & 0xffff] = rk[m].c * vp[m] - rk[m].s * vq[m];
                qr[rk[m].pq >> 16] = rk[m].s * vp[m] + rk[m].c * vq[m];
            }
        }
        __syncwarp();
    }
    return any;
}

// Blocked cyclic Jacobi on the symmetric X (ne x ne, ne a multiple of 16),
// accumulating V <- V J on its first nrows_v rows; W (wcap entries, 16-byte
// aligned: the block's own W of ne (ne + 1) entries, or a shared-memory area
// of psd_sub_elems(ne)) holds the block pairs' subproblems (ne / 16 slices)
// and 16 x 17 scratch tiles for the warps that compute the off-diagonal
// blocks, as many as fit (at least 3 for ne >= 64).  Returns the number of
// sweeps run.
// V[row, R] <- sum_a V[row, R_a] Q[a][r] for every block pair of block
// round br (Q at offset qoff of each pair's slice of W), over the first
// nrows_v rows; units (pair, row group) from t0 in steps of tstride.
template <typename T, int CPT>
__device__ __forceinline__ void psd_v_panel(T *V, const T *W, int slice, int qoff, int ld, int nb, int npairs, int br,
                                            int nrows_v, int t0, int tstride) {
    const int gv = (nrows_v + CPT - 1) / CPT;
    for (int u = t0; u < npairs * gv; u += tstride) {
        const int k = u / gv, g0 = u - k * gv;
        int bI, bJ;
        psd_pair(br, k, nb, bI, bJ);
        const T *Q = W + (size_t)k * slice + qoff;
        T acc[kPsdR][CPT];
#pragma unroll
        for (int r = 0; r < kPsdR; ++r)
#pragma unroll
            for (int m = 0; m < CPT; ++m) acc[r][m] = T(0);
#pragma unroll 4
        for (int a = 0; a < kPsdR; ++a) {
            const int ga = psd_sub_index(a, bI, bJ);
            T y[CPT];
#pragma unroll
            for (int m = 0; m < CPT; ++m) {
                const int row = g0 + m * gv;
                y[m] = row < nrows_v ? V[(size_t)row * ld + ga] : T(0);
            }
#pragma unroll
            for (int r4 = 0; r4 < kPsdR; r4 += 4) {
                T q[4];
                psd_load4(Q + a * kPsdR + r4, q);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int m = 0; m < CPT; ++m) acc[r4 + r][m] = fma(y[m], q[r], acc[r4 + r][m]);
            }
        }
#pragma unroll
        for (int m = 0; m < CPT; ++m) {
            const int row = g0 + m * gv;
            if (row >= nrows_v) continue;
#pragma unroll
            for (int r = 0; r < kPsdR; ++r) V[(size_t)row * ld + psd_sub_index(r, bI, bJ)] = acc[r][m];
        }
    }
}

template <typename T>
__device__ __forceinline__ int psd_jacobi_blocked(T *X, T *V, T *W, int64_t wcap, int ne, int ld, int nrows_v,
                                                  const PsdSmall<T> &sm, T fro) {
    constexpr int CPT = sizeof(T) == 4 ? 2 : 1;     // columns (rows) per thread in the panel products
    const int nb = ne / kPsdB, npairs = nb / 2;
    const int nt = blockDim.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const T eps = PsdEps<T>::v;
    const T floor_abs = eps * fro / static_cast<T>(ne);
    const T stop2 = (PsdEps<T>::off_tol * fro) * (PsdEps<T>::off_tol * fro);
    // subproblems scaled by sc = 2^-e, fro in [2^(e-1), 2^e): entries <= 1
    int fe = 0;
    frexp(fro, &fe);
    const T sc = ldexp(T(1), -fe), isc = ldexp(T(1), fe);
    // V update one block round late on the warps without a subproblem when
    // there are such warps and W holds a second copy of every pair's Q
    const bool defer = npairs < nw && npairs * (kPsdSlice + kPsdR * kPsdR) + kPsdR * kPsdSld <= wcap;
    const int slice = defer ? kPsdSlice + kPsdR * kPsdR : kPsdSlice;
    int vpend = -1;            // block round whose V update is pending
    if (psd_off2(X, ne, ld, sm.red) <= stop2) return 0;
    if (tid == 0) {
        sm.flags[0] = 0;
        sm.flags[1] = 0;
    }
    __syncthreads();
    int sweeps = 0, round = 0;
    while (sweeps < kPsdMaxSweeps) {
        ++sweeps;
        bool any = false;
        for (int br = 0; br < nb - 1; ++br, ++round) {
            int *fl = sm.flags + (round & 1);
            // subproblems: one warp per block pair
            for (int k = warp; k < npairs; k += nw) {
                int bI, bJ;
                psd_pair(br, k, nb, bI, bJ);
                T *S = W + (size_t)k * slice, *Qi = S + kPsdOffQi, *Q = S + kPsdOffQ;
                PsdRot<T> *rot = reinterpret_cast<PsdRot<T> *>(S + kPsdOffRot);
                for (int e = lane; e < kPsdR * kPsdR; e += 32) {
                    const int a = e >> 4, b = e & (kPsdR - 1);
                    const int ga = psd_sub_index(a, bI, bJ), gb = psd_sub_index(b, bI, bJ);
                    // the lower triangle of X, so S is exactly symmetric;
                    // scaled by a power of two to magnitude <= 1
                    S[a * kPsdSld + b] = sc * (ga >= gb ? X[(size_t)ga * ld + gb] : X[(size_t)gb * ld + ga]);
                    Qi[a * kPsdSld + b] = a == b ? T(1) : T(0);
                }
                __syncwarp();
                // the first block round of a sweep also covers the pairs
                // inside each block (every block is in one of its pairs)
                if (psd_sub_sweep(S, Qi, rot, lane, br == 0, eps, floor_abs * sc) && lane == 0) *fl = 1;
                for (int e = lane; e < kPsdR * kPsdR; e += 32) Q[e] = Qi[(e >> 4) * kPsdSld + (e & (kPsdR - 1))];
            }
            if (vpend >= 0 && warp >= npairs)
                psd_v_panel<T, CPT>(V, W, slice, kPsdSlice, ld, nb, npairs, vpend, nrows_v, tid - npairs * 32,
                                    nt - npairs * 32);
            if (tid == 0) sm.flags[(round + 1) & 1] = 0;
            __syncthreads();
            const bool rot = *fl != 0;
            any = any || rot;
            if (rot) {
                // X <- J^T X J, symmetric: the diagonal block of each pair is
                // its rotated S; the block of pairs k > l is
                // Q_k^T X[R_k, R_l] Q_l (one warp: T = X[R_k, R_l] Q_l into
                // the warp's scratch, then Q_k^T T), written with its mirror
                const int nblk = npairs * (npairs - 1) / 2;
                T *scratch = W + (size_t)npairs * slice;
                // warps with a scratch tile in W (at least 3: ne >= 64)
                const int nsw = static_cast<int>(min(static_cast<int64_t>(min(nw, nblk)),
                                                     (wcap - npairs * slice) / (kPsdR * kPsdSld)));
                for (int t = warp; warp < nsw && t < nblk; t += nsw) {
                    int k = 1;
                    while ((k + 1) * k / 2 <= t) ++k;       // t = k (k - 1) / 2 + l, l < k
                    const int l = t - k * (k - 1) / 2;
                    int kI, kJ, lI, lJ;
                    psd_pair(br, k, nb, kI, kJ);
                    psd_pair(br, l, nb, lI, lJ);
                    const T *Qk = W + (size_t)k * slice + kPsdOffQ;
                    const T *Ql = W + (size_t)l * slice + kPsdOffQ;
                    T *Tw = scratch + (size_t)warp * kPsdR * kPsdSld;
                    const int i = lane & (kPsdR - 1), c0 = (lane >> 4) * kPsdB;
                    // T[i][c] = sum_b X[R_k(i), R_l(b)] Q_l[b][c], c in [c0, c0 + 8)
                    {
                        const T *xr = X + (size_t)psd_sub_index(i, kI, kJ) * ld;
                        T acc[kPsdB];
#pragma unroll
                        for (int c = 0; c < kPsdB; ++c) acc[c] = T(0);
#pragma unroll 4
                        for (int b = 0; b < kPsdR; ++b) {
                            const T x = xr[psd_sub_index(b, lI, lJ)];
                            T q[4], q2[4];
                            psd_load4(Ql + b * kPsdR + c0, q);
                            psd_load4(Ql + b * kPsdR + c0 + 4, q2);
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                acc[c] = fma(x, q[c], acc[c]);
                                acc[c + 4] = fma(x, q2[c], acc[c + 4]);
                            }
                        }
#pragma unroll
                        for (int c = 0; c < kPsdB; ++c) Tw[i * kPsdSld + c0 + c] = acc[c];
                    }
                    __syncwarp();
                    // Y[r][c] = sum_i Q_k[i][r] T[i][c]: lane owns column c = lane % 16
                    // and rows r in [c0, c0 + 8)
                    {
                        const int c = i, r0 = c0;
                        T acc[kPsdB];
#pragma unroll
                        for (int r = 0; r < kPsdB; ++r) acc[r] = T(0);
#pragma unroll 4
                        for (int ii = 0; ii < kPsdR; ++ii) {
                            const T tv = Tw[ii * kPsdSld + c];
                            T q[4], q2[4];
                            psd_load4(Qk + ii * kPsdR + r0, q);
                            psd_load4(Qk + ii * kPsdR + r0 + 4, q2);
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                acc[r] = fma(q[r], tv, acc[r]);
                                acc[r + 4] = fma(q2[r], tv, acc[r + 4]);
                            }
                        }
                        const int gc = psd_sub_index(c, lI, lJ);
#pragma unroll
                        for (int r = 0; r < kPsdB; ++r) {
                            const int gr = psd_sub_index(r0 + r, kI, kJ);
                            X[(size_t)gr * ld + gc] = acc[r];
                            X[(size_t)gc * ld + gr] = acc[r];
                        }
                    }
                    __syncwarp();
                }
                // diagonal blocks
                for (int e = tid; e < npairs * kPsdR * kPsdR; e += nt) {
                    const int k = e >> 8, a = (e >> 4) & (kPsdR - 1), b = e & (kPsdR - 1);
                    int bI, bJ;
                    psd_pair(br, k, nb, bI, bJ);
                    X[(size_t)psd_sub_index(a, bI, bJ) * ld + psd_sub_index(b, bI, bJ)] =
                        isc * W[(size_t)k * slice + a * kPsdSld + b];
                }
                if (defer) {
                    // keep this round's Q for the V update, which the warps
                    // without a subproblem run during the next block round
                    for (int e = tid; e < npairs * kPsdR * kPsdR; e += nt) {
                        const int k = e >> 8;
                        W[(size_t)k * slice + kPsdSlice + (e & 255)] = W[(size_t)k * slice + kPsdOffQ + (e & 255)];
                    }
                } else {
                    psd_v_panel<T, CPT>(V, W, slice, kPsdOffQ, ld, nb, npairs, br, nrows_v, tid, nt);
                }
            }
            vpend = defer && rot ? br : -1;
            __syncthreads();
        }
        if (!any || psd_off2(X, ne, ld, sm.red) <= stop2) break;
    }
    if (vpend >= 0) {
        psd_v_panel<T, CPT>(V, W, slice, kPsdSlice, ld, nb, npairs, vpend, nrows_v, tid, nt);
        __syncthreads();
    }
    return sweeps;
}

// Statistics of the projections (device counters, summed with atomics).
struct PsdStats {
    unsigned long long *sweeps;     // Jacobi sweeps
    unsigned long long *fp64;       // blocks reconstructed in FP64
    unsigned long long *calls;      // block projections
};

// Project one block.  io.in(s) returns svec entry s of the point to project;
// io.out(s, p) receives svec entry s of the projection.  X, V, W: matrix
// storage (shared or global); Vkeep: where the eigenvectors persist between
// calls (nullptr: cold start, nothing kept; equal to V: kept in place);
// Wsub: psd_sub_elems(ne) entries of shared memory for the blocked sweeps'
// subproblems when X, V, W are in global memory (nullptr: they use W).
template <typename T, typename IO>
__device__ __forceinline__ void psd_project_block(IO &io, int n, T *X, T *V, T *W, T *Vkeep, const PsdSmall<T> &sm,
                                  PsdStats stats, double fp64_cond, T *Wsub = nullptr) {
    const int ne = psd_ne(n), ld = ne + 1;
    const int64_t len = psd_svec_len(n);
    const T isq2 = T(0.70710678118654752440);
    const bool warm = Vkeep != nullptr;
    // ---- V: the previous eigenvectors, made orthogonal again, or I
    if (warm) {
        if (Vkeep != V)
            for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) {
                const int i = e / ne, j = e - i * ne;
                V[(size_t)i * ld + j] = Vkeep[(size_t)i * ld + j];
            }
        __syncthreads();
        // W = V^T V; H = (3 I - W) / 2 in W; X = V^T; V = X^T H = V H
        psd_gemm_atb<T>(V, V, ne, ld, ne, [&](int i, int k, T acc) {
            W[(size_t)i * ld + k] = (i == k ? T(1.5) : T(0)) - T(0.5) * acc;
        });
        psd_transpose(V, X, ne, ld);
        __syncthreads();
        psd_gemm_atb<T>(X, W, ne, ld, ne, [&](int i, int k, T acc) { V[(size_t)i * ld + k] = acc; });
        __syncthreads();
    } else {
        psd_identity(V, ne, ld);
    }
    // ---- X = smat(input), zero padding
    for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) {
        const int i = e / ne, j = e - i * ne;
        if (i >= n || j >= n) X[(size_t)i * ld + j] = T(0);
    }
    for (int64_t s = threadIdx.x; s < len; s += blockDim.x) {
        int i, j;
        psd_svec_ij(s, n, i, j);
        T x = io.in(s);
        if (i != j) x *= isq2;
        X[(size_t)i * ld + j] = x;
        X[(size_t)j * ld + i] = x;
    }
    __syncthreads();
    if (warm) {
        // X <- V^T X V, then mirrored from its lower triangle
        psd_gemm_atb<T>(X, V, ne, ld, ne, [&](int i, int k, T acc) { W[(size_t)i * ld + k] = acc; });
        __syncthreads();
        psd_gemm_atb<T>(V, W, ne, ld, ne, [&](int i, int k, T acc) { X[(size_t)i * ld + k] = acc; });
        __syncthreads();
        for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) {
            const int i = e / ne, j = e - i * ne;
            if (i < j) X[(size_t)i * ld + j] = X[(size_t)j * ld + i];
        }
        __syncthreads();
    }
    // ---- Frobenius norm, Jacobi
    T f2 = T(0);
    for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) {
        const int i = e / ne, j = e - i * ne;
        const T x = X[(size_t)i * ld + j];
        f2 += x * x;
    }
    f2 = psd_block_sum(f2, sm.red);
    const int sweeps = ne > kPsdBlockedMin
                           ? psd_jacobi_blocked(X, V, Wsub ? Wsub : W, Wsub ? psd_sub_elems(ne) : (int64_t)ne * ld, ne,
                                                ld, n, sm, sqrt(f2))
                           : psd_jacobi(X, V, ne, ld, n, sm, sqrt(f2));
    // ---- eigenvalues, positive set, conditioning
    for (int j = threadIdx.x; j < ne; j += blockDim.x) sm.lam[j] = X[(size_t)j * ld + j];
    __syncthreads();
    if (threadIdx.x == 0) {
        int np = 0;
        T pmax = T(0), pmin = T(INFINITY);
        for (int j = 0; j < n; ++j) {
            const T l = sm.lam[j];
            if (l > T(0)) {
                sm.pos[np++] = j;
                pmax = fmax(pmax, l);
                pmin = fmin(pmin, l);
            }
        }
        sm.flags[2] = np;
        sm.flags[3] = (sizeof(T) < 8 && np > 0 && static_cast<double>(pmax) >= fp64_cond * static_cast<double>(pmin))
                          ? 1 : 0;
        if (stats.calls) {
            atomicAdd(stats.calls, 1ull);
            atomicAdd(stats.sweeps, (unsigned long long)sweeps);
            if (sm.flags[3]) atomicAdd(stats.fp64, 1ull);
        }
    }
    psd_transpose(V, W, ne, ld);       // W = V^T: eigenvectors as rows
    __syncthreads();
    const int npos = sm.flags[2];
    if (sm.flags[3])
        psd_reconstruct<double>(W, sm.lam, sm.pos, npos, X, ne, ld);
    else
        psd_reconstruct<T>(W, sm.lam, sm.pos, npos, X, ne, ld);
    __syncthreads();
    // ---- output in svec form (lower triangle of the symmetric P)
    const T sq2 = T(1.41421356237309504880);
    for (int64_t s = threadIdx.x; s < len; s += blockDim.x) {
        int i, j;
        psd_svec_ij(s, n, i, j);
        T p = i == j ? X[(size_t)i * ld + j] : T(0.5) * (X[(size_t)i * ld + j] + X[(size_t)j * ld + i]) * sq2;
        io.out(s, p);
    }
    // ---- keep the eigenvectors for the next call
    if (warm && Vkeep != V)
        for (int e = threadIdx.x; e < ne * ne; e += blockDim.x) {
            const int i = e / ne, j = e - i * ne;
            Vkeep[(size_t)i * ld + j] = V[(size_t)i * ld + j];
        }
    __syncthreads();
}

}  // namespace scs
