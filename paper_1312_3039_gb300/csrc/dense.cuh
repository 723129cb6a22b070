// Dense column-major products on the CUDA cores, for the family solver's
// direct subspace step (Sec. 4.1 with the dense (I + A^T A)^-1):
//
//     C (M x N) = alpha * A (M x K) * B (K x N) + beta * C
//
// all three column-major with leading dimensions lda, ldb, ldc.  FP32 runs
// 128 x 128 output tiles (8 x 8 per thread: two groups of 4 rows and of 4
// columns, 64 apart, so that a warp's shared-memory vector loads cover
// contiguous 256-byte spans without bank conflicts) when that grid holds at least two
// CTAs per SM and 64 x 64 tiles (4 x 4 per thread) otherwise (few member
// columns: more CTAs, each with less reuse); FP64 64 x 64 tiles; 256
// threads; k-blocks of 8 staged in shared memory, the next
// block's global loads held in registers while the current one is consumed
// (one barrier per k-block).  Edges of every dimension are bounds-checked
// (zero-filled loads, masked stores), so no size needs padding.  CTAs walk the
// M tiles fastest, so the CTAs that read one block of B columns run together
// and B is fetched from HBM about once.  The products are plain FP32 / FP64
// fused multiply-adds in k order: no reduced-precision arithmetic.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace scs {
namespace dense {

constexpr int kGemmThreads = 256;

template <typename T, int BM_, int TM_>
struct GemmTile {
    static constexpr int BM = BM_, BN = BM_, BK = 8, TM = TM_, TN = TM_;
};
template <typename T>
struct VecOf;
template <>
struct VecOf<float> { using type = float4; };
template <>
struct VecOf<double> { using type = double2; };

template <typename T, typename G>
__global__ void __launch_bounds__(kGemmThreads) gemm_nn_kernel(int M, int N, int K, T alpha,
                                                               const T *__restrict__ A, int64_t lda,
                                                               const T *__restrict__ B, int64_t ldb, T beta,
                                                               T *__restrict__ C, int64_t ldc) {
    using V = typename VecOf<T>::type;
    constexpr int BM = G::BM, BN = G::BN, BK = G::BK, TM = G::TM, TN = G::TN;
    constexpr int TX = BN / TN, TY = BM / TM;
    static_assert(TX * TY == kGemmThreads, "one thread per TM x TN sub-tile");
    constexpr int LA = BM * BK / kGemmThreads, LB = BN * BK / kGemmThreads;
    constexpr int PB = 16 / sizeof(T);              // pad of the B rows (keeps 16-byte rows, spreads banks)
    constexpr int GA = TM / 4, GB = TN / 4;       // groups of 4 rows / columns per thread
    constexpr int SA = BM / GA, SB = BN / GB;     // their spacing
    constexpr int V4 = 4 * sizeof(T) / 16;        // vectors per group of 4
    __shared__ __align__(16) T As[2][BK][BM];
    __shared__ __align__(16) T Bs[2][BK][BN + PB];

    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int64_t m0 = (int64_t)blockIdx.x * BM, n0 = (int64_t)blockIdx.y * BN;
    T ra[LA], rb[LB];
    auto load = [&](int k0) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {      // A tile, M fastest: coalesced along the columns of A
            const int idx = tid + r * kGemmThreads;
            const int64_t gi = m0 + idx % BM;
            const int gk = k0 + idx / BM;
            ra[r] = (gi < M && gk < K) ? A[gi + gk * lda] : T(0);
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {      // B tile, K fastest: 8 contiguous entries of a column
            const int idx = tid + r * kGemmThreads;
            const int gk = k0 + idx % BK;
            const int64_t gj = n0 + idx / BK;
            rb[r] = (gj < N && gk < K) ? B[gk + gj * ldb] : T(0);
        }
    };
    auto store = [&](int buf) {
#pragma unroll
        for (int r = 0; r < LA; ++r) {
            const int idx = tid + r * kGemmThreads;
            As[buf][idx / BM][idx % BM] = ra[r];
        }
#pragma unroll
        for (int r = 0; r < LB; ++r) {
            const int idx = tid + r * kGemmThreads;
            Bs[buf][idx % BK][idx / BK] = rb[r];
        }
    };

    T acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

    load(0);
    store(0);
    __syncthreads();
    int buf = 0;
    for (int k0 = 0; k0 < K; k0 += BK) {
        const bool more = k0 + BK < K;
        if (more) load(k0 + BK);
#pragma unroll
        for (int k = 0; k < BK; ++k) {
            T a[TM], b[TN];
#pragma unroll
            for (int g = 0; g < GA; ++g) {
                const V *pa = reinterpret_cast<const V *>(&As[buf][k][g * SA + ty * 4]);
#pragma unroll
                for (int v = 0; v < V4; ++v) reinterpret_cast<V *>(a + 4 * g)[v] = pa[v];
            }
#pragma unroll
            for (int g = 0; g < GB; ++g) {
                const V *pb = reinterpret_cast<const V *>(&Bs[buf][k][g * SB + tx * 4]);
#pragma unroll
                for (int v = 0; v < V4; ++v) reinterpret_cast<V *>(b + 4 * g)[v] = pb[v];
            }
#pragma unroll
            for (int i = 0; i < TM; ++i)
#pragma unroll
                for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (more) store(buf ^ 1);
        __syncthreads();
        buf ^= 1;
    }

#pragma unroll
    for (int j = 0; j < TN; ++j) {
        const int64_t gj = n0 + (j / 4) * SB + tx * 4 + (j % 4);
        if (gj >= N) continue;
        T *col = C + gj * ldc;
#pragma unroll
        for (int i = 0; i < TM; ++i) {
            const int64_t gi = m0 + (i / 4) * SA + ty * 4 + (i % 4);
            if (gi < M) col[gi] = beta == T(0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * col[gi];
        }
    }
}

// Enqueue C = alpha A B + beta C on `stream` (beta == 0: C is not read).
// Empty products (M, N or K zero) scale C by beta (K == 0) or do nothing.
template <typename T, typename G>
inline cudaError_t gemm_nn_tiles(cudaStream_t stream, int M, int N, int K, T alpha, const T *A, int64_t lda,
                                 const T *B, int64_t ldb, T beta, T *C, int64_t ldc) {
    const unsigned gx = static_cast<unsigned>((M + G::BM - 1) / G::BM);
    const unsigned gy = static_cast<unsigned>((N + G::BN - 1) / G::BN);
    if (gy > 65535u) return cudaErrorInvalidConfiguration;
    gemm_nn_kernel<T, G><<<dim3(gx, gy), kGemmThreads, 0, stream>>>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    return cudaGetLastError();
}

template <typename T>
inline cudaError_t gemm_nn(cudaStream_t stream, int M, int N, int K, T alpha, const T *A, int64_t lda, const T *B,
                           int64_t ldb, T beta, T *C, int64_t ldc) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if constexpr (sizeof(T) == 4) {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return cudaErrorInvalidDevice;
        const int64_t big = (int64_t)((M + 127) / 128) * ((N + 127) / 128);
        if (big >= 2 * (int64_t)sms)
            return gemm_nn_tiles<T, GemmTile<T, 128, 8>>(stream, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
    }
    return gemm_nn_tiles<T, GemmTile<T, 64, 4>>(stream, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
}

// ---------------------------------------------------------------------------
// In-place inverse of a symmetric positive definite G (n x n, column-major)
// by Gauss-Jordan elimination without pivoting (the pivots of an SPD matrix
// are positive; for G = I + A^T A they are at least 1).  Step k:
//   colk = G[:, k] with entry k taken as 0; row k of G divided by G[k][k]
//   (with G[k][k] := 1); G[i][j] -= colk_i row_k[j] for i != k (G[i][k]
//   taken as 0).  After the n steps G holds G^-1.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void gj_pivot_kernel(T *G, int n, int k, T *colk) {
    const T piv = G[(size_t)k * n + k];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        colk[i] = i == k ? T(0) : G[(size_t)k * n + i];
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        colk[n + j] = (j == k ? T(1) : G[(size_t)j * n + k]) / piv;
}

template <typename T>
__global__ void gj_update_kernel(T *G, int n, int k, const T *colk) {
    const int64_t total = (int64_t)n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = static_cast<int>(e / n), i = static_cast<int>(e % n);   // column-major: e = j n + i
        const T rkj = colk[n + j];
        if (i == k) G[e] = rkj;
        else G[e] = (j == k ? T(0) : G[e]) - colk[i] * rkj;
    }
}

// Enqueue the n steps on `stream`; colk is device scratch of 2 n entries.
template <typename T>
inline cudaError_t invert_spd_gj(cudaStream_t stream, T *G, int n, T *colk, int grid) {
    for (int k = 0; k < n; ++k) {
        gj_pivot_kernel<T><<<1, 1024, 0, stream>>>(G, n, k, colk);
        gj_update_kernel<T><<<grid, 256, 0, stream>>>(G, n, k, colk);
    }
    return cudaGetLastError();
}

}  // namespace dense
}  // namespace scs
