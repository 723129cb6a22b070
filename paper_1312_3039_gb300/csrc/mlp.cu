// Warm-start network: a multilayer perceptron theta -> predicted scaled
// solution state (u_x, u_y, v_s, u_tau) of a family member, trained and run
// by the kernels of this file (the paper has no learned component; it
// extends Sec. 4.2's warm start).
//
// Layers d_in -> h -> ... -> h -> d_out, GELU after every hidden layer
// (GELU(z) = z Phi(z)), linear output; loss = mean squared error over the
// outputs of a batch; Adam on FP32 master weights.  Products run on the
// tensor cores in BF16 with FP32 accumulation: one GEMM kernel of the form
// C[M x N] = A[M x K] B[N x K]^T (both operands K-contiguous), used as
//   forward   Z   = X W^T + b          (A = X,   B = W)
//   backward  dX  = dZ W               (A = dZ,  B = W^T)
//   backward  dW  = dZ^T X             (A = dZ^T, B = X^T)
// with fused epilogues (bias + GELU with the pre-activation kept; bias; plain).
// Shapes are padded so that every launch meets the kernel's tiling exactly
// (M % 128, N % 64, K % 32, rows 16-byte aligned); padding rows and columns
// of the weights are zero and stay zero (their gradients are zero).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/scs_gpu.h"
#include "common.cuh"
#include "engine_base.h"

namespace scs {
namespace mlp {

constexpr int BM = 128, BN = 64, BK = 32, kGemmThreads = 128;
constexpr int kLds = BK + 8;   // shared-memory row stride (bf16): 80 bytes, conflict-free ldmatrix

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}
__device__ __forceinline__ void ldmatrix_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3, const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(smem_u32(p)));
}
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// epilogues: called with (row, col, value at col, value at col + 1)
struct EpiHidden {   // Z = acc + b (FP32); A = GELU(Z) (BF16)
    float *Z;
    __nv_bfloat16 *A;
    const float *bias;
    int ldz, lda;
    __device__ void operator()(int r, int c, float v0, float v1) const {
        const float z0 = v0 + bias[c], z1 = v1 + bias[c + 1];
        *reinterpret_cast<float2 *>(Z + (size_t)r * ldz + c) = make_float2(z0, z1);
        *reinterpret_cast<__nv_bfloat162 *>(A + (size_t)r * lda + c) = __floats2bfloat162_rn(gelu(z0), gelu(z1));
    }
};
struct EpiBias {     // Z = acc + b (FP32)
    float *Z;
    const float *bias;
    int ldz;
    __device__ void operator()(int r, int c, float v0, float v1) const {
        *reinterpret_cast<float2 *>(Z + (size_t)r * ldz + c) = make_float2(v0 + bias[c], v1 + bias[c + 1]);
    }
};
struct EpiPlain {    // C = acc (FP32)
    float *C;
    int ldc;
    __device__ void operator()(int r, int c, float v0, float v1) const {
        *reinterpret_cast<float2 *>(C + (size_t)r * ldc + c) = make_float2(v0, v1);
    }
};

// C[M x N] = A[M x K] B[N x K]^T; grid (N / BN, M / BM); 4 warps, each a
// 64 x 32 tile of m16n8k16 products; two-stage cp.async pipeline over K.
template <typename Epi>
__global__ void __launch_bounds__(kGemmThreads) gemm_nt_kernel(const __nv_bfloat16 *__restrict__ A, int lda,
                                                               const __nv_bfloat16 *__restrict__ B, int ldb, int K,
                                                               Epi epi) {
    __shared__ __align__(16) __nv_bfloat16 sA[2][BM * kLds];
    __shared__ __align__(16) __nv_bfloat16 sB[2][BN * kLds];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp >> 1, wn = warp & 1;
    const int bm = blockIdx.y * BM, bn = blockIdx.x * BN;
    const __nv_bfloat16 *Ab = A + (size_t)bm * lda, *Bb = B + (size_t)bn * ldb;
    auto load = [&](int stage, int k0) {
        // A: 128 rows x 4 chunks of 8 bf16; B: 64 rows x 4 chunks
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int ch = tid + i * kGemmThreads, r = ch >> 2, c = (ch & 3) * 8;
            cp_async16(&sA[stage][r * kLds + c], Ab + (size_t)r * lda + k0 + c);
        }
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int ch = tid + i * kGemmThreads, r = ch >> 2, c = (ch & 3) * 8;
            cp_async16(&sB[stage][r * kLds + c], Bb + (size_t)r * ldb + k0 + c);
        }
    };
    float acc[4][4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;
    const int KT = K / BK;
    load(0, 0);
    cp_commit();
    for (int kt = 0; kt < KT; ++kt) {
        if (kt + 1 < KT) {
            load((kt + 1) & 1, (kt + 1) * BK);
            cp_commit();
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const __nv_bfloat16 *a_s = sA[kt & 1], *b_s = sB[kt & 1];
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[4][4], bf[2][4];
#pragma unroll
            for (int mi = 0; mi < 4; ++mi) {
                const int r = wm * 64 + mi * 16 + (lane & 15), c = kk + (lane >> 4) * 8;
                ldmatrix_x4(af[mi][0], af[mi][1], af[mi][2], af[mi][3], a_s + r * kLds + c);
            }
#pragma unroll
            for (int nj = 0; nj < 2; ++nj) {
                const int r = wn * 32 + nj * 16 + (lane & 7) + ((lane >> 4) << 3), c = kk + ((lane >> 3) & 1) * 8;
                ldmatrix_x4(bf[nj][0], bf[nj][1], bf[nj][2], bf[nj][3], b_s + r * kLds + c);
            }
#pragma unroll
            for (int mi = 0; mi < 4; ++mi)
#pragma unroll
                for (int ni = 0; ni < 4; ++ni)
                    mma_bf16(acc[mi][ni], af[mi], bf[ni >> 1][(ni & 1) * 2], bf[ni >> 1][(ni & 1) * 2 + 1]);
        }
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
            const int r = bm + wm * 64 + mi * 16 + g, c = bn + wn * 32 + ni * 8 + 2 * t;
            epi(r, c, acc[mi][ni][0], acc[mi][ni][1]);
            epi(r + 8, c, acc[mi][ni][2], acc[mi][ni][3]);
        }
}

// ---------------------------------------------------------------------------
// The same product on the 5th-generation tensor cores (tcgen05): a
// persistent, warp-specialised kernel.  Each CTA walks C tiles of 128 x BNt
// (BNt = 64, 128 or 256; N tiles fastest, so the CTAs of a wave share A rows
// and B stays in L2):
//   warp 0, one thread: TMA copies (cp.async.bulk.tensor, 128-byte swizzle)
//     of the A and B k-blocks into a ring of shared-memory stages; each copy
//     completes on the stage's `full` mbarrier by its byte count;
//   warp 1, one thread: tcgen05.mma (kind::f16, BF16 x BF16 -> FP32) into one
//     of two accumulators in tensor memory (2 x BNt columns); tcgen05.commit
//     frees a stage (`empty`) once its MMAs completed, and hands a finished
//     accumulator to the epilogue (`acc_full`);
//   warps 2-5: the epilogue, tcgen05.ld of the accumulator (a warp reads the
//     32 TMEM lanes of its quarter: rows 32 (warp % 4) ..) into the fused
//     epilogue, then `acc_empty`, so that the MMAs of the next tile run while
//     this one is written out.
// The operand layout in shared memory is K-major with the 128-byte swizzle
// (8-row atoms of 128-byte rows, 1024 bytes apart), the layout the TMA writes
// for a 64-element-wide box.  Every mbarrier wait is bounded: on time-out the
// kernel sets *err, waits (bounded) for its copies and MMAs in flight, frees
// its tensor memory and returns.
// ---------------------------------------------------------------------------
constexpr int TBM = 128, TBN = 64, TBK = 64;             // TBN: the narrowest tile
constexpr int kTcThreads = 192;                          // 6 warps: TMA, MMA, 4 epilogue
constexpr int kTcStageA = TBM * TBK * 2;                 // bytes
constexpr int kTcPipe = 196608;                          // shared-memory bytes of the stage ring
template <int BNt>
__host__ __device__ constexpr int tc_stage_b() { return BNt * TBK * 2; }
template <int BNt>
__host__ __device__ constexpr int tc_stages() { return kTcPipe / (kTcStageA + tc_stage_b<BNt>()); }
template <int BNt>
__host__ __device__ constexpr int tc_smem() { return tc_stages<BNt>() * (kTcStageA + tc_stage_b<BNt>()) + 1024 + 256; }
constexpr uint32_t kTcSpin = 1u << 20;

__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t addr) {
    // K-major, 128-byte swizzle: 8-row atoms of 128-byte rows (64 BF16 of K),
    // 1024 bytes apart (SBO); LBO unused for this layout (1); fixed 0b001 at
    // bits 46-48; layout type 2 (SWIZZLE_128B) at bits 61-63.  A K step of
    // 16 elements moves the start address by 32 bytes inside the atom.
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// byte offset of 16-byte chunk c (0..7) of row r in a 128-byte-swizzled tile
__device__ __forceinline__ int tc_sw128(int r, int c) { return (r >> 3) * 1024 + (r & 7) * 128 + ((c ^ (r & 7)) << 4); }
// kind::f16 instruction descriptor: D FP32, A and B BF16, both K-major, N, M
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < kTcSpin; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(mbar),
                 "r"(bytes)
                 : "memory");
}
// 2-D tiled TMA load of the box at (x = k offset, y = row) into shared memory
__device__ __forceinline__ void tma_load(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(mbar)
        : "memory");
}

// K blocks of a product whose operands are stored in chunks: K block kt lies
// in chunk c = kt / kchunk of the product and reads chunk a[c] of A and b[c]
// of B (each chunk kchunk K blocks wide).  kchunk = 0: one plain K range.
struct TcKMap {
    int kchunk;
    signed char a[8], b[8];
};

// C = A B^T, A M x K and B N x K (K-contiguous, described by tmA and tmB)
template <typename Epi, int BNt>
__global__ void __launch_bounds__(kTcThreads, 1) gemm_nt_tc_kernel(const __grid_constant__ CUtensorMap tmA,
                                                                   const __grid_constant__ CUtensorMap tmB, int M,
                                                                   int N, int K, Epi epi, int *err, TcKMap km) {
    constexpr int S = tc_stages<BNt>();
    constexpr int kStageB = tc_stage_b<BNt>();
    constexpr uint32_t kStageBytes = kTcStageA + kStageB;
    extern __shared__ __align__(16) unsigned char tc_raw[];
    const uint32_t raw = smem_u32(tc_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char *misc = tc_raw + (base - raw) + S * (kTcStageA + kStageB);
    uint64_t *full = reinterpret_cast<uint64_t *>(misc);     // [S] the stage's copies landed
    uint64_t *empty = full + S;                               // [S] the stage's MMAs completed
    uint64_t *acc_full = empty + S;                           // [2] an accumulator is ready
    uint64_t *acc_empty = acc_full + 2;                       // [2] an accumulator was read out
    uint64_t *done = acc_empty + 2;                           // every MMA of the CTA completed
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = M / TBM, nt = N / BNt, ntiles = mt * nt, KT = K / TBK;
    auto sA = [&](int st) { return base + st * kTcStageA; };
    auto sB = [&](int st) { return base + S * kTcStageA + st * kStageB; };
    auto bar = [](uint64_t *b) { return smem_u32(b); };

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(tmem_slot)),
                     "n"(2 * BNt));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    if (tid == 0) {
        for (int st = 0; st < S; ++st) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar(&full[st])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar(&empty[st])));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar(&acc_full[b])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 128;\n" ::"r"(bar(&acc_empty[b])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar(done)));
        asm volatile("fence.mbarrier_init.release.cluster;\n");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    const uint32_t tmem = *tmem_slot;
    bool ok = true;

    if (warp == 0 && lane == 0) {
        // TMA producer
        int it = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int tm = t / nt, tn = t % nt;
            for (int kt = 0; kt < KT; ++kt, ++it) {
                const int s = it % S;
                if (it >= S && !tc_wait(bar(&empty[s]), ((it / S) - 1) & 1)) {
                    ok = false;
                    break;
                }
                int xa = kt * TBK, xb = kt * TBK;
                if (km.kchunk) {
                    const int c = kt / km.kchunk, j = kt % km.kchunk;
                    xa = (km.a[c] * km.kchunk + j) * TBK;
                    xb = (km.b[c] * km.kchunk + j) * TBK;
                }
                mbar_expect(bar(&full[s]), kStageBytes);
                tma_load(sA(s), &tmA, xa, tm * TBM, bar(&full[s]));
                tma_load(sB(s), &tmB, xb, tn * BNt, bar(&full[s]));
            }
        }
        // the copies of the last uses of each stage have landed (bounded)
        for (int j = (it > S ? it - S : 0); j < it; ++j) ok = tc_wait(bar(&full[j % S]), (j / S) & 1) && ok;
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = tc_idesc(TBM, BNt);
        int it = 0, tl = 0;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
            const int b = tl & 1;
            if (tl >= 2 && !tc_wait(bar(&acc_empty[b]), ((tl >> 1) - 1) & 1)) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const uint32_t acc_tm = tmem + (uint32_t)(b * BNt);
            for (int kt = 0; kt < KT; ++kt, ++it) {
                const int s = it % S;
                if (!tc_wait(bar(&full[s]), (it / S) & 1)) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n");
#pragma unroll
                for (int k = 0; k < TBK / 16; ++k) {
                    const uint64_t ad = tc_smem_desc(sA(s) + k * 32), bd = tc_smem_desc(sB(s) + k * 32);
                    const uint32_t acc = (kt > 0 || k > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
                        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc_tm),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                    bar(&empty[s])));
            }
            // the accumulator is handed over even after a time-out, so that
            // the epilogue does not wait in vain
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                bar(&acc_full[b])));
        }
        // every MMA issued above has completed before the memory is freed
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar(done)));
        ok = tc_wait(bar(done), 0) && ok;
    } else if (warp >= 2) {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 = the tile's rows
        const int q = warp & 3;
        const uint32_t lane_base = (uint32_t)(q * 32) << 16;
        int tl = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
            const int b = tl & 1, tm = t / nt, tn = t % nt;
            const bool ready = __all_sync(0xffffffffu, tc_wait(bar(&acc_full[b]), (tl >> 1) & 1));
            if (!ready) {
                ok = false;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n");
            const int r = tm * TBM + q * 32 + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < BNt; c0 += 16) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(tmem + lane_base + (uint32_t)(b * BNt + c0)));
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int j = 0; j < 16; j += 2)
                    epi(r, tn * BNt + c0 + j, __uint_as_float(v[j]), __uint_as_float(v[j + 1]));
            }
            asm volatile("tcgen05.fence::before_thread_sync;\n");
            mbar_arrive(bar(&acc_empty[b]));
        }
    }
    if (!ok) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "n"(2 * BNt));
}

// dst[c][r] = src[r][c] for r < rows, c < cols (BF16; 32 x 32 tiles)
static __global__ void transpose_kernel(const __nv_bfloat16 *__restrict__ src, int lds, __nv_bfloat16 *__restrict__ dst,
                                        int ldd, int rows, int cols) {
    __shared__ __nv_bfloat16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(size_t)r * lds + c] : __float2bfloat16(0.f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) dst[(size_t)c * ldd + r] = tile[threadIdx.x][i];
    }
}

// X (rows x cols FP32, ld cols) -> BF16 (ld ldd, zero columns up to ldd)
static __global__ void to_bf16_kernel(const float *__restrict__ x, int rows, int cols, __nv_bfloat16 *__restrict__ y,
                                      int ldd) {
    const int64_t total = (int64_t)rows * ldd;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = static_cast<int>(e / ldd), c = static_cast<int>(e % ldd);
        y[e] = __float2bfloat16(c < cols ? x[(size_t)r * cols + c] : 0.f);
    }
}

// output layer: dZ = 2 (Y - T) / (rows dout) on the first dout columns, 0 on
// the padding; FP32 (bias gradient) and BF16 copies; per-CTA loss partials
static __global__ void loss_grad_kernel(const float *__restrict__ Y, int ldy, const float *__restrict__ T, int dout,
                                        int rows, float *__restrict__ dz32, __nv_bfloat16 *__restrict__ dz16,
                                        double *__restrict__ part) {
    __shared__ double red[8];
    const double scale = 2.0 / ((double)rows * dout);
    double acc = 0.0;
    const int64_t total = (int64_t)rows * ldy;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = static_cast<int>(e / ldy), c = static_cast<int>(e % ldy);
        float g = 0.f;
        if (c < dout) {
            const float d = Y[e] - T[(size_t)r * dout + c];
            acc += (double)d * d;
            g = static_cast<float>(scale * d);
        }
        dz32[e] = g;
        dz16[e] = __float2bfloat16(g);
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

static __global__ void sum_parts_kernel(const double *__restrict__ part, int n, double scale, double *out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += part[i];
        *out = s * scale;
    }
}

// hidden layer: dZ = dA * GELU'(Z) (FP32 and BF16)
static __global__ void gelu_back_kernel(const float *__restrict__ dA, const float *__restrict__ Z, int64_t len,
                                        float *__restrict__ dz32, __nv_bfloat16 *__restrict__ dz16) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const float g = dA[e] * gelu_grad(Z[e]);
        dz32[e] = g;
        dz16[e] = __float2bfloat16(g);
    }
}

// db[c] = sum over rows of dZ[r][c] (one thread per column, rows in order)
static __global__ void colsum_kernel(const float *__restrict__ dz, int rows, int cols, float *__restrict__ db) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    float s = 0.f;
    for (int r = 0; r < rows; ++r) s += dz[(size_t)r * cols + c];
    db[c] = s;
}

// Adam (bias-corrected) on FP32 master values
static __global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                                   float *__restrict__ v, int64_t len, float lr, float b1, float b2, float eps,
                                   float c1, float c2) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len; e += (int64_t)gridDim.x * blockDim.x) {
        const float gg = g[e];
        const float mm = b1 * m[e] + (1.f - b1) * gg;
        const float vv = b2 * v[e] + (1.f - b2) * gg * gg;
        m[e] = mm;
        v[e] = vv;
        p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

// BF16 copies W (out_p x in_p) and W^T (in_p x out_p) of a FP32 master
static __global__ void weights_bf16_kernel(const float *__restrict__ W, int out_p, int in_p,
                                           __nv_bfloat16 *__restrict__ W16, __nv_bfloat16 *__restrict__ Wt16) {
    const int64_t total = (int64_t)out_p * in_p;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int o = static_cast<int>(e / in_p), i = static_cast<int>(e % in_p);
        const __nv_bfloat16 w = __float2bfloat16(W[e]);
        W16[e] = w;
        Wt16[(size_t)i * out_p + o] = w;
    }
}

inline int round_up(int x, int a) { return (x + a - 1) / a * a; }

// tensor map of a row-major BF16 matrix (rows x cols, leading dimension ld
// elements) read in boxes of box_rows x 64 with the 128-byte swizzle
inline CUtensorMap tc_map(const __nv_bfloat16 *p, int rows, int cols, int ld, int box_rows) {
    static std::mutex mu;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        SCS_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
        if (q != cudaDriverEntryPointSuccess || !fn) throw CudaError("cuTensorMapEncodeTiled unavailable", SCS_DEVICE_ERROR);
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    CUtensorMap m;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(p), dims, strides,
                              box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw CudaError("tensor map encoding failed", SCS_INVALID_INPUT);
    return m;
}

// M, N: the tiles' extent (multiples of 128 and BNt); rows_a, rows_b, cols_a,
// cols_b: the operands' stored extent (rows beyond it read as zeros)
template <typename Epi, int BNt>
void launch_tc(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K, Epi epi, int *err,
               cudaStream_t stream, TcKMap km = TcKMap{}, int rows_a = -1, int rows_b = -1, int cols_a = -1,
               int cols_b = -1) {
    // per device: the kernel's shared-memory attribute set once, its SM count
    constexpr int kDevs = 64;
    static std::mutex mu;
    static int sms[kDevs] = {};
    int dev = 0;
    SCS_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kDevs) throw CudaError("device index beyond the product's table", SCS_INVALID_INPUT);
    int nsm = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (!sms[dev]) {
            SCS_CUDA(cudaFuncSetAttribute(gemm_nt_tc_kernel<Epi, BNt>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tc_smem<BNt>()));
            SCS_CUDA(cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev));
        }
        nsm = sms[dev];
    }
    const CUtensorMap ma = tc_map(A, rows_a < 0 ? M : rows_a, cols_a < 0 ? K : cols_a, lda, TBM),
                      mb = tc_map(B, rows_b < 0 ? N : rows_b, cols_b < 0 ? K : cols_b, ldb, BNt);
    const int tiles = (M / TBM) * (N / BNt);
    gemm_nt_tc_kernel<Epi, BNt><<<std::min(tiles, nsm), kTcThreads, tc_smem<BNt>(), stream>>>(ma, mb, M, N, K, epi, err,
                                                                                              km);
}

// C = A B^T through either kernel; the shape must meet the kernel's tiling
template <typename Epi>
void launch_gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K, Epi epi,
                 bool tc, int *err, cudaStream_t stream) {
    if (lda % 8 || ldb % 8 || (reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15))
        throw CudaError("GEMM operands must have 16-byte aligned rows", SCS_INVALID_INPUT);
    if (tc) {
        if (M % TBM || N % TBN || K % TBK)
            throw CudaError("GEMM shape outside the tcgen05 kernel's tiling", SCS_INVALID_INPUT);
        if (N % 256 == 0)
            launch_tc<Epi, 256>(A, lda, B, ldb, M, N, K, epi, err, stream);
        else if (N % 128 == 0)
            launch_tc<Epi, 128>(A, lda, B, ldb, M, N, K, epi, err, stream);
        else
            launch_tc<Epi, 64>(A, lda, B, ldb, M, N, K, epi, err, stream);
    } else {
        if (M % BM || N % BN || K % BK) throw CudaError("GEMM shape outside the kernel's tiling", SCS_INVALID_INPUT);
        gemm_nt_kernel<Epi><<<dim3(N / BN, M / BM), kGemmThreads, 0, stream>>>(A, lda, B, ldb, K, epi);
    }
    SCS_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// FP32-accurate products on the tensor cores (three-way BF16 split).
//   x = x1 + x2 + x3,  x1 = bf16(x), x2 = bf16(x - x1), x3 = bf16(x - x1 - x2)
// (each difference is exact in FP32, so x - x1 - x2 - x3 is below 2^-24 |x|).
// A sum of products a.b is taken as the six BF16 x BF16 products
//   a1 b1 + a1 b2 + a2 b1 + a1 b3 + a2 b2 + a3 b1
// (the three dropped ones are below 2^-24 |a||b|), in two tcgen05 launches:
// a1 b1 first, then the five smaller products added to it.  The tensor
// cores' FP32 accumulation aligns a group of products to its largest one, so
// in a single accumulator the 2^-16-sized products would lose their low bits
// next to a1 b1 (measured: about 2^-15 relative); summed on their own, their
// accumulation error is 2^-8 smaller.  The operands are stored as three
// chunks of Kp columns each (x1 | x2 | x3, zero-padded from K to Kp); the
// kernel's chunk map reads chunk 0 of A against chunk 0 of B (K' = Kp), then
// chunks (0, 1, 0, 1, 2) of A against (1, 0, 2, 1, 0) of B (K' = 5 Kp).
// ---------------------------------------------------------------------------
// dst (rows x 3 Kp, row-major) from src rows x K: element (r, k) at
// src[r ld + k], or at src[k ld + r] when trans (a column-major source read
// along its rows)
static __global__ void split3_kernel(const float *__restrict__ src, int rows, int K, int64_t ld, int trans, int Kp,
                                     __nv_bfloat16 *__restrict__ dst) {
    const int64_t total = (int64_t)rows * Kp;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / Kp;
        const int k = static_cast<int>(e % Kp);
        const float x = k < K ? (trans ? src[(int64_t)k * ld + r] : src[r * ld + k]) : 0.f;
        const __nv_bfloat16 h1 = __float2bfloat16_rn(x);
        const float r1 = x - __bfloat162float(h1);
        const __nv_bfloat16 h2 = __float2bfloat16_rn(r1);
        const __nv_bfloat16 h3 = __float2bfloat16_rn(r1 - __bfloat162float(h2));
        __nv_bfloat16 *row = dst + r * 3 * (int64_t)Kp;
        row[k] = h1;
        row[Kp + k] = h2;
        row[2 * Kp + k] = h3;
    }
}

// C'(r, c) = alpha acc + beta C'(r, c) stored at C[r ldc + c], r < rows,
// c < cols (beta == 0: C is not read)
struct EpiScaledT {
    float *C;
    int64_t ldc;
    int rows, cols;
    float alpha, beta;
    __device__ void put(int r, int c, float v) const {
        float *p = C + (int64_t)r * ldc + c;
        *p = beta == 0.f ? alpha * v : alpha * v + beta * *p;
    }
    __device__ void operator()(int r, int c, float v0, float v1) const {
        if (r >= rows) return;
        if (c < cols) put(r, c, v0);
        if (c + 1 < cols) put(r, c + 1, v1);
    }
};

void split3_bf16(const float *src, int rows, int K, int64_t ld, int trans, int Kp, __nv_bfloat16 *dst,
                 cudaStream_t stream) {
    const int64_t total = (int64_t)rows * Kp;
    const int grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096)));
    split3_kernel<<<grid, 256, 0, stream>>>(src, rows, K, ld, trans, Kp, dst);
    SCS_CUDA(cudaGetLastError());
}

void gemm_fp32x3(const __nv_bfloat16 *A3, int rows_a, const __nv_bfloat16 *B3, int rows_b, int Kp, float *C,
                 int64_t ldc, float alpha, float beta, int *err, cudaStream_t stream) {
    if (rows_a <= 0 || rows_b <= 0) return;
    if (Kp <= 0 || Kp % TBK || (reinterpret_cast<uintptr_t>(A3) & 15) || (reinterpret_cast<uintptr_t>(B3) & 15))
        throw CudaError("split product: Kp must be a positive multiple of 64, operands 16-byte aligned",
                        SCS_INVALID_INPUT);
    const TcKMap big{Kp / TBK, {0, 0, 0, 0, 0, 0, 0, 0}, {0, 0, 0, 0, 0, 0, 0, 0}};
    const TcKMap small{Kp / TBK, {0, 1, 0, 1, 2, 0, 0, 0}, {1, 0, 2, 1, 0, 0, 0, 0}};
    const int M = round_up(rows_a, TBM), ld = 3 * Kp;
    for (int pass = 0; pass < 2; ++pass) {
        const TcKMap &km = pass == 0 ? big : small;
        const int K = pass == 0 ? Kp : 5 * Kp;
        const EpiScaledT epi{C, ldc, rows_a, rows_b, alpha, pass == 0 ? beta : 1.f};
        if (round_up(rows_b, 256) == round_up(rows_b, 128))
            launch_tc<EpiScaledT, 256>(A3, ld, B3, ld, M, round_up(rows_b, 256), K, epi, err, stream, km, rows_a,
                                       rows_b, ld, ld);
        else if (rows_b > 64)
            launch_tc<EpiScaledT, 128>(A3, ld, B3, ld, M, round_up(rows_b, 128), K, epi, err, stream, km, rows_a,
                                       rows_b, ld, ld);
        else
            launch_tc<EpiScaledT, 64>(A3, ld, B3, ld, M, round_up(rows_b, 64), K, epi, err, stream, km, rows_a,
                                      rows_b, ld, ld);
        SCS_CUDA(cudaGetLastError());
    }
}

class Net {
   public:
    Net(int din, int h, int layers, int dout, int batch, cudaStream_t s) : din_(din), h_(h), L_(layers + 1), dout_(dout),
                                                                           batch_(batch), stream_(s) {
        if (din < 1 || h < 1 || layers < 1 || dout < 1 || batch < BM || batch % BM)
            throw CudaError("network sizes: batch must be a positive multiple of 128", SCS_INVALID_INPUT);
        for (int l = 0; l < L_; ++l) {
            const int in = l == 0 ? din : h, out = l == L_ - 1 ? dout : h;
            // a layer reads its input with the previous layer's padded width
            const int in_p = l == 0 ? round_up(in, 64) : layers_.back().out_p, out_p = round_up(out, 128);
            Layer Y;
            Y.in = in;
            Y.out = out;
            Y.in_p = in_p;
            Y.out_p = out_p;
            Y.W = alloc<float>((size_t)out_p * in_p);
            Y.b = alloc<float>(out_p);
            Y.gW = alloc<float>((size_t)out_p * in_p);
            Y.gb = alloc<float>(out_p);
            Y.mW = alloc<float>((size_t)out_p * in_p);
            Y.vW = alloc<float>((size_t)out_p * in_p);
            Y.mb = alloc<float>(out_p);
            Y.vb = alloc<float>(out_p);
            Y.W16 = alloc<__nv_bfloat16>((size_t)out_p * in_p);
            Y.Wt16 = alloc<__nv_bfloat16>((size_t)out_p * in_p);
            Y.Z = alloc<float>((size_t)batch * out_p);
            Y.A16 = alloc<__nv_bfloat16>((size_t)batch * out_p);
            Y.dz32 = alloc<float>((size_t)batch * out_p);
            Y.dz16 = alloc<__nv_bfloat16>((size_t)batch * out_p);
            Y.dzt16 = alloc<__nv_bfloat16>((size_t)batch * out_p);
            Y.at16 = alloc<__nv_bfloat16>((size_t)batch * in_p);
            Y.dA = alloc<float>((size_t)batch * in_p);
            for (float *p : {Y.W, Y.mW, Y.vW}) SCS_CUDA(cudaMemsetAsync(p, 0, sizeof(float) * out_p * in_p, stream_));
            for (float *p : {Y.b, Y.mb, Y.vb}) SCS_CUDA(cudaMemsetAsync(p, 0, sizeof(float) * out_p, stream_));
            layers_.push_back(Y);
        }
        x16_ = alloc<__nv_bfloat16>((size_t)batch * layers_[0].in_p);
        // tcgen05 products when every padded size meets that kernel's tiling
        tcgen05_ = batch % TBM == 0 && batch % TBK == 0;
        for (const Layer &Y : layers_)
            tcgen05_ = tcgen05_ && Y.in_p % TBK == 0 && Y.out_p % TBN == 0 && Y.out_p % TBK == 0;
        err_ = alloc<int>(1);
        SCS_CUDA(cudaMemsetAsync(err_, 0, sizeof(int), stream_));
        part_ = alloc<double>(1024);
        loss_ = alloc<double>(1);
        SCS_CUDA(cudaStreamSynchronize(stream_));
    }
    ~Net() {
        for (void *p : allocs_) cudaFree(p);
    }

    int64_t param_count() const {
        int64_t c = 0;
        for (const Layer &Y : layers_) c += (int64_t)Y.out * Y.in + Y.out;
        return c;
    }

    // packed host layout: per layer W (out x in, row-major) then b (out)
    void set_params(const float *h) {
        const float *p = h;
        for (Layer &Y : layers_) {
            std::vector<float> W((size_t)Y.out_p * Y.in_p, 0.f), b(Y.out_p, 0.f);
            for (int o = 0; o < Y.out; ++o)
                for (int i = 0; i < Y.in; ++i) W[(size_t)o * Y.in_p + i] = *p++;
            for (int o = 0; o < Y.out; ++o) b[o] = *p++;
            SCS_CUDA(cudaMemcpyAsync(Y.W, W.data(), sizeof(float) * W.size(), cudaMemcpyHostToDevice, stream_));
            SCS_CUDA(cudaMemcpyAsync(Y.b, b.data(), sizeof(float) * b.size(), cudaMemcpyHostToDevice, stream_));
            SCS_CUDA(cudaMemsetAsync(Y.mW, 0, sizeof(float) * W.size(), stream_));
            SCS_CUDA(cudaMemsetAsync(Y.vW, 0, sizeof(float) * W.size(), stream_));
            SCS_CUDA(cudaMemsetAsync(Y.mb, 0, sizeof(float) * b.size(), stream_));
            SCS_CUDA(cudaMemsetAsync(Y.vb, 0, sizeof(float) * b.size(), stream_));
            SCS_CUDA(cudaStreamSynchronize(stream_));
        }
        step_ = 0;
        refresh_bf16();
    }
    void get(float *h, bool grads) {
        float *p = h;
        for (Layer &Y : layers_) {
            std::vector<float> W((size_t)Y.out_p * Y.in_p), b(Y.out_p);
            SCS_CUDA(cudaMemcpyAsync(W.data(), grads ? Y.gW : Y.W, sizeof(float) * W.size(), cudaMemcpyDeviceToHost,
                                     stream_));
            SCS_CUDA(cudaMemcpyAsync(b.data(), grads ? Y.gb : Y.b, sizeof(float) * b.size(), cudaMemcpyDeviceToHost,
                                     stream_));
            SCS_CUDA(cudaStreamSynchronize(stream_));
            for (int o = 0; o < Y.out; ++o)
                for (int i = 0; i < Y.in; ++i) *p++ = W[(size_t)o * Y.in_p + i];
            for (int o = 0; o < Y.out; ++o) *p++ = b[o];
        }
    }

    void refresh_bf16() {
        for (Layer &Y : layers_) {
            weights_bf16_kernel<<<grid((int64_t)Y.out_p * Y.in_p), 256, 0, stream_>>>(Y.W, Y.out_p, Y.in_p, Y.W16,
                                                                                    Y.Wt16);
        }
        SCS_CUDA(cudaGetLastError());
    }

    // forward of `batch_` rows of x (device FP32, batch x din); the output
    // layer's Z (FP32, batch x out_p) holds the prediction
    void forward(const float *x) {
        const Layer &F = layers_[0];
        to_bf16_kernel<<<grid((int64_t)batch_ * F.in_p), 256, 0, stream_>>>(x, batch_, din_, x16_, F.in_p);
        const __nv_bfloat16 *in = x16_;
        for (int l = 0; l < L_; ++l) {
            Layer &Y = layers_[l];
            if (l < L_ - 1) gemm(in, Y.in_p, Y.W16, Y.in_p, batch_, Y.out_p, Y.in_p, EpiHidden{Y.Z, Y.A16, Y.b, Y.out_p, Y.out_p});
            else gemm(in, Y.in_p, Y.W16, Y.in_p, batch_, Y.out_p, Y.in_p, EpiBias{Y.Z, Y.b, Y.out_p});
            in = Y.A16;
        }
        SCS_CUDA(cudaGetLastError());
    }

    // forward + backward: gradients in gW, gb; loss (device double)
    void backward(const float *x, const float *t) {
        forward(x);
        Layer &O = layers_[L_ - 1];
        const int nb = 264;
        loss_grad_kernel<<<nb, 256, 0, stream_>>>(O.Z, O.out_p, t, dout_, batch_, O.dz32, O.dz16, part_);
        sum_parts_kernel<<<1, 32, 0, stream_>>>(part_, nb, 1.0 / ((double)batch_ * dout_), loss_);
        for (int l = L_ - 1; l >= 0; --l) {
            Layer &Y = layers_[l];
            const __nv_bfloat16 *in16 = l == 0 ? x16_ : layers_[l - 1].A16;
            if (l < L_ - 1) {
                // dZ = dA_out * GELU'(Z), dA_out from the layer above
                gelu_back_kernel<<<grid((int64_t)batch_ * Y.out_p), 256, 0, stream_>>>(
                    layers_[l + 1].dA, Y.Z, (int64_t)batch_ * Y.out_p, Y.dz32, Y.dz16);
            }
            // dZ^T and input^T (BF16)
            transpose(Y.dz16, Y.out_p, Y.dzt16, batch_, batch_, Y.out_p);
            transpose(in16, Y.in_p, Y.at16, batch_, batch_, Y.in_p);
            // dW = dZ^T X: (out_p x batch) (in_p x batch)^T
            gemm(Y.dzt16, batch_, Y.at16, batch_, Y.out_p, Y.in_p, batch_, EpiPlain{Y.gW, Y.in_p});
            colsum_kernel<<<(Y.out_p + 255) / 256, 256, 0, stream_>>>(Y.dz32, batch_, Y.out_p, Y.gb);
            // dX = dZ W: (batch x out_p) (in_p x out_p)^T
            if (l > 0) gemm(Y.dz16, Y.out_p, Y.Wt16, Y.out_p, batch_, Y.in_p, Y.out_p, EpiPlain{Y.dA, Y.in_p});
        }
        SCS_CUDA(cudaGetLastError());
    }

    void adam(float lr) {
        ++step_;
        const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
        const float c1 = 1.f - std::pow(b1, (float)step_), c2 = 1.f - std::pow(b2, (float)step_);
        for (Layer &Y : layers_) {
            const int64_t nw = (int64_t)Y.out_p * Y.in_p;
            adam_kernel<<<grid(nw), 256, 0, stream_>>>(Y.W, Y.gW, Y.mW, Y.vW, nw, lr, b1, b2, eps, c1, c2);
            adam_kernel<<<grid(Y.out_p), 256, 0, stream_>>>(Y.b, Y.gb, Y.mb, Y.vb, Y.out_p, lr, b1, b2, eps, c1, c2);
        }
        refresh_bf16();
    }

    double loss_host() {
        double h = 0.0;
        SCS_CUDA(cudaMemcpyAsync(&h, loss_, sizeof(double), cudaMemcpyDeviceToHost, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        return h;
    }

    // prediction of the last forward: rows x dout (FP32) into y
    void copy_output(float *y) {
        const Layer &O = layers_[L_ - 1];
        SCS_CUDA(cudaMemcpy2DAsync(y, sizeof(float) * dout_, O.Z, sizeof(float) * O.out_p, sizeof(float) * dout_,
                                   batch_, cudaMemcpyDefault, stream_));
    }

    template <typename Epi>
    void gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M, int N, int K, Epi epi) {
        launch_gemm(A, lda, B, ldb, M, N, K, epi, tcgen05_, err_, stream_);
    }
    void transpose(const __nv_bfloat16 *src, int lds, __nv_bfloat16 *dst, int ldd, int rows, int cols) {
        transpose_kernel<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, stream_>>>(src, lds, dst, ldd,
                                                                                               rows, cols);
    }
    int grid(int64_t len) const { return static_cast<int>(std::min<int64_t>((len + 255) / 256, 4096)); }

    template <typename U>
    U *alloc(size_t n) {
        void *p = nullptr;
        SCS_CUDA(cudaMalloc(&p, sizeof(U) * (n ? n : 1)));
        allocs_.push_back(p);
        return static_cast<U *>(p);
    }

    struct Layer {
        int in, out, in_p, out_p;
        float *W, *b, *gW, *gb, *mW, *vW, *mb, *vb;
        __nv_bfloat16 *W16, *Wt16;
        float *Z, *dz32, *dA;      // pre-activation; dZ; gradient w.r.t. this layer's input
        __nv_bfloat16 *A16, *dz16, *dzt16, *at16;
    };

    int din_, h_, L_, dout_, batch_;
    int step_ = 0;
    bool tcgen05_ = false;   // products on tcgen05 (else mma.sync); chosen at construction
    int *err_ = nullptr;     // set by a tcgen05 product whose wait timed out
    cudaStream_t stream_;
    std::vector<Layer> layers_;
    std::vector<void *> allocs_;
    __nv_bfloat16 *x16_ = nullptr;
    double *part_ = nullptr, *loss_ = nullptr;
};

// ---------------------------------------------------------------------------
// data helpers of the warm-start pipeline
// ---------------------------------------------------------------------------
// mean and standard deviation of every column (FP64 sums, one thread a column)
static __global__ void column_stats_kernel(const float *__restrict__ d, int64_t rows, int cols, float *mean,
                                           float *sd) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= cols) return;
    double s = 0.0, s2 = 0.0;
    for (int64_t r = 0; r < rows; ++r) {
        const double v = d[r * cols + c];
        s += v;
        s2 += v * v;
    }
    const double mu = s / (double)rows;
    const double var = fmax(s2 / (double)rows - mu * mu, 0.0);
    mean[c] = static_cast<float>(mu);
    sd[c] = static_cast<float>(fmax(sqrt(var), 1e-6 * (1.0 + fabs(mu))));
}

static __global__ void standardize_kernel(float *__restrict__ d, int64_t rows, int cols, const float *__restrict__ mean,
                                          const float *__restrict__ sd) {
    const int64_t total = rows * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int c = static_cast<int>(e % cols);
        d[e] = (d[e] - mean[c]) / sd[c];
    }
}

static __global__ void gather_rows_kernel(const float *__restrict__ src, int cols, const int64_t *__restrict__ idx,
                                          int64_t count, float *__restrict__ dst) {
    const int64_t total = count * cols;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / cols;
        const int c = static_cast<int>(e % cols);
        dst[e] = src[idx[r] * cols + c];
    }
}

// prediction (standardized (u_x, u_y, v_s, u_tau)) -> scaled warm start
// x^ = u_x / tau, y^ = u_y / tau, s^ = v_s / tau with tau = max(u_tau, tau_min)
static __global__ void warm_from_pred_kernel(const float *__restrict__ pred, int64_t ld, const float *__restrict__ mean,
                                             const float *__restrict__ sd, int n, int m, int64_t count, double tau_min,
                                             double *__restrict__ xh, double *__restrict__ yh, double *__restrict__ sh) {
    const int w = n + 2 * m;
    const int64_t total = count * w;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / w;
        const int c = static_cast<int>(e % w);
        const float *p = pred + b * ld;
        const double tau = fmax((double)p[w] * sd[w] + mean[w], tau_min);
        const double v = ((double)p[c] * sd[c] + mean[c]) / tau;
        if (c < n) xh[b * n + c] = v;
        else if (c < n + m) yh[b * m + c - n] = v;
        else sh[b * m + c - n - m] = v;
    }
}

}  // namespace mlp
}  // namespace scs

struct scs_mlp {
    scs::mlp::Net *net = nullptr;
    cudaStream_t stream = nullptr;
    bool own = false;
};

namespace {
template <typename F>
int32_t mlp_guarded(F f) {
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
int grid_of(int64_t len) { return static_cast<int>(std::min<int64_t>((len + 255) / 256, 4096)); }
}  // namespace

extern "C" {

scs_mlp *scs_mlp_create(int32_t d_in, int32_t hidden, int32_t layers, int32_t d_out, int32_t batch, void *stream,
                        int32_t *err) {
    scs_mlp *w = new scs_mlp;
    int32_t e = mlp_guarded([&]() -> int32_t {
        if (stream) {
            w->stream = static_cast<cudaStream_t>(stream);
        } else {
            SCS_CUDA(cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking));
            w->own = true;
        }
        w->net = new scs::mlp::Net(d_in, hidden, layers, d_out, batch, w->stream);
        return 0;
    });
    if (e) {
        delete w->net;
        if (w->own && w->stream) cudaStreamDestroy(w->stream);
        delete w;
        w = nullptr;
    }
    if (err) *err = e;
    return w;
}

int64_t scs_mlp_param_count(scs_mlp *w) { return w && w->net ? w->net->param_count() : -1; }

int32_t scs_mlp_set_params(scs_mlp *w, const float *params) {
    if (!w || !w->net || !params) return SCS_INVALID_INPUT;
    return mlp_guarded([&] { w->net->set_params(params); return 0; });
}

int32_t scs_mlp_get_params(scs_mlp *w, float *params) {
    if (!w || !w->net || !params) return SCS_INVALID_INPUT;
    return mlp_guarded([&] { w->net->get(params, false); return 0; });
}

int32_t scs_mlp_forward(scs_mlp *w, const float *x, float *y) {
    if (!w || !w->net || !x || !y) return SCS_INVALID_INPUT;
    return mlp_guarded([&] {
        w->net->forward(x);
        w->net->copy_output(y);
        SCS_CUDA(cudaStreamSynchronize(w->stream));
        return 0;
    });
}

int32_t scs_mlp_gradients(scs_mlp *w, const float *x, const float *t, float *grads, float *loss) {
    if (!w || !w->net || !x || !t) return SCS_INVALID_INPUT;
    return mlp_guarded([&] {
        w->net->backward(x, t);
        if (grads) w->net->get(grads, true);
        if (loss) *loss = static_cast<float>(w->net->loss_host());
        return 0;
    });
}

int32_t scs_mlp_train_step(scs_mlp *w, const float *x, const float *t, float lr, float *loss) {
    if (!w || !w->net || !x || !t) return SCS_INVALID_INPUT;
    return mlp_guarded([&] {
        w->net->backward(x, t);
        w->net->adam(lr);
        if (loss) *loss = static_cast<float>(w->net->loss_host());
        return 0;
    });
}

int32_t scs_mlp_set_tensor_path(scs_mlp *w, int32_t tcgen05) {
    if (!w || !w->net) return SCS_INVALID_INPUT;
    if (tcgen05) {
        for (const auto &Y : w->net->layers_)
            if (Y.in_p % scs::mlp::TBK || Y.out_p % scs::mlp::TBN || w->net->batch_ % scs::mlp::TBM ||
                Y.out_p % scs::mlp::TBK || w->net->batch_ % scs::mlp::TBK)
                return SCS_UNSUPPORTED;
    }
    w->net->tcgen05_ = tcgen05 != 0;
    return 0;
}

int32_t scs_mlp_error(scs_mlp *w) {
    if (!w || !w->net) return SCS_INVALID_INPUT;
    int h = 0;
    if (cudaMemcpy(&h, w->net->err_, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SCS_DEVICE_ERROR;
    return h ? SCS_DEVICE_ERROR : 0;
}

int32_t scs_bf16_gemm_async(const void *A, int32_t lda, const void *B, int32_t ldb, int32_t M, int32_t N, int32_t K,
                            float *C, int32_t ldc, int32_t tcgen05, int32_t *err, void *stream) {
    if (!A || !B || !C || !err || M <= 0 || N <= 0 || K <= 0 || ldc < N || ldc % 2) return SCS_INVALID_INPUT;
    return mlp_guarded([&]() -> int32_t {
        scs::mlp::launch_gemm(static_cast<const __nv_bfloat16 *>(A), lda, static_cast<const __nv_bfloat16 *>(B), ldb,
                              M, N, K, scs::mlp::EpiPlain{C, ldc}, tcgen05 != 0, reinterpret_cast<int *>(err),
                              static_cast<cudaStream_t>(stream));
        return 0;
    });
}

int32_t scs_bf16_gemm(const void *A, int32_t lda, const void *B, int32_t ldb, int32_t M, int32_t N, int32_t K,
                      float *C, int32_t ldc, int32_t tcgen05, void *stream) {
    if (!A || !B || !C || M <= 0 || N <= 0 || K <= 0 || ldc < N || ldc % 2) return SCS_INVALID_INPUT;
    return mlp_guarded([&]() -> int32_t {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        int *err = nullptr;
        SCS_CUDA(cudaMalloc(&err, sizeof(int)));
        int h = 0;
        try {
            SCS_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
            scs::mlp::launch_gemm(static_cast<const __nv_bfloat16 *>(A), lda, static_cast<const __nv_bfloat16 *>(B),
                                  ldb, M, N, K, scs::mlp::EpiPlain{C, ldc}, tcgen05 != 0, err, s);
            SCS_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
            SCS_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            cudaFree(err);
            throw;
        }
        cudaFree(err);
        return h ? SCS_DEVICE_ERROR : 0;
    });
}

void scs_mlp_destroy(scs_mlp *w) {
    if (!w) return;
    delete w->net;
    if (w->own && w->stream) cudaStreamDestroy(w->stream);
    delete w;
}

int32_t scs_column_stats(const float *data, int64_t rows, int32_t cols, float *mean, float *sd, void *stream) {
    if (!data || rows <= 0 || cols <= 0 || !mean || !sd) return SCS_INVALID_INPUT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    scs::mlp::column_stats_kernel<<<(cols + 127) / 128, 128, 0, s>>>(data, rows, cols, mean, sd);
    return cudaGetLastError() == cudaSuccess ? 0 : SCS_DEVICE_ERROR;
}

int32_t scs_standardize(float *data, int64_t rows, int32_t cols, const float *mean, const float *sd, void *stream) {
    if (!data || rows <= 0 || cols <= 0 || !mean || !sd) return SCS_INVALID_INPUT;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    scs::mlp::standardize_kernel<<<grid_of(rows * cols), 256, 0, s>>>(data, rows, cols, mean, sd);
    return cudaGetLastError() == cudaSuccess ? 0 : SCS_DEVICE_ERROR;
}

int32_t scs_gather_rows(const float *src, int32_t cols, const int64_t *idx, int64_t count, float *dst, void *stream) {
    if (!src || cols <= 0 || !idx || count < 0 || !dst) return SCS_INVALID_INPUT;
    if (!count) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    scs::mlp::gather_rows_kernel<<<grid_of(count * cols), 256, 0, s>>>(src, cols, idx, count, dst);
    return cudaGetLastError() == cudaSuccess ? 0 : SCS_DEVICE_ERROR;
}

int32_t scs_warm_from_prediction(const float *pred, int64_t ld, const float *mean, const float *sd, int32_t n,
                                 int32_t m, int64_t count, double tau_min, double *xh, double *yh, double *sh,
                                 void *stream) {
    if (!pred || !mean || !sd || n <= 0 || m <= 0 || count < 0 || ld < n + 2 * m + 1 || !xh || !yh || !sh ||
        !(tau_min > 0))
        return SCS_INVALID_INPUT;
    if (!count) return 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    scs::mlp::warm_from_pred_kernel<<<grid_of(count * (n + 2 * m)), 256, 0, s>>>(pred, ld, mean, sd, n, m, count,
                                                                                  tau_min, xh, yh, sh);
    return cudaGetLastError() == cudaSuccess ? 0 : SCS_DEVICE_ERROR;
}

}  // extern "C"
