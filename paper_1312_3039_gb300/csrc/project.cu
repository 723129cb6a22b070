// Stand-alone cone projection of a batch of vectors on the device
// (scs_project): Euclidean projection onto K or K* block by block, with the
// squared distance moved summed by a deterministic grid reduction.  The
// same projections as the iteration's kernels (zero/free, nonnegative,
// second-order, PSD by a cold-started Jacobi eigensolver, exponential via
// Moreau, power and its dual via Moreau); used to put predicted warm starts
// back into the cones.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/scs_gpu.h"
#include "common.cuh"
#include "cones.cuh"
#include "engine_base.h"
#include "psd.cuh"

namespace scs {

struct ProjCone {
    int m;                 // rows of one vector
    int z, l;
    int nq;
    const int32_t *q_off;  // row offset of each SOC block
    const int32_t *q_len;
    int ep;                // exponential triples, then dual exponential ones,
    int ed;                // then power triples (pow_a[i] < 0: dual power cone)
    int np;
    const double *pow_a;
    int exp_off;
    int64_t count;         // vectors
    int g_elem, g_soc, g_exp;   // CTAs of each region (grid-stride inside)
    int g_psd;             // CTAs of the PSD launch that ran before (0: none)
    const double *psd_dd;  // their squared distances
};

// Regions: [0, g_exp) exponential, dual exponential and power triples (64
// per CTA pass), then
// [.., + g_soc) one warp per SOC block, then the elementwise rows.
__global__ void __launch_bounds__(kBlock) cone_project_kernel(ProjCone P, int dual, const double *__restrict__ v,
                                                              double *__restrict__ out, ReduceBuf rb,
                                                              double *dist2) {
    double dd = 0.0;
    const int b = blockIdx.x;
    if (b < P.g_exp) {
        const int per = P.ep + P.ed + P.np;
        const int64_t ntri = P.count * per;
        for (int64_t t = (int64_t)b * 64 + threadIdx.x; threadIdx.x < 64 && t < ntri; t += (int64_t)P.g_exp * 64) {
            const int64_t vec = t / per;
            const int tri = static_cast<int>(t % per);
            const int64_t off = vec * P.m + P.exp_off + 3 * tri;
            const double a0 = v[off], a1 = v[off + 1], a2 = v[off + 2];
            double p0, p1, p2;
            if (tri < P.ep + P.ed) {
                // K* of Kexp is Kexp*, of Kexp* is Kexp: onto Kexp* when exactly one holds
                if ((dual != 0) != (tri >= P.ep)) proj_exp_dual(a0, a1, a2, p0, p1, p2);
                else proj_exp(a0, a1, a2, p0, p1, p2);
            } else {
                const double pa = P.pow_a[tri - P.ep - P.ed];
                if ((dual != 0) != (pa < 0.0)) proj_pow_dual(a0, a1, a2, fabs(pa), p0, p1, p2);
                else proj_pow(a0, a1, a2, fabs(pa), p0, p1, p2);
            }
            out[off] = p0; out[off + 1] = p1; out[off + 2] = p2;
            dd += (p0 - a0) * (p0 - a0) + (p1 - a1) * (p1 - a1) + (p2 - a2) * (p2 - a2);
        }
    } else if (b < P.g_exp + P.g_soc) {
        const int lane = threadIdx.x & 31;
        const int64_t nblk = P.count * P.nq;
        const int64_t w0 = (int64_t)(b - P.g_exp) * kWarps + (threadIdx.x >> 5);
        for (int64_t w = w0; w < nblk; w += (int64_t)P.g_soc * kWarps) {
            const int64_t vec = w / P.nq, blk = w % P.nq;
            const int64_t off = vec * P.m + P.q_off[blk];
            const int len = P.q_len[blk];
            double t0 = 0.0, xx = 0.0;
            for (int e = lane; e < len; e += 32) {
                const double t = v[off + e];
                if (e == 0) t0 = t; else xx += t * t;
            }
            xx = warp_sum(xx);
            t0 = __shfl_sync(0xffffffffu, t0, 0);
            const double nx = sqrt(xx);
            double head, tail;
            if (nx <= t0) { head = t0; tail = 1.0; }
            else if (nx <= -t0) { head = 0.0; tail = 0.0; }
            else { head = 0.5 * (t0 + nx); tail = head / nx; }
            for (int e = lane; e < len; e += 32) {
                const double t = v[off + e];
                const double p = e == 0 ? head : tail * t;
                out[off + e] = p;
                dd += (p - t) * (p - t);
            }
        }
    } else {
        const int64_t lin = (int64_t)P.z + P.l;
        const int64_t total = P.count * lin;
        for (int64_t i = (int64_t)(b - P.g_exp - P.g_soc) * kBlock + threadIdx.x; i < total;
             i += (int64_t)P.g_elem * kBlock) {
            const int64_t vec = i / lin, row = i % lin;
            const int64_t off = vec * P.m + row;
            const double t = v[off];
            double p;
            if (row < P.z) p = dual ? t : 0.0;       // K* of {0} is R
            else p = fmax(t, 0.0);
            out[off] = p;
            dd += (p - t) * (p - t);
        }
    }
    double red[1] = {dd}, tot[1];
    if (grid_sum<1>(red, rb, kSiteMisc, tot)) {
        if (threadIdx.x < 32) {
            double extra = 0.0;
            for (int c = threadIdx.x; c < P.g_psd; c += 32) extra += P.psd_dd[c];
            extra = warp_sum(extra);
            if (threadIdx.x == 0) *dist2 = tot[0] + extra;
        }
    }
}

// PSD blocks of a batch: one CTA per (vector, block) pair in grid-stride
// order, FP64, Jacobi from V = I (nothing is kept between calls).  The
// CTA's squared distance goes to dd[blockIdx.x].
struct PsdBatchIO {
    const double *src;
    double *dst;
    int64_t base;
    double dd;
    __device__ double in(int64_t s) const { return src[base + s]; }
    __device__ void out(int64_t s, double p) {
        const double t = src[base + s];
        dst[base + s] = p;
        dd += (p - t) * (p - t);
    }
};

template <bool kSm>
__global__ void __launch_bounds__(kPsdThreads, 1) psd_batch_kernel(const double *__restrict__ v, double *out, int m,
                                                                const int32_t *ord, const int32_t *off, int nblk,
                                                                int64_t count, double *work, int64_t work_stride,
                                                                int small_bytes, int ne_max, double *dd) {
    extern __shared__ __align__(16) unsigned char psd_smem[];
    const PsdSmall<double> sm = psd_small_tables<double>(psd_smem, ne_max);
    double acc = 0.0;
    for (int64_t pr = blockIdx.x; pr < count * nblk; pr += gridDim.x) {
        const int64_t vec = pr / nblk;
        const int blk = static_cast<int>(pr % nblk);
        const int n = ord[blk];
        const int ne = psd_ne(n), ld = ne + 1;
        double *X, *V, *W, *Wsub = nullptr;
        if constexpr (kSm) {
            X = reinterpret_cast<double *>(psd_smem + small_bytes);
            V = X + ne * ld;
            W = V + ne * ld;
        } else {
            X = work + (size_t)blockIdx.x * 3 * work_stride;
            V = X + work_stride;
            W = V + work_stride;
            if (psd_sub_on_chip<double>(ne_max)) Wsub = reinterpret_cast<double *>(psd_smem + small_bytes);
        }
        PsdBatchIO io{v, out, vec * m + off[blk], 0.0};
        psd_project_block<double>(io, n, X, V, W, nullptr, sm, PsdStats{nullptr, nullptr, nullptr}, 0.0, Wsub);
        acc += io.dd;
    }
    acc = psd_block_sum(acc, sm.red);
    if (threadIdx.x == 0) dd[blockIdx.x] = acc;
}

// Region grids for a batch (each region gets CTAs only if it has work).
inline void project_grid(ProjCone &P, int max_ctas) {
    const int64_t lin = P.count * ((int64_t)P.z + P.l);
    const int64_t soc = P.count * P.nq, exp_ = P.count * ((int64_t)P.ep + P.ed + P.np);
    P.g_exp = exp_ ? (int)std::min<int64_t>((exp_ + 63) / 64, max_ctas / 4) : 0;
    P.g_soc = soc ? (int)std::min<int64_t>((soc + kWarps - 1) / kWarps, max_ctas / 4) : 0;
    P.g_elem = lin ? (int)std::min<int64_t>((lin + kBlock - 1) / kBlock, max_ctas / 2) : 0;
    if (P.g_exp + P.g_soc + P.g_elem == 0) P.g_elem = 1;
    if (P.g_exp == 0 && exp_) P.g_exp = 1;
    if (P.g_soc == 0 && soc) P.g_soc = 1;
}

// Validate the cone, fill the SOC tables (host) and the row offsets.
inline int project_setup(const scs_cone *k, int64_t count, ProjCone &P, std::vector<int32_t> &qoff,
                         std::vector<int32_t> &qlen, std::vector<int32_t> &soff, std::string &err) {
    if (!k || count < 0) { err = "bad argument"; return SCS_INVALID_INPUT; }
    if (k->z < 0 || k->l < 0 || k->nq < 0 || k->ns < 0 || k->ep < 0 || k->ed < 0 || k->np < 0 ||
        (k->nq > 0 && !k->q) || (k->ns > 0 && !k->s) || (k->np > 0 && !k->p)) {
        err = "bad cone";
        return SCS_INVALID_INPUT;
    }
    for (int i = 0; i < k->np; ++i)
        if (!(fabs(k->p[i]) > 0.0 && fabs(k->p[i]) < 1.0)) {
            err = "power cone parameter must lie in (-1, 0) or (0, 1)";
            return SCS_INVALID_INPUT;
        }
    int64_t off = (int64_t)k->z + k->l;
    qoff.clear();
    qlen.clear();
    soff.clear();
    for (int i = 0; i < k->nq; ++i) {
        if (k->q[i] < 1) { err = "SOC size must be >= 1"; return SCS_INVALID_INPUT; }
        qoff.push_back((int32_t)off);
        qlen.push_back(k->q[i]);
        off += k->q[i];
    }
    for (int i = 0; i < k->ns; ++i) {
        if (k->s[i] < 1) { err = "PSD order must be >= 1"; return SCS_INVALID_INPUT; }
        if (k->s[i] > kPsdMaxOrder) { err = "PSD order above 1024"; return SCS_UNSUPPORTED; }
        soff.push_back((int32_t)off);
        off += (int64_t)k->s[i] * (k->s[i] + 1) / 2;
        if (off > (int64_t)1 << 30) { err = "cone too large"; return SCS_UNSUPPORTED; }
    }
    P.exp_off = (int)off;
    off += 3 * ((int64_t)k->ep + k->ed + k->np);
    if (off > (int64_t)1 << 30) { err = "cone too large"; return SCS_UNSUPPORTED; }
    P.m = (int)off;
    P.z = k->z;
    P.l = k->l;
    P.nq = k->nq;
    P.ep = k->ep;
    P.ed = k->ed;
    P.np = k->np;
    P.count = count;
    return 0;
}

}  // namespace scs

extern "C" int32_t scs_project(const scs_cone *k, int32_t dual, const double *v, double *out, int64_t count,
                               double *dist2, void *stream) {
    using namespace scs;
    ProjCone P{};
    std::vector<int32_t> qoff, qlen, soff;
    std::string err;
    int rc = project_setup(k, count, P, qoff, qlen, soff, err);
    if (rc) {
        set_last_error("scs_project: " + err);
        return rc;
    }
    if (count == 0 || P.m == 0) {
        if (dist2) *dist2 = 0.0;
        return 0;
    }
    if (!v || !out) {
        set_last_error("scs_project: v and out must be device pointers");
        return SCS_INVALID_INPUT;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) {
        set_last_error("scs_project: no usable CUDA device");
        return SCS_DEVICE_ERROR;
    }
    project_grid(P, sms * 8);
    const int grid = P.g_exp + P.g_soc + P.g_elem;
    // PSD launch: one CTA per (vector, block) pair up to 4 per SM
    const int nps = static_cast<int>(soff.size());
    int n_max = 0;
    for (int i = 0; i < nps; ++i) n_max = std::max(n_max, (int)k->s[i]);
    const int g_psd = nps ? (int)std::min<int64_t>(count * nps, (int64_t)sms * 4) : 0;
    bool on_chip = false;
    const size_t psd_smem = nps ? psd_smem_bytes<double>(n_max, on_chip) : 0;
    const int64_t wstride = nps ? psd_mat_elems(n_max) : 0;
    // scratch for this call: partial sums, arrival counters, SOC and PSD
    // tables, result, PSD partial sums and (large orders) PSD matrices
    double *partials = nullptr, *res = nullptr, *psd_dd = nullptr, *psd_work = nullptr, *pow_tab = nullptr;
    unsigned *counter = nullptr;
    int32_t *tables = nullptr;
    rc = 0;
    const size_t ntab = 2 * qoff.size() + 2 * soff.size() + 2;
    if (cudaMalloc(&partials, sizeof(double) * kMaxRed * grid) || cudaMalloc(&counter, sizeof(unsigned) * kSiteCount) ||
        cudaMalloc(&res, sizeof(double)) || cudaMalloc(&tables, sizeof(int32_t) * ntab) ||
        (nps && cudaMalloc(&psd_dd, sizeof(double) * g_psd)) ||
        (nps && !on_chip && cudaMalloc(&psd_work, sizeof(double) * 3 * wstride * g_psd)) ||
        (k->np > 0 && cudaMalloc(&pow_tab, sizeof(double) * k->np)))
        rc = SCS_DEVICE_ERROR;
    int32_t *t_soff = tables + 2 * qoff.size(), *t_sord = t_soff + soff.size();
    if (!rc) {
        if (!qoff.empty() && (cudaMemcpyAsync(tables, qoff.data(), 4 * qoff.size(), cudaMemcpyHostToDevice, s) ||
                              cudaMemcpyAsync(tables + qoff.size(), qlen.data(), 4 * qlen.size(),
                                              cudaMemcpyHostToDevice, s)))
            rc = SCS_DEVICE_ERROR;
        if (nps && (cudaMemcpyAsync(t_soff, soff.data(), 4 * soff.size(), cudaMemcpyHostToDevice, s) ||
                    cudaMemcpyAsync(t_sord, k->s, 4 * soff.size(), cudaMemcpyHostToDevice, s)))
            rc = SCS_DEVICE_ERROR;
        if (cudaMemsetAsync(counter, 0, sizeof(unsigned) * kSiteCount, s)) rc = SCS_DEVICE_ERROR;
        if (k->np > 0 && cudaMemcpyAsync(pow_tab, k->p, sizeof(double) * k->np, cudaMemcpyHostToDevice, s))
            rc = SCS_DEVICE_ERROR;
    }
    if (!rc && nps) {
        auto kern = on_chip ? psd_batch_kernel<true> : psd_batch_kernel<false>;
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)psd_smem))
            rc = SCS_DEVICE_ERROR;
        if (!rc) {
            kern<<<g_psd, kPsdThreads, psd_smem, s>>>(v, out, P.m, t_sord, t_soff, nps, count, psd_work, wstride,
                                                       (int)psd_small_bytes<double>(psd_ne(n_max)), psd_ne(n_max),
                                                       psd_dd);
            P.g_psd = g_psd;
            P.psd_dd = psd_dd;
        }
    }
    if (!rc) {
        P.q_off = tables;
        P.q_len = tables + qoff.size();
        P.pow_a = pow_tab;
        ReduceBuf rb{partials, counter, grid};
        cone_project_kernel<<<grid, kBlock, 0, s>>>(P, dual ? 1 : 0, v, out, rb, res);
        double h = 0.0;
        if (cudaGetLastError() || cudaMemcpyAsync(&h, res, sizeof(double), cudaMemcpyDeviceToHost, s) ||
            cudaStreamSynchronize(s))
            rc = SCS_DEVICE_ERROR;
        if (!rc && dist2) *dist2 = h;
    }
    cudaFree(partials);
    cudaFree(counter);
    cudaFree(res);
    cudaFree(tables);
    cudaFree(psd_dd);
    cudaFree(psd_work);
    cudaFree(pow_tab);
    if (rc) set_last_error("scs_project: CUDA call failed");
    return rc;
}

// ---------------------------------------------------------------------------
// scs_project_noalloc: the same projection for callers that may not allocate
// device memory -- for example an application whose own memory pool has
// reserved the whole GPU, or a serving process that hands the library fixed
// buffers and a stream and keeps every allocation under its own control.
// Its scratch -- the reduction's arrival counters and partial sums, the SOC
// block tables and the result -- lives in one file-scope device array of
// fixed size, held by every GPU that loads the library until the process
// exits.
// ---------------------------------------------------------------------------
namespace scs {

constexpr int kNoAllocMaxCtas = 1024;      // CTAs of one projection launch
constexpr int kNoAllocMaxSoc = 4096;       // SOC blocks per cone
constexpr size_t kNoAllocCounterOff = 0;                                   // kSiteCount unsigned
constexpr size_t kNoAllocResultOff = 128;                                  // one double
constexpr size_t kNoAllocPartialOff = 256;                                 // kNoAllocMaxCtas doubles
constexpr size_t kNoAllocTableOff = kNoAllocPartialOff + 8 * kNoAllocMaxCtas;   // 2 * kNoAllocMaxSoc int32
constexpr size_t kNoAllocBytes = kNoAllocTableOff + 8 * kNoAllocMaxSoc;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the scratch array, looked up once per device and per
// CUDA context: the address belongs to the context that was current at the
// lookup, so a new context on the device (after cudaDeviceReset, or another
// context made current) triggers a new lookup.
struct NoAllocAddr {
    unsigned long long ctx;   // unique id of the context of the lookup (0: none)
    void *addr;
};
static NoAllocAddr g_noalloc_addr[kNoAllocMaxDevices];
static std::mutex g_noalloc_mutex;

// Unique id of the calling thread's current CUDA context, or 0 when there is
// none or the driver cannot report it (then nothing is cached).  The driver
// functions are reached through the runtime's entry-point query, so the
// library does not link the driver library itself.
static unsigned long long current_context_id() {
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult qf, qg;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &qf) == cudaSuccess &&
            qf == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &qg) == cudaSuccess &&
            qg == cudaDriverEntryPointSuccess && f && g) {
            get_current = reinterpret_cast<GetCurrent>(f);
            get_id = reinterpret_cast<GetId>(g);
        }
    });
    if (!get_current || !get_id) return 0;
    CUcontext c = nullptr;
    unsigned long long id = 0;
    if (get_current(&c) != CUDA_SUCCESS || !c || get_id(c, &id) != CUDA_SUCCESS) return 0;
    return id + 1;   // 0 stays "unknown"
}

}  // namespace scs

extern "C" int32_t scs_project_noalloc(const scs_cone *k, int32_t dual, const double *v, double *out,
                                       int64_t count, double *dist2, void *stream) {
    using namespace scs;
    ProjCone P{};
    std::vector<int32_t> qoff, qlen, soff;
    std::string err;
    int rc = project_setup(k, count, P, qoff, qlen, soff, err);
    if (rc) {
        set_last_error("scs_project_noalloc: " + err);
        return rc;
    }
    if ((int64_t)qoff.size() > kNoAllocMaxSoc) {
        set_last_error("scs_project_noalloc: more than " + std::to_string(kNoAllocMaxSoc) +
                       " SOC blocks in the cone (the fixed scratch holds the tables of at most that many)");
        return SCS_UNSUPPORTED;
    }
    if (!soff.empty()) {
        set_last_error("scs_project_noalloc: PSD blocks need eigensolver matrix scratch; use scs_project");
        return SCS_UNSUPPORTED;
    }
    if (k->np > 0) {
        set_last_error("scs_project_noalloc: power cones need a parameter table; use scs_project");
        return SCS_UNSUPPORTED;
    }
    if (count == 0 || P.m == 0) {
        if (dist2) *dist2 = 0.0;
        return 0;
    }
    if (!v || !out) {
        set_last_error("scs_project_noalloc: v and out must be device pointers");
        return SCS_INVALID_INPUT;
    }
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        set_last_error("scs_project_noalloc: no usable CUDA device (or device ordinal of 64 or more)");
        return SCS_DEVICE_ERROR;
    }
    void *base = nullptr;
    unsigned long long ctx = current_context_id();
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (ctx && g_noalloc_addr[dev].ctx == ctx) base = g_noalloc_addr[dev].addr;
    }
    if (!base) {
        // set-up for this device and context, with the device current: host
        // code cannot use the array's host-side name as a device pointer
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            set_last_error("scs_project_noalloc: cudaGetSymbolAddress of the scratch array failed");
            return SCS_DEVICE_ERROR;
        }
        ctx = current_context_id();   // the lookup creates the context if there was none
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        g_noalloc_addr[dev] = NoAllocAddr{ctx, p};
        base = p;
    }
    unsigned char *sc = static_cast<unsigned char *>(base);
    unsigned *counter = reinterpret_cast<unsigned *>(sc + kNoAllocCounterOff);
    double *res = reinterpret_cast<double *>(sc + kNoAllocResultOff);
    double *partials = reinterpret_cast<double *>(sc + kNoAllocPartialOff);
    int32_t *tables = reinterpret_cast<int32_t *>(sc + kNoAllocTableOff);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    project_grid(P, std::min(sms * 8, kNoAllocMaxCtas));
    const int grid = P.g_exp + P.g_soc + P.g_elem;
    if (grid > kNoAllocMaxCtas) {
        set_last_error("scs_project_noalloc: launch grid above the scratch's 1024 CTAs");
        return SCS_UNSUPPORTED;
    }
    // the counters must start at zero (the array keeps the last call's contents)
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned) * kSiteCount, s) != cudaSuccess) {
        set_last_error("scs_project_noalloc: clearing the scratch counters failed");
        return SCS_DEVICE_ERROR;
    }
    if (!qoff.empty()) {
        if (cudaMemcpyAsync(tables, qoff.data(), 4 * qoff.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(tables + kNoAllocMaxSoc, qlen.data(), 4 * qlen.size(), cudaMemcpyHostToDevice, s) !=
                cudaSuccess) {
            set_last_error("scs_project_noalloc: copying the SOC tables failed");
            return SCS_DEVICE_ERROR;
        }
    }
    P.q_off = tables;
    P.q_len = tables + kNoAllocMaxSoc;
    ReduceBuf rb{partials, counter, grid};
    cone_project_kernel<<<grid, kBlock, 0, s>>>(P, dual ? 1 : 0, v, out, rb, res);
    double h = 0.0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h, res, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_last_error("scs_project_noalloc: the projection launch or its read-back failed");
        return SCS_DEVICE_ERROR;
    }
    if (dist2) *dist2 = h;
    return 0;
}
