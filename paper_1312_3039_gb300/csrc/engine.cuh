// Host side of the device solver: owns the device buffers of one problem,
// performs the setup (equilibration, preconditioner, cached M^-1 h), records
// one ADMM iteration as a CUDA graph whose CG loop is a device-driven
// conditional WHILE node, and runs the solve loop with a termination test
// every `check_interval` iterations.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <stdexcept>
#include <type_traits>
#include <string>
#include <vector>

#include "../../include/scs_gpu.h"
#include "dense.cuh"
#include "engine_base.h"
#include "kernels.cuh"

namespace scs {

// largest n of the direct subspace step (the dense inverse: 512 MB in FP64)
constexpr int kDirectMaxN = 8192;

template <typename T>
class Engine : public EngineBase {
   public:
    Engine(const HostProblem &P, const scs_settings &st) : st_(st) {
        const auto t0 = std::chrono::steady_clock::now();
        m_ = P.m;
        n_ = P.n;
        N_ = n_ + m_ + 1;
        nnz_ = P.nnz;
        SCS_CUDA(cudaSetDevice(st.device));
        device_ = st.device;
        cudaDeviceProp prop;
        SCS_CUDA(cudaGetDeviceProperties(&prop, device_));
        sms_ = prop.multiProcessorCount;
        if (st.cuda_stream) {
            stream_ = static_cast<cudaStream_t>(st.cuda_stream);
        } else {
            SCS_CUDA(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
            own_stream_ = true;
        }
        SCS_CUDA(cudaStreamCreateWithFlags(&body_stream_, cudaStreamNonBlocking));
        cur_ = stream_;
        SCS_CUDA(cudaMallocHost(&Sh_, sizeof(Scalars)));
        setup(P);
        setup_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }

    ~Engine() override {
        cudaSetDevice(device_);
        if (exec_) cudaGraphExecDestroy(exec_);
        if (graph_) cudaGraphDestroy(graph_);
        for (auto &e : ev_) cudaEventDestroy(e);
        for (void *p : allocs_) cudaFree(p);
        if (Sh_) cudaFreeHost(Sh_);
        if (body_stream_) cudaStreamDestroy(body_stream_);
        if (own_stream_ && stream_) cudaStreamDestroy(stream_);
    }

    // -------------------------------------------------------------------
    int reset() override {
        SCS_CUDA(cudaSetDevice(device_));
        set_initial_point();
        SCS_CUDA(cudaStreamSynchronize(stream_));
        warm_pending_ = false;
        return 0;
    }

    int warm_start(const double *x, const double *y, const double *s) override {
        SCS_CUDA(cudaSetDevice(device_));
        // Sec. 4.2: u0 = (x, y, 1), v0 = (0, s, 0) in the scaled problem:
        // x^ = sigma E^-1 x, y^ = rho D^-1 y, s^ = sigma D s
        std::vector<double> u(N_, 0.0), v(N_, 0.0);
        for (int j = 0; j < n_; ++j) u[j] = x ? sigma_ * x[j] / Eh_[j] : 0.0;
        for (int i = 0; i < m_; ++i) {
            u[n_ + i] = y ? rho_ * y[i] / Dh_[i] : 0.0;
            v[n_ + i] = s ? sigma_ * Dh_[i] * s[i] : 0.0;
        }
        u[N_ - 1] = 1.0;
        v[N_ - 1] = 0.0;
        std::vector<T> ut(u.begin(), u.end()), vt(v.begin(), v.end());
        SCS_CUDA(cudaMemcpyAsync(u_, ut.data(), sizeof(T) * N_, cudaMemcpyHostToDevice, stream_));
        SCS_CUDA(cudaMemcpyAsync(v_, vt.data(), sizeof(T) * N_, cudaMemcpyHostToDevice, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        // the warm start is taken to be about as accurate as the tolerances
        double nrm = 0.0;
        for (int i = 0; i < N_; ++i) nrm += u[i] * u[i] + v[i] * v[i];
        reset_counters(std::max(st_.eps_pri, std::max(st_.eps_dual, st_.eps_gap)) * std::sqrt(nrm));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        warm_pending_ = true;
        return 0;
    }

    int iterate(int iters, int sync) override {
        SCS_CUDA(cudaSetDevice(device_));
        run_iters(iters);
        if (sync) SCS_CUDA(cudaStreamSynchronize(stream_));
        return 0;
    }

    // the solve loop's work without its stopping rule: check_interval
    // iterations, the Sec. 3.5 test launch and the host read of the status
    // word, repeated until `iters` iterations are done
    int iterate_checked(int iters, int32_t *status) override {
        SCS_CUDA(cudaSetDevice(device_));
        const int ci = st_.check_interval > 0 ? st_.check_interval : 1;
        for (int k = 0; k < iters;) {
            const int chunk = std::min(ci, iters - k);
            run_iters(chunk);
            k += chunk;
            launch_check();
            SCS_CUDA(cudaMemcpyAsync(Sh_, S_, sizeof(Scalars), cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaStreamSynchronize(stream_));
            if (Sh_->dev_error) throw CudaError("a device wait timed out", SCS_DEVICE_ERROR);
        }
        if (status) *status = iters > 0 ? Sh_->status : 0;
        return 0;
    }

    int iterate_profiled(int iters) override {
        SCS_CUDA(cudaSetDevice(device_));
        if (ev_.empty()) {
            ev_.resize(2);
            for (auto &e : ev_) SCS_CUDA(cudaEventCreate(&e));
        }
        for (int it = 0; it < iters; ++it) {
            if (direct_) {
                launch_K1();
                timed(1, [&] { launch_K2(CondHandle{0, 0}); });
                timed(4, [&] { launch_D1(); launch_D2(); });
                launch_K6();
                if (psd_.npsd) timed(3, [&] { launch_KP(); });
                timed(2, [&] { launch_K7(); });
                continue;
            }
            launch_K1();                  // kind 0 times the CG products q = A p only
            timed(1, [&] { launch_K2(CondHandle{0, 0}); });
            for (int c = 0; c < st_.cg_max_iters; ++c) {
                timed(0, [&] { launch_K3(); });
                timed(1, [&] { launch_K4(); });
                launch_K5(CondHandle{0, 0});
                SCS_CUDA(cudaMemcpyAsync(Sh_, S_, sizeof(Scalars), cudaMemcpyDeviceToHost, stream_));
                SCS_CUDA(cudaStreamSynchronize(stream_));
                if (!Sh_->active) break;
            }
            launch_K6();
            if (psd_.npsd) timed(3, [&] { launch_KP(); });
            timed(2, [&] { launch_K7(); });
        }
        SCS_CUDA(cudaStreamSynchronize(stream_));
        return 0;
    }

    int kernel_time(int kind, double *ms, int64_t *launches) override {
        if (kind < 0 || kind > 4) return SCS_INVALID_INPUT;
        if (ms) *ms = prof_ms_[kind];
        if (launches) *launches = prof_n_[kind];
        prof_ms_[kind] = 0.0;
        prof_n_[kind] = 0;
        return 0;
    }

    int get_iterates(double *u, double *v) override {
        SCS_CUDA(cudaSetDevice(device_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        std::vector<T> h(N_);
        if (u) {
            SCS_CUDA(cudaMemcpy(h.data(), u_, sizeof(T) * N_, cudaMemcpyDeviceToHost));
            for (int i = 0; i < N_; ++i) u[i] = static_cast<double>(h[i]);
        }
        if (v) {
            SCS_CUDA(cudaMemcpy(h.data(), v_, sizeof(T) * N_, cudaMemcpyDeviceToHost));
            for (int i = 0; i < N_; ++i) v[i] = static_cast<double>(h[i]);
        }
        return 0;
    }

    int get_scaling(double *D, double *E, double *sigma, double *rho) override {
        if (D) std::memcpy(D, Dh_.data(), sizeof(double) * m_);
        if (E) std::memcpy(E, Eh_.data(), sizeof(double) * n_);
        if (sigma) *sigma = sigma_;
        if (rho) *rho = rho_;
        return 0;
    }

    void dims(int32_t *m, int32_t *n, int64_t *nnz, int64_t *bytes) override {
        if (m) *m = m_;
        if (n) *n = n_;
        if (nnz) *nnz = nnz_;
        if (bytes) *bytes = bytes_;
    }

    int psd_counters(int64_t *calls, int64_t *sweeps, int64_t *fp64) override {
        SCS_CUDA(cudaSetDevice(device_));
        SCS_CUDA(cudaMemcpyAsync(Sh_, S_, sizeof(Scalars), cudaMemcpyDeviceToHost, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        if (calls) *calls = static_cast<int64_t>(Sh_->psd_calls);
        if (sweeps) *sweeps = static_cast<int64_t>(Sh_->psd_sweeps);
        if (fp64) *fp64 = static_cast<int64_t>(Sh_->psd_fp64);
        return 0;
    }

    int counters(int32_t *iters, int64_t *cg_iters) override {
        SCS_CUDA(cudaSetDevice(device_));
        SCS_CUDA(cudaMemcpyAsync(Sh_, S_, sizeof(Scalars), cudaMemcpyDeviceToHost, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        if (Sh_->dev_error) throw CudaError("a device wait timed out", SCS_DEVICE_ERROR);
        if (iters) *iters = Sh_->k;
        if (cg_iters) *cg_iters = Sh_->cg_total;
        return 0;
    }

    int solve(double *x, double *y, double *s, scs_info *info) override {
        SCS_CUDA(cudaSetDevice(device_));
        const auto t0 = std::chrono::steady_clock::now();
        if (!warm_pending_) set_initial_point();
        warm_pending_ = false;
        int status = 0;
        bool timed_out = false;
        int k = 0;
        const int ci = st_.check_interval > 0 ? st_.check_interval : 1;
        for (;;) {
            const int chunk = std::min(ci, st_.max_iters - k);
            if (chunk > 0) run_iters(chunk);
            k += chunk > 0 ? chunk : 0;
            launch_check();
            SCS_CUDA(cudaMemcpyAsync(Sh_, S_, sizeof(Scalars), cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaStreamSynchronize(stream_));
            status = Sh_->status;
            if (Sh_->dev_error) throw CudaError("a device wait timed out", SCS_DEVICE_ERROR);
            if (status != 0 || k >= st_.max_iters) break;
            if (st_.time_limit_s > 0) {
                const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
                if (el > st_.time_limit_s) { timed_out = true; break; }
            }
        }
        if (status == 0) status = inaccurate_status();
        (void)timed_out;
        // outputs
        output_kernel<T><<<grid_for(n_ + 2 * m_), kBlock, 0, stream_>>>(n_, m_, status, u_, v_, D_, E_, ax_, S_,
                                                                    out_, out_ + n_, out_ + n_ + m_);
        SCS_CUDA(cudaGetLastError());
        // host or device outputs: unified addressing tells them apart
        if (x) SCS_CUDA(cudaMemcpyAsync(x, out_, sizeof(double) * n_, cudaMemcpyDefault, stream_));
        if (y) SCS_CUDA(cudaMemcpyAsync(y, out_ + n_, sizeof(double) * m_, cudaMemcpyDefault, stream_));
        if (s) SCS_CUDA(cudaMemcpyAsync(s, out_ + n_ + m_, sizeof(double) * m_, cudaMemcpyDefault, stream_));
        SCS_CUDA(cudaMemcpyAsync(Sh_, S_, sizeof(Scalars), cudaMemcpyDeviceToHost, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        if (info) {
            info->status = status;
            info->iters = Sh_->k;
            info->cg_iters = static_cast<int32_t>(Sh_->cg_total);
            info->matvecs = Sh_->k + (Sh_->k + kAzEvery - 1) / kAzEvery + 2 * static_cast<int32_t>(Sh_->cg_total) +
                            (direct_ ? Sh_->k : 0);     // the direct step's A d
            info->tau = Sh_->tau;
            info->kappa = Sh_->kappa;
            info->res_pri = Sh_->res_pri;
            info->res_dual = Sh_->res_dual;
            info->gap = Sh_->gap;
            if (status == 1 || status == 2) {
                info->pobj = Sh_->pobj;
                info->dobj = Sh_->dobj;
            } else if (status == -1 || status == -3) {
                info->pobj = NAN;
                info->dobj = 1.0;
            } else if (status == -2 || status == -4) {
                info->pobj = -1.0;
                info->dobj = NAN;
            } else {
                info->pobj = info->dobj = NAN;
            }
            info->setup_s = setup_s;
            info->solve_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        }
        return status;
    }

    // internals (public so that extended device lambdas may be defined in them)
    // ------------------------------------------------------------------ memory
    template <typename U>
    U *dalloc(size_t count) {
        void *p = nullptr;
        if (count == 0) count = 1;
        SCS_CUDA(cudaMalloc(&p, sizeof(U) * count));
        allocs_.push_back(p);
        bytes_ += static_cast<int64_t>(sizeof(U) * count);
        return static_cast<U *>(p);
    }
    void dfree(void *p) {
        for (size_t i = 0; i < allocs_.size(); ++i)
            if (allocs_[i] == p) {
                cudaFree(p);
                allocs_.erase(allocs_.begin() + i);
                return;
            }
    }
    template <typename U>
    U *upload(const std::vector<U> &h) {
        U *d = dalloc<U>(h.size());
        if (!h.empty()) SCS_CUDA(cudaMemcpyAsync(d, h.data(), sizeof(U) * h.size(), cudaMemcpyHostToDevice, stream_));
        return d;
    }
    int grid_for(int64_t len) const {
        int64_t g = (len + kBlock - 1) / kBlock;
        const int64_t cap = static_cast<int64_t>(sms_) * 8;
        if (g > cap) g = cap;
        if (g < 1) g = 1;
        return static_cast<int>(g);
    }

    // ------------------------------------------------------------------ setup
    void setup(const HostProblem &P) {
        // sparse layouts
        // stored layouts of A and A^T; region grids for 8 CTAs per SM
        // one full wave per product: CTAs = SMs x the resident CTAs per SM of
        // the heaviest iteration epilogue that uses the layout
        auto occ = [](auto kern) {
            int n = 0;
            SCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kBlock, 0));
            return std::max(1, std::min(n, 8));
        };
        const int occ_a = std::min(occ(spmv_kernel<T, T, T, EpiAInit<T>>), occ(spmv_kernel<T, T, T, EpiACG<T>>));
        const int occ_at = std::min(occ(spmv_kernel<T, T, T, EpiAtInit<T>>), occ(spmv_kernel<T, T, T, EpiAtCG<T>>));
        // the layouts are planned on the host (row order, row starts,
        // regions, tiles); the plain CSR arrays are uploaded and their rows
        // gathered into stored order on the device
        SpmvLayout<double> LA = spmv_layout(P.a_rowptr, P.a_col, P.a_val, sms_ * occ_a, 0, false);
        SpmvLayout<double> LAt = spmv_layout(P.at_rowptr, P.at_col, P.at_val, sms_ * occ_at, 0, false);
        // CSR(A^T): the host copies, or views of the caller's canonical CSC
        const int32_t *at_cl = P.at_col_view ? P.at_col_view : P.at_col.data();
        const double *at_vl = P.at_val_view ? P.at_val_view : P.at_val.data();
        int32_t *a_rowptr = upload(LA.rowptr), *a_rowid = upload(LA.rowid);
        int32_t *at_rowptr = upload(LAt.rowptr), *at_rowid = upload(LAt.rowid);
        int32_t *a_col = dalloc<int32_t>(nnz_), *at_col = dalloc<int32_t>(nnz_);
        double *a_val64 = dalloc<double>(nnz_), *at_val64 = dalloc<double>(nnz_);
        auto gather = [&](const std::vector<int32_t> &rp, const int32_t *cl, const double *vl, const int32_t *rowid,
                          const int32_t *dst_rp, int rows, int32_t *dst_col, double *dst_val) {
            int32_t *srp = upload(rp), *scl = dalloc<int32_t>(nnz_);
            double *svl = dalloc<double>(nnz_);
            if (nnz_ > 0) {
                SCS_CUDA(cudaMemcpyAsync(scl, cl, sizeof(int32_t) * nnz_, cudaMemcpyHostToDevice, stream_));
                SCS_CUDA(cudaMemcpyAsync(svl, vl, sizeof(double) * nnz_, cudaMemcpyHostToDevice, stream_));
            }
            gather_rows_kernel<<<grid_for((int64_t)rows * 32), kBlock, 0, stream_>>>(rows, rowid, srp, scl, svl, dst_rp,
                                                                                   dst_col, dst_val);
            SCS_CUDA(cudaGetLastError());
            SCS_CUDA(cudaStreamSynchronize(stream_));
            dfree(srp);
            dfree(scl);
            dfree(svl);
        };
        gather(P.a_rowptr, P.a_col.data(), P.a_val.data(), a_rowid, a_rowptr, m_, a_col, a_val64);
        gather(P.at_rowptr, at_cl, at_vl, at_rowid, at_rowptr, n_, at_col, at_val64);
        const int32_t *a_tiles = upload(LA.tile_row), *at_tiles = upload(LAt.tile_row);
        S_ = dalloc<Scalars>(1);
        SCS_CUDA(cudaMemsetAsync(S_, 0, sizeof(Scalars), stream_));
        auto mkcsr = [&](auto *vals, const int32_t *rp, const int32_t *cl, const int32_t *rid,
                         const SpmvLayout<double> &lay, int rows) {
            using V = std::remove_cv_t<std::remove_pointer_t<decltype(vals)>>;
            const bool tiled = !lay.tile_row.empty();
            return Csr<V>{rp, cl, vals, rid, rows, lay.reg, tiled ? (&lay == &LA ? a_tiles : at_tiles) : nullptr,
                          tiled ? static_cast<int32_t>(lay.tile_row.size()) - 1 : 0};
        };
        SCS_CUDA(cudaStreamSynchronize(stream_));     // host layouts are released below

        // vectors
        u_ = dalloc<T>(N_);
        v_ = dalloc<T>(N_);
        b_ = upload(P.b);
        c_ = upload(P.c);
        D_ = dalloc<double>(m_);
        E_ = dalloc<double>(n_);
        p_ = dalloc<double>(n_ + m_);
        ax_ = dalloc<double>(m_);
        out_ = dalloc<double>(n_ + 2 * m_);
        z_ = dalloc<T>(n_);
        r_ = dalloc<T>(n_);
        pv_ = dalloc<T>(n_);
        diag_ = dalloc<T>(n_);
        q_ = dalloc<T>(m_);
        yacc_ = dalloc<T>(m_);
        az_ = dalloc<T>(m_);
        double *tmp_m = dalloc<double>(m_), *tmp_n = dalloc<double>(n_);
        double *red_out = dalloc<double>(4);
        red_out_ = red_out;

        fill(D_, m_, 1.0);
        fill(E_, n_, 1.0);

        // cone tables (row offsets within y)
        ConeDev K{};
        K.z = P.z;
        K.l = P.l;
        K.nq = static_cast<int>(P.q.size());
        K.ep = P.ep;
        std::vector<int32_t> qoff, avg_off, avg_len;
        int32_t off = P.z + P.l;
        for (int32_t qs : P.q) {
            qoff.push_back(off);
            avg_off.push_back(off);
            avg_len.push_back(qs);
            off += qs;
        }
        std::vector<int32_t> psd_off;
        std::vector<int64_t> psd_voff;
        int64_t vtot = 0;
        int psd_nmax = 0;
        for (int32_t ss : P.s) {     // PSD blocks: scaled as one block each
            avg_off.push_back(off);
            avg_len.push_back(ss * (ss + 1) / 2);
            psd_off.push_back(off);
            psd_voff.push_back(vtot);
            vtot += psd_mat_elems(ss);
            psd_nmax = std::max(psd_nmax, static_cast<int>(ss));
            off += ss * (ss + 1) / 2;
        }
        K.exp_off = off;
        K.ed = P.ed;
        K.np = static_cast<int>(P.pw.size());
        const int ntri = P.ep + P.ed + K.np;      // exponential, dual exponential, power: 3 rows each
        for (int e = 0; e < ntri; ++e) {
            avg_off.push_back(off + 3 * e);
            avg_len.push_back(3);
        }
        K.pow_a = K.np ? upload(P.pw) : nullptr;
        K.q_off = upload(qoff);
        K.q_len = upload(P.q);
        // element and SOC ranges: at most one wave of resident CTAs each
        int occ_p = 0;
        SCS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_p, relax_project_kernel<T>, kBlock, 0));
        const int64_t wave = static_cast<int64_t>(sms_) * std::max(1, occ_p);
        K.nb_elem = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(
            wave, (static_cast<int64_t>(n_) + K.z + K.l + kBlock - 1) / kBlock)));
        K.nb_soc = static_cast<int>(std::min<int64_t>(wave, (K.nq + kWarps - 1) / kWarps));
        K.nb_exp = (ntri + kExpPerCta - 1) / kExpPerCta;
        K.npsd = static_cast<int>(P.s.size());
        if (K.npsd) {
            // PSD blocks: eigenvector storage (warm start), per-block step
            // lengths, and global matrices when three do not fit on chip
            PsdDev<T> D{};
            D.npsd = K.npsd;
            D.ord = upload(P.s);
            D.off = upload(psd_off);
            D.voff = upload(psd_voff);
            D.V = dalloc<T>(vtot);
            D.dd = dalloc<double>(K.npsd);
            D.ne_max = psd_ne(psd_nmax);
            bool on_chip = false;
            psd_smem_ = psd_smem_bytes<T>(psd_nmax, on_chip);
            D.smem = on_chip ? 1 : 0;
            D.small_bytes = static_cast<int>(psd_small_bytes<T>(D.ne_max));
            D.fp64_cond = st_.psd_fp64_cond;
            if (!on_chip) {
                D.work_stride = psd_mat_elems(psd_nmax);
                D.work = dalloc<T>(static_cast<size_t>(K.npsd) * 2 * D.work_stride);
            }
            if (on_chip)
                SCS_CUDA(cudaFuncSetAttribute(psd_project_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                              static_cast<int>(psd_smem_)));
            else
                SCS_CUDA(cudaFuncSetAttribute(psd_project_kernel<T, false>,
                                              cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(psd_smem_)));
            SCS_CUDA(cudaMemsetAsync(D.dd, 0, sizeof(double) * K.npsd, stream_));
            K.psd_dd = D.dd;
            psd_ = D;
            psd_identity();
        }
        cone_ = K;
        const int32_t *d_avg_off = upload(avg_off), *d_avg_len = upload(avg_len);
        const int navg = static_cast<int>(avg_off.size());

        // partial sums of the grid reductions: one slot group per CTA of the
        // widest reducing launch (SpMV stream blocks, the projection grid, or
        // the capped grid-stride kernels)
        rb_cap_ = std::max({mkcsr(a_val64, a_rowptr, a_col, a_rowid, LA, m_).grid(),
                            mkcsr(at_val64, at_rowptr, at_col, at_rowid, LAt, n_).grid(), sms_ * 8, proj_grid(), 1});
        rb_.partials = dalloc<double>(static_cast<size_t>(rb_cap_) * kMaxRed);
        rb_.cap = rb_cap_;
        rb_.counter = dalloc<unsigned>(kSiteCount);
        SCS_CUDA(cudaMemsetAsync(rb_.counter, 0, sizeof(unsigned) * kSiteCount, stream_));

        // ---- equilibration, Sec. 5 (FP64) ----
        if (st_.normalize) {
            for (int pass = 0; pass < st_.scale_passes; ++pass) {
                row_sumsq_kernel<<<grid_for((int64_t)m_ * 32), kBlock, 0, stream_>>>(a_rowptr, a_val64, a_rowid, m_, tmp_m);
                row_sumsq_kernel<<<grid_for((int64_t)n_ * 32), kBlock, 0, stream_>>>(at_rowptr, at_val64, at_rowid, n_, tmp_n);
                sqrt_kernel<<<grid_for(m_), kBlock, 0, stream_>>>(tmp_m, m_);
                sqrt_kernel<<<grid_for(n_), kBlock, 0, stream_>>>(tmp_n, n_);
                if (navg)
                    block_mean_kernel<<<grid_for((int64_t)navg * 32), kBlock, 0, stream_>>>(tmp_m, d_avg_off,
                                                                                            d_avg_len, navg,
                                                                                            st_.block_scale);
                inv_sqrt_clamp_kernel<<<grid_for(m_), kBlock, 0, stream_>>>(tmp_m, m_, 1e-4, 1e4, tmp_m, D_);
                inv_sqrt_clamp_kernel<<<grid_for(n_), kBlock, 0, stream_>>>(tmp_n, n_, 1e-4, 1e4, tmp_n, E_);
                scale_vals_kernel<<<grid_for((int64_t)m_ * 32), kBlock, 0, stream_>>>(a_rowptr, a_col, a_val64, a_rowid,
                                                                                      m_, tmp_m, tmp_n);
                scale_vals_kernel<<<grid_for((int64_t)n_ * 32), kBlock, 0, stream_>>>(at_rowptr, at_col, at_val64,
                                                                                      at_rowid, n_, tmp_n, tmp_m);
                SCS_CUDA(cudaGetLastError());
            }
            // sigma = 1 / max(||D b||, 1e-4); rho = mean_i ||row_i(A^)|| / max(||E c||, 1e-4)
            row_sumsq_kernel<<<grid_for((int64_t)m_ * 32), kBlock, 0, stream_>>>(a_rowptr, a_val64, a_rowid, m_, tmp_m);
            sqrt_kernel<<<grid_for(m_), kBlock, 0, stream_>>>(tmp_m, m_);
            const double *Db = D_, *bb = b_, *Ec = E_, *cc = c_, *tm = tmp_m;
            reduce_kernel<<<grid_for(m_), kBlock, 0, stream_>>>(
                [=] __device__(int i) { return tm[i]; }, m_, rb_, red_out + 0);
            reduce_kernel<<<grid_for(m_), kBlock, 0, stream_>>>(
                [=] __device__(int i) { const double t = Db[i] * bb[i]; return t * t; }, m_, rb_, red_out + 1);
            reduce_kernel<<<grid_for(n_), kBlock, 0, stream_>>>(
                [=] __device__(int i) { const double t = Ec[i] * cc[i]; return t * t; }, n_, rb_, red_out + 2);
            double h[3];
            SCS_CUDA(cudaMemcpyAsync(h, red_out, sizeof(h), cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaStreamSynchronize(stream_));
            double mean_row = m_ ? h[0] / m_ : 1.0;
            if (!(mean_row > 0.0)) mean_row = 1.0;
            mean_row_ = mean_row;
            sigma_ = 1.0 / std::max(std::sqrt(h[1]), 1e-4);
            rho_ = mean_row / std::max(std::sqrt(h[2]), 1e-4);
        } else {
            sigma_ = 1.0;
            rho_ = 1.0;
        }
        {
            double *bd = b_, *cd = c_;
            const double *Dd = D_, *Ed = E_;
            const double sg = sigma_, rh = rho_;
            foreach_kernel<<<grid_for(m_), kBlock, 0, stream_>>>([=] __device__(int i) { bd[i] *= sg * Dd[i]; }, m_);
            foreach_kernel<<<grid_for(n_), kBlock, 0, stream_>>>([=] __device__(int j) { cd[j] *= rh * Ed[j]; }, n_);
        }
        // working copies of b^, c^ in the iteration's precision
        if (std::is_same<T, double>::value) {
            bT_ = reinterpret_cast<T *>(b_);
            cT_ = reinterpret_cast<T *>(c_);
        } else {
            bT_ = dalloc<T>(m_);
            cT_ = dalloc<T>(n_);
            T *bt = bT_, *ct = cT_;
            const double *bd = b_, *cd = c_;
            foreach_kernel<<<grid_for(m_), kBlock, 0, stream_>>>([=] __device__(int i) { bt[i] = static_cast<T>(bd[i]); }, m_);
            foreach_kernel<<<grid_for(n_), kBlock, 0, stream_>>>([=] __device__(int j) { ct[j] = static_cast<T>(cd[j]); }, n_);
        }
        // Jacobi preconditioner diag(I + A^T A) = 1 + ||col_j(A^)||^2
        row_sumsq_kernel<<<grid_for((int64_t)n_ * 32), kBlock, 0, stream_>>>(at_rowptr, at_val64, at_rowid, n_, tmp_n);
        {
            T *dg = diag_;
            const double *tn = tmp_n;
            foreach_kernel<<<grid_for(n_), kBlock, 0, stream_>>>(
                [=] __device__(int j) { dg[j] = static_cast<T>(1.0 + tn[j]); }, n_);
        }
        // values in the iteration's precision
        const T *a_val, *at_val;
        if (std::is_same<T, double>::value) {
            a_val = reinterpret_cast<const T *>(a_val64);
            at_val = reinterpret_cast<const T *>(at_val64);
        } else {
            T *av = dalloc<T>(nnz_), *atv = dalloc<T>(nnz_);
            const double *a64 = a_val64, *at64 = at_val64;
            foreach_kernel<<<grid_for(nnz_), kBlock, 0, stream_>>>(
                [=] __device__(int k) { av[k] = static_cast<T>(a64[k]); atv[k] = static_cast<T>(at64[k]); },
                (int)nnz_);
            a_val = av;
            at_val = atv;
        }
        A_ = mkcsr(a_val, a_rowptr, a_col, a_rowid, LA, m_);
        At_ = mkcsr(at_val, at_rowptr, at_col, at_rowid, LAt, n_);
        SCS_CUDA(cudaGetLastError());
        SCS_CUDA(cudaStreamSynchronize(stream_));
        // FP64 values (the same arrays in the FP64 engine) for the termination tests
        A64_ = mkcsr(a_val64, a_rowptr, a_col, a_rowid, LA, m_);
        At64_ = mkcsr(at_val64, at_rowptr, at_col, at_rowid, LAt, n_);
        if (st_.linsys == 1) setup_direct(a_rowptr, a_col, a_val64, a_rowid);

        // reciprocals of the scaling for the termination tests (the FP64
        // divide is slow on this part; the tests run every 20 iterations)
        Dinv_ = dalloc<double>(m_);
        Einv_ = dalloc<double>(n_);
        {
            double *di = Dinv_, *ei = Einv_;
            const double *Dd = D_, *Ed = E_;
            foreach_kernel<<<grid_for(m_), kBlock, 0, stream_>>>([=] __device__(int i) { di[i] = 1.0 / Dd[i]; }, m_);
            foreach_kernel<<<grid_for(n_), kBlock, 0, stream_>>>([=] __device__(int j) { ei[j] = 1.0 / Ed[j]; }, n_);
        }
        // host copies of the scaling (warm start, scs_get_scaling)
        Dh_.resize(m_);
        Eh_.resize(n_);
        SCS_CUDA(cudaMemcpy(Dh_.data(), D_, sizeof(double) * m_, cudaMemcpyDeviceToHost));
        SCS_CUDA(cudaMemcpy(Eh_.data(), E_, sizeof(double) * n_, cudaMemcpyDeviceToHost));

        // scalars
        Scalars sh{};
        sh.relax = st_.alpha;
        sh.eps_pri = st_.eps_pri;
        sh.eps_dual = st_.eps_dual;
        sh.eps_gap = st_.eps_gap;
        sh.eps_infeas = st_.eps_infeas;
        sh.eps_unbdd = st_.eps_unbdd;
        double nb = 0, nc = 0;
        for (double t : P.b) nb += t * t;
        for (double t : P.c) nc += t * t;
        sh.nb = std::sqrt(nb);
        sh.nc = std::sqrt(nc);
        sh.sigma = sigma_;
        sh.rho = rho_;
        sh.hp1 = 1.0;
        sh.cg_rate = st_.cg_rate;
        sh.cg_adapt = st_.cg_adapt;
        sh.cg_tol_rel = st_.cg_tol_rel;
        sh.cg_max = st_.cg_max_iters;
        SCS_CUDA(cudaMemcpy(S_, &sh, sizeof(Scalars), cudaMemcpyHostToDevice));
        compute_p();
        dfree(tmp_m);
        dfree(tmp_n);
        set_initial_point();
        if (st_.use_graph) build_graph();
        SCS_CUDA(cudaStreamSynchronize(stream_));
    }

    // Direct method (Sec. 4.1 with the factorization cached, Sec. 4.2): dense
    // A^ and A^T from the scaled FP64 CSR (stored rows in length-class order,
    // rowid maps them back), G = I + A^T A by the FP64 GEMM, G^-1 in place by
    // FP64 Gauss-Jordan, then kept in the iteration's precision.
    void setup_direct(const int32_t *rp, const int32_t *col, const double *val, const int32_t *rowid) {
        if (n_ > kDirectMaxN || (int64_t)m_ * n_ > ((int64_t)1 << 30))
            throw CudaError("linsys 1 (direct): needs n <= 8192 and m n <= 2^30", SCS_UNSUPPORTED);
        const int m = m_, n = n_;
        const size_t mn = (size_t)m * n, nn = (size_t)n * n;
        double *Ad = dalloc<double>(mn), *Atd = dalloc<double>(mn), *G = dalloc<double>(nn);
        double *colk = dalloc<double>(2 * (size_t)n);
        SCS_CUDA(cudaMemsetAsync(Ad, 0, sizeof(double) * mn, stream_));
        SCS_CUDA(cudaMemsetAsync(Atd, 0, sizeof(double) * mn, stream_));
        foreach_kernel<<<grid_for(m), kBlock, 0, stream_>>>(
            [=] __device__(int r) {
                const int i = rowid[r];
                for (int k = rp[r]; k < rp[r + 1]; ++k) {
                    Ad[(size_t)col[k] * m + i] = val[k];
                    Atd[(size_t)i * n + col[k]] = val[k];
                }
            },
            m);
        foreach_kernel<<<grid_for((int64_t)nn), kBlock, 0, stream_>>>(
            [=] __device__(int64_t e) { G[e] = (e % (n + 1) == 0) ? 1.0 : 0.0; }, (int64_t)nn);
        SCS_CUDA(dense::gemm_nn<double>(stream_, n, n, m, 1.0, Atd, n, Ad, m, 1.0, G, n));   // I + A^T A
        SCS_CUDA(dense::invert_spd_gj<double>(stream_, G, n, colk, grid_for((int64_t)nn)));
        if (std::is_same<T, double>::value) {
            Minv_ = reinterpret_cast<T *>(G);
        } else {
            Minv_ = dalloc<T>(nn);
            T *mi = Minv_;
            foreach_kernel<<<grid_for((int64_t)nn), kBlock, 0, stream_>>>(
                [=] __device__(int64_t e) { mi[e] = static_cast<T>(G[e]); }, (int64_t)nn);
        }
        SCS_CUDA(cudaGetLastError());
        SCS_CUDA(cudaStreamSynchronize(stream_));
        dfree(Ad);
        dfree(Atd);
        dfree(colk);
        if (!std::is_same<T, double>::value) dfree(G);
        direct_ = true;
    }

    // New b, c with the same A (Sec. 4.2): D, E, the layouts and a cached
    // (I + A^T A)^-1 depend on A only and are kept; sigma, rho, b^, c^,
    // p = M^-1 h and 1 + h^T p are recomputed, and the next solve starts cold.
    int update_bc(const double *b, const double *c) override {
        SCS_CUDA(cudaSetDevice(device_));
        double nb = 0.0, nc = 0.0;
        for (int i = 0; i < m_; ++i) nb += b[i] * b[i];
        for (int j = 0; j < n_; ++j) nc += c[j] * c[j];
        SCS_CUDA(cudaMemcpyAsync(b_, b, sizeof(double) * m_, cudaMemcpyHostToDevice, stream_));
        SCS_CUDA(cudaMemcpyAsync(c_, c, sizeof(double) * n_, cudaMemcpyHostToDevice, stream_));
        if (st_.normalize) {
            const double *Db = D_, *bb = b_, *Ec = E_, *cc = c_;
            reduce_kernel<<<grid_for(m_), kBlock, 0, stream_>>>(
                [=] __device__(int i) { const double t = Db[i] * bb[i]; return t * t; }, m_, rb_, red_out_ + 1);
            reduce_kernel<<<grid_for(n_), kBlock, 0, stream_>>>(
                [=] __device__(int i) { const double t = Ec[i] * cc[i]; return t * t; }, n_, rb_, red_out_ + 2);
            double h[2];
            SCS_CUDA(cudaMemcpyAsync(h, red_out_ + 1, sizeof(h), cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaStreamSynchronize(stream_));
            sigma_ = 1.0 / std::max(std::sqrt(h[0]), 1e-4);
            rho_ = mean_row_ / std::max(std::sqrt(h[1]), 1e-4);
        }
        {
            double *bd = b_, *cd = c_;
            const double *Dd = D_, *Ed = E_;
            const double sg = sigma_, rh = rho_;
            foreach_kernel<<<grid_for(m_), kBlock, 0, stream_>>>([=] __device__(int i) { bd[i] *= sg * Dd[i]; }, m_);
            foreach_kernel<<<grid_for(n_), kBlock, 0, stream_>>>([=] __device__(int j) { cd[j] *= rh * Ed[j]; }, n_);
            if (!std::is_same<T, double>::value) {
                T *bt = bT_, *ct = cT_;
                foreach_kernel<<<grid_for(m_), kBlock, 0, stream_>>>(
                    [=] __device__(int i) { bt[i] = static_cast<T>(bd[i]); }, m_);
                foreach_kernel<<<grid_for(n_), kBlock, 0, stream_>>>(
                    [=] __device__(int j) { ct[j] = static_cast<T>(cd[j]); }, n_);
            }
        }
        Scalars sh{};
        SCS_CUDA(cudaMemcpyAsync(&sh, S_, sizeof(Scalars), cudaMemcpyDeviceToHost, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        sh.sigma = sigma_;
        sh.rho = rho_;
        sh.nb = std::sqrt(nb);
        sh.nc = std::sqrt(nc);
        SCS_CUDA(cudaMemcpy(S_, &sh, sizeof(Scalars), cudaMemcpyHostToDevice));
        compute_p();
        set_initial_point();
        warm_pending_ = false;
        SCS_CUDA(cudaStreamSynchronize(stream_));
        return 0;
    }

    // cached p = M^-1 h (Sec. 4.1), h = (c^, b^), solved tightly: CG from
    // zero with the right-hand side r = h, i.e. u = (c^, b^, 0), v = 0; then
    // 1 + h^T p.  The device scalars keep every other field.
    void compute_p() {
        double *red_out = red_out_;
        Scalars sh{};
        SCS_CUDA(cudaMemcpy(&sh, S_, sizeof(Scalars), cudaMemcpyDeviceToHost));
        const Scalars keep = sh;
        sh.cg_rate = 0.0;
        sh.cg_adapt = 0.0;
        sh.dstep = INFINITY;
        sh.cg_tol_rel = std::is_same<T, double>::value ? 1e-14 : 1e-7;
        sh.cg_max = std::max(10 * st_.cg_max_iters, 500);
        sh.k = 0;          // K1 takes the product A z (z restarts from 0 here)
        SCS_CUDA(cudaMemcpyAsync(S_, &sh, sizeof(Scalars), cudaMemcpyHostToDevice, stream_));
        SCS_CUDA(cudaMemsetAsync(u_, 0, sizeof(T) * N_, stream_));
        SCS_CUDA(cudaMemsetAsync(v_, 0, sizeof(T) * N_, stream_));
        SCS_CUDA(cudaMemcpyAsync(u_, cT_, sizeof(T) * n_, cudaMemcpyDeviceToDevice, stream_));
        SCS_CUDA(cudaMemcpyAsync(u_ + n_, bT_, sizeof(T) * m_, cudaMemcpyDeviceToDevice, stream_));
        SCS_CUDA(cudaMemsetAsync(z_, 0, sizeof(T) * n_, stream_));
        launch_K1();
        launch_K2(CondHandle{0, 0});
        for (int c = 0; c < sh.cg_max; c += 16) {
            for (int j = 0; j < 16; ++j) {
                launch_K3();
                launch_K4();
                launch_K5(CondHandle{0, 0});
            }
            SCS_CUDA(cudaMemcpyAsync(Sh_, S_, sizeof(Scalars), cudaMemcpyDeviceToHost, stream_));
            SCS_CUDA(cudaStreamSynchronize(stream_));
            if (!Sh_->active) break;
        }
        {
            double *pd = p_;
            const T *zz = z_, *ya = yacc_;
            const int n = n_;
            foreach_kernel<<<grid_for(n_ + m_), kBlock, 0, stream_>>>(
                [=] __device__(int i) { pd[i] = i < n ? static_cast<double>(zz[i]) : static_cast<double>(ya[i - n]); },
                n_ + m_);
            const double *cc = c_, *bb = b_;
            reduce_kernel<<<grid_for(n_ + m_), kBlock, 0, stream_>>>(
                [=] __device__(int i) { return (i < n ? cc[i] : bb[i - n]) * pd[i]; }, n_ + m_, rb_, red_out + 3);
            if (std::is_same<T, double>::value) {
                pT_ = reinterpret_cast<T *>(p_);
            } else {
                if (!pT_) pT_ = dalloc<T>(n_ + m_);
                T *pt = pT_;
                foreach_kernel<<<grid_for(n_ + m_), kBlock, 0, stream_>>>(
                    [=] __device__(int i) { pt[i] = static_cast<T>(pd[i]); }, n_ + m_);
            }
        }
        double hp;
        SCS_CUDA(cudaMemcpyAsync(&hp, red_out + 3, sizeof(double), cudaMemcpyDeviceToHost, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
        Scalars out = keep;
        out.hp1 = 1.0 + hp;
        SCS_CUDA(cudaMemcpy(S_, &out, sizeof(Scalars), cudaMemcpyHostToDevice));
    }

    // eigenvectors of every PSD block back to I (cold Jacobi start)
    void psd_identity() {
        if (!psd_.npsd) return;
        psd_identity_kernel<T><<<std::min(psd_.npsd, sms_ * 4), kBlock, 0, stream_>>>(psd_.V, psd_.ord, psd_.voff,
                                                                                   psd_.npsd);
        SCS_CUDA(cudaGetLastError());
    }

    void fill(double *d, int len, double val) {
        foreach_kernel<<<grid_for(len), kBlock, 0, stream_>>>([=] __device__(int i) { d[i] = val; }, len);
    }

    void reset_counters(double dstep = INFINITY) {
        // k = 0, cg_total = 0, status = 0, last step length (fields of the device scalars)
        const int zero = 0;
        const int64_t zero64 = 0;
        SCS_CUDA(cudaMemcpyAsync(&S_->dstep, &dstep, sizeof(double), cudaMemcpyHostToDevice, stream_));
        SCS_CUDA(cudaMemcpyAsync(&S_->k, &zero, sizeof(int), cudaMemcpyHostToDevice, stream_));
        SCS_CUDA(cudaMemcpyAsync(&S_->status, &zero, sizeof(int), cudaMemcpyHostToDevice, stream_));
        SCS_CUDA(cudaMemcpyAsync(&S_->cg_total, &zero64, sizeof(int64_t), cudaMemcpyHostToDevice, stream_));
        SCS_CUDA(cudaStreamSynchronize(stream_));
    }

    // Sec. 3.4: u0 = (0, 0, 1), v0 = (0, 0, 1); CG warm start from zero
    void set_initial_point() {
        psd_identity();
        SCS_CUDA(cudaMemsetAsync(u_, 0, sizeof(T) * N_, stream_));
        SCS_CUDA(cudaMemsetAsync(v_, 0, sizeof(T) * N_, stream_));
        SCS_CUDA(cudaMemsetAsync(z_, 0, sizeof(T) * n_, stream_));
        T *uu = u_, *vv = v_;
        const int N = N_;
        foreach_kernel<<<1, 32, 0, stream_>>>([=] __device__(int) { uu[N - 1] = T(1); vv[N - 1] = T(1); }, 1);
        SCS_CUDA(cudaGetLastError());
        reset_counters();
    }

    int inaccurate_status() const {
        const Scalars &s = *Sh_;
        if (!std::isfinite(s.tau) || !std::isfinite(s.kappa)) return SCS_NUMERICAL;
        if (s.tau > 0 && s.tau >= s.kappa) return SCS_SOLVED_INACCURATE;
        if (s.bty < 0 && s.bty <= s.ctx) return SCS_INFEASIBLE_INACCURATE;
        if (s.ctx < 0) return SCS_UNBOUNDED_INACCURATE;
        return s.tau > 0 ? SCS_SOLVED_INACCURATE : SCS_INFEASIBLE_INACCURATE;
    }

    // ------------------------------------------------------------ launches
    int proj_grid() const { return cone_.nb_elem + cone_.nb_soc + cone_.nb_exp; }
    // every reducing launch must fit the partial-sum buffer
    void guard(int grid) const {
        if (grid > rb_cap_ || grid < 1) throw CudaError("reduction grid exceeds its buffer", SCS_DEVICE_ERROR);
    }

    // K1 (the product, every kAzEvery-th iteration) and K1' (from the carried
    // A z): both are launched, the one whose iteration it is not returns at once
    void launch_K1() {
        guard(A_.grid());
        EpiAInit<T> e{u_, v_, bT_, yacc_, az_, S_, n_, N_, 0.0};
        spmv_kernel<T, T, T, EpiAInit<T>><<<A_.grid(), kBlock, 0, cur_>>>(A_, z_, e, rb_);
        yacc_init_kernel<T><<<grid_for(m_), kBlock, 0, cur_>>>(n_, m_, N_, u_, v_, bT_, az_, yacc_, S_, rb_);
    }
    void launch_K2(CondHandle h) {
        guard(At_.grid());
        EpiAtInit<T> e{u_, v_, cT_, diag_, z_, r_, pv_, S_, h, N_, 0.0};
        spmv_kernel<T, T, T, EpiAtInit<T>><<<At_.grid(), kBlock, 0, cur_>>>(At_, yacc_, e, rb_);
    }
    void launch_K3() {
        guard(A_.grid());
        EpiACG<T> e{q_, S_};
        spmv_kernel<T, T, T, EpiACG<T>><<<A_.grid(), kBlock, 0, cur_>>>(A_, pv_, e, rb_);
    }
    void launch_K4() {
        guard(At_.grid());
        EpiAtCG<T> e{diag_, z_, r_, pv_, S_, T(0), q_, yacc_, az_, m_};
        spmv_kernel<T, T, T, EpiAtCG<T>><<<At_.grid(), kBlock, 0, cur_>>>(At_, q_, e, rb_);
    }
    void launch_K5(CondHandle h) {
        cg_update_kernel<T><<<grid_for(n_), kBlock, 0, cur_>>>(n_, m_, q_, yacc_, az_, r_, diag_, pv_, S_, h, rb_);
    }
    void launch_D1() {
        direct_gemv_kernel<T><<<grid_for((int64_t)n_ * 32), kBlock, 0, cur_>>>(n_, Minv_, r_, z_, pv_);
    }
    void launch_D2() {
        guard(A_.grid());
        EpiADirect<T> e{q_, yacc_, az_, S_};
        spmv_kernel<T, T, T, EpiADirect<T>><<<A_.grid(), kBlock, 0, cur_>>>(A_, pv_, e, rb_);
    }
    void launch_K6() {
        smw_kernel<T><<<grid_for(n_ + m_), kBlock, 0, cur_>>>(n_, m_, cT_, bT_, z_, yacc_, S_, rb_);
    }
    void launch_KP() {
        if (!psd_.npsd) return;
        ProjArgs<T> a{n_, m_, N_, u_, v_, pT_, z_, yacc_, S_};
        PsdStats st{&S_->psd_sweeps, &S_->psd_fp64, &S_->psd_calls};
        if (psd_.smem)
            psd_project_kernel<T, true><<<psd_.npsd, kPsdThreads, psd_smem_, cur_>>>(a, psd_, st);
        else
            psd_project_kernel<T, false><<<psd_.npsd, kPsdThreads, psd_smem_, cur_>>>(a, psd_, st);
    }
    void launch_K7() {
        ProjArgs<T> a{n_, m_, N_, u_, v_, pT_, z_, yacc_, S_};
        const int grid = proj_grid();
        guard(grid);
        relax_project_kernel<T><<<grid, kBlock, 0, cur_>>>(a, cone_, rb_);
    }
    void launch_check() {
        guard(A64_.grid());
        guard(At64_.grid());
        EpiChkA<T> ea{u_, v_, b_, Dinv_, ax_, S_, n_, N_, 0.0};
        spmv_kernel<double, T, double, EpiChkA<T>><<<A64_.grid(), kBlock, 0, stream_>>>(A64_, u_, ea, rb_);
        EpiChkAt<T> eb{u_, v_, c_, Einv_, S_, N_, 0.0};
        spmv_kernel<double, T, double, EpiChkAt<T>><<<At64_.grid(), kBlock, 0, stream_>>>(At64_, u_ + n_, eb,
                                                                                                  rb_);
        SCS_CUDA(cudaGetLastError());
    }

    template <typename F>
    void timed(int kind, F f) {
        SCS_CUDA(cudaEventRecord(ev_[0], stream_));
        f();
        SCS_CUDA(cudaEventRecord(ev_[1], stream_));
        SCS_CUDA(cudaEventSynchronize(ev_[1]));
        float ms = 0.f;
        SCS_CUDA(cudaEventElapsedTime(&ms, ev_[0], ev_[1]));
        prof_ms_[kind] += ms;
        prof_n_[kind] += 1;
    }

    // one ADMM iteration without a graph: the CG steps beyond convergence
    // return at once (they read the device flag S->active)
    void launch_iteration_plain() {
        launch_K1();
        launch_K2(CondHandle{0, 0});
        if (direct_) {
            launch_D1();
            launch_D2();
            launch_K6();
            launch_KP();
            launch_K7();
            return;
        }
        for (int c = 0; c < st_.cg_max_iters; ++c) {
            launch_K3();
            launch_K4();
            launch_K5(CondHandle{0, 0});
        }
        launch_K6();
        launch_KP();
        launch_K7();
    }

    void run_iters(int iters) {
        for (int it = 0; it < iters; ++it) {
            if (exec_) {
                SCS_CUDA(cudaGraphLaunch(exec_, stream_));
            } else {
                launch_iteration_plain();
            }
        }
        SCS_CUDA(cudaGetLastError());
    }

    // Graph of one iteration: K1 -> K2 -> WHILE(active){K3 -> K4 -> K5} -> K6 -> K7.
    void build_graph() {
        if (direct_) {      // K1 -> K2 -> KD1 -> KD2 -> K6 -> KP -> K7: no CG loop
            SCS_CUDA(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
            cur_ = stream_;
            launch_K1();
            launch_K2(CondHandle{0, 0});
            launch_D1();
            launch_D2();
            launch_K6();
            launch_KP();
            launch_K7();
            SCS_CUDA(cudaStreamEndCapture(stream_, &graph_));
            SCS_CUDA(cudaGraphInstantiate(&exec_, graph_, 0));
            return;
        }
        SCS_CUDA(cudaGraphCreate(&graph_, 0));
        cudaGraphConditionalHandle h;
        SCS_CUDA(cudaGraphConditionalHandleCreate(&h, graph_, 1, cudaGraphCondAssignDefault));
        CondHandle ch{h, 1};
        SCS_CUDA(cudaStreamBeginCaptureToGraph(stream_, graph_, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        cur_ = stream_;
        launch_K1();
        launch_K2(ch);
        cudaStreamCaptureStatus cs;
        const cudaGraphNode_t *deps = nullptr;
        size_t ndeps = 0;
        cudaGraph_t cap_graph;
        SCS_CUDA(cudaStreamGetCaptureInfo(stream_, &cs, nullptr, &cap_graph, &deps, nullptr, &ndeps));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode;
        SCS_CUDA(cudaGraphAddNode(&cnode, cap_graph, deps, nullptr, ndeps, &cp));
        cudaGraph_t body = cp.conditional.phGraph_out[0];
        SCS_CUDA(cudaStreamUpdateCaptureDependencies(stream_, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
        SCS_CUDA(cudaStreamBeginCaptureToGraph(body_stream_, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
        cur_ = body_stream_;
        launch_K3();
        launch_K4();
        launch_K5(ch);
        cudaGraph_t body_out;
        SCS_CUDA(cudaStreamEndCapture(body_stream_, &body_out));
        cur_ = stream_;
        launch_K6();
        launch_KP();
        launch_K7();
        cudaGraph_t done_graph;
        SCS_CUDA(cudaStreamEndCapture(stream_, &done_graph));
        SCS_CUDA(cudaGraphInstantiate(&exec_, graph_, 0));
        cur_ = stream_;
    }

    // ------------------------------------------------------------------ state
    scs_settings st_;
    int device_ = 0, sms_ = 1;
    int m_ = 0, n_ = 0, N_ = 0;
    int64_t nnz_ = 0, bytes_ = 0;
    cudaStream_t stream_ = nullptr, body_stream_ = nullptr, cur_ = nullptr;
    bool own_stream_ = false, warm_pending_ = false;
    std::vector<void *> allocs_;
    Csr<T> A_{}, At_{};
    Csr<double> A64_{}, At64_{};
    ConeDev cone_{};
    ReduceBuf rb_{};
    int rb_cap_ = 0;
    Scalars *S_ = nullptr, *Sh_ = nullptr;
    T *u_ = nullptr, *v_ = nullptr, *bT_ = nullptr, *cT_ = nullptr, *pT_ = nullptr;
    double *b_ = nullptr, *c_ = nullptr, *D_ = nullptr, *E_ = nullptr;
    double *p_ = nullptr, *ax_ = nullptr, *out_ = nullptr;
    double *Dinv_ = nullptr, *Einv_ = nullptr;   // 1 / D, 1 / E for the termination tests
    T *z_ = nullptr, *r_ = nullptr, *pv_ = nullptr, *diag_ = nullptr, *q_ = nullptr, *yacc_ = nullptr;
    T *az_ = nullptr;      // A^ z_x carried between iterations (kernels.cuh, K1')
    std::vector<double> Dh_, Eh_;
    double sigma_ = 1.0, rho_ = 1.0;
    cudaGraph_t graph_ = nullptr;
    cudaGraphExec_t exec_ = nullptr;
    std::vector<cudaEvent_t> ev_;
    double prof_ms_[5] = {0, 0, 0, 0, 0};
    int64_t prof_n_[5] = {0, 0, 0, 0, 0};
    // direct subspace step (linsys 1): (I + A^T A)^-1, n x n, in T
    bool direct_ = false;
    T *Minv_ = nullptr;
    double *red_out_ = nullptr;   // device scratch of the setup reductions
    double mean_row_ = 1.0;       // mean row norm of A^ (rho's numerator, Sec. 5)
    PsdDev<T> psd_{};
    size_t psd_smem_ = 0;
};

}  // namespace scs
