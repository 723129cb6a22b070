// C ABI of the solver (include/scs_gpu.h): input validation, the host-side
// CSC -> CSR layouts of A and A^T, and dispatch to the FP64 or mixed
// FP32/FP64 device engine.  No C++ exception crosses this boundary.
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/scs_gpu.h"
#include <algorithm>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "engine_base.h"
#include "psd.cuh"

struct scs_work {
    scs::EngineBase *eng = nullptr;
    int device = 0;
};

namespace {

thread_local std::string g_last_error;

void set_error(const std::string &s) { g_last_error = s; }

}  // namespace

void scs::set_last_error(const std::string &s) { set_error(s); }

int scs::validate_and_build(const scs_csc *A, const double *b, const double *c, const scs_cone *k,
                            scs::HostProblem &P) {
    if (!A || !b || !c || !k) { set_error("null argument"); return SCS_INVALID_INPUT; }
    if (A->m <= 0 || A->n <= 0) { set_error("m and n must be positive"); return SCS_INVALID_INPUT; }
    if (!A->colptr || (!A->rowidx && A->colptr[A->n] > 0) || (!A->val && A->colptr[A->n] > 0)) {
        set_error("null CSC array");
        return SCS_INVALID_INPUT;
    }
    const int32_t m = A->m, n = A->n;
    if (A->colptr[0] != 0) { set_error("colptr[0] must be 0"); return SCS_INVALID_INPUT; }
    for (int32_t j = 0; j < n; ++j)
        if (A->colptr[j + 1] < A->colptr[j]) { set_error("colptr must be nondecreasing"); return SCS_INVALID_INPUT; }
    const int64_t nnz_in = A->colptr[n];
    if (nnz_in >= (int64_t)1 << 31) { set_error("nnz must be below 2^31"); return SCS_UNSUPPORTED; }
    for (int64_t t = 0; t < nnz_in; ++t) {
        if (A->rowidx[t] < 0 || A->rowidx[t] >= m) { set_error("row index out of range"); return SCS_INVALID_INPUT; }
        if (!std::isfinite(A->val[t])) { set_error("non-finite entry in A"); return SCS_INVALID_INPUT; }
    }
    for (int32_t i = 0; i < m; ++i)
        if (!std::isfinite(b[i])) { set_error("non-finite entry in b"); return SCS_INVALID_INPUT; }
    for (int32_t j = 0; j < n; ++j)
        if (!std::isfinite(c[j])) { set_error("non-finite entry in c"); return SCS_INVALID_INPUT; }
    // cone
    if (k->z < 0 || k->l < 0 || k->nq < 0 || k->ns < 0 || k->ep < 0 || k->ed < 0 || k->np < 0) {
        set_error("negative cone size");
        return SCS_INVALID_INPUT;
    }
    if ((k->nq > 0 && !k->q) || (k->ns > 0 && !k->s) || (k->np > 0 && !k->p)) { set_error("null cone array"); return SCS_INVALID_INPUT; }
    for (int32_t i = 0; i < k->np; ++i)
        if (!(std::fabs(k->p[i]) > 0.0 && std::fabs(k->p[i]) < 1.0)) {
            set_error("power cone parameter must lie in (-1, 0) or (0, 1)");
            return SCS_INVALID_INPUT;
        }
    int64_t rows = (int64_t)k->z + k->l + 3 * ((int64_t)k->ep + k->ed + k->np);
    for (int32_t i = 0; i < k->nq; ++i) {
        if (k->q[i] < 1) { set_error("SOC size must be >= 1"); return SCS_INVALID_INPUT; }
        rows += k->q[i];
    }
    for (int32_t i = 0; i < k->ns; ++i) {
        if (k->s[i] < 1) { set_error("PSD order must be >= 1"); return SCS_INVALID_INPUT; }
        if (k->s[i] > scs::kPsdMaxOrder) { set_error("PSD order above 1024"); return SCS_UNSUPPORTED; }
        rows += (int64_t)k->s[i] * (k->s[i] + 1) / 2;
    }
    if (rows != m) { set_error("cone sizes do not add up to m"); return SCS_INVALID_INPUT; }

    // CSR of A (counting sort by row; columns visited in order keep each row
    // sorted by column, so duplicates are adjacent and are summed)
    P.m = m;
    P.n = n;
    std::vector<int32_t> cnt(m + 1, 0);
    for (int64_t t = 0; t < nnz_in; ++t) cnt[A->rowidx[t] + 1]++;
    std::vector<int32_t> rp(m + 1, 0);
    for (int32_t i = 0; i < m; ++i) rp[i + 1] = rp[i] + cnt[i + 1];
    std::vector<int32_t> col(nnz_in), pos(rp.begin(), rp.end() - 1);
    std::vector<double> val(nnz_in);
    for (int32_t j = 0; j < n; ++j)
        for (int64_t t = A->colptr[j]; t < A->colptr[j + 1]; ++t) {
            const int32_t i = A->rowidx[t];
            col[pos[i]] = j;
            val[pos[i]] = A->val[t];
            pos[i]++;
        }
    P.a_rowptr.assign(m + 1, 0);
    P.a_col.reserve(nnz_in);
    P.a_val.reserve(nnz_in);
    for (int32_t i = 0; i < m; ++i) {
        // within a row, sort by column (entries of one column may come unsorted)
        std::vector<std::pair<int32_t, double>> row;
        bool sorted = true;
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            if (t > rp[i] && col[t] < col[t - 1]) sorted = false;
        }
        if (!sorted) {
            for (int32_t t = rp[i]; t < rp[i + 1]; ++t) row.emplace_back(col[t], val[t]);
            std::sort(row.begin(), row.end(), [](const auto &a, const auto &b) { return a.first < b.first; });
            for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
                col[t] = row[t - rp[i]].first;
                val[t] = row[t - rp[i]].second;
            }
        }
        for (int32_t t = rp[i]; t < rp[i + 1]; ++t) {
            if (!P.a_col.empty() && (int32_t)P.a_col.size() > P.a_rowptr[i] && P.a_col.back() == col[t]) {
                P.a_val.back() += val[t];
            } else {
                P.a_col.push_back(col[t]);
                P.a_val.push_back(val[t]);
            }
        }
        P.a_rowptr[i + 1] = (int32_t)P.a_col.size();
    }
    P.nnz = (int64_t)P.a_col.size();
    // CSR of A^T from CSR of A (counting sort by column; rows come in order)
    std::vector<int32_t> ccnt(n + 1, 0);
    for (int64_t t = 0; t < P.nnz; ++t) ccnt[P.a_col[t] + 1]++;
    P.at_rowptr.assign(n + 1, 0);
    for (int32_t j = 0; j < n; ++j) P.at_rowptr[j + 1] = P.at_rowptr[j] + ccnt[j + 1];
    P.at_col.resize(P.nnz);
    P.at_val.resize(P.nnz);
    std::vector<int32_t> cpos(P.at_rowptr.begin(), P.at_rowptr.end() - 1);
    for (int32_t i = 0; i < m; ++i)
        for (int32_t t = P.a_rowptr[i]; t < P.a_rowptr[i + 1]; ++t) {
            const int32_t j = P.a_col[t];
            P.at_col[cpos[j]] = i;
            P.at_val[cpos[j]] = P.a_val[t];
            cpos[j]++;
        }
    P.b.assign(b, b + m);
    P.c.assign(c, c + n);
    P.z = k->z;
    P.l = k->l;
    P.ep = k->ep;
    P.ed = k->ed;
    P.pw.assign(k->p, k->p + k->np);
    P.q.assign(k->q, k->q + k->nq);
    P.s.assign(k->s, k->s + k->ns);
    return 0;
}

namespace {

int validate_settings(const scs_settings &s) {
    if (!(s.alpha > 0.0 && s.alpha < 2.0)) { set_error("alpha must lie in (0, 2)"); return SCS_INVALID_INPUT; }
    if (s.max_iters < 0 || s.check_interval < 1 || s.cg_max_iters < 0 || s.scale_passes < 0) {
        set_error("iteration counts out of range");
        return SCS_INVALID_INPUT;
    }
    if (!(s.cg_adapt >= 0.0) || !(s.cg_tol_rel >= 0.0)) { set_error("negative CG tolerance setting"); return SCS_INVALID_INPUT; }
    if (!(s.psd_fp64_cond >= 1.0)) { set_error("psd_fp64_cond must be >= 1"); return SCS_INVALID_INPUT; }
    if (s.precision != 0 && s.precision != 1) { set_error("precision must be 0 or 1"); return SCS_INVALID_INPUT; }
    if (s.block_scale < 0 || s.block_scale > 2) { set_error("block_scale must be 0, 1 or 2"); return SCS_INVALID_INPUT; }
    if (s.linsys != 0 && s.linsys != 1) { set_error("linsys must be 0 or 1"); return SCS_INVALID_INPUT; }
    return 0;
}

template <typename F>
int guarded(F f) {
    try {
        return f();
    } catch (const scs::CudaError &e) {
        set_error(e.what());
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return SCS_DEVICE_ERROR;
    } catch (const std::exception &e) {
        set_error(e.what());
        return SCS_DEVICE_ERROR;
    } catch (...) {
        set_error("unknown error");
        return SCS_DEVICE_ERROR;
    }
}

}  // namespace

extern "C" {

void scs_default_settings(scs_settings *s) {
    if (!s) return;
    std::memset(s, 0, sizeof(*s));
    s->eps_pri = s->eps_dual = s->eps_gap = 1e-4;
    s->eps_infeas = s->eps_unbdd = 1e-4;
    s->alpha = 1.5;
    s->cg_rate = 1.5;
    s->cg_adapt = 0.3;
    s->cg_tol_rel = 0.0;
    s->time_limit_s = 0.0;
    s->psd_fp64_cond = 1e6;
    s->max_iters = 10000;
    s->check_interval = 20;
    s->cg_max_iters = 50;
    s->normalize = 1;
    s->scale_passes = 10;
    s->block_scale = 1;
    s->precision = 1;
    s->use_graph = 1;
    s->verbose = 0;
    s->device = 0;
    s->cuda_stream = nullptr;
    s->linsys = 0;
}

scs_work *scs_init(const scs_csc *A, const double *b, const double *c, const scs_cone *k, const scs_settings *st,
                   int32_t *err) {
    scs_settings s;
    if (st) s = *st; else scs_default_settings(&s);
    scs_work *w = nullptr;
    const int rc = guarded([&]() -> int {
        int r = validate_settings(s);
        if (r) return r;
        scs::HostProblem P;
        r = validate_and_build(A, b, c, k, P);
        if (r) return r;
        w = new scs_work();
        w->device = s.device;
        w->eng = s.precision == 0 ? scs::make_engine_f64(P, s) : scs::make_engine_f32(P, s);
        return 0;
    });
    if (rc != 0) {
        if (w) {
            delete w->eng;
            delete w;
        }
        if (err) *err = rc;
        return nullptr;
    }
    if (err) *err = 0;
    return w;
}

int32_t scs_solve(scs_work *w, double *x, double *y, double *s, scs_info *info) {
    if (!w || !w->eng) { set_error("null work"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->solve(x, y, s, info); });
}

int32_t scs_warm_start(scs_work *w, const double *x, const double *y, const double *s) {
    if (!w || !w->eng) { set_error("null work"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->warm_start(x, y, s); });
}

void scs_finish(scs_work *w) {
    if (!w) return;
    guarded([&] {
        delete w->eng;
        return 0;
    });
    delete w;
}

int32_t scs_reset(scs_work *w) {
    if (!w || !w->eng) { set_error("null work"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->reset(); });
}

int32_t scs_iterate(scs_work *w, int32_t iters, int32_t sync) {
    if (!w || !w->eng || iters < 0) { set_error("bad argument"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->iterate(iters, sync); });
}

int32_t scs_update_bc(scs_work *w, const double *b, const double *c) {
    if (!w || !w->eng || !b || !c) { set_error("bad argument"); return SCS_INVALID_INPUT; }
    int32_t m = 0, n = 0;
    w->eng->dims(&m, &n, nullptr, nullptr);
    for (int32_t i = 0; i < m; ++i)
        if (!std::isfinite(b[i])) { set_error("non-finite entry in b"); return SCS_INVALID_INPUT; }
    for (int32_t j = 0; j < n; ++j)
        if (!std::isfinite(c[j])) { set_error("non-finite entry in c"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->update_bc(b, c); });
}

int32_t scs_iterate_checked(scs_work *w, int32_t iters, int32_t *status) {
    if (!w || !w->eng || iters < 0) { set_error("bad argument"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->iterate_checked(iters, status); });
}

int32_t scs_iterate_profiled(scs_work *w, int32_t iters) {
    if (!w || !w->eng || iters < 0) { set_error("bad argument"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->iterate_profiled(iters); });
}

int32_t scs_kernel_time(scs_work *w, int32_t kind, double *ms, int64_t *launches) {
    if (!w || !w->eng) { set_error("null work"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->kernel_time(kind, ms, launches); });
}

int32_t scs_get_iterates(scs_work *w, double *u, double *v) {
    if (!w || !w->eng) { set_error("null work"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->get_iterates(u, v); });
}

int32_t scs_get_scaling(scs_work *w, double *D, double *E, double *sigma, double *rho) {
    if (!w || !w->eng) { set_error("null work"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->get_scaling(D, E, sigma, rho); });
}

int32_t scs_dims(scs_work *w, int32_t *m, int32_t *n, int64_t *nnz, int64_t *device_bytes) {
    if (!w || !w->eng) { set_error("null work"); return SCS_INVALID_INPUT; }
    w->eng->dims(m, n, nnz, device_bytes);
    return 0;
}

int32_t scs_counters(scs_work *w, int32_t *iters, int64_t *cg_iters) {
    if (!w || !w->eng) { set_error("null work"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->counters(iters, cg_iters); });
}

int32_t scs_psd_counters(scs_work *w, int64_t *calls, int64_t *sweeps, int64_t *fp64_blocks) {
    if (!w || !w->eng) { set_error("null work"); return SCS_INVALID_INPUT; }
    return guarded([&] { return w->eng->psd_counters(calls, sweeps, fp64_blocks); });
}

const char *scs_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
