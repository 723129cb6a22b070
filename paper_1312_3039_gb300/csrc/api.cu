// C ABI of the solver (include/scs_gpu.h): input validation, the host-side
// CSC -> CSR layouts of A and A^T, and dispatch to the FP64 or mixed
// FP32/FP64 device engine.  No C++ exception crosses this boundary.
#include <cmath>
#include <cstring>
#include <string>

#include "../../include/scs_gpu.h"
#include <algorithm>
#include <new>
#include <thread>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "engine_base.h"
#include "host_par.h"
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

namespace {

using scs::host_threads;
using scs::run_parts;

// T + 1 column boundaries splitting the stored entries of a CSC matrix into
// parts of about equal size.
std::vector<int32_t> column_cuts(const int64_t *colptr, int32_t n, int T) { return scs::weight_cuts(colptr, n, T); }

// Canonical CSC (row indices strictly increasing in every column) from any
// CSC: each column sorted by row (stable), entries with equal row summed in
// input order.  Threads over parts of the columns.
void canonicalize(const scs_csc *A, int T, std::vector<int64_t> &cp, std::vector<int32_t> &ri,
                  std::vector<double> &vv) {
    const int32_t n = A->n;
    const int64_t nnz = A->colptr[n];
    ri.resize(nnz);
    vv.resize(nnz);
    std::vector<int64_t> len(n);
    const std::vector<int32_t> cut = column_cuts(A->colptr, n, T);
    std::vector<char> failed(T, 0);
    run_parts(T, [&](int t) {
        try {
            std::vector<int64_t> ord;
            for (int32_t j = cut[t]; j < cut[t + 1]; ++j) {
                const int64_t a = A->colptr[j], e = A->colptr[j + 1];
                ord.resize(e - a);
                for (int64_t u = a; u < e; ++u) ord[u - a] = u;
                std::stable_sort(ord.begin(), ord.end(),
                                 [&](int64_t x, int64_t y) { return A->rowidx[x] < A->rowidx[y]; });
                int64_t w = a;
                for (int64_t u : ord) {
                    if (w > a && ri[w - 1] == A->rowidx[u]) {
                        vv[w - 1] += A->val[u];
                    } else {
                        ri[w] = A->rowidx[u];
                        vv[w] = A->val[u];
                        ++w;
                    }
                }
                len[j] = w - a;
            }
        } catch (...) {
            failed[t] = 1;
        }
    });
    for (char f : failed)
        if (f) throw std::bad_alloc();
    cp.assign(n + 1, 0);
    for (int32_t j = 0; j < n; ++j) cp[j + 1] = cp[j] + len[j];
    // compact in place: column j moves from colptr[j] down to cp[j] <= colptr[j]
    for (int32_t j = 0; j < n; ++j) {
        const int64_t a = A->colptr[j];
        if (cp[j] != a) {
            std::copy(ri.begin() + a, ri.begin() + a + len[j], ri.begin() + cp[j]);
            std::copy(vv.begin() + a, vv.begin() + a + len[j], vv.begin() + cp[j]);
        }
    }
    ri.resize(cp[n]);
    vv.resize(cp[n]);
}

// CSR (rowptr, col, val) of a canonical CSC matrix with m rows: a counting
// sort by row.  The rows are split into T parts; each thread visits every
// column in order and keeps the entries of its own rows, so each CSR row
// comes out sorted by column and the result does not depend on T.
void csc_to_csr(const int64_t *colptr, const int32_t *rowidx, const double *val, int32_t m, int32_t n, int T,
                std::vector<int32_t> &rowptr, std::vector<int32_t> &col, std::vector<double> &out) {
    const int64_t nnz = colptr[n];
    rowptr.assign(m + 1, 0);
    col.resize(nnz);
    out.resize(nnz);
    std::vector<int32_t> r0(T + 1);
    for (int t = 0; t <= T; ++t) r0[t] = static_cast<int32_t>((int64_t)m * t / T);
    std::vector<int64_t> total(T, 0);
    // pass 1: row lengths (into rowptr[i + 1])
    run_parts(T, [&](int t) {
        const uint32_t lo = static_cast<uint32_t>(r0[t]), span = static_cast<uint32_t>(r0[t + 1] - r0[t]);
        int32_t *cnt = rowptr.data() + 1;
        for (int64_t u = 0; u < nnz; ++u) {
            const uint32_t i = static_cast<uint32_t>(rowidx[u]);
            if (i - lo < span) cnt[i]++;
        }
        int64_t s = 0;
        for (uint32_t i = lo; i < lo + span; ++i) s += cnt[i];
        total[t] = s;
    });
    // row starts: the parts' offsets, then a running sum inside each part
    std::vector<int64_t> off(T + 1, 0);
    for (int t = 0; t < T; ++t) off[t + 1] = off[t] + total[t];
    run_parts(T, [&](int t) {
        int64_t s = off[t];
        for (int32_t i = r0[t]; i < r0[t + 1]; ++i) {
            s += rowptr[i + 1];
            rowptr[i + 1] = static_cast<int32_t>(s);
        }
    });
    // pass 2: scatter, columns in order
    std::vector<std::vector<int32_t>> cursor(T);
    for (int t = 0; t < T; ++t) cursor[t].assign(rowptr.begin() + r0[t], rowptr.begin() + r0[t + 1]);
    run_parts(T, [&](int t) {
        const uint32_t lo = static_cast<uint32_t>(r0[t]), span = static_cast<uint32_t>(r0[t + 1] - r0[t]);
        std::vector<int32_t> &pos = cursor[t];
        for (int32_t j = 0; j < n; ++j)
            for (int64_t u = colptr[j]; u < colptr[j + 1]; ++u) {
                const uint32_t i = static_cast<uint32_t>(rowidx[u]);
                if (i - lo < span) {
                    const int32_t w = pos[i - lo]++;
                    col[w] = j;
                    out[w] = val[u];
                }
            }
    });
}

}  // namespace

static int build_problem(const scs_csc *A, const double *b, const double *c, const scs_cone *k,
                         scs::HostProblem &P, bool view_transpose) {
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
    // entries: row range, finiteness, and whether the rows of every column
    // are strictly increasing (then the CSC already is the CSR of A^T)
    const int T = host_threads(nnz_in);
    const std::vector<int32_t> cut = column_cuts(A->colptr, n, T);
    std::vector<char> bad_row(T, 0), bad_val(T, 0), unsorted(T, 0);
    run_parts(T, [&](int t) {
        for (int32_t j = cut[t]; j < cut[t + 1]; ++j)
            for (int64_t u = A->colptr[j]; u < A->colptr[j + 1]; ++u) {
                const int32_t i = A->rowidx[u];
                if (i < 0 || i >= m) bad_row[t] = 1;
                if (!std::isfinite(A->val[u])) bad_val[t] = 1;
                if (u > A->colptr[j] && i <= A->rowidx[u - 1]) unsorted[t] = 1;
            }
    });
    for (int t = 0; t < T; ++t)
        if (bad_row[t]) { set_error("row index out of range"); return SCS_INVALID_INPUT; }
    for (int t = 0; t < T; ++t)
        if (bad_val[t]) { set_error("non-finite entry in A"); return SCS_INVALID_INPUT; }
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

    // CSR of A^T: the canonical CSC of A (A's own arrays when its columns
    // are canonical); CSR of A: its counting-sort transpose
    P.m = m;
    P.n = n;
    const bool canonical = std::none_of(unsorted.begin(), unsorted.end(), [](char f) { return f != 0; });
    if (canonical) {
        P.at_rowptr.resize(n + 1);
        if (view_transpose) {
            P.at_col_view = A->rowidx;
            P.at_val_view = A->val;
        } else {
            P.at_col.resize(nnz_in);
            P.at_val.resize(nnz_in);
        }
        run_parts(T, [&](int t) {
            const int64_t a = A->colptr[cut[t]], e = A->colptr[cut[t + 1]];
            if (!view_transpose) {
                std::copy(A->rowidx + a, A->rowidx + e, P.at_col.begin() + a);
                std::copy(A->val + a, A->val + e, P.at_val.begin() + a);
            }
            for (int32_t j = cut[t]; j < cut[t + 1]; ++j) P.at_rowptr[j + 1] = static_cast<int32_t>(A->colptr[j + 1]);
        });
        csc_to_csr(A->colptr, A->rowidx, A->val, m, n, T, P.a_rowptr, P.a_col, P.a_val);
    } else {
        std::vector<int64_t> cp;
        canonicalize(A, T, cp, P.at_col, P.at_val);
        P.at_rowptr.resize(n + 1);
        for (int32_t j = 0; j <= n; ++j) P.at_rowptr[j] = static_cast<int32_t>(cp[j]);
        csc_to_csr(cp.data(), P.at_col.data(), P.at_val.data(), m, n, host_threads(cp[n]), P.a_rowptr, P.a_col,
                   P.a_val);
    }
    P.nnz = static_cast<int64_t>(P.a_col.size());
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

int scs::validate_and_build(const scs_csc *A, const double *b, const double *c, const scs_cone *k,
                            scs::HostProblem &P, bool view_transpose) {
    try {
        return build_problem(A, b, c, k, P, view_transpose);
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return SCS_DEVICE_ERROR;
    }
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
        // the engine uploads CSR(A^T) before scs_init returns: a canonical
        // CSC's own arrays serve as its columns and values
        r = validate_and_build(A, b, c, k, P, true);
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
