// Host-side interface between the C ABI and the device engines.
#pragma once

#include <stdint.h>

#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/scs_gpu.h"

namespace scs {

struct CudaError : std::runtime_error {
    int code;
    CudaError(const std::string &s, int c) : std::runtime_error(s), code(c) {}
};

#define SCS_CUDA(call)                                                                                  \
    do {                                                                                                \
        cudaError_t e_ = (call);                                                                        \
        if (e_ != cudaSuccess)                                                                          \
            throw ::scs::CudaError(std::string(#call) + ": " + cudaGetErrorString(e_), SCS_DEVICE_ERROR); \
    } while (0)

// The problem after host-side validation and layout (CSR of A and of A^T).
struct HostProblem {
    int32_t m = 0, n = 0;
    int64_t nnz = 0;
    std::vector<int32_t> a_rowptr, a_col, at_rowptr, at_col;
    std::vector<double> a_val, at_val, b, c;
    // CSR(A^T) columns and values as views of the caller's canonical CSC
    // arrays (at_col, at_val left empty); valid while the building call runs
    const int32_t *at_col_view = nullptr;
    const double *at_val_view = nullptr;
    int32_t z = 0, l = 0, ep = 0, ed = 0;
    std::vector<double> pw;     // power-cone parameters (negative: dual power cone)
    std::vector<int32_t> q, s;
};

// Validate A (CSC), b, c and the cone and build the host CSR layouts
// (api.cu); returns 0 or an SCS_* status after setting the error text.
// view_transpose: when the CSC is canonical, leave CSR(A^T)'s columns and
// values as views of its arrays instead of copies.
int validate_and_build(const scs_csc *A, const double *b, const double *c, const scs_cone *k, HostProblem &P,
                       bool view_transpose = false);
// Error text returned by scs_last_error() on this thread.
void set_last_error(const std::string &s);

class EngineBase {
   public:
    virtual ~EngineBase() {}
    virtual int solve(double *x, double *y, double *s, scs_info *info) = 0;
    virtual int warm_start(const double *x, const double *y, const double *s) = 0;
    virtual int reset() = 0;
    virtual int update_bc(const double *b, const double *c) = 0;
    virtual int iterate(int iters, int sync) = 0;
    virtual int iterate_checked(int iters, int32_t *status) = 0;
    virtual int iterate_profiled(int iters) = 0;
    virtual int kernel_time(int kind, double *ms, int64_t *launches) = 0;
    virtual int get_iterates(double *u, double *v) = 0;
    virtual int get_scaling(double *D, double *E, double *sigma, double *rho) = 0;
    virtual void dims(int32_t *m, int32_t *n, int64_t *nnz, int64_t *bytes) = 0;
    virtual int counters(int32_t *iters, int64_t *cg_iters) = 0;
    virtual int psd_counters(int64_t *calls, int64_t *sweeps, int64_t *fp64) = 0;
    double setup_s = 0.0;
};

EngineBase *make_engine_f64(const HostProblem &P, const scs_settings &st);
EngineBase *make_engine_f32(const HostProblem &P, const scs_settings &st);

}  // namespace scs
