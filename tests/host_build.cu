// Host-only harness for the solver's CSC -> CSR build (csrc/api.cu): the C
// ABI's validate_and_build, with the device engines stubbed out, so that the
// CSR layouts of A and A^T can be checked on a machine without a GPU.
#include "../paper_1312_3039_gb300/csrc/api.cu"

namespace scs {
EngineBase *make_engine_f64(const HostProblem &, const scs_settings &) { return nullptr; }
EngineBase *make_engine_f32(const HostProblem &, const scs_settings &) { return nullptr; }
}  // namespace scs

namespace {
scs::HostProblem g_last;
}

extern "C" {

// Builds the problem; returns the status and the sizes (m, n, nnz) of the
// result, whose arrays host_build_copy then copies out.
int host_build(const scs_csc *A, const double *b, const double *c, const scs_cone *k, int64_t *sizes) {
    g_last = scs::HostProblem();
    const int rc = scs::validate_and_build(A, b, c, k, g_last);
    sizes[0] = g_last.m;
    sizes[1] = g_last.n;
    sizes[2] = g_last.nnz;
    return rc;
}

void host_build_copy(int32_t *a_rowptr, int32_t *a_col, double *a_val, int32_t *at_rowptr, int32_t *at_col,
                     double *at_val) {
    const scs::HostProblem &P = g_last;
    std::copy(P.a_rowptr.begin(), P.a_rowptr.end(), a_rowptr);
    std::copy(P.a_col.begin(), P.a_col.end(), a_col);
    std::copy(P.a_val.begin(), P.a_val.end(), a_val);
    std::copy(P.at_rowptr.begin(), P.at_rowptr.end(), at_rowptr);
    std::copy(P.at_col.begin(), P.at_col.end(), at_col);
    std::copy(P.at_val.begin(), P.at_val.end(), at_val);
}

}  // extern "C"
