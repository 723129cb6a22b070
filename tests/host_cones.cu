// Host build of the CUDA path's exponential- and power-cone projections (the
// same __host__ __device__ functions the kernels call), for CPU tests.
#include "../paper_1312_3039_gb300/csrc/cones.cuh"

extern "C" void host_proj_exp(const double *in, double *out, int n, int dual) {
    for (int i = 0; i < n; ++i) {
        if (dual)
            scs::proj_exp_dual(in[3 * i], in[3 * i + 1], in[3 * i + 2], out[3 * i], out[3 * i + 1], out[3 * i + 2]);
        else
            scs::proj_exp(in[3 * i], in[3 * i + 1], in[3 * i + 2], out[3 * i], out[3 * i + 1], out[3 * i + 2]);
    }
}

// FP32 version (the mixed-precision iteration's)
extern "C" void host_proj_exp_f(const float *in, float *out, int n, int dual) {
    for (int i = 0; i < n; ++i) {
        if (dual)
            scs::proj_exp_dual_f(in[3 * i], in[3 * i + 1], in[3 * i + 2], out[3 * i], out[3 * i + 1], out[3 * i + 2]);
        else
            scs::proj_exp_f(in[3 * i], in[3 * i + 1], in[3 * i + 2], out[3 * i], out[3 * i + 1], out[3 * i + 2]);
    }
}

// power cone Kpow^a (dual = 0) or its dual (dual = 1), one a per triple
extern "C" void host_proj_pow(const double *in, const double *a, double *out, int n, int dual) {
    for (int i = 0; i < n; ++i) {
        if (dual)
            scs::proj_pow_dual(in[3 * i], in[3 * i + 1], in[3 * i + 2], a[i], out[3 * i], out[3 * i + 1], out[3 * i + 2]);
        else
            scs::proj_pow(in[3 * i], in[3 * i + 1], in[3 * i + 2], a[i], out[3 * i], out[3 * i + 1], out[3 * i + 2]);
    }
}

extern "C" void host_proj_pow_f(const float *in, const float *a, float *out, int n, int dual) {
    for (int i = 0; i < n; ++i) {
        if (dual)
            scs::proj_pow_dual(in[3 * i], in[3 * i + 1], in[3 * i + 2], a[i], out[3 * i], out[3 * i + 1], out[3 * i + 2]);
        else
            scs::proj_pow(in[3 * i], in[3 * i + 1], in[3 * i + 2], a[i], out[3 * i], out[3 * i + 1], out[3 * i + 2]);
    }
}
