/*
 * scs_gpu.h -- C ABI of the GB300 splitting conic solver.
 *
 * Solves the primal-dual pair of cone programs (Sec. 2, Eq. "e-coneprob")
 *
 *     minimize  c^T x   subject to  A x + s = b,  s in K
 *     maximize -b^T y   subject to  -A^T y + r = c,  r = 0,  y in K*
 *
 * by ADMM on the homogeneous self-dual embedding (Sec. 2.3, Eq. "e-hsd";
 * iteration Eq. "e-SCS" with over-relaxation, Sec. 3.3), projecting onto the
 * subspace with the indirect method of Sec. 4.1 (Jacobi-preconditioned CG on
 * I + A^T A, warm-started, stopped at zeta^k = (1/k)^cg_rate, Sec. 6.1) and
 * onto the cone block by block.  Data are equilibrated as in Sec. 5 and
 * termination follows Sec. 3.5 / Sec. 5 ("Scaled termination criteria").
 *
 * Every step of the iteration runs in CUDA kernels on one GPU; the host only
 * validates input, builds the sparse layouts, launches and reads a status
 * word every `check_interval` iterations.
 *
 * Conventions
 *   - All symbols are extern "C"; no C++ exception crosses the ABI.  Every
 *     call returns a status (or NULL plus *err) and never aborts the process.
 *   - Row order of K: `z` zero rows, `l` nonnegative rows, SOC blocks of sizes
 *     q[0..nq) (head first: {(t, x): ||x|| <= t}), PSD blocks of orders
 *     s[0..ns) in svec form (lower triangle column by column, off-diagonal
 *     entries times sqrt 2), `ep` exponential triples (x, y, z) with
 *     Kexp = closure{y > 0, y e^(x/y) <= z}, `ed` triples of its dual, and
 *     one triple per power-cone parameter p[i] (Sec. 6.1).
 *   - Host pointers unless stated.  Inputs are copied during the call; the
 *     caller keeps ownership.  A work object owns all device memory it uses
 *     until scs_finish.
 *   - One work object must not be used by two threads at once; distinct work
 *     objects are independent (each has its own CUDA stream unless one is
 *     given in the settings).
 */
#ifndef SCS_GPU_H
#define SCS_GPU_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes (Sec. 2.3: tau > 0 gives a solution, kappa > 0 a certificate) */
enum {
    SCS_SOLVED = 1,                 /* optimality tests of Sec. 3.5 passed                */
    SCS_SOLVED_INACCURATE = 2,      /* max_iters / time limit reached, tau dominant       */
    SCS_UNFINISHED = 0,
    SCS_INFEASIBLE = -1,            /* y/(-b^T y) certifies primal infeasibility (Sec. 2.2) */
    SCS_UNBOUNDED = -2,             /* x/(-c^T x) certifies dual infeasibility (Sec. 2.2)   */
    SCS_INFEASIBLE_INACCURATE = -3,
    SCS_UNBOUNDED_INACCURATE = -4,
    SCS_INVALID_INPUT = -10,
    SCS_DEVICE_ERROR = -11,
    SCS_TIMEOUT = -12,
    SCS_NUMERICAL = -13,
    SCS_UNSUPPORTED = -14           /* cone type or size this build does not handle       */
};

/* A in compressed sparse column form, 0-based.  colptr has n+1 entries,
 * rowidx/val have colptr[n] entries; row indices inside a column need not be
 * sorted; duplicate entries are summed; nnz must be below 2^31. */
typedef struct {
    int32_t m, n;
    const int64_t *colptr;
    const int32_t *rowidx;
    const double *val;
} scs_csc;

/* K = {0}^z x R+^l x SOC(q_0) x ... x PSD(s_0) x ... x Kexp^ep x (Kexp*)^ed
 * x Kpow(p_0) x ... (Sec. 6.1), rows in that order.  p[i] in (0, 1) is the
 * power cone Kpow^a = {(x, y, z): x^a y^(1-a) >= |z|, x, y >= 0}, a = p[i];
 * p[i] in (-1, 0) its dual (Kpow^a)* = {(u/a)^a (v/(1-a))^(1-a) >= |w|,
 * u, v >= 0} with a = -p[i]; each takes three rows (x, y, z).  Only the
 * single-problem solver and scs_project take ed, np > 0. */
typedef struct {
    int32_t z, l;
    const int32_t *q;
    int32_t nq;
    const int32_t *s;
    int32_t ns;
    int32_t ep;
    int32_t ed;                 /* dual exponential triples: K holds Kexp* itself */
    const double *p;            /* power-cone parameters, np of them          */
    int32_t np;
} scs_cone;

typedef struct {
    double eps_pri, eps_dual, eps_gap;    /* Sec. 3.5 tolerances                        */
    double eps_infeas, eps_unbdd;         /* Sec. 3.5 certificate tolerances            */
    double alpha;                         /* relaxation, Sec. 3.3; in (0, 2)            */
    double cg_rate;                       /* zeta^k = (1/k)^cg_rate; <= 0 disables it   */
    double cg_adapt;                      /* and at cg_adapt * ||(u^k, v^k) - (u^k-1, v^k-1)||
                                             (0 disables; see scs_default_settings)     */
    double cg_tol_rel;                    /* CG also stops at cg_tol_rel * ||u^k + v^k|| */
    double time_limit_s;                  /* <= 0: none                                 */
    double psd_fp64_cond;                 /* FP32 engine: a PSD block whose positive
                                             eigenvalues spread wider than this (max /
                                             min >= psd_fp64_cond) sums V max(L,0) V^T in
                                             FP64 (Sec. 6.1 projection); INFINITY: never */
    int32_t max_iters;
    int32_t check_interval;               /* termination test every this many iterations */
    int32_t cg_max_iters;                 /* cap on CG steps per ADMM iteration          */
    int32_t normalize;                    /* 1: equilibrate (Sec. 5); 0: use data as is   */
    int32_t scale_passes;                 /* equilibration passes                       */
    int32_t block_scale;                  /* one D value per SOC / PSD / exp block: the
                                             0 mean, 1 root mean square (default) or 2
                                             maximum of the block's row norms (Sec. 5)  */
    int32_t precision;                    /* 0: FP64 throughout; 1: FP32 A and CG, FP64
                                             iterates, residuals, gap and certificates */
    int32_t use_graph;                    /* 1: one CUDA graph per iteration with the CG
                                             loop as a device-side conditional node     */
    int32_t verbose;
    int32_t device;                       /* CUDA device ordinal                        */
    void *cuda_stream;                    /* cudaStream_t to run on, or NULL            */
    int32_t linsys;                       /* subspace step (Sec. 4.1): 0 indirect (PCG on
                                             I + A^T A); 1 direct: (I + A^T A)^-1 formed
                                             once at scs_init (FP64 Gauss-Jordan on the
                                             device) and reused by every iteration and
                                             warm-started solve (Sec. 4.2); n <= 8192 and
                                             m n <= 2^30 (SCS_UNSUPPORTED otherwise)    */
} scs_settings;

typedef struct {
    int32_t status;
    int32_t iters;                        /* ADMM iterations done                        */
    int32_t cg_iters;                     /* CG steps over the solve                     */
    int32_t matvecs;                      /* iters + ceil(iters / 20) + 2 * cg_iters: one
                                             A^T product per iteration outside CG, the A
                                             product of the CG's warm start on every 20th
                                             iteration (A z is carried in between), two
                                             per CG step (Table 5 counts 2 per iteration
                                             outside CG); linsys 1 adds one A product per
                                             iteration and takes no CG step             */
    double pobj, dobj;                    /* c^T x and -b^T y of the returned point      */
    double res_pri, res_dual, gap;        /* unscaled ||Ax+s-b||, ||A^T y+c||, |c^T x+b^T y| */
    double tau, kappa;
    double setup_s, solve_s;              /* wall time of scs_init and of scs_solve      */
} scs_info;

typedef struct scs_work scs_work;

/* Fill *s with defaults: eps 1e-4, alpha 1.5, cg_rate 1.5, cg_adapt 0.3,
 * cg_tol_rel 0, psd_fp64_cond 1e6,
 * max_iters 10000, check_interval 20, cg_max_iters 50, normalize 1,
 * scale_passes 10, block_scale 1, precision 1, use_graph 1, device 0,
 * linsys 0. */
void scs_default_settings(scs_settings *s);

/* Validate and copy A, b (m), c (n) and the cone to the device, equilibrate
 * (Sec. 5), form the Jacobi preconditioner diag(I + A^T A) and the cached
 * p = M^-1 h and 1 + h^T p (Sec. 4.1), set u0 = (0,0,1), v0 = (0,0,1)
 * (Sec. 3.4).  Returns NULL and sets *err (if err is not NULL) to an SCS_*
 * status on failure; scs_last_error() then describes it. */
scs_work *scs_init(const scs_csc *A, const double *b, const double *c,
                   const scs_cone *k, const scs_settings *st, int32_t *err);

/* Run the iteration from the current starting point (cold, or the one set by
 * scs_warm_start) until a Sec. 3.5 test passes, max_iters or the time limit.
 * x (n), y (m), s (m) receive, in host or device memory (unified addressing
 * tells them apart; the call returns when the copies are done), the solution
 * (status 1, 2) or
 * the certificate (status -1: y with b^T y = -1, x and s NaN; status -2: x
 * with c^T x = -1, s = -A x, y NaN).  Any output pointer may be NULL.  info
 * may be NULL.  The next call starts cold unless scs_warm_start is called. */
int32_t scs_solve(scs_work *w, double *x, double *y, double *s, scs_info *info);

/* Sec. 4.2 warm start: the next scs_solve starts from u0 = (x, y, 1),
 * v0 = (0, s, 0) (mapped into the scaled problem).  Host arrays of length n,
 * m, m; NULL entries are taken as zero.  The cached factor data and the CG
 * warm-start vector are kept. */
int32_t scs_warm_start(scs_work *w, const double *x, const double *y, const double *s);

/* Free everything the work object owns.  NULL is accepted. */
void scs_finish(scs_work *w);

/* ---- extensions (not in the paper's interface) ---------------------------- */

/* Sec. 4.2, repeated solves with the same A: new b (m) and c (n), host
 * arrays.  The scaling D, E, the sparse layouts and (linsys 1) the cached
 * (I + A^T A)^-1 depend on A only and are kept; sigma, rho, the scaled b^,
 * c^ and the cached p = M^-1 h are recomputed.  The next scs_solve starts
 * cold unless scs_warm_start is called after this. */
int32_t scs_update_bc(scs_work *w, const double *b, const double *c);

/* Reset the iterates to u0 = (0,0,1), v0 = (0,0,1) and the CG warm start to 0. */
int32_t scs_reset(scs_work *w);

/* Run exactly `iters` ADMM iterations from the current iterates, without
 * termination tests (benchmarking, resume).  Asynchronous on the work's
 * stream unless `sync` is nonzero. */
int32_t scs_iterate(scs_work *w, int32_t iters, int32_t sync);

/* Exactly `iters` ADMM iterations from the current iterates with the work
 * scs_solve does around them: every check_interval iterations the Sec. 3.5
 * tests run on the device and the host reads the status word (synchronising
 * the stream), but the call does not stop when a test passes (benchmarking
 * the solve's per-iteration cost).  *status (may be NULL) receives the last
 * check's result (0: no test passed; see the status codes). */
int32_t scs_iterate_checked(scs_work *w, int32_t iters, int32_t *status);

/* Copy the raw scaled iterates u = (x, y, tau) and v = (0, s, kappa), each of
 * length n + m + 1, to host arrays (either may be NULL). */
int32_t scs_get_iterates(scs_work *w, double *u, double *v);

/* Copy the scaling (Sec. 5) to host arrays D (m) and E (n), and sigma, rho. */
int32_t scs_get_scaling(scs_work *w, double *D, double *E, double *sigma, double *rho);

/* Per-kernel device time since the last call (CUDA events on the work's
 * stream, collected only by scs_iterate_profiled).  kind: 0 = SpMV with A in
 * the CG loop, 1 = SpMV with A^T in the CG loop, 2 = cone projection of the
 * non-PSD rows, 3 = projection of the PSD blocks, 4 = the direct subspace
 * step (linsys 1: the dense solve and its A product).
 * Writes the summed milliseconds and the launch count. */
int32_t scs_iterate_profiled(scs_work *w, int32_t iters);
int32_t scs_kernel_time(scs_work *w, int32_t kind, double *ms, int64_t *launches);

/* Iteration counters since the last reset / warm start / solve start: ADMM
 * iterations and CG steps (synchronises the work's stream). */
int32_t scs_counters(scs_work *w, int32_t *iters, int64_t *cg_iters);

/* PSD projection statistics since scs_init (Sec. 6.1 eigendecomposition per
 * block): block projections done, the Jacobi sweeps they took, and how many
 * of them summed the reconstruction V max(Lambda, 0) V^T in FP64 (blocks whose
 * eigenvalue magnitudes spread over more than 1e6, FP32 engine only).  Any
 * pointer may be NULL; synchronises the work's stream. */
int32_t scs_psd_counters(scs_work *w, int64_t *calls, int64_t *sweeps, int64_t *fp64_blocks);

/* Sizes of the work object's problem and the device bytes it holds. */
int32_t scs_dims(scs_work *w, int32_t *m, int32_t *n, int64_t *nnz, int64_t *device_bytes);

/* Euclidean projection, on the device, of `count` vectors stacked back to
 * back (each of the cone's length m, rows ordered as in scs_cone) onto K
 * (dual = 0) or onto K* (dual = 1): block by block, the zero cone (its dual
 * is all of R), the nonnegative and second-order cones (self-dual), the
 * exponential and power cones and their duals (Sec. 6.1; the duals through
 * Moreau, Eq. "e-moreau").  This puts a predicted warm start back into the cones.
 * v and out are device pointers to count * m doubles (out may equal v);
 * *dist2 (host, may be NULL) receives the sum over all vectors of
 * ||out - v||^2.  Runs on `stream` (a cudaStream_t, or NULL for the legacy
 * default stream) of the current device and returns when it is done.  It
 * allocates a device scratch buffer for the call (PSD blocks of order above
 * 96 add three order x order FP64 matrices per CTA).  PSD blocks (order at
 * most 1024) are projected by eigendecomposition, Sec. 6.1, with a
 * cold-started FP64 Jacobi eigensolver. */
int32_t scs_project(const scs_cone *k, int32_t dual, const double *v, double *out, int64_t count,
                    double *dist2, void *stream);

/* scs_project for callers that may not allocate device memory -- for
 * example an application whose own memory pool has already reserved the
 * whole GPU, or a serving process that gives the library its buffers and
 * stream and keeps every device allocation under its own control.
 * The paper has no counterpart: this is a property of the library.
 * Same arguments, result and stream semantics as scs_project (it returns
 * once the projection is done), but the call allocates nothing: its scratch
 * (the reduction's counters and partial sums, the SOC block tables and the
 * result) lives in one fixed-size device array inside the library, which
 * every GPU that loads the library holds (about 41 KB) until the process
 * exits.
 *   - Set-up: the first call on a device (and again after that device's
 *     CUDA context is replaced, e.g. by cudaDeviceReset) looks up the
 *     array's device address, with the device current; make that first
 *     call before any stream capture.
 *   - Limits: at most 4096 SOC blocks per cone, no PSD blocks (their
 *     eigensolver needs matrix scratch) and no power cones (their parameter
 *     table); SCS_UNSUPPORTED otherwise, with the reason in scs_last_error().
 *   - Every call shares the one array, and each call clears the part that
 *     must start at zero; calls that overlap on the GPU (different streams or
 *     threads at the same time) race on it and must not be issued. */
int32_t scs_project_noalloc(const scs_cone *k, int32_t dual, const double *v, double *out, int64_t count,
                            double *dist2, void *stream);

/* ---- batched persistent solver ----------------------------------------------
 * Many independent small programs solved together: the same iteration as
 * scs_solve (Eq. "e-SCS", indirect subspace step Sec. 4.1, equilibration
 * Sec. 5, tests Sec. 3.5), one CTA per program at a time inside one
 * persistent launch captured in a CUDA graph, the program's iterates and CG
 * vectors in shared memory.  Extends the paper's repeated-solve setting
 * (Sec. 4.2) to many programs at once; the paper has no batched form.
 * Cones: zero, nonnegative and second-order only (SCS_UNSUPPORTED
 * otherwise, including any exponential, power or PSD block); a program must fit one CTA's shared memory (about 4 (2 N + 6 n
 * + 4 m) bytes in FP32, N = n + m + 1).  No time limit. */
typedef struct scs_batch scs_batch;

/* count programs: A[i] (CSC, host), b and c concatenated in program order
 * (sum of m_i, sum of n_i doubles), cones k[i]; settings as for scs_init
 * (precision 0: FP64, 1: FP32 iterates with FP64 tests).  Runs the setup
 * launch (equilibration, Jacobi diagonal, p = M^-1 h per program) and the
 * autotuner (team size and long-row split timed on a sample of programs).
 * Returns NULL with *err set on failure. */
scs_batch *scs_batch_init(int32_t count, const scs_csc *A, const double *b, const double *c, const scs_cone *k,
                          const scs_settings *st, int32_t *err);

/* Solve every program from a cold start, or from the points of
 * scs_batch_warm_start.  x (sum n_i), y, s (sum m_i) in program order receive
 * each solution or certificate as scs_solve does; info[count] the per-program
 * status and counters (setup_s / solve_s are the batch's).  Any pointer may be
 * NULL.  Returns 0, or an error status for the whole call. */
int32_t scs_batch_solve(scs_batch *w, double *x, double *y, double *s, scs_info *info);

/* Sec. 4.2 warm start of every program (concatenated host arrays; NULL
 * entries are zero); used by the next scs_batch_solve only. */
int32_t scs_batch_warm_start(scs_batch *w, const double *x, const double *y, const double *s);

/* Exactly `iters` iterations of every program from its current iterates,
 * without termination tests (parity tests, timing). */
int32_t scs_batch_iterate(scs_batch *w, int32_t iters);

/* Scaled iterates u, v (n_i + m_i + 1 doubles each, host) of program index. */
int32_t scs_batch_get_iterates(scs_batch *w, int32_t index, double *u, double *v);

/* What the autotuner chose (threads per program, rows longer than row_split
 * nonzeros summed by a warp) and the time it and the setup took (ms). */
int32_t scs_batch_config(scs_batch *w, int32_t *threads, int32_t *row_split, double *tune_ms, double *setup_ms);

void scs_batch_finish(scs_batch *w);

/* ---- family solver: members sharing A and the cone -------------------------
 * Many programs with the same A and cone and their own b, c (the setting of
 * Sec. 4.2 where only b and c change between solves).  The equilibration
 * D, E (Sec. 5) depends on A only and is shared; sigma, rho are per member.
 * The subspace step uses the dense (I + A^T A)^-1, formed once in FP64 on the
 * device, so one iteration of all members is three dense products over the
 * member columns (FP32 or FP64 GEMMs) plus one fused update launch; the
 * Sec. 3.5 tests run every check_interval iterations.  Cones: zero,
 * nonnegative, SOC; dense A^ must have at most 2^31 entries.  The paper has
 * no batched family form; each member follows the paper's iteration with an
 * exact subspace solve. */
typedef struct scs_family scs_family;

/* A (CSC, host, shared), cone, count members; b: count x m, c: count x n
 * (host, member-major).  Returns NULL with *err set on failure. */
scs_family *scs_family_init(const scs_csc *A, const scs_cone *k, int32_t count, const double *b, const double *c,
                            const scs_settings *st, int32_t *err);

/* New b, c for every member (same layout); the shared inverse is kept. */
int32_t scs_family_set_data(scs_family *w, const double *b, const double *c);

/* Warm start of every member for the next solve, u0 = (x^, y^, 1),
 * v0 = (0, s^, 0) (Sec. 4.2).  device_scaled = 0: host arrays in the
 * caller's units (count x n, m, m); 1: device FP64 arrays already in each
 * member's scaled space.  NULL arrays are zero. */
int32_t scs_family_warm_start(scs_family *w, const double *x, const double *y, const double *s,
                              int32_t device_scaled);

/* Iterate every member until each has passed a test (or max_iters); x, y, s
 * (count x n, m, m) receive each member's solution or certificate as
 * scs_solve gives it, in host memory (device_out = 0) or device memory (1);
 * info[count] (host) the status and iteration count at which each member
 * stopped.  Any pointer may be NULL. */
int32_t scs_family_solve(scs_family *w, double *x, double *y, double *s, scs_info *info, int32_t device_out);

/* Exactly `iters` iterations of every member, no tests (parity tests). */
int32_t scs_family_iterate(scs_family *w, int32_t iters);

/* Scaled iterates u, v (n + m + 1 each, host) of one member. */
int32_t scs_family_get_iterates(scs_family *w, int32_t index, double *u, double *v);

/* Each member's scaled HSD state when it stopped, divided by its u_tau
 * (so (x^, y^, s^, 1) for a solved member), as float, count x (n + 2m + 1),
 * copied to dst (host or device). */
int32_t scs_family_snapshots(scs_family *w, float *dst);

/* Map each member's point from its scaled space to the caller's units
 * (Sec. 5: x = E x^ / sigma, y = D y^ / rho, s = s^ / (sigma D)), the inverse
 * of the warm-start mapping, so that a prediction made for the family can
 * warm-start the single-problem solver (scs_warm_start, Sec. 4.2) of the same
 * member.  All six arrays are device FP64, count x n, m, m (member-major);
 * synchronises the family's stream. */
int32_t scs_family_unscale(scs_family *w, const double *xh, const double *yh, const double *sh, double *x, double *y,
                           double *s);

int32_t scs_family_dims(scs_family *w, int32_t *n, int32_t *m, int32_t *count);
void scs_family_finish(scs_family *w);

/* ---- learned warm start --------------------------------------------------
 * A multilayer perceptron (d_in -> hidden x layers (GELU) -> d_out) that maps a
 * family member's parameter theta to its predicted scaled state
 * (u_x, u_y, v_s, u_tau); trained by MSE with Adam; BF16 tensor-core
 * products with FP32 accumulation and FP32 master weights.  The paper has no
 * learned component: this extends the warm start of Sec. 4.2.  All device
 * pointers; calls run on the network's stream (NULL: a private one). */
typedef struct scs_mlp scs_mlp;

/* batch: rows of every forward / training call, a positive multiple of 128. */
scs_mlp *scs_mlp_create(int32_t d_in, int32_t hidden, int32_t layers, int32_t d_out, int32_t batch, void *stream,
                        int32_t *err);
int64_t scs_mlp_param_count(scs_mlp *w);
/* Host FP32 parameters, per layer W (out x in, row-major) then b (out);
 * setting them also clears the optimiser state. */
int32_t scs_mlp_set_params(scs_mlp *w, const float *params);
int32_t scs_mlp_get_params(scs_mlp *w, float *params);
/* y (batch x d_out, FP32, device or host) = network(x) for x (batch x d_in,
 * FP32, device); synchronises. */
int32_t scs_mlp_forward(scs_mlp *w, const float *x, float *y);
/* Loss and gradients (host, packed like the parameters) for targets t
 * (batch x d_out, FP32, device); grads or loss may be NULL. */
int32_t scs_mlp_gradients(scs_mlp *w, const float *x, const float *t, float *grads, float *loss);
/* One Adam step (learning rate lr) on a batch; *loss (host) if not NULL
 * (then the call synchronises). */
int32_t scs_mlp_train_step(scs_mlp *w, const float *x, const float *t, float lr, float *loss);
/* Products on the 5th-generation tensor cores (tcgen05.mma with tensor-memory
 * accumulators, the default when every padded size allows it) or on the
 * warp-level mma.sync kernel (tcgen05 = 0); SCS_UNSUPPORTED if a padded size
 * is outside the tcgen05 kernel's tiling (multiples of 64, batch of 128). */
int32_t scs_mlp_set_tensor_path(scs_mlp *w, int32_t tcgen05);
/* 0, or SCS_DEVICE_ERROR if a tcgen05 product's bounded wait ever timed out
 * (its output is then not written); synchronises. */
int32_t scs_mlp_error(scs_mlp *w);
void scs_mlp_destroy(scs_mlp *w);

/* The network's product alone, for tests and tuning: C (M x N, FP32, ld ldc)
 * = A (M x K, BF16, ld lda) B (N x K, BF16, ld ldb)^T on the device, through
 * the tcgen05 kernel (tcgen05 = 1: M % 128, N % 64, K % 64) or the mma.sync
 * kernel (M % 128, N % 64, K % 32); rows 16-byte aligned.  Allocates a small
 * status word; synchronises `stream`. */
int32_t scs_bf16_gemm(const void *A, int32_t lda, const void *B, int32_t ldb, int32_t M, int32_t N, int32_t K,
                      float *C, int32_t ldc, int32_t tcgen05, void *stream);
/* The same product enqueued on `stream` only (no allocation, no
 * synchronisation), so that back-to-back launches can be timed: err is a
 * device int32 the caller zeroes beforehand; a tcgen05 launch sets it to 1
 * if a bounded wait timed out.  Shapes are checked on the host
 * (SCS_INVALID_INPUT); returns 0 once the launch is enqueued. */
int32_t scs_bf16_gemm_async(const void *A, int32_t lda, const void *B, int32_t ldb, int32_t M, int32_t N, int32_t K,
                            float *C, int32_t ldc, int32_t tcgen05, int32_t *err, void *stream);

/* The family solver's dense product alone (Sec. 4.1 direct step in dense
 * form), for tests and tuning: C (M x N) = alpha A (M x K) B (K x N) +
 * beta C, all column-major device arrays with leading dimensions lda >= M,
 * ldb >= K, ldc >= M; precision 0: FP64, 1: FP32 (alpha, beta rounded to
 * FP32), both plain CUDA-core fused multiply-adds in k order, enqueued on
 * `stream` (no allocation, no synchronisation); precision 2: FP32 operands
 * through the tensor cores, each split three ways into BF16 (x = x1 + x2 +
 * x3) and the six cross products above 2^-24 |a||b| accumulated in FP32 by
 * two tcgen05 products (a1 b1, then the five smaller ones added to it; the
 * FP32 family solver's path; this call allocates its scratch and
 * synchronises).  beta == 0 does not read C.
 * SCS_INVALID_INPUT for bad sizes or pointers, SCS_DEVICE_ERROR if the
 * launch fails. */
int32_t scs_dense_gemm(int32_t precision, int32_t M, int32_t N, int32_t K, double alpha, const void *A, int64_t lda,
                       const void *B, int64_t ldb, double beta, void *C, int64_t ldc, void *stream);

/* Device helpers of the warm-start pipeline (FP32 row-major data):
 * per-column mean and standard deviation; in-place standardisation
 * (d - mean) / sd; row gather dst[r] = src[idx[r]]. */
int32_t scs_column_stats(const float *data, int64_t rows, int32_t cols, float *mean, float *sd, void *stream);
int32_t scs_standardize(float *data, int64_t rows, int32_t cols, const float *mean, const float *sd, void *stream);
int32_t scs_gather_rows(const float *src, int32_t cols, const int64_t *idx, int64_t count, float *dst, void *stream);
/* A standardised prediction (count rows of ld >= n + 2m + 1 floats: u_x, u_y,
 * v_s, u_tau) to the scaled warm start x^ = u_x / tau, y^ = u_y / tau,
 * s^ = v_s / tau with tau = max(u_tau, tau_min) (FP64 device arrays count x n,
 * m, m); project y^ onto K* and s^ onto K afterwards (scs_project). */
int32_t scs_warm_from_prediction(const float *pred, int64_t ld, const float *mean, const float *sd, int32_t n,
                                 int32_t m, int64_t count, double tau_min, double *xh, double *yh, double *sh,
                                 void *stream);

/* Human-readable description of the most recent error on this thread. */
const char *scs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SCS_GPU_H */
