/*
 * pexp.h -- C ABI of the GB300 Paraexp exponential block Krylov (PEBK) library.
 *
 * Method: G.L. Kooij, M.A. Botchev, B.J. Geurts, "A block Krylov subspace
 * implementation of the time-parallel Paraexp method and its extension for
 * nonlinear partial differential equations", arXiv:1509.04567.
 *
 * The library solves the semi-discrete linear initial value problem
 *     u'(t) = A u(t) + g(t),  u(0) = u0,  t in [0, T]                 (Sec. 2.1, eq. ivp2)
 * for A the second-order central-difference advection-diffusion operator
 * (Sec. 3.1), by the time-parallel Paraexp decomposition (Sec. 2.2, Fig. 3):
 * shift by u0 (eq. linivp_shift), split the source over P subintervals
 * (eq. piecewiseSource_linivp), compress each subinterval's source samples by a
 * truncated thin SVD into g ~ U p(t) (eq. svd_appr), integrate every subproblem
 * (eq. linivpSubproblem) with an exponential block Krylov method
 * (eq. blockKrylovSubspace) and sum the subsolutions (eq. superposition).
 * The viscous Burgers equation is solved by waveform relaxation around the same
 * linear solver (Sec. 2.3-2.4, eq. ivp3, Fig. 5).
 *
 * Conventions for every entry point:
 *   - Return value: PEXP_OK (0) or a negative status code (below).  No C++
 *     exception crosses this boundary.  pexp_status_string() names a code.
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; the
 *     library reads/writes them in stream order on the context's stream and
 *     never frees them.  Pointers named *_host are host pointers (pinned memory
 *     gives the fastest copies); the call returns after the results are in them.
 *   - A state vector is n contiguous values, n = nx (1D) or nx*ny (2D, unknown
 *     (ix, iy) at index iy*nx + ix).  A time series of states (sources G,
 *     solutions Y) is n_out consecutive vectors: element (i, k) -- value k at
 *     output time t_i -- is at offset i*n + k ("time-major").
 *   - Output times are uniform: t_i = i*T/(n_out-1), i = 0..n_out-1.  Subinterval
 *     boundaries snap to this grid: T_j = t_{floor(j*(n_out-1)/P)}.
 *   - dtype arguments are PEXP_F64 (double) or PEXP_F32 (float).
 *   - A call is synchronous with respect to the host unless stated otherwise:
 *     it returns when its device work has completed (the Krylov loop reads
 *     convergence flags back to the host).
 *   - Errors: invalid sizes/options -> PEXP_ERR_INVALID_ARG with nothing
 *     written; CUDA runtime failure -> PEXP_ERR_CUDA; workspace allocation
 *     failure -> PEXP_ERR_OOM.
 */
#ifndef PEXP_H
#define PEXP_H

#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status codes */
#define PEXP_OK                     0
#define PEXP_ERR_INVALID_ARG       -1
#define PEXP_ERR_OOM               -2
#define PEXP_ERR_CUDA              -3
#define PEXP_ERR_BREAKDOWN         -4  /* Krylov block lost all directions unexpectedly */
#define PEXP_ERR_NOT_CONVERGED     -5  /* a subproblem missed tol within the step budget; output written */
#define PEXP_ERR_WR_NOT_CONVERGED  -6  /* waveform relaxation hit wr_max_iter; last iterate written */
#define PEXP_ERR_TIMEOUT           -7  /* a bounded device-side wait expired */
#define PEXP_ERR_UNSUPPORTED       -8  /* valid request not implemented for this operator/precision */
#define PEXP_ERR_SCRATCH_LIMIT     -9  /* request needs more than the fixed scratch of pexp_sai_solve_noalloc */
#define PEXP_ERR_WR_DIVERGED      -10  /* waveform relaxation updates grew wr_diverge times in a row; last iterate written */

/* ---------------------------------------------------------------- enumerations */
#define PEXP_BC_PERIODIC   0
#define PEXP_BC_DIRICHLET0 1

#define PEXP_KRYLOV_POLY 0   /* polynomial block Krylov space span{U, AU, A^2U, ...} (eq. blockKrylovSubspace) */
#define PEXP_KRYLOV_SAI  1   /* shift-and-invert space of (I - gamma A)^{-1} (Sec. 2.1, cited acceleration) */

#define PEXP_FP64  0         /* every n-length array and all arithmetic in FP64 */
#define PEXP_MIXED 1         /* n-length Krylov data in FP32 with FP32 arithmetic; small matrices in FP64 */

#define PEXP_F64 0
#define PEXP_F32 1

#define PEXP_NODES_UNIFORM   0   /* source sampled at the output times (Sec. 4's uniform samples) */
#define PEXP_NODES_CHEBYSHEV 1   /* source sampled at n_samp Chebyshev points per subinterval (Sec. 3) */

/* ---------------------------------------------------------------- descriptors */
/* The operator A of eq. ivp2: second-order central differences of
 * -a u_x + nu u_xx (Sec. 3.1), per dimension; 2D is the sum A_x + A_y.
 *   (A u)_i = nu (u_{i-1} - 2u_i + u_{i+1})/dx^2 - a (u_{i+1} - u_{i-1})/(2 dx)
 * dx = L/n (periodic) or L/(n+1) (homogeneous Dirichlet, interior points). */
typedef struct {
    int     dim;        /* 1 or 2 */
    int64_t nx, ny;     /* mesh points per dimension (ny ignored for dim 1) */
    int     bc;         /* PEXP_BC_* */
    double  ax, ay;     /* advection velocities */
    double  nu;         /* diffusivity */
    double  Lx, Ly;     /* domain lengths */
} pexp_operator;

/* Solver options.  Defaults: pexp_default_options(). */
typedef struct {
    double T;            /* final time */
    int    P;            /* number of subintervals, 1 <= P <= n_out-1 (Sec. 2.2) */
    int    n_out;        /* number of output times, >= 2 (the source sample times unless nodes = 1) */
    double tol;          /* relative tolerance of each EBK subproblem (Sec. 3, "tol") */
    double svd_tol;      /* keep singular values sigma_i > svd_tol*sigma_1 (Sec. 2.1) */
    int    max_rank;     /* cap on the retained rank m = block width, <= PEXP_MAX_RANK */
    int    restart_len;  /* block steps per Krylov cycle (Sec. 3: 20) */
    int    max_restarts; /* restart cycles after the first (Sec. 2.1, Sec. 3); the step budget is
                          * restart_len*(max_restarts+1) <= PEXP_MAX_STEPS.  0: one cycle that may grow to
                          * restart_len steps.  > 0: a subproblem not converged after restart_len steps of
                          * a cycle starts a new cycle for the error of the cycles so far, from the range
                          * of the cycle's rank-b residual (I - V V^T) A V, coupled to the previous cycle
                          * in one block lower-triangular projected problem; each cycle orthogonalises
                          * against its own blocks only.  Restarted solves run the dense-projection
                          * driver (not the fused kernels); report.sub_restarts counts the cycles. */
    int    krylov;       /* PEXP_KRYLOV_* */
    double sai_gamma;    /* SAI pole gamma = sai_gamma * T / P (nominal subinterval length) */
    int    precision;    /* PEXP_FP64 or PEXP_MIXED */
    int    wr_max_iter;  /* waveform relaxation iteration limit (Fig. 5, K) */
    double wr_tol;       /* stop when max_i||u_{k+1}(t_i)-u_k(t_i)|| <= wr_tol*max_i||u_{k+1}(t_i)|| */
    int    burgers_form; /* 0: -(u_{i+1}^2-u_{i-1}^2)/(4dx);  1: -u_i(u_{i+1}-u_{i-1})/(2dx) */
    int    diagnostics;  /* bit 0: measure the orthogonality of every Krylov basis (report.orth_max) */
    int    jacobian;     /* Burgers WR: 0 = Picard (eq. ivp3); 1 = averaged-Jacobian correction (eq. ivp4,
                          * one Jacobian per subinterval at its time-averaged iterate, eq. piecewiseJac) */
    int    wr_diverge;   /* Burgers WR: stop with PEXP_ERR_WR_DIVERGED once the relative update has grown
                          * this many iterations in a row (0 = never) */
    /* Linear solves: solve only the subproblems j = sub_first .. sub_last-1 (0-based, eq.
     * linivpSubproblem) and sum their solutions (eq. superposition); 0, 0 = all.  Outputs up to
     * T_{sub_first} are set to zero and u0 is added only when sub_first = 0, so the solutions
     * of disjoint ranges add up to the full solve (the subintervals split over several GPUs). */
    int    sub_first;
    int    sub_last;
    /* Linear solves: where the source is sampled (Sec. 3: "the sample points per subinterval
     * are Chebyshev nodes").  PEXP_NODES_UNIFORM (default): at the output times, G has n_out
     * rows.  PEXP_NODES_CHEBYSHEV: at n_samp (2 .. PEXP_MAX_SAMPLES) Chebyshev extrema of every
     * subinterval [T_{j-1}, T_j], the i-th at T_{j-1} + (T_j - T_{j-1}) (1 - cos(pi i/(n_samp-1)))/2,
     * both ends included and shared with the neighbour: G has P*(n_samp-1)+1 rows, subinterval
     * j's (1-based) at rows (j-1)*(n_samp-1) .. j*(n_samp-1).  The cubic spline of the source
     * model runs through these samples and the outputs stay at the uniform times.  Not for
     * pexp_solve_burgers (PEXP_ERR_UNSUPPORTED), whose source samples are its iterate's. */
    int    nodes;
    int    n_samp;
} pexp_options;

#define PEXP_DIAG_ORTH  1   /* measure the orthogonality of every Krylov basis */
#define PEXP_DIAG_KTIME 2   /* time kernel classes with CUDA events (report.k_*) */
#define PEXP_DIAG_NOCOOP 4  /* launch every Krylov pass on its own: no cooperative launches (a
                               single-column periodic window of up to 2^18 points otherwise runs
                               its shift-and-invert passes, and its Gram-Schmidt passes, as one
                               grid-synchronised launch each); the results are the same bit for bit */
/* With PEXP_DIAG_KTIME, bits 8..15 of `diagnostics` choose the classes that are timed:
 * bit 8 + PEXP_KC_x times class x; no bit set times every class.  Each timed launch
 * costs two event records on the host, so timing one class perturbs a solve least. */
#define PEXP_DIAG_KTIME_CLASS(cls) (1 << (8 + (cls)))
/* With PEXP_DIAG_KTIME, bits 16..19 = k > 0 time a sample of about 1 in 2^k of the launches
 * of the chosen classes, picked by a fixed pseudo-random sequence (so that no kernel of a
 * repeating launch pattern is favoured); report.k_* then cover the sampled launches only.
 * Events between the kernels of a Krylov step stop their launches from overlapping, so
 * sampling keeps the timing from slowing the solve it measures. */
#define PEXP_DIAG_KTIME_SAMPLE(k) ((k) << 16)

/* kernel classes of report.k_ms / k_launches / k_bytes */
#define PEXP_KC_SAI     0   /* shift-and-invert recurrence solve */
#define PEXP_KC_STENCIL 1   /* operator stencil (A V, A^T V) */
#define PEXP_KC_PROJ    2   /* tall-skinny projections X^T Y (Gram-Schmidt, Galerkin, Gram) */
#define PEXP_KC_UPDATE  3   /* tall-skinny block updates X T */
#define PEXP_KC_SMALL   4   /* per-subinterval small FP64 kernels */
#define PEXP_KC_SOURCE  5   /* source Gram matrix and source block */
#define PEXP_KC_RECON   6   /* reconstruction of the outputs */
#define PEXP_KC_COUNT   8

#define PEXP_MAX_RANK   16    /* largest block width */
#define PEXP_MAX_STEPS  64    /* largest Krylov step budget restart_len*(max_restarts+1) */
#define PEXP_MAX_SAMPLES 112  /* largest number of samples in one subinterval: the FP64 source
                                 Gram tile, 8 (s|1) 256 bytes, fits one CTA's shared memory */
#define PEXP_REPORT_SUBS 128  /* per-subinterval report entries (the first 128 subintervals) */
#define PEXP_REPORT_WR   64   /* WR update history entries (the first 64 iterations) */

/* Per-call report (host memory, optional). */
typedef struct {
    int    status;
    int    n_sub;             /* P */
    int    rank_max;          /* max_j m_j (retained source rank) */
    int    rank_min;
    int    k_nh_max;          /* max block steps of the source (nonhomogeneous) parts */
    int    k_hom_max;         /* max steps of the homogeneous continuation windows */
    int    k_hom_sum;         /* total homogeneous steps */
    int    not_converged;     /* number of Krylov solves that missed tol */
    double est_max;           /* largest final error estimate (relative) */
    double sigma_ratio_max;   /* max_j sigma_{m_j+1}/sigma_1 (first dropped singular value) */
    int    wr_iters;          /* waveform relaxation iterations made */
    double wr_delta;          /* last relative WR update */
    double time_ms;           /* device time of the solve (CUDA events) */
    double t_source_ms;       /* phase times (CUDA events): source compression */
    double t_krylov_ms;       /*   nonhomogeneous block Krylov solves (all subintervals) */
    double t_hom_ms;          /*   homogeneous continuation chain */
    double t_recon_ms;        /*   reconstruction of all output times */
    double orth_max;          /* max over bases of max|V^T V - I| (PEXP_DIAG_ORTH), else -1 */
    double k_ms[PEXP_KC_COUNT];      /* PEXP_DIAG_KTIME: summed kernel time per class (ms) */
    int    k_launches[PEXP_KC_COUNT];/*   launches per class */
    double k_bytes[PEXP_KC_COUNT];   /*   bytes the kernels move per class: each array once per launch,
                                      *   the low parts of an FP32 working block included */
    double bytes_alg;         /* algorithmic HBM bytes: each array counted once per pass the method needs */
    int    launches;          /* kernels launched by the call */
    double k_bytes_alg[PEXP_KC_COUNT];/* PEXP_DIAG_KTIME: algorithmic bytes per class: every array at its
                                      *   storage width (FP32 working block at 4 bytes), once per launch */
    int    sub_rank[PEXP_REPORT_SUBS];      /* retained source rank m_j of subinterval j = 1.. */
    int    sub_steps[PEXP_REPORT_SUBS];     /* block steps of subproblem j's nonhomogeneous part */
    int    sub_hom_steps[PEXP_REPORT_SUBS]; /* steps of the homogeneous continuation on subinterval j */
    int    sub_restarts[PEXP_REPORT_SUBS];  /* Krylov restart cycles of subproblem j's nonhomogeneous part */
    double wr_history[PEXP_REPORT_WR];      /* relative WR update of iterations 1, 2, ... */
} pexp_report;

typedef struct pexp_ctx pexp_ctx;

/* ---------------------------------------------------------------- context */
/* Create a context on CUDA device `device` using `cuda_stream` (a cudaStream_t,
 * NULL = the legacy default stream; borrowed, not destroyed).  The context owns a
 * device workspace that grows on demand and is freed by pexp_destroy. */
int pexp_create(pexp_ctx** out, int device, void* cuda_stream);
int pexp_destroy(pexp_ctx* ctx);
int pexp_set_stream(pexp_ctx* ctx, void* cuda_stream);
void pexp_default_options(pexp_options* opts);
const char* pexp_status_string(int status);

/* ---------------------------------------------------------------- solvers */
/* Paraexp-EBK linear solve (Sec. 2.2, Fig. 3).
 *   y0_dev: n FP64 values (always FP64: the shift g_hat = A u0 + g of eq. linivp_shift
 *   multiplies the rounding error of u0 by ||A||, up to ~4e9 on fine meshes, so u0 must
 *   carry full precision whatever the precision of the solve).  G_dev: n_out*n source samples g(t_i)
 *   (time-major, dtype g_dtype; with opts->nodes = PEXP_NODES_CHEBYSHEV, P*(n_samp-1)+1 samples at
 *   the Chebyshev points) or NULL for g = 0.  Y_dev: n_out*n outputs
 *   u(t_i) (time-major, dtype y_dtype); must not overlap G_dev or y0_dev.
 * Returns PEXP_ERR_NOT_CONVERGED (outputs still written) when a Krylov solve missed tol. */
int pexp_solve_linear(pexp_ctx* ctx, const pexp_operator* op, const pexp_options* opts,
                      const void* y0_dev, const void* G_dev, int g_dtype,
                      void* Y_dev, int y_dtype, pexp_report* rep);

/* Same solve with HOST buffers (y0 FP64 as above): copies y0 and G in, solves, copies Y out. */
int pexp_solve_linear_host(pexp_ctx* ctx, const pexp_operator* op, const pexp_options* opts,
                           const void* y0_host, const void* G_host, int g_dtype,
                           void* Y_host, int y_dtype, pexp_report* rep);

/* Viscous Burgers u_t + u u_x = nu u_xx + f by waveform relaxation (Sec. 2.3-2.4, Fig. 5),
 * plain Picard form (eq. ivp3): A = nu D2 from `op` (its advection velocity must be 0).
 *   u0_dev: n FP64 values.  forcing_dev: optional n_out*n samples f(t_i) or NULL.
 *   init_dev: optional first iterate (n_out*n) or NULL for u0 at every time.
 *   U_dev: n_out*n output, the last iterate (also on PEXP_ERR_WR_NOT_CONVERGED).
 * forcing, init and U have dtype `dtype`. */
int pexp_solve_burgers(pexp_ctx* ctx, const pexp_operator* op, const pexp_options* opts,
                       const void* u0_dev, const void* forcing_dev, const void* init_dev,
                       void* U_dev, int dtype, pexp_report* rep);

/* ---------------------------------------------------------------- batched solves
 * Many independent problems of uneven size (Sec. 2.2's solve per instance).  One problem:
 * an operator, options and caller-owned device buffers, as for pexp_solve_linear. */
typedef struct {
    pexp_operator op;
    pexp_options  opts;
    const void*   y0_dev;   /* n FP64 values */
    const void*   G_dev;    /* n_out*n source samples (time-major, g_dtype) or NULL */
    int           g_dtype;
    void*         Y_dev;    /* n_out*n outputs (time-major, y_dtype) */
    int           y_dtype;
} pexp_problem;

/* Solves `count` problems (probs: host array).  The problems run concurrently on the
 * context's batch workers -- each a private stream and workspace driven by a host thread
 * -- largest first (by n * (n_out + 40 P)); the number of workers is the context's tuned
 * value (pexp_autotune) or 4.  The workers' streams wait for the work queued so far on the
 * context's stream before starting, and the context's stream waits for them at the end.
 * reps: host array of `count` reports or NULL; reps[i].status is problem i's status.
 * Returns PEXP_OK when every problem returned PEXP_OK, else the first other status in
 * problem order; PEXP_ERR_INVALID_ARG (nothing run) when a problem fails validation.
 * The call is synchronous. */
int pexp_solve_batched(pexp_ctx* ctx, int count, const pexp_problem* probs, pexp_report* reps);

/* Tunes the batched solve for this device.  If `path` names a readable table written by
 * this call on a GPU with the same name and SM count, its worker count is loaded;
 * otherwise the given problems are solved with 1, 2, 4, 8 and 16 workers (each once to
 * warm up and once timed), the fastest count is kept in the context, and the table is
 * written to `path` (NULL: not written).  The problems' outputs are overwritten. */
int pexp_autotune(pexp_ctx* ctx, int count, const pexp_problem* probs, const char* path);

/* ---------------------------------------------------------------- kernel-level entry points
 * Single steps of the hot path, exposed for testing and composition.  All
 * pointers are device pointers in FP64 unless a dtype is given. */

/* Y = A X (transpose != 0: Y = A^T X) for `nvec` vectors of length n stored at
 * X + c*n, Y + c*n (Sec. 3.1 stencil).  dtype PEXP_F64 or PEXP_F32. */
int pexp_apply_operator(pexp_ctx* ctx, const pexp_operator* op, const void* X_dev, void* Y_dev,
                        int nvec, int dtype, int transpose);

/* Y = (I - gamma A)^{-1} X for `nvec` vectors (shift-and-invert operator of Sec. 2.1),
 * 1D operators, periodic (constant-coefficient recurrences) or homogeneous Dirichlet (the
 * factored solve of pexp_jacobian_sai_solve); 2D: PEXP_ERR_UNSUPPORTED. */
int pexp_sai_solve(pexp_ctx* ctx, const pexp_operator* op, double gamma, const void* X_dev,
                   void* Y_dev, int nvec, int dtype);

/* Y = (I - gamma (A + J))^{-1} X for `nvec` vectors (Sec. 2.1's shift-and-invert operator for
 * the operator A + J_k of the averaged-Jacobian iteration, Sec. 2.4 eq. ivpSubproblem), 1D
 * operators, periodic or homogeneous Dirichlet.  ubar_dev: n FP64 values, the state at which J
 * is the Jacobian of the conservative Burgers term -(u_{i+1}^2 - u_{i-1}^2)/(4 dx), or NULL for
 * J = 0 (then this is the solve of pexp_sai_solve, by the variable-coefficient kernels).
 * Returns PEXP_ERR_UNSUPPORTED for 2D operators or when I - gamma (A + J) is not diagonally
 * dominant (the factorisation takes no pivots). */
int pexp_jacobian_sai_solve(pexp_ctx* ctx, const pexp_operator* op, double gamma, const double* ubar_dev,
                            const void* X_dev, void* Y_dev, int nvec, int dtype);

/* E_b = exp(M_b) for `batch` dense row-major N x N FP64 matrices, M and E
 * consecutive in memory (Pade-13 scaling and squaring, Higham 2005). N <= 128. */
int pexp_small_expm(pexp_ctx* ctx, const double* M_dev, double* E_dev, int N, int batch);

/* g(t_i) = -u u_x at every row of U (n_out rows of n), conservative (form 0,
 * -(u_{i+1}^2 - u_{i-1}^2)/(4 dx), which conserves the discrete mean) or advective
 * (form 1, -u_i (u_{i+1} - u_{i-1})/(2 dx)) central differences (Sec. 4: the paper
 * does not fix the discretisation of the nonlinear term). */
int pexp_burgers_source(pexp_ctx* ctx, const pexp_operator* op, const void* U_dev, void* G_dev,
                        int n_rows, int dtype, int form);

/* ---------------------------------------------------------------- allocation-free entry point
 * The paper has no counterpart: this is a deployment variant of pexp_sai_solve.
 *
 * Y = (I - gamma A)^{-1} X for `nvec` vectors, computed by the same kernels as
 * pexp_sai_solve, but with no context and no allocation: the call makes no
 * cudaMalloc, cudaFree or other allocating call of CUDA or any library.  It is
 * for callers that cannot allocate device memory at the point of the call:
 *   - code that runs under a fixed device-memory budget whose memory another
 *     allocator (e.g. a framework's caching allocator) has already reserved, so a
 *     cudaMalloc would fail or fragment that pool;
 *   - code on latency-critical streams, where cudaMalloc/cudaFree may synchronise
 *     the whole device and stall the other streams.
 * Its scratch (chunk summaries of the two recurrences and the vector pointer
 * tables) lives in one statically sized device array of PEXP_NOALLOC_SCRATCH_BYTES
 * that every GPU which loads the library holds until the process exits.
 *
 *   op:     1D periodic operator (else PEXP_ERR_UNSUPPORTED); gamma > 0.
 *   X_dev:  nvec input vectors of length n = op->nx at X_dev + k*n (device, read).
 *   Y_dev:  nvec output vectors, same layout (device, written); must not overlap X_dev.
 *   dtype:  PEXP_F64 or PEXP_F32 (the element type of X and Y).
 *   cuda_stream: cudaStream_t of the current device (NULL = legacy default stream).
 * Size limit: 8 * (2*nvec + 4*ceil(n/2048)*nvec) <= PEXP_NOALLOC_SCRATCH_BYTES
 * (n = 2^20: nvec <= 127); larger requests return PEXP_ERR_SCRATCH_LIMIT before any
 * CUDA call.  Invalid arguments return PEXP_ERR_INVALID_ARG; CUDA failures PEXP_ERR_CUDA.
 *
 * The call runs on the calling thread's current device and is asynchronous: it
 * returns once its kernels are enqueued on cuda_stream; the caller synchronises.
 * The first call on a device also looks up the device address of the scratch array
 * (once per device, thread-safe); make that first call before any stream capture
 * begins.  Under CUDA's lazy module loading (the default), that first call is also
 * when the driver loads the library's device code on the device, and with it the
 * scratch array: device memory is taken then, once, and a first call made after the
 * caller's budget is fully reserved can fail with PEXP_ERR_CUDA.  A caller under a fixed
 * budget makes one call (any valid size) before reserving it; later calls take no
 * device memory.  Every call, on any stream, shares the one array, which keeps the last
 * call's contents; nothing in it needs to start at zero (each call writes every
 * entry it reads).  Calls that overlap on the GPU (concurrent streams, or calls from
 * several threads without ordering) race on the scratch and give wrong results. */
#define PEXP_NOALLOC_SCRATCH_BYTES (2u << 20)
int pexp_sai_solve_noalloc(const pexp_operator* op, double gamma, const void* X_dev, void* Y_dev,
                           int nvec, int dtype, void* cuda_stream);

/* Self-test of the bounded wait of the grid barriers that the cooperative launches use
 * (no counterpart in the paper; it checks this library's own synchronisation).  Launches a
 * small cooperative grid on the context's stream whose CTAs pass four barriers; with
 * absent_cta >= 0 that CTA leaves at once, so the others' wait expires after about 1 s.
 * Blocks until the launch ends.  Returns PEXP_OK when every barrier completed,
 * PEXP_ERR_TIMEOUT when a wait expired (the barrier words are then reset and the context
 * stays usable), PEXP_ERR_UNSUPPORTED where a cooperative launch is not possible. */
int pexp_selftest_barrier(pexp_ctx* ctx, int absent_cta);

#ifdef __cplusplus
}
#endif
#endif /* PEXP_H */
