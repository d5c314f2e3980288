// Shared declarations of the PEBK CUDA library (sm_103a).
//
// Translation units:
//   tall.cu   -- kernels over n-length data: central-difference stencil,
//                shift-and-invert solve, batched tall-skinny products,
//                reconstruction, Burgers source, conversions;
//   small.cu  -- per-subinterval kernels on small FP64 matrices: source SVD by
//                Jacobi, block orthonormalisation (pivoted Cholesky), cubic
//                coefficient model, Pade exponential, projected time stepping;
//   solver.cu -- host orchestration and the C ABI of include/pexp.h.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pexp.h"

namespace pexp {

constexpr int kNumSM = 152;  // GB300: 2 dies x 76 SMs

// One dimension of the central-difference operator (Sec. 3.1):
//   (A u)_i += d ((u_{i-1} - u_i) + (u_{i+1} - u_i)) - c (u_{i+1} - u_{i-1}),
// d = nu/dx^2, c = a/(2 dx).  The difference form keeps the rounding error
// relative to the (small) result for smooth data.
struct Dim1 {
    int64_t n;       // points in this dimension
    int64_t stride;  // element stride between neighbours in this dimension
    double d, c;
    int periodic;
};

struct OpDesc {
    int dim;
    int64_t n;   // total unknowns
    Dim1 x, y;
};

// One task of a batched tall-skinny product over rows 0..n-1.
//   TN:  out (p x q, column-major, ld p) = X'^T Y'
//   NN:  Z (n x q) = alpha X' Tm + beta Z          (Tm p x q, column-major, ld ldt)
// X' = X + xs 1^T (xs optional, FP64), Y' = [Y(:, 0:q1) | Y2(:, 0:q-q1)] + ys 1^T.
// All tall arrays column-major with leading dimensions in elements.
// NN may run in place (Z == X, p == q <= 16).
template <typename T>
struct TsTask {
    const T* X;
    const T* Y;
    const T* Y2;
    T* Z;
    const double* Tm;
    const double* xs;
    const double* ys;
    double* out;
    int64_t ldx, ldy, ldy2, ldz;
    int p, q, q1, ldt;
    double alpha, beta;
};

// Double-float update task for FP32 data (see k_ts_nn_df):
//   Z = alpha (X + xs 1^T) Tm [+ Z], X and Z given as (hi, lo) FP32 array pairs;
//   the low array of X covers its first pl columns (pl = 0: all p columns).
struct DfTask {
    const float* Xh;
    const float* Xl;
    int pl;
    const double* xs;
    int64_t ldx;
    float* Zh;
    float* Zl;
    int64_t ldz;
    const double* Tm;
    int ldt, p, q, accumulate;
    double alpha;
};

// Reconstruction task: for output rows r = 0..ns-1 (coefficient rows r0 + r),
//   Out[(i0 + r) * ldo + k] = u0[k] + sum_a V1[a*ld1 + k] C1[(r0+r)*ldc1 + a]
//                                   + sum_a V2[a*ld2 + k] C2[(r0+r)*ldc2 + a]
// with u0 optional; K1 or K2 may be zero.
template <typename T>
struct ReconTask {
    const T* V1; const double* C1; int64_t ld1; int K1, ldc1;
    const T* V2; const double* C2; int64_t ld2; int K2, ldc2;
    int r0, ns;
    int64_t i0;
};

// Grid barrier words of cooperative launches (grid_bar below).
struct GridBar {
    unsigned* count;
    unsigned* gen;
    int* err;
};

struct SaiCoef {
    double alpha, beta, inv_c;   // (I - gamma A) = c (I - alpha S^{-1})(I - beta S)
    double alpha_n, beta_n;      // alpha^n, beta^n (circular closure)
};

// Factors of a tridiagonal shift-and-invert matrix with coefficients that vary along x:
//   (I - gamma A_w) = (I - diag(lam) S^{-1}) diag(d) (I - diag(mu) S),  S the cyclic shift,
// so (I - gamma A_w)^{-1} x is two first-order recurrences, y_i = x_i + lam_i y_{i-1} and
// z_i = y_i / d_i, x_i = z_i + mu_i x_{i+1}.  Bounded (homogeneous Dirichlet) meshes have
// lam_0 = mu_{n-1} = 0: the recurrences do not wrap around.  Arrays of n FP64 values.
struct VarSai {
    const double* lam;
    const double* mu;
    const double* dinv;
};

// A window's tridiagonal operator for the variable-coefficient solve: the 1D
// central-difference operator plus, when ubar != NULL, the Jacobian of the conservative
// Burgers term -(u_{i+1}^2 - u_{i-1}^2)/(4 dx) at the state ubar:
//   (J v)_i = -(ubar_{i+1} v_{i+1} - ubar_{i-1} v_{i-1}) / (2 dx)   (Sec. 2.3, eq. jacobian)
struct VarOpTask {
    const double* ubar;   // n values or NULL (A alone)
    double* lam;          // outputs: factors of (I - gamma A_w), n values each
    double* mu;
    double* dinv;
    int* flag;            // set to 1 when a row of (I - gamma A_w) is not diagonally dominant
};

// ---------------------------------------------------------------- vsai.cu
// Factors of (I - gamma (A + J(ubar_w))) for every task: each thread runs the diagonal
// recurrence d_i = b_i - a_i c_{i-1} / d_{i-1} over its chunk after `warm` steps of
// warm-up from the left (the recurrence contracts towards its periodic solution; bounded
// meshes start exactly at i = 0).
void launch_vsai_factor(const Dim1& x, double gamma, double inv2dx, const VarOpTask* tasks_dev, int ntasks,
                        int64_t warm, cudaStream_t s);
// Warm-up length that takes the diagonal recurrence to its limit to rounding: the
// contraction per step is about 1 - 2/sqrt(g), g = gamma * (largest off-diagonal of A_w).
int64_t vsai_warmup(const Dim1& x, double gamma, double inv2dx, double umax);
// Y = (I - gamma A_w)^{-1} X for nvec vectors, vector v with the factors coef[v] (device
// array).  Same layout, low parts and skip flags as launch_sai_solve_lo.
template <typename T>
void launch_vsai_solve(int64_t n, const VarSai* coef, const T* const* X, const T* const* Xlo, T* const* Y,
                       T* const* Ylo, int nvec, double* scratch, cudaStream_t s, const int* const* skip = nullptr);
// Time average of the iterate over each subinterval by the trapezoidal rule on its
// samples (eq. piecewiseJac): ubar_j = mean of U rows idx_j .. idx_{j+1} with half weights
// at both ends.  Writes FP64 (P x n) and T copies; umax_bits[j] (zeroed by the caller)
// receives max_k |ubar_j[k]| as the bits of a non-negative double.
template <typename T>
void launch_window_average(const T* U, int64_t n, const int* idx_dev, int P, double* ubar64, T* ubarT,
                           unsigned long long* umax_bits, cudaStream_t s);
// Shifted source of the averaged-Jacobian iteration on each subinterval (eq. sourceParallel
// read as A u0 + g_k - J_j (u_k - u0)): row r of the window-major output holds window
// rw[r]'s sample at output time ri[r]:  out_r = Au0 + G[ri] - J(ubar_{rw}) (U[ri] - u0).
template <typename T>
void launch_jac_source(const Dim1& x, double inv2dx, const double* Au0, const double* u0, const T* G, const T* U,
                       const double* ubar64, const int* rw, const int* ri, int nrows, T* out, cudaStream_t s);

// Y += J X (transpose != 0: J^T X), J the Jacobian of the conservative Burgers term at the
// per-vector state U[v] (FP64, n values); for FP32 data X may carry low parts Xlo and Y is
// kept as a (Yh, Yl) pair (Yl may be NULL for FP64 data).
template <typename T>
void launch_jac_add(int64_t n, int periodic, double inv2dx, const double* const* U, const T* const* X,
                    const float* const* Xlo, T* const* Yh, T* const* Yl, int nvec, int transpose, cudaStream_t s);

// ---------------------------------------------------------------- tall.cu
SaiCoef sai_coefficients(const OpDesc& op, double gamma);
size_t sai_scratch_doubles(int64_t n, int nvec);
size_t ts_tn_partial_doubles(int ntasks, int max_pq, int64_t n);

template <typename T>
void launch_stencil(const OpDesc& op, const T* X, T* Y, int nvec, int transpose, cudaStream_t s);
template <typename T>
void launch_stencil_ptrs(const OpDesc& op, const T* const* X, T* const* Y, int nvec, int transpose,
                         cudaStream_t s);
void launch_stencil_df(const OpDesc& op, const float* const* X, const float* const* Xl, float* const* Yh,
                       float* const* Yl, int nvec, int transpose, cudaStream_t s);
template <typename T>
void launch_burgers_source(const OpDesc& op, const T* U, T* G, int nrows, int form, double inv2dx,
                           cudaStream_t s);
template <typename T>
void launch_sai_solve(const OpDesc& op, const SaiCoef& cf, const T* const* X, T* const* Y, T* const* Ylo, int nvec,
                      double* scratch, cudaStream_t s);
// Same with input low parts (FP32 data: X + Xlo is a double-float input; NULL = none) and
// optional per-vector skip flags (vector v is left untouched while *skip[v] != 0).
template <typename T>
void launch_sai_solve_lo(const OpDesc& op, const SaiCoef& cf, const T* const* X, const T* const* Xlo, T* const* Y,
                         T* const* Ylo, int nvec, double* scratch, cudaStream_t s, const int* const* skip = nullptr);
// The three passes of the solve of one vector (x: no low part) in one cooperative launch
// with grid barriers between them; the same arithmetic as launch_sai_solve_lo, so the same
// result.  Returns false (nothing launched) where a cooperative launch is not possible.
template <typename T>
bool launch_sai_coop(const OpDesc& op, const SaiCoef& cf, const T* x, T* y, T* ylo, double* scratch, const int* skip,
                     GridBar bar, cudaStream_t s);
// Largest grid (at most `want`) whose CTAs are all resident at once, 0 without cooperative launch.
int coop_grid(const void* kernel, int threads, size_t smem, int want);
// Cooperative launch of up to 64 CTAs passing 4 barriers; CTA `absent` (>= 0) skips them.
// Returns the grid size, 0 where a cooperative launch is not possible.
int launch_bar_selftest(GridBar bar, int absent, cudaStream_t s);
template <typename T>
void launch_ts_tn(const TsTask<T>* tasks_dev, int ntasks, int max_pq, int max_q, int64_t n, double* partial,
                  cudaStream_t s, int exact = 0);
template <typename T>
void launch_ts_nn(const TsTask<T>* tasks_dev, int ntasks, int max_pq, int64_t n, cudaStream_t s);
// max_ns: most samples of a task; max_k: most basis columns (K1 + K2) of a task
template <typename T, typename TO>
void launch_recon(const ReconTask<T>* tasks_dev, int ntasks, int max_ns, int64_t n, const double* u0,
                  TO* out, int64_t ldo, int max_k, cudaStream_t s);
template <typename TI, typename TO>
void launch_convert(const TI* x, TO* y, int64_t count, cudaStream_t s);
// rows of A minus rows of B: partial[row] = ||A_row - B_row||^2, partial[nrows + row] = ||A_row||^2
template <typename T>
void launch_row_diff_norms(const T* A, const T* B, int64_t n, int nrows, double* out, cudaStream_t s);

template <typename T>
void launch_add(T* y, const T* x, int64_t count, cudaStream_t s);
// max_q: most block columns q of any task (<= 16); q <= 4 takes a two-row kernel
void launch_ts_nn_df(const DfTask* tasks_dev, int ntasks, int max_pq, int64_t n, cudaStream_t s, int max_q = 16);
template <typename T>
// split: 2n floats of scratch (FP32 data: u as a double-float pair)
void launch_row_dots(const double* u, const T* G, int64_t n, int nrows, double* out, float* split, cudaStream_t s);

int fail_cuda(cudaError_t e, const char* what, const char* file, int line);

// Raises a kernel's dynamic shared-memory limit on the current device to at least `bytes`.
// The limit is a process-wide attribute of the kernel: it is only ever raised, under a lock,
// so that launches from several host threads (batched solves) never find it lowered by
// another thread that needed less.
void smem_optin_raw(const void* kernel, size_t bytes);
template <typename K>
inline void smem_optin(K* kernel, size_t bytes) {
    smem_optin_raw(reinterpret_cast<const void*>(kernel), bytes);
}

// Programmatic dependent launch for the kernels of a Krylov step, which run back to back
// on one stream.  Such a kernel is launched with programmatic stream serialization, so
// its launch may overlap the kernel before it; it calls pdl_entry() before its first
// memory access: griddepcontrol.wait returns once the grids it depends on have completed
// and their writes are visible (at once when it was launched without the attribute), then
// griddepcontrol.launch_dependents lets the next kernel of the stream be launched.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Grid-wide barrier for kernels launched cooperatively (every CTA resident at once):
// an arrival counter and a generation word in global memory, shared by the launches of one
// stream.  The wait is bounded: a CTA that sees no progress for 1 s sets *err and stops
// waiting, and once *err is set every CTA skips the remaining barriers (and its callers the
// remaining work), so a launch always ends.  The host resets the three words after an error.
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Returns false (in every thread of the CTA) once the barrier has failed.
__device__ __forceinline__ bool grid_bar(const GridBar& g) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* vgen = g.gen;
        volatile int* verr = g.err;
        int ok = *verr == 0;
        if (ok) {
            const unsigned my = *vgen;
            __threadfence();
            const unsigned nb = gridDim.x * gridDim.y * gridDim.z;
            if (atomicAdd(g.count, 1u) == nb - 1) {
                atomicExch(g.count, 0u);
                __threadfence();
                atomicAdd(g.gen, 1u);
            } else {
                const unsigned long long t0 = global_ns();
                while (*vgen == my && *verr == 0) {
                    if (global_ns() - t0 > 1000000000ull) {
                        atomicExch(g.err, 1);
                        break;
                    }
                    __nanosleep(64);
                }
            }
            __threadfence();
            ok = *verr == 0;
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args&&... args) {
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kernel, static_cast<Args&&>(args)...);
}

}  // namespace pexp

#define PEXP_CUDA_TRY(expr)                                                                \
    do {                                                                                   \
        cudaError_t _e = (expr);                                                           \
        if (_e != cudaSuccess) return ::pexp::fail_cuda(_e, #expr, __FILE__, __LINE__);    \
    } while (0)
