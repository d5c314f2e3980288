// Per-subinterval ("window") small-matrix state and kernels of the PEBK solver.
#pragma once

#include "common.cuh"

namespace pexp {

// Layout of the FP64 per-window buffer (one slab of `stride` doubles per window)
// and of the int per-window buffer.  Matrices are column-major.
struct WinLayout {
    int s_max;     // samples per window
    int b_max;     // block width
    int K_max;     // basis columns = b_max * (kmax + 1)
    int N_max;     // augmented matrix size = K_max + 4 b_max
    int ycols;     // column blocks of the step projections: 3 (A V, A^T V, W) or 5 with low parts
    int64_t stride;
    int64_t off_gram;  // s_max x s_max     Gram of the source samples
    int64_t off_zs;    // s_max x b_max     U = Ghat zs
    int64_t off_C;     // b_max x s_max     coefficient samples (ld b_max)
    int64_t off_coef;  // (s_max-1) x 4 x b_max cubic coefficients [(r*4+l)*b_max + k]
    int64_t off_H;     // K_max x K_max     Galerkin matrix V^T A V
    int64_t off_out1;  // (K_max + b_max) x ycols b_max   projections of step i
    int64_t off_h2;    // K_max x b_max     second Gram-Schmidt pass
    int64_t off_gw;    // b_max x b_max     Gram of the new block
    int64_t off_T;     // b_max x b_max     block scaling
    int64_t off_Y;     // s_max x K_max     projected solution at the samples, row r at r*K_max
    int64_t off_Yp;    // s_max x K_max     previous step's projected solution
    int64_t off_scal;  // 16 scalars
    int64_t off_scr;   // 9 N_max^2 scratch (augmented matrix, exponential, Pade work)
    int istride;
};

// int fields
enum { WI_B = 0, WI_CONV, WI_STEPS, WI_S, WI_KIND, WI_KEPT, WI_STATUS, WI_K, WI_I0, WI_COUNT = 16 };
// double scalars at off_scal
enum { WS_BETA = 0, WS_EST, WS_SCALE, WS_SIGRATIO, WS_H, WS_PRE, WS_COUNT = 16 };

enum { KIND_SOURCE = 0, KIND_HOM = 1 };

WinLayout make_layout(int s_max, int b_max, int kmax, int ycols = 3);

// Partial sums of the fused Krylov kernels: window k of the launch list owns chunks
// [k*nchunks, (k+1)*nchunks) of `part`, `pstride` doubles each (NULL: dense inputs).
struct Parts {
    const double* part;
    int nchunks, pstride;
};

// Sum of entry e over the chunks of task `task`, computed by one warp (all lanes get it):
// lanes take chunks lane, lane+32, ... and the lane sums meet in a fixed shuffle tree.
__device__ __forceinline__ double parts_sum_warp(const Parts& p, int task, int e) {
    const int lane = threadIdx.x & 31;
    const double* base = p.part + (size_t)task * p.nchunks * p.pstride + e;
    double s = 0.0;
#pragma unroll 4
    for (int c = lane; c < p.nchunks; c += 32) s += base[(size_t)c * p.pstride];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    return s;
}

// Launchers.  `wins` is a device array of window indices (nw entries).
// The Gram matrix of the shifted samples G_hat = A u0 1^T + G is assembled from its
// parts: off_gram holds G^T G, dots[i] = (A u0) . g(t_i) (NULL: no source),
// *nrm2 = ||A u0||^2.
void launch_source_eig(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, double thr,
                       int max_rank, const double* dots, const double* nrm2, cudaStream_t s,
                       Parts gp = Parts{nullptr, 0, 0});
void launch_start_orth(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, cudaStream_t s);
void launch_block_orth(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, int pass, int step,
                       double defl, cudaStream_t s, Parts gp = Parts{nullptr, 0, 0});
void launch_spline(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, double h, cudaStream_t s);
// With fused partials (E, F, h1, pre of the step) and the operator coefficients d, c:
// H[a, i] = -d E - c F, H[i, a] = -d E + c F; h1 and pre are stored at out1.
// b_launch: largest block width among the windows (0: unknown, the matrices stay in global memory
// unless the layout's largest matrix fits in shared memory)
// only_ef != 0 (fused partials): h1 and pre are left to another kernel.
// jcoef != 0 (fused partials): the partials also hold the Jacobian sums Ja, Jb of
// launch_step_proj, and H gets jcoef * Ja in its new column and jcoef * Jb in its new row
// (jcoef = 1/(2 dx): the Jacobian of the conservative Burgers term).
void launch_project(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, int step, double h,
                    double tol, double scale_ref, cudaStream_t s, Parts fp = Parts{nullptr, 0, 0}, double d = 0.0,
                    double cadv = 0.0, int b_launch = 0, int only_ef = 0, double jcoef = 0.0);
void launch_small_expm_batch(const double* M, double* E, int N, int batch, double* scratch, cudaStream_t s);
size_t small_expm_scratch_doubles(int N);
void init_pade_constants();

}  // namespace pexp
