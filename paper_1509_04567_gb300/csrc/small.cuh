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
    int64_t off_yk;    // 2 x K_max         projected state at two knots (Chebyshev samples)
    int istride;
};

// int fields
// WI_S: source samples of a source window (output times of a homogeneous one); WI_SOUT: output
// times of a source window whose samples are not its output times (0: the same as WI_S);
// WI_CHEB: the source samples are the window's Chebyshev points (knots of the spline).
enum { WI_B = 0, WI_CONV, WI_STEPS, WI_S, WI_KIND, WI_KEPT, WI_STATUS, WI_K, WI_I0, WI_SOUT, WI_CHEB, WI_COUNT = 16 };
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

// Cholesky QR with diagonal pivoting and deflation of one new Krylov block (k_block_orth):
//   pass 1: Gram G of W after Gram-Schmidt; columns whose remaining norm is below
//           defl * (largest column norm of W before Gram-Schmidt) are dropped;
//           T maps W to the kept orthonormal directions (columns 0..r-1), the rest 0.
//   pass 2: re-orthonormalise the kept columns (Cholesky of their Gram).
// Entered by warp 0 of the calling CTA (all lanes: the Gram may be summed from the chunk
// partials gp of launch-list entry `task`); thread 0 factors, writes T (b x b, column-major)
// to Tout and returns the kept count r (other threads return 0).  `kept`: pass 2's
// candidate count (< 0: the window's WI_KEPT).  `owner`: also write the window's state (the
// pre-Gram-Schmidt norm, WI_KEPT, and WI_CONV when the block is empty).  sG: b*b shared doubles.
// pp (pass 1): the pre-Gram-Schmidt norms summed from the projection pass's partials (entries
// pre_off + c of launch-list entry `task`) into spre (b shared doubles) instead of read from
// the window's state.
// BM: the largest block width b the caller passes (sizes the factorisation's local arrays).
template <int BM = PEXP_MAX_RANK>
__device__ __forceinline__ int block_orth_body(const WinLayout& L, double* D, int* I, int task, int pass, int step,
                                               double defl, Parts gp, int kept, double* sG, double* Tout, bool owner,
                                               Parts pp = Parts{nullptr, 0, 0}, int pre_off = 0,
                                               double* spre = nullptr) {
    const int b = I[WI_B];
    if (gp.part) {
        for (int e = 0; e < b * b; ++e) {
            const double v = parts_sum_warp(gp, task, e);
            if (threadIdx.x == 0) sG[e] = v;
        }
    }
    if (pass == 1 && pp.part) {
        for (int c = 0; c < b; ++c) {
            const double v = parts_sum_warp(pp, task, pre_off + c);
            if (threadIdx.x == 0) spre[c] = v;
        }
    }
    __syncwarp();
    if (threadIdx.x != 0) return 0;
    const double* G0 = D + L.off_gw;
    double G[BM * BM], R[BM * BM];
    int perm[BM];
    for (int e = 0; e < b * b; ++e) {
        G[e] = gp.part ? sG[e] : G0[e];
        R[e] = 0.0;
    }
    for (int k = 0; k < b; ++k) perm[k] = k;
    double lim2;
    int ncand = b;
    if (pass == 1) {
        // pre-Gram-Schmidt norms: diagonal of W^T W stored in out1 rows [step*b, step*b+b),
        // in the last column block (fused path: b values after h1 at out1)
        const int ldo = (step + 1) * b;
        const double* o1 = D + L.off_out1;
        const int wc = (L.ycols - 1) * b;
        double pre = 0.0;
        for (int c = 0; c < b; ++c)
            pre = fmax(pre, pp.part ? spre[c] : gp.part ? o1[step * b * b + c] : o1[(step * b + c) + (wc + c) * ldo]);
        lim2 = defl * defl * pre;
        if (owner) D[L.off_scal + WS_PRE] = sqrt(pre);
    } else {
        lim2 = 0.25;  // kept columns have unit norm after pass 1, dropped ones are zero
        ncand = kept >= 0 ? kept : I[WI_KEPT];
    }
    int r = 0;
    for (int k = 0; k < ncand; ++k) {
        int j = k;
        if (pass == 1) {
            for (int l = k + 1; l < b; ++l)
                if (G[l + l * b] > G[j + j * b]) j = l;
        }
        if (!(G[j + j * b] > lim2)) break;
        if (j != k) {  // symmetric swap of rows/cols k and j, and of the R columns
            for (int l = 0; l < b; ++l) { double t = G[k + l * b]; G[k + l * b] = G[j + l * b]; G[j + l * b] = t; }
            for (int l = 0; l < b; ++l) { double t = G[l + k * b]; G[l + k * b] = G[l + j * b]; G[l + j * b] = t; }
            for (int l = 0; l < k; ++l) { double t = R[l + k * b]; R[l + k * b] = R[l + j * b]; R[l + j * b] = t; }
            int t = perm[k]; perm[k] = perm[j]; perm[j] = t;
        }
        const double rkk = sqrt(G[k + k * b]);
        R[k + k * b] = rkk;
        for (int l = k + 1; l < b; ++l) R[k + l * b] = G[k + l * b] / rkk;
        for (int l = k + 1; l < b; ++l)
            for (int l2 = k + 1; l2 < b; ++l2) G[l + l2 * b] -= R[k + l * b] * R[k + l2 * b];
        ++r;
    }
    // T = P[:, 0:r] R[0:r, 0:r]^{-1}
    double Ri[BM * BM];
    for (int e = 0; e < b * b; ++e) Ri[e] = 0.0;
    for (int j = 0; j < r; ++j) {
        Ri[j + j * b] = 1.0 / R[j + j * b];
        for (int i = j - 1; i >= 0; --i) {
            double v = 0.0;
            for (int k = i + 1; k <= j; ++k) v += R[i + k * b] * Ri[k + j * b];
            Ri[i + j * b] = -v / R[i + i * b];
        }
    }
    double* T = Tout;
    for (int e = 0; e < b * b; ++e) T[e] = 0.0;
    for (int k = 0; k < r; ++k)
        for (int j = 0; j <= k; ++j) T[perm[j] + k * b] = Ri[j + k * b];
    if (pass == 1 && owner) {
        I[WI_KEPT] = r;
        if (r == 0) I[WI_CONV] = 1;  // invariant subspace reached: the projection is exact
    }
    return r;
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
// h: the output spacing; a window with WI_CHEB set takes its knots at its Chebyshev points
// (WI_S of them over (WI_SOUT - 1) h), otherwise at the multiples of h.
void launch_spline(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, double h, cudaStream_t s);
// With fused partials (E, F, h1, pre of the step) and the operator coefficients d, c:
// H[a, i] = -d E - c F, H[i, a] = -d E + c F; h1 and pre are stored at out1.
// b_launch: largest block width among the windows (0: unknown, the matrices stay in global memory
// unless the layout's largest matrix fits in shared memory)
// only_ef != 0 (fused partials): h1 and pre are left to another kernel.
// jcoef != 0 (fused partials): the partials also hold the Jacobian sums Ja, Jb of
// launch_step_proj, and H gets jcoef * Ja in its new column and jcoef * Jb in its new row
// (jcoef = 1/(2 dx): the Jacobian of the conservative Burgers term).
// rc0, rc0p (dense projections only): first blocks of the current and the previous restart
// cycle; the new block's H entries outside its cycle are set to 0, except the row of a cycle's
// first block over the previous cycle (0, 0: no restarts).
void launch_project(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, int step, double h,
                    double tol, double scale_ref, cudaStream_t s, Parts fp = Parts{nullptr, 0, 0}, double d = 0.0,
                    double cadv = 0.0, int b_launch = 0, int only_ef = 0, double jcoef = 0.0, int rc0 = 0,
                    int rc0p = 0);
void launch_small_expm_batch(const double* M, double* E, int N, int batch, double* scratch, cudaStream_t s);
size_t small_expm_scratch_doubles(int N);
void init_pade_constants();

}  // namespace pexp
