// Fused kernels of one block Krylov step for 1D operators (see krylov.cu).
#pragma once

#include "common.cuh"

namespace pexp {

// V: basis of one window, column-major, leading dimension ld; columns [0, p) hold
// V_{1:i}; the working block W occupies columns [p, p + b) (FP32 data: its low
// parts are in Wl, same layout).
template <typename T>
struct StepTask {
    const T* V;
    int64_t ld;
    int p;
    const int* conv;  // the window's convergence flag: the kernels skip a converged window (NULL: never)
    const T* ubar;    // Jacobian launches: the state of the window's Burgers Jacobian (n values)
};

// W <- W - V h (mode 0/1) or W <- W T (scale), h/T a dense FP64 matrix (hm, ld ldh).
template <typename T>
struct UpdTask {
    const T* V;       // V_{1:i} (mode 0/1); unused by the scale kernel
    T* Wh;            // working block (hi)
    float* Wl;        // FP32 data: low parts; NULL for FP64
    T* out;           // scale kernel, final pass: destination of the rounded block (else NULL)
    int64_t ld;
    int p;
    const double* hm;
    int ldh;
    const int* conv;  // the window's convergence flag: the kernels skip a converged window (NULL: never)
};

struct KGeom {
    int nchunks;
    int64_t rows;
};
KGeom krylov_geom(int ntasks, int64_t n);
// upper bound of ntasks * krylov_geom(ntasks, n).nchunks over ntasks <= ntasks_max
size_t krylov_partial_slots(int ntasks_max, int64_t n);

// All launchers take the row-chunk geometry g (the same for every task of a step) and
// write the partials of task k at partial + (k * g.nchunks + chunk) * pstride.
// partial layout of k_step_proj per (task, chunk): E (p x b) | F (p x b) | h1 (p x b) | pre (b)
// and, with jac, Ja (p x b) | Jb (p x b) after them:
//   Ja[a, i] = sum_r ubar_r v_i,r (v_a,r+1 - v_a,r-1),  Jb[a, i] = sum_r ubar_r v_a,r (v_i,r+1 - v_i,r-1),
// so that v_a^T J v_i = Ja / (2 dx) and v_i^T J v_a = Jb / (2 dx) for the Jacobian J of the
// conservative Burgers term at ubar (summation by parts, zero ghosts on bounded meshes).
// p = columns of V_{1:i} (the same for every task of the launch)
template <typename T>
void launch_step_proj(const StepTask<T>* tasks, int ntasks, int b, int p, int64_t n, int periodic, KGeom g,
                      double* partial, int pstride, cudaStream_t s, bool jac = false);
// mode 0 and 1: W -= V h (h = tk.hm, p x b), partial G = W^T W (b x b); mode 0 subtracts
// in double-float (FP32 data), mode 1 with FP32 products (second-pass coefficients).
// Mode 1 with hpart: h is summed by each CTA from the chunk partials at hpart (task-major,
// stride hstride, g.nchunks chunks) instead of read from tk.hm; `partial` must not overlap them.
template <typename T>
void launch_update(const UpdTask<T>* tasks, int ntasks, int b, int p_max, int64_t n, int mode, KGeom g,
                   double* partial, int pstride, cudaStream_t s, const double* hpart = nullptr, int hstride = 0);
// W <- W T (T = tk.hm, b x b) and partial h = V^T W (p x b) of the result
template <typename T>
void launch_scale_proj(const UpdTask<T>* tasks, int ntasks, int b, int p, int64_t n, KGeom g, double* partial,
                       int pstride, cudaStream_t s);
// partial G = X^T X (b x b, b = task.p <= 4) of the block X = task.Wh
template <typename T>
void launch_block_gram(const UpdTask<T>* tasks, int ntasks, int64_t n, KGeom g, double* partial, int pstride,
                       cudaStream_t s);
// W <- W T; gram != 0: partial G = W^T W; task.out != NULL: result rounded into task.out
template <typename T>
void launch_scale(const UpdTask<T>* tasks, int ntasks, int b, int64_t n, int gram, KGeom g, double* partial,
                  int pstride, cudaStream_t s);
struct WinLayout;
// The scale and second projection pass fuse into one kernel (k_scale_proj) for a basis of p
// columns and block width b with elements of tsize bytes.
bool proj_fused(int p, int b, size_t tsize);
// Part B of a fused Krylov step (passes u[0..3]: update0, scale_proj, update1, scale, with the
// two Cholesky QRs between them) for window w, block width b, in one cooperative launch:
// the same arithmetic and results as the separate launches.  The partial sums take
// g.nchunks * (2 psg + ps2) doubles of kp.  Returns false (nothing launched) for b != 1,
// an unfused width p, or where a cooperative launch is not possible.
template <typename T>
bool launch_gs_coop(const UpdTask<T>* u, int b, int p, int64_t n, KGeom g, double* kp, int ps2, int psg,
                    const WinLayout& L, double* wd, int* wi, int w, int step, double defl, GridBar bar, cudaStream_t s);
// Part B of a fused step with the partial-sum and Cholesky-QR kernels folded into the passes
// (bitwise the same results as update + sum + block_orth + scale_proj + ... launched apart):
// update0 summing h1 from the projection partials (entries hoff + [0, p b)); scale_proj after
// the first QR (Gram partials gpart, pre-Gram-Schmidt norms at entry pre_off of the projection
// partials ppart); scale after the second QR.  wins: the window of each task.
template <typename T>
void launch_update0_h(const UpdTask<T>* tasks, int ntasks, int b, int p, int64_t n, KGeom g, double* partial,
                      int pstride, const double* hpart, int hstride, int hoff, cudaStream_t s);
template <typename T>
void launch_scale_proj_qr(const UpdTask<T>* tasks, int ntasks, int b, int64_t n, KGeom g, double* partial, int pstride,
                          const WinLayout& L, double* wd, int* wi, const int* wins, int step, double defl,
                          const double* gpart, int gstride, const double* ppart, int ppstride, int pre_off,
                          cudaStream_t s);
template <typename T>
void launch_scale_qr(const UpdTask<T>* tasks, int ntasks, int b, int64_t n, KGeom g, const WinLayout& L, double* wd,
                     int* wi, const int* wins, int step, double defl, const double* gpart, int gstride, cudaStream_t s);
constexpr int kKrylovMaxB = 4;   // block widths handled by the fused kernels
// Sums the per-CTA partials of each task into wd + wins[task] * stride + off (ne entries).
// Entries [e0, e0 + ne) of each partial go to entries [0, ne) of the output.
// Windows whose flag wi[w * istride + conv_field] is set are skipped.
void launch_sum_parts(const double* part, int nchunks, int pstride, int ne, double* wd, int64_t stride, int64_t off,
                      const int* wins, int ntasks, const int* wi, int istride, int conv_field, cudaStream_t s,
                      int e0 = 0);
// Gram matrices of the source windows: X[k] points at the first of sv[k] (<= 31)
// consecutive length-n vectors; partial (chunk) results s x s, both halves.
template <typename T>
void launch_source_gram(const T* const* X, const int* sv, int ntasks, int s_max, int64_t n, KGeom g, double* partial,
                        int pstride, cudaStream_t st);

}  // namespace pexp
