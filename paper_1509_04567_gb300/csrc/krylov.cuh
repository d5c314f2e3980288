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
};

// W <- W - V h (mode 0/1) or W <- W T (scale).  h/T come either from a dense
// FP64 matrix (hm, ld ldh) or, when hpart != NULL, from the sum over `hchunks`
// partial results of the previous kernel (stride hstride, offset hoff per chunk).
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
    const double* hpart;
    int hchunks, hstride;
};

struct KGeom {
    int nchunks;
    int64_t rows;
};
KGeom krylov_geom(int ntasks, int64_t n);
size_t krylov_partial_doubles(int ntasks, int p_max, int b_max, int64_t n);
size_t krylov_update_smem(int p_max, int b, size_t tsize);

// All launchers take the row-chunk geometry g (the same for every task of a step) and
// write the partials of task k at partial + (k * g.nchunks + chunk) * pstride.
// partial layout of k_step_proj per (task, chunk): E (p x b) | F (p x b) | h1 (p x b) | pre (b)
template <typename T>
void launch_step_proj(const StepTask<T>* tasks, int ntasks, int b, int64_t n, int periodic, KGeom g,
                      double* partial, int pstride, cudaStream_t s);
// mode 0: W -= V h, partial h2 = V^T W (p x b);  mode 1: W -= V h, partial G = W^T W (b x b)
template <typename T>
void launch_update(const UpdTask<T>* tasks, int ntasks, int b, int p_max, int64_t n, int mode, KGeom g,
                   double* partial, int pstride, cudaStream_t s);
// W <- W T; gram != 0: partial G = W^T W; task.out != NULL: result rounded into task.out
template <typename T>
void launch_scale(const UpdTask<T>* tasks, int ntasks, int b, int64_t n, int gram, KGeom g, double* partial,
                  int pstride, cudaStream_t s);
constexpr int kKrylovMaxB = 4;   // block widths handled by the fused kernels
// Gram matrices of the source windows: X[k] points at the first of sv[k] (<= 31)
// consecutive length-n vectors; partial (chunk) results s x s, both halves.
template <typename T>
void launch_source_gram(const T* const* X, const int* sv, int ntasks, int s_max, int64_t n, KGeom g, double* partial,
                        int pstride, cudaStream_t st);

}  // namespace pexp
