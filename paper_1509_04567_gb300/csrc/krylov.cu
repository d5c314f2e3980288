// Fused tall-skinny kernels of one block Krylov step (1D operators), sm_103a.
//
// The Galerkin matrix H = V^T A V of the central-difference operator is formed
// by summation by parts: for (A v)_r = d (v_{r-1} - 2 v_r + v_{r+1})
//                                      - c (v_{r+1} - v_{r-1}),
//   v_a^T A v_i = -d sum_r dv_a,r dv_i,r - c sum_r v_a,r (v_i,r+1 - v_i,r-1),
// dv_r = v_{r+1} - v_r (periodic indices; homogeneous Dirichlet adds the
// r = -1 term dv_{-1} = v_0).  Products of first differences carry no
// cancellation, so FP32 products are accurate to FP32 relative to H, whereas
// v_a^T (A v_i) would multiply the rounding of A v_i by ||A||.
//
// Kernels (one CTA = 256 threads works on a row chunk of one window):
//   k_step_proj     E = dV^T dV_i, F = V^T (S V_i - S^-1 V_i), h1 = V^T W, pre = diag(W^T W)
//   k_update_proj   W <- W - V h1, then h2 = V^T W      (classical Gram-Schmidt, both passes)
//   k_update_gram   W <- W - V h2, then G = W^T W
//   k_scale_gram    W <- W T, then G = W^T W (optional); final pass rounds W into the basis
// Partial sums of each CTA go to a buffer and are summed, in a fixed order, by
// the small per-window kernels that consume them.
//
// FP32 data: products in FP32, per-lane sums compensated (Neumaier), lanes and
// CTAs combined in FP64; the working block W is a (hi, lo) pair updated in
// double-float so that Gram-Schmidt cancellation leaves no FP32-sized noise.
#include <algorithm>

#include "common.cuh"
#include "krylov.cuh"
#include "small.cuh"

namespace pexp {

namespace {

template <typename T>
struct Sum;
template <>
struct Sum<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x, double y) { s = fma(x, y, s); }
    __device__ __forceinline__ double get() const { return s; }
};
template <>
struct Sum<float> {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x, float y) {
        const float v = x * y;
        const float t = s + v;
        const float bp = t - s;
        c += (s - (t - bp)) + (v - bp);   // exact rounding error of s + v (branch-free two-sum)
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// double-float helpers for the working block of FP32 data
struct F2 {
    float hi, lo;
};
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
    const float h = s + e;
    return F2{h, e - (h - s)};
}
__device__ __forceinline__ F2 f2_mulf(float a, F2 b) {   // a (FP32) * (hi, lo)
    const float p = a * b.hi;
    float e = fmaf(a, b.hi, -p);
    e = fmaf(a, b.lo, e);
    const float h = p + e;
    return F2{h, e - (h - p)};
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float h = p + e;
    return F2{h, e - (h - p)};
}
__device__ __forceinline__ F2 f2_from(double v) {
    const float h = (float)v;
    return F2{h, (float)(v - (double)h)};
}

constexpr int kThreads = 256;
constexpr int kTile = 256;   // rows staged in shared memory per iteration

__device__ __forceinline__ int64_t wrap(int64_t r, int64_t n) { return r < 0 ? r + n : (r >= n ? r - n : r); }

}  // namespace

// =====================================================================================
// k_step_proj
// =====================================================================================
template <typename T, int B>
__global__ void __launch_bounds__(kThreads) k_step_proj(const StepTask<T>* __restrict__ tasks, int64_t n, int periodic,
                                                        int64_t rows, int nchunks, int pstride,
                                                        double* __restrict__ partial) {
    const StepTask<T> tk = tasks[blockIdx.y];
    const int ch = blockIdx.x;
    const int64_t r0 = (int64_t)ch * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    const int p = tk.p;   // columns of V_{1:i}
    const T* Vi = tk.V + (int64_t)(p - B) * tk.ld;   // last block of V_{1:i}
    const T* W = tk.V + (int64_t)p * tk.ld;          // working block (slot i+1)
    __shared__ T sD[B][kTile], sC[B][kTile], sW[B][kTile];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // each warp owns columns a = warp, warp + 8, ... (at most 8 per warp kept in registers)
    constexpr int GMAX = 6;
    Sum<T> E[GMAX][B], F[GMAX][B], Hh[GMAX][B];
    Sum<T> pre[B];
#pragma unroll
    for (int g = 0; g < GMAX; ++g)
#pragma unroll
        for (int c = 0; c < B; ++c) {
            E[g][c].zero();
            F[g][c].zero();
            Hh[g][c].zero();
        }
#pragma unroll
    for (int c = 0; c < B; ++c) pre[c].zero();
    const int ng = (p + 7) / 8;   // columns per warp
    double* pout = partial + ((size_t)blockIdx.y * nchunks + ch) * pstride;
    // column groups beyond GMAX are handled in extra passes over the chunk
    for (int g0 = 0; g0 < ng; g0 += GMAX) {
        for (int64_t t0 = r0; t0 < r1; t0 += kTile) {
            const int nt = (int)((t0 + kTile <= r1) ? kTile : (r1 - t0));
            __syncthreads();
            for (int e = threadIdx.x; e < B * kTile; e += kThreads) {
                const int c = e / kTile, k = e % kTile;
                if (k < nt) {
                    const int64_t r = t0 + k;
                    const T* v = Vi + (int64_t)c * tk.ld;
                    const T vr = v[r];
                    T vp, vm;
                    if (periodic) {
                        vp = v[wrap(r + 1, n)];
                        vm = v[wrap(r - 1, n)];
                    } else {
                        vp = (r + 1 < n) ? v[r + 1] : T(0);
                        vm = (r > 0) ? v[r - 1] : T(0);
                    }
                    sD[c][k] = vp - vr;
                    sC[c][k] = vp - vm;
                    sW[c][k] = W[(int64_t)c * tk.ld + r];
                }
            }
            __syncthreads();
            if (g0 == 0 && warp == 0) {
                for (int k = lane; k < nt; k += 32)
#pragma unroll
                    for (int c = 0; c < B; ++c) pre[c].add(sW[c][k], sW[c][k]);
            }
#pragma unroll
            for (int g = 0; g < GMAX; ++g) {
                const int a = (g0 + g) * 8 + warp;
                if (g0 + g >= ng || a >= p) continue;
                const T* va = tk.V + (int64_t)a * tk.ld;
                for (int k = lane; k < nt; k += 32) {
                    const int64_t r = t0 + k;
                    const T x = va[r];
                    T xn;
                    if (periodic) xn = va[wrap(r + 1, n)];
                    else xn = (r + 1 < n) ? va[r + 1] : T(0);
                    const T dx = xn - x;
#pragma unroll
                    for (int c = 0; c < B; ++c) {
                        E[g][c].add(dx, sD[c][k]);
                        F[g][c].add(x, sC[c][k]);
                        Hh[g][c].add(x, sW[c][k]);
                    }
                }
            }
        }
        // Dirichlet: the ghost term dv_{-1} dv_{-1} = v_0 v_0 belongs to the chunk holding row 0
        // warp reductions and partial output for this column group
#pragma unroll
        for (int g = 0; g < GMAX; ++g) {
            const int a = (g0 + g) * 8 + warp;
            if (g0 + g >= ng || a >= p) continue;
            double extra[B];
#pragma unroll
            for (int c = 0; c < B; ++c) extra[c] = 0.0;
            if (!periodic && r0 == 0 && lane == 0) {
#pragma unroll
                for (int c = 0; c < B; ++c) extra[c] = (double)tk.V[(int64_t)a * tk.ld] * (double)Vi[(int64_t)c * tk.ld];
            }
#pragma unroll
            for (int c = 0; c < B; ++c) {
                const double e = wsum(E[g][c].get() + extra[c]);
                const double f = wsum(F[g][c].get());
                const double hh = wsum(Hh[g][c].get());
                if (lane == 0) {
                    pout[a + c * p] = e;
                    pout[p * B + a + c * p] = f;
                    pout[2 * p * B + a + c * p] = hh;
                }
                E[g][c].zero();
                F[g][c].zero();
                Hh[g][c].zero();
            }
        }
    }
    if (warp == 0) {
#pragma unroll
        for (int c = 0; c < B; ++c) {
            const double v = wsum(pre[c].get());
            if (lane == 0) pout[3 * p * B + c] = v;
        }
    }
}

// =====================================================================================
// Gram-Schmidt update fused with the next projection (mode 0) or Gram matrix (mode 1):
//   W <- W - V h;   mode 0: partial h2 = V^T W;   mode 1: partial G = W^T W.
// A row tile of V is staged in shared memory: rows update W (row-parallel), then
// warps own columns of V for the projection (column-parallel), V read once.
// =====================================================================================
template <typename T, int B>
__device__ __forceinline__ void load_coeffs(const UpdTask<T>& tk, int nc, double* sh) {
    // nc = number of coefficient entries (p*B or B*B); summed over partial chunks if given
    if (tk.hpart) {
        const Parts pp{tk.hpart, tk.hchunks, tk.hstride};
        for (int e = threadIdx.x >> 5; e < nc; e += kThreads / 32) {
            const double v = parts_sum_warp(pp, 0, e);
            if ((threadIdx.x & 31) == 0) sh[e] = v;
        }
        return;
    }
    for (int e = threadIdx.x; e < nc; e += kThreads) {
        {
            const int rows = (nc == B * B) ? B : tk.p;
            const int a = e % rows, c = e / rows;
            sh[e] = tk.hm[a + (int64_t)c * tk.ldh];
        }
    }
}

template <typename T, int B, int MODE>
__global__ void __launch_bounds__(kThreads) k_update(const UpdTask<T>* __restrict__ tasks, int64_t n, int64_t rows,
                                                     int nchunks, int pstride, double* __restrict__ partial) {
    const UpdTask<T> tk = tasks[blockIdx.y];
    const int ch = blockIdx.x;
    const int64_t r0 = (int64_t)ch * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    const int p = tk.p;
    extern __shared__ double sh_upd[];
    double* sh = sh_upd;                                       // p x B coefficients
    T* sV = reinterpret_cast<T*>(sh + ((p * B + 1) & ~1));    // p x kTile
    T* sW = sV + (size_t)p * kTile;                            // B x kTile (rounded new W)
    load_coeffs<T, B>(tk, p * B, sh);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int GMAX = 6;
    const int ng = (p + 7) / 8;
    Sum<T> acc[GMAX][B];
    Sum<T> gram[B][B];
#pragma unroll
    for (int g = 0; g < GMAX; ++g)
#pragma unroll
        for (int c = 0; c < B; ++c) acc[g][c].zero();
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) gram[i][j].zero();
    double* pout = partial + ((size_t)blockIdx.y * nchunks + ch) * pstride;
    for (int g0 = 0; g0 < (MODE == 0 ? ng : 1); g0 += GMAX) {
        for (int64_t t0 = r0; t0 < r1; t0 += kTile) {
            const int nt = (int)((t0 + kTile <= r1) ? kTile : (r1 - t0));
            __syncthreads();
            for (int e = threadIdx.x; e < p * kTile; e += kThreads) {
                const int a = e / kTile, k = e % kTile;
                if (k < nt) sV[(size_t)a * kTile + k] = tk.V[(int64_t)a * tk.ld + t0 + k];
            }
            __syncthreads();
            // row-parallel update (first column group only), or reload of the updated W
            for (int k = threadIdx.x; k < nt; k += kThreads) {
                const int64_t r = t0 + k;
                if (g0 == 0) {
                    if constexpr (sizeof(T) == 4) {
                        F2 w[B];
#pragma unroll
                        for (int c = 0; c < B; ++c) w[c] = F2{tk.Wh[(int64_t)c * tk.ld + r], tk.Wl[(int64_t)c * tk.ld + r]};
                        for (int a = 0; a < p; ++a) {
                            const float x = sV[(size_t)a * kTile + k];
#pragma unroll
                            for (int c = 0; c < B; ++c) w[c] = f2_add(w[c], f2_mulf(x, f2_from(-sh[a + c * p])));
                        }
#pragma unroll
                        for (int c = 0; c < B; ++c) {
                            tk.Wh[(int64_t)c * tk.ld + r] = w[c].hi;
                            tk.Wl[(int64_t)c * tk.ld + r] = w[c].lo;
                            sW[c * kTile + k] = w[c].hi + w[c].lo;
                        }
                    } else {
                        double w[B];
#pragma unroll
                        for (int c = 0; c < B; ++c) w[c] = tk.Wh[(int64_t)c * tk.ld + r];
                        for (int a = 0; a < p; ++a) {
                            const double x = sV[(size_t)a * kTile + k];
#pragma unroll
                            for (int c = 0; c < B; ++c) w[c] = fma(-sh[a + c * p], x, w[c]);
                        }
#pragma unroll
                        for (int c = 0; c < B; ++c) {
                            tk.Wh[(int64_t)c * tk.ld + r] = w[c];
                            sW[c * kTile + k] = w[c];
                        }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < B; ++c) {
                        T v = tk.Wh[(int64_t)c * tk.ld + r];
                        if constexpr (sizeof(T) == 4) v += tk.Wl[(int64_t)c * tk.ld + r];
                        sW[c * kTile + k] = v;
                    }
                }
                if (MODE == 1) {
#pragma unroll
                    for (int i = 0; i < B; ++i)
#pragma unroll
                        for (int j = 0; j < B; ++j) gram[i][j].add(sW[i * kTile + k], sW[j * kTile + k]);
                }
            }
            if (MODE == 0) {
                __syncthreads();
#pragma unroll
                for (int g = 0; g < GMAX; ++g) {
                    const int a = (g0 + g) * 8 + warp;
                    if (g0 + g >= ng || a >= p) continue;
                    for (int k = lane; k < nt; k += 32) {
                        const T x = sV[(size_t)a * kTile + k];
#pragma unroll
                        for (int c = 0; c < B; ++c) acc[g][c].add(x, sW[c * kTile + k]);
                    }
                }
            }
        }
        if (MODE == 0) {
#pragma unroll
            for (int g = 0; g < GMAX; ++g) {
                const int a = (g0 + g) * 8 + warp;
                if (g0 + g >= ng || a >= p) continue;
#pragma unroll
                for (int c = 0; c < B; ++c) {
                    const double v = wsum(acc[g][c].get());
                    if (lane == 0) pout[a + c * p] = v;
                    acc[g][c].zero();
                }
            }
        }
    }
    if (MODE == 1) {
        __shared__ double sg[kThreads / 32][B * B];
#pragma unroll
        for (int i = 0; i < B; ++i)
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const double v = wsum(gram[i][j].get());
                if (lane == 0) sg[warp][i + j * B] = v;
            }
        __syncthreads();
        for (int e = threadIdx.x; e < B * B; e += kThreads) {
            double s = 0.0;
            for (int w2 = 0; w2 < kThreads / 32; ++w2) s += sg[w2][e];
            pout[e] = s;
        }
    }
}

// =====================================================================================
// Block scaling W <- W T (T: B x B), with the Gram matrix of the result (gram != 0)
// or, for the final pass, the result rounded into the basis slot task.out.
// =====================================================================================
template <typename T, int B>
__global__ void __launch_bounds__(kThreads) k_scale(const UpdTask<T>* __restrict__ tasks, int64_t n, int64_t rows,
                                                    int nchunks, int gramflag, int pstride,
                                                    double* __restrict__ partial) {
    const UpdTask<T> tk = tasks[blockIdx.y];
    const int ch = blockIdx.x;
    const int64_t r0 = (int64_t)ch * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    __shared__ double sh[B * B];
    load_coeffs<T, B>(tk, B * B, sh);
    __syncthreads();
    Sum<T> gram[B][B];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) gram[i][j].zero();
    for (int64_t r = r0 + threadIdx.x; r < r1; r += kThreads) {
        T res[B];
        if constexpr (sizeof(T) == 4) {
            F2 x[B], z[B];
#pragma unroll
            for (int c = 0; c < B; ++c) {
                x[c] = F2{tk.Wh[(int64_t)c * tk.ld + r], tk.Wl[(int64_t)c * tk.ld + r]};
                z[c] = F2{0.f, 0.f};
            }
#pragma unroll
            for (int a = 0; a < B; ++a)
#pragma unroll
                for (int c = 0; c < B; ++c) z[c] = f2_add(z[c], f2_mul(x[a], f2_from(sh[a + c * B])));
#pragma unroll
            for (int c = 0; c < B; ++c) {
                res[c] = z[c].hi + z[c].lo;
                if (tk.out) {
                    tk.out[(int64_t)c * tk.ld + r] = res[c];
                } else {
                    tk.Wh[(int64_t)c * tk.ld + r] = z[c].hi;
                    tk.Wl[(int64_t)c * tk.ld + r] = z[c].lo;
                }
            }
        } else {
            double x[B];
#pragma unroll
            for (int c = 0; c < B; ++c) x[c] = tk.Wh[(int64_t)c * tk.ld + r];
#pragma unroll
            for (int c = 0; c < B; ++c) {
                double z = 0.0;
#pragma unroll
                for (int a = 0; a < B; ++a) z = fma(x[a], sh[a + c * B], z);
                res[c] = z;
                if (tk.out) tk.out[(int64_t)c * tk.ld + r] = z;
                else tk.Wh[(int64_t)c * tk.ld + r] = z;
            }
        }
        if (gramflag) {
#pragma unroll
            for (int i = 0; i < B; ++i)
#pragma unroll
                for (int j = 0; j < B; ++j) gram[i][j].add(res[i], res[j]);
        }
    }
    if (gramflag) {
        __shared__ double sg[kThreads / 32][B * B];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        double* pout = partial + ((size_t)blockIdx.y * nchunks + ch) * pstride;
#pragma unroll
        for (int i = 0; i < B; ++i)
#pragma unroll
            for (int j = 0; j < B; ++j) {
                const double v = wsum(gram[i][j].get());
                if (lane == 0) sg[warp][i + j * B] = v;
            }
        __syncthreads();
        for (int e = threadIdx.x; e < B * B; e += kThreads) {
            double s = 0.0;
            for (int w2 = 0; w2 < kThreads / 32; ++w2) s += sg[w2][e];
            pout[e] = s;
        }
    }
}

// =====================================================================================
// Gram matrix of the source samples of one window: G = X^T X, X = s columns of the
// time-major source (consecutive rows of the n_out x n array).  A row tile of X is
// staged in shared memory; thread t owns entries (a, c), a <= c, and sums FP32
// products with compensation; CTAs write partial Gram matrices (s x s, both halves).
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreads) k_source_gram(const T* const* __restrict__ Xp, const int* __restrict__ sv,
                                                          int64_t n, int64_t rows, int nchunks, int pstride,
                                                          double* __restrict__ partial) {
    const int task = blockIdx.y;
    const T* X = Xp[task];
    const int s = sv[task];
    const int ch = blockIdx.x;
    const int64_t r0 = (int64_t)ch * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    extern __shared__ double sh_gram[];
    T* sX = reinterpret_cast<T*>(sh_gram);   // s x kTile
    const int npair = s * (s + 1) / 2;
    // up to 9 (a, c) pairs per thread: s <= 64
    constexpr int MAXP = 9;
    int pa[MAXP], pc[MAXP];
    int np = 0;
    for (int q = threadIdx.x; q < npair && np < MAXP; q += kThreads) {
        int a = 0, rem = q;
        while (rem >= s - a) { rem -= s - a; ++a; }
        pa[np] = a;
        pc[np] = a + rem;
        ++np;
    }
    Sum<T> acc[MAXP];
#pragma unroll
    for (int q = 0; q < MAXP; ++q) acc[q].zero();
    for (int64_t t0 = r0; t0 < r1; t0 += kTile) {
        const int nt = (int)((t0 + kTile <= r1) ? kTile : (r1 - t0));
        __syncthreads();
        for (int e = threadIdx.x; e < s * kTile; e += kThreads) {
            const int a = e / kTile, k = e % kTile;
            if (k < nt) sX[a * kTile + k] = X[(int64_t)a * n + t0 + k];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXP; ++q) {
            if (q >= np) break;
            const T* xa = sX + pa[q] * kTile;
            const T* xc = sX + pc[q] * kTile;
            for (int k = 0; k < nt; ++k) acc[q].add(xa[k], xc[k]);
        }
    }
    double* pout = partial + ((size_t)task * nchunks + ch) * pstride;
#pragma unroll
    for (int q = 0; q < MAXP; ++q) {
        if (q >= np) break;
        const double v = acc[q].get();
        pout[pa[q] + pc[q] * s] = v;
        pout[pc[q] + pa[q] * s] = v;
    }
}

// =====================================================================================
// launchers
// =====================================================================================
KGeom krylov_geom(int ntasks, int64_t n) {
    KGeom g;
    const int want = std::max(1, (4 * kNumSM + ntasks - 1) / ntasks);
    const int64_t maxch = std::max<int64_t>(1, (n + kTile - 1) / kTile);
    g.nchunks = (int)std::min<int64_t>(want, maxch);
    g.rows = (n + g.nchunks - 1) / g.nchunks;
    g.rows = (g.rows + kTile - 1) / kTile * kTile;
    g.nchunks = (int)((n + g.rows - 1) / g.rows);
    return g;
}

size_t krylov_partial_doubles(int ntasks, int p_max, int b_max, int64_t n) {
    const KGeom g = krylov_geom(ntasks, n);
    const size_t stride = (size_t)3 * p_max * b_max + b_max;
    return (size_t)ntasks * g.nchunks * std::max<size_t>(stride, (size_t)b_max * b_max) + 64;
}

size_t krylov_update_smem(int p_max, int b, size_t tsize) {
    return sizeof(double) * (size_t)((p_max * b + 1) & ~1) + tsize * (size_t)(p_max + b) * kTile;
}

#define PEXP_B_DISPATCH(b, CALL)     \
    switch (b) {                      \
        case 1: { constexpr int BB = 1; CALL; } break; \
        case 2: { constexpr int BB = 2; CALL; } break; \
        case 3: { constexpr int BB = 3; CALL; } break; \
        case 4: { constexpr int BB = 4; CALL; } break; \
        default: break;               \
    }

template <typename T>
void launch_step_proj(const StepTask<T>* tasks, int ntasks, int b, int64_t n, int periodic, KGeom g,
                      double* partial, int pstride, cudaStream_t s) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    PEXP_B_DISPATCH(b, (k_step_proj<T, BB><<<grid, kThreads, 0, s>>>(tasks, n, periodic, g.rows, g.nchunks, pstride, partial)));
}

template <typename T>
void launch_update(const UpdTask<T>* tasks, int ntasks, int b, int p_max, int64_t n, int mode, KGeom g,
                   double* partial, int pstride, cudaStream_t s) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    const size_t sm = krylov_update_smem(p_max, b, sizeof(T));
    if (mode == 0) {
        PEXP_B_DISPATCH(b, ({
            if (sm > 48 * 1024) cudaFuncSetAttribute(k_update<T, BB, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_update<T, BB, 0><<<grid, kThreads, sm, s>>>(tasks, n, g.rows, g.nchunks, pstride, partial);
        }));
    } else {
        PEXP_B_DISPATCH(b, ({
            if (sm > 48 * 1024) cudaFuncSetAttribute(k_update<T, BB, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
            k_update<T, BB, 1><<<grid, kThreads, sm, s>>>(tasks, n, g.rows, g.nchunks, pstride, partial);
        }));
    }
}

template <typename T>
void launch_scale(const UpdTask<T>* tasks, int ntasks, int b, int64_t n, int gram, KGeom g, double* partial,
                  int pstride, cudaStream_t s) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    PEXP_B_DISPATCH(b, (k_scale<T, BB><<<grid, kThreads, 0, s>>>(tasks, n, g.rows, g.nchunks, gram, pstride, partial)));
}

template <typename T>
void launch_source_gram(const T* const* X, const int* sv, int ntasks, int s_max, int64_t n, KGeom g, double* partial,
                        int pstride, cudaStream_t st) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    const size_t sm = sizeof(T) * (size_t)s_max * kTile;
    if (sm > 48 * 1024) cudaFuncSetAttribute(k_source_gram<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_source_gram<T><<<grid, kThreads, sm, st>>>(X, sv, n, g.rows, g.nchunks, pstride, partial);
}

#define PEXP_KRY_INST(T)                                                                                           \
    template void launch_step_proj<T>(const StepTask<T>*, int, int, int64_t, int, KGeom, double*, int, cudaStream_t); \
    template void launch_update<T>(const UpdTask<T>*, int, int, int, int64_t, int, KGeom, double*, int, cudaStream_t); \
    template void launch_scale<T>(const UpdTask<T>*, int, int, int64_t, int, KGeom, double*, int, cudaStream_t); \
    template void launch_source_gram<T>(const T* const*, const int*, int, int, int64_t, KGeom, double*, int, cudaStream_t);
PEXP_KRY_INST(double)
PEXP_KRY_INST(float)

}  // namespace pexp
