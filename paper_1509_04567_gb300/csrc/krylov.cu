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
// Kernels (CTA = 256 threads on a chunk of 1024-8192 rows of one window):
//   k_step_proj  E = dV^T dV_i, F = V^T (S V_i - S^-1 V_i), h1 = V^T W, pre = diag(W^T W)
//   k_update0    W <- W - V h1, then G = W^T W           (first Gram-Schmidt pass)
//   k_scale_proj W <- W T1 (Cholesky QR), then h2 = V^T W
//   k_update1    W <- W - V h2, then G = W^T W           (second pass; each CTA sums
//                h2 from the k_scale_proj partials itself)
//   k_scale      W <- W T2; the final pass rounds W into the basis
// i.e. block classical Gram-Schmidt with Cholesky QR, applied twice (BCGS2).
//
// Memory-level parallelism: every thread owns rows and issues the loads of all the
// columns it needs for a row before using any of them (the update passes take two rows
// at a time, W first), so a CTA keeps tens of KB in flight; the +-1 neighbours of the stencil sums come from adjacent lanes (warps
// overlap by one row on each side).  Sums: each thread accumulates FP32 (FP64 data:
// FP64) products of its rows; warps reduce in the data type; the 8 warps and the
// CTAs are combined in FP64 (one partial per CTA, summed in a fixed order by the
// consumer).  FP64 arithmetic runs at 1/64 of the FP32 rate on this GPU, so it is
// kept out of the per-row work of the FP32 kernels.  The Galerkin sums E and F are
// compensated (per-thread two-product/two-sum, two-sum warp tree): the projected
// matrix multiplies their rounding by ||H|| over each subinterval, and plain FP32
// sums left a solution error of several 1e-6 at 2^20 points.
//
// FP32 data: the working block W is a (hi, lo) pair updated in double-float, so that
// Gram-Schmidt cancellation leaves no FP32-sized noise.  The first pass subtracts
// V h1 with exact FP32 products x*h_hi (FMA) and a compensated sum; the second pass
// coefficients h2 are at the orthogonality-error level, so FP32 products suffice.
// The second pass works on the block normalised by the first Cholesky QR: a block
// whose columns are nearly dependent (condition kappa) would otherwise turn the
// ~1e-10 residual of the projections into a kappa-times larger loss of orthogonality.
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

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
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
constexpr int kWarps = kThreads / 32;
constexpr int kTile = 256;    // rows per shared-memory tile of k_source_gram
constexpr int kHalo = 30;     // active rows per warp in k_step_proj (lanes 1..30)

// per-thread accumulator budget (registers) of the projection kernels
// (two CTAs of 256 threads per SM: at most 128 registers per thread; the kernels built
// for three, at 80 registers, keep fewer columns per CTA)
template <typename T>
struct Budget {
    static constexpr int acc = 72;
};
template <>
struct Budget<double> {
    static constexpr int acc = 36;
};
template <typename T, int B, bool JAC = false>
struct Group {
    // columns per CTA of k_step_proj: FP32 data keep E and F as compensated (s, c) pairs
    // (5 registers per column and block column), FP64 data plain sums (3 doubles); FP32
    // single columns take 8, which fits 3 CTAs per SM (80 registers)
    static constexpr int step = sizeof(T) == 4 ? (B == 1 ? 8 : 16 / B) : Budget<T>::acc / (3 * B);
    static constexpr int vtw = Budget<T>::acc / (B + 1);     // columns per CTA of k_vtw
    static constexpr int ctas = (sizeof(T) == 4 && B == 1) ? 3 : 2;   // CTAs per SM k_step_proj is built for
};
// the Jacobian launches keep two more compensated sums (Ja, Jb) per column and block column
template <typename T, int B>
struct Group<T, B, true> {
    static constexpr int step = sizeof(T) == 4 ? (B == 1 ? 4 : (8 / B > 1 ? 8 / B : 1)) : (Budget<T>::acc / (5 * B) > 1 ? Budget<T>::acc / (5 * B) : 1);
    static constexpr int vtw = Budget<T>::acc / (B + 1);
    static constexpr int ctas = 2;
};
constexpr int kFuseP = 16;   // k_scale_proj keeps V^T W accumulators for up to 16 columns

template <typename T>
__device__ __forceinline__ T ldg(const T* p) { return __ldg(p); }

// s + c += x * y: FP32 sums keep the rounding errors of the product and of the sum in c
// (two-product by FMA, two-sum); FP64 sums are plain FMAs.
__device__ __forceinline__ void comp_add(float& s, float& c, float x, float y) {
    const float p = x * y;
    const float pe = fmaf(x, y, -p);
    const float t = s + p;
    const float bp = t - s;
    c += ((s - (t - bp)) + (p - bp)) + pe;
    s = t;
}
__device__ __forceinline__ void comp_add(double& s, double&, double x, double y) { s = fma(x, y, s); }

// Reduce per-thread values over the CTA: warp sums in the data type, then the 8 warp
// results in FP64 by thread e for entry e.  sred: kWarps x ne doubles.
template <typename T>
__device__ __forceinline__ void warp_to_smem(T v, double* sred, int ne, int e) {
    const T s = warp_sum(v);
    if ((threadIdx.x & 31) == 0) sred[(threadIdx.x >> 5) * ne + e] = (double)s;
}
// Same for a compensated (hi, lo) pair: the warp tree adds with two-sum.
__device__ __forceinline__ void warp_to_smem2(float hi, float lo, double* sred, int ne, int e) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o), l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        const float sum = hi + h2;
        const float bp = sum - hi;
        const float err = (hi - (sum - bp)) + (h2 - bp);
        hi = sum;
        lo = lo + l2 + err;
    }
    if ((threadIdx.x & 31) == 0) sred[(threadIdx.x >> 5) * ne + e] = (double)hi + (double)lo;
}
__device__ __forceinline__ void warp_to_smem2(double hi, double lo, double* sred, int ne, int e) {
    warp_to_smem(hi + lo, sred, ne, e);
}
__device__ __forceinline__ double cta_entry(const double* sred, int ne, int e) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) s += sred[w * ne + e];
    return s;
}

}  // namespace

// =====================================================================================
// k_step_proj: grid (chunks, tasks, column groups).  Group z owns columns
// [z*PG, z*PG + PG) of V_{1:p}; group 0 also sums diag(W^T W).
// =====================================================================================
template <typename T, int B, bool JAC>
__global__ void __launch_bounds__(kThreads, Group<T, B, JAC>::ctas) k_step_proj(const StepTask<T>* __restrict__ tasks, int64_t n, int periodic,
                                                        int64_t rows, int nchunks, int pstride,
                                                        double* __restrict__ partial) {
    pdl_entry();
    constexpr int PG = Group<T, B, JAC>::step;
    constexpr int NK = JAC ? 5 : 3;   // sums per column pair: E, F, h1 (+ Ja, Jb)
    constexpr int NE = NK * PG * B + B;
    __shared__ double sred[kWarps * NE];
    const StepTask<T> tk = tasks[blockIdx.y];
    if (tk.conv && *tk.conv) return;
    const int p = tk.p;
    const int a0 = blockIdx.z * PG;
    if (a0 >= p) return;
    const int na = min(PG, p - a0);
    const int64_t ld = tk.ld;
    const T* __restrict__ Va = tk.V + (int64_t)a0 * ld;
    const T* __restrict__ Vi = tk.V + (int64_t)(p - B) * ld;   // last block of V_{1:p}
    const T* __restrict__ W = tk.V + (int64_t)p * ld;          // working block (slot p)
    const int64_t r0 = (int64_t)blockIdx.x * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const bool grp0 = blockIdx.z == 0;
    T aE[PG][B], aF[PG][B], cE[PG][B], cF[PG][B], aH[PG][B], aP[B];
    T aJa[PG][B], cJa[PG][B], aJb[PG][B], cJb[PG][B];
#pragma unroll
    for (int q = 0; q < PG; ++q)
#pragma unroll
        for (int c = 0; c < B; ++c) {
            aE[q][c] = aF[q][c] = cE[q][c] = cF[q][c] = aH[q][c] = T(0);
            aJa[q][c] = cJa[q][c] = aJb[q][c] = cJb[q][c] = T(0);
        }
#pragma unroll
    for (int c = 0; c < B; ++c) aP[c] = T(0);
    // Dirichlet: the r = -1 term dv_{-1} = v_0 of the E sums, in the chunk holding row 0
    if (!periodic && r0 == 0 && threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < PG; ++q)
#pragma unroll
            for (int c = 0; c < B; ++c)
                if (q < na) aE[q][c] = Va[(int64_t)q * ld] * Vi[(int64_t)c * ld];
    }
    // lanes 1..30 of each warp own rows; lanes 0 and 31 load the rows before and after
    for (int64_t base = r0; base < r1; base += (int64_t)kHalo * kWarps) {
        const int64_t r = base + (int64_t)warp * kHalo + lane - 1;
        const bool act = lane >= 1 && lane <= kHalo && r < r1;
        const bool need = r <= r1;   // r >= r0 - 1 holds by construction
        bool ok;
        int64_t rp;
        if (periodic) {
            ok = need;
            rp = r < 0 ? r + n : (r >= n ? r - n : r);
        } else {
            ok = need && r >= 0 && r < n;
            rp = r;
        }
        T x[PG], vi[B], w[B];
#pragma unroll
        for (int q = 0; q < PG; ++q) x[q] = (ok && q < na) ? ldg(Va + (int64_t)q * ld + rp) : T(0);
#pragma unroll
        for (int c = 0; c < B; ++c) {
            vi[c] = ok ? ldg(Vi + (int64_t)c * ld + rp) : T(0);
            w[c] = act ? ldg(W + (int64_t)c * ld + rp) : T(0);
        }
        T D[B], C[B];
#pragma unroll
        for (int c = 0; c < B; ++c) {
            const T vr = __shfl_down_sync(0xffffffffu, vi[c], 1);
            const T vl = __shfl_up_sync(0xffffffffu, vi[c], 1);
            D[c] = vr - vi[c];
            C[c] = vr - vl;
        }

        T ub = T(0);
        if constexpr (JAC) ub = act ? ldg(tk.ubar + rp) : T(0);
#pragma unroll
        for (int q = 0; q < PG; ++q) {
            const T xr = __shfl_down_sync(0xffffffffu, x[q], 1);
            T xl = T(0);
            if constexpr (JAC) xl = __shfl_up_sync(0xffffffffu, x[q], 1);
            if (act && q < na) {
                const T dx = xr - x[q];
#pragma unroll
                for (int c = 0; c < B; ++c) {
                    comp_add(aE[q][c], cE[q][c], dx, D[c]);
                    comp_add(aF[q][c], cF[q][c], x[q], C[c]);
                    aH[q][c] = fma(x[q], w[c], aH[q][c]);
                    if constexpr (JAC) {
                        comp_add(aJa[q][c], cJa[q][c], ub * vi[c], xr - xl);
                        comp_add(aJb[q][c], cJb[q][c], ub * x[q], C[c]);
                    }
                }
            }
        }
        if (act && grp0) {
#pragma unroll
            for (int c = 0; c < B; ++c) aP[c] = fma(w[c], w[c], aP[c]);
        }
    }
#pragma unroll
    for (int q = 0; q < PG; ++q) {
        if (q < na) {
#pragma unroll
            for (int c = 0; c < B; ++c) {
                warp_to_smem2(aE[q][c], cE[q][c], sred, NE, (q * B + c) * NK + 0);
                warp_to_smem2(aF[q][c], cF[q][c], sred, NE, (q * B + c) * NK + 1);
                warp_to_smem(aH[q][c], sred, NE, (q * B + c) * NK + 2);
                if constexpr (JAC) {
                    warp_to_smem2(aJa[q][c], cJa[q][c], sred, NE, (q * B + c) * NK + 3);
                    warp_to_smem2(aJb[q][c], cJb[q][c], sred, NE, (q * B + c) * NK + 4);
                }
            }
        }
    }
    if (grp0) {
#pragma unroll
        for (int c = 0; c < B; ++c) warp_to_smem(aP[c], sred, NE, NK * PG * B + c);
    }
    __syncthreads();
    double* pout = partial + ((size_t)blockIdx.y * nchunks + blockIdx.x) * pstride;
    for (int e = threadIdx.x; e < NE; e += kThreads) {
        if (e < NK * PG * B) {
            const int kind = e % NK, qc = e / NK, q = qc / B, c = qc % B;
            // kinds 0..2 at kind * p * B; Ja, Jb after pre (3 p B + B)
            const int base = kind < 3 ? kind * p * B : 3 * p * B + B + (kind - 3) * p * B;
            if (q < na) pout[base + (a0 + q) + c * p] = cta_entry(sred, NE, e);
        } else if (grp0) {
            pout[3 * p * B + (e - NK * PG * B)] = cta_entry(sred, NE, e);
        }
    }
}

// =====================================================================================
// Coefficients of the update kernels: dense FP64 (tk.hm, leading dimension tk.ldh),
// staged in shared memory -- as (hi, lo) FP32 pairs for FP32 data.
// =====================================================================================
template <typename T>
struct Coef;
template <>
struct Coef<float> {
    using type = float2;
    __device__ static type make(double v) {
        const float h = (float)v;
        return make_float2(h, (float)(v - (double)h));
    }
};
template <>
struct Coef<double> {
    using type = double;
    __device__ static type make(double v) { return v; }
};

template <typename T>
__device__ __forceinline__ void stage_coeffs(const UpdTask<T>& tk, int rows_h, int cols, typename Coef<T>::type* sh) {
    for (int e = threadIdx.x; e < rows_h * cols; e += kThreads) {
        const int a = e % rows_h, c = e / rows_h;
        sh[e] = Coef<T>::make(tk.hm[a + (int64_t)c * tk.ldh]);
    }
    __syncthreads();
}

// W <- W - V h for one row: FP32 data in double-float with exact products x*h_hi
// (FMA) and a compensated sum; FP64 data with FMAs.  Columns [q0, q0 + Q) of V.
template <int Q, int B>
__device__ __forceinline__ void sub_vh(const float (&x)[Q], const float2* sh, int p, int q0, float (&sh_)[B],
                                       float (&sl_)[B]) {
#pragma unroll
    for (int c = 0; c < B; ++c) {
        float s = sh_[c], l = sl_[c];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            if (q0 + q < p) {
                const float2 h = sh[(q0 + q) + c * p];
                const float ph = x[q] * h.x;
                float pe = fmaf(x[q], h.x, -ph);
                pe = fmaf(x[q], h.y, pe);
                const float t = s + ph;
                const float bp = t - s;
                l += ((s - (t - bp)) + (ph - bp)) + pe;
                s = t;
            }
        }
        sh_[c] = s;
        sl_[c] = l;
    }
}
template <int Q, int B>
__device__ __forceinline__ void sub_vh(const double (&x)[Q], const double* sh, int p, int q0, double (&sh_)[B],
                                       double (&)[B]) {
#pragma unroll
    for (int c = 0; c < B; ++c) {
        double s = sh_[c];
#pragma unroll
        for (int q = 0; q < Q; ++q)
            if (q0 + q < p) s = fma(x[q], sh[(q0 + q) + c * p], s);
        sh_[c] = s;
    }
}

// =====================================================================================
// k_update0: W <- W - V h1 (first Gram-Schmidt pass) and partial G = W^T W.
// Each thread takes R rows per iteration and issues all their loads (W first, then the
// columns of V in groups of Q) before using any, so a row costs one memory round trip.
// =====================================================================================
constexpr int kUpdQ = 8;   // columns of V per load group of the update kernels
constexpr int kUpdR = 2;   // rows per thread per iteration of the update kernels
template <int B>
constexpr int kUpdCtas = B <= 2 ? 4 : 2;   // resident CTAs per SM the update kernels are built for
template <int B>
constexpr int kScaleProjCtas = B == 1 ? 3 : 2;   // and the scale-projection kernel

template <typename T, int B>
__device__ __forceinline__ void k_update0_body(const UpdTask<T>& tk, int64_t n, int64_t rows, int nchunks, int pstride, double* __restrict__ partial, int bx, int by) {

    using CT = typename Coef<T>::type;
    constexpr int Q = kUpdQ, R = kUpdR;
    constexpr int NE = B * B;
    extern __shared__ double sh_dyn[];
    CT* sh = reinterpret_cast<CT*>(sh_dyn);
    __shared__ double sred[kWarps * NE];
    const int p = tk.p;
    stage_coeffs<T>(tk, p, B, sh);
    const int64_t ld = tk.ld;
    const int64_t r0 = (int64_t)bx * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    T g[B][B];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) g[i][j] = T(0);
    for (int64_t base = r0; base < r1; base += (int64_t)R * kThreads) {
        int64_t r[R];
        bool act[R];
        T wh[R][B], wl[R][B], s[R][B], l[R][B];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            r[u] = base + (int64_t)u * kThreads + threadIdx.x;
            act[u] = r[u] < r1;
#pragma unroll
            for (int c = 0; c < B; ++c) {
                wh[u][c] = act[u] ? tk.Wh[(int64_t)c * ld + r[u]] : T(0);
                if constexpr (sizeof(T) == 4) wl[u][c] = act[u] ? tk.Wl[(int64_t)c * ld + r[u]] : 0.f;
                s[u][c] = l[u][c] = T(0);
            }
        }
        for (int q0 = 0; q0 < p; q0 += Q) {
            T x[R][Q];
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int q = 0; q < Q; ++q)
                    x[u][q] = (act[u] && q0 + q < p) ? ldg(tk.V + (int64_t)(q0 + q) * ld + r[u]) : T(0);
#pragma unroll
            for (int u = 0; u < R; ++u) sub_vh<Q, B>(x[u], sh, p, q0, s[u], l[u]);
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            T wr[B];
#pragma unroll
            for (int c = 0; c < B; ++c) {
                if constexpr (sizeof(T) == 4) {
                    const F2 wv = f2_add(F2{wh[u][c], wl[u][c]}, F2{-s[u][c], -l[u][c]});
                    if (act[u]) {
                        tk.Wh[(int64_t)c * ld + r[u]] = wv.hi;
                        tk.Wl[(int64_t)c * ld + r[u]] = wv.lo;
                    }
                    wr[c] = wv.hi + wv.lo;
                } else {
                    const T wv = wh[u][c] - s[u][c];
                    if (act[u]) tk.Wh[(int64_t)c * ld + r[u]] = wv;
                    wr[c] = wv;
                }
            }
#pragma unroll
            for (int i = 0; i < B; ++i)
#pragma unroll
                for (int j = 0; j < B; ++j) g[i][j] = fma(wr[i], wr[j], g[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) warp_to_smem(g[i][j], sred, NE, i + j * B);
    __syncthreads();
    double* pout = partial + ((size_t)by * nchunks + bx) * pstride;
    for (int e = threadIdx.x; e < NE; e += kThreads) pout[e] = cta_entry(sred, NE, e);
}

template <typename T, int B>
__global__ void __launch_bounds__(kThreads, kUpdCtas<B>) k_update0(const UpdTask<T>* __restrict__ tasks, int64_t n, int64_t rows,
                                                         int nchunks, int pstride, double* __restrict__ partial) {    pdl_entry();
    const UpdTask<T> tk = tasks[blockIdx.y];
    if (tk.conv && *tk.conv) return;
    k_update0_body<T, B>(tk, n, rows, nchunks, pstride, partial, blockIdx.x, blockIdx.y);
}

// W <- W T for one row (T: B x B FP64 in shared memory); FP32 data in double-float.
template <int B>
__device__ __forceinline__ void scale_row(float (&xh)[B], float (&xl)[B], const float2* sT, float (&res)[B]) {
    F2 z[B];
#pragma unroll
    for (int c = 0; c < B; ++c) {
        z[c] = F2{0.f, 0.f};
#pragma unroll
        for (int a = 0; a < B; ++a) {
            const float2 t = sT[a + c * B];
            z[c] = f2_add(z[c], f2_mul(F2{xh[a], xl[a]}, F2{t.x, t.y}));
        }
    }
#pragma unroll
    for (int c = 0; c < B; ++c) {
        xh[c] = z[c].hi;
        xl[c] = z[c].lo;
        res[c] = z[c].hi + z[c].lo;
    }
}
template <int B>
__device__ __forceinline__ void scale_row(double (&xh)[B], double (&)[B], const double* sT, double (&res)[B]) {
    double z[B];
#pragma unroll
    for (int c = 0; c < B; ++c) {
        z[c] = 0.0;
#pragma unroll
        for (int a = 0; a < B; ++a) z[c] = fma(xh[a], sT[a + c * B], z[c]);
    }
#pragma unroll
    for (int c = 0; c < B; ++c) xh[c] = res[c] = z[c];
}

// =====================================================================================
// k_scale_proj: W <- W T1 (normalisation of the block after the first Gram-Schmidt
// pass) and partial h2 = V^T W of the normalised block, p <= kFuseP.  Computing the
// second-pass coefficients from the normalised block keeps their error from being
// magnified by the block's conditioning.
// =====================================================================================
template <typename T, int B>
__device__ __forceinline__ void k_scale_proj_body(const UpdTask<T>& tk, int64_t n, int64_t rows, int nchunks, int pstride, double* __restrict__ partial, int bx, int by) {

    constexpr int Q = kFuseP;
    constexpr int NE = Q * B;
    using CT = typename Coef<T>::type;
    __shared__ CT sT[B * B];
    __shared__ double sred[kWarps * NE];
    const int p = tk.p;
    for (int e = threadIdx.x; e < B * B; e += kThreads) sT[e] = Coef<T>::make(tk.hm[(e % B) + (int64_t)(e / B) * tk.ldh]);
    __syncthreads();
    const int64_t ld = tk.ld;
    const int64_t r0 = (int64_t)bx * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    T acc[Q][B];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int c = 0; c < B; ++c) acc[q][c] = T(0);
    for (int64_t base = r0; base < r1; base += kThreads) {
        const int64_t r = base + threadIdx.x;
        const bool act = r < r1;
        T x[Q], xh[B], xl[B], res[B];
#pragma unroll
        for (int q = 0; q < Q; ++q) x[q] = (act && q < p) ? ldg(tk.V + (int64_t)q * ld + r) : T(0);
#pragma unroll
        for (int c = 0; c < B; ++c) {
            xh[c] = act ? tk.Wh[(int64_t)c * ld + r] : T(0);
            if constexpr (sizeof(T) == 4) xl[c] = act ? tk.Wl[(int64_t)c * ld + r] : 0.f;
        }
        scale_row<B>(xh, xl, sT, res);
        if (act) {
#pragma unroll
            for (int c = 0; c < B; ++c) {
                tk.Wh[(int64_t)c * ld + r] = xh[c];
                if constexpr (sizeof(T) == 4) tk.Wl[(int64_t)c * ld + r] = xl[c];
            }
        }
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int c = 0; c < B; ++c) acc[q][c] = fma(x[q], res[c], acc[q][c]);
    }
#pragma unroll
    for (int q = 0; q < Q; ++q)
        if (q < p) {
#pragma unroll
            for (int c = 0; c < B; ++c) warp_to_smem(acc[q][c], sred, NE, q + c * Q);
        }
    __syncthreads();
    double* pout = partial + ((size_t)by * nchunks + bx) * pstride;
    for (int e = threadIdx.x; e < NE; e += kThreads) {
        const int q = e % Q, c = e / Q;
        if (q < p) pout[q + c * p] = cta_entry(sred, NE, e);
    }
}

template <typename T, int B>
__global__ void __launch_bounds__(kThreads, kScaleProjCtas<B>) k_scale_proj(const UpdTask<T>* __restrict__ tasks, int64_t n,
                                                            int64_t rows, int nchunks, int pstride,
                                                            double* __restrict__ partial) {    pdl_entry();
    const UpdTask<T> tk = tasks[blockIdx.y];
    if (tk.conv && *tk.conv) return;
    k_scale_proj_body<T, B>(tk, n, rows, nchunks, pstride, partial, blockIdx.x, blockIdx.y);
}

// =====================================================================================
// k_vtw: partial h = V^T W over columns [z*PG, z*PG + PG) (grid z), W = hi + lo rounded.
// =====================================================================================
template <typename T, int B>
__global__ void __launch_bounds__(kThreads, 2) k_vtw(const UpdTask<T>* __restrict__ tasks, int64_t n, int64_t rows,
                                                  int nchunks, int pstride, double* __restrict__ partial) {
    constexpr int PG = Group<T, B>::vtw;
    constexpr int NE = PG * B;
    __shared__ double sred[kWarps * NE];
    const UpdTask<T> tk = tasks[blockIdx.y];
    if (tk.conv && *tk.conv) return;
    const int p = tk.p;
    const int a0 = blockIdx.z * PG;
    if (a0 >= p) return;
    const int na = min(PG, p - a0);
    const int64_t ld = tk.ld;
    const int64_t r0 = (int64_t)blockIdx.x * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    T acc[PG][B];
#pragma unroll
    for (int q = 0; q < PG; ++q)
#pragma unroll
        for (int c = 0; c < B; ++c) acc[q][c] = T(0);
    for (int64_t base = r0; base < r1; base += kThreads) {
        const int64_t r = base + threadIdx.x;
        const bool act = r < r1;
        T x[PG], w[B];
#pragma unroll
        for (int q = 0; q < PG; ++q) x[q] = (act && q < na) ? ldg(tk.V + (int64_t)(a0 + q) * ld + r) : T(0);
#pragma unroll
        for (int c = 0; c < B; ++c) {
            T v = act ? tk.Wh[(int64_t)c * ld + r] : T(0);
            if constexpr (sizeof(T) == 4) v += act ? tk.Wl[(int64_t)c * ld + r] : 0.f;
            w[c] = v;
        }
#pragma unroll
        for (int q = 0; q < PG; ++q)
#pragma unroll
            for (int c = 0; c < B; ++c) acc[q][c] = fma(x[q], w[c], acc[q][c]);
    }
#pragma unroll
    for (int q = 0; q < PG; ++q)
        if (q < na) {
#pragma unroll
            for (int c = 0; c < B; ++c) warp_to_smem(acc[q][c], sred, NE, q + c * PG);
        }
    __syncthreads();
    double* pout = partial + ((size_t)blockIdx.y * nchunks + blockIdx.x) * pstride;
    for (int e = threadIdx.x; e < NE; e += kThreads) {
        const int q = e % PG, c = e / PG;
        if (q < na) pout[(a0 + q) + c * p] = cta_entry(sred, NE, e);
    }
}

// =====================================================================================
// k_update1: W <- W - V h2 (second Gram-Schmidt pass) and partial G = W^T W.
// h2 is at the orthogonality-error level, so V h2 is formed with FP32 products.
// Loads as in k_update0: R rows per thread, W first, V in groups of Q columns.
// =====================================================================================
template <typename T, int B>
__device__ __forceinline__ void k_update1_body(const UpdTask<T>& tk, int64_t n, int64_t rows, int nchunks, int pstride, double* __restrict__ partial, const double* __restrict__ hpart, int hstride, int bx, int by) {

    constexpr int Q = kUpdQ, R = kUpdR;
    constexpr int NE = B * B;
    extern __shared__ double sh_dyn[];
    T* sh = reinterpret_cast<T*>(sh_dyn);
    __shared__ double sred[kWarps * NE];
    const int p = tk.p;
    if (hpart) {
        // h2 straight from the chunk partials of k_scale_proj (p x B, column-major), summed
        // in the fixed order of parts_sum_warp: every CTA gets the same coefficients, and
        // the same ones that a separate summing kernel would have stored
        const Parts hp{hpart, nchunks, hstride};
        for (int e = threadIdx.x >> 5; e < p * B; e += kWarps) {
            const double v = parts_sum_warp(hp, by, e);
            if ((threadIdx.x & 31) == 0) sh[e] = (T)v;
        }
    } else {
        for (int e = threadIdx.x; e < p * B; e += kThreads) sh[e] = (T)tk.hm[(e % p) + (int64_t)(e / p) * tk.ldh];
    }
    __syncthreads();
    const int64_t ld = tk.ld;
    const int64_t r0 = (int64_t)bx * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    T g[B][B];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) g[i][j] = T(0);
    for (int64_t base = r0; base < r1; base += (int64_t)R * kThreads) {
        int64_t r[R];
        bool act[R];
        T wh[R][B], wl[R][B], s[R][B];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            r[u] = base + (int64_t)u * kThreads + threadIdx.x;
            act[u] = r[u] < r1;
#pragma unroll
            for (int c = 0; c < B; ++c) {
                wh[u][c] = act[u] ? tk.Wh[(int64_t)c * ld + r[u]] : T(0);
                if constexpr (sizeof(T) == 4) wl[u][c] = act[u] ? tk.Wl[(int64_t)c * ld + r[u]] : 0.f;
                s[u][c] = T(0);
            }
        }
        for (int q0 = 0; q0 < p; q0 += Q) {
            T x[R][Q];
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int q = 0; q < Q; ++q)
                    x[u][q] = (act[u] && q0 + q < p) ? ldg(tk.V + (int64_t)(q0 + q) * ld + r[u]) : T(0);
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int c = 0; c < B; ++c)
#pragma unroll
                    for (int q = 0; q < Q; ++q)
                        if (q0 + q < p) s[u][c] = fma(x[u][q], sh[(q0 + q) + c * p], s[u][c]);
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            T wr[B];
#pragma unroll
            for (int c = 0; c < B; ++c) {
                if constexpr (sizeof(T) == 4) {
                    const F2 wv = f2_add(F2{wh[u][c], wl[u][c]}, F2{-s[u][c], 0.f});
                    if (act[u]) {
                        tk.Wh[(int64_t)c * ld + r[u]] = wv.hi;
                        tk.Wl[(int64_t)c * ld + r[u]] = wv.lo;
                    }
                    wr[c] = wv.hi + wv.lo;
                } else {
                    const T wv = wh[u][c] - s[u][c];
                    if (act[u]) tk.Wh[(int64_t)c * ld + r[u]] = wv;
                    wr[c] = wv;
                }
            }
#pragma unroll
            for (int i = 0; i < B; ++i)
#pragma unroll
                for (int j = 0; j < B; ++j) g[i][j] = fma(wr[i], wr[j], g[i][j]);
        }
    }
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) warp_to_smem(g[i][j], sred, NE, i + j * B);
    __syncthreads();
    double* pout = partial + ((size_t)by * nchunks + bx) * pstride;
    for (int e = threadIdx.x; e < NE; e += kThreads) pout[e] = cta_entry(sred, NE, e);
}

template <typename T, int B>
__global__ void __launch_bounds__(kThreads, kUpdCtas<B>) k_update1(const UpdTask<T>* __restrict__ tasks, int64_t n, int64_t rows,
                                                      int nchunks, int pstride, double* __restrict__ partial,
                                                      const double* __restrict__ hpart, int hstride) {    pdl_entry();
    const UpdTask<T> tk = tasks[blockIdx.y];
    if (tk.conv && *tk.conv) return;
    k_update1_body<T, B>(tk, n, rows, nchunks, pstride, partial, hpart, hstride, blockIdx.x, blockIdx.y);
}

// =====================================================================================
// k_scale: W <- W T (T: B x B, dense FP64), with the Gram matrix of the result
// (gram != 0) or, for the final pass, the result rounded into the basis slot task.out.
// Four rows per thread per iteration, loads first.
// =====================================================================================
template <typename T, int B>
__device__ __forceinline__ void k_scale_body(const UpdTask<T>& tk, int64_t n, int64_t rows, int nchunks, int gramflag, int pstride, double* __restrict__ partial, int bx, int by) {

    constexpr int U = 4;
    constexpr int NE = B * B;
    using CT = typename Coef<T>::type;
    __shared__ CT sT[B * B];
    __shared__ double sred[kWarps * NE];
    for (int e = threadIdx.x; e < B * B; e += kThreads) sT[e] = Coef<T>::make(tk.hm[(e % B) + (int64_t)(e / B) * tk.ldh]);
    __syncthreads();
    const int64_t ld = tk.ld;
    const int64_t r0 = (int64_t)bx * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    T g[B][B];
#pragma unroll
    for (int i = 0; i < B; ++i)
#pragma unroll
        for (int j = 0; j < B; ++j) g[i][j] = T(0);
    for (int64_t base = r0; base < r1; base += (int64_t)kThreads * U) {
        T xh[U][B], xl[U][B];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = base + (int64_t)u * kThreads + threadIdx.x;
            const bool act = r < r1;
#pragma unroll
            for (int c = 0; c < B; ++c) {
                xh[u][c] = act ? tk.Wh[(int64_t)c * ld + r] : T(0);
                if constexpr (sizeof(T) == 4) xl[u][c] = act ? tk.Wl[(int64_t)c * ld + r] : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = base + (int64_t)u * kThreads + threadIdx.x;
            const bool act = r < r1;
            T res[B];
            scale_row<B>(xh[u], xl[u], sT, res);
            if (act) {
#pragma unroll
                for (int c = 0; c < B; ++c) {
                    if (tk.out) {
                        tk.out[(int64_t)c * ld + r] = res[c];
                    } else {
                        tk.Wh[(int64_t)c * ld + r] = xh[u][c];
                        if constexpr (sizeof(T) == 4) tk.Wl[(int64_t)c * ld + r] = xl[u][c];
                    }
                }
            }
            if (gramflag) {
#pragma unroll
                for (int i = 0; i < B; ++i)
#pragma unroll
                    for (int j = 0; j < B; ++j) g[i][j] = fma(res[i], res[j], g[i][j]);
            }
        }
    }
    if (gramflag) {
#pragma unroll
        for (int i = 0; i < B; ++i)
#pragma unroll
            for (int j = 0; j < B; ++j) warp_to_smem(g[i][j], sred, NE, i + j * B);
        __syncthreads();
        double* pout = partial + ((size_t)by * nchunks + bx) * pstride;
        for (int e = threadIdx.x; e < NE; e += kThreads) pout[e] = cta_entry(sred, NE, e);
    }
}

template <typename T, int B>
__global__ void __launch_bounds__(kThreads, 2) k_scale(const UpdTask<T>* __restrict__ tasks, int64_t n, int64_t rows,
                                                       int nchunks, int gramflag, int pstride,
                                                       double* __restrict__ partial) {    pdl_entry();
    const UpdTask<T> tk = tasks[blockIdx.y];
    if (tk.conv && *tk.conv) return;
    k_scale_body<T, B>(tk, n, rows, nchunks, gramflag, pstride, partial, blockIdx.x, blockIdx.y);
}

// =====================================================================================
// k_block_gram: partial G = X^T X of an n x b block (b <= 4, task.Wh, ld task.ld, b = task.p),
// compensated FP32 sums for FP32 data.
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreads) k_block_gram(const UpdTask<T>* __restrict__ tasks, int64_t n, int64_t rows,
                                                         int nchunks, int pstride, double* __restrict__ partial) {
    constexpr int BM = 4;
    constexpr int NE = BM * BM;
    __shared__ double sred[kWarps * NE];
    const UpdTask<T> tk = tasks[blockIdx.y];
    const int b = tk.p;
    const int64_t ld = tk.ld;
    const int64_t r0 = (int64_t)blockIdx.x * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    T gs[BM][BM], gc[BM][BM];
#pragma unroll
    for (int i = 0; i < BM; ++i)
#pragma unroll
        for (int j = 0; j < BM; ++j) gs[i][j] = gc[i][j] = T(0);
    constexpr int U = 4;
    for (int64_t base = r0; base < r1; base += (int64_t)kThreads * U) {
        T x[U][BM];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t r = base + (int64_t)u * kThreads + threadIdx.x;
#pragma unroll
            for (int c = 0; c < BM; ++c) x[u][c] = (r < r1 && c < b) ? ldg(tk.Wh + (int64_t)c * ld + r) : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int i = 0; i < BM; ++i)
#pragma unroll
                for (int j = i; j < BM; ++j) comp_add(gs[i][j], gc[i][j], x[u][i], x[u][j]);
    }
#pragma unroll
    for (int i = 0; i < BM; ++i)
#pragma unroll
        for (int j = i; j < BM; ++j) warp_to_smem2(gs[i][j], gc[i][j], sred, NE, i + j * BM);
    __syncthreads();
    double* pout = partial + ((size_t)blockIdx.y * nchunks + blockIdx.x) * pstride;
    for (int e = threadIdx.x; e < b * b; e += kThreads) {
        const int i = e % b, j = e / b;
        const int lo = i < j ? i : j, hi = i < j ? j : i;
        pout[e] = cta_entry(sred, NE, lo + hi * BM);
    }
}

template <typename T>
void launch_block_gram(const UpdTask<T>* tasks, int ntasks, int64_t n, KGeom g, double* partial, int pstride,
                       cudaStream_t s) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    k_block_gram<T><<<grid, kThreads, 0, s>>>(tasks, n, g.rows, g.nchunks, pstride, partial);
}

// =====================================================================================
// Sum of per-CTA partials into a dense FP64 block of each window's slab:
// out(task) = wd + wins[task] * stride + off, entries [0, ne).
// =====================================================================================
__global__ void __launch_bounds__(kThreads) k_sum_parts(const double* __restrict__ part, int nchunks, int pstride, int e0,
                                                        int ne, double* __restrict__ wd, int64_t stride, int64_t off,
                                                        const int* __restrict__ wins, const int* __restrict__ wi,
                                                        int istride, int conv_field) {
    pdl_entry();
    if (wi && wi[(int64_t)wins[blockIdx.x] * istride + conv_field]) return;
    const Parts pp{part, nchunks, pstride};
    double* out = wd + (int64_t)wins[blockIdx.x] * stride + off;
    for (int e = threadIdx.x >> 5; e < ne; e += kWarps) {
        const double v = parts_sum_warp(pp, blockIdx.x, e0 + e);
        if ((threadIdx.x & 31) == 0) out[e] = v;
    }
}

// =====================================================================================
// Gram matrix of the source samples of one window: G = X^T X, X = s columns of the
// time-major source (consecutive rows of the n_out x n array).  A row tile of X is
// staged in shared memory; thread t owns entries (a, c), a <= c, and sums FP32
// products with compensation; CTAs write partial Gram matrices (s x s, both halves).
// =====================================================================================
template <typename T, int MAXP>
__global__ void __launch_bounds__(kThreads) k_source_gram(const T* const* __restrict__ Xp, const int* __restrict__ sv,
                                                          int64_t n, int64_t rows, int nchunks, int pstride,
                                                          double* __restrict__ partial) {
    // One thread per Gram entry (a, c), a <= c (up to MAXP of them), a compensated sum over
    // the chunk's rows in order.  The tile is stored row-major with an odd row stride: the
    // lanes of a warp read different columns of one row, which fall in different banks (a
    // column-major tile with a stride of kTile put them all in one bank).
    const int task = blockIdx.y;
    const T* X = Xp[task];
    const int s = sv[task];
    const int ch = blockIdx.x;
    const int64_t r0 = (int64_t)ch * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    extern __shared__ double sh_gram[];
    const int sp = s | 1;
    T* sX = reinterpret_cast<T*>(sh_gram);   // kTile x sp, row k at sX + k * sp
    const int npair = s * (s + 1) / 2;
    // up to MAXP (a, c) pairs per thread: 9 for s <= 64, 25 for s <= 112 (npair <= MAXP kThreads)
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
            const int a = e / kTile, k = e % kTile;   // coalesced along k in global memory
            if (k < nt) sX[k * sp + a] = X[(int64_t)a * n + t0 + k];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < MAXP; ++q) {
            if (q >= np) break;
            const T* xa = sX + pa[q];
            const T* xc = sX + pc[q];
            for (int k = 0; k < nt; ++k) acc[q].add(xa[k * sp], xc[k * sp]);
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
// Part B of a fused step with its small steps folded in (separate launches):
//   k_update0_h:     k_update0 with h1 summed by every CTA from the projection pass's
//                    partials (entries hoff + [0, p B) of its task);
//   k_scale_proj_qr: the first Cholesky QR (k_block_orth pass 1, with the pre-Gram-Schmidt
//                    norms from the projection partials) in every CTA, then k_scale_proj;
//   k_scale_qr:      the second Cholesky QR in every CTA, then k_scale (rounded into the slot).
// The sums run in the fixed order of parts_sum_warp, so every CTA gets the values that the
// separate summing and QR kernels store, and the results are the same bit for bit.  CTA 0
// of each window writes the window's state (the QR's T, kept count, convergence).
// =====================================================================================
constexpr int kH1Max = PEXP_MAX_STEPS * kKrylovMaxB * kKrylovMaxB;   // p B <= 64 * 4 * 4
template <typename T, int B>
__global__ void __launch_bounds__(kThreads, kUpdCtas<B>) k_update0_h(const UpdTask<T>* __restrict__ tasks, int64_t n,
                                                                     int64_t rows, int nchunks, int pstride,
                                                                     double* __restrict__ partial,
                                                                     const double* __restrict__ hpart, int hstride,
                                                                     int hoff) {
    pdl_entry();
    __shared__ double sH[kH1Max];
    const UpdTask<T> tk0 = tasks[blockIdx.y];
    if (tk0.conv && *tk0.conv) return;
    const int p = tk0.p;
    const Parts hp{hpart, nchunks, hstride};
    for (int e = threadIdx.x >> 5; e < p * B; e += kWarps) {
        const double v = parts_sum_warp(hp, blockIdx.y, hoff + e);
        if ((threadIdx.x & 31) == 0) sH[e] = v;
    }
    __syncthreads();
    UpdTask<T> tk = tk0;
    tk.hm = sH;
    tk.ldh = p;
    k_update0_body<T, B>(tk, n, rows, nchunks, pstride, partial, blockIdx.x, blockIdx.y);
}

template <typename T, int B>
__global__ void __launch_bounds__(kThreads, kScaleProjCtas<B>) k_scale_proj_qr(
    const UpdTask<T>* __restrict__ tasks, int64_t n, int64_t rows, int nchunks, int pstride, double* __restrict__ partial,
    WinLayout L, double* __restrict__ wd, int* __restrict__ wi, const int* __restrict__ wins, int step, double defl,
    const double* __restrict__ gpart, int gstride, const double* __restrict__ ppart, int ppstride, int pre_off) {
    pdl_entry();
    const UpdTask<T> tk0 = tasks[blockIdx.y];
    if (tk0.conv && *tk0.conv) return;
    __shared__ double sG[B * B], sT[B * B], spre[B];
    __shared__ int s_r;
    const int w = wins[blockIdx.y];
    double* D = wd + (int64_t)w * L.stride;
    int* I = wi + (int64_t)w * L.istride;
    if (threadIdx.x < 32) {
        const int r = block_orth_body<B>(L, D, I, blockIdx.y, 1, step, defl, Parts{gpart, nchunks, gstride}, -1, sG, sT,
                                      blockIdx.x == 0, Parts{ppart, nchunks, ppstride}, pre_off, spre);
        if (threadIdx.x == 0) {
            s_r = r;
            if (blockIdx.x == 0)
                for (int e = 0; e < B * B; ++e) D[L.off_T + e] = sT[e];
        }
    }
    __syncthreads();
    if (s_r == 0) return;   // no direction kept: CTA 0 marked the window converged
    UpdTask<T> tk = tk0;
    tk.hm = sT;
    tk.ldh = B;
    k_scale_proj_body<T, B>(tk, n, rows, nchunks, pstride, partial, blockIdx.x, blockIdx.y);
}

template <typename T, int B>
__global__ void __launch_bounds__(kThreads, 2) k_scale_qr(const UpdTask<T>* __restrict__ tasks, int64_t n, int64_t rows,
                                                         int nchunks, WinLayout L, double* __restrict__ wd,
                                                         int* __restrict__ wi, const int* __restrict__ wins, int step,
                                                         double defl, const double* __restrict__ gpart, int gstride) {
    pdl_entry();
    const UpdTask<T> tk0 = tasks[blockIdx.y];
    if (tk0.conv && *tk0.conv) return;
    __shared__ double sG[B * B], sT[B * B];
    const int w = wins[blockIdx.y];
    double* D = wd + (int64_t)w * L.stride;
    int* I = wi + (int64_t)w * L.istride;
    if (threadIdx.x < 32) {
        block_orth_body<B>(L, D, I, blockIdx.y, 2, step, defl, Parts{gpart, nchunks, gstride}, -1, sG, sT, blockIdx.x == 0);
        if (threadIdx.x == 0 && blockIdx.x == 0)
            for (int e = 0; e < B * B; ++e) D[L.off_T + e] = sT[e];
    }
    __syncthreads();
    UpdTask<T> tk = tk0;
    tk.hm = sT;
    tk.ldh = B;
    k_scale_body<T, B>(tk, n, rows, nchunks, 0, 0, nullptr, blockIdx.x, blockIdx.y);
}

// =====================================================================================
// k_gs_coop: part B of a fused Krylov step (the four passes above and the two Cholesky QRs
// between them) for one window in one cooperative launch.  CTAs take chunks blockIdx.x,
// blockIdx.x + gridDim.x, ... of the same row geometry and meet at grid barriers, so every
// partial sum, and every result, is the one the separate launches produce.  The Cholesky
// QRs run in every CTA from the same fixed-order sums (CTA 0 alone writes the window's
// state).  The partial sums of the three passes go to three separate regions of kp, since a
// CTA may still be summing one pass's partials while another writes the next pass's.
// The convergence flag is read once at entry: the projected solve on the other stream may
// set it while this kernel runs, and every CTA must still reach every barrier.
// =====================================================================================
template <typename T, int B>
__global__ void __launch_bounds__(kThreads, 3) k_gs_coop(UpdTask<T> u1, UpdTask<T> u3, UpdTask<T> u2, UpdTask<T> u4,
                                                         int64_t n, int64_t rows, int nchunks, double* __restrict__ kp,
                                                         int ps2, int psg, WinLayout L, double* __restrict__ wd,
                                                         int* __restrict__ wi, int w, int step, double defl,
                                                         GridBar bar) {
    bool active = !(u1.conv && *(volatile const int*)u1.conv);
    double* D = wd + (int64_t)w * L.stride;
    int* I = wi + (int64_t)w * L.istride;
    double* pg1 = kp;
    double* ph2 = pg1 + (size_t)nchunks * psg;
    double* pg2 = ph2 + (size_t)nchunks * ps2;
    __shared__ double sG[B * B], sT1[B * B], sT2[B * B];
    __shared__ int s_r;
    // pass 1: W <- W - V h1 (h1 stored by the projection pass), Gram partials
    if (active)
        for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) k_update0_body<T, B>(u1, n, rows, nchunks, psg, pg1, ch, 0);
    if (!grid_bar(bar)) return;
    if (active && threadIdx.x < 32) {
        const int r = block_orth_body<B>(L, D, I, 0, 1, step, defl, Parts{pg1, nchunks, psg}, -1, sG, sT1, blockIdx.x == 0);
        if (threadIdx.x == 0) {
            s_r = r;
            if (blockIdx.x == 0)
                for (int e = 0; e < B * B; ++e) D[L.off_T + e] = sT1[e];
        }
    }
    __syncthreads();
    const int r1 = active ? s_r : 0;
    if (r1 == 0) active = false;   // no direction kept: CTA 0 marked the window converged
    // W <- W T1, h2 partials
    UpdTask<T> t3 = u3;
    t3.hm = sT1;
    t3.ldh = B;
    if (active)
        for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x) k_scale_proj_body<T, B>(t3, n, rows, nchunks, ps2, ph2, ch, 0);
    if (!grid_bar(bar)) return;
    // pass 2: W <- W - V h2 (h2 summed from the partials by every CTA), Gram partials
    if (active)
        for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x)
            k_update1_body<T, B>(u2, n, rows, nchunks, psg, pg2, ph2, ps2, ch, 0);
    if (!grid_bar(bar)) return;
    if (active && threadIdx.x < 32) {
        block_orth_body<B>(L, D, I, 0, 2, step, defl, Parts{pg2, nchunks, psg}, r1, sG, sT2, blockIdx.x == 0);
        if (threadIdx.x == 0 && blockIdx.x == 0)
            for (int e = 0; e < B * B; ++e) D[L.off_T + e] = sT2[e];
    }
    __syncthreads();
    // W T2 rounded into the basis slot
    UpdTask<T> t4 = u4;
    t4.hm = sT2;
    t4.ldh = B;
    if (active)
        for (int ch = blockIdx.x; ch < nchunks; ch += gridDim.x)
            k_scale_body<T, B>(t4, n, rows, nchunks, 0, psg, nullptr, ch, 0);
}

// =====================================================================================
// launchers
// =====================================================================================
KGeom krylov_geom(int ntasks, int64_t n) {
    // 1024 .. 8192 rows per CTA; batches of many tasks take the 8192-row floor, and a
    // single task (one window of the homogeneous chain) is cut into 3 chunks per SM, so
    // that its launches run in one wave at the 3 CTAs per SM its kernels are built for
    KGeom g;
    const int64_t lo = std::max<int64_t>(1, (n + 8191) / 8192);
    const int64_t hi = std::max<int64_t>(1, (n + 1023) / 1024);
    const int64_t want = (3 * kNumSM + ntasks - 1) / std::max(1, ntasks);
    const int64_t ch = std::min(std::max(want, lo), hi);
    g.rows = (n + ch - 1) / ch;
    g.rows = (g.rows + kTile - 1) / kTile * kTile;
    g.nchunks = (int)((n + g.rows - 1) / g.rows);
    return g;
}

size_t krylov_partial_slots(int ntasks_max, int64_t n) {
    // ntasks * nchunks(ntasks) <= ntasks * ceil(n / 8192) + 3 * kNumSM + ntasks for every ntasks <= ntasks_max
    const int64_t lo = std::max<int64_t>(1, (n + 8191) / 8192);
    return (size_t)ntasks_max * (size_t)(lo + 1) + 8 * kNumSM + 64;
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
void launch_step_proj(const StepTask<T>* tasks, int ntasks, int b, int p, int64_t n, int periodic, KGeom g,
                      double* partial, int pstride, cudaStream_t s, bool jac) {
    if (ntasks <= 0) return;
    if (jac) {
        PEXP_B_DISPATCH(b, ({
            constexpr int PG = Group<T, BB, true>::step;
            dim3 grid(g.nchunks, ntasks, (p + PG - 1) / PG);
            launch_pdl(k_step_proj<T, BB, true>, grid, dim3(kThreads), 0, s, tasks, n, periodic, g.rows, g.nchunks, pstride,
                       partial);
        }));
        return;
    }
    PEXP_B_DISPATCH(b, ({
        constexpr int PG = Group<T, BB>::step;
        dim3 grid(g.nchunks, ntasks, (p + PG - 1) / PG);
        launch_pdl(k_step_proj<T, BB, false>, grid, dim3(kThreads), 0, s, tasks, n, periodic, g.rows, g.nchunks, pstride, partial);
    }));
}

bool proj_fused(int p, int b, size_t tsize) { return p <= kFuseP && (size_t)p * b * tsize <= 128; }

template <typename T>
void launch_update(const UpdTask<T>* tasks, int ntasks, int b, int p, int64_t n, int mode, KGeom g, double* partial,
                   int pstride, cudaStream_t s, const double* hpart, int hstride) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    if (mode == 0) {
        const size_t sm = (size_t)p * b * (sizeof(T) == 4 ? sizeof(float2) : sizeof(double)) + 16;
        PEXP_B_DISPATCH(b, (launch_pdl(k_update0<T, BB>, grid, dim3(kThreads), sm, s, tasks, n, g.rows, g.nchunks, pstride, partial)));
    } else {
        const size_t sm = (size_t)p * b * sizeof(T) + 16;
        PEXP_B_DISPATCH(b, (launch_pdl(k_update1<T, BB>, grid, dim3(kThreads), sm, s, tasks, n, g.rows, g.nchunks, pstride,
                                       partial, hpart, hstride)));
    }
}

template <typename T>
void launch_scale_proj(const UpdTask<T>* tasks, int ntasks, int b, int p, int64_t n, KGeom g, double* partial,
                       int pstride, cudaStream_t s) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    if (proj_fused(p, b, sizeof(T))) {
        PEXP_B_DISPATCH(b, (launch_pdl(k_scale_proj<T, BB>, grid, dim3(kThreads), 0, s, tasks, n, g.rows, g.nchunks, pstride, partial)));
    } else {
        PEXP_B_DISPATCH(b, ({
            launch_pdl(k_scale<T, BB>, grid, dim3(kThreads), 0, s, tasks, n, g.rows, g.nchunks, 0, pstride, (double*)nullptr);
            constexpr int PG = Group<T, BB>::vtw;
            dim3 g3(g.nchunks, ntasks, (p + PG - 1) / PG);
            k_vtw<T, BB><<<g3, kThreads, 0, s>>>(tasks, n, g.rows, g.nchunks, pstride, partial);
        }));
    }
}

template <typename T>
void launch_scale(const UpdTask<T>* tasks, int ntasks, int b, int64_t n, int gram, KGeom g, double* partial,
                  int pstride, cudaStream_t s) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    PEXP_B_DISPATCH(b, (launch_pdl(k_scale<T, BB>, grid, dim3(kThreads), 0, s, tasks, n, g.rows, g.nchunks, gram, pstride, partial)));
}

void launch_sum_parts(const double* part, int nchunks, int pstride, int ne, double* wd, int64_t stride, int64_t off,
                      const int* wins, int ntasks, const int* wi, int istride, int conv_field, cudaStream_t s, int e0) {
    if (ntasks <= 0 || ne <= 0) return;
    launch_pdl(k_sum_parts, dim3(ntasks), dim3(kThreads), 0, s, part, nchunks, pstride, e0, ne, wd, stride, off, wins, wi, istride,
                                            conv_field);
}

template <typename T>
void launch_source_gram(const T* const* X, const int* sv, int ntasks, int s_max, int64_t n, KGeom g, double* partial,
                        int pstride, cudaStream_t st) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    // the sample tile: kTile rows of stride s_max | 1
    const size_t sm = sizeof(T) * (size_t)(s_max | 1) * kTile;
    static_assert(64 * 65 / 2 <= 9 * kThreads && 112 * 113 / 2 <= 25 * kThreads, "Gram pairs per thread");
    if (s_max <= 64) {
        if (sm > 32 * 1024) smem_optin(k_source_gram<T, 9>, sm);
        k_source_gram<T, 9><<<grid, kThreads, sm, st>>>(X, sv, n, g.rows, g.nchunks, pstride, partial);
    } else {
        if (sm > 32 * 1024) smem_optin(k_source_gram<T, 25>, sm);
        k_source_gram<T, 25><<<grid, kThreads, sm, st>>>(X, sv, n, g.rows, g.nchunks, pstride, partial);
    }
}

template <typename T>
void launch_update0_h(const UpdTask<T>* tasks, int ntasks, int b, int p, int64_t n, KGeom g, double* partial,
                      int pstride, const double* hpart, int hstride, int hoff, cudaStream_t s) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    const size_t sm = (size_t)p * b * (sizeof(T) == 4 ? sizeof(float2) : sizeof(double)) + 16;
    PEXP_B_DISPATCH(b, (launch_pdl(k_update0_h<T, BB>, grid, dim3(kThreads), sm, s, tasks, n, g.rows, g.nchunks, pstride,
                                   partial, hpart, hstride, hoff)));
}

template <typename T>
void launch_scale_proj_qr(const UpdTask<T>* tasks, int ntasks, int b, int64_t n, KGeom g, double* partial, int pstride,
                          const WinLayout& L, double* wd, int* wi, const int* wins, int step, double defl,
                          const double* gpart, int gstride, const double* ppart, int ppstride, int pre_off,
                          cudaStream_t s) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    PEXP_B_DISPATCH(b, (launch_pdl(k_scale_proj_qr<T, BB>, grid, dim3(kThreads), 0, s, tasks, n, g.rows, g.nchunks,
                                   pstride, partial, L, wd, wi, wins, step, defl, gpart, gstride, ppart, ppstride,
                                   pre_off)));
}

template <typename T>
void launch_scale_qr(const UpdTask<T>* tasks, int ntasks, int b, int64_t n, KGeom g, const WinLayout& L, double* wd,
                     int* wi, const int* wins, int step, double defl, const double* gpart, int gstride, cudaStream_t s) {
    if (ntasks <= 0) return;
    dim3 grid(g.nchunks, ntasks);
    PEXP_B_DISPATCH(b, (launch_pdl(k_scale_qr<T, BB>, grid, dim3(kThreads), 0, s, tasks, n, g.rows, g.nchunks, L, wd, wi,
                                   wins, step, defl, gpart, gstride)));
}

template <typename T>
bool launch_gs_coop(const UpdTask<T>* u, int b, int p, int64_t n, KGeom g, double* kp, int ps2, int psg,
                    const WinLayout& L, double* wd, int* wi, int w, int step, double defl, GridBar bar, cudaStream_t s) {
    if (b != 1 || !proj_fused(p, b, sizeof(T))) return false;
    constexpr int BB = 1;
    const size_t sm = (size_t)p * BB * (sizeof(T) == 4 ? sizeof(float2) : sizeof(double)) + 16;
    const void* fn = reinterpret_cast<const void*>(k_gs_coop<T, BB>);
    const size_t sm_max = (size_t)kFuseP * BB * (sizeof(T) == 4 ? sizeof(float2) : sizeof(double)) + 16;
    const int grid = coop_grid(fn, kThreads, sm_max, g.nchunks);
    if (grid <= 0) return false;
    UpdTask<T> u1 = u[0], u3 = u[1], u2 = u[2], u4 = u[3];
    int64_t nn = n, rows = g.rows;
    int nch = g.nchunks, a2 = ps2, ag = psg, ww = w, st = step;
    WinLayout LL = L;
    double dd = defl;
    void* args[] = {&u1, &u3, &u2, &u4, &nn, &rows, &nch, &kp, &a2, &ag, &LL, &wd, &wi, &ww, &st, &dd, &bar};
    if (cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kThreads), args, sm, s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

#define PEXP_KRY_INST(T)                                                                                           \
    template void launch_update0_h<T>(const UpdTask<T>*, int, int, int, int64_t, KGeom, double*, int, const double*, int, \
                                      int, cudaStream_t);                                                          \
    template void launch_scale_proj_qr<T>(const UpdTask<T>*, int, int, int64_t, KGeom, double*, int, const WinLayout&,   \
                                          double*, int*, const int*, int, double, const double*, int, const double*, int, \
                                          int, cudaStream_t);                                                      \
    template void launch_scale_qr<T>(const UpdTask<T>*, int, int, int64_t, KGeom, const WinLayout&, double*, int*,       \
                                     const int*, int, double, const double*, int, cudaStream_t);                    \
    template bool launch_gs_coop<T>(const UpdTask<T>*, int, int, int64_t, KGeom, double*, int, int, const WinLayout&, \
                                    double*, int*, int, int, double, GridBar, cudaStream_t);               \
    template void launch_step_proj<T>(const StepTask<T>*, int, int, int, int64_t, int, KGeom, double*, int, cudaStream_t, bool); \
    template void launch_update<T>(const UpdTask<T>*, int, int, int, int64_t, int, KGeom, double*, int, cudaStream_t, \
                                   const double*, int);                                                             \
    template void launch_scale<T>(const UpdTask<T>*, int, int, int64_t, int, KGeom, double*, int, cudaStream_t); \
    template void launch_scale_proj<T>(const UpdTask<T>*, int, int, int, int64_t, KGeom, double*, int, cudaStream_t); \
    template void launch_block_gram<T>(const UpdTask<T>*, int, int64_t, KGeom, double*, int, cudaStream_t); \
    template void launch_source_gram<T>(const T* const*, const int*, int, int, int64_t, KGeom, double*, int, cudaStream_t);
PEXP_KRY_INST(double)
PEXP_KRY_INST(float)

}  // namespace pexp
