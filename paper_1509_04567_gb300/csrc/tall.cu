// Kernels over n-length data for the PEBK hot path (sm_103a).
//
//  * central-difference stencil Y = A X (Sec. 3.1), 1D/2D, periodic/Dirichlet;
//  * shift-and-invert solve Y = (I - gamma A)^{-1} X (Sec. 2.1) for 1D periodic A;
//  * batched tall-skinny products X^T Y (projections, Gram matrices) and
//    X T (block updates) used by block Gram-Schmidt and the source compression;
//  * reconstruction u(t_i) = u0 + V y(t_i) (eq. superposition);
//  * Burgers nonlinear source -u u_x (Sec. 4) and small helpers.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>

#include "common.cuh"
#include "sai.cuh"

namespace pexp {

void smem_optin_raw(const void* kernel, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> cap;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    size_t& c = cap[{dev, kernel}];
    if (bytes > c) {
        cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        c = bytes;
    }
}

int coop_grid(const void* kernel, int threads, size_t smem, int want) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, int> cap;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    auto it = cap.find({dev, kernel});
    if (it == cap.end()) {
        int coop = 0, sms = 0, per = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem) != cudaSuccess) {
            cudaGetLastError();
            per = 0;
        }
        it = cap.emplace(std::make_pair(dev, kernel), coop ? per * sms : 0).first;
    }
    return it->second <= 0 ? 0 : std::min(want, it->second);
}

int fail_cuda(cudaError_t e, const char* what, const char* file, int line) {
    fprintf(stderr, "pexp: CUDA error %s (%d) in %s at %s:%d\n", cudaGetErrorString(e), (int)e, what, file,
            line);
    return PEXP_ERR_CUDA;
}

static int grid_for(int64_t work, int threads, int per_thread = 1) {
    int64_t b = (work + (int64_t)threads * per_thread - 1) / ((int64_t)threads * per_thread);
    if (b < 1) b = 1;
    if (b > 65535LL * 8) b = 65535LL * 8;
    return (int)b;
}

// =====================================================================================
// Stencil
// =====================================================================================
template <typename T>
__device__ __forceinline__ T stencil_at(const OpDesc& op, const T* __restrict__ x, int64_t k, int transpose) {
    const T u = x[k];
    T acc = T(0);
    {
        const Dim1& D = op.x;
        int64_t ix = (op.dim == 1) ? k : (k % D.n);
        T um, up;
        if (ix > 0) um = x[k - 1];
        else um = D.periodic ? x[k + D.n - 1] : T(0);
        if (ix < D.n - 1) up = x[k + 1];
        else up = D.periodic ? x[k - (D.n - 1)] : T(0);
        const T d = T(D.d), c = transpose ? T(-D.c) : T(D.c);
        acc = d * ((um - u) + (up - u)) - c * (up - um);
    }
    if (op.dim == 2) {
        const Dim1& D = op.y;
        int64_t iy = k / op.x.n;
        T um, up;
        if (iy > 0) um = x[k - D.stride];
        else um = D.periodic ? x[k + (D.n - 1) * D.stride] : T(0);
        if (iy < D.n - 1) up = x[k + D.stride];
        else up = D.periodic ? x[k - (D.n - 1) * D.stride] : T(0);
        const T d = T(D.d), c = transpose ? T(-D.c) : T(D.c);
        acc += d * ((um - u) + (up - u)) - c * (up - um);
    }
    return acc;
}

template <typename T>
__global__ void __launch_bounds__(256) k_stencil(OpDesc op, const T* const* __restrict__ Xp,
                                                 T* const* __restrict__ Yp, const T* Xb, T* Yb,
                                                 int transpose) {
    const int v = blockIdx.y;
    const T* x = Xp ? Xp[v] : Xb + (int64_t)v * op.n;
    T* y = Yp ? Yp[v] : Yb + (int64_t)v * op.n;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < op.n;
         k += (int64_t)gridDim.x * blockDim.x)
        y[k] = stencil_at(op, x, k, transpose);
}

template <typename T>
void launch_stencil(const OpDesc& op, const T* X, T* Y, int nvec, int transpose, cudaStream_t s) {
    if (nvec <= 0) return;
    dim3 g(std::min(grid_for(op.n, 256), std::max(1, 4 * kNumSM * 8 / nvec + 1)), nvec);
    k_stencil<T><<<g, 256, 0, s>>>(op, nullptr, nullptr, X, Y, transpose);
}

template <typename T>
void launch_stencil_ptrs(const OpDesc& op, const T* const* X, T* const* Y, int nvec, int transpose,
                         cudaStream_t s) {
    if (nvec <= 0) return;
    dim3 g(std::min(grid_for(op.n, 256), std::max(1, 4 * kNumSM * 8 / nvec + 1)), nvec);
    k_stencil<T><<<g, 256, 0, s>>>(op, X, Y, nullptr, nullptr, transpose);
}

// Double-float stencil for FP32 data: (hi, lo) = A x or A^T x to ~2^-48 relative,
// from the exact FP32 values of x.  The Galerkin matrix V^T A V of the FP32 basis is
// built from these: rounding A x to FP32 would perturb it by far more than the
// basis rounding itself, because A amplifies the high-frequency part of x.
struct DF2 {
    float hi, lo;
};
__device__ __forceinline__ DF2 two_diff(float a, float b) {
    const float s = a - b;
    const float bb = s - a;
    const float e = (a - (s - bb)) - (b + bb);
    return DF2{s, e};
}
__device__ __forceinline__ DF2 df2_add(DF2 a, DF2 b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
    const float h = s + e;
    return DF2{h, e - (h - s)};
}
__device__ __forceinline__ DF2 df2_mul(DF2 a, DF2 b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float h = p + e;
    return DF2{h, e - (h - p)};
}
__device__ __forceinline__ DF2 df2_from(double v) {
    const float h = (float)v;
    return DF2{h, (float)(v - (double)h)};
}

__device__ __forceinline__ DF2 stencil_df_dim(const Dim1& D, const float* __restrict__ x, const float* __restrict__ xl,
                                             int64_t k, int64_t idx, float u, float ul, int transpose) {
    float um, up, uml = 0.f, upl = 0.f;
    int64_t km = -1, kp = -1;
    if (idx > 0) km = k - D.stride;
    else if (D.periodic) km = k + (D.n - 1) * D.stride;
    if (idx < D.n - 1) kp = k + D.stride;
    else if (D.periodic) kp = k - (D.n - 1) * D.stride;
    um = km >= 0 ? x[km] : 0.f;
    up = kp >= 0 ? x[kp] : 0.f;
    if (xl) {
        uml = km >= 0 ? xl[km] : 0.f;
        upl = kp >= 0 ? xl[kp] : 0.f;
    }
    // differences of (hi + lo) values: exact hi difference plus the lo difference
    const DF2 dm = df2_add(two_diff(um, u), DF2{uml - ul, 0.f});
    const DF2 dp = df2_add(two_diff(up, u), DF2{upl - ul, 0.f});
    const DF2 dc = df2_add(two_diff(up, um), DF2{upl - uml, 0.f});
    const DF2 d = df2_from(D.d), c = df2_from(transpose ? -D.c : D.c);
    const DF2 t1 = df2_mul(d, df2_add(dm, dp));
    const DF2 t2 = df2_mul(c, dc);
    return df2_add(t1, DF2{-t2.hi, -t2.lo});
}

__global__ void __launch_bounds__(256) k_stencil_df(OpDesc op, const float* const* __restrict__ Xp,
                                                   const float* const* __restrict__ Xl,
                                                   float* const* __restrict__ Yh, float* const* __restrict__ Yl,
                                                   int transpose) {
    const int v = blockIdx.y;
    const float* x = Xp[v];
    const float* xl = Xl ? Xl[v] : nullptr;
    float* yh = Yh[v];
    float* yl = Yl[v];
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < op.n; k += (int64_t)gridDim.x * blockDim.x) {
        const float u = x[k];
        const float ul = xl ? xl[k] : 0.f;
        DF2 r = stencil_df_dim(op.x, x, xl, k, (op.dim == 1) ? k : (k % op.x.n), u, ul, transpose);
        if (op.dim == 2) r = df2_add(r, stencil_df_dim(op.y, x, xl, k, k / op.x.n, u, ul, transpose));
        yh[k] = r.hi;
        yl[k] = r.lo;
    }
}

void launch_stencil_df(const OpDesc& op, const float* const* X, const float* const* Xl, float* const* Yh,
                       float* const* Yl, int nvec, int transpose, cudaStream_t s) {
    if (nvec <= 0) return;
    dim3 g(std::min(grid_for(op.n, 256), std::max(1, 4 * kNumSM * 8 / nvec + 1)), nvec);
    k_stencil_df<<<g, 256, 0, s>>>(op, X, Xl, Yh, Yl, transpose);
}

// =====================================================================================
// Burgers source g = -u u_x (Sec. 4), conservative or advective central form
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(256) k_burgers(OpDesc op, const T* __restrict__ U, T* __restrict__ G,
                                                 int form, double inv2dx) {
    const int64_t row = blockIdx.y;
    const T* u = U + row * op.n;
    T* g = G + row * op.n;
    const int periodic = op.x.periodic;
    const T h2 = T(inv2dx);
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < op.n;
         k += (int64_t)gridDim.x * blockDim.x) {
        T um, up;
        if (k > 0) um = u[k - 1];
        else um = periodic ? u[op.n - 1] : T(0);
        if (k < op.n - 1) up = u[k + 1];
        else up = periodic ? u[0] : T(0);
        if (form == 0) g[k] = -(up - um) * (up + um) * (h2 * T(0.5));   // -(u_{k+1}^2 - u_{k-1}^2)/(4 dx)
        else g[k] = -u[k] * (up - um) * h2;                               // -u_k (u_{k+1} - u_{k-1})/(2 dx)
    }
}

template <typename T>
void launch_burgers_source(const OpDesc& op, const T* U, T* G, int nrows, int form, double inv2dx,
                           cudaStream_t s) {
    if (nrows <= 0) return;
    dim3 g(std::min(grid_for(op.n, 256), std::max(1, 4 * kNumSM * 8 / nrows + 1)), nrows);
    k_burgers<T><<<g, 256, 0, s>>>(op, U, G, form, inv2dx);
}

// =====================================================================================
// Shift-and-invert solve for a 1D periodic operator.
//
// (I - gamma A) has constant diagonals p (sub), q (main), r (super) and wraps
// around.  It factors as c (I - alpha S^{-1})(I - beta S) with S the cyclic
// shift, |alpha|, |beta| < 1, c = (q + sqrt(q^2 - 4 p r)) / 2, alpha = -p/c,
// beta = -r/c.  So y = (1/c) x with
//     w_i = v_i + alpha w_{i-1}      (forward, circular)
//     x_i = w_i + beta  x_{i+1}      (backward, circular)
// Each recurrence is a scan of affine maps f(z) = a z + b: chunks of 2048
// elements per CTA (8 per thread), a CTA-wide scan, and a circular sum over
// chunk summaries for the carry into each chunk (terms decay like alpha^2048).
// Three passes, each reading the input: forward chunk summaries; forward values
// in registers -> backward chunk summaries (w is not stored); forward values
// again (the same arithmetic, so the same w) -> backward values -> output.
// =====================================================================================

SaiCoef sai_coefficients(const OpDesc& op, double gamma) {
    const Dim1& D = op.x;
    // (A u)_i = (d + c) u_{i-1} - 2 d u_i + (d - c) u_{i+1}
    const double p = -gamma * (D.d + D.c);
    const double q = 1.0 + 2.0 * gamma * D.d;
    const double r = -gamma * (D.d - D.c);
    const double disc = q * q - 4.0 * p * r;
    const double c = 0.5 * (q + sqrt(disc));
    SaiCoef cf;
    cf.alpha = -p / c;
    cf.beta = -r / c;
    cf.inv_c = 1.0 / c;
    cf.alpha_n = pow(cf.alpha, (double)D.n);
    cf.beta_n = pow(cf.beta, (double)D.n);
    return cf;
}

size_t sai_scratch_doubles(int64_t n, int nvec) {
    const int64_t nch = (n + kSaiChunk - 1) / kSaiChunk;
    return (size_t)4 * nch * nvec;
}

// Resident CTAs per SM the three passes are built for (48 registers): their CTA scans are
// latency-bound, so more CTAs in flight hide more of it.
constexpr int kSaiCtas = 5;

// Pass 1: chunk summaries of the forward recurrence with zero carry-in (chunk ch of vector v).
template <typename T>
__device__ __forceinline__ void sai_fwd_ends_body(int64_t n, int nch, double alpha, const T* x, const T* xl,
                                                  double* __restrict__ ends, double* __restrict__ decays, int v,
                                                  int ch) {
    using R = typename SaiR<T>::R;
    __shared__ R sa[kSaiThreads], sb[kSaiThreads];
    const int64_t start = (int64_t)ch * kSaiChunk + (int64_t)threadIdx.x * kSaiPer;
    T vals[kSaiPer], lows[kSaiPer];
    const int cnt = sai_load(x, n, start, vals);
    if (xl) sai_load(xl, n, start, lows);
    const R al = rfrom<R>(alpha);
    R b = rfrom<R>(0.0);
#pragma unroll
    for (int j = 0; j < kSaiPer; ++j)
        if (j < cnt) b = rfma(al, b, load_r<T, R>(vals[j], xl ? lows[j] : T(0)));
    R a = ipow(al, cnt);
    R ea, eb, ta, tb;
    cta_affine_scan<R>(a, b, false, sa, sb, ea, eb, ta, tb);
    if (threadIdx.x == 0) {
        ends[(int64_t)v * nch + ch] = rdbl(tb);
        decays[(int64_t)v * nch + ch] = rdbl(ta);
    }
}

// Pass 2: forward values with carries (kept in registers) -> summaries of the
// backward recurrence of w with zero carry from the right.
template <typename T>
__device__ __forceinline__ void sai_fwd_apply_body(int64_t n, int nch, double alpha, double beta, double alpha_n,
                                                   const T* x, const T* xl, const double* __restrict__ fends,
                                                   const double* __restrict__ fdecays, double* __restrict__ bends,
                                                   double* __restrict__ bdecays, int v, int ch) {
    using R = typename SaiR<T>::R;
    __shared__ R sa[kSaiThreads], sb[kSaiThreads];
    __shared__ double carry_in;
    const int64_t start = (int64_t)ch * kSaiChunk + (int64_t)threadIdx.x * kSaiPer;
    T vals[kSaiPer], lows[kSaiPer];
    const int cnt = sai_load(x, n, start, vals);
    if (xl) sai_load(xl, n, start, lows);
    // warp 0 computes the carry while the loads are in flight; it is read after the first scan
    if (threadIdx.x < 32) {
        const double cv = sai_carry_warp(fends + (int64_t)v * nch, fdecays + (int64_t)v * nch, nch, ch, +1, alpha_n);
        if (threadIdx.x == 0) carry_in = cv;
    }
    R wv[kSaiPer];
    sai_forward_values<T, R>(vals, lows, xl != nullptr, cnt, rfrom<R>(alpha), &carry_in, sa, sb, wv);
    const R be = rfrom<R>(beta);
    R gb = rfrom<R>(0.0);
#pragma unroll
    for (int j = kSaiPer - 1; j >= 0; --j)
        if (j < cnt) gb = rfma(be, gb, wv[j]);
    R ga = ipow(be, cnt);
    R ea, eb, ta, tb;
    cta_affine_scan<R>(ga, gb, true, sa, sb, ea, eb, ta, tb);
    if (threadIdx.x == 0) {
        bends[(int64_t)v * nch + ch] = rdbl(tb);
        bdecays[(int64_t)v * nch + ch] = rdbl(ta);
    }
}

// Pass 3: the forward values again (same inputs and arithmetic as pass 2, so the
// same w), then the backward recurrence with carries, scaled by 1/c, into Y.
template <typename T>
__device__ __forceinline__ void sai_bwd_apply_body(int64_t n, int nch, double alpha, double alpha_n, double beta,
                                                   double beta_n, double inv_c, const T* x, const T* xl, T* y, T* ylo,
                                                   const double* __restrict__ fends,
                                                   const double* __restrict__ fdecays,
                                                   const double* __restrict__ bends,
                                                   const double* __restrict__ bdecays, int v, int ch) {
    using R = typename SaiR<T>::R;
    __shared__ R sa[kSaiThreads], sb[kSaiThreads];
    __shared__ double carry_f, carry_b;
    const int64_t start = (int64_t)ch * kSaiChunk + (int64_t)threadIdx.x * kSaiPer;
    T vals[kSaiPer], lows[kSaiPer];
    const int cnt = sai_load(x, n, start, vals);
    if (xl) sai_load(xl, n, start, lows);
    // the two carries side by side while the loads are in flight: warp 0 the forward one (read
    // after the first scan), warp 1 the backward one (read after the second)
    if (threadIdx.x < 32) {
        const double cf = sai_carry_warp(fends + (int64_t)v * nch, fdecays + (int64_t)v * nch, nch, ch, +1, alpha_n);
        if (threadIdx.x == 0) carry_f = cf;
    } else if (threadIdx.x < 64) {
        const double cb = sai_carry_warp(bends + (int64_t)v * nch, bdecays + (int64_t)v * nch, nch, ch, -1, beta_n);
        if (threadIdx.x == 32) carry_b = cb;
    }
    R wv[kSaiPer];
    sai_forward_values<T, R>(vals, lows, xl != nullptr, cnt, rfrom<R>(alpha), &carry_f, sa, sb, wv);
    const R be = rfrom<R>(beta);
    R gb = rfrom<R>(0.0);
#pragma unroll
    for (int j = kSaiPer - 1; j >= 0; --j)
        if (j < cnt) gb = rfma(be, gb, wv[j]);
    R ga = ipow(be, cnt);
    R ea, eb, ta, tb;
    cta_affine_scan<R>(ga, gb, true, sa, sb, ea, eb, ta, tb);
    R xv = rfma(ea, rfrom<R>(carry_b), eb);
    const R ic = rfrom<R>(inv_c);
    T oh[kSaiPer], ol[kSaiPer];
#pragma unroll
    for (int j = kSaiPer - 1; j >= 0; --j) {
        if (j < cnt) {
            xv = rfma(be, xv, wv[j]);
            split_r(rmul(xv, ic), ylo != nullptr, oh[j], ol[j]);
        } else {
            oh[j] = ol[j] = T(0);
        }
    }
    sai_store(y, n, start, cnt, oh);
    if (ylo) sai_store(ylo, n, start, cnt, ol);
}

template <typename T>
__global__ void __launch_bounds__(kSaiThreads, kSaiCtas) k_sai_fwd_ends(int64_t n, int nch, double alpha,
                                                              const T* const* __restrict__ Xp,
                                                              const T* const* __restrict__ Xlo,
                                                              double* __restrict__ ends,
                                                              double* __restrict__ decays,
                                                              const int* const* __restrict__ skip) {
    pdl_entry();
    const int v = blockIdx.y;
    if (skip && skip[v] && *skip[v]) return;
    sai_fwd_ends_body<T>(n, nch, alpha, Xp[v], Xlo ? Xlo[v] : nullptr, ends, decays, v, blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(kSaiThreads, kSaiCtas) k_sai_fwd_apply(int64_t n, int nch, double alpha, double beta,
                                                               double alpha_n, const T* const* __restrict__ Xp,
                                                               const T* const* __restrict__ Xlo,
                                                               const double* __restrict__ fends,
                                                               const double* __restrict__ fdecays,
                                                               double* __restrict__ bends,
                                                               double* __restrict__ bdecays,
                                                               const int* const* __restrict__ skip) {
    pdl_entry();
    const int v = blockIdx.y;
    if (skip && skip[v] && *skip[v]) return;
    sai_fwd_apply_body<T>(n, nch, alpha, beta, alpha_n, Xp[v], Xlo ? Xlo[v] : nullptr, fends, fdecays, bends, bdecays, v,
                          blockIdx.x);
}

template <typename T>
__global__ void __launch_bounds__(kSaiThreads, kSaiCtas) k_sai_bwd_apply(int64_t n, int nch, double alpha, double alpha_n,
                                                               double beta, double beta_n, double inv_c,
                                                               const T* const* __restrict__ Xp,
                                                               const T* const* __restrict__ Xlo,
                                                               T* const* __restrict__ Yp, T* const* __restrict__ Ylo,
                                                               const double* __restrict__ fends,
                                                               const double* __restrict__ fdecays,
                                                               const double* __restrict__ bends,
                                                               const double* __restrict__ bdecays,
                                                               const int* const* __restrict__ skip) {
    pdl_entry();
    const int v = blockIdx.y;
    if (skip && skip[v] && *skip[v]) return;
    sai_bwd_apply_body<T>(n, nch, alpha, alpha_n, beta, beta_n, inv_c, Xp[v], Xlo ? Xlo[v] : nullptr, Yp[v],
                          Ylo ? Ylo[v] : nullptr, fends, fdecays, bends, bdecays, v, blockIdx.x);
}

// The three passes of one vector's solve in one cooperative launch: CTAs take chunks
// ch = blockIdx.x, blockIdx.x + gridDim.x, ... in every pass, with the same arithmetic as the
// three kernels above (so the same result), and meet at a grid barrier between passes.
// `skip`: the window's convergence flag, read once at entry (the whole solve is skipped).
template <typename T>
__global__ void __launch_bounds__(kSaiThreads) k_sai_coop(int64_t n, int nch, SaiCoef cf, const T* __restrict__ x,
                                                          T* __restrict__ y, T* __restrict__ ylo,
                                                          double* __restrict__ scr, const int* __restrict__ skip,
                                                          GridBar bar) {
    const bool active = !(skip && *(volatile const int*)skip);
    double* fends = scr;
    double* fdec = fends + nch;
    double* bends = fdec + nch;
    double* bdec = bends + nch;
    if (active)
        for (int ch = blockIdx.x; ch < nch; ch += gridDim.x) sai_fwd_ends_body<T>(n, nch, cf.alpha, x, nullptr, fends, fdec, 0, ch);
    if (!grid_bar(bar)) return;
    // a CTA's chunks run one after another: a barrier between them keeps the next chunk's
    // carries (written by warps 0 and 1) from overtaking the reads of the last chunk's
    if (active)
        for (int ch = blockIdx.x; ch < nch; ch += gridDim.x) {
            sai_fwd_apply_body<T>(n, nch, cf.alpha, cf.beta, cf.alpha_n, x, nullptr, fends, fdec, bends, bdec, 0, ch);
            __syncthreads();
        }
    if (!grid_bar(bar)) return;
    if (active)
        for (int ch = blockIdx.x; ch < nch; ch += gridDim.x) {
            sai_bwd_apply_body<T>(n, nch, cf.alpha, cf.alpha_n, cf.beta, cf.beta_n, cf.inv_c, x, nullptr, y, ylo, fends,
                                  fdec, bends, bdec, 0, ch);
            __syncthreads();
        }
}

template <typename T>
void launch_sai_solve(const OpDesc& op, const SaiCoef& cf, const T* const* X, T* const* Y, T* const* Ylo, int nvec,
                      double* scratch, cudaStream_t s) {
    launch_sai_solve_lo<T>(op, cf, X, nullptr, Y, Ylo, nvec, scratch, s, nullptr);
}

template <typename T>
void launch_sai_solve_lo(const OpDesc& op, const SaiCoef& cf, const T* const* X, const T* const* Xlo, T* const* Y,
                         T* const* Ylo, int nvec, double* scratch, cudaStream_t s, const int* const* skip) {
    if (nvec <= 0) return;
    const int64_t n = op.n;
    const int nch = (int)((n + kSaiChunk - 1) / kSaiChunk);
    double* fends = scratch;
    double* fdec = fends + (size_t)nch * nvec;
    double* bends = fdec + (size_t)nch * nvec;
    double* bdec = bends + (size_t)nch * nvec;
    dim3 g(nch, nvec);
    launch_pdl(k_sai_fwd_ends<T>, g, dim3(kSaiThreads), 0, s, n, nch, cf.alpha, X, Xlo, fends, fdec, skip);
    launch_pdl(k_sai_fwd_apply<T>, g, dim3(kSaiThreads), 0, s, n, nch, cf.alpha, cf.beta, cf.alpha_n, X, Xlo, fends,
               (const double*)fdec, bends, bdec, skip);
    launch_pdl(k_sai_bwd_apply<T>, g, dim3(kSaiThreads), 0, s, n, nch, cf.alpha, cf.alpha_n, cf.beta, cf.beta_n,
               cf.inv_c, X, Xlo, Y, Ylo, (const double*)fends, (const double*)fdec, (const double*)bends,
               (const double*)bdec, skip);
}

template <typename T>
bool launch_sai_coop(const OpDesc& op, const SaiCoef& cf, const T* x, T* y, T* ylo, double* scratch, const int* skip,
                     GridBar bar, cudaStream_t s) {
    int64_t n = op.n;
    int nch = (int)((n + kSaiChunk - 1) / kSaiChunk);
    const int g = coop_grid(reinterpret_cast<const void*>(k_sai_coop<T>), kSaiThreads, 0, nch);
    if (g <= 0) return false;
    SaiCoef c = cf;
    void* args[] = {&n, &nch, &c, &x, &y, &ylo, &scratch, &skip, &bar};
    if (cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_sai_coop<T>), dim3(g), dim3(kSaiThreads), args, 0,
                                    s) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

// Self-test of the bounded grid barrier: the CTAs of a cooperative launch pass `rounds`
// barriers, except CTA `absent` (>= 0), which leaves at once, so that the others' wait runs
// out after its time limit and sets the error word.
__global__ void k_bar_selftest(GridBar bar, int rounds, int absent) {
    if ((int)blockIdx.x == absent) return;
    for (int i = 0; i < rounds; ++i)
        if (!grid_bar(bar)) return;
}

int launch_bar_selftest(GridBar bar, int absent, cudaStream_t s) {
    const int g = coop_grid(reinterpret_cast<const void*>(k_bar_selftest), 256, 0, 64);
    if (g <= 0) return 0;
    int rounds = 4;
    void* args[] = {&bar, &rounds, &absent};
    if (cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_bar_selftest), dim3(g), dim3(256), args, 0, s) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return g;
}

// =====================================================================================
// Batched tall-skinny products
// =====================================================================================
template <typename T>
struct Acc;
template <>
struct Acc<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x, double y) { s = fma(x, y, s); }
    __device__ __forceinline__ double get() const { return s; }
};
// FP32 products summed with Neumaier's compensated summation: the running error
// stays near the FP32 unit roundoff independent of the number of rows.
template <>
struct Acc<float> {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x, float y) {
        const float v = x * y;
        const float t = s + v;
        if (fabsf(s) >= fabsf(v)) c += (s - t) + v;
        else c += (v - t) + s;
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

// FP32 data, exact products (x*y = p + e via FMA) summed in a double-float (hi, lo)
// accumulator: the Gram matrix of FP32 data comes out accurate to ~1e-14.
struct AccDF {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = 0.f; lo = 0.f; }
    __device__ __forceinline__ void add(float x, float y) {
        const float p = x * y;
        const float e = fmaf(x, y, -p);
        const float s = hi + p;
        const float bp = s - hi;
        const float err = (hi - (s - bp)) + (p - bp);
        const float l = lo + (err + e);
        hi = s + l;
        lo = l - (hi - s);
    }
    __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};
template <typename T, bool EXACT>
struct AccSel { using type = Acc<T>; };
template <>
struct AccSel<float, true> { using type = AccDF; };

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

struct TnGeom {
    int nchunks;
    int64_t rows;
};
static TnGeom tn_geom(int ntasks, int64_t n) {
    TnGeom g;
    int want = (4 * kNumSM + ntasks - 1) / ntasks;
    int64_t maxch = (n + 2047) / 2048;
    g.nchunks = (int)std::max<int64_t>(1, std::min<int64_t>(want, maxch));
    g.rows = (n + g.nchunks - 1) / g.nchunks;
    g.rows = (g.rows + 31) / 32 * 32;
    g.nchunks = (int)((n + g.rows - 1) / g.rows);
    return g;
}

// Upper bound for any launch with at most `ntasks` tasks: ntasks * nchunks <= 4*152 + ntasks.
size_t ts_tn_partial_doubles(int ntasks, int max_pq, int64_t n) {
    (void)n;
    return (size_t)(4 * kNumSM + ntasks + 8) * (size_t)max_pq;
}

template <typename T, int GA, int QM, bool EXACT>
__global__ void __launch_bounds__(256) k_ts_tn(const TsTask<T>* __restrict__ tasks, int64_t n, int64_t rows,
                                               int nchunks, int pq_stride, double* __restrict__ partial) {
    const TsTask<T> tk = tasks[blockIdx.y];
    const int ch = blockIdx.x;
    const int64_t r0 = (int64_t)ch * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    double* pout = partial + ((size_t)blockIdx.y * nchunks + ch) * pq_stride;
    const int p = tk.p, q = tk.q, q1 = tk.q1;
    for (int a0 = warp * GA; a0 < p; a0 += nw * GA) {
        typename AccSel<T, EXACT>::type acc[GA][QM];
#pragma unroll
        for (int g = 0; g < GA; ++g)
#pragma unroll
            for (int c = 0; c < QM; ++c) acc[g][c].zero();
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            T yv[QM];
            const T ysh = tk.ys ? T(tk.ys[r]) : T(0);
#pragma unroll
            for (int c = 0; c < QM; ++c) {
                if (c < q) yv[c] = (c < q1 ? (tk.Y ? tk.Y[(int64_t)c * tk.ldy + r] : T(0)) : tk.Y2[(int64_t)(c - q1) * tk.ldy2 + r]) + ysh;
                else yv[c] = T(0);
            }
            const T xsh = tk.xs ? T(tk.xs[r]) : T(0);
#pragma unroll
            for (int g = 0; g < GA; ++g) {
                const int a = a0 + g;
                if (a < p) {
                    const T xv = (tk.X ? tk.X[(int64_t)a * tk.ldx + r] : T(0)) + xsh;
#pragma unroll
                    for (int c = 0; c < QM; ++c)
                        if (c < q) acc[g][c].add(xv, yv[c]);
                }
            }
        }
#pragma unroll
        for (int g = 0; g < GA; ++g) {
            const int a = a0 + g;
#pragma unroll
            for (int c = 0; c < QM; ++c) {
                double v = warp_sum(acc[g][c].get());
                if (lane == 0 && a < p && c < q) pout[a + c * p] = v;
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_ts_reduce(const TsTask<T>* __restrict__ tasks, int nchunks, int pq_stride,
                                                   const double* __restrict__ partial) {
    const TsTask<T> tk = tasks[blockIdx.x];
    const int pq = tk.p * tk.q;
    const double* base = partial + (size_t)blockIdx.x * nchunks * pq_stride;
    for (int e = threadIdx.x; e < pq; e += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < nchunks; ++c) s += base[(size_t)c * pq_stride + e];
        tk.out[e] = s;
    }
}

// The accumulator tile (columns of X per warp pass x columns of Y) is chosen from
// max_q.  exact != 0 selects exact-product double-float accumulation for FP32 data.
template <typename T, bool EXACT>
static void tn_dispatch(const TsTask<T>* tasks_dev, int ntasks, int max_pq, int max_q, int64_t n, double* partial,
                        cudaStream_t s) {
    TnGeom g = tn_geom(ntasks, n);
    dim3 grid(g.nchunks, ntasks);
    if (max_q <= 4) k_ts_tn<T, 4, 4, EXACT><<<grid, 256, 0, s>>>(tasks_dev, n, g.rows, g.nchunks, max_pq, partial);
    else if (max_q <= 8) k_ts_tn<T, 4, 8, EXACT><<<grid, 256, 0, s>>>(tasks_dev, n, g.rows, g.nchunks, max_pq, partial);
    else if (max_q <= 16) k_ts_tn<T, 2, 16, EXACT><<<grid, 256, 0, s>>>(tasks_dev, n, g.rows, g.nchunks, max_pq, partial);
    else k_ts_tn<T, 1, 48, EXACT><<<grid, 256, 0, s>>>(tasks_dev, n, g.rows, g.nchunks, max_pq, partial);
    k_ts_reduce<T><<<ntasks, 256, 0, s>>>(tasks_dev, g.nchunks, max_pq, partial);
}

template <typename T>
void launch_ts_tn(const TsTask<T>* tasks_dev, int ntasks, int max_pq, int max_q, int64_t n, double* partial,
                  cudaStream_t s, int exact) {
    if (ntasks <= 0) return;
    if (exact) tn_dispatch<T, true>(tasks_dev, ntasks, max_pq, max_q, n, partial, s);
    else tn_dispatch<T, false>(tasks_dev, ntasks, max_pq, max_q, n, partial, s);
}

template <typename T, int QM>
__global__ void __launch_bounds__(256) k_ts_nn(const TsTask<T>* __restrict__ tasks, int64_t n) {
    const TsTask<T> tk = tasks[blockIdx.y];
    extern __shared__ double smem_nn[];
    T* sT = reinterpret_cast<T*>(smem_nn);
    const int p = tk.p, q = tk.q;
    for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
        const int a = e % p, c = e / p;
        sT[e] = T(tk.Tm[a + (int64_t)c * tk.ldt]);
    }
    __syncthreads();
    const bool inplace = (const void*)tk.Z == (const void*)tk.X;
    const T alpha = T(tk.alpha), beta = T(tk.beta);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const T xsh = tk.xs ? T(tk.xs[r]) : T(0);
        T acc[QM];
#pragma unroll
        for (int c = 0; c < QM; ++c) acc[c] = T(0);
        if (inplace) {
            T xr[QM];
#pragma unroll
            for (int a = 0; a < QM; ++a) xr[a] = (a < p) ? tk.X[(int64_t)a * tk.ldx + r] + xsh : T(0);
#pragma unroll
            for (int a = 0; a < QM; ++a)
                if (a < p) {
#pragma unroll
                    for (int c = 0; c < QM; ++c)
                        if (c < q) acc[c] = fma(xr[a], sT[a + c * p], acc[c]);
                }
        } else {
            for (int a = 0; a < p; ++a) {
                const T xv = (tk.X ? tk.X[(int64_t)a * tk.ldx + r] : T(0)) + xsh;
#pragma unroll
                for (int c = 0; c < QM; ++c)
                    if (c < q) acc[c] = fma(xv, sT[a + c * p], acc[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < QM; ++c)
            if (c < q) {
                T* z = tk.Z + (int64_t)c * tk.ldz + r;
                *z = (tk.beta == 0.0) ? alpha * acc[c] : fma(beta, *z, alpha * acc[c]);
            }
    }
}

template <typename T>
void launch_ts_nn(const TsTask<T>* tasks_dev, int ntasks, int max_pq, int64_t n, cudaStream_t s) {
    if (ntasks <= 0) return;
    int bx = std::max(1, std::min(grid_for(n, 256), (4 * kNumSM * 4 + ntasks - 1) / ntasks));
    dim3 grid(bx, ntasks);
    size_t sm = (size_t)max_pq * sizeof(T);
    if (sm > 32 * 1024) smem_optin(k_ts_nn<T, 16>, sm);
    k_ts_nn<T, 16><<<grid, 256, sm, s>>>(tasks_dev, n);
}

// Double-float block update for FP32 data (the working block of a Krylov step):
//   Z = alpha (X + xs 1^T) T  [+ Z]
// X and Z are (hi, lo) pairs of FP32 arrays (a missing lo array means 0, and for
// Z means "round to FP32"); products and sums are error-free to ~2^-48, so the
// cancellation of Gram-Schmidt leaves no FP32-sized noise in the new direction.
// QM: most block columns q of Z this instantiation handles (4: the small blocks of the source
// and continuation formations, fewer accumulators); R: rows per thread per iteration, all
// their loads issued before any is used; PB: columns of X per batch of loads.
template <int QM, int R, int PB>
__global__ void __launch_bounds__(256, 2) k_ts_nn_df(const DfTask* __restrict__ tasks, int64_t n, int64_t rows) {
    const DfTask tk = tasks[blockIdx.y];
    extern __shared__ float smem_df[];
    const int p = tk.p, q = tk.q;
    float2* Tc = reinterpret_cast<float2*>(smem_df);   // alpha T as (hi, lo), p x q
    float2* cs = Tc + p * q;                            // column sums of alpha T (the xs term)
    for (int e = threadIdx.x; e < p * q; e += blockDim.x) {
        const int a = e % p, c = e / p;
        const double v = tk.alpha * tk.Tm[a + (int64_t)c * tk.ldt];
        const float h = (float)v;
        Tc[e] = make_float2(h, (float)(v - (double)h));
    }
    if (tk.xs && threadIdx.x < q) {
        double sum = 0.0;
        for (int a = 0; a < p; ++a) sum += tk.alpha * tk.Tm[a + (int64_t)threadIdx.x * tk.ldt];
        const float h = (float)sum;
        cs[threadIdx.x] = make_float2(h, (float)(sum - (double)h));
    }
    __syncthreads();
    const int pl = (tk.Xl && tk.pl > 0) ? tk.pl : (tk.Xl ? p : 0);   // columns of X with a low part
    const int64_t r0 = (int64_t)blockIdx.x * rows;
    const int64_t r1 = (r0 + rows < n) ? r0 + rows : n;
    for (int64_t base = r0; base < r1; base += (int64_t)R * blockDim.x) {
        int64_t r[R];
        bool act[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            r[u] = base + (int64_t)u * blockDim.x + threadIdx.x;
            act[u] = r[u] < r1;
        }
        // Z[r, c] = sum_a (X[r, a] (+ xs[r])) T[a, c]: exact FP32 products x * t_hi (FMA), the
        // small terms in a second sum, the running sums compensated (two-sum)
        float sh[R][QM], sl[R][QM];
#pragma unroll
        for (int u = 0; u < R; ++u)
#pragma unroll
            for (int c = 0; c < QM; ++c) sh[u][c] = sl[u][c] = 0.f;
        for (int a0 = 0; a0 < p; a0 += PB) {
            float x[R][PB], xl[R][PB];
#pragma unroll
            for (int u = 0; u < R; ++u)
#pragma unroll
                for (int j = 0; j < PB; ++j) {
                    const int a = a0 + j;
                    x[u][j] = (act[u] && a < p && tk.Xh) ? tk.Xh[(int64_t)a * tk.ldx + r[u]] : 0.f;
                    xl[u][j] = (act[u] && a < pl) ? tk.Xl[(int64_t)a * tk.ldx + r[u]] : 0.f;
                }
#pragma unroll
            for (int c = 0; c < QM; ++c) {
                if (c >= q) break;
#pragma unroll
                for (int j = 0; j < PB; ++j) {
                    if (a0 + j >= p) break;
                    const float2 t = Tc[(a0 + j) + c * p];   // one coefficient pair, used by every row
#pragma unroll
                    for (int u = 0; u < R; ++u) {
                        const float ph = x[u][j] * t.x;
                        float pe = fmaf(x[u][j], t.x, -ph);
                        pe = fmaf(x[u][j], t.y, pe);
                        pe = fmaf(xl[u][j], t.x, pe);
                        const float w = sh[u][c] + ph;
                        const float bp = w - sh[u][c];
                        sl[u][c] += ((sh[u][c] - (w - bp)) + (ph - bp)) + pe;
                        sh[u][c] = w;
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < R; ++u) {
            if (!act[u]) continue;
            DF xsd = DF{0.f, 0.f};
            if (tk.xs) {
                const double v = tk.xs[r[u]];
                const float h = (float)v;
                xsd = DF{h, (float)(v - (double)h)};
            }
#pragma unroll
            for (int c = 0; c < QM; ++c) {
                if (c >= q) break;
                DF z = df_fast2sum(sh[u][c], sl[u][c]);
                if (tk.xs) z = df_add(z, df_mul(xsd, DF{cs[c].x, cs[c].y}));
                const int64_t o = (int64_t)c * tk.ldz + r[u];
                if (tk.accumulate) z = df_add(z, DF{tk.Zh[o], tk.Zl ? tk.Zl[o] : 0.f});
                if (tk.Zl) {
                    tk.Zh[o] = z.hi;
                    tk.Zl[o] = z.lo;
                } else {
                    tk.Zh[o] = z.hi + z.lo;
                }
            }
        }
    }
}

void launch_ts_nn_df(const DfTask* tasks_dev, int ntasks, int max_pq, int64_t n, cudaStream_t s, int max_q) {
    if (ntasks <= 0) return;
    // row chunks of >= 256 rows, about 8 CTAs per SM in total
    const int64_t maxch = std::max<int64_t>(1, (n + 255) / 256);
    const int64_t want = std::max<int64_t>(1, (8 * kNumSM + ntasks - 1) / ntasks);
    const int64_t ch = std::min(want, maxch);
    int64_t rows = (n + ch - 1) / ch;
    rows = (rows + 255) / 256 * 256;
    dim3 grid((unsigned)((n + rows - 1) / rows), ntasks);
    size_t sm = ((size_t)max_pq + 16) * sizeof(float2);
    if (max_q <= 4) {
        if (sm > 32 * 1024) smem_optin(k_ts_nn_df<4, 1, 16>, sm);
        k_ts_nn_df<4, 1, 16><<<grid, 256, sm, s>>>(tasks_dev, n, rows);
    } else {
        if (sm > 32 * 1024) smem_optin(k_ts_nn_df<16, 1, 16>, sm);
        k_ts_nn_df<16, 1, 16><<<grid, 256, sm, s>>>(tasks_dev, n, rows);
    }
}

// out[i] = sum_k u[k] * G[i*n + k] for the rows i < nrows.  FP64 data: FP64 FMAs.  FP32 data:
// u enters as a double-float pair (uh, ul) prepared once; the products uh*g are exact (FMA),
// the sums compensated, all in FP32 units (FP64 runs at 1/64 of the FP32 rate here).
__device__ __forceinline__ void dot_acc(float& s, float& c, float uh, float ul, float g) {
    const float p = uh * g;
    float pe = fmaf(uh, g, -p);
    pe = fmaf(ul, g, pe);
    const float t = s + p;
    const float bp = t - s;
    c += ((s - (t - bp)) + (p - bp)) + pe;
    s = t;
}
__global__ void __launch_bounds__(256) k_row_dots_f(const float* __restrict__ uh, const float* __restrict__ ul,
                                                    const float* __restrict__ G, int64_t n, double* __restrict__ out) {
    constexpr int U = 4;
    const int64_t row = blockIdx.x;
    const float* g = G + row * n;
    float s = 0.f, c = 0.f;
    for (int64_t k0 = (int64_t)threadIdx.x; k0 < n; k0 += (int64_t)blockDim.x * U) {
        float gv[U], hv[U], lv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int64_t k = k0 + (int64_t)u * blockDim.x;
            const bool ok = k < n;
            gv[u] = ok ? g[k] : 0.f;
            hv[u] = ok ? __ldg(uh + k) : 0.f;
            lv[u] = ok ? __ldg(ul + k) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) dot_acc(s, c, hv[u], lv[u], gv[u]);
    }
    double v = (double)s + (double)c;
    __shared__ double red[8];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[row] = t;
    }
}
__global__ void __launch_bounds__(256) k_row_dots_d(const double* __restrict__ u, const double* __restrict__ G,
                                                    int64_t n, double* __restrict__ out) {
    const int64_t row = blockIdx.x;
    const double* g = G + row * n;
    double s = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s = fma(u[k], g[k], s);
    __shared__ double red[8];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        out[row] = t;
    }
}
__global__ void k_split_df(const double* __restrict__ u, float* __restrict__ uh, float* __restrict__ ul, int64_t n) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const double v = u[k];
        const float h = (float)v;
        uh[k] = h;
        ul[k] = (float)(v - (double)h);
    }
}
template <typename T>
void launch_row_dots(const double* u, const T* G, int64_t n, int nrows, double* out, float* split, cudaStream_t s) {
    if (nrows <= 0) return;
    if constexpr (sizeof(T) == 4) {
        k_split_df<<<std::min(grid_for(n, 256), 4 * kNumSM * 8), 256, 0, s>>>(u, split, split + n, n);
        k_row_dots_f<<<nrows, 256, 0, s>>>(split, split + n, G, n, out);
    } else {
        (void)split;
        k_row_dots_d<<<nrows, 256, 0, s>>>(u, G, n, out);
    }
}

// =====================================================================================
// Reconstruction u(t) = u0 + V y(t)
//
// FP64 data accumulate with FMAs.  FP32 data accumulate V y with FP32 FMAs and add u0
// last, as an exact (hi, lo) pair of the FP64 initial condition, by two-sum: the
// correction V y is small against u0 at early times, so rounding u0 itself to FP32 (a
// relative 6e-8 per element) was the larger part of the early-time error there.
// =====================================================================================
template <typename T>
struct ReconAcc;
template <>
struct ReconAcc<double> {
    using C = double;
    double s;
    __device__ __forceinline__ static C coef(double v) { return v; }
    __device__ __forceinline__ void init(double u) { s = u; }
    __device__ __forceinline__ void add(double v, C c) { s = fma(v, c, s); }
    template <typename TO>
    __device__ __forceinline__ TO get(double) const { return TO(s); }
};
template <>
struct ReconAcc<float> {
    using C = float;
    float s;
    __device__ __forceinline__ static C coef(double v) { return (float)v; }
    __device__ __forceinline__ void init(double) { s = 0.f; }
    __device__ __forceinline__ void add(float v, C c) { s = fmaf(v, c, s); }
    // u0 + s with u0 = hi + lo (hi = FP32 rounding of u0): two-sum of s and hi, then lo
    template <typename TO>
    __device__ __forceinline__ TO get(double u) const {
        const float hi = (float)u;
        const float lo = (float)(u - (double)hi);
        const float t = s + hi;
        const float bp = t - s;
        const float e = (s - (t - bp)) + (hi - bp);
        if constexpr (sizeof(TO) == 8) return (double)t + (double)(e + lo);
        else return t + (e + lo);
    }
};

template <typename T, typename TO, int RM>
__global__ void __launch_bounds__(256) k_recon(const ReconTask<T>* __restrict__ tasks, int64_t n,
                                               const double* __restrict__ u0, TO* __restrict__ out, int64_t ldo,
                                               int64_t rows) {
    constexpr int AB = 8;   // basis columns per batch of loads
    using Acc = ReconAcc<T>;
    using CT = typename Acc::C;
    const ReconTask<T> tk = tasks[blockIdx.y];
    extern __shared__ double smem_rc[];
    const int K = tk.K1 + tk.K2;
    const int ng = (tk.ns + RM - 1) / RM;   // groups of RM samples
    // coefficients: sc[(g * K + a) * RM + r] = C(sample g*RM + r, column a) (0 past ns)
    CT* sc = reinterpret_cast<CT*>(smem_rc);
    for (int e = threadIdx.x; e < ng * K * RM; e += blockDim.x) {
        const int r = e % RM, a = (e / RM) % K, g = e / (RM * K);
        const int smp = g * RM + r;
        double v = 0.0;
        if (smp < tk.ns)
            v = (a < tk.K1) ? tk.C1[(int64_t)(tk.r0 + smp) * tk.ldc1 + a]
                            : tk.C2[(int64_t)(tk.r0 + smp) * tk.ldc2 + (a - tk.K1)];
        sc[e] = Acc::coef(v);
    }
    __syncthreads();
    const int64_t k0 = (int64_t)blockIdx.x * rows;
    const int64_t k1 = (k0 + rows < n) ? k0 + rows : n;
    for (int64_t kb = k0; kb < k1; kb += blockDim.x) {
        const int64_t k = kb + threadIdx.x;
        const bool act = k < k1;
        const double base = (act && u0) ? u0[k] : 0.0;
        for (int g = 0; g < ng; ++g) {
            Acc acc[RM];
#pragma unroll
            for (int r = 0; r < RM; ++r) acc[r].init(base);
            for (int a0 = 0; a0 < K; a0 += AB) {
                T v[AB];
#pragma unroll
                for (int j = 0; j < AB; ++j) {
                    const int a = a0 + j;
                    v[j] = T(0);
                    if (act && a < K)
                        v[j] = (a < tk.K1) ? tk.V1[(int64_t)a * tk.ld1 + k] : tk.V2[(int64_t)(a - tk.K1) * tk.ld2 + k];
                }
#pragma unroll
                for (int j = 0; j < AB; ++j) {
                    if (a0 + j >= K) break;
                    const CT* cj = sc + ((int64_t)g * K + a0 + j) * RM;
#pragma unroll
                    for (int r = 0; r < RM; ++r) acc[r].add(v[j], cj[r]);
                }
            }
            if (act) {
#pragma unroll
                for (int r = 0; r < RM; ++r)
                    if (g * RM + r < tk.ns) out[(tk.i0 + g * RM + r) * ldo + k] = acc[r].template get<TO>(base);
            }
        }
    }
}

// max_ns: most samples of a task; max_k: most basis columns (K1 + K2) of a task.
template <typename T, typename TO>
void launch_recon(const ReconTask<T>* tasks_dev, int ntasks, int max_ns, int64_t n, const double* u0, TO* out,
                  int64_t ldo, int max_k, cudaStream_t s) {
    if (ntasks <= 0) return;
    const int64_t maxch = std::max<int64_t>(1, (n + 255) / 256);
    const int64_t want = std::max<int64_t>(1, (8 * kNumSM + ntasks - 1) / ntasks);
    const int64_t ch = std::min(want, maxch);
    int64_t rows = (n + ch - 1) / ch;
    rows = (rows + 255) / 256 * 256;
    dim3 grid((unsigned)((n + rows - 1) / rows), ntasks);
    const size_t ng = (size_t)(std::max(max_ns, 1) + 16) / 17;
    const size_t sm = ng * (size_t)std::max(max_k, 1) * 17 * sizeof(typename ReconAcc<T>::C);
    if (sm > 32 * 1024)
        smem_optin(k_recon<T, TO, 17>, sm);
    k_recon<T, TO, 17><<<grid, 256, sm, s>>>(tasks_dev, n, u0, out, ldo, rows);
}

// =====================================================================================
// Helpers
// =====================================================================================
template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ x, TO* __restrict__ y, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = TO(x[i]);
}
template <typename TI, typename TO>
void launch_convert(const TI* x, TO* y, int64_t count, cudaStream_t s) {
    if (count <= 0) return;
    k_convert<TI, TO><<<std::min(grid_for(count, 256), 4 * kNumSM * 8), 256, 0, s>>>(x, y, count);
}

template <typename T>
__global__ void k_add(T* __restrict__ y, const T* __restrict__ x, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        y[i] += x[i];
}
template <typename T>
void launch_add(T* y, const T* x, int64_t count, cudaStream_t s) {
    if (count <= 0) return;
    k_add<T><<<std::min(grid_for(count, 256), 4 * kNumSM * 8), 256, 0, s>>>(y, x, count);
}

template <typename T>
__global__ void __launch_bounds__(256) k_row_diff_norms(const T* __restrict__ A, const T* __restrict__ B, int64_t n,
                                                       int nrows, double* __restrict__ out) {
    const int row = blockIdx.x;
    const T* a = A + (int64_t)row * n;
    const T* b = B + (int64_t)row * n;
    double sd = 0.0, sa = 0.0;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        const double av = (double)a[k], bv = (double)b[k];
        sd = fma(av - bv, av - bv, sd);
        sa = fma(av, av, sa);
    }
    __shared__ double r1[8], r2[8];
    sd = warp_sum(sd);
    sa = warp_sum(sa);
    if ((threadIdx.x & 31) == 0) {
        r1[threadIdx.x >> 5] = sd;
        r2[threadIdx.x >> 5] = sa;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0, t2 = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += r1[w];
            t2 += r2[w];
        }
        out[row] = t1;
        out[nrows + row] = t2;
    }
}
template <typename T>
void launch_row_diff_norms(const T* A, const T* B, int64_t n, int nrows, double* out, cudaStream_t s) {
    if (nrows <= 0) return;
    k_row_diff_norms<T><<<nrows, 256, 0, s>>>(A, B, n, nrows, out);
}

// ---------------------------------------------------------------- instantiations
#define PEXP_INST_T(T)                                                                                    \
    template void launch_stencil<T>(const OpDesc&, const T*, T*, int, int, cudaStream_t);                 \
    template void launch_stencil_ptrs<T>(const OpDesc&, const T* const*, T* const*, int, int, cudaStream_t); \
    template void launch_burgers_source<T>(const OpDesc&, const T*, T*, int, int, double, cudaStream_t);  \
    template void launch_sai_solve<T>(const OpDesc&, const SaiCoef&, const T* const*, T* const*, T* const*,  \
                                      int, double*, cudaStream_t);                                        \
    template void launch_sai_solve_lo<T>(const OpDesc&, const SaiCoef&, const T* const*, const T* const*,       \
                                         T* const*, T* const*, int, double*, cudaStream_t, const int* const*); \
    template bool launch_sai_coop<T>(const OpDesc&, const SaiCoef&, const T*, T*, T*, double*, const int*, GridBar, \
                                     cudaStream_t);                                                          \
    template void launch_ts_tn<T>(const TsTask<T>*, int, int, int, int64_t, double*, cudaStream_t, int);   \
    template void launch_ts_nn<T>(const TsTask<T>*, int, int, int64_t, cudaStream_t);                     \
    template void launch_recon<T, float>(const ReconTask<T>*, int, int, int64_t, const double*, float*,    \
                                         int64_t, int, cudaStream_t);                                     \
    template void launch_recon<T, double>(const ReconTask<T>*, int, int, int64_t, const double*, double*,  \
                                          int64_t, int, cudaStream_t);                                    \
    template void launch_row_diff_norms<T>(const T*, const T*, int64_t, int, double*, cudaStream_t); \
    template void launch_add<T>(T*, const T*, int64_t, cudaStream_t);                                   \
    template void launch_row_dots<T>(const double*, const T*, int64_t, int, double*, float*, cudaStream_t);
PEXP_INST_T(double)
PEXP_INST_T(float)
template void launch_convert<double, float>(const double*, float*, int64_t, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, int64_t, cudaStream_t);
template void launch_convert<double, double>(const double*, double*, int64_t, cudaStream_t);
template void launch_convert<float, float>(const float*, float*, int64_t, cudaStream_t);

}  // namespace pexp
