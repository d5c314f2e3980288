// Device helpers of the chunked affine-scan solves of periodic (and bounded) first-order
// recurrences x_i = a_i x_{i-1} + b_i (sai solve in tall.cu, variable-coefficient solve in
// vsai.cu): double-float arithmetic for FP32 data, warp and CTA scans of affine maps,
// vectorised loads and stores of a thread's run of elements, and the circular carry
// over chunk summaries.
#pragma once

#include "common.cuh"

namespace pexp {

constexpr int kSaiThreads = 256;
constexpr int kSaiPer = 8;
constexpr int kSaiChunk = kSaiThreads * kSaiPer;

// Arithmetic of the recurrences.  FP64 data use double.  FP32 data use a
// double-float pair (hi, lo) -- Dekker/Knuth error-free sum and FMA product --
// because the recurrences accumulate ~1/(1-alpha) terms and plain FP32 rounding
// would leave smooth, correlated errors of ~1e-6 in every solve.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_fast2sum(float a, float b) {
    const float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return df_fast2sum(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_fast2sum(p, e);
}
__device__ __forceinline__ double rmul(double a, double b) { return a * b; }
__device__ __forceinline__ DF rmul(DF a, DF b) { return df_mul(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ DF rfma(DF a, DF b, DF c) { return df_add(df_mul(a, b), c); }
__device__ __forceinline__ double rdbl(double a) { return a; }
__device__ __forceinline__ double rdbl(DF a) { return (double)a.hi + (double)a.lo; }
template <typename R> __device__ __forceinline__ R rfrom(double x);
template <> __device__ __forceinline__ double rfrom<double>(double x) { return x; }
template <> __device__ __forceinline__ DF rfrom<DF>(double x) {
    const float h = (float)x;
    return DF{h, (float)(x - (double)h)};
}
template <typename T> struct SaiR { using R = double; };
template <> struct SaiR<float> { using R = DF; };
template <typename T, typename R> __device__ __forceinline__ T rto(R x);
template <> __device__ __forceinline__ double rto<double, double>(double x) { return x; }
template <> __device__ __forceinline__ float rto<float, DF>(DF x) { return x.hi + x.lo; }
template <typename T, typename R> __device__ __forceinline__ R load_r(T hi, T lo);
template <> __device__ __forceinline__ double load_r<double, double>(double hi, double lo) { return hi; }
template <> __device__ __forceinline__ DF load_r<float, DF>(float hi, float lo) { return DF{hi, lo}; }

// Shuffles of a recurrence value (FP64, or a double-float pair).
__device__ __forceinline__ double rshfl_up(double v, int d) { return __shfl_up_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double rshfl_down(double v, int d) { return __shfl_down_sync(0xffffffffu, v, d); }
__device__ __forceinline__ double rshfl_idx(double v, int l) { return __shfl_sync(0xffffffffu, v, l); }
__device__ __forceinline__ DF rshfl_up(DF v, int d) {
    return DF{__shfl_up_sync(0xffffffffu, v.hi, d), __shfl_up_sync(0xffffffffu, v.lo, d)};
}
__device__ __forceinline__ DF rshfl_down(DF v, int d) {
    return DF{__shfl_down_sync(0xffffffffu, v.hi, d), __shfl_down_sync(0xffffffffu, v.lo, d)};
}
__device__ __forceinline__ DF rshfl_idx(DF v, int l) {
    return DF{__shfl_sync(0xffffffffu, v.hi, l), __shfl_sync(0xffffffffu, v.lo, l)};
}

// Scan of affine maps f(z) = a z + b over the CTA in "virtual" order v (v = t forward,
// v = NT-1-t backward); map v is applied after maps < v.  Returns the exclusive
// composition for this thread and the CTA total.  Warps scan with shuffles (Kogge-Stone);
// one warp then composes the warp totals: two barriers per scan.
template <typename R>
__device__ __forceinline__ void cta_affine_scan(R a, R b, bool reverse, R* sa, R* sb, R& ea, R& eb, R& ta,
                                                R& tb) {
    constexpr int NW = kSaiThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lv = reverse ? 31 - lane : lane;        // virtual lane
    const int wv = reverse ? NW - 1 - warp : warp;    // virtual warp
    // inclusive scan within the warp in virtual order
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const R pa = reverse ? rshfl_down(a, d) : rshfl_up(a, d);
        const R pb = reverse ? rshfl_down(b, d) : rshfl_up(b, d);
        if (lv >= d) {
            b = rfma(a, pb, b);
            a = rmul(a, pa);
        }
    }
    // exclusive within the warp: the inclusive value of the previous virtual lane
    const int last = reverse ? 0 : 31;
    R xa = reverse ? rshfl_down(a, 1) : rshfl_up(a, 1);
    R xb = reverse ? rshfl_down(b, 1) : rshfl_up(b, 1);
    if (lv == 0) {
        xa = rfrom<R>(1.0);
        xb = rfrom<R>(0.0);
    }
    if (lane == last) {
        sa[wv] = a;
        sb[wv] = b;
    }
    __syncthreads();
    if (warp == 0) {
        // exclusive scan of the warp totals (NW <= 32) in virtual warp order; lanes < NW only
        // read lanes < NW, so log2(NW) shuffle rounds give them their full prefixes
        R wa = lane < NW ? sa[lane] : rfrom<R>(1.0);
        R wb = lane < NW ? sb[lane] : rfrom<R>(0.0);
#pragma unroll
        for (int d = 1; d < NW; d <<= 1) {
            const R pa = rshfl_up(wa, d), pb = rshfl_up(wb, d);
            if (lane >= d) {
                wb = rfma(wa, pb, wb);
                wa = rmul(wa, pa);
            }
        }
        const R ta_ = rshfl_idx(wa, NW - 1), tb_ = rshfl_idx(wb, NW - 1);
        R pa = rshfl_up(wa, 1), pb = rshfl_up(wb, 1);
        if (lane == 0) {
            pa = rfrom<R>(1.0);
            pb = rfrom<R>(0.0);
        }
        __syncwarp();
        if (lane < NW) {
            sa[lane] = pa;   // exclusive prefix of virtual warp `lane`
            sb[lane] = pb;
        }
        if (lane == 0) {
            sa[NW] = ta_;
            sb[NW] = tb_;
        }
    }
    __syncthreads();
    const R pa = sa[wv], pb = sb[wv];
    // this thread's exclusive map = (within-warp exclusive) after (previous warps)
    ea = rmul(xa, pa);
    eb = rfma(xa, pb, xb);
    ta = sa[NW];
    tb = sb[NW];
    __syncthreads();   // the shared arrays are reused by the next scan
}

// Loads and stores of a thread's kSaiPer consecutive elements: 16-byte vector
// accesses when the run is whole and aligned, else element by element.
template <typename T>
__device__ __forceinline__ bool sai_vec_ok(const T* p, int64_t n, int64_t start) {
    return start + kSaiPer <= n && ((reinterpret_cast<uintptr_t>(p + start) & 15u) == 0);
}
__device__ __forceinline__ void sai_vload(const float* p, float* v) {
#pragma unroll
    for (int j = 0; j < kSaiPer / 4; ++j) {
        const float4 a = reinterpret_cast<const float4*>(p)[j];
        v[4 * j] = a.x;
        v[4 * j + 1] = a.y;
        v[4 * j + 2] = a.z;
        v[4 * j + 3] = a.w;
    }
}
__device__ __forceinline__ void sai_vload(const double* p, double* v) {
#pragma unroll
    for (int j = 0; j < kSaiPer / 2; ++j) {
        const double2 a = reinterpret_cast<const double2*>(p)[j];
        v[2 * j] = a.x;
        v[2 * j + 1] = a.y;
    }
}
__device__ __forceinline__ void sai_vstore(float* p, const float* v) {
#pragma unroll
    for (int j = 0; j < kSaiPer / 4; ++j)
        reinterpret_cast<float4*>(p)[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
}
__device__ __forceinline__ void sai_vstore(double* p, const double* v) {
#pragma unroll
    for (int j = 0; j < kSaiPer / 2; ++j) reinterpret_cast<double2*>(p)[j] = make_double2(v[2 * j], v[2 * j + 1]);
}
template <typename T>
__device__ __forceinline__ int sai_load(const T* x, int64_t n, int64_t start, T* vals) {
    if (sai_vec_ok(x, n, start)) {
        sai_vload(x + start, vals);
        return kSaiPer;
    }
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < kSaiPer; ++j) {
        int64_t k = start + j;
        if (k < n) {
            vals[j] = x[k];
            cnt = j + 1;
        } else {
            vals[j] = T(0);
        }
    }
    return cnt;
}
template <typename T>
__device__ __forceinline__ void sai_store(T* y, int64_t n, int64_t start, int cnt, const T* vals) {
    if (cnt == kSaiPer && sai_vec_ok(y, n, start)) {
        sai_vstore(y + start, vals);
        return;
    }
#pragma unroll
    for (int j = 0; j < kSaiPer; ++j)
        if (j < cnt) y[start + j] = vals[j];
}
// Split of a recurrence value into the stored pair: FP64 as is; FP32 as (hi, lo)
// when a low-part array is given (the working block keeps double-float
// precision), else rounded.
__device__ __forceinline__ void split_r(double v, bool pair, double& h, double& l) {
    h = v;
    l = 0.0;
}
__device__ __forceinline__ void split_r(DF v, bool pair, float& h, float& l) {
    if (pair) {
        h = v.hi;
        l = v.lo;
    } else {
        h = v.hi + v.lo;
        l = 0.f;
    }
}

template <typename R>
__device__ __forceinline__ R ipow(R x, int e) {
    R r = rfrom<R>(1.0);
    for (int i = 0; i < e; ++i) r = rmul(r, x);
    return r;
}

// Circular carry into chunk `ch` from the chunk summaries: sum_k prod_k * end_{c_k} / (1 - rho^n),
// c_k = ch - dir*k (circular), prod_k = product of the decays of c_1..c_{k-1}.  Evaluated by
// one warp, 32 summaries at a time (decays multiply along a warp scan), until the running
// product drops below 1e-30.  Must be called by all 32 lanes of warp 0.
__device__ __forceinline__ double sai_carry_warp(const double* ends, const double* decays, int nch, int ch, int dir,
                                                 double rho_n) {
    const int lane = threadIdx.x & 31;
    double sum = 0.0, base = 1.0;
    for (int k0 = 1; k0 <= nch; k0 += 32) {
        const int k = k0 + lane;
        double e = 0.0, d = 1.0;
        if (k <= nch) {
            int cidx = ch - dir * k;
            cidx %= nch;
            if (cidx < 0) cidx += nch;
            e = ends[cidx];
            d = decays[cidx];
        }
        // exclusive prefix product of the decays within the warp
        double incl = d;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double up = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl *= up;
        }
        double excl = __shfl_up_sync(0xffffffffu, incl, 1);
        if (lane == 0) excl = 1.0;
        double term = base * excl * e;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) term += __shfl_xor_sync(0xffffffffu, term, o);
        sum += term;
        base *= __shfl_sync(0xffffffffu, incl, 31);
        if (fabs(base) < 1e-30) break;
    }
    return sum / (1.0 - rho_n);
}

// Forward values w of this thread's elements (cnt of them, registers): the local maps
// composed over the CTA and the circular carry into the chunk.  Contains barriers.  The carry
// is read from shared memory after the CTA scan, so the warp that computes it may write it
// up to the scan's first barrier: its computation overlaps the other warps' local work.
template <typename T, typename R>
__device__ __forceinline__ void sai_forward_values(const T* vals, const T* lows, bool has_lo, int cnt, R al,
                                                   const double* carry_sm, R* sa, R* sb, R* wv) {
    R b = rfrom<R>(0.0);
#pragma unroll
    for (int j = 0; j < kSaiPer; ++j)
        if (j < cnt) b = rfma(al, b, load_r<T, R>(vals[j], has_lo ? lows[j] : T(0)));
    R a = ipow(al, cnt);
    R ea, eb, ta, tb;
    cta_affine_scan<R>(a, b, false, sa, sb, ea, eb, ta, tb);
    R w = rfma(ea, rfrom<R>(*carry_sm), eb);
#pragma unroll
    for (int j = 0; j < kSaiPer; ++j) {
        if (j < cnt) w = rfma(al, w, load_r<T, R>(vals[j], has_lo ? lows[j] : T(0)));
        wv[j] = w;
    }
}

}  // namespace pexp
