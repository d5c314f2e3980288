// Variable-coefficient shift-and-invert solve and the per-subinterval kernels of the
// averaged-Jacobian waveform relaxation (Sec. 2.3-2.4, eqs. ivp4, piecewiseJac,
// ivpSubproblem), sm_103a.
//
// On subinterval j the operator is A + J_j, J_j the Jacobian of the Burgers term at the
// subinterval's time-averaged iterate.  A + J_j is tridiagonal (cyclic on a periodic mesh)
// with coefficients that vary along x, so the shift-and-invert matrix M = I - gamma (A + J_j)
// no longer factors into two constant recurrences.  It factors as
//     M = (I - diag(lam) S^{-1}) diag(d) (I - diag(mu) S),
// with M's sub-, main and super-diagonals a_i, b_i, c_i:
//     d_i = b_i - a_i c_{i-1} / d_{i-1},  lam_i = -a_i / d_{i-1},  mu_i = -c_i / d_i.
// The d recurrence is a contraction for a diagonally dominant M (the Burgers workload has
// cell Peclet numbers far below 2), so its periodic solution is reached from any start in
// a warm-up of ~40 sqrt(g) steps, g = gamma * off-diagonal: each chunk of 2048 rows warms
// up from the left on its own, with no global step.  A bounded mesh (a_0 = c_{n-1} = 0)
// starts exactly at row 0.
//
// The solve is then the two affine recurrences of the constant-coefficient solve in
// tall.cu with per-element coefficients: the same chunked CTA scans, circular carries over
// chunk summaries (the carry's geometric factor is the product of all chunk decays), and
// three passes over the input, the forward values recomputed in the last pass.
#include <math.h>

#include <algorithm>

#include "common.cuh"
#include "sai.cuh"

namespace pexp {

namespace {

constexpr int kFacThreads = 64;

// Row i of A + J(ubar): sub (coefficient of v_{i-1}), diag, super (coefficient of v_{i+1}).
__device__ __forceinline__ void op_row(const Dim1& x, const double* ubar, double inv2dx, int64_t i, double& l,
                                       double& m, double& r) {
    const int64_t n = x.n;
    l = x.d + x.c;
    m = -2.0 * x.d;
    r = x.d - x.c;
    if (ubar) {
        const int64_t im = i == 0 ? n - 1 : i - 1, ip = i == n - 1 ? 0 : i + 1;
        l += ubar[im] * inv2dx;
        r -= ubar[ip] * inv2dx;
    }
    if (!x.periodic) {
        if (i == 0) l = 0.0;
        if (i == n - 1) r = 0.0;
    }
}

__global__ void __launch_bounds__(kFacThreads) k_vsai_factor(Dim1 x, double gamma, double inv2dx,
                                                             const VarOpTask* __restrict__ tasks, int64_t warm) {
    const VarOpTask tk = tasks[blockIdx.y];
    const int64_t n = x.n;
    const int64_t p0 = ((int64_t)blockIdx.x * kFacThreads + threadIdx.x) * kSaiChunk;
    if (p0 >= n) return;
    const int64_t p1 = min(p0 + (int64_t)kSaiChunk, n);
    // M = I - gamma A: a_i = -gamma l_i, b_i = 1 - gamma m_i, c_i = -gamma r_i
    double d, cprev;
    int64_t q;
    if (!x.periodic && p0 <= warm) {
        q = 0;
        d = 1.0;       // d_{-1}: a_0 = 0, so any nonzero value gives d_0 = b_0
        cprev = 0.0;
    } else {
        q = p0 - warm;   // may wrap (periodic): indices mod n
        d = 0.0;
        double l, m, r;
        const int64_t qm = ((q - 1) % n + n) % n;
        op_row(x, tk.ubar, inv2dx, qm, l, m, r);
        d = 1.0 - gamma * m;   // start: the diagonal itself
        cprev = -gamma * r;
    }
    bool bad = false;
    for (int64_t i = q; i < p1; ++i) {
        const int64_t k = ((i % n) + n) % n;
        double l, m, r;
        op_row(x, tk.ubar, inv2dx, k, l, m, r);
        const double a = -gamma * l, b = 1.0 - gamma * m, c = -gamma * r;
        const double lam = -a / d;
        const double dn = b + lam * cprev;   // b - a c_{i-1} / d_{i-1}
        if (i >= p0) {
            tk.lam[k] = lam;
            tk.dinv[k] = 1.0 / dn;
            tk.mu[k] = -c / dn;
            if (fabs(b) < fabs(a) + fabs(c)) bad = true;
        }
        d = dn;
        cprev = c;
    }
    if (bad) *tk.flag = 1;
}

template <typename R>
__device__ __forceinline__ R load_coef(const double* p, int64_t k, int64_t n) {
    return rfrom<R>(k < n ? __ldg(p + k) : 0.0);
}

// Product of all chunk decays of one vector (the recurrence's factor around the circle),
// by warp 0; every lane returns it.
__device__ __forceinline__ double decay_product_warp(const double* decays, int nch) {
    const int lane = threadIdx.x & 31;
    double pr = 1.0;
    for (int c = lane; c < nch; c += 32) pr *= decays[c];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pr *= __shfl_xor_sync(0xffffffffu, pr, o);
    return pr;
}

// Forward values y of this thread's run with per-element lam (registers), carry-in
// `carry` before the chunk.  Contains barriers.
template <typename T, typename R>
__device__ __forceinline__ void vsai_forward_values(const T* vals, const T* lows, bool has_lo, int cnt, const R* lam,
                                                    double carry, R* sa, R* sb, R* wv) {
    R b = rfrom<R>(0.0), a = rfrom<R>(1.0);
#pragma unroll
    for (int j = 0; j < kSaiPer; ++j)
        if (j < cnt) {
            b = rfma(lam[j], b, load_r<T, R>(vals[j], has_lo ? lows[j] : T(0)));
            a = rmul(a, lam[j]);
        }
    R ea, eb, ta, tb;
    cta_affine_scan<R>(a, b, false, sa, sb, ea, eb, ta, tb);
    R w = rfma(ea, rfrom<R>(carry), eb);
#pragma unroll
    for (int j = 0; j < kSaiPer; ++j) {
        if (j < cnt) w = rfma(lam[j], w, load_r<T, R>(vals[j], has_lo ? lows[j] : T(0)));
        wv[j] = w;
    }
}

// Pass 1: forward chunk summaries with zero carry-in.
template <typename T>
__global__ void __launch_bounds__(kSaiThreads) k_vsai_fwd_ends(int64_t n, int nch, const VarSai* __restrict__ coef,
                                                               const T* const* __restrict__ Xp,
                                                               const T* const* __restrict__ Xlo,
                                                               double* __restrict__ ends, double* __restrict__ decays,
                                                               const int* const* __restrict__ skip) {
    pdl_entry();
    using R = typename SaiR<T>::R;
    __shared__ R sa[kSaiThreads], sb[kSaiThreads];
    const int v = blockIdx.y, ch = blockIdx.x;
    if (skip && skip[v] && *skip[v]) return;
    const VarSai cf = coef[v];
    const T* x = Xp[v];
    const T* xl = Xlo ? Xlo[v] : nullptr;
    const int64_t start = (int64_t)ch * kSaiChunk + (int64_t)threadIdx.x * kSaiPer;
    T vals[kSaiPer], lows[kSaiPer];
    const int cnt = sai_load(x, n, start, vals);
    if (xl) sai_load(xl, n, start, lows);
    R b = rfrom<R>(0.0), a = rfrom<R>(1.0);
#pragma unroll
    for (int j = 0; j < kSaiPer; ++j)
        if (j < cnt) {
            const R lj = load_coef<R>(cf.lam, start + j, n);
            b = rfma(lj, b, load_r<T, R>(vals[j], xl ? lows[j] : T(0)));
            a = rmul(a, lj);
        }
    R ea, eb, ta, tb;
    cta_affine_scan<R>(a, b, false, sa, sb, ea, eb, ta, tb);
    if (threadIdx.x == 0) {
        ends[(int64_t)v * nch + ch] = rdbl(tb);
        decays[(int64_t)v * nch + ch] = rdbl(ta);
    }
}

// Pass 2: forward values with carries, z = y / d, and the summaries of the backward
// recurrence of z with zero carry from the right.
template <typename T>
__global__ void __launch_bounds__(kSaiThreads) k_vsai_fwd_apply(int64_t n, int nch, const VarSai* __restrict__ coef,
                                                                const T* const* __restrict__ Xp,
                                                                const T* const* __restrict__ Xlo,
                                                                const double* __restrict__ fends,
                                                                const double* __restrict__ fdecays,
                                                                double* __restrict__ bends,
                                                                double* __restrict__ bdecays,
                                                                const int* const* __restrict__ skip) {
    pdl_entry();
    using R = typename SaiR<T>::R;
    __shared__ R sa[kSaiThreads], sb[kSaiThreads];
    __shared__ double carry_in;
    const int v = blockIdx.y, ch = blockIdx.x;
    if (skip && skip[v] && *skip[v]) return;
    const VarSai cf = coef[v];
    if (threadIdx.x < 32) {
        const double* fe = fends + (int64_t)v * nch;
        const double* fd = fdecays + (int64_t)v * nch;
        const double rho = decay_product_warp(fd, nch);
        const double cv = sai_carry_warp(fe, fd, nch, ch, +1, rho);
        if (threadIdx.x == 0) carry_in = cv;
    }
    const T* x = Xp[v];
    const T* xl = Xlo ? Xlo[v] : nullptr;
    const int64_t start = (int64_t)ch * kSaiChunk + (int64_t)threadIdx.x * kSaiPer;
    T vals[kSaiPer], lows[kSaiPer];
    const int cnt = sai_load(x, n, start, vals);
    if (xl) sai_load(xl, n, start, lows);
    R lam[kSaiPer];
#pragma unroll
    for (int j = 0; j < kSaiPer; ++j) lam[j] = load_coef<R>(cf.lam, start + j, n);
    __syncthreads();   // carry_in
    R wv[kSaiPer];
    vsai_forward_values<T, R>(vals, lows, xl != nullptr, cnt, lam, carry_in, sa, sb, wv);
    R gb = rfrom<R>(0.0), ga = rfrom<R>(1.0);
#pragma unroll
    for (int j = kSaiPer - 1; j >= 0; --j)
        if (j < cnt) {
            const R mj = load_coef<R>(cf.mu, start + j, n);
            const R zj = rmul(wv[j], load_coef<R>(cf.dinv, start + j, n));
            gb = rfma(mj, gb, zj);
            ga = rmul(ga, mj);
        }
    R ea, eb, ta, tb;
    cta_affine_scan<R>(ga, gb, true, sa, sb, ea, eb, ta, tb);
    if (threadIdx.x == 0) {
        bends[(int64_t)v * nch + ch] = rdbl(tb);
        bdecays[(int64_t)v * nch + ch] = rdbl(ta);
    }
}

// Pass 3: the forward values again, z = y / d, then the backward recurrence with carries.
template <typename T>
__global__ void __launch_bounds__(kSaiThreads) k_vsai_bwd_apply(int64_t n, int nch, const VarSai* __restrict__ coef,
                                                                const T* const* __restrict__ Xp,
                                                                const T* const* __restrict__ Xlo,
                                                                T* const* __restrict__ Yp, T* const* __restrict__ Ylo,
                                                                const double* __restrict__ fends,
                                                                const double* __restrict__ fdecays,
                                                                const double* __restrict__ bends,
                                                                const double* __restrict__ bdecays,
                                                                const int* const* __restrict__ skip) {
    pdl_entry();
    using R = typename SaiR<T>::R;
    __shared__ R sa[kSaiThreads], sb[kSaiThreads];
    __shared__ double carry_f, carry_b;
    const int v = blockIdx.y, ch = blockIdx.x;
    if (skip && skip[v] && *skip[v]) return;
    const VarSai cf = coef[v];
    if (threadIdx.x < 32) {
        const double* fe = fends + (int64_t)v * nch;
        const double* fd = fdecays + (int64_t)v * nch;
        const double* be = bends + (int64_t)v * nch;
        const double* bd = bdecays + (int64_t)v * nch;
        const double rf = decay_product_warp(fd, nch);
        const double rb = decay_product_warp(bd, nch);
        const double cfv = sai_carry_warp(fe, fd, nch, ch, +1, rf);
        const double cbv = sai_carry_warp(be, bd, nch, ch, -1, rb);
        if (threadIdx.x == 0) {
            carry_f = cfv;
            carry_b = cbv;
        }
    }
    const T* x = Xp[v];
    const T* xl = Xlo ? Xlo[v] : nullptr;
    T* y = Yp[v];
    T* ylo = Ylo ? Ylo[v] : nullptr;
    const int64_t start = (int64_t)ch * kSaiChunk + (int64_t)threadIdx.x * kSaiPer;
    T vals[kSaiPer], lows[kSaiPer];
    const int cnt = sai_load(x, n, start, vals);
    if (xl) sai_load(xl, n, start, lows);
    R lam[kSaiPer];
#pragma unroll
    for (int j = 0; j < kSaiPer; ++j) lam[j] = load_coef<R>(cf.lam, start + j, n);
    __syncthreads();   // carry_f, carry_b
    R wv[kSaiPer];
    vsai_forward_values<T, R>(vals, lows, xl != nullptr, cnt, lam, carry_f, sa, sb, wv);
    R mu[kSaiPer];
    R gb = rfrom<R>(0.0), ga = rfrom<R>(1.0);
#pragma unroll
    for (int j = kSaiPer - 1; j >= 0; --j) {
        mu[j] = load_coef<R>(cf.mu, start + j, n);
        wv[j] = rmul(wv[j], load_coef<R>(cf.dinv, start + j, n));   // z = y / d
        if (j < cnt) {
            gb = rfma(mu[j], gb, wv[j]);
            ga = rmul(ga, mu[j]);
        }
    }
    R ea, eb, ta, tb;
    cta_affine_scan<R>(ga, gb, true, sa, sb, ea, eb, ta, tb);
    R xv = rfma(ea, rfrom<R>(carry_b), eb);
    T oh[kSaiPer], ol[kSaiPer];
#pragma unroll
    for (int j = kSaiPer - 1; j >= 0; --j) {
        if (j < cnt) {
            xv = rfma(mu[j], xv, wv[j]);
            split_r(xv, ylo != nullptr, oh[j], ol[j]);
        } else {
            oh[j] = ol[j] = T(0);
        }
    }
    sai_store(y, n, start, cnt, oh);
    if (ylo) sai_store(ylo, n, start, cnt, ol);
}

// Trapezoidal time mean of the iterate over each subinterval; grid (row chunks, P).
template <typename T>
__global__ void __launch_bounds__(256) k_window_average(const T* __restrict__ U, int64_t n,
                                                        const int* __restrict__ idx, double* __restrict__ ubar64,
                                                        T* __restrict__ ubarT, unsigned long long* __restrict__ umax_bits) {
    const int j = blockIdx.y;
    const int i0 = idx[j], i1 = idx[j + 1];
    const double inv = 1.0 / (double)(i1 - i0);
    double mx = 0.0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.5 * ((double)U[(int64_t)i0 * n + k] + (double)U[(int64_t)i1 * n + k]);
        for (int i = i0 + 1; i < i1; ++i) s += (double)U[(int64_t)i * n + k];
        s *= inv;
        ubar64[(int64_t)j * n + k] = s;
        ubarT[(int64_t)j * n + k] = (T)s;
        mx = fmax(mx, fabs(s));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(umax_bits + j, (unsigned long long)__double_as_longlong(mx));
}

// Window-major shifted source of the averaged-Jacobian iteration; grid (row chunks, rows).
template <typename T>
__global__ void __launch_bounds__(256) k_jac_source(Dim1 x, double inv2dx, const double* __restrict__ Au0,
                                                    const double* __restrict__ u0, const T* __restrict__ G,
                                                    const T* __restrict__ U, const double* __restrict__ ubar64,
                                                    const int* __restrict__ rw, const int* __restrict__ ri,
                                                    T* __restrict__ out) {
    const int64_t n = x.n;
    const int r = blockIdx.y;
    const int i = ri[r];
    const double* ub = ubar64 + (int64_t)rw[r] * n;
    const T* g = G + (int64_t)i * n;
    const T* u = U + (int64_t)i * n;
    T* o = out + (int64_t)r * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t km = k - 1, kp = k + 1;
        double em = 0.0, ep = 0.0, um = 0.0, up = 0.0;
        if (x.periodic) {
            if (km < 0) km += n;
            if (kp >= n) kp -= n;
        }
        if (km >= 0) { em = (double)u[km] - u0[km]; um = ub[km]; }
        if (kp < n) { ep = (double)u[kp] - u0[kp]; up = ub[kp]; }
        // J (u - u0) with (J v)_k = -(ubar_{k+1} v_{k+1} - ubar_{k-1} v_{k-1}) / (2 dx)
        const double je = -(up * ep - um * em) * inv2dx;
        o[k] = (T)(Au0[k] + (double)g[k] - je);
    }
}

// Y += J X (transpose: J^T X) for the Jacobian of the conservative Burgers term at the
// per-vector state U[v]:  (J x)_k = -(u_{k+1} x_{k+1} - u_{k-1} x_{k-1}) / (2 dx),
// (J^T x)_k = u_k (x_{k+1} - x_{k-1}) / (2 dx).  FP64 arithmetic; FP32 data read x as
// (hi, lo) and keep the result as a (hi, lo) pair.  Grid (row chunks, vectors).
template <typename T>
__global__ void __launch_bounds__(256) k_jac_add(int64_t n, int periodic, double inv2dx,
                                                 const double* const* __restrict__ Up, const T* const* __restrict__ Xp,
                                                 const float* const* __restrict__ Xlo, T* const* __restrict__ Yh,
                                                 T* const* __restrict__ Yl, int transpose) {
    const int v = blockIdx.y;
    const double* u = Up[v];
    const T* x = Xp[v];
    const float* xl = Xlo ? Xlo[v] : nullptr;
    T* yh = Yh[v];
    T* yl = Yl ? Yl[v] : nullptr;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t km = k - 1, kp = k + 1;
        if (periodic) {
            if (km < 0) km += n;
            if (kp >= n) kp -= n;
        }
        double xm = 0.0, xp = 0.0, um = 0.0, up = 0.0;
        if (km >= 0) { xm = (double)x[km] + (xl ? (double)xl[km] : 0.0); um = u[km]; }
        if (kp < n) { xp = (double)x[kp] + (xl ? (double)xl[kp] : 0.0); up = u[kp]; }
        const double j = transpose ? u[k] * (xp - xm) * inv2dx : -(up * xp - um * xm) * inv2dx;
        double y = (double)yh[k] + (yl ? (double)yl[k] : 0.0) + j;
        const T h = (T)y;
        yh[k] = h;
        if (yl) yl[k] = (T)(y - (double)h);
    }
}

}  // namespace

template <typename T>
void launch_jac_add(int64_t n, int periodic, double inv2dx, const double* const* U, const T* const* X,
                    const float* const* Xlo, T* const* Yh, T* const* Yl, int nvec, int transpose, cudaStream_t s) {
    if (nvec <= 0) return;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, std::max<int64_t>(1, 8 * kNumSM / nvec + 1));
    k_jac_add<T><<<dim3((unsigned)blocks, nvec), 256, 0, s>>>(n, periodic, inv2dx, U, X, Xlo, Yh, Yl, transpose);
}

void launch_vsai_factor(const Dim1& x, double gamma, double inv2dx, const VarOpTask* tasks_dev, int ntasks,
                        int64_t warm, cudaStream_t s) {
    if (ntasks <= 0) return;
    const int64_t nch = (x.n + kSaiChunk - 1) / kSaiChunk;
    dim3 g((unsigned)((nch + kFacThreads - 1) / kFacThreads), ntasks);
    k_vsai_factor<<<g, kFacThreads, 0, s>>>(x, gamma, inv2dx, tasks_dev, warm);
}

int64_t vsai_warmup(const Dim1& x, double gamma, double inv2dx, double umax) {
    const double g = gamma * (x.d + fabs(x.c) + umax * inv2dx);
    const double w = 40.0 * sqrt(1.0 + g) + 64.0;
    const double cap = x.periodic ? 2.0 * (double)x.n : (double)x.n;
    return (int64_t)std::min(w, cap);
}

template <typename T>
void launch_vsai_solve(int64_t n, const VarSai* coef, const T* const* X, const T* const* Xlo, T* const* Y,
                       T* const* Ylo, int nvec, double* scratch, cudaStream_t s, const int* const* skip) {
    if (nvec <= 0) return;
    const int nch = (int)((n + kSaiChunk - 1) / kSaiChunk);
    double* fends = scratch;
    double* fdec = fends + (size_t)nch * nvec;
    double* bends = fdec + (size_t)nch * nvec;
    double* bdec = bends + (size_t)nch * nvec;
    dim3 g(nch, nvec);
    launch_pdl(k_vsai_fwd_ends<T>, g, dim3(kSaiThreads), 0, s, n, nch, coef, X, Xlo, fends, fdec, skip);
    launch_pdl(k_vsai_fwd_apply<T>, g, dim3(kSaiThreads), 0, s, n, nch, coef, X, Xlo, (const double*)fends,
               (const double*)fdec, bends, bdec, skip);
    launch_pdl(k_vsai_bwd_apply<T>, g, dim3(kSaiThreads), 0, s, n, nch, coef, X, Xlo, Y, Ylo, (const double*)fends,
               (const double*)fdec, (const double*)bends, (const double*)bdec, skip);
}

template <typename T>
void launch_window_average(const T* U, int64_t n, const int* idx_dev, int P, double* ubar64, T* ubarT,
                           unsigned long long* umax_bits, cudaStream_t s) {
    if (P <= 0) return;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, std::max<int64_t>(1, 4 * kNumSM / P + 1));
    k_window_average<T><<<dim3((unsigned)blocks, P), 256, 0, s>>>(U, n, idx_dev, ubar64, ubarT, umax_bits);
}

template <typename T>
void launch_jac_source(const Dim1& x, double inv2dx, const double* Au0, const double* u0, const T* G, const T* U,
                       const double* ubar64, const int* rw, const int* ri, int nrows, T* out, cudaStream_t s) {
    if (nrows <= 0) return;
    const int64_t blocks = std::min<int64_t>((x.n + 255) / 256, std::max<int64_t>(1, 8 * kNumSM / nrows + 1));
    k_jac_source<T><<<dim3((unsigned)blocks, nrows), 256, 0, s>>>(x, inv2dx, Au0, u0, G, U, ubar64, rw, ri, out);
}

#define PEXP_VSAI_INST(T)                                                                                         \
    template void launch_vsai_solve<T>(int64_t, const VarSai*, const T* const*, const T* const*, T* const*,          \
                                       T* const*, int, double*, cudaStream_t, const int* const*);                   \
    template void launch_window_average<T>(const T*, int64_t, const int*, int, double*, T*, unsigned long long*,     \
                                           cudaStream_t);                                                            \
    template void launch_jac_source<T>(const Dim1&, double, const double*, const double*, const T*, const T*,         \
                                       const double*, const int*, const int*, int, T*, cudaStream_t);               \
    template void launch_jac_add<T>(int64_t, int, double, const double* const*, const T* const*, const float* const*, \
                                    T* const*, T* const*, int, int, cudaStream_t);
PEXP_VSAI_INST(double)
PEXP_VSAI_INST(float)

}  // namespace pexp
