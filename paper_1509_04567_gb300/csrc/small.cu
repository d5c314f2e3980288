// Per-subinterval small-matrix kernels (FP64, one CTA per window).
//
//  * source compression (Sec. 2.1): eigen-decomposition of the s x s Gram matrix
//    of the source samples by cyclic Jacobi rotations; the retained singular
//    triplets give U = Ghat Z_m Sigma_m^{-1} and coefficients Sigma_m Z_m^T;
//  * block orthonormalisation of a new Krylov block: Cholesky QR with diagonal
//    pivoting; directions whose remaining norm falls below a threshold relative
//    to the block's norm before Gram-Schmidt are dropped (block deflation);
//  * the cubic coefficient model p(t) (eq. svd_appr): not-a-knot cubic spline;
//  * the projected problem y' = H y + E_1 p(t) (or y' = H y, y(0) = beta e_1),
//    integrated exactly through the exponential of an augmented matrix, which is
//    computed by Pade scaling and squaring (Higham, SIAM J. Matrix Anal. Appl.
//    26 (2005), degrees 3/5/7/9/13 with their published theta_m bounds).
#include <math.h>

#include <algorithm>

#include <mutex>

#include "small.cuh"

namespace pexp {

WinLayout make_layout(int s_max, int b_max, int kmax, int ycols) {
    WinLayout L;
    L.s_max = s_max;
    L.b_max = b_max;
    L.ycols = ycols;
    L.K_max = b_max * (kmax + 1);
    L.N_max = L.K_max + 4 * b_max;
    int64_t o = 0;
    auto take = [&](int64_t cnt) {
        int64_t r = o;
        o += (cnt + 7) / 8 * 8;
        return r;
    };
    L.off_gram = take((int64_t)s_max * s_max);
    L.off_zs = take((int64_t)s_max * b_max);
    L.off_C = take((int64_t)b_max * s_max);
    L.off_coef = take((int64_t)std::max(1, s_max - 1) * 4 * b_max);
    L.off_H = take((int64_t)L.K_max * L.K_max);
    L.off_out1 = take((int64_t)(L.K_max + b_max) * ycols * b_max);
    L.off_h2 = take((int64_t)L.K_max * b_max);
    L.off_gw = take((int64_t)b_max * b_max);
    L.off_T = take((int64_t)b_max * b_max);
    L.off_Y = take((int64_t)s_max * L.K_max);
    L.off_Yp = take((int64_t)s_max * L.K_max);
    L.off_scal = take(WS_COUNT);
    L.off_scr = take((int64_t)9 * L.N_max * L.N_max);
    L.off_yk = take((int64_t)2 * L.K_max);
    L.stride = o;
    L.istride = WI_COUNT;
    return L;
}

// ---------------------------------------------------------------- Pade constants
__constant__ double c_pade[5][14];
static const int kPadeDeg[5] = {3, 5, 7, 9, 13};
// theta_m: largest ||A||_1 for which the degree-m diagonal Pade approximant meets
// double precision (Higham 2005, Table 2.3).
__constant__ double c_theta[5] = {1.495585217958292e-2, 2.539398330063230e-1, 9.504178996162932e-1,
                                  2.097847961257068e0, 5.371920351148152e0};

void init_pade_constants() {
    // constant memory is per device: the coefficients go to each device once
    static std::mutex mu;
    static bool done[128] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(mu);
    if (dev < 0 || dev >= 128 || done[dev]) return;
    double h[5][14] = {};
    for (int d = 0; d < 5; ++d) {
        const int m = kPadeDeg[d];
        // numerator coefficients of the [m/m] Pade approximant of exp:
        // c_j = (2m-j)! m! / ((2m)! j! (m-j)!),  c_{j+1} = c_j (m-j) / ((2m-j)(j+1))
        double c = 1.0;
        for (int j = 0; j <= m; ++j) {
            h[d][j] = c;
            c = c * (double)(m - j) / ((double)(2 * m - j) * (double)(j + 1));
        }
    }
    cudaMemcpyToSymbol(c_pade, h, sizeof(h));
    done[dev] = true;
}

// ---------------------------------------------------------------- CTA helpers
__device__ __forceinline__ int kPadeDeg_dev(int d) { return d == 0 ? 3 : d == 1 ? 5 : d == 2 ? 7 : d == 3 ? 9 : 13; }

__device__ __forceinline__ void cta_mm(const double* A, const double* B, double* C, int N) {
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i = e % N, j = e / N;
        double s = 0.0;
        for (int k = 0; k < N; ++k) s = fma(A[i + k * N], B[k + j * N], s);
        C[e] = s;
    }
    __syncthreads();
}

__device__ double cta_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
    __syncthreads();
    return r;
}

// Solve P X = Q in place (X overwrites Q) by Gaussian elimination with partial pivoting.
__device__ void cta_solve(double* P, double* Q, int N) {
    __shared__ int s_piv;
    const int lane = threadIdx.x & 31;
    for (int k = 0; k < N; ++k) {
        if (threadIdx.x < 32) {
            double best = -1.0;
            int bi = k;
            for (int i = k + lane; i < N; i += 32) {
                const double v = fabs(P[i + k * N]);
                if (v > best) { best = v; bi = i; }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (lane == 0) s_piv = bi;
        }
        __syncthreads();
        const int pv = s_piv;
        if (pv != k) {
            for (int j = threadIdx.x; j < N; j += blockDim.x) {
                double t = P[k + j * N]; P[k + j * N] = P[pv + j * N]; P[pv + j * N] = t;
                t = Q[k + j * N]; Q[k + j * N] = Q[pv + j * N]; Q[pv + j * N] = t;
            }
        }
        __syncthreads();
        const double d = P[k + k * N];
        for (int i = k + 1 + threadIdx.x; i < N; i += blockDim.x) P[i + k * N] /= d;
        __syncthreads();
        const int rem = N - k - 1;
        for (int e = threadIdx.x; e < rem * (rem + N); e += blockDim.x) {
            const int i = k + 1 + e % rem;
            const int jj = e / rem;
            if (jj < rem) {
                const int j = k + 1 + jj;
                P[i + j * N] -= P[i + k * N] * P[k + j * N];
            } else {
                const int j = jj - rem;
                Q[i + j * N] -= P[i + k * N] * Q[k + j * N];
            }
        }
        __syncthreads();
    }
    for (int k = N - 1; k >= 0; --k) {
        const double d = P[k + k * N];
        for (int j = threadIdx.x; j < N; j += blockDim.x) Q[k + j * N] /= d;
        __syncthreads();
        for (int e = threadIdx.x; e < k * N; e += blockDim.x) {
            const int i = e % k, j = e / k;
            Q[i + j * N] -= P[i + k * N] * Q[k + j * N];
        }
        __syncthreads();
    }
}

// E = exp(A) for an N x N column-major A (destroyed).  w: 7 N^2 doubles.
__device__ void cta_expm(double* A, int N, double* E, double* w) {
    __shared__ double red[32];
    // 1-norm: largest absolute column sum
    double cs = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double s = 0.0;
        for (int i = 0; i < N; ++i) s += fabs(A[i + j * N]);
        cs = fmax(cs, s);
    }
    const double nrm = cta_max(cs, red);
    int d = 4, sq = 0;
    for (int t = 0; t < 4; ++t)
        if (nrm <= c_theta[t]) { d = t; break; }
    if (d == 4 && nrm > c_theta[4]) {
        sq = (int)ceil(log2(nrm / c_theta[4]));
        if (sq < 0) sq = 0;
        const double sc = ldexp(1.0, -sq);
        for (int e = threadIdx.x; e < N * N; e += blockDim.x) A[e] *= sc;
        __syncthreads();
    }
    const int NN = N * N;
    double* A2 = w;
    double* A4 = w + NN;
    double* A6 = w + 2 * NN;
    double* U = w + 3 * NN;
    double* V = w + 4 * NN;
    double* T1 = w + 5 * NN;
    double* T2 = w + 6 * NN;
    const double* c = c_pade[d];
    const int m = kPadeDeg_dev(d);
    cta_mm(A, A, A2, N);
    if (m >= 5) cta_mm(A2, A2, A4, N);
    if (m >= 7) cta_mm(A4, A2, A6, N);
    if (m == 9) cta_mm(A6, A2, T2, N);  // A8 in T2
    if (m == 13) {
        for (int e = threadIdx.x; e < NN; e += blockDim.x) T1[e] = c[13] * A6[e] + c[11] * A4[e] + c[9] * A2[e];
        __syncthreads();
        cta_mm(A6, T1, U, N);
        for (int e = threadIdx.x; e < NN; e += blockDim.x) {
            const double id = (e % N == e / N) ? 1.0 : 0.0;
            U[e] += c[7] * A6[e] + c[5] * A4[e] + c[3] * A2[e] + c[1] * id;
            T2[e] = c[12] * A6[e] + c[10] * A4[e] + c[8] * A2[e];
        }
        __syncthreads();
        cta_mm(A, U, T1, N);   // odd part
        cta_mm(A6, T2, V, N);
        for (int e = threadIdx.x; e < NN; e += blockDim.x) {
            const double id = (e % N == e / N) ? 1.0 : 0.0;
            V[e] += c[6] * A6[e] + c[4] * A4[e] + c[2] * A2[e] + c[0] * id;
        }
        __syncthreads();
    } else {
        for (int e = threadIdx.x; e < NN; e += blockDim.x) {
            const double id = (e % N == e / N) ? 1.0 : 0.0;
            double u = c[1] * id + c[3] * A2[e];
            double v = c[0] * id + c[2] * A2[e];
            if (m >= 5) { u += c[5] * A4[e]; v += c[4] * A4[e]; }
            if (m >= 7) { u += c[7] * A6[e]; v += c[6] * A6[e]; }
            if (m >= 9) { u += c[9] * T2[e]; v += c[8] * T2[e]; }
            U[e] = u;
            V[e] = v;
        }
        __syncthreads();
        cta_mm(A, U, T1, N);
    }
    // r_m(A) = (V - U_odd)^{-1} (V + U_odd)
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
        const double u = T1[e], v = V[e];
        U[e] = v - u;
        E[e] = v + u;
    }
    __syncthreads();
    cta_solve(U, E, N);
    for (int k = 0; k < sq; ++k) {
        cta_mm(E, E, T1, N);
        for (int e = threadIdx.x; e < NN; e += blockDim.x) E[e] = T1[e];
        __syncthreads();
    }
}

// =====================================================================================
// Source compression: Jacobi eigen-decomposition of the Gram matrix (Sec. 2.1)
// =====================================================================================
constexpr int kEigThreads = 64;
constexpr int kEigRows = (PEXP_MAX_SAMPLES + kEigThreads - 1) / kEigThreads;   // rows per thread

__global__ void __launch_bounds__(kEigThreads) k_source_eig(WinLayout L, double* __restrict__ wd, int* __restrict__ wi,
                                                   const int* __restrict__ wins, double thr, int max_rank,
                                                   const double* __restrict__ dots, const double* __restrict__ nrm2,
                                                   Parts gp) {
    const int w = wins[blockIdx.x];
    double* D = wd + (int64_t)w * L.stride;
    int* I = wi + (int64_t)w * L.istride;
    const int s = I[WI_S];
    extern __shared__ double sm_eig[];
    double* A = sm_eig;          // s x s
    double* Z = A + s * s;       // s x s eigenvectors (columns)
    __shared__ double rot[3];
    __shared__ int order[PEXP_MAX_SAMPLES];
    __shared__ int s_more;
    const double* G = D + L.off_gram;
    const int i0 = I[WI_I0];
    const double na2 = *nrm2;
    for (int e = threadIdx.x; e < s * s; e += blockDim.x) {
        const int i = e % s, j = e / s;
        // (A u0 + g_i) . (A u0 + g_j) = ||A u0||^2 + (A u0).g_i + (A u0).g_j + g_i . g_j
        A[e] = na2 + (dots ? (dots[i0 + i] + dots[i0 + j]) + (gp.part ? 0.0 : G[e]) : 0.0);
        Z[e] = (i == j) ? 1.0 : 0.0;
    }
    if (dots && gp.part) {
        __syncthreads();
        for (int e = threadIdx.x >> 5; e < s * s; e += (int)(blockDim.x >> 5)) {
            const double v = parts_sum_warp(gp, blockIdx.x, e);
            if ((threadIdx.x & 31) == 0) A[e] += v;
        }
    }
    __syncthreads();
    for (int sweep = 0; sweep < 40; ++sweep) {
        if (threadIdx.x == 0) {
            double off = 0.0, dia = 0.0;
            for (int j = 0; j < s; ++j)
                for (int i = 0; i < s; ++i) {
                    const double v = A[i + j * s] * A[i + j * s];
                    if (i == j) dia += v; else off += v;
                }
            s_more = (off > 1e-32 * dia) ? 1 : 0;
        }
        __syncthreads();
        if (!s_more) break;
        for (int p = 0; p < s - 1; ++p)
            for (int q = p + 1; q < s; ++q) {
                if (threadIdx.x == 0) {
                    const double apq = A[p + q * s];
                    double c = 1.0, sn = 0.0, t = 0.0;
                    if (fabs(apq) > 1e-300) {
                        const double th = (A[q + q * s] - A[p + p * s]) / (2.0 * apq);
                        t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        sn = t * c;
                    }
                    rot[0] = c; rot[1] = sn; rot[2] = t;
                }
                __syncthreads();
                const double c = rot[0], sn = rot[1], t = rot[2];
                if (sn != 0.0) {
                    // rows k = threadIdx.x + kEigThreads u: all reads before the barrier, all writes after
                    double akp[kEigRows], akq[kEigRows], zkp[kEigRows], zkq[kEigRows];
#pragma unroll
                    for (int u = 0; u < kEigRows; ++u) {
                        const int k = threadIdx.x + kEigThreads * u;
                        akp[u] = akq[u] = zkp[u] = zkq[u] = 0.0;
                        if (k < s) {
                            akp[u] = A[k + p * s]; akq[u] = A[k + q * s];
                            zkp[u] = Z[k + p * s]; zkq[u] = Z[k + q * s];
                        }
                    }
                    __syncthreads();
#pragma unroll
                    for (int u = 0; u < kEigRows; ++u) {
                        const int k = threadIdx.x + kEigThreads * u;
                        if (k < s) {
                            if (k != p && k != q) {
                                const double np = c * akp[u] - sn * akq[u], nq = sn * akp[u] + c * akq[u];
                                A[k + p * s] = np; A[p + k * s] = np;
                                A[k + q * s] = nq; A[q + k * s] = nq;
                            }
                            Z[k + p * s] = c * zkp[u] - sn * zkq[u];
                            Z[k + q * s] = sn * zkp[u] + c * zkq[u];
                        }
                    }
                    const int k = threadIdx.x;
                    if (k == 0) {
                        const double apq = A[p + q * s];
                        A[p + p * s] -= t * apq;
                        A[q + q * s] += t * apq;
                        A[p + q * s] = 0.0;
                        A[q + p * s] = 0.0;
                    }
                }
                __syncthreads();
            }
    }
    if (threadIdx.x == 0) {
        for (int i = 0; i < s; ++i) order[i] = i;
        for (int i = 1; i < s; ++i) {  // insertion sort, descending eigenvalue
            int o = order[i], j = i - 1;
            while (j >= 0 && A[order[j] * (s + 1)] < A[o * (s + 1)]) { order[j + 1] = order[j]; --j; }
            order[j + 1] = o;
        }
        const double l1 = A[order[0] * (s + 1)];
        const double sig1 = l1 > 0 ? sqrt(l1) : 0.0;
        int m = 0;
        if (sig1 > 0) {
            for (int i = 0; i < s; ++i) {
                const double li = A[order[i] * (s + 1)];
                const double si = li > 0 ? sqrt(li) : 0.0;
                if (si > thr * sig1) m = i + 1; else break;
            }
            if (m > max_rank) m = max_rank;
            if (m > L.b_max) m = L.b_max;
            if (m < 1) m = 1;
        }
        I[WI_B] = m;
        double* sc = D + L.off_scal;
        if (m < s && sig1 > 0) {
            const double lm = A[order[m] * (s + 1)];
            sc[WS_SIGRATIO] = (lm > 0 ? sqrt(lm) : 0.0) / sig1;
        } else {
            sc[WS_SIGRATIO] = 0.0;
        }
    }
    __syncthreads();
    const int m = I[WI_B];
    double* zs = D + L.off_zs;   // s x b_max, ld s_max
    double* C = D + L.off_C;     // b_max x s, ld b_max
    for (int e = threadIdx.x; e < s * m; e += blockDim.x) {
        const int i = e % s, k = e / s;
        const int col = order[k];
        const double lk = A[col * (s + 1)];
        const double sk = lk > 0 ? sqrt(lk) : 0.0;
        zs[i + k * L.s_max] = (sk > 0) ? Z[i + col * s] / sk : 0.0;
        C[k + i * L.b_max] = sk * Z[i + col * s];
    }
}

void launch_source_eig(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, double thr, int max_rank,
                       const double* dots, const double* nrm2, cudaStream_t s, Parts gp) {
    if (nw <= 0) return;
    size_t sm = (size_t)2 * L.s_max * L.s_max * sizeof(double);
    if (sm > 32 * 1024) smem_optin(k_source_eig, sm);
    k_source_eig<<<nw, kEigThreads, sm, s>>>(L, wd, wi, wins, thr, max_rank, dots, nrm2, gp);
}

// =====================================================================================
// Start block: Cholesky of the Gram matrix of U (source) or of z (homogeneous).
//   source: T = R^{-1}, C <- R C;  homogeneous: T = 1/beta, beta = ||z||.
// =====================================================================================
__global__ void k_start_orth(WinLayout L, double* __restrict__ wd, int* __restrict__ wi, const int* __restrict__ wins) {
    const int w = wins[blockIdx.x];
    double* D = wd + (int64_t)w * L.stride;
    int* I = wi + (int64_t)w * L.istride;
    if (threadIdx.x != 0) return;
    const int b = I[WI_B];
    const double* G = D + L.off_gw;   // b x b, ld b
    double R[PEXP_MAX_RANK * PEXP_MAX_RANK];
    double Ti[PEXP_MAX_RANK * PEXP_MAX_RANK];
    for (int e = 0; e < b * b; ++e) { R[e] = 0.0; Ti[e] = 0.0; }
    int ok = 1;
    for (int j = 0; j < b; ++j) {
        double d = G[j + j * b];
        for (int k = 0; k < j; ++k) d -= R[k + j * b] * R[k + j * b];
        if (!(d > 0.0)) { ok = 0; d = 1e-300; }
        const double rjj = sqrt(d);
        R[j + j * b] = rjj;
        for (int l = j + 1; l < b; ++l) {
            double v = G[j + l * b];
            for (int k = 0; k < j; ++k) v -= R[k + j * b] * R[k + l * b];
            R[j + l * b] = v / rjj;
        }
    }
    // Ti = R^{-1} (upper triangular)
    for (int j = 0; j < b; ++j) {
        Ti[j + j * b] = 1.0 / R[j + j * b];
        for (int i = j - 1; i >= 0; --i) {
            double v = 0.0;
            for (int k = i + 1; k <= j; ++k) v += R[i + k * b] * Ti[k + j * b];
            Ti[i + j * b] = -v / R[i + i * b];
        }
    }
    double* T = D + L.off_T;
    for (int e = 0; e < b * b; ++e) T[e] = Ti[e];
    if (I[WI_KIND] == KIND_SOURCE) {
        double* C = D + L.off_C;
        const int s = I[WI_S];
        for (int i = 0; i < s; ++i) {
            double col[PEXP_MAX_RANK];
            for (int k = 0; k < b; ++k) col[k] = C[k + i * L.b_max];
            for (int k = 0; k < b; ++k) {
                double v = 0.0;
                for (int l = k; l < b; ++l) v += R[k + l * b] * col[l];
                C[k + i * L.b_max] = v;
            }
        }
    } else {
        D[L.off_scal + WS_BETA] = ok ? R[0] : 0.0;
        if (!ok) {
            // zero start vector: nothing to continue, the window is done with an empty basis
            I[WI_CONV] = 1;
            I[WI_K] = 0;
            I[WI_STEPS] = 0;
            for (int e = 0; e < b * b; ++e) T[e] = 0.0;
            return;
        }
    }
    if (!ok) I[WI_STATUS] = PEXP_ERR_BREAKDOWN;
}

void launch_start_orth(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, cudaStream_t s) {
    if (nw <= 0) return;
    k_start_orth<<<nw, 32, 0, s>>>(L, wd, wi, wins);
}

// =====================================================================================
// New Krylov block: Cholesky QR with diagonal pivoting and deflation.
//   pass 1: Gram G of W after Gram-Schmidt; columns whose remaining norm is below
//           defl * (largest column norm of W before Gram-Schmidt) are dropped;
//           T maps W to the kept orthonormal directions (columns 0..r-1), the rest 0.
//   pass 2: re-orthonormalise the kept columns (Cholesky of their Gram).
// =====================================================================================
__global__ void k_block_orth(WinLayout L, double* __restrict__ wd, int* __restrict__ wi, const int* __restrict__ wins,
                             int pass, int step, double defl, Parts gp) {
    pdl_entry();
    const int w = wins[blockIdx.x];
    double* D = wd + (int64_t)w * L.stride;
    int* I = wi + (int64_t)w * L.istride;
    if (I[WI_CONV]) return;  // converged (at this step's projection, or earlier)
    __shared__ double sG[PEXP_MAX_RANK * PEXP_MAX_RANK];
    block_orth_body(L, D, I, blockIdx.x, pass, step, defl, gp, -1, sG, D + L.off_T, true);
}

void launch_block_orth(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, int pass, int step,
                       double defl, cudaStream_t s, Parts gp) {
    if (nw <= 0) return;
    launch_pdl(k_block_orth, dim3(nw), dim3(32), 0, s, L, wd, wi, wins, pass, step, defl, gp);
}

// =====================================================================================
// Not-a-knot cubic spline through the coefficient samples C[:, i] at tau_i = i h
// (a line for 2 samples, a parabola for 3).  coef[(r*4 + l)*b_max + k] multiplies
// theta^l on [tau_r, tau_{r+1}].  Second derivatives sigma_i solve
//   h sigma_{i-1} + 4h sigma_i + h sigma_{i+1} = 6 (y_{i+1} - 2 y_i + y_{i-1}) / h
// with sigma_0, sigma_{s-1} eliminated by the not-a-knot conditions
// (continuous third derivative at tau_1 and tau_{s-2}).
// =====================================================================================
// Chebyshev knots of a window of length dT: tau_i = dT (1 - cos(pi i/(s-1))) / 2 (both ends exact).
__device__ __forceinline__ double cheb_knot(int i, int s, double dT) {
    if (i <= 0) return 0.0;
    if (i >= s - 1) return dT;
    return 0.5 * dT * (1.0 - cospi((double)i / (double)(s - 1)));
}

// The same not-a-knot spline through s samples at the Chebyshev knots of a window of length dT
// (spacings h_r = tau_{r+1} - tau_r):
//   h_{i-1} sigma_{i-1} + 2 (h_{i-1} + h_i) sigma_i + h_i sigma_{i+1}
//       = 6 ((y_{i+1} - y_i)/h_i - (y_i - y_{i-1})/h_{i-1}),  i = 1 .. s-2,
// with sigma_0 = sigma_1 + (h_0/h_1)(sigma_1 - sigma_2) and
// sigma_{s-1} = sigma_{s-2} + (h_{s-2}/h_{s-3})(sigma_{s-2} - sigma_{s-3}) (not-a-knot) substituted
// into the first and last rows; a line for 2 samples, the parabola through 3.
template <typename Y, typename Put>
__device__ void spline_knots(int s, double dT, Y y, Put put) {
    double hk[PEXP_MAX_SAMPLES];
    for (int r = 0; r + 1 < s; ++r) hk[r] = cheb_knot(r + 1, s, dT) - cheb_knot(r, s, dT);
    if (s == 2) {
        put(0, y(0), (y(1) - y(0)) / hk[0], 0.0, 0.0);
        return;
    }
    if (s == 3) {
        const double f01 = (y(1) - y(0)) / hk[0], f12 = (y(2) - y(1)) / hk[1];
        const double f012 = (f12 - f01) / (hk[0] + hk[1]);
        put(0, y(0), f01 - f012 * hk[0], f012, 0.0);
        put(1, y(1), f01 + f012 * hk[0], f012, 0.0);
        return;
    }
    double sig[PEXP_MAX_SAMPLES], cp[PEXP_MAX_SAMPLES];
    const int nI = s - 2;
    for (int i = 1; i <= nI; ++i) {
        const double h0 = hk[i - 1], h1 = hk[i];
        const double rhs = 6.0 * ((y(i + 1) - y(i)) / h1 - (y(i) - y(i - 1)) / h0);
        double a = h0, d = 2.0 * (h0 + h1), c = h1;
        if (i == 1) {   // sigma_0 eliminated
            d += h0 * (1.0 + h0 / h1);
            c -= h0 * h0 / h1;
            a = 0.0;
        }
        if (i == nI) {  // sigma_{s-1} eliminated
            d += h1 * (1.0 + h1 / h0);
            a -= h1 * h1 / h0;
            c = 0.0;
        }
        if (i == 1) {
            cp[i] = c / d;
            sig[i] = rhs / d;
        } else {
            const double m = d - a * cp[i - 1];
            cp[i] = c / m;
            sig[i] = (rhs - a * sig[i - 1]) / m;
        }
    }
    for (int i = nI - 1; i >= 1; --i) sig[i] -= cp[i] * sig[i + 1];
    sig[0] = sig[1] + hk[0] / hk[1] * (sig[1] - sig[2]);
    sig[s - 1] = sig[s - 2] + hk[s - 2] / hk[s - 3] * (sig[s - 2] - sig[s - 3]);
    for (int r = 0; r < s - 1; ++r) {
        const double hr = hk[r];
        const double c1 = (y(r + 1) - y(r)) / hr - hr * (2.0 * sig[r] + sig[r + 1]) / 6.0;
        put(r, y(r), c1, 0.5 * sig[r], (sig[r + 1] - sig[r]) / (6.0 * hr));
    }
}

__global__ void k_spline(WinLayout L, double* __restrict__ wd, int* __restrict__ wi, const int* __restrict__ wins,
                         double h) {
    const int w = wins[blockIdx.x];
    double* D = wd + (int64_t)w * L.stride;
    int* I = wi + (int64_t)w * L.istride;
    const int b = I[WI_B], s = I[WI_S];
    const int k = threadIdx.x;
    if (k >= b) return;
    const double* C = D + L.off_C;
    double* cf = D + L.off_coef;
    auto y = [&](int i) { return C[k + i * L.b_max]; };
    auto put = [&](int r, double c0, double c1, double c2, double c3) {
        cf[(r * 4 + 0) * L.b_max + k] = c0;
        cf[(r * 4 + 1) * L.b_max + k] = c1;
        cf[(r * 4 + 2) * L.b_max + k] = c2;
        cf[(r * 4 + 3) * L.b_max + k] = c3;
    };
    if (I[WI_CHEB]) {
        spline_knots(s, (I[WI_SOUT] - 1) * h, y, put);
        return;
    }
    if (s == 2) {
        put(0, y(0), (y(1) - y(0)) / h, 0.0, 0.0);
        return;
    }
    if (s == 3) {
        const double f01 = (y(1) - y(0)) / h, f12 = (y(2) - y(1)) / h, f012 = (f12 - f01) / (2.0 * h);
        put(0, y(0), f01 - f012 * h, f012, 0.0);
        put(1, y(1), f01 + f012 * h, f012, 0.0);
        return;
    }
    // unknowns sigma_1..sigma_{s-2}: tridiagonal (sub a, diag d, super c), rhs r
    double sig[PEXP_MAX_SAMPLES], cp[PEXP_MAX_SAMPLES];
    const int nI = s - 2;
    // uniform spacing: row 1 and row s-2 become 6h sigma = rhs after elimination
    for (int i = 1; i <= nI; ++i) {
        const double rhs = 6.0 * (y(i + 1) - 2.0 * y(i) + y(i - 1)) / h;
        double a = h, d = 4.0 * h, c = h;
        if (i == 1) { d += 2.0 * h; c -= h; a = 0.0; }        // sigma_0 = 2 sigma_1 - sigma_2
        if (i == nI) { d += 2.0 * h; a -= (i == 1 ? 0.0 : h); c = 0.0; }  // sigma_{s-1} = 2 sigma_{s-2} - sigma_{s-3}
        if (i == 1 && nI == 1) { a = 0.0; c = 0.0; }
        // Thomas forward sweep
        if (i == 1) {
            cp[i] = c / d;
            sig[i] = rhs / d;
        } else {
            const double m = d - a * cp[i - 1];
            cp[i] = c / m;
            sig[i] = (rhs - a * sig[i - 1]) / m;
        }
    }
    for (int i = nI - 1; i >= 1; --i) sig[i] -= cp[i] * sig[i + 1];
    sig[0] = 2.0 * sig[1] - sig[2 < s - 1 ? 2 : 1];
    sig[s - 1] = 2.0 * sig[s - 2] - sig[s - 3];
    if (s == 4) {  // both eliminations act on a 2 x 2 system: sigma_0 uses sigma_2, sigma_3 uses sigma_1
        sig[0] = 2.0 * sig[1] - sig[2];
        sig[3] = 2.0 * sig[2] - sig[1];
    }
    for (int r = 0; r < s - 1; ++r) {
        const double c1 = (y(r + 1) - y(r)) / h - h * (2.0 * sig[r] + sig[r + 1]) / 6.0;
        put(r, y(r), c1, 0.5 * sig[r], (sig[r + 1] - sig[r]) / (6.0 * h));
    }
}

void launch_spline(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, double h, cudaStream_t s) {
    if (nw <= 0) return;
    k_spline<<<nw, 32, 0, s>>>(L, wd, wi, wins, h);
}

// =====================================================================================
// Projected problem of block step `step` (basis V_{1:step}, K = step*b columns).
//   1. add block `step` of H = V^T A V from the projections of this step;
//   2. E = exp(M) of the augmented matrix
//        M = [[h H, h E_1, 0, 0, 0], [0, 0, I, 0, 0], [0, 0, 0, I, 0], [0, 0, 0, 0, I], [0]*5]
//      (homogeneous windows: M = h H), so that E holds e^{hH} and h phi_{l+1}(hH) E_1;
//   3. y(tau_{r+1}) = e^{hH} y(tau_r) + sum_l l! h^l [h phi_{l+1}(hH) E_1] c_{r,l}
//      from y(0) = 0 (source) or beta e_1 (homogeneous);
//   4. est = max_r ||y_step(tau_r) - y_{step-1}(tau_r)||, converged when
//      step >= 2 and est <= tol * max(scale_ref, max_r ||y(tau_r)||).
// =====================================================================================
// One step of length hh of the projected source problem from the state yin: the exponential of
// the augmented matrix M(hh) (as in k_project), then
//   yout = e^{hh H} yin + sum_l l! hh^l [hh phi_{l+1}(hh H) E_1] c_{r,l}
// with the cubic coefficients of knot interval r.  yout: K_max entries (zero beyond K).
__device__ void project_step(const WinLayout& L, const double* D, const double* H, int K, int b, int N, double hh,
                             int r, const double* yin, double* yout, double* M, double* E, double* work) {
    const int KM = L.K_max;
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i = e % N, j = e / N;
        double v = 0.0;
        if (i < K && j < K) v = hh * H[i + j * KM];
        else if (i < b && j >= K && j < K + b && (j - K) == i) v = hh;
        else if (i >= K && j >= K) {
            const int bi = (i - K) / b, bj = (j - K) / b;
            if (bj == bi + 1 && (i - K) % b == (j - K) % b) v = 1.0;
        }
        M[e] = v;
    }
    __syncthreads();
    cta_expm(M, N, E, work);
    const double* cf = D + L.off_coef;
    for (int a = threadIdx.x; a < KM; a += blockDim.x) {
        double v = 0.0;
        if (a < K) {
            for (int j = 0; j < K; ++j) v = fma(E[a + j * N], yin[j], v);
            double f = 1.0, hl = 1.0;
            for (int l = 0; l < 4; ++l) {
                double t = 0.0;
                for (int k = 0; k < b; ++k) t = fma(E[a + (K + l * b + k) * N], cf[(r * 4 + l) * L.b_max + k], t);
                v = fma(f * hl, t, v);
                hl *= hh;
                f *= (double)(l + 1);
            }
        }
        yout[a] = v;
    }
    __syncthreads();
}

// Projected source problem of a window sampled at its s Chebyshev knots (the spline's knots),
// solved at its srow output times q h, q = 0 .. srow-1: the state is carried from knot to
// knot, and an output time inside a knot interval is reached from the state at the knot
// before it with that interval's cubic (output times at a knot take its state).  Y's rows
// are the output times; the previous step's rows go to Yp first.
__device__ void project_cheb(const WinLayout& L, double* D, const double* H, int K, int b, int N, int s, int srow,
                             double h, double* M, double* E, double* work) {
    const int KM = L.K_max;
    double* Y = D + L.off_Y;
    double* Yp = D + L.off_Yp;
    const int Kp = K - b;
    for (int e = threadIdx.x; e < srow * KM; e += blockDim.x) {
        const int a = e % KM;
        Yp[e] = (a < Kp) ? Y[e] : 0.0;
    }
    __syncthreads();
    double* yc = D + L.off_yk;   // state at the current knot
    double* yn = yc + KM;
    for (int a = threadIdx.x; a < KM; a += blockDim.x) Y[a] = yc[a] = 0.0;
    __syncthreads();
    const double dT = (srow - 1) * h;
    const double eps = 1e-14 * dT;
    int q = 1;
    for (int r = 0; r + 1 < s; ++r) {
        const double ta = cheb_knot(r, s, dT), tb = cheb_knot(r + 1, s, dT);
        for (; q < srow && q * h < tb - eps; ++q) {
            double* yq = Y + (int64_t)q * KM;
            const double th = q * h - ta;
            if (th <= eps) {
                for (int a = threadIdx.x; a < KM; a += blockDim.x) yq[a] = yc[a];
                __syncthreads();
            } else {
                project_step(L, D, H, K, b, N, th, r, yc, yq, M, E, work);
            }
        }
        project_step(L, D, H, K, b, N, tb - ta, r, yc, yn, M, E, work);
        for (int a = threadIdx.x; a < KM; a += blockDim.x) yc[a] = yn[a];
        __syncthreads();
        for (; q < srow && fabs(q * h - tb) <= eps; ++q) {
            double* yq = Y + (int64_t)q * KM;
            for (int a = threadIdx.x; a < KM; a += blockDim.x) yq[a] = yc[a];
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(256) k_project(WinLayout L, double* __restrict__ wd, int* __restrict__ wi,
                                                 const int* __restrict__ wins, int step, double h, double tol,
                                                 double scale_ref, Parts fp, double dcoef, double ccoef, int nsm,
                                                 int only_ef, double jcoef, int rc0, int rc0p) {
    extern __shared__ double sm_proj[];   // 9 nsm^2 doubles when nsm > 0
    const int w = wins[blockIdx.x];
    double* D = wd + (int64_t)w * L.stride;
    int* I = wi + (int64_t)w * L.istride;
    __shared__ double red[32];
    if (I[WI_CONV]) return;  // converged at an earlier step (e.g. invariant subspace)
    const int b = I[WI_B], s = I[WI_S], kind = I[WI_KIND];
    const int K = step * b;
    const int ldo = (step + 1) * b;
    const int KM = L.K_max;
    double* H = D + L.off_H;
    const double* o1 = D + L.off_out1;
    // column blocks of out1: [0,b) V^T A V_i, [b,2b) V^T A^T V_i, and with ycols == 5 the
    // low parts [2b,3b), [3b,4b) of the same products (FP32 data)
    const bool lo = L.ycols == 5;
    if (fp.part) {
        // fused partials: E (K x b) | F (K x b) | h1 (K x b) | pre (b) per chunk
        double* o1w = D + L.off_out1;
        // only_ef: h1 and pre are summed into out1 by another kernel (the Gram-Schmidt
        // passes run concurrently with this one)
        const int nfield = only_ef ? 2 * K * b : 3 * K * b + b;
        // Jacobian sums Ja, Jb (K x b each) follow pre in the partials
        const int nj = jcoef != 0.0 ? 2 * K * b : 0;
        const int nwarps = blockDim.x >> 5;
        for (int e2 = threadIdx.x >> 5; e2 < nfield + nj; e2 += nwarps) {
            const int e = e2 < nfield ? e2 : 3 * K * b + b + (e2 - nfield);
            const double sacc = parts_sum_warp(fp, blockIdx.x, e);
            if ((threadIdx.x & 31) != 0) continue;
            if (e2 >= nfield) {
                D[L.off_scr + 2 * K * b + (e2 - nfield)] = sacc;   // Ja then Jb
            } else if (e < 2 * K * b) {
                // E and F: stage in the scratch area for the H assembly below
                D[L.off_scr + e] = sacc;
            } else {
                o1w[e - 2 * K * b] = sacc;   // h1 (K x b) then pre (b)
            }
        }
        __syncthreads();
        const double* Es = D + L.off_scr;
        const double* Fs = Es + K * b;
        const double* Ja = Fs + K * b;
        const double* Jb = Ja + K * b;
        for (int e = threadIdx.x; e < K * b; e += blockDim.x) {
            const int a = e % K, c = e / K;
            const double ja = nj ? jcoef * Ja[e] : 0.0, jb = nj ? jcoef * Jb[e] : 0.0;
            H[a + ((step - 1) * b + c) * KM] = -dcoef * Es[e] - ccoef * Fs[e] + ja;
            if (a < (step - 1) * b) H[((step - 1) * b + c) + a * KM] = -dcoef * Es[e] + ccoef * Fs[e] + jb;
        }
    } else {
        // restart cycles (rc0: first block of the current cycle, rc0p: of the previous one):
        // the new block couples to its own cycle, and as the first block of a cycle also
        // through its row to the previous cycle (the residual's range); other entries are 0
        const int k0 = rc0 * b, k0p = rc0p * b;
        const bool first = rc0 > 0 && step - 1 == rc0;
        for (int e = threadIdx.x; e < K * b; e += blockDim.x) {
            const int a = e % K, c = e / K;
            double v = o1[a + c * ldo];
            if (lo) v += o1[a + (2 * b + c) * ldo];
            H[a + ((step - 1) * b + c) * KM] = (a >= k0) ? v : 0.0;
        }
        for (int e = threadIdx.x; e < (step - 1) * b * b; e += blockDim.x) {
            const int a = e % ((step - 1) * b), c = e / ((step - 1) * b);
            double v = o1[a + (b + c) * ldo];
            if (lo) v += o1[a + (3 * b + c) * ldo];
            H[((step - 1) * b + c) + a * KM] = (a >= k0 || (first && a >= k0p)) ? v : 0.0;
        }
    }
    __syncthreads();
    const int N = (kind == KIND_SOURCE) ? K + 4 * b : K;
    // the augmented matrix, its exponential and the Pade work space: in shared memory when
    // they fit (each small product then costs shared-memory latency, not L2 latency)
    const int64_t mstride = nsm > 0 ? (int64_t)nsm * nsm : (int64_t)L.N_max * L.N_max;
    double* M = nsm > 0 ? sm_proj : D + L.off_scr;
    double* E = M + mstride;
    double* work = E + mstride;
    // Chebyshev samples: the knots are not the output times (one exponential per step, below)
    const bool cheb = kind == KIND_SOURCE && I[WI_CHEB];
    const int srow = cheb ? I[WI_SOUT] : s;   // rows of Y: the window's output times
    double* Y = D + L.off_Y;
    double* Yp = D + L.off_Yp;
    if (cheb) {
        project_cheb(L, D, H, K, b, N, s, srow, h, M, E, work);
    } else {
    for (int e = threadIdx.x; e < N * N; e += blockDim.x) {
        const int i = e % N, j = e / N;
        double v = 0.0;
        if (i < K && j < K) v = h * H[i + j * KM];
        else if (kind == KIND_SOURCE) {
            if (i < b && j >= K && j < K + b && (j - K) == i) v = h;
            else if (i >= K && j >= K) {
                const int bi = (i - K) / b, bj = (j - K) / b;
                if (bj == bi + 1 && (i - K) % b == (j - K) % b) v = 1.0;
            }
        }
        M[e] = v;
    }
    __syncthreads();
    cta_expm(M, N, E, work);
    const int Kp = K - b;
    for (int e = threadIdx.x; e < s * KM; e += blockDim.x) {
        const int a = e % KM;
        Yp[e] = (a < Kp) ? Y[e] : 0.0;
    }
    __syncthreads();
    const double beta = D[L.off_scal + WS_BETA];
    for (int a = threadIdx.x; a < KM; a += blockDim.x) Y[a] = (kind == KIND_HOM && a == 0) ? beta : 0.0;
    __syncthreads();
    const double* cf = D + L.off_coef;
    for (int r = 0; r + 1 < s; ++r) {
        const double* yr = Y + (int64_t)r * KM;
        double* yn = Y + (int64_t)(r + 1) * KM;
        for (int a = threadIdx.x; a < KM; a += blockDim.x) {
            double v = 0.0;
            if (a < K) {
                for (int j = 0; j < K; ++j) v = fma(E[a + j * N], yr[j], v);
                if (kind == KIND_SOURCE) {
                    double f = 1.0, hl = 1.0;
                    for (int l = 0; l < 4; ++l) {
                        double t = 0.0;
                        for (int k = 0; k < b; ++k)
                            t = fma(E[a + (K + l * b + k) * N], cf[(r * 4 + l) * L.b_max + k], t);
                        v = fma(f * hl, t, v);
                        hl *= h;
                        f *= (double)(l + 1);
                    }
                }
            }
            yn[a] = v;
        }
        __syncthreads();
    }
    }
    double dmax = 0.0, nmax = 0.0;
    for (int r = threadIdx.x; r < srow; r += blockDim.x) {
        double dd = 0.0, nn = 0.0, cc = 0.0;
        for (int a = 0; a < K; ++a) {
            const double y = Y[(int64_t)r * KM + a];
            const double df = y - Yp[(int64_t)r * KM + a];
            dd = fma(df, df, dd);
            nn = fma(y, y, nn);
            if (rc0 > 0 && a >= rc0 * b) cc = fma(y, y, cc);
        }
        // in a restart cycle the estimate also covers the cycle's own part of the solution
        dmax = fmax(dmax, sqrt(fmax(dd, cc)));
        nmax = fmax(nmax, sqrt(nn));
    }
    dmax = cta_max(dmax, red);
    nmax = cta_max(nmax, red);
    if (threadIdx.x == 0) {
        const double scale = fmax(scale_ref, nmax);
        D[L.off_scal + WS_EST] = (scale > 0) ? dmax / scale : 0.0;
        D[L.off_scal + WS_SCALE] = scale;
        I[WI_STEPS] = step;
        I[WI_K] = K;
        // no stop at the first step of a restart cycle: the new direction alone barely moves
        // the solution, and the estimate is far below the error there
        if (step >= 2 && dmax <= tol * scale && (rc0 == 0 || step - rc0 >= 2)) I[WI_CONV] = 1;
    }
}

void launch_project(const WinLayout& L, double* wd, int* wi, const int* wins, int nw, int step, double h, double tol,
                    double scale_ref, cudaStream_t s, Parts fp, double d, double cadv, int b_launch, int only_ef,
                    double jcoef, int rc0, int rc0p) {
    if (nw <= 0) return;
    // largest augmented matrix of this launch: step * b + 4 b (source windows)
    const int nl = b_launch > 0 ? std::min(L.N_max, (step + 4) * b_launch) : L.N_max;
    const size_t sm = (size_t)9 * nl * nl * sizeof(double);
    if (sm <= 200u * 1024u) {
        if (sm > 32 * 1024) smem_optin(k_project, sm);
        k_project<<<nw, 256, sm, s>>>(L, wd, wi, wins, step, h, tol, scale_ref, fp, d, cadv, nl, only_ef, jcoef, rc0,
                                      rc0p);
    } else {
        k_project<<<nw, 256, 0, s>>>(L, wd, wi, wins, step, h, tol, scale_ref, fp, d, cadv, 0, only_ef, jcoef, rc0, rc0p);
    }
}

// =====================================================================================
// Batched exponential of dense N x N matrices (row-major in and out).
// =====================================================================================
__global__ void __launch_bounds__(256) k_expm_batch(const double* __restrict__ M, double* __restrict__ Eo, int N,
                                                    double* __restrict__ scratch) {
    const int bidx = blockIdx.x;
    const int NN = N * N;
    double* A = scratch + (size_t)bidx * 9 * NN;
    double* E = A + NN;
    double* w = E + NN;
    // row-major in -> column-major work copy (A^T of the column-major view)
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
        const int i = e % N, j = e / N;
        A[i + j * N] = M[(size_t)bidx * NN + i * N + j];
    }
    __syncthreads();
    cta_expm(A, N, E, w);
    for (int e = threadIdx.x; e < NN; e += blockDim.x) {
        const int i = e % N, j = e / N;
        Eo[(size_t)bidx * NN + i * N + j] = E[i + j * N];
    }
}

size_t small_expm_scratch_doubles(int N) { return (size_t)9 * N * N; }

void launch_small_expm_batch(const double* M, double* E, int N, int batch, double* scratch, cudaStream_t s) {
    if (batch <= 0) return;
    k_expm_batch<<<batch, 256, 0, s>>>(M, E, N, scratch);
}

}  // namespace pexp
