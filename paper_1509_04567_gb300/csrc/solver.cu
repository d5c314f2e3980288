// Host orchestration of the Paraexp exponential block Krylov (PEBK) solver and the
// C ABI of include/pexp.h.
//
// Linear solve (Sec. 2.2, Fig. 3), on one GPU:
//   1. shift by u0: g_hat = A u0 + g (eq. linivp_shift); subinterval j owns the
//      samples t_{idx_{j-1}} .. t_{idx_j};
//   2. source compression per subinterval, all subintervals in one batch:
//      Gram matrix of g_hat samples, Jacobi eigen-decomposition, U = G_hat Z S^{-1},
//      Cholesky re-orthonormalisation, not-a-knot cubic coefficient model;
//   3. nonhomogeneous parts of all subproblems in one batch: block Krylov steps
//      (shift-and-invert solve or stencil, explicit Galerkin projection H = V^T A V,
//      block classical Gram-Schmidt with re-orthogonalisation, Cholesky QR twice),
//      exact projected solve at the window's samples, stop on the change between
//      successive steps;
//   4. homogeneous parts: by superposition (eq. superposition) the homogeneous
//      continuations of all earlier subproblems add up, on window m, to
//      exp((t - T_{m-1}) A) z_{m-1} with z_{m-1} = u_hat(T_{m-1}); one single-vector
//      Krylov solve per window carries that sum (P - 1 solves instead of P(P-1)/2);
//   5. reconstruction u(t_i) = u0 + V_nh y_nh(t_i) + V_h y_h(t_i), all windows in one batch.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "krylov.cuh"
#include "small.cuh"

using namespace pexp;

// ---------------------------------------------------------------- kernel-class timer
// Optional CUDA-event timing of kernel classes: events recorded around launches on the
// solve's stream, read back once the solve has completed.
struct KTimer {
    bool on = false;
    unsigned mask = 0xffu;   // timed classes (bit = PEXP_KC_*)
    unsigned sample = 0;     // time about 1 in 2^sample of the launches of those classes
    uint32_t rng = 0;        // xorshift32 state of the sample choice (fixed seed per call)
    bool pick() {
        if (!sample) return true;
        rng ^= rng << 13;
        rng ^= rng >> 17;
        rng ^= rng << 5;
        return (rng & ((1u << sample) - 1u)) == 0;
    }
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    struct Rec {
        int cls;
        cudaEvent_t a, b;
        double bytes, alg;
    };
    std::vector<Rec> recs;
    cudaEvent_t next() {
        if (used == pool.size()) {
            cudaEvent_t e;
            cudaEventCreate(&e);
            pool.push_back(e);
        }
        return pool[used++];
    }
    void reset(bool enable, unsigned classes, unsigned sample_log2) {
        on = enable;
        mask = classes ? classes : 0xffu;
        sample = sample_log2 < 16 ? sample_log2 : 15;
        rng = 0x9e3779b9u;
        used = 0;
        recs.clear();
    }
    ~KTimer() {
        for (auto e : pool) cudaEventDestroy(e);
    }
};

// ---------------------------------------------------------------- context
struct pexp_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    char* ws = nullptr;   // device workspace (small state, scratch)
    size_t ws_cap = 0;
    size_t ws_top = 0;
    char* bs = nullptr;   // device pool of the Krylov bases, sized once the block widths are known
    size_t bs_cap = 0;
    size_t bs_top = 0;
    // task staging: a ring of slots (pinned host | device), each guarded by an event so a
    // slot is rewritten only after its previous host-to-device copy has run
    char* stage_h[2] = {nullptr, nullptr};
    char* stage_d[2] = {nullptr, nullptr};
    size_t stage_cap = 0;   // bytes per slot
    cudaEvent_t slot_ev[16] = {};
    bool slot_busy[16] = {};
    int slot_next = 0;
    int* flags_h = nullptr;  // pinned copies of the per-window int state (lookahead of the Krylov loop)
    size_t flags_cap = 0;
    cudaEvent_t flag_ev[4] = {};   // one per pinned copy (kFlagBufs)
    // second stream: the projected solve of a Krylov step runs beside the Gram-Schmidt passes
    cudaStream_t s2 = nullptr;
    cudaEvent_t ev_sp = nullptr, ev_pj = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaEvent_t evp[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};   // phase boundaries
    int launches = 0;
    // host copies for host-pointer solves: outputs leave window by window on a copy stream
    void* io_d = nullptr;
    size_t io_cap = 0;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev_out = nullptr;
    // grid-barrier words (count, generation, error) of the cooperative launches on `stream`
    unsigned* bar = nullptr;
    // cooperative launches allowed: not for the workers of a batched solve, whose solves run
    // side by side (two grids that each fill the GPU must not wait on each other)
    bool coop = true;
    // batched solves: worker contexts, each on a stream of its own
    std::vector<pexp_ctx*> workers;
    int batch_workers = 0;    // tuned count (0: default)
    bool owns_stream = false; // a worker's stream belongs to it
    KTimer kt;
};

namespace {

constexpr size_t kAlign = 256;

// Relative thresholds below which a new Krylov direction counts as already in the
// space (block deflation): its norm after Gram-Schmidt over its norm before.  FP32
// data keep the working block in double-float, so directions far below FP32 rounding
// are still resolved; dropping them (a threshold near sqrt of FP32 epsilon) left the
// rounding noise of the stored basis, magnified by the shift-and-invert step,
// unresolved in the projected problem.
#ifndef PEXP_DEFL_FP64
#define PEXP_DEFL_FP64 1e-10
#endif
#ifndef PEXP_DEFL_FP32
#define PEXP_DEFL_FP32 1e-8
#endif
#ifndef PEXP_TN_EXACT_FP32
#define PEXP_TN_EXACT_FP32 0
#endif
constexpr size_t kStageBytes = 8u << 20;   // per half of the staging area
constexpr int kSlots = 16;                   // ring slots over both halves
constexpr int kFlagBufs = 4;                 // pinned copies of the window flags in flight
constexpr int kLookahead = 1;                // steps between queueing a step and reading its flags
static_assert(kLookahead + 1 <= kFlagBufs, "a flag copy is read before its buffer is reused");
static_assert(std::extent<decltype(pexp_ctx::flag_ev)>::value == kFlagBufs, "one event per flag copy");

// NVTX ranges of a solve's phases, shown by profilers (ncu, nsys) on the host timeline: one
// range at a time, the next phase closing the current one; the destructor closes the last
// (also when a phase throws).
struct NvtxPhases {
    bool open = false;
    void next(const char* name) {
        if (open) nvtxRangePop();
        nvtxRangePushA(name);
        open = true;
    }
    ~NvtxPhases() {
        if (open) nvtxRangePop();
    }
};

struct OomError {};
struct StatusError {
    int code;
};

void* ws_alloc(pexp_ctx* c, size_t bytes) {
    size_t off = (c->ws_top + kAlign - 1) / kAlign * kAlign;
    if (off + bytes > c->ws_cap) throw OomError();
    c->ws_top = off + bytes;
    return c->ws + off;
}

// Reserve `need` bytes of workspace up front (grows the buffer between calls).
int ws_reserve(pexp_ctx* c, size_t need) {
    if (need <= c->ws_cap) return PEXP_OK;
    if (c->ws) cudaFree(c->ws);
    c->ws = nullptr;
    c->ws_cap = 0;
    size_t cap = need + need / 8 + (64u << 20);
    if (cudaMalloc(&c->ws, cap) != cudaSuccess) {
        cudaGetLastError();
        if (cudaMalloc(&c->ws, need) != cudaSuccess) {
            cudaGetLastError();
            return PEXP_ERR_OOM;
        }
        cap = need;
    }
    c->ws_cap = cap;
    return PEXP_OK;
}

void* bs_alloc(pexp_ctx* c, size_t bytes) {
    size_t off = (c->bs_top + kAlign - 1) / kAlign * kAlign;
    if (off + bytes > c->bs_cap) throw OomError();
    c->bs_top = off + bytes;
    return c->bs + off;
}

int bs_reserve(pexp_ctx* c, size_t need) {
    c->bs_top = 0;
    if (need <= c->bs_cap) return PEXP_OK;
    if (c->bs) cudaFree(c->bs);
    c->bs = nullptr;
    c->bs_cap = 0;
    if (cudaMalloc(&c->bs, need) != cudaSuccess) {
        cudaGetLastError();
        return PEXP_ERR_OOM;
    }
    c->bs_cap = need;
    return PEXP_OK;
}

// Task staging: host-side byte buffer copied to the device in one transfer.
// Task arrays for one group of launches: filled on the host, copied to the device in one
// stream-ordered copy.  Each Stage takes the next slot of the context's ring; the host may
// run ahead of the device by up to kSlots - 1 stages.
struct Stage {
    pexp_ctx* c;
    int slot;
    char* h;
    char* d;
    size_t used = 0;
    Stage(pexp_ctx* c_, int) : c(c_) {
        slot = c->slot_next;
        c->slot_next = (slot + 1) % kSlots;
        if (c->slot_busy[slot]) {
            cudaEventSynchronize(c->slot_ev[slot]);
            c->slot_busy[slot] = false;
        }
        const int per = kSlots / 2;
        h = c->stage_h[slot / per] + (size_t)(slot % per) * c->stage_cap;
        d = c->stage_d[slot / per] + (size_t)(slot % per) * c->stage_cap;
    }
    template <typename X>
    X* put(const X* src, size_t count) {
        size_t off = (used + 15) / 16 * 16;
        size_t bytes = sizeof(X) * count;
        if (off + bytes > c->stage_cap) throw OomError();
        memcpy(h + off, src, bytes);
        used = off + bytes;
        return reinterpret_cast<X*>(d + off);
    }
    void flush() {
        if (!used) return;
        cudaMemcpyAsync(d, h, used, cudaMemcpyHostToDevice, c->stream);
        cudaEventRecord(c->slot_ev[slot], c->stream);
        c->slot_busy[slot] = true;
    }
};

// Time a launch sequence as kernel class `cls` moving `bytes` (the low parts of an FP32
// working block included) of which `alg` are algorithmic (every array at its storage
// width; alg < 0: the same as bytes).
template <typename F>
void timed(pexp_ctx* c, int cls, double bytes, F&& f, cudaStream_t on = nullptr, bool on_set = false,
           double alg = -1.0) {
    if (!c->kt.on || !((c->kt.mask >> cls) & 1u) || !c->kt.pick()) {
        f();
        return;
    }
    cudaStream_t st = on_set ? on : c->stream;
    cudaEvent_t a = c->kt.next(), b = c->kt.next();
    cudaEventRecord(a, st);
    f();
    cudaEventRecord(b, st);
    c->kt.recs.push_back({cls, a, b, bytes, alg < 0 ? bytes : alg});
}

void check_launch(pexp_ctx* c) {
    c->launches++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fail_cuda(e, "kernel launch", __FILE__, __LINE__);
        throw StatusError{PEXP_ERR_CUDA};
    }
}

void sync(pexp_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        fail_cuda(e, "cudaStreamSynchronize", __FILE__, __LINE__);
        throw StatusError{PEXP_ERR_CUDA};
    }
}

void d2h(pexp_ctx* c, void* dst, const void* src, size_t bytes) {
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) {
        fail_cuda(e, "cudaMemcpyAsync D2H", __FILE__, __LINE__);
        throw StatusError{PEXP_ERR_CUDA};
    }
    sync(c);
}

// Partial-sum buffers of the fused Krylov kernels and the source Gram kernel: one slot
// per (task, row chunk), each as wide as the largest partial (step projections at the
// last step, or an s x s Gram matrix).
size_t kpart_doubles(int P, int64_t n, int kmax, int b_cap, int smax) {
    // step projections with the Jacobian sums: 5 p b + b per chunk (p <= kmax b)
    const size_t width = std::max<size_t>((size_t)(5 * kmax * b_cap * b_cap + b_cap + b_cap * b_cap), (size_t)smax * smax);
    return krylov_partial_slots(P, n) * width + 64;
}

OpDesc make_opdesc(const pexp_operator& op) {
    OpDesc d;
    memset(&d, 0, sizeof(d));
    d.dim = op.dim;
    auto dim1 = [&](int64_t n, double a, double L, int64_t stride) {
        Dim1 r;
        const double dx = (op.bc == PEXP_BC_PERIODIC) ? L / (double)n : L / (double)(n + 1);
        r.n = n;
        r.stride = stride;
        r.d = op.nu / (dx * dx);
        r.c = a / (2.0 * dx);
        r.periodic = op.bc == PEXP_BC_PERIODIC;
        return r;
    };
    d.x = dim1(op.nx, op.ax, op.Lx, 1);
    if (op.dim == 2) {
        d.y = dim1(op.ny, op.ay, op.Ly, op.nx);
        d.n = op.nx * op.ny;
    } else {
        d.n = op.nx;
    }
    return d;
}

int validate(const pexp_operator* op, const pexp_options* o) {
    if (!op || !o) return PEXP_ERR_INVALID_ARG;
    if (op->dim != 1 && op->dim != 2) return PEXP_ERR_INVALID_ARG;
    if (op->nx < 3 || (op->dim == 2 && op->ny < 3)) return PEXP_ERR_INVALID_ARG;
    if (op->bc != PEXP_BC_PERIODIC && op->bc != PEXP_BC_DIRICHLET0) return PEXP_ERR_INVALID_ARG;
    if (!(op->nu >= 0.0) || !(op->Lx > 0.0) || (op->dim == 2 && !(op->Ly > 0.0))) return PEXP_ERR_INVALID_ARG;
    if (o->n_out < 2 || o->P < 1 || o->P > o->n_out - 1) return PEXP_ERR_INVALID_ARG;
    if (!(o->T > 0.0) || !(o->tol > 0.0) || !(o->svd_tol >= 0.0)) return PEXP_ERR_INVALID_ARG;
    if (o->max_rank < 1 || o->restart_len < 1 || o->max_restarts < 0) return PEXP_ERR_INVALID_ARG;
    if (o->restart_len * (o->max_restarts + 1) > PEXP_MAX_STEPS) return PEXP_ERR_INVALID_ARG;
    if (o->krylov != PEXP_KRYLOV_POLY && o->krylov != PEXP_KRYLOV_SAI) return PEXP_ERR_INVALID_ARG;
    if (o->precision != PEXP_FP64 && o->precision != PEXP_MIXED) return PEXP_ERR_INVALID_ARG;
    if (o->krylov == PEXP_KRYLOV_SAI && !(o->sai_gamma > 0.0)) return PEXP_ERR_INVALID_ARG;
    // largest subinterval sample count
    const int P = o->P, nt = o->n_out;
    int smax = 0;
    for (int j = 1; j <= P; ++j) {
        const int i0 = (int)(((int64_t)(j - 1) * (nt - 1)) / P), i1 = (int)(((int64_t)j * (nt - 1)) / P);
        smax = std::max(smax, i1 - i0 + 1);
    }
    if (smax > PEXP_MAX_SAMPLES) return PEXP_ERR_INVALID_ARG;
    if (o->nodes != PEXP_NODES_UNIFORM && o->nodes != PEXP_NODES_CHEBYSHEV) return PEXP_ERR_INVALID_ARG;
    if (o->nodes == PEXP_NODES_CHEBYSHEV && (o->n_samp < 2 || o->n_samp > PEXP_MAX_SAMPLES)) return PEXP_ERR_INVALID_ARG;
    if (!(o->sub_first == 0 && o->sub_last == 0) && !(0 <= o->sub_first && o->sub_first < o->sub_last && o->sub_last <= P))
        return PEXP_ERR_INVALID_ARG;
    if (o->krylov == PEXP_KRYLOV_SAI && op->dim != 1) return PEXP_ERR_UNSUPPORTED;
    return PEXP_OK;
}

// ---------------------------------------------------------------- Krylov driver
template <typename T>
struct Win {
    int w;        // window index in the small-state arrays
    T* V;         // basis, n x K_max column-major (ld n)
    T* S;         // scratch n x (ycols-1) b: A V_i, A^T V_i (and their low parts for FP32 data)
    int b;        // block width
    float* Wlo;   // FP32 data: low parts of the working block (n x b); NULL for FP64
    float* V1lo;  // FP32 data: low parts of the start block while it is formed (n x b); NULL for FP64
    VarSai vs{};                  // variable-coefficient solves: the window's factors
    const T* ubar = nullptr;      // Jacobian windows: the state of J (Galerkin sums)
    const double* ubar64 = nullptr;   // the same in FP64 (operator applications)
};

// Per-subinterval operators of a solve.  The averaged-Jacobian waveform relaxation gives
// subinterval j the tridiagonal operator A + J_j (Sec. 2.4, eq. piecewiseJac); a bounded
// mesh with the shift-and-invert space has one factored operator for all subintervals.
template <typename T>
struct WinOps {
    bool var = false;                 // shift-and-invert solves use the factors vs[j]
    std::vector<VarSai> vs;           // P entries
    bool jac = false;                 // Galerkin sums and operator applications include J_j
    std::vector<const T*> ubar;       // P entries: the state of J_j (T)
    std::vector<const double*> ubar64;   // and in FP64
    double inv2dx = 0.0;
    const T* Gwin = nullptr;          // window-major shifted source (rows idx_j + j ...), or NULL:
                                      // time-major G shifted by A u0 in every window
};


template <typename T>
struct Solver {
    pexp_ctx* c;
    cudaStream_t st;
    OpDesc od;
    int64_t n;
    const pexp_options* o;
    WinLayout L;
    double* wd;
    int* wi;
    double* partial;
    double* sai_scr;
    SaiCoef sai;
    double h;
    int kmax;
    double defl;
    double scale_ref;
    double* diag = nullptr;   // K_max x 48 doubles for the orthogonality diagnostic
    double* kpart[2] = {nullptr, nullptr};   // partial sums of the fused Krylov kernels
    bool fused = false;                        // 1D operator and block widths <= kKrylovMaxB
    bool var = false;                          // per-window variable-coefficient shift-and-invert solves
    bool jac = false;                          // per-window Jacobian terms in the operator
    double inv2dx = 0.0;
    std::vector<int> wi_host;
    std::vector<int> restarts;                 // restart cycles begun, per window
    bool coop_used = false;                    // a cooperative launch ran (check_coop reads its error word)

    GridBar gbar() const { return GridBar{c->bar, c->bar + 1, reinterpret_cast<int*>(c->bar + 2)}; }
    // A single window of one column (a link of the homogeneous chain) on a periodic constant-
    // coefficient operator: the shift-and-invert passes and part B of each step run as one
    // cooperative launch each (the same arithmetic, 2 launches instead of 9).  Only while the
    // step's grids are under one wave (n <= 2^18): a grid barrier costs ~3.5 us, more than the
    // launch gap that programmatic dependent launch leaves between full-size kernels (measured
    // at 2^20 points: 164 ms per solve cooperative, 152 ms separate; 2^15: 24.5 vs 27.5 ms).
    bool coop_ok(const std::vector<Win<T>>& act) const {
        return c->coop && act.size() == 1 && act[0].b == 1 && !var && !jac && od.dim == 1 && od.x.periodic &&
               o->krylov == PEXP_KRYLOV_SAI && !(o->diagnostics & PEXP_DIAG_NOCOOP) &&
               krylov_geom(1, n).nchunks < 3 * kNumSM;
    }
    // Separate launches with the partial-sum and Cholesky-QR kernels folded into the passes of
    // part B (update0 sums h1, scale_proj and scale factor their QRs): a single window (a link
    // of the chain, where 3 fewer launches per step pay; in the batched phase every CTA re-summing
    // the partials costs more than the launches it saves: 2^20 points, 152.4 against 150.0 ms),
    // its basis in the fused width range, and the step not cooperative
    bool fold_ok(const std::vector<Win<T>>& act, int step) const {
        if (act.size() != 1 || coop_ok(act)) return false;
        for (const auto& W : act)
            if (!proj_fused(step * W.b, W.b, sizeof(T))) return false;
        return true;
    }
    // after the cooperative launches: a bounded grid barrier that gave up ends the solve
    void check_coop() {
        if (!coop_used) return;
        int err = 0;
        d2h(c, &err, c->bar + 2, sizeof(int));
        if (err) {
            cudaMemsetAsync(c->bar, 0, 3 * sizeof(unsigned), st);
            sync(c);
            throw StatusError{PEXP_ERR_TIMEOUT};
        }
    }

    T* slot(const Win<T>& W, int blk) const { return W.V + (int64_t)blk * W.b * n; }
    double* D(int w) const { return wd + (int64_t)w * L.stride; }

    // max |V^T V - I| over the first K columns of V (diagnostic, one pass over V per 48 columns).
    // Restart cycles are orthonormal each, not to one another: the defect is taken per cycle
    // (restart_len blocks of b columns).
    double orth_defect_cycles(const T* V, int K, int b) {
        if (o->max_restarts <= 0 || b <= 0) return orth_defect(V, K);
        const int cw = o->restart_len * b;
        double m = 0.0;
        for (int k0 = 0; k0 < K; k0 += cw) m = std::max(m, orth_defect(V + (int64_t)k0 * n, std::min(cw, K - k0)));
        return m;
    }

    double orth_defect(const T* V, int K) {
        if (K <= 0) return 0.0;
        std::vector<double> G((size_t)K * K);
        for (int c0 = 0; c0 < K; c0 += 48) {
            const int q = std::min(48, K - c0);
            Stage sg(c, 0);
            TsTask<T> t;
            memset(&t, 0, sizeof(t));
            t.X = V; t.ldx = n; t.p = K; t.Y = V + (int64_t)c0 * n; t.ldy = n; t.q = q; t.q1 = q;
            t.out = diag;
            const TsTask<T>* dt = sg.put(&t, 1);
            sg.flush();
            launch_ts_tn<T>(dt, 1, K * q, q, n, partial, st, 1);
            check_launch(c);
            d2h(c, G.data() + (size_t)c0 * K, t.out, sizeof(double) * K * q);
        }
        double m = 0.0;
        for (int j = 0; j < K; ++j) {
            // zero columns (deflated directions) are skipped
            if (G[(size_t)j * K + j] < 0.5) continue;
            for (int i = 0; i < K; ++i) {
                if (G[(size_t)i * K + i] < 0.5) continue;
                m = std::max(m, fabs(G[(size_t)j * K + i] - (i == j ? 1.0 : 0.0)));
            }
        }
        return m;
    }

    // Fused block Krylov steps (1D operators, block widths <= kKrylovMaxB): per step one
    // projection pass (Galerkin sums by parts, first Gram-Schmidt coefficients, norms),
    // the projected solve, and four passes for block Gram-Schmidt with Cholesky QR,
    // applied twice: update + Gram, scaling + second projection, update + Gram, scaling.
    //
    // Every kernel of a step skips a window whose convergence flag is set, so the host does
    // not wait for a step's flags before queueing the next step: the flags of step k come
    // back by an asynchronous copy and are read (to drop converged windows) after step k+1
    // has been queued.  A window converged at step k costs one step of empty launches.
    int run_fused(std::vector<Win<T>> ws, int* max_steps) {
        int notconv = 0;
        *max_steps = 0;
        std::stable_sort(ws.begin(), ws.end(), [](const Win<T>& a, const Win<T>& b) { return a.b < b.b; });
        std::vector<Win<T>> act = ws;
        const int periodic = od.x.periodic;
        const size_t nint = wi_host.size();
        if (c->flags_cap < kFlagBufs * nint) {
            if (c->flags_h) cudaFreeHost(c->flags_h);
            c->flags_h = nullptr;
            c->flags_cap = 0;
            if (cudaMallocHost(&c->flags_h, sizeof(int) * kFlagBufs * nint) != cudaSuccess) throw OomError();
            c->flags_cap = kFlagBufs * nint;
        }
        for (int k = 0; k < kFlagBufs; ++k)
            if (!c->flag_ev[k]) cudaEventCreateWithFlags(&c->flag_ev[k], cudaEventDisableTiming);
        auto conv_of = [&](const Win<T>& W) { return wi + (size_t)W.w * L.istride + WI_CONV; };
        // a cooperative step leaves its projected solve running on the second stream into the
        // next step's shift-and-invert launch (which needs neither its result nor its buffers);
        // the next projection pass, which reuses the partial sums it reads, waits for it
        bool pj_pending = false;
        for (int step = 1; step <= kmax && !act.empty(); ++step) {
            const int na = (int)act.size();
            int bmax = 0;
            for (auto& W : act) bmax = std::max(bmax, W.b);
            const KGeom g = krylov_geom(na, n);
            const int ps1 = (jac ? 5 : 3) * step * bmax * bmax + bmax;   // step_proj partial stride
            // ---- part A
            Stage sa(c, 0);
            std::vector<const T*> xin;
            std::vector<T*> yout, ylo;
            std::vector<StepTask<T>> st1(na);
            std::vector<int> wl(na);
            std::vector<const int*> skip;
            std::vector<VarSai> vcs;
            for (int a = 0; a < na; ++a) {
                const Win<T>& W = act[a];
                T* Vi = slot(W, step - 1);
                T* Wn = slot(W, step);
                // the solve takes the stored (rounded) block: the projected matrix is formed
                // from the stored basis, and any part of the input outside it (e.g. a low part
                // of the rounding) would follow the wrong projected dynamics
                for (int cc = 0; cc < W.b; ++cc) {
                    xin.push_back(Vi + (int64_t)cc * n);
                    yout.push_back(Wn + (int64_t)cc * n);
                    ylo.push_back(W.Wlo ? reinterpret_cast<T*>(W.Wlo) + (int64_t)cc * n : nullptr);
                    skip.push_back(conv_of(W));
                    vcs.push_back(W.vs);
                }
                st1[a] = StepTask<T>{W.V, n, step * W.b, conv_of(W), W.ubar};
                wl[a] = W.w;
            }
            const int nv = (int)xin.size();
            const T* const* d_xin = sa.put(xin.data(), nv);
            T* const* d_yout = sa.put(yout.data(), nv);
            T* const* d_ylo = std::is_same<T, float>::value ? sa.put(ylo.data(), nv) : nullptr;
            const StepTask<T>* d_st1 = sa.put(st1.data(), na);
            const int* const* d_skip = sa.put(skip.data(), nv);
            const int* d_wl = sa.put(wl.data(), na);
            const VarSai* d_vcs = var ? sa.put(vcs.data(), nv) : nullptr;
            sa.flush();
            const double w = sizeof(T);
            const double wout = std::is_same<T, float>::value ? 8.0 : w;
            if (o->krylov == PEXP_KRYLOV_SAI) {
                bool one = false;
                timed(c, PEXP_KC_SAI, (double)nv * n * (w + wout), [&] {
                    if (coop_ok(act))
                        one = launch_sai_coop<T>(od, sai, xin[0], yout[0], ylo[0], sai_scr, conv_of(act[0]), gbar(), st);
                    if (one) coop_used = true;
                    else if (var) launch_vsai_solve<T>(n, d_vcs, d_xin, nullptr, d_yout, d_ylo, nv, sai_scr, st, d_skip);
                    else launch_sai_solve_lo<T>(od, sai, d_xin, nullptr, d_yout, d_ylo, nv, sai_scr, st, d_skip);
                }, nullptr, false, 2.0 * nv * n * w);
                if (!one) c->launches += 2;   // the solve is three kernels; check_launch below counts one
            } else {
                timed(c, PEXP_KC_STENCIL, (double)nv * n * (w + w), [&] { launch_stencil_ptrs<T>(od, d_xin, d_yout, nv, 0, st); });
                for (const auto& W : act)
                    if (W.Wlo) cudaMemsetAsync(W.Wlo, 0, sizeof(float) * (size_t)n * W.b, st);
            }
            check_launch(c);
            double by1 = 0;
            for (auto& W : act) by1 += (double)n * (step + 1) * W.b * w;
            if (pj_pending) {
                cudaStreamWaitEvent(st, c->ev_pj, 0);
                pj_pending = false;
            }
            timed(c, PEXP_KC_PROJ, by1, [&] {
                for (int a0 = 0; a0 < na;) {
                    int a1 = a0;
                    while (a1 < na && act[a1].b == act[a0].b) ++a1;
                    launch_step_proj<T>(d_st1 + a0, a1 - a0, act[a0].b, step * act[a0].b, n, periodic, g,
                                        kpart[0] + (size_t)a0 * g.nchunks * ps1, ps1, st, jac);
                    check_launch(c);
                    a0 = a1;
                }
            });
            // h1 and the pre-Gram-Schmidt norms for the passes below; the projected solve (the
            // Galerkin matrix, its exponential, the convergence test) runs on the second stream
            // beside them: it is FP64-bound on one SM per window, the passes are HBM-bound
            cudaEventRecord(c->ev_sp, st);
            if (!fold_ok(act, step)) timed(c, PEXP_KC_SMALL, 0.0, [&] {
                for (int a0 = 0; a0 < na;) {
                    int a1 = a0;
                    while (a1 < na && act[a1].b == act[a0].b) ++a1;
                    const int bb = act[a0].b, pp = step * bb;
                    launch_sum_parts(kpart[0] + (size_t)a0 * g.nchunks * ps1, g.nchunks, ps1, pp * bb + bb, wd, L.stride,
                                     L.off_out1, d_wl + a0, a1 - a0, wi, L.istride, WI_CONV, st, 2 * pp * bb);
                    check_launch(c);
                    a0 = a1;
                }
            });
            // a cooperative part B fills the GPU: queue it first, so that the projected solve
            // starts beside the next step's shift-and-invert launch instead of holding back its grid
            const bool coop_step = coop_ok(act);
            if (coop_step && step < kmax) part_b(act, step);
            cudaStreamWaitEvent(c->s2, c->ev_sp, 0);
            timed(c, PEXP_KC_SMALL, 0.0, [&] {
                launch_project(L, wd, wi, d_wl, na, step, h, o->tol, scale_ref, c->s2, Parts{kpart[0], g.nchunks, ps1},
                               od.x.d, od.x.c, bmax, 1, jac ? inv2dx : 0.0);
            }, c->s2, true);
            check_launch(c);
            cudaEventRecord(c->ev_pj, c->s2);
            if (!coop_step && step < kmax) part_b(act, step);
            int* fl = c->flags_h + (size_t)(step % kFlagBufs) * nint;
            // The flags of this step go back behind its projected solve, on its stream, so that
            // no copy and no wait sit between the main stream's kernels (programmatic dependent
            // launch chains part B into the next step's shift-and-invert passes, which need
            // neither the projected solve's results nor its buffers; a window it marks converged
            // costs them one step of work that is never used).  The next projection pass, which
            // overwrites the partial sums the projected solve reads, waits for it.  The host
            // reads the flags of the step kLookahead before, so that it prepares the next
            // launches while the device runs this step.
            cudaMemcpyAsync(fl, wi, sizeof(int) * nint, cudaMemcpyDeviceToHost, c->s2);
            cudaEventRecord(c->flag_ev[step % kFlagBufs], c->s2);
            pj_pending = true;
            if (step > kLookahead) {
                const int old = (step - kLookahead) % kFlagBufs;
                cudaEventSynchronize(c->flag_ev[old]);
                const int* F = c->flags_h + (size_t)old * nint;
                std::vector<Win<T>> next;
                for (auto& W : act)
                    if (!F[(size_t)W.w * L.istride + WI_CONV]) next.push_back(W);
                act.swap(next);
            }
        }
        if (pj_pending) cudaStreamWaitEvent(st, c->ev_pj, 0);
        d2h(c, wi_host.data(), wi, sizeof(int) * nint);
        for (auto& W : ws) {
            const int* I = &wi_host[(size_t)W.w * L.istride];
            *max_steps = std::max(*max_steps, I[WI_STEPS]);
            if (!I[WI_CONV]) ++notconv;
        }
        return notconv;
    }

    // Part B of a fused step: block classical Gram-Schmidt with Cholesky QR, twice (BCGS2).
    // Part B of a fused step: block classical Gram-Schmidt with Cholesky QR, twice (BCGS2).
    // All its partial sums go through kpart[1]: kpart[0] holds the step projections, which
    // the projected solve on the second stream may still be reading.
    void part_b(const std::vector<Win<T>>& act, int step) {
        if (coop_ok(act)) {
            // the same four passes and two QRs as below, for the single window, in one launch
            const Win<T>& W = act[0];
            T* Wn = slot(W, step);
            const int p = step * W.b;
            UpdTask<T> u[4];
            memset(u, 0, sizeof(u));
            UpdTask<T> t;
            memset(&t, 0, sizeof(t));
            t.V = W.V; t.Wh = Wn; t.Wl = W.Wlo; t.ld = n; t.p = p;
            t.conv = wi + (size_t)W.w * L.istride + WI_CONV;
            t.hm = D(W.w) + L.off_out1; t.ldh = p;   // h1 from the projection pass
            u[0] = t;
            t.hm = nullptr; t.ldh = W.b;              // W <- W T1 (T1 from the first QR), h2 = V^T W
            u[1] = t;
            u[2] = t;                                 // W <- W - V h2 (h2 summed from the partials)
            memset(&t, 0, sizeof(t));
            t.Wh = Wn; t.Wl = W.Wlo; t.ld = n; t.p = W.b; t.ldh = W.b;
            t.conv = wi + (size_t)W.w * L.istride + WI_CONV;
            t.out = Wn;                               // W T2 rounded into the slot
            u[3] = t;
            const KGeom gb = krylov_geom(1, n);
            const double w = sizeof(T);
            const double wl_ = std::is_same<T, float>::value ? 8.0 : w;
            const double pb = (double)p, bb = (double)W.b;
            const double bytes = 2.0 * n * (pb * w + 2 * bb * wl_) + (double)n * (pb * w + 2 * bb * wl_) +
                                 (double)n * bb * (wl_ + w);
            const double alg = 3.0 * n * (pb * w + 2 * bb * w) + 2.0 * n * bb * w;
            bool one = false;
            timed(c, PEXP_KC_UPDATE, bytes, [&] {
                one = launch_gs_coop<T>(u, W.b, p, n, gb, kpart[1], p * W.b, W.b * W.b, L, wd, wi, W.w, step, defl,
                                        gbar(), st);
            }, nullptr, false, alg);
            if (one) {
                coop_used = true;
                ++c->launches;
                return;
            }
        }
        {
            const double w = sizeof(T);
            const int nb = (int)act.size();
            const KGeom gb = krylov_geom(nb, n);
            int bmb = 0;
            for (auto& W : act) bmb = std::max(bmb, W.b);
            const int ps2 = step * bmb * bmb;   // h2 partial stride
            const int psg = bmb * bmb;          // Gram partial stride
            Stage sb(c, 1);
            std::vector<UpdTask<T>> u1(nb), u2(nb), u3(nb), u4(nb);
            std::vector<int> wl2(nb);
            for (int a = 0; a < nb; ++a) {
                const Win<T>& W = act[a];
                T* Wn = slot(W, step);
                const int p = step * W.b;
                UpdTask<T> t;
                memset(&t, 0, sizeof(t));
                t.V = W.V; t.Wh = Wn; t.Wl = W.Wlo; t.ld = n; t.p = p;
                t.conv = wi + (size_t)W.w * L.istride + WI_CONV;
                t.hm = D(W.w) + L.off_out1; t.ldh = p;                         // h1 from the projection pass
                u1[a] = t;
                t.hm = D(W.w) + L.off_T; t.ldh = W.b;                          // W <- W T1, h2 = V^T W
                u3[a] = t;
                t.hm = D(W.w) + L.off_h2; t.ldh = p;                           // unused: the pass sums h2 itself
                u2[a] = t;
                memset(&t, 0, sizeof(t));
                t.Wh = Wn; t.Wl = W.Wlo; t.ld = n; t.p = W.b; t.hm = D(W.w) + L.off_T; t.ldh = W.b;
                t.conv = wi + (size_t)W.w * L.istride + WI_CONV;
                t.out = Wn;
                u4[a] = t;                                                     // final: W T2 rounded into the slot
                wl2[a] = W.w;
            }
            const UpdTask<T>* d1 = sb.put(u1.data(), nb);
            const UpdTask<T>* d2 = sb.put(u2.data(), nb);
            const UpdTask<T>* d3 = sb.put(u3.data(), nb);
            const UpdTask<T>* d4 = sb.put(u4.data(), nb);
            const int* d_wl2 = sb.put(wl2.data(), nb);
            sb.flush();
            double pb = 0, bb = 0;
            for (auto& W : act) { pb += (double)step * W.b; bb += W.b; }
            const double wl_ = std::is_same<T, float>::value ? 8.0 : w;   // bytes per element of the working block
            auto groups = [&](auto&& f) {
                for (int a0 = 0; a0 < nb;) {
                    int a1 = a0;
                    while (a1 < nb && act[a1].b == act[a0].b) ++a1;
                    f(a0, a1, act[a0].b);
                    a0 = a1;
                }
            };
            const double alg_upd = (double)n * (pb * w + 2 * bb * w);
            if (fold_ok(act, step)) {
                // partial sums: Gram of pass 1 | h2 | Gram of pass 2, each pass's in its own
                // region (a kernel reads one pass's partials while writing the next one's)
                const size_t rg = (size_t)nb * gb.nchunks * psg, rh = (size_t)nb * gb.nchunks * ps2;
                double* pg1 = kpart[1];
                double* ph2 = pg1 + rg;
                double* pg2 = ph2 + rh;
                const int ps1 = (jac ? 5 : 3) * step * bmb * bmb + bmb;   // projection partial stride
                timed(c, PEXP_KC_UPDATE, (double)n * (pb * w + 2 * bb * wl_), [&] {
                    groups([&](int a0, int a1, int b) {
                        launch_update0_h<T>(d1 + a0, a1 - a0, b, step * b, n, gb, pg1 + (size_t)a0 * gb.nchunks * psg, psg,
                                            kpart[0] + (size_t)a0 * gb.nchunks * ps1, ps1, 2 * step * b * b, st);
                        check_launch(c);
                    });
                }, nullptr, false, alg_upd);
                timed(c, PEXP_KC_UPDATE, (double)n * (pb * w + 2 * bb * wl_), [&] {
                    groups([&](int a0, int a1, int b) {
                        launch_scale_proj_qr<T>(d3 + a0, a1 - a0, b, n, gb, ph2 + (size_t)a0 * gb.nchunks * ps2, ps2, L, wd, wi,
                                                d_wl2 + a0, step, defl, pg1 + (size_t)a0 * gb.nchunks * psg, psg,
                                                kpart[0] + (size_t)a0 * gb.nchunks * ps1, ps1, 3 * step * b * b, st);
                        check_launch(c);
                    });
                }, nullptr, false, alg_upd);
                timed(c, PEXP_KC_UPDATE, (double)n * (pb * w + 2 * bb * wl_), [&] {
                    groups([&](int a0, int a1, int b) {
                        launch_update<T>(d2 + a0, a1 - a0, b, step * b, n, 1, gb, pg2 + (size_t)a0 * gb.nchunks * psg, psg, st,
                                         ph2 + (size_t)a0 * gb.nchunks * ps2, ps2);
                        check_launch(c);
                    });
                }, nullptr, false, alg_upd);
                timed(c, PEXP_KC_UPDATE, (double)n * bb * (wl_ + w), [&] {
                    groups([&](int a0, int a1, int b) {
                        launch_scale_qr<T>(d4 + a0, a1 - a0, b, n, gb, L, wd, wi, d_wl2 + a0, step, defl,
                                           pg2 + (size_t)a0 * gb.nchunks * psg, psg, st);
                        check_launch(c);
                    });
                }, nullptr, false, 2.0 * n * bb * w);
                return;
            }
            // pass 1: W <- W - V h1 (Gram of the result), Cholesky QR with deflation
            timed(c, PEXP_KC_UPDATE, (double)n * (pb * w + 2 * bb * wl_), [&] {
                groups([&](int a0, int a1, int b) {
                    launch_update<T>(d1 + a0, a1 - a0, b, step * b, n, 0, gb, kpart[1] + (size_t)a0 * gb.nchunks * psg, psg, st);
                    check_launch(c);
                });
            }, nullptr, false, alg_upd);
            timed(c, PEXP_KC_SMALL, 0.0, [&] {
                launch_block_orth(L, wd, wi, d_wl2, nb, 1, step, defl, st, Parts{kpart[1], gb.nchunks, psg});
            });
            check_launch(c);
            // pass 2: W <- W T1 and h2 = V^T W; W <- W - V h2 (Gram), Cholesky QR; round into the basis
            timed(c, PEXP_KC_UPDATE, (double)n * (pb * w + 2 * bb * wl_), [&] {
                groups([&](int a0, int a1, int b) {
                    launch_scale_proj<T>(d3 + a0, a1 - a0, b, step * b, n, gb, kpart[1] + (size_t)a0 * gb.nchunks * ps2, ps2, st);
                    check_launch(c);
                });
            }, nullptr, false, alg_upd);
            // the second pass sums h2 from the partials above itself; its Gram partials go after
            // them in the same buffer (ps2 + psg <= the buffer's width per chunk slot)
            const size_t off2 = (size_t)nb * gb.nchunks * ps2;
            timed(c, PEXP_KC_UPDATE, (double)n * (pb * w + 2 * bb * wl_), [&] {
                groups([&](int a0, int a1, int b) {
                    launch_update<T>(d2 + a0, a1 - a0, b, step * b, n, 1, gb, kpart[1] + off2 + (size_t)a0 * gb.nchunks * psg,
                                     psg, st, kpart[1] + (size_t)a0 * gb.nchunks * ps2, ps2);
                    check_launch(c);
                });
            }, nullptr, false, alg_upd);
            timed(c, PEXP_KC_SMALL, 0.0, [&] {
                launch_block_orth(L, wd, wi, d_wl2, nb, 2, step, defl, st, Parts{kpart[1] + off2, gb.nchunks, psg});
            });
            check_launch(c);
            timed(c, PEXP_KC_UPDATE, (double)n * bb * (wl_ + w), [&] {
                groups([&](int a0, int a1, int b) {
                    launch_scale<T>(d4 + a0, a1 - a0, b, n, 0, gb, nullptr, psg, st);
                    check_launch(c);
                });
            }, nullptr, false, 2.0 * n * bb * w);
        }
    }

    // Runs block Krylov steps for the windows `ws` (each with its start block already
    // orthonormal in V block 0).  Returns the number of windows that missed tol.
    int run(std::vector<Win<T>> ws, int kind, int* max_steps) {
        if (fused) return run_fused(ws, max_steps);
        int notconv = 0;
        *max_steps = 0;
        std::vector<Win<T>> act = ws;
        // restart cycles (max_restarts > 0): every window starts together, so the cycles of all
        // active windows begin at the same block: c0 (current cycle), c0p (previous cycle)
        const int rlen = o->max_restarts > 0 ? o->restart_len : 0;
        int c0 = 0, c0p = 0;
        for (int step = 1; step <= kmax && !act.empty(); ++step) {
            const int na = (int)act.size();
            // ---- part A: operator applications, projections, projected solve
            Stage sa(c, 0);
            std::vector<const T*> xin;
            std::vector<T*> yout, ylo, yav, yatv, yavl, yatvl;
            std::vector<const float*> xlo;
            std::vector<VarSai> vcs;
            std::vector<const double*> ubv;
            const int yc = L.ycols;   // 3 (FP64) or 5 (FP32 data: A V and A^T V carry low parts)
            // TN1 over X = V_{1:step+1} (the working block W sits in slot step) and
            // Y = [A V_i, A^T V_i, (low parts), W]; Y is split into launches of <= 48 columns
            std::vector<std::vector<TsTask<T>>> tn1;
            std::vector<int> wl(na);
            for (int a = 0; a < na; ++a) {
                const Win<T>& W = act[a];
                T* Vi = slot(W, step - 1);
                T* Wn = slot(W, step);
                for (int cc = 0; cc < W.b; ++cc) {
                    xin.push_back(Vi + (int64_t)cc * n);
                    yout.push_back(Wn + (int64_t)cc * n);
                    ylo.push_back(W.Wlo ? reinterpret_cast<T*>(W.Wlo) + (int64_t)cc * n : nullptr);
                    yav.push_back(W.S + (int64_t)cc * n);
                    yatv.push_back(W.S + (int64_t)(W.b + cc) * n);
                    yavl.push_back(W.S + (int64_t)(2 * W.b + cc) * n);
                    yatvl.push_back(W.S + (int64_t)(3 * W.b + cc) * n);
                    xlo.push_back(step == 1 && W.V1lo ? W.V1lo + (int64_t)cc * n : nullptr);
                    vcs.push_back(W.vs);
                    ubv.push_back(W.ubar64);
                }
                const int ldo = (step + 1) * W.b;
                const int qs = (yc - 1) * W.b;   // columns of S
                int sl = 0;
                for (int c0 = 0; c0 < qs + W.b; ++sl) {
                    TsTask<T> t;
                    memset(&t, 0, sizeof(t));
                    t.X = W.V;
                    t.ldx = n;
                    t.p = ldo;
                    t.out = D(W.w) + L.off_out1 + (int64_t)c0 * ldo;
                    if (c0 < qs) {
                        const int q = std::min(48, qs - c0);
                        t.Y = W.S + (int64_t)c0 * n; t.ldy = n; t.q = q; t.q1 = q;
                        // the working block joins the last S slice when it fits
                        if (c0 + q == qs && q + W.b <= 48) { t.Y2 = Wn; t.ldy2 = n; t.q = q + W.b; }
                        c0 += t.q;
                    } else {
                        t.Y = Wn; t.ldy = n; t.q = W.b; t.q1 = W.b;
                        c0 += W.b;
                    }
                    if ((int)tn1.size() <= sl) tn1.emplace_back();
                    tn1[sl].push_back(t);
                }
                wl[a] = W.w;
            }
            const int nv = (int)xin.size();
            const T* const* d_xin = sa.put(xin.data(), nv);
            T* const* d_yout = sa.put(yout.data(), nv);
            T* const* d_ylo = std::is_same<T, float>::value ? sa.put(ylo.data(), nv) : nullptr;
            T* const* d_yav = sa.put(yav.data(), nv);
            T* const* d_yatv = sa.put(yatv.data(), nv);
            T* const* d_yavl = std::is_same<T, float>::value ? sa.put(yavl.data(), nv) : nullptr;
            T* const* d_yatvl = std::is_same<T, float>::value ? sa.put(yatvl.data(), nv) : nullptr;
            // at step 1 the Galerkin block V_1^T A V_1 uses the unrounded start block on one
            // side: the FP32 rounding error d of V_1 would otherwise add d^T A d ~ |d|^2 ||A||
            // to it, a spurious damping of the dominant component
            const float* const* d_xlo = (std::is_same<T, float>::value && step == 1) ? sa.put(xlo.data(), nv) : nullptr;
            std::vector<const TsTask<T>*> d_tn1(tn1.size());
            std::vector<int> tn1_pq(tn1.size(), 0), tn1_q(tn1.size(), 0);
            for (size_t sl = 0; sl < tn1.size(); ++sl) {
                for (auto& t : tn1[sl]) {
                    tn1_pq[sl] = std::max(tn1_pq[sl], t.p * t.q);
                    tn1_q[sl] = std::max(tn1_q[sl], t.q);
                }
                d_tn1[sl] = sa.put(tn1[sl].data(), tn1[sl].size());
            }
            const int* d_wl = sa.put(wl.data(), na);
            const VarSai* d_vcs = var ? sa.put(vcs.data(), nv) : nullptr;
            const double* const* d_ubv = jac ? sa.put(ubv.data(), nv) : nullptr;
            sa.flush();
            const double w = sizeof(T);
            const double wout = std::is_same<T, float>::value ? 8.0 : w;   // hi + lo for FP32 data
            if (o->krylov == PEXP_KRYLOV_SAI) {
                timed(c, PEXP_KC_SAI, (double)nv * n * (w + wout), [&] {
                    if (var) launch_vsai_solve<T>(n, d_vcs, d_xin, nullptr, d_yout, d_ylo, nv, sai_scr, st);
                    else launch_sai_solve<T>(od, sai, d_xin, d_yout, d_ylo, nv, sai_scr, st);
                }, nullptr, false, 2.0 * nv * n * w);
                c->launches += 2;   // the solve is three kernels; check_launch below counts one
            } else {
                launch_stencil_ptrs<T>(od, d_xin, d_yout, nv, 0, st);
                for (const auto& W : act)
                    if (W.Wlo) cudaMemsetAsync(W.Wlo, 0, sizeof(float) * (size_t)n * W.b, st);
            }
            check_launch(c);
            timed(c, PEXP_KC_STENCIL, 2.0 * nv * n * (w + wout), [&] {
                if constexpr (std::is_same<T, float>::value) {
                    launch_stencil_df(od, reinterpret_cast<const float* const*>(d_xin), d_xlo,
                                      reinterpret_cast<float* const*>(d_yav), reinterpret_cast<float* const*>(d_yavl), nv, 0, st);
                    check_launch(c);
                    launch_stencil_df(od, reinterpret_cast<const float* const*>(d_xin), d_xlo,
                                      reinterpret_cast<float* const*>(d_yatv), reinterpret_cast<float* const*>(d_yatvl), nv, 1, st);
                    check_launch(c);
                } else {
                    launch_stencil_ptrs<T>(od, d_xin, d_yav, nv, 0, st);
                    check_launch(c);
                    launch_stencil_ptrs<T>(od, d_xin, d_yatv, nv, 1, st);
                    check_launch(c);
                }
                if (jac) {
                    // (A + J_j) V_i and (A + J_j)^T V_i: the Jacobian of each window added in FP64
                    const float* const* xl32 = std::is_same<T, float>::value ? d_xlo : nullptr;
                    launch_jac_add<T>(n, od.x.periodic, inv2dx, d_ubv, d_xin, xl32, d_yav,
                                      std::is_same<T, float>::value ? d_yavl : nullptr, nv, 0, st);
                    check_launch(c);
                    launch_jac_add<T>(n, od.x.periodic, inv2dx, d_ubv, d_xin, xl32, d_yatv,
                                      std::is_same<T, float>::value ? d_yatvl : nullptr, nv, 1, st);
                    check_launch(c);
                }
            }, nullptr, false, 4.0 * nv * n * w);
            for (size_t sl = 0; sl < tn1.size(); ++sl) {
                double by = 0;
                for (auto& t : tn1[sl]) by += (double)n * (t.p + t.q) * w;
                timed(c, PEXP_KC_PROJ, by, [&] {
                    launch_ts_tn<T>(d_tn1[sl], (int)tn1[sl].size(), tn1_pq[sl], tn1_q[sl], n, partial, st,
                                    std::is_same<T, float>::value ? 1 : 0);
                    check_launch(c);
                });
            }
            timed(c, PEXP_KC_SMALL, 0.0, [&] {
                launch_project(L, wd, wi, d_wl, na, step, h, o->tol, scale_ref, st, Parts{nullptr, 0, 0}, 0.0, 0.0, 0, 0,
                               0.0, c0, c0p);
            });
            check_launch(c);
            // ---- convergence flags
            d2h(c, wi_host.data(), wi, sizeof(int) * wi_host.size());
            std::vector<Win<T>> next;
            for (auto& W : act) {
                const int* I = &wi_host[(size_t)W.w * L.istride];
                *max_steps = std::max(*max_steps, I[WI_STEPS]);
                if (!I[WI_CONV]) next.push_back(W);
            }
            if (step == kmax) {
                notconv += (int)next.size();
                break;
            }
            act.swap(next);
            if (act.empty()) break;
            // ---- part B: Gram-Schmidt (two passes) and Cholesky QR (two passes)
            const int nb = (int)act.size();
            Stage sb(c, 1);
            std::vector<TsTask<T>> nn1(nb), tn2(nb), nn2(nb), tn3(nb), nn3(nb);
            std::vector<int> wl2(nb);
            int mpq1 = 0, mpq2 = 0, mq2 = 0, mpq3 = 0, mq3 = 0;
            // the block made at this step starts the next restart cycle
            const bool restart = rlen > 0 && step - c0 == rlen;
            for (int a = 0; a < nb; ++a) {
                const Win<T>& W = act[a];
                T* Wn = slot(W, step);
                // Gram-Schmidt against the blocks of the current cycle, columns [k0, k0 + p)
                const int b = W.b, k0 = c0 * W.b, p = (step - c0) * b, ldo = (step + 1) * b;
                TsTask<T> t;
                memset(&t, 0, sizeof(t));
                // W -= V_{cycle} h1, h1 = out1[k0:k0+p, 2b:3b]
                t.X = W.V + (int64_t)k0 * n; t.ldx = n; t.p = p; t.q = b;
                t.Z = Wn; t.ldz = n;
                t.Tm = D(W.w) + L.off_out1 + (int64_t)2 * b * ldo + k0; t.ldt = ldo;
                t.alpha = -1.0; t.beta = 1.0;
                nn1[a] = t;
                mpq1 = std::max(mpq1, p * b);
                // h2 = V^T W
                memset(&t, 0, sizeof(t));
                t.X = W.V + (int64_t)k0 * n; t.ldx = n; t.p = p;
                t.Y = Wn; t.ldy = n; t.q = b; t.q1 = b;
                t.out = D(W.w) + L.off_h2;
                tn2[a] = t;
                mpq2 = std::max(mpq2, p * b);
                mq2 = std::max(mq2, b);
                // W -= V h2
                t = nn1[a];
                t.Tm = D(W.w) + L.off_h2; t.ldt = p;
                nn2[a] = t;
                // Gram of W
                memset(&t, 0, sizeof(t));
                t.X = Wn; t.ldx = n; t.p = b;
                t.Y = Wn; t.ldy = n; t.q = b; t.q1 = b;
                t.out = D(W.w) + L.off_gw;
                tn3[a] = t;
                mpq3 = std::max(mpq3, b * b);
                mq3 = std::max(mq3, b);
                // W <- W T (in place)
                memset(&t, 0, sizeof(t));
                t.X = Wn; t.ldx = n; t.p = b; t.q = b;
                t.Z = Wn; t.ldz = n;
                t.Tm = D(W.w) + L.off_T; t.ldt = b;
                t.alpha = 1.0; t.beta = 0.0;
                nn3[a] = t;
                wl2[a] = W.w;
            }
            const TsTask<T>* d_tn2 = sb.put(tn2.data(), nb);
            const TsTask<T>* d_tn3 = sb.put(tn3.data(), nb);
            const int* d_wl2 = sb.put(wl2.data(), nb);
            if constexpr (std::is_same<T, float>::value) {
                // FP32 data: the working block stays a double-float pair (slot = hi, Wlo = lo)
                // through both Gram-Schmidt updates and both Cholesky scalings; the
                // final scaling rounds the orthonormal block to FP32 in place.
                std::vector<DfTask> d1(nb), d2(nb), d3(nb), d4(nb);
                for (int a = 0; a < nb; ++a) {
                    const Win<T>& W = act[a];
                    float* Wn = slot(W, step);
                    const int b = W.b, k0 = c0 * W.b, p = (step - c0) * b, ldo = (step + 1) * b;
                    DfTask t;
                    memset(&t, 0, sizeof(t));
                    t.Xh = W.V + (int64_t)k0 * n; t.ldx = n; t.Zh = Wn; t.Zl = W.Wlo; t.ldz = n;
                    t.Tm = D(W.w) + L.off_out1 + (int64_t)(L.ycols - 1) * b * ldo + k0; t.ldt = ldo;
                    t.p = p; t.q = b; t.alpha = -1.0; t.accumulate = 1;
                    d1[a] = t;
                    t.Tm = D(W.w) + L.off_h2; t.ldt = p;
                    d2[a] = t;
                    memset(&t, 0, sizeof(t));
                    t.Xh = Wn; t.Xl = W.Wlo; t.ldx = n; t.Zh = Wn; t.Zl = W.Wlo; t.ldz = n;
                    t.Tm = D(W.w) + L.off_T; t.ldt = b; t.p = b; t.q = b; t.alpha = 1.0; t.accumulate = 0;
                    d3[a] = t;
                    // a block that starts a shift-and-invert restart cycle keeps its low part
                    // for the residual direction formed from it below
                    if (!(restart && o->krylov == PEXP_KRYLOV_SAI)) t.Zl = nullptr;
                    d4[a] = t;
                }
                const DfTask* dd1 = sb.put(d1.data(), nb);
                const DfTask* dd2 = sb.put(d2.data(), nb);
                const DfTask* dd3 = sb.put(d3.data(), nb);
                const DfTask* dd4 = sb.put(d4.data(), nb);
                sb.flush();
                double pb = 0, bb = 0;   // sum of p*b and of b over the active windows
                for (auto& W : act) { pb += (double)(step - c0) * W.b; bb += W.b; }
                const double nn = (double)n;
                // pass 1, Cholesky QR of the result, then the second pass on the normalised block
                // (as the fused kernels do): second-pass coefficients taken from the block before
                // normalisation carry its conditioning into the basis's orthogonality
                timed(c, PEXP_KC_UPDATE, nn * (pb * 4 + bb * 16), [&] { launch_ts_nn_df(dd1, nb, mpq1, n, st, mq3); }, nullptr, false, nn * (pb * 4 + bb * 8)); check_launch(c);
                timed(c, PEXP_KC_PROJ, nn * bb * 4, [&] { launch_ts_tn<T>(d_tn3, nb, mpq3, mq3, n, partial, st, 1); }); check_launch(c);
                timed(c, PEXP_KC_SMALL, 0.0, [&] { launch_block_orth(L, wd, wi, d_wl2, nb, 1, step, defl, st); }); check_launch(c);
                timed(c, PEXP_KC_UPDATE, nn * bb * 16, [&] { launch_ts_nn_df(dd3, nb, mpq3, n, st, mq3); }, nullptr, false, nn * bb * 8); check_launch(c);
                timed(c, PEXP_KC_PROJ, nn * (pb + bb) * 4, [&] { launch_ts_tn<T>(d_tn2, nb, mpq2, mq2, n, partial, st, PEXP_TN_EXACT_FP32); }); check_launch(c);
                timed(c, PEXP_KC_UPDATE, nn * (pb * 4 + bb * 16), [&] { launch_ts_nn_df(dd2, nb, mpq1, n, st, mq3); }, nullptr, false, nn * (pb * 4 + bb * 8)); check_launch(c);
                timed(c, PEXP_KC_PROJ, nn * bb * 4, [&] { launch_ts_tn<T>(d_tn3, nb, mpq3, mq3, n, partial, st, 1); }); check_launch(c);
                timed(c, PEXP_KC_SMALL, 0.0, [&] { launch_block_orth(L, wd, wi, d_wl2, nb, 2, step, defl, st); }); check_launch(c);
                timed(c, PEXP_KC_UPDATE, nn * bb * 12, [&] { launch_ts_nn_df(dd4, nb, mpq3, n, st, mq3); }, nullptr, false, nn * bb * 8); check_launch(c);
            } else {
                const TsTask<T>* d_nn1 = sb.put(nn1.data(), nb);
                const TsTask<T>* d_nn2 = sb.put(nn2.data(), nb);
                const TsTask<T>* d_nn3 = sb.put(nn3.data(), nb);
                sb.flush();
                double pb = 0, bb = 0;
                for (auto& W : act) { pb += (double)(step - c0) * W.b; bb += W.b; }
                const double nn = (double)n * 8.0;
                timed(c, PEXP_KC_UPDATE, nn * (pb + 2 * bb), [&] { launch_ts_nn<T>(d_nn1, nb, mpq1, n, st); }); check_launch(c);
                timed(c, PEXP_KC_PROJ, nn * (pb + bb), [&] { launch_ts_tn<T>(d_tn2, nb, mpq2, mq2, n, partial, st, 0); }); check_launch(c);
                timed(c, PEXP_KC_UPDATE, nn * (pb + 2 * bb), [&] { launch_ts_nn<T>(d_nn2, nb, mpq1, n, st); }); check_launch(c);
                timed(c, PEXP_KC_PROJ, nn * bb, [&] { launch_ts_tn<T>(d_tn3, nb, mpq3, mq3, n, partial, st, 0); }); check_launch(c);
                timed(c, PEXP_KC_SMALL, 0.0, [&] { launch_block_orth(L, wd, wi, d_wl2, nb, 1, step, defl, st); }); check_launch(c);
                timed(c, PEXP_KC_UPDATE, nn * 2 * bb, [&] { launch_ts_nn<T>(d_nn3, nb, mpq3, n, st); }); check_launch(c);
                timed(c, PEXP_KC_PROJ, nn * bb, [&] { launch_ts_tn<T>(d_tn3, nb, mpq3, mq3, n, partial, st, 0); }); check_launch(c);
                timed(c, PEXP_KC_SMALL, 0.0, [&] { launch_block_orth(L, wd, wi, d_wl2, nb, 2, step, defl, st); }); check_launch(c);
                timed(c, PEXP_KC_UPDATE, nn * 2 * bb, [&] { launch_ts_nn<T>(d_nn3, nb, mpq3, n, st); }); check_launch(c);
            }
            if (restart) {
                if (o->krylov == PEXP_KRYLOV_SAI) restart_block(act, step, c0);
                for (auto& W : act) ++restarts[W.w];
                c0p = c0;
                c0 = step;
            }
        }
        return notconv;
    }

    // First block of a restart cycle in the shift-and-invert space.  After `step` blocks of the
    // cycle that starts at block c0, the Galerkin solution V_c y_c(t) leaves the residual
    // (I - V_c V_c^T) A V_c y_c(t), of rank b: with M = (I - gamma A)^{-1}, the cycle's Arnoldi
    // relation M V_c = V_c Ht + V' h E^T (V' the block just made in slot `step`) gives
    //     (I - V_c V_c^T) A V_c = q h E^T Ht^{-1} / gamma,   q = V' - gamma (I - V_c V_c^T) A V'.
    // The next cycle's space starts from q, orthonormalised (two Cholesky QRs) into the slot.
    // FP32 data: V' is the double-float block (slot, Wlo), so that gamma A V' carries no
    // amplified rounding of a stored vector.  (In the polynomial space the range is V' itself.)
    void restart_block(const std::vector<Win<T>>& act, int step, int c0) {
        const int nb = (int)act.size();
        const double gamma = o->sai_gamma * o->T / (double)o->P;
        int bmax = 0;
        for (auto& W : act) bmax = std::max(bmax, W.b);
        std::vector<double> mg((size_t)bmax * bmax, 0.0);   // -gamma I
        for (int i = 0; i < bmax; ++i) mg[(size_t)i * bmax + i] = -gamma;
        Stage sr(c, 1);
        const double* d_mg = sr.put(mg.data(), mg.size());
        std::vector<const T*> xin;
        std::vector<const float*> xlo;
        std::vector<T*> yav, yavl;
        std::vector<TsTask<T>> th(nb), tq(nb), tg(nb), ts(nb);
        std::vector<DfTask> da(nb), dh(nb), dl(nb), d3(nb), d4(nb);
        std::vector<int> wl(nb);
        int mpq = 0;
        for (int a = 0; a < nb; ++a) {
            const Win<T>& W = act[a];
            T* Wn = slot(W, step);
            const int b = W.b, k0 = c0 * b, p = (step - c0) * b;
            for (int cc = 0; cc < b; ++cc) {
                xin.push_back(Wn + (int64_t)cc * n);
                xlo.push_back(W.Wlo ? W.Wlo + (int64_t)cc * n : nullptr);
                yav.push_back(W.S + (int64_t)cc * n);
                yavl.push_back(W.S + (int64_t)(2 * b + cc) * n);
            }
            TsTask<T> t;
            // h = V_c^T (A V') (FP32 data: the high and the low part of A V' side by side)
            memset(&t, 0, sizeof(t));
            t.X = W.V + (int64_t)k0 * n; t.ldx = n; t.p = p;
            t.Y = W.S; t.ldy = n; t.q1 = b; t.q = b;
            if (W.Wlo) { t.Y2 = W.S + (int64_t)2 * b * n; t.ldy2 = n; t.q = 2 * b; }
            t.out = D(W.w) + L.off_h2;
            th[a] = t;
            mpq = std::max(mpq, p * t.q);
            // FP64: q = V' - gamma A V' + gamma V_c h
            memset(&t, 0, sizeof(t));
            t.X = W.S; t.ldx = n; t.p = b; t.q = b; t.Z = Wn; t.ldz = n; t.Tm = d_mg; t.ldt = bmax;
            t.alpha = 1.0; t.beta = 1.0;
            tq[a] = t;
            memset(&t, 0, sizeof(t));
            t.X = W.V + (int64_t)k0 * n; t.ldx = n; t.p = p; t.q = b; t.Z = Wn; t.ldz = n;
            t.Tm = D(W.w) + L.off_h2; t.ldt = p; t.alpha = gamma; t.beta = 1.0;
            tg[a] = t;
            // Gram of the block and its scaling (Cholesky QR)
            memset(&t, 0, sizeof(t));
            t.X = Wn; t.ldx = n; t.p = b; t.Y = Wn; t.ldy = n; t.q = b; t.q1 = b; t.out = D(W.w) + L.off_gw;
            ts[a] = t;
            if constexpr (std::is_same<T, float>::value) {
                DfTask d;
                memset(&d, 0, sizeof(d));
                d.Xh = W.S; d.Xl = W.S + (int64_t)2 * b * n; d.ldx = n; d.Zh = Wn; d.Zl = W.Wlo; d.ldz = n;
                d.Tm = d_mg; d.ldt = bmax; d.p = b; d.q = b; d.alpha = 1.0; d.accumulate = 1;
                da[a] = d;
                memset(&d, 0, sizeof(d));
                d.Xh = W.V + (int64_t)k0 * n; d.ldx = n; d.Zh = Wn; d.Zl = W.Wlo; d.ldz = n;
                d.Tm = D(W.w) + L.off_h2; d.ldt = p; d.p = p; d.q = b; d.alpha = gamma; d.accumulate = 1;
                dh[a] = d;
                d.Tm = D(W.w) + L.off_h2 + (int64_t)p * b;   // the low part's products
                dl[a] = d;
                memset(&d, 0, sizeof(d));
                d.Xh = Wn; d.Xl = W.Wlo; d.ldx = n; d.Zh = Wn; d.Zl = W.Wlo; d.ldz = n;
                d.Tm = D(W.w) + L.off_T; d.ldt = b; d.p = b; d.q = b; d.alpha = 1.0; d.accumulate = 0;
                d3[a] = d;
                d.Zl = nullptr;
                d4[a] = d;
            }
            wl[a] = W.w;
        }
        const int nv = (int)xin.size();
        const T* const* d_xin = sr.put(xin.data(), nv);
        T* const* d_yav = sr.put(yav.data(), nv);
        const float* const* d_xlo = std::is_same<T, float>::value ? sr.put(xlo.data(), nv) : nullptr;
        T* const* d_yavl = std::is_same<T, float>::value ? sr.put(yavl.data(), nv) : nullptr;
        const TsTask<T>* d_th = sr.put(th.data(), nb);
        const TsTask<T>* d_tq = sr.put(tq.data(), nb);
        const TsTask<T>* d_tg = sr.put(tg.data(), nb);
        const TsTask<T>* d_ts = sr.put(ts.data(), nb);
        const DfTask* d_da = std::is_same<T, float>::value ? sr.put(da.data(), nb) : nullptr;
        const DfTask* d_dh = std::is_same<T, float>::value ? sr.put(dh.data(), nb) : nullptr;
        const DfTask* d_dl = std::is_same<T, float>::value ? sr.put(dl.data(), nb) : nullptr;
        const DfTask* d_d3 = std::is_same<T, float>::value ? sr.put(d3.data(), nb) : nullptr;
        const DfTask* d_d4 = std::is_same<T, float>::value ? sr.put(d4.data(), nb) : nullptr;
        const int* d_wl = sr.put(wl.data(), nb);
        sr.flush();
        int bm = 0;
        for (auto& W : act) bm = std::max(bm, W.b);
        // A V' (FP32 data: of the double-float pair, as a double-float pair)
        if constexpr (std::is_same<T, float>::value) {
            launch_stencil_df(od, reinterpret_cast<const float* const*>(d_xin), d_xlo,
                              reinterpret_cast<float* const*>(d_yav), reinterpret_cast<float* const*>(d_yavl), nv, 0, st);
        } else {
            launch_stencil_ptrs<T>(od, d_xin, d_yav, nv, 0, st);
        }
        check_launch(c);
        launch_ts_tn<T>(d_th, nb, mpq, std::is_same<T, float>::value ? 2 * bm : bm, n, partial, st,
                        std::is_same<T, float>::value ? 1 : 0);
        check_launch(c);
        if constexpr (std::is_same<T, float>::value) {
            launch_ts_nn_df(d_da, nb, bm * bm, n, st, bm); check_launch(c);
            launch_ts_nn_df(d_dh, nb, mpq, n, st, bm); check_launch(c);
            launch_ts_nn_df(d_dl, nb, mpq, n, st, bm); check_launch(c);
        } else {
            launch_ts_nn<T>(d_tq, nb, bm * bm, n, st); check_launch(c);
            launch_ts_nn<T>(d_tg, nb, mpq, n, st); check_launch(c);
        }
        // two Cholesky QRs of q (deflation relative to this step's pre-Gram-Schmidt norms)
        for (int pass = 1; pass <= 2; ++pass) {
            launch_ts_tn<T>(d_ts, nb, bm * bm, bm, n, partial, st, std::is_same<T, float>::value ? 1 : 0);
            check_launch(c);
            launch_block_orth(L, wd, wi, d_wl, nb, pass, step, defl, st);
            check_launch(c);
            if constexpr (std::is_same<T, float>::value) {
                launch_ts_nn_df(pass == 1 ? d_d3 : d_d4, nb, bm * bm, n, st, bm);
            } else {
                // W <- W T in place, as the final scaling of a step
                std::vector<TsTask<T>> sc(nb);
                for (int a = 0; a < nb; ++a) {
                    TsTask<T> t;
                    memset(&t, 0, sizeof(t));
                    T* Wn = slot(act[a], step);
                    t.X = Wn; t.ldx = n; t.p = act[a].b; t.q = act[a].b; t.Z = Wn; t.ldz = n;
                    t.Tm = D(act[a].w) + L.off_T; t.ldt = act[a].b; t.alpha = 1.0; t.beta = 0.0;
                    sc[a] = t;
                }
                Stage sq(c, 0);
                const TsTask<T>* d_sc = sq.put(sc.data(), nb);
                sq.flush();
                launch_ts_nn<T>(d_sc, nb, bm * bm, n, st);
            }
            check_launch(c);
        }
    }
};

template <typename T>
T* as(void* p) { return reinterpret_cast<T*>(p); }

struct Partition {
    std::vector<int> idx;   // P+1 boundaries
    int smax = 0;
};
Partition make_partition(int n_out, int P) {
    Partition r;
    r.idx.resize(P + 1);
    for (int j = 0; j <= P; ++j) r.idx[j] = (int)(((int64_t)j * (n_out - 1)) / P);
    for (int j = 1; j <= P; ++j) r.smax = std::max(r.smax, r.idx[j] - r.idx[j - 1] + 1);
    return r;
}

// Source samples of the subintervals: the output times (nodes = PEXP_NODES_UNIFORM), or n_samp
// Chebyshev points per subinterval sharing the ends (Sec. 3), rows j (n_samp - 1) .. of G.
struct SrcPartition {
    bool cheb = false;
    std::vector<int> idx;   // P+1 first rows: subinterval j's samples are rows idx[j] .. idx[j+1]
    int smax = 0;           // largest sample count of a subinterval
    int rows = 0;           // rows of G
};
SrcPartition make_src_partition(const pexp_options* o, const Partition& pt) {
    SrcPartition r;
    r.cheb = o->nodes == PEXP_NODES_CHEBYSHEV;
    if (!r.cheb) {
        r.idx = pt.idx;
        r.smax = pt.smax;
        r.rows = o->n_out;
        return r;
    }
    r.idx.resize(o->P + 1);
    for (int j = 0; j <= o->P; ++j) r.idx[j] = j * (o->n_samp - 1);
    r.smax = o->n_samp;
    r.rows = o->P * (o->n_samp - 1) + 1;
    return r;
}
int src_rows_of(const pexp_options* o) {
    return o->nodes == PEXP_NODES_CHEBYSHEV ? o->P * (o->n_samp - 1) + 1 : o->n_out;
}

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Upper bound of the workspace a linear solve needs (bytes).
template <typename T>
size_t linear_workspace_bytes(int64_t n, const pexp_options* o, int g_conv, int b_cap) {
    const int P = o->P;
    Partition pt = make_partition(o->n_out, P);
    const SrcPartition sp = make_src_partition(o, pt);
    const int smax = std::max(pt.smax, sp.smax);
    const int kmax = o->restart_len * (o->max_restarts + 1);
    WinLayout L = make_layout(smax, b_cap, kmax, sizeof(T) == 8 ? 3 : 5);
    size_t s = 0;
    s += align_up(sizeof(double) * n * 2);                                  // u0, A u0
    if (g_conv) s += align_up(sizeof(T) * (size_t)n * sp.rows);            // converted G
    s += align_up(sizeof(double) * L.stride * 2 * P);                       // window state
    s += align_up(sizeof(int) * L.istride * 2 * P);
    s += align_up(sizeof(double) * (ts_tn_partial_doubles(P, std::max(std::max(smax * smax, 48 * (L.K_max + b_cap)), 48 * L.K_max), n) + 512));
    s += align_up(sizeof(double) * (size_t)L.K_max * 48);                   // orthogonality diagnostic
    s += 2 * align_up(sizeof(double) * kpart_doubles(P, n, kmax, b_cap, smax));
    s += align_up(sizeof(double) * sai_scratch_doubles(n, P * b_cap) + 64);
    s += align_up(sizeof(double) * (sp.rows + P));                          // (A u0) . g(t_i)
    s += align_up(sizeof(double) * 3 * (size_t)n) + kAlign;                 // bounded-mesh SAI factors
    if (sizeof(T) == 4) s += align_up(sizeof(float) * n * 2);               // A u0 as a double-float pair
    s += (size_t)(4 * P + 32) * kAlign;   // alignment of the per-window allocations
    return s;
}

template <typename T, typename TO>
int solve_linear_typed(pexp_ctx* c, const pexp_operator* op, const pexp_options* o, const double* u0d,
                       const void* G_dev, int g_dtype, TO* Y, pexp_report* rep, const WinOps<T>* wo, TO* Y_host) {
    cudaStream_t st = c->stream;
    Solver<T> S;
    S.c = c;
    S.st = st;
    S.o = o;
    S.od = make_opdesc(*op);
    const int64_t n = S.od.n;
    S.n = n;
    const int P = o->P, n_out = o->n_out;
    Partition pt = make_partition(n_out, P);
    // source samples: the output times, or each subinterval's Chebyshev points
    const SrcPartition sp = make_src_partition(o, pt);
    const int smax = std::max(pt.smax, sp.smax);
    S.kmax = o->restart_len * (o->max_restarts + 1);
    S.h = o->T / (double)(n_out - 1);
    const bool fp64 = sizeof(T) == 8;
    S.defl = fp64 ? PEXP_DEFL_FP64 : PEXP_DEFL_FP32;
    const double svd_floor = fp64 ? 1e-7 : 1e-5;
    const int b_cap = std::min(std::min(o->max_rank, PEXP_MAX_RANK), sp.smax);
    S.L = make_layout(smax, b_cap, S.kmax, fp64 ? 3 : 5);
    const WinLayout& L = S.L;
    // the subproblems solved: j in [ja, jb) (all by default); their solutions are zero before T_ja
    const bool ranged = !(o->sub_first == 0 && o->sub_last == 0);
    const int ja = ranged ? o->sub_first : 0, jb = ranged ? o->sub_last : P;

    // ---- buffers
    double* Au0 = as<double>(ws_alloc(c, sizeof(double) * n));
    const T* G = nullptr;
    if (G_dev) {
        const bool same = (g_dtype == PEXP_F64) == fp64;
        if (same) {
            G = reinterpret_cast<const T*>(G_dev);
        } else {
            T* Gc = as<T>(ws_alloc(c, sizeof(T) * (size_t)n * sp.rows));
            if (g_dtype == PEXP_F64) launch_convert<double, T>(reinterpret_cast<const double*>(G_dev), Gc, n * sp.rows, st);
            else launch_convert<float, T>(reinterpret_cast<const float*>(G_dev), Gc, n * sp.rows, st);
            check_launch(c);
            G = Gc;
        }
    }
    // window-major pre-shifted source (averaged-Jacobian WR): window j's s_j samples start at
    // row idx_j + j, and the shift by A u0 is already in them
    const T* Gw = wo ? wo->Gwin : nullptr;
    const bool have_src = G || Gw;
    const int src_rows = Gw ? n_out + P - 1 : sp.rows;
    auto src_first = [&](int j) -> const T* {
        if (Gw) return Gw + (int64_t)(pt.idx[j] + j) * n;
        return G ? G + (int64_t)sp.idx[j] * n : nullptr;
    };
    auto src_count = [&](int j) { return sp.idx[j + 1] - sp.idx[j] + 1; };
    // a bounded mesh with the shift-and-invert space: one factored operator for all windows
    WinOps<T> wo_bounded;
    if (!wo && o->krylov == PEXP_KRYLOV_SAI && !S.od.x.periodic) {
        const double gamma = o->sai_gamma * o->T / (double)P;
        double* fac = as<double>(ws_alloc(c, sizeof(double) * 3 * (size_t)n));
        int* flag = as<int>(ws_alloc(c, sizeof(int) * 4));
        cudaMemsetAsync(flag, 0, sizeof(int), st);
        Stage sf(c, 0);
        VarOpTask vt{nullptr, fac, fac + n, fac + 2 * n, flag};
        const VarOpTask* dvt = sf.put(&vt, 1);
        sf.flush();
        launch_vsai_factor(S.od.x, gamma, 0.0, dvt, 1, vsai_warmup(S.od.x, gamma, 0.0, 0.0), st);
        check_launch(c);
        int fl = 0;
        d2h(c, &fl, flag, sizeof(int));
        if (fl) throw StatusError{PEXP_ERR_UNSUPPORTED};
        wo_bounded.var = true;
        wo_bounded.vs.assign(P, VarSai{fac, fac + n, fac + 2 * n});
        wo = &wo_bounded;
    }
    S.var = wo && wo->var;
    S.jac = wo && wo->jac;
    S.inv2dx = wo ? wo->inv2dx : 0.0;
    auto win_ops = [&](Win<T>& W, int j) {
        if (!wo) return;
        if (wo->var) W.vs = wo->vs[j];
        if (wo->jac) {
            W.ubar = wo->ubar[j];
            W.ubar64 = wo->ubar64[j];
        }
    };
    const int nwin = 2 * P;   // [0, P): source windows j=1..P; [P, 2P): homogeneous windows m=1..P
    S.wd = as<double>(ws_alloc(c, sizeof(double) * L.stride * nwin));
    S.wi = as<int>(ws_alloc(c, sizeof(int) * L.istride * nwin));
    const size_t part_n = ts_tn_partial_doubles(P, std::max(std::max(smax * smax, 48 * (L.K_max + b_cap)), 48 * L.K_max), n) + 512;
    S.partial = as<double>(ws_alloc(c, sizeof(double) * part_n));
    S.diag = as<double>(ws_alloc(c, sizeof(double) * (size_t)L.K_max * 48));
    const size_t kpart_n = kpart_doubles(P, n, S.kmax, b_cap, smax);
    for (int k = 0; k < 2; ++k) S.kpart[k] = as<double>(ws_alloc(c, sizeof(double) * kpart_n));
    S.sai_scr = as<double>(ws_alloc(c, sizeof(double) * (sai_scratch_doubles(n, P * b_cap) + 64)));
    // one pole for every window: gamma = sai_gamma * T / P (the nominal subinterval length)
    if (o->krylov == PEXP_KRYLOV_SAI && !S.var) S.sai = sai_coefficients(S.od, o->sai_gamma * o->T / (double)P);
    S.wi_host.assign((size_t)L.istride * nwin, 0);
    S.restarts.assign(nwin, 0);

    // ---- initial window state
    {
        std::vector<int> wih((size_t)L.istride * nwin, 0);
        for (int j = 0; j < P; ++j) {
            wih[(size_t)j * L.istride + WI_S] = src_count(j);
            wih[(size_t)j * L.istride + WI_KIND] = KIND_SOURCE;
            wih[(size_t)j * L.istride + WI_I0] = Gw ? pt.idx[j] + j : sp.idx[j];
            if (sp.cheb) {
                wih[(size_t)j * L.istride + WI_SOUT] = pt.idx[j + 1] - pt.idx[j] + 1;
                wih[(size_t)j * L.istride + WI_CHEB] = 1;
            }
            wih[(size_t)(P + j) * L.istride + WI_S] = pt.idx[j + 1] - pt.idx[j] + 1;
            wih[(size_t)(P + j) * L.istride + WI_KIND] = KIND_HOM;
            wih[(size_t)(P + j) * L.istride + WI_B] = 1;
        }
        cudaMemcpyAsync(S.wi, wih.data(), sizeof(int) * wih.size(), cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(S.wd, 0, sizeof(double) * L.stride * nwin, st);
        sync(c);   // wih goes out of scope
    }

    NvtxPhases nvtx;
    nvtx.next("pexp: shift and source compression");
    cudaEventRecord(c->evp[0], st);
    // ---- shift: A u0, ||u0||, ||A u0||^2, (A u0) . g(t_i)
    double* nrm = S.partial + part_n - 8;   // [0] = ||u0||^2, [1] = ||A u0||^2
    double* dots = have_src ? as<double>(ws_alloc(c, sizeof(double) * src_rows)) : nullptr;
    float* au0_split = (G && sizeof(T) == 4) ? as<float>(ws_alloc(c, sizeof(float) * n * 2)) : nullptr;
    if (Gw) {
        // the window-major source carries its shift: no A u0 term in the Gram or in U
        cudaMemsetAsync(Au0, 0, sizeof(double) * n, st);
        cudaMemsetAsync(dots, 0, sizeof(double) * src_rows, st);
    } else {
        launch_stencil<double>(S.od, u0d, Au0, 1, 0, st);
        check_launch(c);
    }
    {
        Stage s0(c, 0);
        TsTask<double> t[2];
        memset(t, 0, sizeof(t));
        t[0].X = u0d; t[0].ldx = n; t[0].p = 1; t[0].Y = u0d; t[0].ldy = n; t[0].q = 1; t[0].q1 = 1; t[0].out = nrm;
        t[1].X = Au0; t[1].ldx = n; t[1].p = 1; t[1].Y = Au0; t[1].ldy = n; t[1].q = 1; t[1].q1 = 1; t[1].out = nrm + 1;
        const TsTask<double>* dt = s0.put(t, 2);
        s0.flush();
        launch_ts_tn<double>(dt, 2, 1, 1, n, S.partial, st, 0);
        check_launch(c);
        if (G && !Gw) {
            launch_row_dots<T>(Au0, G, n, sp.rows, dots, au0_split, st);
            check_launch(c);
        }
        double nn = 0;
        d2h(c, &nn, nrm, sizeof(double));
        S.scale_ref = sqrt(nn);
    }

    // ---- source compression, all subintervals: Gram of g_hat = A u0 + g from
    // G^T G (per window), (A u0) . g(t_i) and ||A u0||^2
    std::vector<int> all(P);
    for (int j = 0; j < P; ++j) all[j] = j;
    {
        Stage s1(c, 0);
        std::vector<TsTask<T>> tg(P);
        for (int j = 0; j < P; ++j) {
            TsTask<T> t;
            memset(&t, 0, sizeof(t));
            const int s = src_count(j);
            t.X = src_first(j);
            t.ldx = n; t.p = s;
            t.Y = t.X; t.ldy = n; t.q = s; t.q1 = s;
            t.out = S.D(j) + L.off_gram;
            tg[j] = t;
        }
        std::vector<const T*> gx(P);
        std::vector<int> gs(P);
        for (int j = 0; j < P; ++j) {
            gx[j] = src_first(j);
            gs[j] = src_count(j);
        }
        const T* const* dgx = s1.put(gx.data(), P);
        const int* dgs = s1.put(gs.data(), P);
        const int* dall = s1.put(all.data(), P);
        s1.flush();
        const KGeom gg = krylov_geom(P, n);
        const int psg = sp.smax * sp.smax;
        if (have_src) {
            timed(c, PEXP_KC_SOURCE, (double)n * src_rows * sizeof(T),
                  [&] { launch_source_gram<T>(dgx, dgs, P, sp.smax, n, gg, S.kpart[0], psg, st); });
            check_launch(c);
        }
        launch_source_eig(L, S.wd, S.wi, dall, P, std::max(o->svd_tol, svd_floor), b_cap, dots, nrm + 1, st,
                          Parts{have_src ? S.kpart[0] : nullptr, gg.nchunks, psg});
        check_launch(c);
        d2h(c, S.wi_host.data(), S.wi, sizeof(int) * S.wi_host.size());
    }
    std::vector<int> mj(P);
    int b_max = 0, b_min = 1 << 30;
    for (int j = 0; j < P; ++j) {
        mj[j] = (j >= ja && j < jb) ? S.wi_host[(size_t)j * L.istride + WI_B] : 0;
        if (j < ja || j >= jb) continue;
        b_max = std::max(b_max, mj[j]);
        b_min = std::min(b_min, mj[j]);
    }
    // restart cycles run in the dense-projection driver
    S.fused = (S.od.dim == 1) && (b_max <= kKrylovMaxB) && o->max_restarts == 0;
    // bases laid out with the actual widths, in the basis pool
    {
        size_t need = 0;
        for (int j = 0; j < P; ++j)
            if (mj[j] > 0)
                need += align_up(sizeof(T) * (size_t)n * mj[j] * (S.kmax + 1)) + align_up(sizeof(T) * (size_t)n * (L.ycols - 1) * mj[j]) +
                        (std::is_same<T, float>::value ? 2 * align_up(sizeof(float) * (size_t)n * mj[j]) : 0);
        need += (size_t)P * align_up(sizeof(T) * (size_t)n * (S.kmax + 1));   // homogeneous bases
        need += align_up(sizeof(T) * (size_t)n * (L.ycols - 1)) + 3 * align_up(sizeof(float) * (size_t)n) + (size_t)(6 * P + 8) * kAlign;
        const int r = bs_reserve(c, need);
        if (r) throw StatusError{r};
    }
    std::vector<Win<T>> src;
    std::vector<T*> Vnh(P, nullptr);
    for (int j = 0; j < P; ++j) {
        if (mj[j] == 0) continue;
        Win<T> W;
        W.w = j;
        W.b = mj[j];
        W.V = as<T>(bs_alloc(c, sizeof(T) * (size_t)n * W.b * (S.kmax + 1)));
        W.S = as<T>(bs_alloc(c, sizeof(T) * (size_t)n * (L.ycols - 1) * W.b));
        W.Wlo = std::is_same<T, float>::value ? as<float>(bs_alloc(c, sizeof(float) * (size_t)n * W.b)) : nullptr;
        W.V1lo = std::is_same<T, float>::value ? as<float>(bs_alloc(c, sizeof(float) * (size_t)n * W.b)) : nullptr;
        win_ops(W, j);
        Vnh[j] = W.V;
        src.push_back(W);
    }
    {
        const int ns = (int)src.size();
        Stage s2(c, 1);
        std::vector<TsTask<T>> tu(ns), tgr(ns), tsc(ns);
        std::vector<int> wl(ns);
        int mpq = 0, mq = 0, mpqg = 0;
        for (int a = 0; a < ns; ++a) {
            const Win<T>& W = src[a];
            const int j = W.w;
            const int s = src_count(j);
            TsTask<T> t;
            memset(&t, 0, sizeof(t));
            t.X = src_first(j); t.ldx = n; t.xs = Au0; t.p = s; t.q = W.b;
            t.Z = W.V; t.ldz = n; t.Tm = S.D(j) + L.off_zs; t.ldt = L.s_max; t.alpha = 1.0; t.beta = 0.0;
            tu[a] = t;
            mpq = std::max(mpq, s * W.b);
            memset(&t, 0, sizeof(t));
            t.X = W.V; t.ldx = n; t.p = W.b; t.Y = W.V; t.ldy = n; t.q = W.b; t.q1 = W.b;
            t.out = S.D(j) + L.off_gw;
            tgr[a] = t;
            mpqg = std::max(mpqg, W.b * W.b);
            mq = std::max(mq, W.b);
            memset(&t, 0, sizeof(t));
            t.X = W.V; t.ldx = n; t.p = W.b; t.q = W.b; t.Z = W.V; t.ldz = n;
            t.Tm = S.D(j) + L.off_T; t.ldt = W.b; t.alpha = 1.0; t.beta = 0.0;
            tsc[a] = t;
            wl[a] = j;
        }
        const TsTask<T>* dtu = s2.put(tu.data(), ns);
        const TsTask<T>* dtg = s2.put(tgr.data(), ns);
        const TsTask<T>* dts = s2.put(tsc.data(), ns);
        const int* dwl = s2.put(wl.data(), ns);
        const DfTask* ddu = nullptr;
        const DfTask* dds = nullptr;
        if constexpr (std::is_same<T, float>::value) {
            // U = (A u0 1^T + G) Z S^{-1} in double-float: the columns of G_hat nearly
            // cancel for the smaller singular values.
            std::vector<DfTask> du(ns);
            for (int a = 0; a < ns; ++a) {
                DfTask t;
                memset(&t, 0, sizeof(t));
                t.Xh = tu[a].X; t.ldx = n; t.xs = Au0; t.Zh = tu[a].Z; t.Zl = src[a].V1lo; t.ldz = n;
                t.Tm = tu[a].Tm; t.ldt = tu[a].ldt; t.p = tu[a].p; t.q = tu[a].q; t.alpha = 1.0;
                du[a] = t;
            }
            ddu = s2.put(du.data(), ns);
            // re-orthonormalisation of the start block keeps its low part
            std::vector<DfTask> dsc(ns);
            for (int a = 0; a < ns; ++a) {
                DfTask t;
                memset(&t, 0, sizeof(t));
                t.Xh = src[a].V; t.Xl = src[a].V1lo; t.ldx = n; t.Zh = src[a].V; t.Zl = src[a].V1lo; t.ldz = n;
                t.Tm = tsc[a].Tm; t.ldt = tsc[a].ldt; t.p = src[a].b; t.q = src[a].b; t.alpha = 1.0;
                dsc[a] = t;
            }
            dds = s2.put(dsc.data(), ns);
        }
        s2.flush();
        if (ddu) launch_ts_nn_df(ddu, ns, mpq, n, st, mq);
        else launch_ts_nn<T>(dtu, ns, mpq, n, st);
        check_launch(c);
        if (mq <= 4) {
            // Gram of the start blocks: streamed partials, summed into each window's slab
            std::vector<UpdTask<T>> gtk(ns);
            for (int a = 0; a < ns; ++a) {
                UpdTask<T> t;
                memset(&t, 0, sizeof(t));
                t.Wh = src[a].V; t.ld = n; t.p = src[a].b;
                gtk[a] = t;
            }
            Stage sg(c, 0);
            const UpdTask<T>* dgt = sg.put(gtk.data(), ns);
            sg.flush();
            const KGeom gq = krylov_geom(ns, n);
            launch_block_gram<T>(dgt, ns, n, gq, S.kpart[1], mq * mq, st); check_launch(c);
            launch_sum_parts(S.kpart[1], gq.nchunks, mq * mq, mq * mq, S.wd, L.stride, L.off_gw, dwl, ns, nullptr, 0, 0,
                             st);
            check_launch(c);
        } else {
            launch_ts_tn<T>(dtg, ns, mpqg, mq, n, S.partial, st, 1); check_launch(c);
        }
        launch_start_orth(L, S.wd, S.wi, dwl, ns, st); check_launch(c);
        if (dds) launch_ts_nn_df(dds, ns, mpqg, n, st, mq);
        else launch_ts_nn<T>(dts, ns, mpqg, n, st);
        check_launch(c);
        launch_spline(L, S.wd, S.wi, dwl, ns, S.h, st); check_launch(c);
        sync(c);   // staging half 1 is reused by the Krylov loop
    }

    nvtx.next("pexp: nonhomogeneous block Krylov");
    cudaEventRecord(c->evp[1], st);
    // the Krylov steps take the rounded start block (see the note on the solve's input)
    for (auto& W : src) W.V1lo = nullptr;
    // ---- nonhomogeneous parts, all subintervals in one batch
    int k_nh = 0;
    int notconv = S.run(src, KIND_SOURCE, &k_nh);
    d2h(c, S.wi_host.data(), S.wi, sizeof(int) * S.wi_host.size());
    std::vector<int> Knh(P, 0);
    for (int j = 0; j < P; ++j) Knh[j] = S.wi_host[(size_t)j * L.istride + WI_K];
    double orth_max = -1.0;
    if (o->diagnostics & PEXP_DIAG_ORTH) {
        orth_max = 0.0;
        for (int j = 0; j < P; ++j)
            if (Vnh[j]) orth_max = std::max(orth_max, S.orth_defect_cycles(Vnh[j], Knh[j], mj[j]));
    }

    nvtx.next("pexp: homogeneous chain");
    cudaEventRecord(c->evp[2], st);
    // ---- homogeneous chain over windows 2..P
    std::vector<T*> Vh(P, nullptr);
    std::vector<int> Kh(P, 0), steps_h(P, 0);
    const double* u0_out = ja == 0 ? u0d : nullptr;   // u0 belongs to the range that starts at t = 0
    // reconstruction task of window m: its nonhomogeneous part and (m >= 1) the continuation
    // of the solution from T_m; the first sample of a window m >= 1 is the last of window m - 1
    auto recon_task = [&](int m) {
        ReconTask<T> rt;
        memset(&rt, 0, sizeof(rt));
        const int s = pt.idx[m + 1] - pt.idx[m] + 1;
        if (Vnh[m]) { rt.V1 = Vnh[m]; rt.C1 = S.D(m) + L.off_Y; rt.ld1 = n; rt.K1 = Knh[m]; rt.ldc1 = L.K_max; }
        if (m >= 1 && Vh[m] && Kh[m] > 0) { rt.V2 = Vh[m]; rt.C2 = S.D(P + m) + L.off_Y; rt.ld2 = n; rt.K2 = Kh[m]; rt.ldc2 = L.K_max; }
        rt.r0 = (m == 0) ? 0 : 1;
        rt.ns = s - rt.r0;
        rt.i0 = pt.idx[m] + rt.r0;
        return rt;
    };
    // host outputs: a window's rows are final once its continuation is solved, so they are
    // reconstructed then and copied out on the copy stream while the chain goes on
    auto emit_window = [&](int m) {
        const ReconTask<T> rt = recon_task(m);
        Stage so(c, 1);
        const ReconTask<T>* drt = so.put(&rt, 1);
        so.flush();
        timed(c, PEXP_KC_RECON, (double)n * (rt.K1 + rt.K2) * sizeof(T) + (double)n * rt.ns * sizeof(TO),
              [&] { launch_recon<T, TO>(drt, 1, rt.ns, n, u0_out, Y, n, std::max(1, rt.K1 + rt.K2), st); });
        check_launch(c);
        cudaEventRecord(c->ev_out, st);
        cudaStreamWaitEvent(c->cs, c->ev_out, 0);
        const cudaError_t e = cudaMemcpyAsync(Y_host + (size_t)rt.i0 * n, Y + (size_t)rt.i0 * n,
                                              sizeof(TO) * (size_t)rt.ns * n, cudaMemcpyDeviceToHost, c->cs);
        if (e != cudaSuccess) {
            fail_cuda(e, "cudaMemcpyAsync D2H (window outputs)", __FILE__, __LINE__);
            throw StatusError{PEXP_ERR_CUDA};
        }
    };
    if (ja > 0) {
        // rows before and at T_ja: the range's solution is zero there
        const size_t zr = (size_t)pt.idx[ja] + 1;
        cudaMemsetAsync(Y, 0, sizeof(TO) * zr * n, st);
        if (Y_host) {
            cudaEventRecord(c->ev_out, st);
            cudaStreamWaitEvent(c->cs, c->ev_out, 0);
            cudaMemcpyAsync(Y_host, Y, sizeof(TO) * zr * n, cudaMemcpyDeviceToHost, c->cs);
        }
    }
    // the first window of the range has no continuation: its rows are final already
    if (Y_host) emit_window(ja);
    int k_hom_max = 0, k_hom_sum = 0;
    T* Sh = as<T>(bs_alloc(c, sizeof(T) * (size_t)n * (L.ycols - 1)));
    float* Whlo = std::is_same<T, float>::value ? as<float>(bs_alloc(c, sizeof(float) * (size_t)n)) : nullptr;
    // low part of z while it is formed and normalised
    float* Vh1lo_buf = std::is_same<T, float>::value ? as<float>(bs_alloc(c, sizeof(float) * (size_t)n)) : nullptr;
    for (int m = 1; m < P; ++m) {   // 0-based window m needs z at T_m (end of window m-1)
        if (m <= ja) continue;      // nothing of subproblems ja.. exists before T_ja
        Vh[m] = as<T>(bs_alloc(c, sizeof(T) * (size_t)n * (S.kmax + 1)));
        const int wprev = m - 1;
        const int sprev = pt.idx[m] - pt.idx[m - 1] + 1;
        Stage s3(c, 0);
        ReconTask<T> rt;
        memset(&rt, 0, sizeof(rt));
        rt.V1 = Vnh[wprev]; rt.C1 = S.D(wprev) + L.off_Y; rt.ld1 = n; rt.K1 = Vnh[wprev] ? Knh[wprev] : 0; rt.ldc1 = L.K_max;
        if (m - 1 >= 1) {
            rt.V2 = Vh[m - 1]; rt.C2 = S.D(P + m - 1) + L.off_Y; rt.ld2 = n; rt.K2 = Kh[m - 1]; rt.ldc2 = L.K_max;
        }
        rt.r0 = sprev - 1; rt.ns = 1; rt.i0 = 0;
        const ReconTask<T>* drt = s3.put(&rt, 1);
        TsTask<T> tsc;
        memset(&tsc, 0, sizeof(tsc));
        tsc.X = Vh[m]; tsc.ldx = n; tsc.p = 1; tsc.q = 1; tsc.Z = Vh[m]; tsc.ldz = n;
        tsc.Tm = S.D(P + m) + L.off_T; tsc.ldt = 1; tsc.alpha = 1.0; tsc.beta = 0.0;
        UpdTask<T> zg;
        memset(&zg, 0, sizeof(zg));
        zg.Wh = Vh[m]; zg.ld = n; zg.p = 1;
        const UpdTask<T>* dzg = s3.put(&zg, 1);
        const TsTask<T>* dts = s3.put(&tsc, 1);
        int wsel = P + m;
        const int* dw = s3.put(&wsel, 1);
        // FP32 data: z = u_hat(T_m) and its normalisation in double-float, then rounded into
        // the start vector: the window's Krylov space and its projected matrix both use that
        // rounded vector, so the rounding (white noise) is resolved by the projected problem
        // instead of following the dynamics of the start vector
        const DfTask* dz = nullptr;
        int nz = 0;
        DfTask zt[3];
        memset(zt, 0, sizeof(zt));
        float* Vh1lo = Vh1lo_buf;
        if constexpr (std::is_same<T, float>::value) {
            int acc = 0;
            if (rt.K1 > 0) {
                DfTask& t = zt[nz++];
                t.Xh = rt.V1; t.ldx = n; t.Zh = Vh[m]; t.Zl = Vh1lo; t.ldz = n;
                t.Tm = rt.C1 + (int64_t)rt.r0 * rt.ldc1; t.ldt = rt.K1; t.p = rt.K1; t.q = 1; t.alpha = 1.0;
                t.accumulate = acc;
                acc = 1;
            }
            if (rt.K2 > 0) {
                DfTask& t = zt[nz++];
                t.Xh = rt.V2; t.ldx = n; t.Zh = Vh[m]; t.Zl = Vh1lo; t.ldz = n;
                t.Tm = rt.C2 + (int64_t)rt.r0 * rt.ldc2; t.ldt = rt.K2;
                t.p = rt.K2; t.q = 1; t.alpha = 1.0; t.accumulate = acc;
            }
            DfTask& t = zt[2];
            t.Xh = Vh[m]; t.Xl = Vh1lo; t.ldx = n; t.Zh = Vh[m]; t.Zl = Vh1lo; t.ldz = n;
            t.Tm = S.D(P + m) + L.off_T; t.ldt = 1; t.p = 1; t.q = 1; t.alpha = 1.0;
            dz = s3.put(zt, 3);
        }
        s3.flush();
        const int maxc = std::max(1, (rt.K1 + rt.K2));
        if (dz) {
            if (nz == 0) cudaMemsetAsync(Vh[m], 0, sizeof(T) * (size_t)n, st);
            for (int k = 0; k < nz; ++k) {
                launch_ts_nn_df(dz + k, 1, std::max(rt.K1, rt.K2), n, st, 1);
                check_launch(c);
            }
        } else {
            launch_recon<T, T>(drt, 1, 1, n, nullptr, Vh[m], n, maxc, st); check_launch(c);
        }
        {
            // ||z||^2 for the normalisation: streamed partials summed into the window's slab
            const KGeom gz = krylov_geom(1, n);
            launch_block_gram<T>(dzg, 1, n, gz, S.kpart[1], 1, st); check_launch(c);
            launch_sum_parts(S.kpart[1], gz.nchunks, 1, 1, S.wd, L.stride, L.off_gw, dw, 1, nullptr, 0, 0, st);
            check_launch(c);
        }
        launch_start_orth(L, S.wd, S.wi, dw, 1, st); check_launch(c);
        if (dz) launch_ts_nn_df(dz + 2, 1, 1, n, st, 1);
        else launch_ts_nn<T>(dts, 1, 1, n, st);
        check_launch(c);
        // a zero z (nothing to continue) is marked converged with an empty basis on the device
        std::vector<Win<T>> one(1);
        one[0].w = P + m; one[0].V = Vh[m]; one[0].S = Sh; one[0].b = 1; one[0].Wlo = Whlo; one[0].V1lo = nullptr;
        win_ops(one[0], m);   // the continuation on subinterval m has that subinterval's operator
        int kh = 0;
        notconv += S.run(one, KIND_HOM, &kh);
        const int kk = S.wi_host[(size_t)(P + m) * L.istride + WI_K];   // state after the last step
        Kh[m] = kk;
        if (o->diagnostics & PEXP_DIAG_ORTH) orth_max = std::max(orth_max, S.orth_defect_cycles(Vh[m], kk, 1));
        k_hom_max = std::max(k_hom_max, kh);
        k_hom_sum += kh;
        steps_h[m] = kh;
        if (Y_host) emit_window(m);
    }
    S.check_coop();

    nvtx.next("pexp: reconstruction");
    cudaEventRecord(c->evp[3], st);
    if (Y_host) {
        // every window has been reconstructed and is on its way to the host
        cudaEventRecord(c->evp[4], st);
        sync(c);
        const cudaError_t e = cudaStreamSynchronize(c->cs);
        if (e != cudaSuccess) {
            fail_cuda(e, "cudaStreamSynchronize (copy stream)", __FILE__, __LINE__);
            throw StatusError{PEXP_ERR_CUDA};
        }
    } else {
        // ---- reconstruction of all windows in one launch
        Stage s4(c, 1);
        std::vector<ReconTask<T>> rts;
        int maxc = 1, maxns = 1;
        for (int m = ja; m < P; ++m) {
            const ReconTask<T> rt = recon_task(m);
            maxc = std::max(maxc, rt.K1 + rt.K2);
            maxns = std::max(maxns, rt.ns);
            rts.push_back(rt);
        }
        const ReconTask<T>* drt = s4.put(rts.data(), rts.size());
        s4.flush();
        double kt = 0;
        for (auto& r : rts) kt += r.K1 + r.K2;
        timed(c, PEXP_KC_RECON, (double)n * kt * sizeof(T) + (double)n * n_out * sizeof(TO),
              [&] { launch_recon<T, TO>(drt, (int)rts.size(), maxns, n, u0_out, Y, n, maxc, st); });
        check_launch(c);
        cudaEventRecord(c->evp[4], st);
        sync(c);
    }

    if (rep) {
        float ms[4] = {0, 0, 0, 0};
        for (int k = 0; k < 4; ++k) cudaEventElapsedTime(&ms[k], c->evp[k], c->evp[k + 1]);
        rep->t_source_ms = ms[0];
        rep->t_krylov_ms = ms[1];
        rep->t_hom_ms = ms[2];
        rep->t_recon_ms = ms[3];
        double est_max = 0, sig_max = 0;
        for (int j = 0; j < P; ++j) {
            double sc[WS_COUNT];
            d2h(c, sc, S.D(j) + L.off_scal, sizeof(sc));
            est_max = std::max(est_max, sc[WS_EST]);
            sig_max = std::max(sig_max, sc[WS_SIGRATIO]);
        }
        rep->n_sub = P;
        rep->rank_max = b_max;
        rep->rank_min = b_min;
        rep->k_nh_max = k_nh;
        rep->k_hom_max = k_hom_max;
        rep->k_hom_sum = k_hom_sum;
        rep->not_converged = notconv;
        rep->est_max = est_max;
        rep->sigma_ratio_max = sig_max;
        rep->orth_max = orth_max;
        for (int j = 0; j < std::min(P, PEXP_REPORT_SUBS); ++j) {
            rep->sub_rank[j] = mj[j];
            rep->sub_steps[j] = mj[j] > 0 ? S.wi_host[(size_t)j * L.istride + WI_STEPS] : 0;
            rep->sub_hom_steps[j] = steps_h[j];
            rep->sub_restarts[j] = S.restarts[j];
        }
        const double w = (double)sizeof(T);
        double bytes = 0;
        // algorithmic bytes, each array counted once per pass the method needs: two passes
        // over the source samples and the write of U per window; per Krylov step of a
        // window, the basis reads of the projection and Gram-Schmidt passes (2k(k+1) columns
        // over k steps) and ~14 column passes of the working block; the homogeneous chain
        // likewise; the reconstruction below
        for (int j = 0; j < P; ++j) {
            const int s = src_count(j);
            bytes += 2.0 * n * s * w + (double)n * mj[j] * w;
            const double k = Knh[j] / std::max(1, mj[j]);
            bytes += (double)n * mj[j] * w * (2.0 * k * (k + 1) + 14.0 * k);
            if (j >= 1) { const double kh = Kh[j]; bytes += (double)n * w * (2.0 * kh * (kh + 1) + 14.0 * kh); }
        }
        bytes += (double)n * n_out * (double)sizeof(TO);
        rep->bytes_alg = bytes;
    }
    return notconv ? PEXP_ERR_NOT_CONVERGED : PEXP_OK;
}

int solve_linear_dispatch(pexp_ctx* c, const pexp_operator* op, const pexp_options* o, const void* y0_dev,
                          const void* G_dev, int g_dtype, void* Y_dev, int y_dtype, pexp_report* rep,
                          size_t keep_top, const WinOps<double>* wo64 = nullptr, const WinOps<float>* wo32 = nullptr,
                          void* Y_host = nullptr) {
    const OpDesc od = make_opdesc(*op);
    const int64_t n = od.n;
    const bool fp64 = o->precision == PEXP_FP64;
    Partition pt = make_partition(o->n_out, o->P);
    const int b_cap = std::min(std::min(o->max_rank, PEXP_MAX_RANK), make_src_partition(o, pt).smax);
    const int g_conv = G_dev && ((g_dtype == PEXP_F64) != fp64);
    size_t need = keep_top +
                  (fp64 ? linear_workspace_bytes<double>(n, o, g_conv, b_cap)
                        : linear_workspace_bytes<float>(n, o, g_conv, b_cap));
    if (need > c->ws_cap) {
        if (keep_top) return PEXP_ERR_OOM;   // cannot move live buffers of the caller
        int r = ws_reserve(c, need);
        if (r) return r;
    }
    c->ws_top = keep_top;
    // the initial condition is FP64 in every precision (A u0 amplifies its rounding by ||A||)
    const double* u0d = reinterpret_cast<const double*>(y0_dev);
    if (fp64) {
        if (y_dtype == PEXP_F64)
            return solve_linear_typed<double, double>(c, op, o, u0d, G_dev, g_dtype, as<double>(Y_dev), rep, wo64,
                                                      as<double>(Y_host));
        return solve_linear_typed<double, float>(c, op, o, u0d, G_dev, g_dtype, as<float>(Y_dev), rep, wo64,
                                                 as<float>(Y_host));
    }
    if (y_dtype == PEXP_F64)
        return solve_linear_typed<float, double>(c, op, o, u0d, G_dev, g_dtype, as<double>(Y_dev), rep, wo32,
                                                 as<double>(Y_host));
    return solve_linear_typed<float, float>(c, op, o, u0d, G_dev, g_dtype, as<float>(Y_dev), rep, wo32, as<float>(Y_host));
}

template <typename F>
int guarded(F&& f) {
    try {
        return f();
    } catch (const OomError&) {
        return PEXP_ERR_OOM;
    } catch (const StatusError& e) {
        return e.code;
    } catch (const std::bad_alloc&) {
        return PEXP_ERR_OOM;
    } catch (...) {
        return PEXP_ERR_CUDA;
    }
}

}  // namespace

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

void pexp_default_options(pexp_options* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->T = 1.0;
    o->P = 1;
    o->n_out = 2;
    o->tol = 1e-8;
    o->svd_tol = 1e-12;
    o->max_rank = 16;
    o->restart_len = 20;
    o->max_restarts = 0;
    o->krylov = PEXP_KRYLOV_SAI;
    o->sai_gamma = 0.1;
    o->precision = PEXP_FP64;
    o->wr_max_iter = 50;
    o->wr_tol = 1e-6;
    o->burgers_form = 0;
    o->jacobian = 0;
    o->wr_diverge = 3;
}

const char* pexp_status_string(int s) {
    switch (s) {
        case PEXP_OK: return "ok";
        case PEXP_ERR_INVALID_ARG: return "invalid argument";
        case PEXP_ERR_OOM: return "out of device memory";
        case PEXP_ERR_CUDA: return "CUDA error";
        case PEXP_ERR_BREAKDOWN: return "Krylov breakdown";
        case PEXP_ERR_NOT_CONVERGED: return "Krylov tolerance not reached";
        case PEXP_ERR_WR_NOT_CONVERGED: return "waveform relaxation not converged";
        case PEXP_ERR_TIMEOUT: return "device wait timed out";
        case PEXP_ERR_UNSUPPORTED: return "unsupported operator/precision combination";
        case PEXP_ERR_SCRATCH_LIMIT: return "request exceeds the fixed scratch of the allocation-free entry point";
        case PEXP_ERR_WR_DIVERGED: return "waveform relaxation diverged (the update grew in successive iterations)";
        default: return "unknown status";
    }
}

int pexp_create(pexp_ctx** out, int device, void* stream) {
    if (!out) return PEXP_ERR_INVALID_ARG;
    *out = nullptr;
    pexp_ctx* c = new (std::nothrow) pexp_ctx();
    if (!c) return PEXP_ERR_OOM;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess) { delete c; return PEXP_ERR_CUDA; }
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    c->stage_cap = kStageBytes / (kSlots / 2);
    for (int h = 0; h < 2; ++h) {
        if (cudaMallocHost(&c->stage_h[h], kStageBytes) != cudaSuccess ||
            cudaMalloc(&c->stage_d[h], kStageBytes) != cudaSuccess) {
            pexp_destroy(c);
            return PEXP_ERR_OOM;
        }
    }
    for (int k = 0; k < kSlots; ++k) cudaEventCreateWithFlags(&c->slot_ev[k], cudaEventDisableTiming);
    if (cudaStreamCreateWithFlags(&c->s2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_sp, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_pj, cudaEventDisableTiming) != cudaSuccess) {
        pexp_destroy(c);
        return PEXP_ERR_CUDA;
    }
    cudaEventCreate(&c->ev0);
    cudaEventCreate(&c->ev1);
    for (int k = 0; k < 5; ++k) cudaEventCreate(&c->evp[k]);
    if (cudaMalloc(&c->bar, 256) != cudaSuccess || cudaMemset(c->bar, 0, 256) != cudaSuccess) {
        pexp_destroy(c);
        return PEXP_ERR_OOM;
    }
    init_pade_constants();
    *out = c;
    return PEXP_OK;
}

int pexp_destroy(pexp_ctx* c) {
    if (!c) return PEXP_OK;
    for (pexp_ctx* w : c->workers) pexp_destroy(w);
    c->workers.clear();
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->owns_stream && c->stream) {
        cudaStreamDestroy(c->stream);
        c->stream = nullptr;
    }
    if (c->ws) cudaFree(c->ws);
    if (c->bs) cudaFree(c->bs);
    if (c->bar) cudaFree(c->bar);
    for (int h = 0; h < 2; ++h) {
        if (c->stage_h[h]) cudaFreeHost(c->stage_h[h]);
        if (c->stage_d[h]) cudaFree(c->stage_d[h]);
    }
    if (c->io_d) cudaFree(c->io_d);
    for (int k = 0; k < kSlots; ++k)
        if (c->slot_ev[k]) cudaEventDestroy(c->slot_ev[k]);
    if (c->flags_h) cudaFreeHost(c->flags_h);
    for (int k = 0; k < kFlagBufs; ++k)
        if (c->flag_ev[k]) cudaEventDestroy(c->flag_ev[k]);
    if (c->s2) {
        cudaStreamSynchronize(c->s2);
        cudaStreamDestroy(c->s2);
    }
    if (c->cs) {
        cudaStreamSynchronize(c->cs);
        cudaStreamDestroy(c->cs);
    }
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    if (c->ev_sp) cudaEventDestroy(c->ev_sp);
    if (c->ev_pj) cudaEventDestroy(c->ev_pj);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    for (int k = 0; k < 5; ++k)
        if (c->evp[k]) cudaEventDestroy(c->evp[k]);
    delete c;
    return PEXP_OK;
}

int pexp_set_stream(pexp_ctx* c, void* stream) {
    if (!c) return PEXP_ERR_INVALID_ARG;
    c->stream = reinterpret_cast<cudaStream_t>(stream);
    return PEXP_OK;
}

}  // extern "C"

namespace {
// One linear solve with device inputs; Y_host != NULL: the outputs are also copied to Y_host
// window by window as they are completed (the host entry point).
int solve_linear_entry(pexp_ctx* c, const pexp_operator* op, const pexp_options* o, const void* y0_dev,
                       const void* G_dev, int g_dtype, void* Y_dev, int y_dtype, pexp_report* rep, void* Y_host) {
    if (!c || !y0_dev || !Y_dev) return PEXP_ERR_INVALID_ARG;
    if ((g_dtype != PEXP_F64 && g_dtype != PEXP_F32) || (y_dtype != PEXP_F64 && y_dtype != PEXP_F32))
        return PEXP_ERR_INVALID_ARG;
    int v = validate(op, o);
    if (v) return v;
    if (rep) memset(rep, 0, sizeof(*rep));
    cudaSetDevice(c->device);
    c->launches = 0;
    c->kt.reset((o->diagnostics & PEXP_DIAG_KTIME) != 0, ((unsigned)o->diagnostics >> 8) & 0xffu,
                ((unsigned)o->diagnostics >> 16) & 0xfu);
    cudaEventRecord(c->ev0, c->stream);
    int r = guarded([&] {
        return solve_linear_dispatch(c, op, o, y0_dev, G_dev, g_dtype, Y_dev, y_dtype, rep, 0, nullptr, nullptr, Y_host);
    });
    cudaEventRecord(c->ev1, c->stream);
    cudaEventSynchronize(c->ev1);
    if (rep && c->kt.on) {
        for (auto& k : c->kt.recs) {
            float ms = 0;
            cudaEventElapsedTime(&ms, k.a, k.b);
            rep->k_ms[k.cls] += ms;
            rep->k_launches[k.cls] += 1;
            rep->k_bytes[k.cls] += k.bytes;
            rep->k_bytes_alg[k.cls] += k.alg;
        }
    }
    if (rep) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        rep->time_ms = ms;
        rep->launches = c->launches;
        rep->status = r;
    }
    return r;
}
}  // namespace

extern "C" {

int pexp_solve_linear(pexp_ctx* c, const pexp_operator* op, const pexp_options* o, const void* y0_dev,
                      const void* G_dev, int g_dtype, void* Y_dev, int y_dtype, pexp_report* rep) {
    return solve_linear_entry(c, op, o, y0_dev, G_dev, g_dtype, Y_dev, y_dtype, rep, nullptr);
}

int pexp_selftest_barrier(pexp_ctx* c, int absent_cta) {
    if (!c) return PEXP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    const GridBar bar{c->bar, c->bar + 1, reinterpret_cast<int*>(c->bar + 2)};
    if (launch_bar_selftest(bar, absent_cta, c->stream) <= 0) return PEXP_ERR_UNSUPPORTED;
    int err = 0;
    PEXP_CUDA_TRY(cudaMemcpyAsync(&err, c->bar + 2, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PEXP_CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (err) {
        PEXP_CUDA_TRY(cudaMemsetAsync(c->bar, 0, 3 * sizeof(unsigned), c->stream));
        PEXP_CUDA_TRY(cudaStreamSynchronize(c->stream));
        return PEXP_ERR_TIMEOUT;
    }
    return PEXP_OK;
}

int pexp_solve_linear_host(pexp_ctx* c, const pexp_operator* op, const pexp_options* o, const void* y0_host,
                           const void* G_host, int g_dtype, void* Y_host, int y_dtype, pexp_report* rep) {
    if (!c || !y0_host || !Y_host) return PEXP_ERR_INVALID_ARG;
    int v = validate(op, o);
    if (v) return v;
    const OpDesc od = make_opdesc(*op);
    const size_t n = (size_t)od.n;
    const size_t ys = (y_dtype == PEXP_F64) ? 8 : 4, gs = (g_dtype == PEXP_F64) ? 8 : 4;
    const size_t grows = (size_t)src_rows_of(o);
    const size_t bytes = align_up(n * 8) + (G_host ? align_up(n * grows * gs) : 0) + align_up(n * o->n_out * ys);
    cudaSetDevice(c->device);
    if (bytes > c->io_cap) {
        if (c->io_d) cudaFree(c->io_d);
        c->io_d = nullptr;
        c->io_cap = 0;
        if (cudaMalloc(&c->io_d, bytes) != cudaSuccess) { cudaGetLastError(); return PEXP_ERR_OOM; }
        c->io_cap = bytes;
    }
    char* p = reinterpret_cast<char*>(c->io_d);
    void* y0d = p;
    p += align_up(n * 8);
    void* Gd = nullptr;
    if (G_host) { Gd = p; p += align_up(n * grows * gs); }
    void* Yd = p;
    PEXP_CUDA_TRY(cudaMemcpyAsync(y0d, y0_host, n * 8, cudaMemcpyHostToDevice, c->stream));
    if (G_host) PEXP_CUDA_TRY(cudaMemcpyAsync(Gd, G_host, n * grows * gs, cudaMemcpyHostToDevice, c->stream));
    // the outputs leave window by window on the copy stream while the continuation chain runs
    return solve_linear_entry(c, op, o, y0d, Gd, g_dtype, Yd, y_dtype, rep, Y_host);
}

}  // extern "C"

namespace {

constexpr int kDefaultBatchWorkers = 4;

double problem_cost(const pexp_problem& p) {
    const double n = (double)p.op.nx * (p.op.dim == 2 ? (double)p.op.ny : 1.0);
    return n * ((double)p.opts.n_out + 40.0 * p.opts.P);
}

int ensure_workers(pexp_ctx* c, int k) {
    while ((int)c->workers.size() < k) {
        cudaSetDevice(c->device);
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return PEXP_ERR_CUDA;
        pexp_ctx* w = nullptr;
        const int r = pexp_create(&w, c->device, st);
        if (r) {
            cudaStreamDestroy(st);
            return r;
        }
        w->owns_stream = true;
        w->coop = false;
        c->workers.push_back(w);
    }
    return PEXP_OK;
}

int run_batched(pexp_ctx* c, int count, const pexp_problem* probs, pexp_report* reps, int k) {
    k = std::max(1, std::min(k, count));
    int r = ensure_workers(c, k);
    if (r) return r;
    cudaSetDevice(c->device);
    // the workers start after the work queued on the caller's stream
    PEXP_CUDA_TRY(cudaEventRecord(c->ev0, c->stream));
    for (int w = 0; w < k; ++w) PEXP_CUDA_TRY(cudaStreamWaitEvent(c->workers[w]->stream, c->ev0, 0));
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int a, int b) { return problem_cost(probs[a]) > problem_cost(probs[b]); });
    std::vector<int> st(count, PEXP_OK);
    std::atomic<int> next{0};
    auto work = [&](pexp_ctx* w) {
        for (;;) {
            const int q = next.fetch_add(1);
            if (q >= count) break;
            const int i = order[q];
            const pexp_problem& p = probs[i];
            pexp_report local;
            st[i] = solve_linear_entry(w, &p.op, &p.opts, p.y0_dev, p.G_dev, p.g_dtype, p.Y_dev, p.y_dtype,
                                       reps ? &reps[i] : &local, nullptr);
        }
    };
    std::vector<std::thread> th;
    for (int w = 1; w < k; ++w) th.emplace_back(work, c->workers[w]);
    work(c->workers[0]);
    for (auto& t : th) t.join();
    // later work on the caller's stream comes after every worker's
    for (int w = 0; w < k; ++w) {
        PEXP_CUDA_TRY(cudaEventRecord(c->workers[w]->ev1, c->workers[w]->stream));
        PEXP_CUDA_TRY(cudaStreamWaitEvent(c->stream, c->workers[w]->ev1, 0));
    }
    for (int i = 0; i < count; ++i)
        if (st[i] != PEXP_OK) return st[i];
    return PEXP_OK;
}

std::string device_key(int dev) {
    cudaDeviceProp pr;
    if (cudaGetDeviceProperties(&pr, dev) != cudaSuccess) return "unknown";
    return std::string(pr.name) + " sm" + std::to_string(pr.multiProcessorCount);
}

}  // namespace

extern "C" {

int pexp_solve_batched(pexp_ctx* c, int count, const pexp_problem* probs, pexp_report* reps) {
    if (!c || count < 0 || (count > 0 && !probs)) return PEXP_ERR_INVALID_ARG;
    for (int i = 0; i < count; ++i) {
        const pexp_problem& p = probs[i];
        if (!p.y0_dev || !p.Y_dev) return PEXP_ERR_INVALID_ARG;
        if ((p.g_dtype != PEXP_F64 && p.g_dtype != PEXP_F32) || (p.y_dtype != PEXP_F64 && p.y_dtype != PEXP_F32))
            return PEXP_ERR_INVALID_ARG;
        const int v = validate(&p.op, &p.opts);
        if (v) return v;
    }
    if (reps) memset(reps, 0, sizeof(pexp_report) * (size_t)count);
    if (count == 0) return PEXP_OK;
    return run_batched(c, count, probs, reps, c->batch_workers > 0 ? c->batch_workers : kDefaultBatchWorkers);
}

int pexp_autotune(pexp_ctx* c, int count, const pexp_problem* probs, const char* path) {
    if (!c || count < 1 || !probs) return PEXP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    const std::string key = device_key(c->device);
    if (path) {
        // a table for this device: {"device": "<name> sm<count>", "batch_workers": k, ...}
        FILE* f = fopen(path, "r");
        if (f) {
            std::string txt;
            char buf[4096];
            size_t got;
            while ((got = fread(buf, 1, sizeof(buf), f)) > 0) txt.append(buf, got);
            fclose(f);
            const size_t dk = txt.find("\"device\": \"" + key + "\"");
            const size_t bw = txt.find("\"batch_workers\": ");
            if (dk != std::string::npos && bw != std::string::npos) {
                const int k = atoi(txt.c_str() + bw + 17);
                if (k >= 1 && k <= 64) {
                    c->batch_workers = k;
                    return PEXP_OK;
                }
            }
        }
    }
    for (int i = 0; i < count; ++i) {
        const int v = validate(&probs[i].op, &probs[i].opts);
        if (v) return v;
    }
    const int cand[] = {1, 2, 4, 8, 16};
    double best_ms = 1e300;
    int best = kDefaultBatchWorkers;
    std::string timings;
    for (int k : cand) {
        int r = run_batched(c, count, probs, nullptr, k);   // warm-up: workspaces grown
        if (r != PEXP_OK && r != PEXP_ERR_NOT_CONVERGED) return r;
        cudaStreamSynchronize(c->stream);
        const auto t0 = std::chrono::steady_clock::now();
        r = run_batched(c, count, probs, nullptr, k);
        cudaStreamSynchronize(c->stream);
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (r != PEXP_OK && r != PEXP_ERR_NOT_CONVERGED) return r;
        char e[64];
        snprintf(e, sizeof(e), "%s\"%d\": %.3f", timings.empty() ? "" : ", ", k, ms);
        timings += e;
        if (ms < best_ms) {
            best_ms = ms;
            best = k;
        }
    }
    c->batch_workers = best;
    if (path) {
        FILE* f = fopen(path, "w");
        if (!f) return PEXP_ERR_INVALID_ARG;
        fprintf(f, "{\"device\": \"%s\", \"batch_workers\": %d, \"problems\": %d, \"timings_ms\": {%s}}\n",
                key.c_str(), best, count, timings.c_str());
        fclose(f);
    }
    return PEXP_OK;
}

int pexp_solve_burgers(pexp_ctx* c, const pexp_operator* op, const pexp_options* o, const void* u0_dev,
                       const void* forcing_dev, const void* init_dev, void* U_dev, int dtype, pexp_report* rep) {
    if (!c || !u0_dev || !U_dev || !op || !o) return PEXP_ERR_INVALID_ARG;
    if (op->dim != 1 || op->ax != 0.0) return PEXP_ERR_INVALID_ARG;
    if (dtype != PEXP_F64 && dtype != PEXP_F32) return PEXP_ERR_INVALID_ARG;
    if (o->wr_max_iter < 1 || !(o->wr_tol > 0) || o->wr_diverge < 0) return PEXP_ERR_INVALID_ARG;
    if (o->jacobian != 0 && o->jacobian != 1) return PEXP_ERR_INVALID_ARG;
    int v = validate(op, o);
    if (v) return v;
    // the source samples of waveform relaxation are the iterate's, at the output times
    if (o->nodes != PEXP_NODES_UNIFORM) return PEXP_ERR_UNSUPPORTED;
    // the averaged Jacobian: conservative form, shift-and-invert space, iterates in the
    // solver's own precision
    if (o->jacobian && (o->burgers_form != 0 || o->krylov != PEXP_KRYLOV_SAI ||
                        (dtype == PEXP_F64) != (o->precision == PEXP_FP64)))
        return PEXP_ERR_UNSUPPORTED;
    if (rep) memset(rep, 0, sizeof(*rep));
    cudaSetDevice(c->device);
    const OpDesc od = make_opdesc(*op);
    const int64_t n = od.n;
    const int nt = o->n_out;
    const size_t es = dtype == PEXP_F64 ? 8 : 4;
    const double inv2dx = 1.0 / (2.0 * (op->bc == PEXP_BC_PERIODIC ? op->Lx / n : op->Lx / (n + 1)));
    c->launches = 0;
    cudaEventRecord(c->ev0, c->stream);
    int status = guarded([&]() -> int {
        const bool fp64 = o->precision == PEXP_FP64;
        const int P = o->P;
        Partition pt = make_partition(nt, P);
        const int wrows = nt + P - 1;   // window-major source rows (boundary samples twice)
        const bool jac = o->jacobian != 0;
        // live WR buffers at the bottom of the workspace: previous iterate, source, norms, and for
        // the averaged Jacobian the window states, the factors and the window-major source
        size_t keep = align_up(es * n * nt) * 2 + align_up(sizeof(double) * 2 * nt) + kAlign;
        if (jac)
            keep += align_up(sizeof(double) * n) + align_up(sizeof(double) * (size_t)P * n) + align_up(es * (size_t)P * n) +
                    align_up(sizeof(double) * 3 * (size_t)P * n) + align_up(es * (size_t)wrows * n) +
                    align_up(sizeof(int) * (P + 1)) + 2 * align_up(sizeof(int) * wrows) + align_up(8 * (size_t)P) +
                    align_up(sizeof(int) * P) + align_up(sizeof(VarOpTask) * P) + 16 * kAlign;
        const int b_cap = std::min(std::min(o->max_rank, PEXP_MAX_RANK), pt.smax);
        const int g_conv = jac ? 0 : ((dtype == PEXP_F64) != fp64);
        size_t need = keep + align_up(sizeof(double) * n) +
                      (fp64 ? linear_workspace_bytes<double>(n, o, g_conv, b_cap)
                            : linear_workspace_bytes<float>(n, o, g_conv, b_cap));
        int r = ws_reserve(c, need);
        if (r) return r;
        c->ws_top = 0;
        char* Uprev = reinterpret_cast<char*>(ws_alloc(c, es * n * nt));
        char* Gk = reinterpret_cast<char*>(ws_alloc(c, es * n * nt));
        double* norms = as<double>(ws_alloc(c, sizeof(double) * 2 * nt));
        // averaged-Jacobian buffers and the fixed per-window operator descriptors
        WinOps<double> wo64;
        WinOps<float> wo32;
        double *Au0 = nullptr, *ubar64 = nullptr, *fac = nullptr;
        char *ubarT = nullptr, *Gwin = nullptr;
        int *idx_d = nullptr, *rw_d = nullptr, *ri_d = nullptr, *flags = nullptr;
        unsigned long long* umax_bits = nullptr;
        VarOpTask* vtasks = nullptr;
        const double gamma = o->sai_gamma * o->T / (double)P;
        if (jac) {
            Au0 = as<double>(ws_alloc(c, sizeof(double) * n));
            ubar64 = as<double>(ws_alloc(c, sizeof(double) * (size_t)P * n));
            ubarT = reinterpret_cast<char*>(ws_alloc(c, es * (size_t)P * n));
            fac = as<double>(ws_alloc(c, sizeof(double) * 3 * (size_t)P * n));
            Gwin = reinterpret_cast<char*>(ws_alloc(c, es * (size_t)wrows * n));
            idx_d = as<int>(ws_alloc(c, sizeof(int) * (P + 1)));
            rw_d = as<int>(ws_alloc(c, sizeof(int) * wrows));
            ri_d = as<int>(ws_alloc(c, sizeof(int) * wrows));
            umax_bits = reinterpret_cast<unsigned long long*>(ws_alloc(c, 8 * (size_t)P));
            flags = as<int>(ws_alloc(c, sizeof(int) * P));
            vtasks = reinterpret_cast<VarOpTask*>(ws_alloc(c, sizeof(VarOpTask) * P));
            std::vector<int> rw, ri;
            for (int j = 0; j < P; ++j)
                for (int i = pt.idx[j]; i <= pt.idx[j + 1]; ++i) {
                    rw.push_back(j);
                    ri.push_back(i);
                }
            std::vector<VarOpTask> vt(P);
            for (int j = 0; j < P; ++j) {
                double* f = fac + 3 * (size_t)j * n;
                vt[j] = VarOpTask{ubar64 + (size_t)j * n, f, f + n, f + 2 * n, flags + j};
                const VarSai vs{f, f + n, f + 2 * n};
                wo64.vs.push_back(vs);
                wo32.vs.push_back(vs);
                wo64.ubar.push_back(reinterpret_cast<const double*>(ubarT) + (size_t)j * n);
                wo32.ubar.push_back(reinterpret_cast<const float*>(ubarT) + (size_t)j * n);
                wo64.ubar64.push_back(ubar64 + (size_t)j * n);
                wo32.ubar64.push_back(ubar64 + (size_t)j * n);
            }
            wo64.var = wo32.var = true;
            wo64.jac = wo32.jac = true;
            wo64.inv2dx = wo32.inv2dx = inv2dx;
            wo64.Gwin = reinterpret_cast<const double*>(Gwin);
            wo32.Gwin = reinterpret_cast<const float*>(Gwin);
            PEXP_CUDA_TRY(cudaMemcpyAsync(idx_d, pt.idx.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice, c->stream));
            PEXP_CUDA_TRY(cudaMemcpyAsync(rw_d, rw.data(), sizeof(int) * wrows, cudaMemcpyHostToDevice, c->stream));
            PEXP_CUDA_TRY(cudaMemcpyAsync(ri_d, ri.data(), sizeof(int) * wrows, cudaMemcpyHostToDevice, c->stream));
            PEXP_CUDA_TRY(cudaMemcpyAsync(vtasks, vt.data(), sizeof(VarOpTask) * P, cudaMemcpyHostToDevice, c->stream));
            launch_stencil<double>(od, reinterpret_cast<const double*>(u0_dev), Au0, 1, 0, c->stream);
            check_launch(c);
            sync(c);   // the host vectors above go out of scope
        }
        const size_t top = c->ws_top;
        // first iterate
        if (init_dev) {
            cudaMemcpyAsync(Uprev, init_dev, es * n * nt, cudaMemcpyDeviceToDevice, c->stream);
        } else {
            for (int i = 0; i < nt; ++i) {
                if (dtype == PEXP_F64)
                    cudaMemcpyAsync(Uprev + es * n * i, u0_dev, es * n, cudaMemcpyDeviceToDevice, c->stream);
                else
                    launch_convert<double, float>(reinterpret_cast<const double*>(u0_dev), as<float>(Uprev + es * n * i), n, c->stream);
            }
        }
        std::vector<double> nh(2 * nt);
        int status_l = PEXP_ERR_WR_NOT_CONVERGED;
        double delta = 0;
        int it = 0, grew = 0;
        pexp_report lrep;
        for (it = 1; it <= o->wr_max_iter; ++it) {
            if (dtype == PEXP_F64) launch_burgers_source<double>(od, as<double>(Uprev), as<double>(Gk), nt, o->burgers_form, inv2dx, c->stream);
            else launch_burgers_source<float>(od, as<float>(Uprev), as<float>(Gk), nt, o->burgers_form, inv2dx, c->stream);
            check_launch(c);
            if (forcing_dev) {
                if (dtype == PEXP_F64) launch_add<double>(as<double>(Gk), reinterpret_cast<const double*>(forcing_dev), n * nt, c->stream);
                else launch_add<float>(as<float>(Gk), reinterpret_cast<const float*>(forcing_dev), n * nt, c->stream);
                check_launch(c);
            }
            int lr;
            if (jac) {
                // J_{k,j} at the trapezoidal time mean of the iterate over subinterval j (eq.
                // piecewiseJac); the factors of I - gamma (A + J_{k,j}); the shifted source
                // A u0 + g_k - J_{k,j} (u_k - u0) of every subinterval (eq. sourceParallel)
                PEXP_CUDA_TRY(cudaMemsetAsync(umax_bits, 0, 8 * (size_t)P, c->stream));
                PEXP_CUDA_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * P, c->stream));
                if (dtype == PEXP_F64)
                    launch_window_average<double>(as<double>(Uprev), n, idx_d, P, ubar64, as<double>(ubarT), umax_bits, c->stream);
                else
                    launch_window_average<float>(as<float>(Uprev), n, idx_d, P, ubar64, as<float>(ubarT), umax_bits, c->stream);
                check_launch(c);
                std::vector<unsigned long long> ub(P);
                d2h(c, ub.data(), umax_bits, 8 * (size_t)P);
                double umax = 0.0;
                for (int j = 0; j < P; ++j) {
                    double x;
                    memcpy(&x, &ub[j], sizeof(double));
                    umax = std::max(umax, x);
                }
                launch_vsai_factor(od.x, gamma, inv2dx, vtasks, P, vsai_warmup(od.x, gamma, inv2dx, umax), c->stream);
                check_launch(c);
                if (dtype == PEXP_F64)
                    launch_jac_source<double>(od.x, inv2dx, Au0, reinterpret_cast<const double*>(u0_dev), as<double>(Gk),
                                              as<double>(Uprev), ubar64, rw_d, ri_d, wrows, as<double>(Gwin), c->stream);
                else
                    launch_jac_source<float>(od.x, inv2dx, Au0, reinterpret_cast<const double*>(u0_dev), as<float>(Gk),
                                             as<float>(Uprev), ubar64, rw_d, ri_d, wrows, as<float>(Gwin), c->stream);
                check_launch(c);
                std::vector<int> fl(P);
                d2h(c, fl.data(), flags, sizeof(int) * P);
                for (int j = 0; j < P; ++j)
                    if (fl[j]) return PEXP_ERR_UNSUPPORTED;   // I - gamma (A + J) not diagonally dominant
                lr = solve_linear_dispatch(c, op, o, u0_dev, nullptr, dtype, U_dev, dtype, &lrep, top, &wo64, &wo32);
            } else {
                lr = solve_linear_dispatch(c, op, o, u0_dev, Gk, dtype, U_dev, dtype, &lrep, top);
            }
            if (lr != PEXP_OK && lr != PEXP_ERR_NOT_CONVERGED) return lr;
            if (dtype == PEXP_F64) launch_row_diff_norms<double>(as<double>(U_dev), as<double>(Uprev), n, nt, norms, c->stream);
            else launch_row_diff_norms<float>(as<float>(U_dev), as<float>(Uprev), n, nt, norms, c->stream);
            check_launch(c);
            d2h(c, nh.data(), norms, sizeof(double) * 2 * nt);
            double dmax = 0, umax = 0;
            for (int i = 0; i < nt; ++i) {
                dmax = std::max(dmax, sqrt(nh[i]));
                umax = std::max(umax, sqrt(nh[nt + i]));
            }
            const double prev_delta = delta;
            delta = umax > 0 ? dmax / umax : 0.0;
            if (rep) {
                rep->k_nh_max = std::max(rep->k_nh_max, lrep.k_nh_max);
                rep->k_hom_max = std::max(rep->k_hom_max, lrep.k_hom_max);
                rep->rank_max = std::max(rep->rank_max, lrep.rank_max);
                rep->not_converged += lrep.not_converged;
                rep->bytes_alg += lrep.bytes_alg + 3.0 * es * n * nt;
                if (it <= PEXP_REPORT_WR) rep->wr_history[it - 1] = delta;
                memcpy(rep->sub_rank, lrep.sub_rank, sizeof(rep->sub_rank));
                memcpy(rep->sub_steps, lrep.sub_steps, sizeof(rep->sub_steps));
                memcpy(rep->sub_hom_steps, lrep.sub_hom_steps, sizeof(rep->sub_hom_steps));
                memcpy(rep->sub_restarts, lrep.sub_restarts, sizeof(rep->sub_restarts));
            }
            if (delta <= o->wr_tol) { status_l = PEXP_OK; break; }
            // divergence: the update grew in wr_diverge successive iterations
            grew = (it >= 2 && delta > prev_delta) ? grew + 1 : 0;
            if (o->wr_diverge > 0 && grew >= o->wr_diverge) { status_l = PEXP_ERR_WR_DIVERGED; break; }
            cudaMemcpyAsync(Uprev, U_dev, es * n * nt, cudaMemcpyDeviceToDevice, c->stream);
        }
        if (rep) {
            rep->wr_iters = std::min(it, o->wr_max_iter);
            rep->wr_delta = delta;
            rep->n_sub = o->P;
        }
        return status_l;
    });
    cudaEventRecord(c->ev1, c->stream);
    cudaEventSynchronize(c->ev1);
    if (rep) {
        float ms = 0;
        cudaEventElapsedTime(&ms, c->ev0, c->ev1);
        rep->time_ms = ms;
        rep->launches = c->launches;
        rep->status = status;
    }
    return status;
}

int pexp_apply_operator(pexp_ctx* c, const pexp_operator* op, const void* X, void* Y, int nvec, int dtype,
                        int transpose) {
    if (!c || !op || !X || !Y || nvec < 1) return PEXP_ERR_INVALID_ARG;
    if (op->dim != 1 && op->dim != 2) return PEXP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    const OpDesc od = make_opdesc(*op);
    if (dtype == PEXP_F64) launch_stencil<double>(od, as<double>(const_cast<void*>(X)), as<double>(Y), nvec, transpose, c->stream);
    else if (dtype == PEXP_F32) launch_stencil<float>(od, as<float>(const_cast<void*>(X)), as<float>(Y), nvec, transpose, c->stream);
    else return PEXP_ERR_INVALID_ARG;
    PEXP_CUDA_TRY(cudaGetLastError());
    PEXP_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return PEXP_OK;
}

int pexp_jacobian_sai_solve(pexp_ctx* c, const pexp_operator* op, double gamma, const double* ubar, const void* X,
                            void* Y, int nvec, int dtype) {
    if (!c || !op || !X || !Y || nvec < 1 || !(gamma > 0)) return PEXP_ERR_INVALID_ARG;
    if (op->dim != 1) return PEXP_ERR_UNSUPPORTED;
    if (op->nx < 3 || !(op->Lx > 0.0) || !(op->nu >= 0.0)) return PEXP_ERR_INVALID_ARG;
    if (dtype != PEXP_F64 && dtype != PEXP_F32) return PEXP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    const OpDesc od = make_opdesc(*op);
    const int64_t n = od.n;
    const double inv2dx = 1.0 / (2.0 * (op->bc == PEXP_BC_PERIODIC ? op->Lx / n : op->Lx / (n + 1)));
    return guarded([&]() -> int {
        const size_t es = dtype == PEXP_F64 ? 8 : 4;
        size_t need = align_up(sizeof(double) * (sai_scratch_doubles(n, nvec) + 64)) + align_up(sizeof(double) * 3 * n) +
                      align_up(sizeof(double) * (n + 64)) + 4 * kAlign;
        int r = ws_reserve(c, need);
        if (r) return r;
        c->ws_top = 0;
        double* scr = as<double>(ws_alloc(c, sizeof(double) * (sai_scratch_doubles(n, nvec) + 64)));
        double* fac = as<double>(ws_alloc(c, sizeof(double) * 3 * n));
        int* flag = as<int>(ws_alloc(c, sizeof(int) * 4));
        PEXP_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), c->stream));
        double umax = 0.0;
        if (ubar) {
            // max |ubar| for the warm-up length of the factorisation
            std::vector<double> hu(n);
            PEXP_CUDA_TRY(cudaMemcpyAsync(hu.data(), ubar, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
            sync(c);
            for (double x : hu) umax = std::max(umax, fabs(x));
        }
        Stage sg(c, 0);
        VarOpTask vt{ubar, fac, fac + n, fac + 2 * n, flag};
        const VarOpTask* dvt = sg.put(&vt, 1);
        std::vector<const void*> xs(nvec);
        std::vector<void*> ys(nvec);
        std::vector<VarSai> vcs(nvec, VarSai{fac, fac + n, fac + 2 * n});
        for (int v = 0; v < nvec; ++v) {
            xs[v] = reinterpret_cast<const char*>(X) + es * n * v;
            ys[v] = reinterpret_cast<char*>(Y) + es * n * v;
        }
        const void* const* dx = sg.put(xs.data(), nvec);
        void* const* dy = sg.put(ys.data(), nvec);
        const VarSai* dv = sg.put(vcs.data(), nvec);
        sg.flush();
        launch_vsai_factor(od.x, gamma, inv2dx, dvt, 1, vsai_warmup(od.x, gamma, inv2dx, umax), c->stream);
        check_launch(c);
        int fl = 0;
        d2h(c, &fl, flag, sizeof(int));
        if (fl) return PEXP_ERR_UNSUPPORTED;
        if (dtype == PEXP_F64)
            launch_vsai_solve<double>(n, dv, reinterpret_cast<const double* const*>(dx), nullptr,
                                      reinterpret_cast<double* const*>(dy), nullptr, nvec, scr, c->stream);
        else
            launch_vsai_solve<float>(n, dv, reinterpret_cast<const float* const*>(dx), nullptr,
                                     reinterpret_cast<float* const*>(dy), nullptr, nvec, scr, c->stream);
        check_launch(c);
        c->launches += 2;
        sync(c);
        return PEXP_OK;
    });
}

int pexp_sai_solve(pexp_ctx* c, const pexp_operator* op, double gamma, const void* X, void* Y, int nvec,
                   int dtype) {
    if (!c || !op || !X || !Y || nvec < 1 || !(gamma > 0)) return PEXP_ERR_INVALID_ARG;
    if (op->dim != 1) return PEXP_ERR_UNSUPPORTED;
    if (op->bc != PEXP_BC_PERIODIC) return pexp_jacobian_sai_solve(c, op, gamma, nullptr, X, Y, nvec, dtype);
    if (dtype != PEXP_F64 && dtype != PEXP_F32) return PEXP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    const OpDesc od = make_opdesc(*op);
    const int64_t n = od.n;
    return guarded([&]() -> int {
        const size_t es = dtype == PEXP_F64 ? 8 : 4;
        size_t need = align_up(sizeof(double) * (sai_scratch_doubles(n, nvec) + 64)) + 2 * kAlign;
        int r = ws_reserve(c, need);
        if (r) return r;
        c->ws_top = 0;
        double* scr = as<double>(ws_alloc(c, sizeof(double) * (sai_scratch_doubles(n, nvec) + 64)));
        Stage sg(c, 0);
        std::vector<const void*> xs(nvec);
        std::vector<void*> ys(nvec);
        for (int v = 0; v < nvec; ++v) {
            xs[v] = reinterpret_cast<const char*>(X) + es * n * v;
            ys[v] = reinterpret_cast<char*>(Y) + es * n * v;
        }
        const void* const* dx = sg.put(xs.data(), nvec);
        void* const* dy = sg.put(ys.data(), nvec);
        sg.flush();
        const SaiCoef cf = sai_coefficients(od, gamma);
        if (dtype == PEXP_F64)
            launch_sai_solve<double>(od, cf, reinterpret_cast<const double* const*>(dx), reinterpret_cast<double* const*>(dy), nullptr, nvec, scr, c->stream);
        else
            launch_sai_solve<float>(od, cf, reinterpret_cast<const float* const*>(dx), reinterpret_cast<float* const*>(dy), nullptr, nvec, scr, c->stream);
        check_launch(c);
        sync(c);
        return PEXP_OK;
    });
}

int pexp_small_expm(pexp_ctx* c, const double* M, double* E, int N, int batch) {
    if (!c || !M || !E || N < 1 || N > 128 || batch < 1) return PEXP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    return guarded([&]() -> int {
        size_t need = align_up(sizeof(double) * small_expm_scratch_doubles(N) * batch) + kAlign;
        int r = ws_reserve(c, need);
        if (r) return r;
        c->ws_top = 0;
        double* scr = as<double>(ws_alloc(c, sizeof(double) * small_expm_scratch_doubles(N) * batch));
        launch_small_expm_batch(M, E, N, batch, scr, c->stream);
        check_launch(c);
        sync(c);
        return PEXP_OK;
    });
}

int pexp_burgers_source(pexp_ctx* c, const pexp_operator* op, const void* U, void* G, int n_rows, int dtype,
                        int form) {
    if (!c || !op || !U || !G || n_rows < 1 || op->dim != 1) return PEXP_ERR_INVALID_ARG;
    cudaSetDevice(c->device);
    const OpDesc od = make_opdesc(*op);
    const int64_t n = od.n;
    const double inv2dx = 1.0 / (2.0 * (op->bc == PEXP_BC_PERIODIC ? op->Lx / n : op->Lx / (n + 1)));
    if (dtype == PEXP_F64) launch_burgers_source<double>(od, as<double>(const_cast<void*>(U)), as<double>(G), n_rows, form, inv2dx, c->stream);
    else if (dtype == PEXP_F32) launch_burgers_source<float>(od, as<float>(const_cast<void*>(U)), as<float>(G), n_rows, form, inv2dx, c->stream);
    else return PEXP_ERR_INVALID_ARG;
    PEXP_CUDA_TRY(cudaGetLastError());
    PEXP_CUDA_TRY(cudaStreamSynchronize(c->stream));
    return PEXP_OK;
}

}  // extern "C"
