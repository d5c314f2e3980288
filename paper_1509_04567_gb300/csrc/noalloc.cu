// pexp_sai_solve_noalloc: the shift-and-invert solve of pexp_sai_solve for callers
// that cannot allocate device memory (a fixed budget already reserved by another
// allocator, or streams that must not stall on cudaMalloc/cudaFree).  The scratch is
// a file-scope device array; its device address is looked up once per device.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "common.cuh"

using namespace pexp;

namespace {

constexpr size_t kScratchDoubles = PEXP_NOALLOC_SCRATCH_BYTES / sizeof(double);
constexpr int kMaxDevices = 64;

// The scratch: one file-scope device array, one copy on every device that loads this
// module.  Device code may name it directly; host code may not pass the name to a kernel
// (on the host it denotes a host-side shadow, not a device address), so its device
// address is looked up with cudaGetSymbolAddress, once per device.
static __device__ __align__(256) double g_sai_scratch[kScratchDoubles];

std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device `dev`; NULL on failure.
double* scratch_for(int dev) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        double* ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_sai_scratch);
        if (e != cudaSuccess || !ptr) {
            fprintf(stderr, "pexp_sai_solve_noalloc: cudaGetSymbolAddress failed on device %d: %s\n", dev,
                    cudaGetErrorString(e));
            return nullptr;
        }
        g_scratch_ptr[dev] = ptr;
    }
    return g_scratch_ptr[dev];
}

// Pointer tables of the nvec vectors, written into the scratch on the device.
__global__ void k_vector_tables(const char* X, char* Y, int64_t vec_bytes, int nvec, const void** xp, void** yp) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < nvec) {
        xp[v] = X + (int64_t)v * vec_bytes;
        yp[v] = Y + (int64_t)v * vec_bytes;
    }
}

}  // namespace

extern "C" int pexp_sai_solve_noalloc(const pexp_operator* op, double gamma, const void* X_dev, void* Y_dev,
                                      int nvec, int dtype, void* cuda_stream) {
    if (!op || !X_dev || !Y_dev || nvec < 1 || !(gamma > 0) || !isfinite(gamma)) return PEXP_ERR_INVALID_ARG;
    if (dtype != PEXP_F64 && dtype != PEXP_F32) return PEXP_ERR_INVALID_ARG;
    if (op->dim != 1 || op->bc != PEXP_BC_PERIODIC) return PEXP_ERR_UNSUPPORTED;
    if (op->nx < 3 || !(op->Lx > 0) || !(op->nu >= 0) || !isfinite(op->nu) || !isfinite(op->ax) || !isfinite(op->Lx))
        return PEXP_ERR_INVALID_ARG;
    const int64_t n = op->nx;
    // pointer tables (2 nvec slots) + forward/backward chunk ends and decays
    if (n > (int64_t)1 << 40 || (double)nvec * 2.0 + (double)sai_scratch_doubles(n, 1) * nvec > (double)kScratchDoubles)
        return PEXP_ERR_SCRATCH_LIMIT;
    const size_t es = dtype == PEXP_F64 ? sizeof(double) : sizeof(float);
    const char* xb = static_cast<const char*>(X_dev);
    const char* yb = static_cast<const char*>(Y_dev);
    const size_t bytes = es * (size_t)n * (size_t)nvec;
    if (xb < yb + bytes && yb < xb + bytes) return PEXP_ERR_INVALID_ARG;

    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PEXP_ERR_CUDA;
    double* scr = scratch_for(dev);
    if (!scr) return PEXP_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);

    const void** xp = reinterpret_cast<const void**>(scr);
    void** yp = reinterpret_cast<void**>(scr + nvec);
    double* summaries = scr + 2 * (size_t)nvec;

    OpDesc od;
    memset(&od, 0, sizeof(od));
    od.dim = 1;
    od.n = n;
    const double dx = op->Lx / (double)n;
    od.x.n = n;
    od.x.stride = 1;
    od.x.d = op->nu / (dx * dx);
    od.x.c = op->ax / (2.0 * dx);
    od.x.periodic = 1;
    const SaiCoef cf = sai_coefficients(od, gamma);

    k_vector_tables<<<(nvec + 127) / 128, 128, 0, s>>>(xb, const_cast<char*>(yb), (int64_t)(es * n), nvec, xp, yp);
    if (dtype == PEXP_F64)
        launch_sai_solve<double>(od, cf, reinterpret_cast<const double* const*>(xp),
                                 reinterpret_cast<double* const*>(yp), nullptr, nvec, summaries, s);
    else
        launch_sai_solve<float>(od, cf, reinterpret_cast<const float* const*>(xp),
                                reinterpret_cast<float* const*>(yp), nullptr, nvec, summaries, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "pexp_sai_solve_noalloc: kernel launch failed: %s\n", cudaGetErrorString(e));
        return PEXP_ERR_CUDA;
    }
    return PEXP_OK;
}
