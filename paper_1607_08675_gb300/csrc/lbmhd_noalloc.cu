// lbmhd_noalloc.cu -- diagnostics of a caller-owned state buffer without
// any device allocation.
//
// Some callers cannot call cudaMalloc: a host application that hands out
// all device memory from its own arena and forbids allocation after
// start-up, or a latency-critical loop that cannot afford the implicit
// device synchronisation of cudaMalloc / cudaFree.  For them the FP64
// diagnostics reduction runs here with its per-block partial sums in a
// fixed, file-scope device array instead of memory from lbmhd_create.
#include <stdint.h>

#include <mutex>

#include "lbmhd_internal.h"

namespace lbmhd {

// Room for the partial rows of the largest diagnostics grid: the reduction
// launches at most 1024 blocks (whatever the lattice size), 12 FP64 sums
// each, so 1024 * 12 doubles = 96 KiB.  Every GPU that loads the library
// holds this array until the process exits.
constexpr int kNoAllocRows = 1024;
constexpr int kNoAllocCols = 12;
static __device__ __align__(256) double g_noalloc_partials[kNoAllocRows * kNoAllocCols];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_addr[kMaxDevices] = {};

// The name g_noalloc_partials in host code is only a stand-in for the
// symbol; the device address must be looked up once per device, with that
// device current.
int scratch_for_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error(std::string("cudaGetDevice: ") + cudaGetErrorString(e));
        return LBMHD_ECUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal beyond the 64 devices this entry point supports");
        return LBMHD_EINVAL;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess || !p) {
            set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            return LBMHD_ECUDA;
        }
        g_addr[dev] = (double*)p;
    }
    *out = g_addr[dev];
    return LBMHD_OK;
}

}  // namespace
}  // namespace lbmhd

using namespace lbmhd;

extern "C" int lbmhd_diagnostics_noalloc(const void* state, int precision, int nx, int ny,
                                         long long plane_stride, double fp16_scale, double* out,
                                         void* stream) {
    if (!state || !out) {
        set_error("state and out must be device pointers");
        return LBMHD_EINVAL;
    }
    if (storage_bytes(precision) == 0) {
        set_error("unknown precision");
        return LBMHD_EINVAL;
    }
    // A pointer carved out of a caller's arena may sit anywhere; the kernel
    // reads whole stored values and writes FP64 sums, so misalignment is
    // refused here, before anything reaches the GPU.
    if ((uintptr_t)state % storage_bytes(precision) != 0) {
        set_error("state must be aligned to the stored value size (8 B FP64 / FF, 4 B FP32, "
                  "2 B FP16)");
        return LBMHD_EINVAL;
    }
    if ((uintptr_t)out % sizeof(double) != 0) {
        set_error("out must be 8-byte aligned");
        return LBMHD_EINVAL;
    }
    if (nx < 1 || ny < 1 || (long long)nx * ny > (1LL << 30)) {
        set_error("nx, ny must be >= 1 with nx*ny <= 2^30 nodes");
        return LBMHD_EINVAL;
    }
    if (precision == LBMHD_FP16_DEV && !(fp16_scale > 0.0 && fp16_scale < 1e30)) {
        set_error("fp16_scale must be positive and finite");
        return LBMHD_EINVAL;
    }
    if (plane_stride < (long long)nx * ny) {
        set_error("plane_stride must be at least nx*ny elements");
        return LBMHD_EINVAL;
    }
    Geom g;
    g.nx = nx;
    g.ny = ny;
    g.ps = plane_stride;
    if (diag_num_blocks(g, precision) > kNoAllocRows) {
        set_error("diagnostics grid exceeds the 1024 partial rows of the static scratch");
        return LBMHD_EINVAL;
    }
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc) return rc;
    HostColl c = {};
    c.scale = 1.0f;
    c.inv_scale = 1.0f;
    if (precision == LBMHD_FP16_DEV) {
        c.scale = (float)fp16_scale;
        c.inv_scale = (float)(1.0 / fp16_scale);
    }
    // Every row the final pass reads is written by the same call, so nothing
    // in the scratch has to start at zero.
    cudaError_t e = launch_diag(precision, state, scratch, out, g, c, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        set_error(std::string("diagnostics launch: ") + cudaGetErrorString(e));
        return LBMHD_ECUDA;
    }
    return LBMHD_OK;
}
