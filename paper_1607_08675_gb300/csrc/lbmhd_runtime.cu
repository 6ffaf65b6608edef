// lbmhd_runtime.cu -- the C ABI of include/lbmhd.h: handle lifetime,
// parameter validation, buffers, stream-ordered transfers, CUDA-graph
// replay of long step sequences, error reporting.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "lbmhd_internal.h"

namespace lbmhd {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

size_t storage_bytes(int prec) {
    switch (prec) {
        case LBMHD_FP64:
        case LBMHD_FF: return 8;
        case LBMHD_FP32:
        case LBMHD_FP32_DEV: return 4;
        case LBMHD_FP16_DEV: return 2;
    }
    return 0;
}

// Plane strides are a multiple of 64 elements (at least 128 bytes), so
// every row segment a warp loads is vector aligned whenever nx is a
// multiple of the vector width.
long long plane_stride(int nx, int ny) {
    const long long n = (long long)nx * ny;
    return (n + 63) / 64 * 64;
}

}  // namespace lbmhd

using namespace lbmhd;

namespace {

constexpr int kGraphSteps = 64;  // even: a replay leaves the buffer parity unchanged

int fail(int code, const std::string& msg) {
    set_error(msg);
    return code;
}

int cuda_fail(lbmhd_t* h, cudaError_t e, const char* where) {
    if (h) h->failed = true;
    cudaGetLastError();  // clear a sticky launch error where possible
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return LBMHD_ECUDA;
}

#define LBMHD_CK(h, call)                                    \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
    } while (0)

bool is_finite(double v) { return std::isfinite(v); }

}  // namespace

int lbmhd::validate_params(int nx, int ny, const lbmhd_params* p) {
    if (!p) return fail(LBMHD_EINVAL, "params is NULL");
    if (p->abi_version != LBMHD_ABI_VERSION)
        return fail(LBMHD_EVERSION, "params.abi_version does not match LBMHD_ABI_VERSION");
    if (nx < 1 || ny < 1) return fail(LBMHD_EINVAL, "nx and ny must be >= 1");
    if ((long long)nx * ny > (1LL << 30)) return fail(LBMHD_EINVAL, "nx*ny exceeds 2^30 nodes");
    if (storage_bytes(p->precision) == 0) return fail(LBMHD_EINVAL, "unknown precision");
    const double v[] = {p->tau_nu, p->tau_eta, p->C_S, p->delta, p->s5, p->s6, p->s7, p->s8,
                        p->fp16_scale};
    for (double x : v)
        if (!is_finite(x)) return fail(LBMHD_EINVAL, "non-finite parameter");
    if (!(p->tau_nu > 0.5) || !(p->tau_eta > 0.5))
        return fail(LBMHD_EINVAL, "tau_nu and tau_eta must exceed 1/2 (positive nu, eta)");
    if (p->C_S < 0.0) return fail(LBMHD_EINVAL, "C_S must be >= 0");
    if (!(p->delta > 0.0)) return fail(LBMHD_EINVAL, "delta must be > 0");
    for (double s : {p->s5, p->s6, p->s7, p->s8})
        if (s > 0.0 && !(s < 2.0)) return fail(LBMHD_EINVAL, "given rates s5..s8 must lie in (0, 2)");
    if (!(p->fp16_scale > 0.0)) return fail(LBMHD_EINVAL, "fp16_scale must be > 0");
    if (p->les < 0 || p->les > 3) return fail(LBMHD_EINVAL, "les must be 0, 1, 2 or 3");
    if (p->check_finite_every < 0) return fail(LBMHD_EINVAL, "check_finite_every must be >= 0");
    // bulk viscosity (Sec. 4.3) at the base rates
    const double s4 = 1.0 / p->tau_nu;
    const double s7 = p->s7 > 0.0 ? p->s7 : s4, s8 = p->s8 > 0.0 ? p->s8 : s4;
    const double xi = -1.0 / 9.0 - 1.0 / (9.0 * s4) - 1.0 / (15.0 * s7) + 2.0 / (5.0 * s8);
    if (!(xi > 0.0)) return fail(LBMHD_EINVAL, "s7, s8 give a non-positive bulk viscosity");
    return LBMHD_OK;
}

namespace {

HostColl make_coll(const lbmhd_params* p) {
    HostColl c;
    c.tn = p->tau_nu;
    c.te = p->tau_eta;
    const double cd2 = p->C_S * p->delta * p->delta;
    c.k18 = 18.0 * cd2;
    c.k36 = 36.0 * cd2;
    c.s5 = p->s5 > 0.0 ? p->s5 : 1.0 / p->tau_nu;
    c.s6 = p->s6 > 0.0 ? p->s6 : 1.0 / p->tau_nu;
    c.tie5 = p->s5 > 0.0 ? 0 : 1;
    c.tie6 = p->s6 > 0.0 ? 0 : 1;
    c.s7 = p->s7 > 0.0 ? p->s7 : 0.0;
    c.s8 = p->s8 > 0.0 ? p->s8 : 0.0;
    c.les = p->les == 1 ? 1 : 0;
    c.kin = p->les >= 2 ? p->les : 0;  // 2: filtered equilibria, 3: cross-helicity
    c.d2 = p->delta * p->delta;
    c.scale = (float)p->fp16_scale;
    c.inv_scale = (float)(1.0 / p->fp16_scale);
    return c;
}

int check_handle(lbmhd_t* h) {
    if (!h) return fail(LBMHD_EINVAL, "handle is NULL");
    if (h->failed) return fail(LBMHD_ECUDA, "handle is unusable after a CUDA error");
    return LBMHD_OK;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

long long ncell(const lbmhd_t* h) { return (long long)h->geom.nx * h->geom.ny; }

int read_flag(lbmhd_t* h) {
    int flag = 0;
    LBMHD_CK(h, cudaMemcpyAsync(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LBMHD_CK(h, cudaStreamSynchronize(h->stream));
    if (flag & 2) return fail(LBMHD_ETIMEOUT, "a bounded device wait expired in the step kernel");
    if (flag & 1) return fail(LBMHD_ENONFINITE, "non-finite density detected");
    return LBMHD_OK;
}

cudaError_t launch_one(lbmhd_t* h, const void* src, void* dst) {
    if (h->coll.kin)
        return launch_step_kinetic(h->p.precision, h->kin_two_pass != 0, h->sm_count, src, dst,
                                   h->d_kin, h->geom, h->coll, h->stream);
    if (h->tma_w > 0)
        return launch_step_tma(h->p.precision, h->tma_w, h->sm_count, src, dst, h->geom, h->coll,
                               h->d_flag, h->stream);
    return launch_step(h->p.precision, h->vec, h->block, 0, src, dst, h->geom, h->coll, h->stream);
}

cudaError_t one_step(lbmhd_t* h) {
    cudaError_t e = launch_one(h, h->buf[h->cur], h->buf[1 - h->cur]);
    if (e == cudaSuccess) {
        h->cur = 1 - h->cur;
        h->launches += h->coll.kin && h->kin_two_pass ? 2 : 1;
    }
    return e;
}

}  // namespace

extern "C" {

void lbmhd_params_default(lbmhd_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->abi_version = LBMHD_ABI_VERSION;
    p->precision = LBMHD_FP64;
    p->tau_nu = 0.6;
    p->tau_eta = 0.6;
    p->C_S = 0.1;
    p->delta = 1.0;
    p->les = 1;
    p->check_finite_every = 0;
    p->fp16_scale = 1024.0;
    p->stream = nullptr;
}

int lbmhd_bytes_per_cell(int precision) { return (int)(2 * kNumPlanes * storage_bytes(precision)); }

int lbmhd_create(int nx, int ny, const lbmhd_params* p, lbmhd_t** out) {
    if (!out) return fail(LBMHD_EINVAL, "out is NULL");
    int rc = validate_params(nx, ny, p);
    if (rc) return rc;
    lbmhd_t* h = new (std::nothrow) lbmhd_t();
    if (!h) return fail(LBMHD_ENOMEM, "host allocation failed");
    std::memset((void*)h, 0, sizeof(*h));
    h->p = *p;
    h->geom.nx = nx;
    h->geom.ny = ny;
    h->geom.ps = plane_stride(nx, ny);
    h->coll = make_coll(p);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(nullptr, e, "cudaGetDevice");
    }
    if (p->stream) {
        h->stream = (cudaStream_t)p->stream;
        h->own_stream = false;
        // the legacy and per-thread default streams cannot be captured
        h->capturable = p->stream != (void*)cudaStreamLegacy &&
                        p->stream != (void*)cudaStreamPerThread;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return cuda_fail(nullptr, e, "cudaStreamCreateWithFlags");
        }
        h->own_stream = true;
        h->capturable = true;
    }
    const size_t bytes = (size_t)kNumPlanes * h->geom.ps * storage_bytes(p->precision);
    const size_t pbytes = (size_t)diag_num_blocks(h->geom, p->precision) * 12 * sizeof(double);
    void* mem[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    const size_t sizes[5] = {bytes, bytes, pbytes, 12 * sizeof(double), sizeof(int)};
    for (int i = 0; i < 5; ++i) {
        e = cudaMalloc(&mem[i], sizes[i]);
        if (e != cudaSuccess) {
            for (int j = 0; j < i; ++j) cudaFree(mem[j]);
            if (h->own_stream) cudaStreamDestroy(h->stream);
            delete h;
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? LBMHD_ENOMEM : LBMHD_ECUDA,
                        std::string("device allocation failed: ") + cudaGetErrorString(e));
        }
    }
    h->buf[0] = mem[0];
    h->buf[1] = mem[1];
    if (p->les >= 2) {
        const size_t kb = (size_t)5 * h->geom.ps *
                          (p->precision == LBMHD_FP64 || p->precision == LBMHD_FF ? 8 : 4);
        e = cudaMalloc(&h->d_kin, kb);
        if (e != cudaSuccess) {
            for (int j = 0; j < 5; ++j) cudaFree(mem[j]);
            if (h->own_stream) cudaStreamDestroy(h->stream);
            delete h;
            cudaGetLastError();
            return fail(LBMHD_ENOMEM, "device allocation failed (filtered-equilibrium moments)");
        }
    }
    h->d_partials = (double*)mem[2];
    h->d_diag = (double*)mem[3];
    h->d_flag = (int*)mem[4];
    cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream);
    // Default launch shape, measured on GB300 at 8192^2: four nodes per
    // thread in 64-thread blocks for FP32 storage (46.0K MLUPS, 1.03x the
    // measured copy bandwidth), eight nodes (16-byte loads) in 32-thread
    // blocks for FP16 storage (82.0K MLUPS, 0.92x), two nodes in 128-thread
    // blocks for FP64 (FP64-pipe bound) and for double-word FF storage;
    // narrower vectors when nx is not a multiple.
    const int want = p->precision == LBMHD_FP64 || p->precision == LBMHD_FF
                         ? 2
                         : (p->precision == LBMHD_FP16_DEV ? 8 : 4);
    h->vec = 1;
    for (int v = want; v > 1; v >>= 1)
        if (nx % v == 0) {
            h->vec = v;
            break;
        }
    h->block = h->vec == 8 ? 32 : (h->vec == 4 ? 64 : (p->precision == LBMHD_FF ? 256 : 128));
    h->tma_w = 0;
    // Kinetic steps: the fused kernel where it is faster (measured at 8192^2
    // / 4096^2, MLUPS fused vs two-pass: FP32 les 2 33.5K vs 23.7K, les 3
    // 37.1K vs 22.3K; FP16 38.9K vs 26.6K; FF les 3 8.2K vs 7.2K), the
    // two-pass kernels where the arithmetic dominates and occupancy wins (FP64
    // les 2 1.36K vs 1.39K, les 3 1.57K vs 1.58K; FF les 2 6.7K vs 7.6K).
    h->kin_two_pass = p->precision == LBMHD_FP64 || (p->precision == LBMHD_FF && p->les == 2);
    if (cudaDeviceGetAttribute(&h->sm_count, cudaDevAttrMultiProcessorCount, h->device) !=
            cudaSuccess ||
        h->sm_count < 1)
        h->sm_count = 1;
    h->cur = 0;
    *out = h;
    return LBMHD_OK;
}

int lbmhd_set_launch(lbmhd_t* h, int vec, int block) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (h->coll.kin) {
        if (vec != 0 && vec != 1)
            return fail(LBMHD_EINVAL, "les 2, 3: vec 1 (fused kernel) or 0 (two-pass kernels)");
        h->kin_two_pass = vec == 0;
    } else if (vec == 0) {
        if (!tma_variant_ok(h->p.precision, block, h->geom.nx))
            return fail(LBMHD_EINVAL,
                        "TMA-staged step: FP32/FP16 storage, tile 128, 256 or 512 dividing nx");
        h->tma_w = block;
    } else {
        if (!step_variant_ok(h->p.precision, vec, h->geom.nx))
            return fail(LBMHD_EINVAL,
                        "vector width must be 1, 2, 4 (or 8 for FP16 storage) and divide nx");
        if (block < 32 || block > 256 || block % 32)
            return fail(LBMHD_EINVAL, "block must be a multiple of 32 in [32, 256]");
        h->vec = vec;
        h->block = block;
        h->tma_w = 0;
    }
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    return LBMHD_OK;
}

int lbmhd_get_launch(const lbmhd_t* h, int* vec, int* block) {
    if (!h || !vec || !block) return fail(LBMHD_EINVAL, "NULL argument");
    if (h->coll.kin) {
        *vec = h->kin_two_pass ? 0 : 1;
        const bool wide = h->p.precision == LBMHD_FP64 || h->p.precision == LBMHD_FF;
        *block = h->kin_two_pass ? 256 : (wide ? 128 : 256) + 32;
        return LBMHD_OK;
    }
    *vec = h->tma_w > 0 ? 0 : h->vec;
    *block = h->tma_w > 0 ? h->tma_w : h->block;
    return LBMHD_OK;
}

int lbmhd_init_device(lbmhd_t* h, const double* rho, const double* ux, const double* uy,
                      const double* bx, const double* by) {
    TraceRange trace_("lbmhd_init_device");
    int rc = check_handle(h);
    if (rc) return rc;
    if (!rho || !ux || !uy || !bx || !by) return fail(LBMHD_EINVAL, "NULL field");
    DeviceGuard dg(h->device);
    LBMHD_CK(h, launch_init(h->p.precision, rho, ux, uy, bx, by, h->buf[h->cur], h->geom, h->coll,
                            h->stream));
    LBMHD_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    h->initialised = true;
    h->steps = 0;
    return LBMHD_OK;
}

// The host arrays of lbmhd_init / lbmhd_moments: when all five are pinned
// host memory the kernels address them in place (over the CPU-GPU link;
// no staging copy, no temporary); otherwise (pageable memory) they are
// staged through a temporary device copy.
static bool device_views(const double* const* host, const double** dev) {
    for (int i = 0; i < 5; ++i) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, host[i]) != cudaSuccess || a.type != cudaMemoryTypeHost ||
            !a.devicePointer) {
            cudaGetLastError();
            return false;
        }
        dev[i] = (const double*)a.devicePointer;
    }
    return true;
}

int lbmhd_init(lbmhd_t* h, const double* rho, const double* ux, const double* uy,
               const double* bx, const double* by) {
    TraceRange trace_("lbmhd_init");
    int rc = check_handle(h);
    if (rc) return rc;
    if (!rho || !ux || !uy || !bx || !by) return fail(LBMHD_EINVAL, "NULL field");
    DeviceGuard dg(h->device);
    const long long n = ncell(h);
    const double* src[5] = {rho, ux, uy, bx, by};
    const double* dev[5];
    double* tmp = nullptr;
    if (!device_views(src, dev)) {
        LBMHD_CK(h, cudaMallocAsync((void**)&tmp, 5 * n * sizeof(double), h->stream));
        for (int i = 0; i < 5; ++i) {
            LBMHD_CK(h, cudaMemcpyAsync(tmp + i * n, src[i], n * sizeof(double),
                                        cudaMemcpyHostToDevice, h->stream));
            dev[i] = tmp + i * n;
        }
    }
    LBMHD_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    LBMHD_CK(h, launch_init(h->p.precision, dev[0], dev[1], dev[2], dev[3], dev[4],
                            h->buf[h->cur], h->geom, h->coll, h->stream, h->d_flag));
    if (tmp) LBMHD_CK(h, cudaFreeAsync(tmp, h->stream));
    int flag = 0;
    LBMHD_CK(h, cudaMemcpyAsync(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LBMHD_CK(h, cudaStreamSynchronize(h->stream));
    h->steps = 0;
    if (flag & 8) {
        h->initialised = false;
        LBMHD_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
        return fail(LBMHD_EINVAL, "rho must be positive and finite (the handle needs a new init)");
    }
    h->initialised = true;
    return LBMHD_OK;
}

int lbmhd_step(lbmhd_t* h, int n) {
    TraceRange trace_("lbmhd_step");
    int rc = check_handle(h);
    if (rc) return rc;
    if (n < 0) return fail(LBMHD_EINVAL, "n must be >= 0");
    if (!h->initialised) return fail(LBMHD_ESTATE, "lbmhd_step before lbmhd_init");
    DeviceGuard dg(h->device);
    const int every = h->p.check_finite_every;
    int done = 0;
    while (done < n) {
        const int left = n - done;
        if (left >= kGraphSteps && h->cur == 0 && every == 0 && h->capturable) {
            if (!h->graph) {
                cudaGraph_t g = nullptr;
                LBMHD_CK(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
                for (int s = 0; s < kGraphSteps; ++s) {
                    const int a = s & 1;
                    cudaError_t e = launch_one(h, h->buf[a], h->buf[1 - a]);
                    if (e != cudaSuccess) {
                        cudaStreamEndCapture(h->stream, &g);
                        if (g) cudaGraphDestroy(g);
                        return cuda_fail(h, e, "launch_step (capture)");
                    }
                }
                LBMHD_CK(h, cudaStreamEndCapture(h->stream, &g));
                cudaError_t e = cudaGraphInstantiate(&h->graph, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
                h->graph_steps = kGraphSteps;
            }
            LBMHD_CK(h, cudaGraphLaunch(h->graph, h->stream));
            h->launches += kGraphSteps * (h->coll.kin && h->kin_two_pass ? 2 : 1);
            done += kGraphSteps;
            h->steps += kGraphSteps;
            continue;
        }
        LBMHD_CK(h, one_step(h));
        ++done;
        ++h->steps;
        if (every > 0 && h->steps % every == 0)
            LBMHD_CK(h, launch_check_finite(h->p.precision, h->buf[h->cur], h->d_flag, h->geom,
                                            h->coll, h->stream));
    }
    return LBMHD_OK;
}

int lbmhd_moments_device(lbmhd_t* h, double* rho, double* ux, double* uy, double* bx,
                         double* by) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!rho || !ux || !uy || !bx || !by) return fail(LBMHD_EINVAL, "NULL field");
    if (!h->initialised) return fail(LBMHD_ESTATE, "moments before lbmhd_init");
    DeviceGuard dg(h->device);
    LBMHD_CK(h, launch_moments(h->p.precision, h->buf[h->cur], rho, ux, uy, bx, by, h->geom,
                               h->coll, h->stream));
    return LBMHD_OK;
}

int lbmhd_moments(lbmhd_t* h, double* rho, double* ux, double* uy, double* bx, double* by) {
    TraceRange trace_("lbmhd_moments");
    int rc = check_handle(h);
    if (rc) return rc;
    if (!rho || !ux || !uy || !bx || !by) return fail(LBMHD_EINVAL, "NULL field");
    if (!h->initialised) return fail(LBMHD_ESTATE, "moments before lbmhd_init");
    DeviceGuard dg(h->device);
    const long long n = ncell(h);
    double* dst[5] = {rho, ux, uy, bx, by};
    const double* dev[5];
    if (device_views(dst, dev)) {
        rc = lbmhd_moments_device(h, (double*)dev[0], (double*)dev[1], (double*)dev[2],
                                  (double*)dev[3], (double*)dev[4]);
        if (rc) return rc;
        return read_flag(h);
    }
    double* tmp = nullptr;
    LBMHD_CK(h, cudaMallocAsync((void**)&tmp, 5 * n * sizeof(double), h->stream));
    rc = lbmhd_moments_device(h, tmp, tmp + n, tmp + 2 * n, tmp + 3 * n, tmp + 4 * n);
    if (rc) {
        cudaFreeAsync(tmp, h->stream);
        return rc;
    }
    for (int i = 0; i < 5; ++i)
        LBMHD_CK(h, cudaMemcpyAsync(dst[i], tmp + i * n, n * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->stream));
    LBMHD_CK(h, cudaFreeAsync(tmp, h->stream));
    return read_flag(h);
}

int lbmhd_diagnostics(lbmhd_t* h, lbmhd_diag* out) {
    TraceRange trace_("lbmhd_diagnostics");
    int rc = check_handle(h);
    if (rc) return rc;
    if (!out) return fail(LBMHD_EINVAL, "out is NULL");
    if (!h->initialised) return fail(LBMHD_ESTATE, "diagnostics before lbmhd_init");
    DeviceGuard dg(h->device);
    double v[12];
    LBMHD_CK(h, launch_diag(h->p.precision, h->buf[h->cur], h->d_partials, h->d_diag, h->geom,
                            h->coll, h->stream));
    LBMHD_CK(h, cudaMemcpyAsync(v, h->d_diag, sizeof(v), cudaMemcpyDeviceToHost, h->stream));
    rc = read_flag(h);
    out->mass = v[0];
    out->mom_x = v[1];
    out->mom_y = v[2];
    out->bsum_x = v[3];
    out->bsum_y = v[4];
    out->E_kin = v[5];
    out->E_mag = v[6];
    out->enstrophy = v[7];
    out->cross_helicity = v[8];
    out->divB_max = v[9];
    out->divB_rms = v[10];
    out->current_sq = v[11];
    out->step = h->steps;
    return rc;
}

int lbmhd_get_state(lbmhd_t* h, double* state) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!state) return fail(LBMHD_EINVAL, "state is NULL");
    if (!h->initialised) return fail(LBMHD_ESTATE, "get_state before lbmhd_init");
    DeviceGuard dg(h->device);
    const long long n = ncell(h);
    double* tmp = nullptr;
    LBMHD_CK(h, cudaMallocAsync((void**)&tmp, kNumPlanes * n * sizeof(double), h->stream));
    LBMHD_CK(h, launch_get_state(h->p.precision, h->buf[h->cur], tmp, h->geom, h->coll, h->stream));
    LBMHD_CK(h, cudaMemcpyAsync(state, tmp, kNumPlanes * n * sizeof(double), cudaMemcpyDeviceToHost,
                                h->stream));
    LBMHD_CK(h, cudaFreeAsync(tmp, h->stream));
    LBMHD_CK(h, cudaStreamSynchronize(h->stream));
    return LBMHD_OK;
}

int lbmhd_get_state_raw(lbmhd_t* h, void* state, size_t bytes) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!state) return fail(LBMHD_EINVAL, "state is NULL");
    const size_t sb = storage_bytes(h->p.precision), n = (size_t)ncell(h);
    if (bytes != kNumPlanes * n * sb) return fail(LBMHD_EINVAL, "bytes != 19 * nx * ny * value size");
    if (!h->initialised) return fail(LBMHD_ESTATE, "get_state_raw before lbmhd_init");
    DeviceGuard dg(h->device);
    // the 19 planes, packed (the device planes are padded to the plane stride)
    LBMHD_CK(h, cudaMemcpy2DAsync(state, n * sb, h->buf[h->cur], (size_t)h->geom.ps * sb, n * sb,
                                  kNumPlanes, cudaMemcpyDeviceToHost, h->stream));
    LBMHD_CK(h, cudaStreamSynchronize(h->stream));
    return LBMHD_OK;
}

int lbmhd_set_state_raw(lbmhd_t* h, const void* state, size_t bytes) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!state) return fail(LBMHD_EINVAL, "state is NULL");
    const size_t sb = storage_bytes(h->p.precision), n = (size_t)ncell(h);
    if (bytes != kNumPlanes * n * sb) return fail(LBMHD_EINVAL, "bytes != 19 * nx * ny * value size");
    DeviceGuard dg(h->device);
    LBMHD_CK(h, cudaMemcpy2DAsync(h->buf[h->cur], (size_t)h->geom.ps * sb, state, n * sb, n * sb,
                                  kNumPlanes, cudaMemcpyHostToDevice, h->stream));
    LBMHD_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    LBMHD_CK(h, cudaStreamSynchronize(h->stream));
    h->initialised = true;
    return LBMHD_OK;
}

int lbmhd_set_state(lbmhd_t* h, const double* state) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!state) return fail(LBMHD_EINVAL, "state is NULL");
    DeviceGuard dg(h->device);
    const long long n = ncell(h);
    double* tmp = nullptr;
    LBMHD_CK(h, cudaMallocAsync((void**)&tmp, kNumPlanes * n * sizeof(double), h->stream));
    LBMHD_CK(h, cudaMemcpyAsync(tmp, state, kNumPlanes * n * sizeof(double), cudaMemcpyHostToDevice,
                                h->stream));
    LBMHD_CK(h, launch_set_state(h->p.precision, tmp, h->buf[h->cur], h->geom, h->coll, h->stream));
    LBMHD_CK(h, cudaFreeAsync(tmp, h->stream));
    LBMHD_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    LBMHD_CK(h, cudaStreamSynchronize(h->stream));
    h->initialised = true;
    return LBMHD_OK;
}

int lbmhd_copy_rows(lbmhd_t* dst, int dst_row, lbmhd_t* src, int src_row, int nrows) {
    int rc = check_handle(dst);
    if (rc) return rc;
    rc = check_handle(src);
    if (rc) return rc;
    if (dst->geom.nx != src->geom.nx || dst->p.precision != src->p.precision)
        return fail(LBMHD_EINVAL, "handles differ in nx or precision");
    if (nrows < 0 || dst_row < 0 || src_row < 0 || dst_row + nrows > dst->geom.ny ||
        src_row + nrows > src->geom.ny)
        return fail(LBMHD_EINVAL, "row range outside a lattice");
    if (!src->initialised) return fail(LBMHD_ESTATE, "source not initialised");
    if (nrows == 0) return LBMHD_OK;
    DeviceGuard dg(dst->device);
    // order after the source's pending work
    cudaEvent_t ev;
    LBMHD_CK(dst, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    LBMHD_CK(dst, cudaEventRecord(ev, src->stream));
    LBMHD_CK(dst, cudaStreamWaitEvent(dst->stream, ev, 0));
    cudaEventDestroy(ev);
    const size_t sb = storage_bytes(dst->p.precision);
    const size_t row = (size_t)dst->geom.nx * sb;
    // one strided copy: 19 planes of nrows contiguous rows each
    LBMHD_CK(dst, cudaMemcpy2DAsync(
                      (char*)dst->buf[dst->cur] + (size_t)dst_row * row, dst->geom.ps * sb,
                      (const char*)src->buf[src->cur] + (size_t)src_row * row, src->geom.ps * sb,
                      (size_t)nrows * row, kNumPlanes, cudaMemcpyDeviceToDevice, dst->stream));
    dst->initialised = true;
    return LBMHD_OK;
}

int lbmhd_step_rows(lbmhd_t* h, int y0, int y1) {
    TraceRange trace_("lbmhd_step_rows");
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->initialised) return fail(LBMHD_ESTATE, "lbmhd_step_rows before lbmhd_init");
    if (y0 < 0 || y1 > h->geom.ny || y0 >= y1)
        return fail(LBMHD_EINVAL, "need 0 <= y0 < y1 <= ny");
    DeviceGuard dg(h->device);
    const void* src = h->buf[h->cur];
    void* dst = h->buf[1 - h->cur];
    cudaError_t e;
    if (h->coll.kin)
        e = launch_step_kinetic(h->p.precision, h->kin_two_pass != 0, h->sm_count, src, dst,
                                h->d_kin, h->geom, h->coll, h->stream, y0, y1);
    else
        e = launch_step(h->p.precision, h->vec, h->block, 0, src, dst, h->geom, h->coll,
                        h->stream, y0, y1);
    if (e != cudaSuccess) return cuda_fail(h, e, "lbmhd_step_rows");
    h->launches += h->coll.kin && h->kin_two_pass ? 2 : 1;
    return LBMHD_OK;
}

int lbmhd_step_commit(lbmhd_t* h) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!h->initialised) return fail(LBMHD_ESTATE, "lbmhd_step_commit before lbmhd_init");
    h->cur = 1 - h->cur;
    ++h->steps;
    return LBMHD_OK;
}

namespace {
int row_planes(lbmhd_t* h, bool pack, int row, unsigned mask, void* buf, void* stream) {
    int rc = check_handle(h);
    if (rc) return rc;
    if (!buf) return fail(LBMHD_EINVAL, "buf is NULL");
    if (row < 0 || row >= h->geom.ny) return fail(LBMHD_EINVAL, "row outside the lattice");
    if (mask >> kNumPlanes) return fail(LBMHD_EINVAL, "plane_mask has bits above plane 18");
    if ((uintptr_t)buf % storage_bytes(h->p.precision))
        return fail(LBMHD_EINVAL, "buf must be aligned to the stored value size");
    if (pack && !h->initialised) return fail(LBMHD_ESTATE, "lbmhd_pack_row before lbmhd_init");
    int planes[kNumPlanes], n = 0;
    for (int p = 0; p < kNumPlanes; ++p)
        if (mask >> p & 1u) planes[n++] = p;
    DeviceGuard dg(h->device);
    const cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
    const cudaError_t e =
        launch_row_planes(h->p.precision, pack, h->buf[h->cur], h->geom, row, planes, n, buf, st);
    if (e != cudaSuccess) return cuda_fail(h, e, pack ? "lbmhd_pack_row" : "lbmhd_unpack_row");
    if (!pack) h->initialised = true;
    return LBMHD_OK;
}
}  // namespace

int lbmhd_pack_row(lbmhd_t* h, int row, unsigned plane_mask, void* buf, void* stream) {
    return row_planes(h, true, row, plane_mask, buf, stream);
}

int lbmhd_unpack_row(lbmhd_t* h, int row, unsigned plane_mask, const void* buf, void* stream) {
    return row_planes(h, false, row, plane_mask, const_cast<void*>(buf), stream);
}

int lbmhd_sync(lbmhd_t* h) {
    int rc = check_handle(h);
    if (rc) return rc;
    DeviceGuard dg(h->device);
    return read_flag(h);
}

int64_t lbmhd_step_count(const lbmhd_t* h) { return h ? h->steps : 0; }

int64_t lbmhd_launch_count(const lbmhd_t* h) { return h ? h->launches : 0; }

void lbmhd_destroy(lbmhd_t* h) {
    if (!h) return;
    DeviceGuard dg(h->device);
    if (!h->failed) cudaStreamSynchronize(h->stream);
    free_tape(h);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
    cudaFree(h->d_partials);
    cudaFree(h->d_diag);
    cudaFree(h->d_flag);
    cudaFree(h->d_kin);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char* lbmhd_last_error(void) { return g_err.c_str(); }

}  // extern "C"
