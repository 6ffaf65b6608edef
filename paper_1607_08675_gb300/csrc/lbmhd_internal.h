// lbmhd_internal.h -- declarations shared by the library's translation
// units (kernel launchers and the handle).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "lbmhd.h"

#include <nvtx3/nvToolsExt.h>

namespace lbmhd {

// A named range on the calling thread for profilers (NVTX; a no-op unless a
// tool is attached), held for the duration of an entry point.
struct TraceRange {
    explicit TraceRange(const char* name) { nvtxRangePushA(name); }
    ~TraceRange() { nvtxRangePop(); }
    TraceRange(const TraceRange&) = delete;
    TraceRange& operator=(const TraceRange&) = delete;
};


constexpr int kNumPlanes = 19;  // 9 f_i, then g_k (x, y) for k = 0..4

// Host-side copy of the collision parameters; converted to the arithmetic
// type of a precision by the launchers.
struct HostColl {
    double tn, te, k18, k36, s5, s6, s7, s8;
    int les;
    float scale, inv_scale;  // FP16_DEV encoding
    int tie5, tie6;          // s5 / s6 are the tied 1/tau_nu
    int kin;                 // 2: filtered equilibria, 3: cross-helicity closure, 0: neither
    double d2;               // Delta^2
};

// Geometry of one lattice in device memory: 19 planes of ps elements each,
// node (x, y) at y*nx + x within a plane.
struct Geom {
    int nx, ny;
    long long ps;  // plane stride in elements (padded)
};

size_t storage_bytes(int prec);   // bytes of one stored value
long long plane_stride(int nx, int ny);

// Fused stream-collide step: src -> dst (both 19 planes).  vec = nodes per
// thread along x (1, 2, 4; nx % vec == 0), block = threads per block,
// max_blocks = 0 for an exact cover, else a grid-stride cap.  Rows
// [y0, y1) of dst only (y1 < 0: every row); the pull wraps periodically.
cudaError_t launch_step(int prec, int vec, int block, int max_blocks, const void* src, void* dst,
                        const Geom& g, const HostColl& c, cudaStream_t st, int y0 = 0,
                        int y1 = -1);
bool step_variant_ok(int prec, int vec, int nx);

// TMA-staged step (lbmhd_step_tma.cu): W threads = nodes per row tile,
// persistent grid of `grid` CTAs; a timed-out wait sets bit 2 of *status.
bool tma_variant_ok(int prec, int W, int nx);

// Kinetic-LES step (lbmhd_kinetic.cu), les = 2 or 3.  Default: one fused
// launch (column strips swept down in y, moments of the next row in a
// shared-memory ring).  two_pass: conserved moments of the streamed
// populations into `mom` (5 planes of the arithmetic type, plane stride
// g.ps), then the step.  Both give the same bits.
// Kinetic-LES step of an ensemble (lbmhd_kinetic.cu), one CTA per work
// unit.  fused: the one-pass kernel, a unit being one strip-segment of a run
// (kinetic_fused_strip(prec) columns wide; RunDev::kstrips, kseglen);
// otherwise the moments pass and the step, a unit being `block` nodes.
// runs: device array of RunDev<R> (lbmhd_batch_run.cuh); mom: the runs'
// moment planes (two-pass only).
cudaError_t launch_batch_kinetic(int prec, int kin, bool fused, const void* runs,
                                 const int* unit_run, unsigned nunits, int block, const void* src,
                                 void* dst, void* mom, float inv_s, cudaStream_t st);
int kinetic_fused_strip(int prec);
// Rows [y0, y1) of dst only (y1 < 0: every row); moments are formed for
// rows y0 - 1 .. y1 (periodic).
cudaError_t launch_step_kinetic(int prec, bool two_pass, int sm_count, const void* src,
                                void* dst, void* mom, const Geom& g, const HostColl& c,
                                cudaStream_t st, int y0 = 0, int y1 = -1);
// Gather (pack) or scatter (unpack) the planes planes[0 .. nplanes) of row
// `row` of a 19-plane state to / from buf, nplanes * nx stored values in
// plane order (lbmhd_aux.cu).
cudaError_t launch_row_planes(int prec, bool pack, void* state, const Geom& g, int row,
                              const int* planes, int nplanes, void* buf, cudaStream_t st);
cudaError_t launch_step_tma(int prec, int W, int grid, const void* src, void* dst, const Geom& g,
                            const HostColl& c, int* status, cudaStream_t st);

// Equilibrium initialisation from five FP64 fields the device can address
// (device memory or pinned host memory).  With bad != nullptr, a density
// that is not positive and finite sets bit 3 (value 8) of *bad.
cudaError_t launch_init(int prec, const double* rho, const double* ux, const double* uy,
                        const double* bx, const double* by, void* state, const Geom& g,
                        const HostColl& c, cudaStream_t st, int* bad = nullptr);
// Moments of a stored state into five FP64 device fields.
cudaError_t launch_moments(int prec, const void* state, double* rho, double* ux, double* uy,
                           double* bx, double* by, const Geom& g, const HostColl& c,
                           cudaStream_t st);
// Decode to / encode from 19 FP64 planes of nx*ny (unpadded).
cudaError_t launch_get_state(int prec, const void* state, double* out, const Geom& g,
                             const HostColl& c, cudaStream_t st);
cudaError_t launch_set_state(int prec, const double* in, void* state, const Geom& g,
                             const HostColl& c, cudaStream_t st);
// Sets bit 1 of *flag if the density or the magnetic rest population is
// not finite anywhere.
cudaError_t launch_check_finite(int prec, const void* state, int* flag, const Geom& g,
                                const HostColl& c, cudaStream_t st);

// Diagnostics: per-block FP64 partials then one fixed-order final pass.
int diag_num_blocks(const Geom& g, int prec);
cudaError_t launch_diag(int prec, const void* state, double* partials, double* out12,
                        const Geom& g, const HostColl& c, cudaStream_t st);

void set_error(const std::string& msg);

// Frees the adjoint tape of a handle (lbmhd_adjoint.cu).
void free_tape(lbmhd_t* h);

// Parameter validation shared by lbmhd_create and lbmhd_batch_create
// (status code; message through set_error).
int validate_params(int nx, int ny, const lbmhd_params* p);

}  // namespace lbmhd

struct lbmhd_t {
    lbmhd::Geom geom;
    lbmhd_params p;
    lbmhd::HostColl coll;
    int device;
    cudaStream_t stream;
    bool own_stream;
    bool capturable;
    void* buf[2];
    int cur;
    bool initialised;
    bool failed;
    int64_t steps;
    int64_t launches;
    void* tape;  // adjoint checkpoints (lbmhd_adjoint.cu), NULL when none
    void* d_kin; // les = 2: streamed conserved moments (5 planes)
    double* d_partials;
    double* d_diag;
    int* d_flag;
    int vec, block;   // register kernel: nodes per thread, threads per block
    int tma_w;        // > 0: TMA-staged kernel with this tile width
    int kin_two_pass; // les 2, 3: moments pass + step instead of the fused kernel
    int sm_count;
    cudaGraphExec_t graph;
    int graph_steps;
};
