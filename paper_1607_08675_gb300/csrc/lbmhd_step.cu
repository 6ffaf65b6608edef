// lbmhd_step.cu -- the fused pull-stream + collide kernel of one LB-MHD
// time step over a single lattice (Sec. 1.2 streaming, Sec. 3 MRT / SRT
// collisions).  The per-thread work is step_body (lbmhd_step_body.cuh): a
// warp covers 32*V consecutive nodes of one row, loads each of the 19
// planes once with aligned vector loads, takes the x-halo from the
// neighbouring lane by a shuffle and collides in registers.  All HBM
// traffic is the 19 plane reads and 19 plane writes per node.
#include "lbmhd_internal.h"
#include "lbmhd_step_body.cuh"

namespace lbmhd {

template <int P, int V>
__global__ void __launch_bounds__(256) step_kernel(const typename Fmt<P>::S* __restrict__ src,
                                                   typename Fmt<P>::S* __restrict__ dst, int nx,
                                                   int ny, long long ps, unsigned total,
                                                   unsigned total_pad,
                                                   Coll<typename Fmt<P>::R> c, float scale,
                                                   float inv_scale, int y0) {
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total_pad; t += stride)
        step_body<P, V>(src, dst, nx, ny, ps, t, total, c, scale, inv_scale, y0);
}

template <int P, int V>
static cudaError_t launch_pv(int block, int max_blocks, const void* src, void* dst, const Geom& g,
                             const HostColl& hc, cudaStream_t st, int y0, int y1) {
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    const unsigned total = (unsigned)((long long)g.nx / V * (y1 - y0));
    const unsigned total_pad = (total + 31u) / 32u * 32u;
    long long blocks = ((long long)total_pad + block - 1) / block;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    step_kernel<P, V><<<(unsigned)blocks, block, 0, st>>>(
        (const S*)src, (S*)dst, g.nx, g.ny, g.ps, total, total_pad, coll_for_prec<R>(hc, P), hc.scale,
        hc.inv_scale, y0);
    return cudaGetLastError();
}

bool step_variant_ok(int prec, int vec, int nx) {
    if (prec < 0 || prec > 4) return false;
    if (vec != 1 && vec != 2 && vec != 4 && !(vec == 8 && prec == P_FP16_DEV)) return false;
    return nx % vec == 0;
}

cudaError_t launch_step(int prec, int vec, int block, int max_blocks, const void* src, void* dst,
                        const Geom& g, const HostColl& c, cudaStream_t st, int y0, int y1) {
    if (y1 < 0) y1 = g.ny;
#define LBMHD_CASE(P)                                                                      \
    case P:                                                                                \
        switch (vec) {                                                                     \
            case 1: return launch_pv<P, 1>(block, max_blocks, src, dst, g, c, st, y0, y1); \
            case 2: return launch_pv<P, 2>(block, max_blocks, src, dst, g, c, st, y0, y1); \
            case 4: return launch_pv<P, 4>(block, max_blocks, src, dst, g, c, st, y0, y1); \
        }                                                                                  \
        break;
    switch (prec) {
        LBMHD_CASE(P_FP64)
        LBMHD_CASE(P_FP32)
        LBMHD_CASE(P_FP32_DEV)
        LBMHD_CASE(P_FF)
        case P_FP16_DEV:
            switch (vec) {
                case 1: return launch_pv<P_FP16_DEV, 1>(block, max_blocks, src, dst, g, c, st, y0, y1);
                case 2: return launch_pv<P_FP16_DEV, 2>(block, max_blocks, src, dst, g, c, st, y0, y1);
                case 4: return launch_pv<P_FP16_DEV, 4>(block, max_blocks, src, dst, g, c, st, y0, y1);
                case 8: return launch_pv<P_FP16_DEV, 8>(block, max_blocks, src, dst, g, c, st, y0, y1);
            }
            break;
    }
#undef LBMHD_CASE
    return cudaErrorInvalidValue;
}

}  // namespace lbmhd
