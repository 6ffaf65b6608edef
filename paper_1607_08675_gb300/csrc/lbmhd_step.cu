// lbmhd_step.cu -- the fused pull-stream + collide kernel of one LB-MHD
// time step (Sec. 1.2 streaming, Sec. 3 MRT / SRT collisions).
//
// Layout: 19 SoA planes per buffer, x fastest.  A warp covers 32*V
// consecutive nodes of one row; each thread loads V nodes of every plane
// with one aligned vector load.  The pull of an x-shifted plane needs the
// element just left (c_x = +1) or right (c_x = -1) of the thread's
// segment: it comes from the neighbouring lane by a warp shuffle, and only
// a lane at a warp edge or at the periodic wrap loads it from memory.  All
// HBM traffic is therefore the 19 coalesced plane reads and 19 plane
// writes per node; the collision runs in registers.
#include "lbmhd_device.cuh"
#include "lbmhd_internal.h"

namespace lbmhd {

template <class S, int V>
struct alignas(sizeof(S) * V) Pack {
    S v[V];
};

template <class S>
__device__ __forceinline__ S shfl_up1(S v) {
    return __shfl_up_sync(0xffffffffu, v, 1);
}
template <>
__device__ __forceinline__ unsigned short shfl_up1(unsigned short v) {
    return (unsigned short)__shfl_up_sync(0xffffffffu, (unsigned)v, 1);
}
template <class S>
__device__ __forceinline__ S shfl_down1(S v) {
    return __shfl_down_sync(0xffffffffu, v, 1);
}
template <>
__device__ __forceinline__ unsigned short shfl_down1(unsigned short v) {
    return (unsigned short)__shfl_down_sync(0xffffffffu, (unsigned)v, 1);
}

template <int P, int V>
__global__ void __launch_bounds__(256) step_kernel(const typename Fmt<P>::S* __restrict__ src,
                                                   typename Fmt<P>::S* __restrict__ dst, int nx,
                                                   int ny, long long ps, unsigned total,
                                                   unsigned total_pad,
                                                   Coll<typename Fmt<P>::R> c, float scale,
                                                   float inv_scale) {
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    const int lane = threadIdx.x & 31;
    const unsigned nxv = (unsigned)(nx / V);
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total_pad; t += stride) {
        const bool live = t < total;
        const unsigned tc = live ? t : total - 1;
        const int y = (int)(tc / nxv);
        const int x0 = (int)(tc - (unsigned)y * nxv) * V;
        const int ym = y == 0 ? ny - 1 : y - 1;
        const int yp = y == ny - 1 ? 0 : y + 1;
        const bool has_left = lane > 0 && x0 > 0;
        const bool has_right = lane < 31 && x0 + V < nx;
        const int xl = x0 == 0 ? nx - 1 : x0 - 1;
        const int xr = x0 + V == nx ? 0 : x0 + V;

        S raw[kPlanes][V];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const int cx = plane_cx(p), cy = plane_cy(p);
            const int row = cy == 0 ? y : (cy > 0 ? ym : yp);
            const S* base = src + p * ps + (long long)row * nx;
            const Pack<S, V> pk = *reinterpret_cast<const Pack<S, V>*>(base + x0);
            if (cx == 0) {
#pragma unroll
                for (int k = 0; k < V; ++k) raw[p][k] = pk.v[k];
            } else if (cx > 0) {
                S prev = shfl_up1(pk.v[V - 1]);
                if (!has_left) prev = base[xl];
                raw[p][0] = prev;
#pragma unroll
                for (int k = 1; k < V; ++k) raw[p][k] = pk.v[k - 1];
            } else {
                S next = shfl_down1(pk.v[0]);
                if (!has_right) next = base[xr];
#pragma unroll
                for (int k = 0; k < V - 1; ++k) raw[p][k] = pk.v[k + 1];
                raw[p][V - 1] = next;
            }
        }

#pragma unroll
        for (int k = 0; k < V; ++k) {
            R d[9], g[10];
#pragma unroll
            for (int i = 0; i < 9; ++i) d[i] = Fmt<P>::dec(raw[i][k], i, inv_scale);
#pragma unroll
            for (int q = 0; q < 10; ++q) g[q] = Fmt<P>::dec(raw[9 + q][k], 9 + q, inv_scale);
            collide<R>(d, g, c);
#pragma unroll
            for (int i = 0; i < 9; ++i) raw[i][k] = Fmt<P>::enc(d[i], i, scale);
#pragma unroll
            for (int q = 0; q < 10; ++q) raw[9 + q][k] = Fmt<P>::enc(g[q], 9 + q, scale);
        }

        if (live) {
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) {
                Pack<S, V> o;
#pragma unroll
                for (int k = 0; k < V; ++k) o.v[k] = raw[p][k];
                *reinterpret_cast<Pack<S, V>*>(dst + p * ps + (long long)y * nx + x0) = o;
            }
        }
    }
}

template <class R>
static Coll<R> to_coll(const HostColl& h) {
    Coll<R> c;
    c.tn = (R)h.tn;
    c.te = (R)h.te;
    c.tn2 = (R)(h.tn * h.tn);
    c.te2 = (R)(h.te * h.te);
    c.k18 = (R)h.k18;
    c.k36 = (R)h.k36;
    c.s5 = (R)h.s5;
    c.s6 = (R)h.s6;
    c.s7 = (R)h.s7;
    c.s8 = (R)h.s8;
    c.les = h.les;
    return c;
}

template <int P, int V>
static cudaError_t launch_pv(int block, int max_blocks, const void* src, void* dst, const Geom& g,
                             const HostColl& hc, cudaStream_t st) {
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    const unsigned total = (unsigned)((long long)g.nx / V * g.ny);
    const unsigned total_pad = (total + 31u) / 32u * 32u;
    long long blocks = ((long long)total_pad + block - 1) / block;
    if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
    step_kernel<P, V><<<(unsigned)blocks, block, 0, st>>>(
        (const S*)src, (S*)dst, g.nx, g.ny, g.ps, total, total_pad, to_coll<R>(hc), hc.scale,
        hc.inv_scale);
    return cudaGetLastError();
}

bool step_variant_ok(int prec, int vec, int nx) {
    if (prec < 0 || prec > 3) return false;
    if (vec != 1 && vec != 2 && vec != 4) return false;
    return nx % vec == 0;
}

cudaError_t launch_step(int prec, int vec, int block, int max_blocks, const void* src, void* dst,
                        const Geom& g, const HostColl& c, cudaStream_t st) {
#define LBMHD_CASE(P)                                                              \
    case P:                                                                        \
        switch (vec) {                                                             \
            case 1: return launch_pv<P, 1>(block, max_blocks, src, dst, g, c, st); \
            case 2: return launch_pv<P, 2>(block, max_blocks, src, dst, g, c, st); \
            case 4: return launch_pv<P, 4>(block, max_blocks, src, dst, g, c, st); \
        }                                                                          \
        break;
    switch (prec) {
        LBMHD_CASE(P_FP64)
        LBMHD_CASE(P_FP32)
        LBMHD_CASE(P_FP32_DEV)
        LBMHD_CASE(P_FP16_DEV)
    }
#undef LBMHD_CASE
    return cudaErrorInvalidValue;
}

}  // namespace lbmhd
