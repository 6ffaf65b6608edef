// lbmhd_step_tma.cu -- the fused stream-collide step with its loads staged
// through shared memory by bulk asynchronous copies (TMA, cp.async.bulk)
// in a multi-stage ring, for the FP32 and FP16 storage formats.
//
// Why: the register kernel (lbmhd_step.cu) moves exactly the algorithmic
// bytes but keeps too few of them in flight (its loads live in registers,
// so occupancy caps the memory parallelism).  Here one persistent CTA per
// SM walks row tiles of W nodes; one elected thread keeps the next
// STAGES-1 tiles' 19 plane rows in flight as bulk copies completing on
// mbarriers, while all W threads collide the current tile out of shared
// memory (one node per thread) and store the result rows with coalesced
// stores.
//
// Tile (y, x0): plane p is pulled from row y - c_py.  Planes with c_px = +1
// also need the element left of x0, planes with c_px = -1 the element right
// of x0 + W - 1; their copies are widened by one 16-byte granule on that
// side (bulk copies move 16-byte multiples from 16-byte aligned
// addresses), and at the periodic row ends the granule comes from the
// other end of the row in a separate 16-byte copy.  Shared row of plane p:
// [H granule | W nodes | H granule], node x at index H + x.
//
// Every wait on an mbarrier is bounded: past ~2 s the kernel records
// LBMHD_ETIMEOUT in the status word, drains its own copies (bounded again)
// and returns.
#include <cuda_fp16.h>

#include "lbmhd_bulk.cuh"
#include "lbmhd_internal.h"
#include "lbmhd_step_body.cuh"

namespace lbmhd {

template <int P, int W, int STAGES>
struct TmaCfg {
    using S = typename Fmt<P>::S;
    static constexpr int H = 16 / (int)sizeof(S);  // one 16-byte granule
    static constexpr int ROW = W + 2 * H;           // elements per staged plane row
    static constexpr int STAGE_ELEMS = kPlanes * ROW;
    static constexpr size_t STAGE_BYTES = (size_t)STAGE_ELEMS * sizeof(S);
    // one 8-byte mbarrier per stage after the stage buffers
    static constexpr size_t BAR_BYTES = ((size_t)STAGES * 8 + 127) / 128 * 128;
    static constexpr size_t SMEM = STAGES * STAGE_BYTES + BAR_BYTES;
    static_assert(STAGE_BYTES % 16 == 0 && (ROW * sizeof(S)) % 16 == 0,
                  "bulk-copy destinations must stay 16-byte aligned");
    static_assert(BAR_BYTES >= STAGES * 8, "room for every stage barrier");
    static_assert(SMEM <= 227 * 1024, "dynamic shared memory per CTA");
};

// Issue the copies of tile t into stage buffer sb (one thread).
template <int P, int W, int STAGES>
__device__ __forceinline__ void issue_tile(const typename Fmt<P>::S* __restrict__ src,
                                           typename Fmt<P>::S* sb, unsigned long long* bar,
                                           long long t, int tiles_x, int nx, int ny,
                                           long long ps) {
    using C = TmaCfg<P, W, STAGES>;
    using S = typename C::S;
    constexpr int H = C::H;
    const int y = (int)(t / tiles_x);
    const int x0 = (int)(t - (long long)y * tiles_x) * W;
    const bool left_wrap = x0 == 0;
    const bool right_wrap = x0 + W == nx;
    // bytes: 19 rows of W nodes, one granule per x-shifted plane (6 of f, 4 of g)
    mbar_expect_tx(bar, (unsigned)((kPlanes * W + 10 * H) * sizeof(S)));
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = plane_cx(p), cy = plane_cy(p);
        int row = y - cy;
        row = row < 0 ? row + ny : (row >= ny ? row - ny : row);
        const S* g = src + p * ps + (long long)row * nx;
        S* s = sb + p * C::ROW;
        if (cx == 0) {
            bulk_g2s(s + H, g + x0, W * sizeof(S), bar);
        } else if (cx > 0) {  // needs node x0 - 1
            if (left_wrap) {
                bulk_g2s(s + H, g + x0, W * sizeof(S), bar);
                bulk_g2s(s, g + (nx - H), H * sizeof(S), bar);
            } else {
                bulk_g2s(s, g + (x0 - H), (W + H) * sizeof(S), bar);
            }
        } else {  // needs node x0 + W
            if (right_wrap) {
                bulk_g2s(s + H, g + x0, W * sizeof(S), bar);
                bulk_g2s(s + H + W, g, H * sizeof(S), bar);
            } else {
                bulk_g2s(s + H, g + x0, (W + H) * sizeof(S), bar);
            }
        }
    }
}

template <int P, int W, int STAGES>
__global__ void __launch_bounds__(W) step_tma_kernel(const typename Fmt<P>::S* __restrict__ src,
                                                     typename Fmt<P>::S* __restrict__ dst,
                                                     int nx, int ny, long long ps,
                                                     Coll<typename Fmt<P>::R> c, float scale,
                                                     float inv_scale, int* status) {
    using C = TmaCfg<P, W, STAGES>;
    using S = typename C::S;
    using R = typename Fmt<P>::R;
    constexpr int H = C::H;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S* stage = reinterpret_cast<S*>(smem_raw);
    unsigned long long* full =
        reinterpret_cast<unsigned long long*>(smem_raw + STAGES * C::STAGE_BYTES);
    __shared__ int abort_flag;

    const int tiles_x = nx / W;
    const long long ntiles = (long long)tiles_x * ny;
    const int tid = threadIdx.x;
    // tiles of this CTA: blockIdx.x + k * gridDim.x, k = 0 .. my_n - 1
    const long long my_n =
        blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < STAGES; ++s) mbar_init(&full[s], 1);
        mbar_init_fence();
    }
    __syncthreads();
    long long issued = 0;  // meaningful in thread 0 only
    if (tid == 0)
        for (; issued < STAGES && issued < my_n; ++issued)
            issue_tile<P, W, STAGES>(src, stage + issued * C::STAGE_ELEMS, &full[issued],
                                     blockIdx.x + issued * gridDim.x, tiles_x, nx, ny, ps);

    long long k = 0;
    for (; k < my_n; ++k) {
        const int s = (int)(k % STAGES);
        if (!mbar_wait_bounded(&full[s], (unsigned)((k / STAGES) & 1))) atomicExch(&abort_flag, 1);
        __syncthreads();
        if (abort_flag) break;
        const long long t = blockIdx.x + k * gridDim.x;
        const int y = (int)(t / tiles_x);
        const int x0 = (int)(t - (long long)y * tiles_x) * W;
        const S* sb = stage + s * C::STAGE_ELEMS;

        R d[9], g[10];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const S v = sb[p * C::ROW + H + tid - plane_cx(p)];
            if (p < 9) d[p] = Fmt<P>::dec(v, p, inv_scale);
            else g[p - 9] = Fmt<P>::dec(v, p, inv_scale);
        }
        // all reads of stage s are done after this barrier: refill it with
        // tile k + STAGES, keeping STAGES tiles in flight during the collision
        __syncthreads();
        if (tid == 0 && issued < my_n) {
            issue_tile<P, W, STAGES>(src, stage + s * C::STAGE_ELEMS, &full[s],
                                     blockIdx.x + issued * gridDim.x, tiles_x, nx, ny, ps);
            ++issued;
        }
        collide<R, Fmt<P>::kScaled>(d, g, c);
        S* out = dst + (long long)y * nx + x0 + tid;
#pragma unroll
        for (int i = 0; i < 9; ++i) out[i * ps] = Fmt<P>::enc(d[i], i, scale);
#pragma unroll
        for (int q = 0; q < 10; ++q) out[(9 + q) * ps] = Fmt<P>::enc(g[q], 9 + q, scale);
    }

    if (abort_flag && tid == 0) {
        // drain this CTA's own copies still in flight (bounded), then report
        for (long long kk = k; kk < issued; ++kk)
            if (!mbar_wait_bounded(&full[kk % STAGES], (unsigned)((kk / STAGES) & 1))) break;
        atomicOr(status, 2);
    }
}

template <int P, int W, int STAGES>
static cudaError_t launch_tma_pws(const void* src, void* dst, const Geom& g, const Coll<typename Fmt<P>::R>& c,
                                  float scale, float inv_scale, int* status, int grid,
                                  cudaStream_t st) {
    using C = TmaCfg<P, W, STAGES>;
    auto k = step_tma_kernel<P, W, STAGES>;
    static bool attr_set = false;  // per process; the attribute is per function
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    using S = typename Fmt<P>::S;
    k<<<grid, W, C::SMEM, st>>>((const S*)src, (S*)dst, g.nx, g.ny, g.ps, c, scale, inv_scale,
                                status);
    return cudaGetLastError();
}

// Tile widths offered: W threads per CTA = nodes per tile.  Stages fill
// about 160 KB of shared memory.
bool tma_variant_ok(int prec, int W, int nx) {
    if (prec != P_FP32 && prec != P_FP32_DEV && prec != P_FP16_DEV) return false;
    if (W != 128 && W != 256 && W != 512) return false;
    const int gran = prec == P_FP16_DEV ? 8 : 4;
    return nx % W == 0 && nx % gran == 0 && nx >= W;
}

cudaError_t launch_step_tma(int prec, int W, int grid, const void* src, void* dst, const Geom& g,
                            const HostColl& hc, int* status, cudaStream_t st) {
    const Coll<float> c = coll_for_prec<float>(hc, prec);
#define LBMHD_TMA(P, WW, SS) \
    return launch_tma_pws<P, WW, SS>(src, dst, g, c, hc.scale, hc.inv_scale, status, grid, st)
    switch (prec) {
        case P_FP32:
            if (W == 128) LBMHD_TMA(P_FP32, 128, 16);
            if (W == 256) LBMHD_TMA(P_FP32, 256, 8);
            if (W == 512) LBMHD_TMA(P_FP32, 512, 4);
            break;
        case P_FP32_DEV:
            if (W == 128) LBMHD_TMA(P_FP32_DEV, 128, 16);
            if (W == 256) LBMHD_TMA(P_FP32_DEV, 256, 8);
            if (W == 512) LBMHD_TMA(P_FP32_DEV, 512, 4);
            break;
        case P_FP16_DEV:
            if (W == 128) LBMHD_TMA(P_FP16_DEV, 128, 24);
            if (W == 256) LBMHD_TMA(P_FP16_DEV, 256, 16);
            if (W == 512) LBMHD_TMA(P_FP16_DEV, 512, 8);
            break;
    }
#undef LBMHD_TMA
    return cudaErrorInvalidValue;
}

}  // namespace lbmhd
