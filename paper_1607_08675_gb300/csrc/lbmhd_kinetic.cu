// lbmhd_kinetic.cu -- the steps that need gradients of the resolved fields:
// the paper's own kinetic LES (les = 2, Sec. 4.1) and the cross-helicity
// closure of Carati et al. (les = 3, Eqs. CHClosureV/B, whose rates are built
// from u and B gradients).  For les = 2 the collision relaxes towards the filtered equilibria
// M^eq + Delta^2 M^(Delta), whose corrections need gradients of the
// resolved conserved moments at the current step.  Two kernels:
//  1. kin_moments_kernel: rho, jx, jy, Bx, By of the populations streamed
//     into every node (pull + sums) into five planes;
//  2. step_kin_kernel: per node, pull the populations, take central
//     differences of those planes at x +- 1, y +- 1, form the corrections
//     (filtered_shift) and collide (collide<..., KIN>) -- or, for les = 3,
//     the closure's relaxation times (carati_taus) and collide with them.
// One node per thread; neighbouring threads share the moment loads in L1.
#include "lbmhd_internal.h"
#include "lbmhd_step_body.cuh"

namespace lbmhd {

namespace {

__device__ __forceinline__ int wrapk(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

template <int P>
__global__ void __launch_bounds__(256) kin_moments_kernel(const typename Fmt<P>::S* __restrict__ src,
                                                          typename Fmt<P>::R* __restrict__ mom,
                                                          int nx, int ny, long long ps,
                                                          float inv_s) {
    using R = typename Fmt<P>::R;
    const long long n = (long long)nx * ny;
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(node / nx), x = (int)(node - (long long)y * nx);
        R d[kPlanes];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p)
            d[p] = Fmt<P>::dec(src[p * ps + (long long)wrapk(y - plane_cy(p), ny) * nx +
                                   wrapk(x - plane_cx(p), nx)],
                               p, 1.0f);
        R drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
        R jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
        R jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
        R bx = (d[9] + d[11]) + (d[13] + d[15]) + d[17];
        R by = (d[10] + d[12]) + (d[14] + d[16]) + d[18];
        if (Fmt<P>::kScaled) {  // stored values carry the FP16 storage scale
            drho *= (R)inv_s;
            jx *= (R)inv_s;
            jy *= (R)inv_s;
            bx *= (R)inv_s;
            by *= (R)inv_s;
        }
        mom[node] = R(1) + drho;
        mom[ps + node] = jx;
        mom[2 * ps + node] = jy;
        mom[3 * ps + node] = bx;
        mom[4 * ps + node] = by;
    }
}

template <int P, int MODE>
__global__ void __launch_bounds__(256) step_kin_kernel(const typename Fmt<P>::S* __restrict__ src,
                                                       typename Fmt<P>::S* __restrict__ dst,
                                                       const typename Fmt<P>::R* __restrict__ mom,
                                                       int nx, int ny, long long ps,
                                                       Coll<typename Fmt<P>::R> c) {
    using R = typename Fmt<P>::R;
    const long long n = (long long)nx * ny;
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const int y = (int)(node / nx), x = (int)(node - (long long)y * nx);
        R d[9], g[10];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const R v = Fmt<P>::dec(src[p * ps + (long long)wrapk(y - plane_cy(p), ny) * nx +
                                        wrapk(x - plane_cx(p), nx)],
                                    p, 1.0f);
            if (p < 9) d[p] = v;
            else g[p - 9] = v;
        }
        const long long xp = (long long)y * nx + wrapk(x + 1, nx);
        const long long xm = (long long)y * nx + wrapk(x - 1, nx);
        const long long yp = (long long)wrapk(y + 1, ny) * nx + x;
        const long long ym = (long long)wrapk(y - 1, ny) * nx + x;
        if (MODE == 2) {
            R fld[5], gx[5], gy[5], sh[4];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                const R* m = mom + q * ps;
                fld[q] = m[node];
                gx[q] = R(0.5) * (m[xp] - m[xm]);
                gy[q] = R(0.5) * (m[yp] - m[ym]);
            }
            filtered_shift<R>(fld, gx, gy, c.d2, sh);
            if (Fmt<P>::kScaled)
#pragma unroll
                for (int q = 0; q < 4; ++q) sh[q] *= c.scl;
            collide<R, Fmt<P>::kScaled, true>(d, g, c, sh);
        } else {
            // u = j / rho at the four neighbours, B as stored
            const R* m0 = mom;
            const R ixp = R(1) / m0[xp], ixm = R(1) / m0[xm], iyp = R(1) / m0[yp],
                    iym = R(1) / m0[ym];
            R gu[2][2], gb[2][2], taus[2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const R* mj = mom + (1 + a) * ps;
                const R* mb = mom + (3 + a) * ps;
                gu[a][0] = R(0.5) * (mj[xp] * ixp - mj[xm] * ixm);
                gu[a][1] = R(0.5) * (mj[yp] * iyp - mj[ym] * iym);
                gb[a][0] = R(0.5) * (mb[xp] - mb[xm]);
                gb[a][1] = R(0.5) * (mb[yp] - mb[ym]);
            }
            carati_taus<R>(gu, gb, c.cd2, c.tn, c.te, taus);
            collide<R, Fmt<P>::kScaled, false, true>(d, g, c, taus);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) dst[i * ps + node] = Fmt<P>::enc(d[i], i, 1.0f);
#pragma unroll
        for (int q = 0; q < 10; ++q) dst[(9 + q) * ps + node] = Fmt<P>::enc(g[q], 9 + q, 1.0f);
    }
}

unsigned kin_grid(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65535LL * 8 ? 65535LL * 8 : b));
}

template <int P>
cudaError_t launch_p(const void* src, void* dst, void* mom, const Geom& g, const HostColl& hc,
                     cudaStream_t st) {
    auto step = hc.kin == 3 ? step_kin_kernel<P, 3> : step_kin_kernel<P, 2>;
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    const long long n = (long long)g.nx * g.ny;
    kin_moments_kernel<P><<<kin_grid(n), 256, 0, st>>>((const S*)src, (R*)mom, g.nx, g.ny, g.ps,
                                                       hc.inv_scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    step<<<kin_grid(n), 256, 0, st>>>((const S*)src, (S*)dst, (const R*)mom, g.nx, g.ny, g.ps,
                                      coll_for_prec<R>(hc, P));
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_kinetic(int prec, const void* src, void* dst, void* mom, const Geom& g,
                                const HostColl& c, cudaStream_t st) {
    switch (prec) {
        case P_FP64: return launch_p<P_FP64>(src, dst, mom, g, c, st);
        case P_FP32: return launch_p<P_FP32>(src, dst, mom, g, c, st);
        case P_FP32_DEV: return launch_p<P_FP32_DEV>(src, dst, mom, g, c, st);
        case P_FP16_DEV: return launch_p<P_FP16_DEV>(src, dst, mom, g, c, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbmhd
