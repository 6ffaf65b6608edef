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
// The default is a fused one-pass kernel (below) with the same arithmetic.
// This file is compiled without FMA contraction (-fmad=false), so that the
// two kernels, whose code is shaped differently, round every operation the
// same way and give the same bits.
#include "lbmhd_batch_run.cuh"
#include "lbmhd_internal.h"
#include "lbmhd_step_body.cuh"

namespace lbmhd {

namespace {

__device__ __forceinline__ int wrapk(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// One node of the moments pass: rho, jx, jy, Bx, By of the populations
// streamed into node `node` (pull + sums), into the five planes of mom.
template <int P>
__device__ __forceinline__ void kin_moments_node(const typename Fmt<P>::S* __restrict__ src,
                                                 typename Fmt<P>::R* __restrict__ mom, int nx,
                                                 int ny, long long ps, long long node,
                                                 float inv_s) {
    using R = typename Fmt<P>::R;
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

// One node of the step: pull, central differences of the moment planes at
// x +- 1, y +- 1, then the filtered-equilibrium collision (MODE 2) or the
// cross-helicity closure's relaxation times (MODE 3).
template <int P, int MODE>
__device__ __forceinline__ void kin_step_node(const typename Fmt<P>::S* __restrict__ src,
                                              typename Fmt<P>::S* __restrict__ dst,
                                              const typename Fmt<P>::R* __restrict__ mom, int nx,
                                              int ny, long long ps, long long node,
                                              const Coll<typename Fmt<P>::R>& c) {
    using R = typename Fmt<P>::R;
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
        collide_xf<R, Fmt<P>::kScaled, true>(d, g, c, sh);
    } else {
        // u = j / rho at the four neighbours, B as stored
        const R* m0 = mom;
        const R ixp = recip(m0[xp]), ixm = recip(m0[xm]), iyp = recip(m0[yp]),
                iym = recip(m0[ym]);
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
        collide_xf<R, Fmt<P>::kScaled, false, true>(d, g, c, taus);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) dst[i * ps + node] = Fmt<P>::enc(d[i], i, 1.0f);
#pragma unroll
    for (int q = 0; q < 10; ++q) dst[(9 + q) * ps + node] = Fmt<P>::enc(g[q], 9 + q, 1.0f);
}

// Moments of the rows ra, ra + 1, ..., ra + nrows - 1 (periodic; ra >= -1).
template <int P>
__global__ void __launch_bounds__(256) kin_moments_kernel(const typename Fmt<P>::S* __restrict__ src,
                                                          typename Fmt<P>::R* __restrict__ mom,
                                                          int nx, int ny, long long ps,
                                                          float inv_s, int ra, int nrows) {
    const long long n = (long long)nx * nrows;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(t / nx);
        const long long node = (long long)wrapk(ra + r, ny) * nx + (t - (long long)r * nx);
        kin_moments_node<P>(src, mom, nx, ny, ps, node, inv_s);
    }
}

// The step of rows y0 .. y0 + nrows - 1.
template <int P, int MODE>
__global__ void __launch_bounds__(256) step_kin_kernel(const typename Fmt<P>::S* __restrict__ src,
                                                       typename Fmt<P>::S* __restrict__ dst,
                                                       const typename Fmt<P>::R* __restrict__ mom,
                                                       int nx, int ny, long long ps,
                                                       Coll<typename Fmt<P>::R> c, int y0,
                                                       int nrows) {
    const long long n = (long long)nx * nrows, base = (long long)y0 * nx;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
         t += (long long)gridDim.x * blockDim.x)
        kin_step_node<P, MODE>(src, dst, mom, nx, ny, ps, base + t, c);
}

// ---- fused one-pass variant -------------------------------------------------
// A CTA owns a strip of SW columns [x0, x0 + sw) and a segment of rows
// [y0, y1), and sweeps down it, keeping the conserved moments of the
// populations streamed into consecutive rows (the sw strip nodes and the
// two periodic halo columns x0 - 1, x0 + sw) in a ring of 5 rows in shared
// memory.  Per row y: phase A pulls the populations of row y + 1 and forms
// their moments, a barrier, then phase B collides row y with the central
// differences from the ring and the populations phase A pulled one row
// earlier, kept in registers.  Every stored value is read from DRAM once,
// so the step moves the 152 B/node (FP32) of a plain step instead of the
// two-pass 268 B.  Ring of 5 rows: phase A of row y + 2 (slot j + 3) may
// run while a slower thread still reads rows y - 1 .. y + 1 (slots j ..
// j + 2) in phase B, and no thread gets further ahead without passing the
// next barrier.  Moments, differences and collision are the arithmetic of
// the two-pass kernels, so both give the same bits.
//
// Addressing: plane p starts at base + p * ps; inside a plane a node is a
// 32-bit offset y * nx + x (a lattice has at most 2^30 nodes).
// U2: the row loop is unrolled by two with the kept populations in two
// register sets used alternately, so no per-row copies of the 19 values.
// Measured on GB300 at 8192^2, FP32, MLUPS (fraction of the measured copy
// bandwidth at 152 B/node): les 2 with U2 38.8K (0.87), without 33.4K; les 3
// without 38.4K (0.86), with 36.4K -- the register schedule decides, so the
// choice is per closure.
constexpr int kRing = 5;

template <int P>
__device__ __forceinline__ void sum_moments(const typename Fmt<P>::R (&d)[kPlanes], float inv_s,
                                            typename Fmt<P>::R (&m)[5]) {
    using R = typename Fmt<P>::R;
    R drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    R jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    R jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    R bx = (d[9] + d[11]) + (d[13] + d[15]) + d[17];
    R by = (d[10] + d[12]) + (d[14] + d[16]) + d[18];
    if (Fmt<P>::kScaled) {
        drho *= (R)inv_s;
        jx *= (R)inv_s;
        jy *= (R)inv_s;
        bx *= (R)inv_s;
        by *= (R)inv_s;
    }
    m[0] = R(1) + drho;
    m[1] = jx;
    m[2] = jy;
    m[3] = bx;
    m[4] = by;
}

// The work of one CTA of SW + 32 threads on one strip-segment of one lattice
// (src, dst: 19 planes of stride ps).  ring: the CTA's shared moment rows.
template <int P, int MODE, int SW, bool U2>
__device__ __forceinline__ void kin_fused_body(
    const typename Fmt<P>::S* __restrict__ src, typename Fmt<P>::S* __restrict__ dst,
    long long ps, int nx, int ny, int x0, int y0, int y1, const Coll<typename Fmt<P>::R>& c,
    float inv_s, typename Fmt<P>::R (*ring)[5][SW + 2]) {
    using R = typename Fmt<P>::R;
    const int tid = threadIdx.x;
    const int sw = min(SW, nx - x0);
    // moment position of this thread: strip node, left halo, right halo
    int pos = -1, xm = 0;
    if (tid < sw) {
        pos = tid + 1;
        xm = x0 + tid;
    } else if (tid == sw) {
        pos = 0;
        xm = wrapk(x0 - 1, nx);
    } else if (tid == sw + 1) {
        pos = sw + 1;
        xm = wrapk(x0 + sw, nx);
    }
    const unsigned xw = (unsigned)wrapk(xm - 1, nx), xe = (unsigned)wrapk(xm + 1, nx);
    // populations streamed into (xm, yy): plane p from (xm - c_px, yy - c_py)
    auto pull = [&](int yy, R (&v)[kPlanes]) {
        const unsigned rm = (unsigned)wrapk(yy - 1, ny) * (unsigned)nx;
        const unsigned r0 = (unsigned)yy * (unsigned)nx;
        const unsigned rp = (unsigned)wrapk(yy + 1, ny) * (unsigned)nx;
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const int cx = plane_cx(p), cy = plane_cy(p);
            const unsigned row = cy == 0 ? r0 : (cy > 0 ? rm : rp);
            const unsigned col = cx == 0 ? (unsigned)xm : (cx > 0 ? xw : xe);
            v[p] = Fmt<P>::dec(src[p * ps + (row + col)], p, 1.0f);
        }
    };
    // phase A: pulled populations of (xm, yy) into v, their moments into a slot
    auto phase_a = [&](int yy, int slot, R (&v)[kPlanes]) {
        if (pos < 0) return;
        pull(wrapk(yy, ny), v);
        R m[5];
        sum_moments<P>(v, inv_s, m);
#pragma unroll
        for (int q = 0; q < 5; ++q) ring[slot][q][pos] = m[q];
    };
    // phase B: collide node (x0 + tid, y), pulled populations in v, with the
    // moment rows y - 1, y, y + 1 in slots sm, s0, sp
    auto phase_b = [&](int y, int sm, int s0, int sp, const R (&v)[kPlanes]) {
        const int i = tid + 1;
        R d[9], g[10];
#pragma unroll
        for (int p = 0; p < 9; ++p) d[p] = v[p];
#pragma unroll
        for (int q = 0; q < 10; ++q) g[q] = v[9 + q];
        if (MODE == 2) {
            R fld[5], gx[5], gy[5], sh[4];
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                fld[q] = ring[s0][q][i];
                gx[q] = R(0.5) * (ring[s0][q][i + 1] - ring[s0][q][i - 1]);
                gy[q] = R(0.5) * (ring[sp][q][i] - ring[sm][q][i]);
            }
            filtered_shift<R>(fld, gx, gy, c.d2, sh);
            if (Fmt<P>::kScaled)
#pragma unroll
                for (int q = 0; q < 4; ++q) sh[q] *= c.scl;
            collide_xf<R, Fmt<P>::kScaled, true>(d, g, c, sh);
        } else {
            const R ixp = recip(ring[s0][0][i + 1]), ixm = recip(ring[s0][0][i - 1]),
                    iyp = recip(ring[sp][0][i]), iym = recip(ring[sm][0][i]);
            R gu[2][2], gb[2][2], taus[2];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                gu[a][0] = R(0.5) * (ring[s0][1 + a][i + 1] * ixp - ring[s0][1 + a][i - 1] * ixm);
                gu[a][1] = R(0.5) * (ring[sp][1 + a][i] * iyp - ring[sm][1 + a][i] * iym);
                gb[a][0] = R(0.5) * (ring[s0][3 + a][i + 1] - ring[s0][3 + a][i - 1]);
                gb[a][1] = R(0.5) * (ring[sp][3 + a][i] - ring[sm][3 + a][i]);
            }
            carati_taus<R>(gu, gb, c.cd2, c.tn, c.te, taus);
            collide_xf<R, Fmt<P>::kScaled, false, true>(d, g, c, taus);
        }
        const unsigned node = (unsigned)y * (unsigned)nx + (unsigned)xm;
#pragma unroll
        for (int q = 0; q < 9; ++q) dst[q * ps + node] = Fmt<P>::enc(d[q], q, 1.0f);
#pragma unroll
        for (int q = 0; q < 10; ++q) dst[(9 + q) * ps + node] = Fmt<P>::enc(g[q], 9 + q, 1.0f);
    };
    R va[kPlanes], vb[kPlanes];
    phase_a(y0 - 1, 0, va);
    phase_a(y0, 1, va);
    // one row: moments of row y + 1 (pulled into nxt), barrier, collide row
    // y (pulled into cur one row earlier)
    auto row = [&](int y, int j, R (&cur)[kPlanes], R (&nxt)[kPlanes]) {
        phase_a(y + 1, (j + 2) % kRing, nxt);
        __syncthreads();
        if (tid < sw) phase_b(y, j % kRing, (j + 1) % kRing, (j + 2) % kRing, cur);
    };
    if (U2) {
        int y = y0, j = 0;
        for (; y + 1 < y1; y += 2, j += 2) {
            row(y, j, va, vb);
            row(y + 1, j + 1, vb, va);
        }
        if (y < y1) row(y, j, va, vb);
    } else {
        for (int y = y0, j = 0; y < y1; ++y, ++j) {
            row(y, j, va, vb);
#pragma unroll
            for (int p = 0; p < kPlanes; ++p) va[p] = vb[p];
        }
    }
}

// Rows [ya, yb) of the lattice, cut into segments of seglen rows.
template <int P, int MODE, int SW, int MINB, bool U2>
__global__ void __launch_bounds__(SW + 32, MINB) step_kin_fused_kernel(
    const typename Fmt<P>::S* __restrict__ src, typename Fmt<P>::S* __restrict__ dst, int nx,
    int ny, long long ps, int ya, int yb, int seglen, Coll<typename Fmt<P>::R> c, float inv_s) {
    using R = typename Fmt<P>::R;
    __shared__ R ring[kRing][5][SW + 2];
    const int y0 = ya + blockIdx.y * seglen;
    kin_fused_body<P, MODE, SW, U2>(src, dst, ps, nx, ny, blockIdx.x * SW, y0,
                                    min(y0 + seglen, yb), c, inv_s, ring);
}

// Fused-kernel shape per format: strip width SW (FP64 and FF hold twice the
// registers per value), CTAs per SM the register budget is sized for, and
// the two-row unroll for the filtered equilibria (les 2).
template <int P>
struct FusedShape {
    static constexpr bool kWide = P == P_FP64 || P == P_FF;
    static constexpr int SW = kWide ? 128 : 256;
    static constexpr int MINB = kWide ? 2 : 3;
};

// Row segments per strip for about four waves of resident CTAs; each
// segment forms two moment rows again.
inline int fused_seglen(int nx, int ny, int sw, int minb, int sm_count) {
    const int nstrips = (nx + sw - 1) / sw;
    const long long want = 4LL * minb * (sm_count > 0 ? sm_count : 1);
    long long nseg = (want + nstrips - 1) / nstrips;
    if (nseg > ny) nseg = ny;
    if (nseg < 1) nseg = 1;
    return (int)((ny + nseg - 1) / nseg);
}

template <int P>
cudaError_t launch_fused(const void* src, void* dst, const Geom& g, const HostColl& hc,
                         int sm_count, cudaStream_t st, int y0, int y1) {
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    constexpr int SW = FusedShape<P>::SW, MINB = FusedShape<P>::MINB;
    const int nstrips = (g.nx + SW - 1) / SW;
    const int rows = y1 - y0;
    const int seglen = fused_seglen(g.nx, rows, SW, MINB, sm_count);
    const int nseg = (rows + seglen - 1) / seglen;
    const dim3 grid((unsigned)nstrips, (unsigned)nseg);
    auto k = hc.kin == 3 ? step_kin_fused_kernel<P, 3, SW, MINB, false>
                         : step_kin_fused_kernel<P, 2, SW, MINB, true>;
    k<<<grid, SW + 32, 0, st>>>((const S*)src, (S*)dst, g.nx, g.ny, g.ps, y0, y1, seglen,
                                coll_for_prec<R>(hc, P), hc.inv_scale);
    return cudaGetLastError();
}

// ---- ensembles -------------------------------------------------------------
// One CTA per work unit of an ensemble (a unit belongs to one run; the
// ensemble's unit map gives the run), one node per thread: the moments pass
// and the step of the two-pass kernels, node for node, so every run evolves
// bit-identically to its own lattice.
template <int P>
__global__ void __launch_bounds__(256) batch_kin_moments_kernel(
    const RunDev<typename Fmt<P>::R>* __restrict__ runs, const int* __restrict__ unit_run,
    const typename Fmt<P>::S* __restrict__ src, typename Fmt<P>::R* __restrict__ mom, float inv_s) {
    const RunDev<typename Fmt<P>::R>& rd = runs[unit_run[blockIdx.x]];
    const unsigned t = (blockIdx.x - rd.unit0) * blockDim.x + threadIdx.x;
    if (t < rd.total) kin_moments_node<P>(src + rd.off, mom + rd.moff, rd.nx, rd.ny, rd.ps, t, inv_s);
}

template <int P, int MODE>
__global__ void __launch_bounds__(256) batch_kin_step_kernel(
    const RunDev<typename Fmt<P>::R>* __restrict__ runs, const int* __restrict__ unit_run,
    const typename Fmt<P>::S* __restrict__ src, typename Fmt<P>::S* __restrict__ dst,
    const typename Fmt<P>::R* __restrict__ mom) {
    const RunDev<typename Fmt<P>::R>& rd = runs[unit_run[blockIdx.x]];
    const unsigned t = (blockIdx.x - rd.unit0) * blockDim.x + threadIdx.x;
    if (t < rd.total)
        kin_step_node<P, MODE>(src + rd.off, dst + rd.off, mom + rd.moff, rd.nx, rd.ny, rd.ps, t,
                               rd.c);
}

// The fused kernel over an ensemble: one CTA per work unit, a unit being one
// strip-segment of one run (unit_run gives the run; the unit's place in the
// run's strips x segments follows from the run's first unit), so every run
// evolves bit-identically to its own lattice.
template <int P, int MODE, int SW, int MINB, bool U2>
__global__ void __launch_bounds__(SW + 32, MINB) batch_kin_fused_kernel(
    const RunDev<typename Fmt<P>::R>* __restrict__ runs, const int* __restrict__ unit_run,
    const typename Fmt<P>::S* __restrict__ src, typename Fmt<P>::S* __restrict__ dst,
    float inv_s) {
    using R = typename Fmt<P>::R;
    __shared__ R ring[kRing][5][SW + 2];
    const RunDev<R>& rd = runs[unit_run[blockIdx.x]];
    const int l = (int)(blockIdx.x - rd.unit0);
    const int strip = l % rd.kstrips, seg = l / rd.kstrips;
    const int y0 = seg * rd.kseglen;
    kin_fused_body<P, MODE, SW, U2>(src + rd.off, dst + rd.off, rd.ps, rd.nx, rd.ny, strip * SW,
                                    y0, min(y0 + rd.kseglen, rd.ny), rd.c, inv_s, ring);
}

template <int P>
cudaError_t launch_batch_p(int kin, bool fused, const void* runs, const int* unit_run,
                           unsigned nunits, int block, const void* src, void* dst, void* mom,
                           float inv_s, cudaStream_t st) {
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    const RunDev<R>* rd = (const RunDev<R>*)runs;
    if (fused) {
        constexpr int SW = FusedShape<P>::SW, MINB = FusedShape<P>::MINB;
        auto k = kin == 3 ? batch_kin_fused_kernel<P, 3, SW, MINB, false>
                          : batch_kin_fused_kernel<P, 2, SW, MINB, true>;
        k<<<nunits, SW + 32, 0, st>>>(rd, unit_run, (const S*)src, (S*)dst, inv_s);
        return cudaGetLastError();
    }
    batch_kin_moments_kernel<P><<<nunits, block, 0, st>>>(rd, unit_run, (const S*)src, (R*)mom,
                                                          inv_s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    auto step = kin == 3 ? batch_kin_step_kernel<P, 3> : batch_kin_step_kernel<P, 2>;
    step<<<nunits, block, 0, st>>>(rd, unit_run, (const S*)src, (S*)dst, (const R*)mom);
    return cudaGetLastError();
}

unsigned kin_grid(long long n) {
    long long b = (n + 255) / 256;
    return (unsigned)(b < 1 ? 1 : (b > 65535LL * 8 ? 65535LL * 8 : b));
}

template <int P>
cudaError_t launch_p(const void* src, void* dst, void* mom, const Geom& g, const HostColl& hc,
                     cudaStream_t st, int y0, int y1) {
    auto step = hc.kin == 3 ? step_kin_kernel<P, 3> : step_kin_kernel<P, 2>;
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    // moments of rows y0 - 1 .. y1 (the whole lattice when that covers it)
    int ra = y0 - 1, mrows = y1 - y0 + 2;
    if (mrows >= g.ny) {
        ra = 0;
        mrows = g.ny;
    }
    kin_moments_kernel<P><<<kin_grid((long long)g.nx * mrows), 256, 0, st>>>(
        (const S*)src, (R*)mom, g.nx, g.ny, g.ps, hc.inv_scale, ra, mrows);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    step<<<kin_grid((long long)g.nx * (y1 - y0)), 256, 0, st>>>(
        (const S*)src, (S*)dst, (const R*)mom, g.nx, g.ny, g.ps, coll_for_prec<R>(hc, P), y0,
        y1 - y0);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_kinetic(int prec, int kin, bool fused, const void* runs,
                                 const int* unit_run, unsigned nunits, int block, const void* src,
                                 void* dst, void* mom, float inv_s, cudaStream_t st) {
#define LBMHD_KB(P)                                                                             \
    case P:                                                                                     \
        return launch_batch_p<P>(kin, fused, runs, unit_run, nunits, block, src, dst, mom, inv_s, \
                                 st);
    switch (prec) {
        LBMHD_KB(P_FP64)
        LBMHD_KB(P_FP32)
        LBMHD_KB(P_FP32_DEV)
        LBMHD_KB(P_FP16_DEV)
        LBMHD_KB(P_FF)
    }
#undef LBMHD_KB
    return cudaErrorInvalidValue;
}

int kinetic_fused_strip(int prec) {
    switch (prec) {
        case P_FP64: return FusedShape<P_FP64>::SW;
        case P_FF: return FusedShape<P_FF>::SW;
        case P_FP32: return FusedShape<P_FP32>::SW;
        case P_FP32_DEV: return FusedShape<P_FP32_DEV>::SW;
        case P_FP16_DEV: return FusedShape<P_FP16_DEV>::SW;
    }
    return 0;
}

cudaError_t launch_step_kinetic(int prec, bool two_pass, int sm_count, const void* src,
                                void* dst, void* mom, const Geom& g, const HostColl& c,
                                cudaStream_t st, int y0, int y1) {
    if (y1 < 0) y1 = g.ny;
    if (!two_pass) {
        switch (prec) {
            case P_FP64: return launch_fused<P_FP64>(src, dst, g, c, sm_count, st, y0, y1);
            case P_FP32: return launch_fused<P_FP32>(src, dst, g, c, sm_count, st, y0, y1);
            case P_FP32_DEV: return launch_fused<P_FP32_DEV>(src, dst, g, c, sm_count, st, y0, y1);
            case P_FP16_DEV: return launch_fused<P_FP16_DEV>(src, dst, g, c, sm_count, st, y0, y1);
            case P_FF: return launch_fused<P_FF>(src, dst, g, c, sm_count, st, y0, y1);
        }
        return cudaErrorInvalidValue;
    }
    switch (prec) {
        case P_FP64: return launch_p<P_FP64>(src, dst, mom, g, c, st, y0, y1);
        case P_FP32: return launch_p<P_FP32>(src, dst, mom, g, c, st, y0, y1);
        case P_FP32_DEV: return launch_p<P_FP32_DEV>(src, dst, mom, g, c, st, y0, y1);
        case P_FP16_DEV: return launch_p<P_FP16_DEV>(src, dst, mom, g, c, st, y0, y1);
        case P_FF: return launch_p<P_FF>(src, dst, mom, g, c, st, y0, y1);
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbmhd
