// lbmhd_adjoint.cu -- the hand-written discrete adjoint of the fused
// stream-collide step, and its checkpointed driver.
//
// A step maps the stored state x_t to x_{t+1} = C(S(x_t)) node by node:
// S pulls f_i from x - c_i and g_k from x - C_k, C is the collision
// (collide() in lbmhd_device.cuh).  Its transpose Jacobian applied to an
// adjoint lambda_{t+1} is, per node y,
//     mu(y) = J_C(z(y))^T lambda_{t+1}(y),   z(y) = S(x_t)(y),
// followed by the transpose of the pull, a push:
//     lambda_t,p(y - c_p) = mu_p(y).
// One kernel does both: it pulls z from x_t like the forward step,
// recomputes the collision's intermediates in registers, runs their
// derivatives in reverse order (collide_adjoint) and scatters mu.  The
// same pass accumulates the parameter sensitivities lambda . dC/d(tau_nu,
// tau_eta, 18 C_S Delta^2, 36 C_S Delta^2) in FP64 (per-block partial sums,
// then a fixed-order reduction: deterministic).
//
// The derivative of |x| and of sqrt at 0 (the local strain and current
// magnitudes Q and J) is taken as 0.  The forward intermediates are
// recomputed with the same reciprocal and square root as the forward step.
//
// Driver: lbmhd_adjoint_record runs the forward from given fields keeping
// FP64 checkpoints every K steps; lbmhd_adjoint_backward seeds lambda_T
// from the gradient of the final moments, then walks the segments in
// reverse: restore the checkpoint, recompute the segment's states with the
// forward kernel (bit-identical to the recorded run), and apply the
// adjoint step backwards through them.  Finally lambda_0 goes through the
// Jacobian of the equilibrium initialisation to the initial fields.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include <type_traits>

#include "lbmhd_internal.h"
#include "lbmhd_step_body.cuh"

namespace lbmhd {

// Reverse-mode derivative of collide<R> at the pulled node state (d, g):
// given the adjoint (ld, lg) of the outputs, returns the adjoint (md, mg)
// of the inputs and th = d/d(tau_nu, tau_eta, k18, k36) of lambda . C.
// a / b in the arithmetic type: IEEE division for float and double, the
// double-word reciprocal for double-word; and a value as FP64.
template <class R>
__device__ __forceinline__ R quot(R a, R b) {
    return a / b;
}
__device__ __forceinline__ ff quot(ff a, ff b) { return a * rcp(b); }
__device__ __forceinline__ double to_f64(float v) { return v; }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(ff v) { return (double)v.hi + (double)v.lo; }

template <class R>
__device__ __forceinline__ void collide_adjoint(const R (&d)[9], const R (&g)[10],
                                                const R (&ld)[9], const R (&lg)[10],
                                                const Coll<R>& c, R (&md)[9], R (&mg)[10],
                                                R (&th)[4]) {
    // ---- forward intermediates (same expressions as collide) -------------
    const R drho = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const R jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    const R jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    const R rho = R(1) + drho;
    const R irho = rcp(rho);
    const R ux = jx * irho, uy = jy * irho;
    const R bx = (g[0] + g[2]) + (g[4] + g[6]) + g[8];
    const R by = (g[1] + g[3]) + (g[5] + g[7]) + g[9];
    const R dsum = (d[5] + d[6]) + (d[7] + d[8]);
    const R m3 = (d[5] - d[6]) + (d[7] - d[8]);
    const R m4 = (d[1] + d[3]) - (d[2] + d[4]);
    const R m5 = R(2) * (d[3] - d[1]) + (d[5] - d[6]) + (d[8] - d[7]);
    const R m6 = R(2) * (d[4] - d[2]) + (d[5] + d[6]) - (d[7] + d[8]);
    const R m7 = R(4) * d[0] - R(5) * ((d[1] + d[2]) + (d[3] + d[4])) + R(4) * dsum;
    const R m8 = R(4) * d[0] - dsum;
    const R j2 = jx * jx + jy * jy;
    const R j2i = j2 * irho;
    const R n3 = m3 - (jx * jy * irho - bx * by);
    const R n4 = m4 - ((jx * jx - jy * jy) * irho - bx * bx + by * by);
    const R n5 = m5 + jx;
    const R n6 = m6 + jy;
    const R n7 = m7 + R(3) * j2i;
    const R n8 = m8 - (R(5) / R(3) * drho - R(3) * j2i);
    const R E = ux * by - uy * bx;
    R tau_e = c.tn, tau_m = c.te, Q = R(0), rA = R(1), X = R(0), J = R(0), rB = R(1);
    if (c.les) {
        Q = sqrt_(n4 * n4 + R(4) * (n3 * n3));
        rA = sqrt_(c.tn2 + c.k18 * Q * irho);
        tau_e = R(0.5) * (c.tn + rA);
        X = (g[3] - g[7]) - (g[4] - g[8]) - R(2) * E;
        J = fabs(X);
        rB = sqrt_(c.te2 + c.k36 * J);
        tau_m = R(0.5) * (c.te + rB);
    }
    const R snu = rcp(tau_e);
    const bool t7 = !(c.s7 > R(0)), t8 = !(c.s8 > R(0));
    const R s7 = t7 ? snu : c.s7;
    const R s8 = t8 ? snu : c.s8;
    const R sm = rcp(tau_m);
    const R third = R(1) / R(3), sixth = R(1) / R(6);
    const R e3 = R(3) * E;
    const R geq[10] = {third * bx,        third * by,        sixth * bx,        sixth * (by + e3),
                       sixth * (bx - e3), sixth * by,        sixth * bx,        sixth * (by - e3),
                       sixth * (bx + e3), sixth * by};

    // ---- reverse sweep ----------------------------------------------------
    // magnetic: g' = (1 - sm) g + sm g^eq
    R smb = R(0), gq[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) {
        mg[q] = (R(1) - sm) * lg[q];
        smb += lg[q] * (geq[q] - g[q]);
        gq[q] = sm * lg[q];
    }
    R bxb = third * gq[0] + sixth * ((gq[2] + gq[4]) + (gq[6] + gq[8]));
    R byb = third * gq[1] + sixth * ((gq[3] + gq[5]) + (gq[7] + gq[9]));
    R Eb = R(0.5) * ((gq[3] - gq[4]) - (gq[7] - gq[8]));

    // density: d' = d - sum_j a_j T_j, so a_j-bar = -T_j . ld
    const R lsum = (ld[5] + ld[6]) + (ld[7] + ld[8]);
    const R ab3 = -((ld[5] - ld[6]) + (ld[7] - ld[8]));
    const R ab4 = -((ld[1] + ld[3]) - (ld[2] + ld[4]));
    const R ab5 = -(R(2) * (ld[3] - ld[1]) + (ld[5] - ld[6]) + (ld[8] - ld[7]));
    const R ab6 = -(R(2) * (ld[4] - ld[2]) + (ld[5] + ld[6]) - (ld[7] + ld[8]));
    const R ab7 = -(R(4) * ld[0] - R(5) * ((ld[1] + ld[2]) + (ld[3] + ld[4])) + R(4) * lsum);
    const R ab8 = -(R(4) * ld[0] - lsum);
#pragma unroll
    for (int i = 0; i < 9; ++i) md[i] = ld[i];

    // a3 = snu n3/4, a4 = snu n4/4, a5 = s5 n5/12, a6 = s6 n6/12,
    // a7 = s7 n7/180, a8 = s8 n8/20
    R snub = R(0.25) * (ab3 * n3 + ab4 * n4);
    R nb3 = R(0.25) * ab3 * snu;
    R nb4 = R(0.25) * ab4 * snu;
    const R nb5 = ab5 * c.s5 * (R(1) / R(12));
    const R nb6 = ab6 * c.s6 * (R(1) / R(12));
    const R nb7 = ab7 * s7 * (R(1) / R(180));
    const R nb8 = ab8 * s8 * (R(1) / R(20));
    const R s5b = ab5 * n5 * (R(1) / R(12));
    const R s6b = ab6 * n6 * (R(1) / R(12));
    const R s7b = ab7 * n7 * (R(1) / R(180));
    const R s8b = ab8 * n8 * (R(1) / R(20));
    if (t7) snub += s7b;
    if (t8) snub += s8b;
    R tnb = R(0), teb = R(0), k18b = R(0), k36b = R(0);
    if (c.tie5) tnb -= s5b * c.s5 * c.s5;  // s5 = 1/tau_nu
    if (c.tie6) tnb -= s6b * c.s6 * c.s6;
    const R taueb = -snub * snu * snu;      // snu = 1/tau_e
    const R taumb = -smb * sm * sm;         // sm = 1/tau_m
    R irhob = R(0);
    if (c.les) {
        // tau_m = (te + sqrt(te^2 + k36 J)) / 2
        teb += R(0.5) * taumb;
        const R Bb = quot(taumb * R(0.25), rB);
        teb += Bb * R(2) * c.te;
        k36b += Bb * J;
        const R Jb = Bb * c.k36;
        const R Xb = X > R(0) ? Jb : (X < R(0) ? -Jb : R(0));
        mg[3] += Xb;
        mg[7] -= Xb;
        mg[4] -= Xb;
        mg[8] += Xb;
        Eb -= R(2) * Xb;
        // tau_e = (tn + sqrt(tn^2 + k18 Q / rho)) / 2
        tnb += R(0.5) * taueb;
        const R Ab = quot(taueb * R(0.25), rA);
        tnb += Ab * R(2) * c.tn;
        k18b += Ab * Q * irho;
        const R Qb = Ab * c.k18 * irho;
        irhob += Ab * c.k18 * Q;
        if (Q > R(0)) {
            nb4 += quot(Qb * n4, Q);
            nb3 += quot(Qb * R(4) * n3, Q);
        }
    } else {
        tnb += taueb;
        teb += taumb;
    }
    // E = ux by - uy bx
    R uxb = Eb * by, uyb = -Eb * bx;
    byb += Eb * ux;
    bxb -= Eb * uy;
    // n8 = m8 - 5/3 drho + 3 j2i ; n7 = m7 + 3 j2i ; n6 = m6 + jy ; n5 = m5 + jx
    R drhob = -(R(5) / R(3)) * nb8;
    R j2ib = R(3) * (nb8 + nb7);
    R jxb = nb5, jyb = nb6;
    // n4 = m4 - (jx^2 - jy^2) irho + bx^2 - by^2
    jxb -= R(2) * jx * irho * nb4;
    jyb += R(2) * jy * irho * nb4;
    irhob -= (jx * jx - jy * jy) * nb4;
    bxb += R(2) * bx * nb4;
    byb -= R(2) * by * nb4;
    // n3 = m3 - jx jy irho + bx by
    jxb -= jy * irho * nb3;
    jyb -= jx * irho * nb3;
    irhob -= jx * jy * nb3;
    bxb += by * nb3;
    byb += bx * nb3;
    // j2i = (jx^2 + jy^2) irho
    jxb += R(2) * jx * irho * j2ib;
    jyb += R(2) * jy * irho * j2ib;
    irhob += j2 * j2ib;
    // ux = jx irho, uy = jy irho
    jxb += uxb * irho;
    jyb += uyb * irho;
    irhob += uxb * jx + uyb * jy;
    // irho = 1 / (1 + drho)
    drhob -= irho * irho * irhob;
    // m_j = T_j . d (j = 3..8), drho = sum d, jx, jy
    const R mb3 = nb3, mb4 = nb4, mb5 = nb5, mb6 = nb6, mb7 = nb7, mb8 = nb8;
    const R q78 = R(4) * mb7 - mb8;
    md[0] += R(4) * (mb7 + mb8) + drhob;
    md[1] += mb4 - R(2) * mb5 - R(5) * mb7 + drhob + jxb;
    md[2] += -mb4 - R(2) * mb6 - R(5) * mb7 + drhob + jyb;
    md[3] += mb4 + R(2) * mb5 - R(5) * mb7 + drhob - jxb;
    md[4] += -mb4 + R(2) * mb6 - R(5) * mb7 + drhob - jyb;
    md[5] += (mb3 + mb5) + (mb6 + q78) + drhob + jxb + jyb;
    md[6] += (mb6 - mb3) - (mb5 - q78) + drhob - jxb + jyb;
    md[7] += (mb3 - mb5) - (mb6 - q78) + drhob - jxb - jyb;
    md[8] += (mb5 - mb3) - (mb6 - q78) + drhob + jxb - jyb;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        mg[2 * k] += bxb;
        mg[2 * k + 1] += byb;
    }
    th[0] = tnb;
    th[1] = teb;
    th[2] = k18b;
    th[3] = k36b;
}

namespace {

constexpr int kAdjBlock = 256;
// Grid of at most 8 blocks per SM of a 152-SM GB300 (two resident at 114
// registers, four waves): each thread sweeps many nodes, so its one final
// conversion and warp reduction of the sensitivity sums stays small.
constexpr int kAdjMaxBlocks = 8 * 152;

__device__ __forceinline__ int wrapi(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One adjoint step.  x: stored state before the forward step (19 planes of
// storage type S); lin: lambda_{t+1}; lout: lambda_t (type R, same plane
// stride).  partials: 4 doubles per block, summed over the steps of a
// backward sweep -- each block adds into its own slot and the steps run in
// order on one stream, so the sums are deterministic; one reduction over
// the blocks follows the sweep.
template <int P>
__global__ void __launch_bounds__(kAdjBlock) adj_step_kernel(
    const typename Fmt<P>::S* __restrict__ x, const typename Fmt<P>::R* __restrict__ lin,
    typename Fmt<P>::R* __restrict__ lout, int nx, int ny, long long ps,
    Coll<typename Fmt<P>::R> c, float inv_scale, double* __restrict__ partials) {
    using R = typename Fmt<P>::R;
    const long long n = (long long)nx * ny;
    // per-thread sensitivity sums: FP64 for FP64 storage; double-word for
    // the FP32 forms, which keeps FP64 instructions out of the node loop
    using Acc = typename std::conditional<std::is_same<R, double>::value, double, ff>::type;
    Acc acc[4] = {Acc(0), Acc(0), Acc(0), Acc(0)};
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        // lattices hold at most 2^30 nodes: 32-bit division
        const int y = (int)((unsigned)node / (unsigned)nx), xx = (int)node - y * nx;
        R d[9], g[10], ld[9], lg[10], md[9], mg[10], th[4];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const long long src =
                (long long)wrapi(y - plane_cy(p), ny) * nx + wrapi(xx - plane_cx(p), nx);
            const R v = Fmt<P>::dec(x[p * ps + src], p, inv_scale);
            const R l = lin[p * ps + node];
            if (p < 9) {
                d[p] = v;
                ld[p] = l;
            } else {
                g[p - 9] = v;
                lg[p - 9] = l;
            }
        }
        collide_adjoint<R>(d, g, ld, lg, c, md, mg, th);
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const long long dst =
                (long long)wrapi(y - plane_cy(p), ny) * nx + wrapi(xx - plane_cx(p), nx);
            lout[p * ps + dst] = p < 9 ? md[p] : mg[p - 9];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if constexpr (std::is_same<R, float>::value) dw_accumulate(acc[q], th[q]);
            else acc[q] += th[q];
        }
    }
    __shared__ double red[kAdjBlock / 32][4];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        double a;
        a = to_f64(acc[q]);
        const double w = warp_sum_d(a);
        if (lane == 0) red[warp][q] = w;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kAdjBlock / 32; ++w) s += red[w][threadIdx.x];
        partials[(long long)blockIdx.x * 4 + threadIdx.x] += s;  // this block's slot
    }
}

// acc[q] += sum over blocks of partials (fixed order, one block).
__global__ void adj_reduce_kernel(const double* __restrict__ partials, int nblocks, double* acc) {
    __shared__ double red[kAdjBlock / 32][4];
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 4; ++q) a[q] += partials[(long long)b * 4 + q];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double w = warp_sum_d(a[q]);
        if (lane == 0) red[warp][q] = w;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0.0;
        for (int w = 0; w < kAdjBlock / 32; ++w) s += red[w][threadIdx.x];
        acc[threadIdx.x] += s;
    }
}

// lambda_T from the gradient of the final moments (rho, u, B) of state x:
// d rho / d f_i = 1, d u_a / d f_i = (c_ia - u_a) / rho, d B_a / d g_kb = delta_ab.
template <int P>
__global__ void adj_seed_kernel(const typename Fmt<P>::S* __restrict__ x,
                                const double* __restrict__ gr, const double* __restrict__ gux,
                                const double* __restrict__ guy, const double* __restrict__ gbx,
                                const double* __restrict__ gby, typename Fmt<P>::R* lam, int nx,
                                int ny, long long ps, float inv_scale) {
    using R = typename Fmt<P>::R;
    const long long n = (long long)nx * ny;
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        double d[9], drho = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            d[i] = to_f64(Fmt<P>::dec(x[i * ps + node], i, inv_scale));
            drho += d[i];
        }
        const double jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
        const double jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
        const double rho = 1.0 + drho, ux = jx / rho, uy = jy / rho;
        const double a = gr ? gr[node] : 0.0, bu = gux ? gux[node] : 0.0,
                     bv = guy ? guy[node] : 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i)
            lam[i * ps + node] =
                (R)(a + (bu * (plane_cx(i) - ux) + bv * (plane_cy(i) - uy)) / rho);
        const double cbx = gbx ? gbx[node] : 0.0, cby = gby ? gby[node] : 0.0;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            lam[(9 + 2 * k) * ps + node] = (R)cbx;
            lam[(10 + 2 * k) * ps + node] = (R)cby;
        }
    }
}

// lambda_0 through the Jacobian of the equilibrium initialisation (Sec. 3
// equilibria) to d/d(rho0, u0, B0).
template <class R>
__global__ void adj_init_kernel(const R* __restrict__ lam, const double* __restrict__ f0,
                                double* dr, double* dux, double* duy, double* dbx, double* dby,
                                int nx, int ny, long long ps) {
    const long long n = (long long)nx * ny;
    for (long long node = blockIdx.x * (long long)blockDim.x + threadIdx.x; node < n;
         node += (long long)gridDim.x * blockDim.x) {
        const double rho = f0[node], u = f0[n + node], v = f0[2 * n + node];
        const double Bx = f0[3 * n + node], By = f0[4 * n + node];
        const double u2 = u * u + v * v;
        double gr = 0.0, gu = 0.0, gv = 0.0, gbx = 0.0, gby = 0.0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double l = to_f64(lam[i * ps + node]);
            const double cx = plane_cx(i), cy = plane_cy(i), w = plane_rest<double>(i);
            const double cu = cx * u + cy * v, cb = cx * Bx + cy * By, c2 = cx * cx + cy * cy;
            gr += l * w * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u2);
            gu += l * w * rho * (3.0 * cx + 9.0 * cu * cx - 3.0 * u);
            gv += l * w * rho * (3.0 * cy + 9.0 * cu * cy - 3.0 * v);
            gbx += l * 4.5 * w * (Bx * c2 - 2.0 * cb * cx);
            gby += l * 4.5 * w * (By * c2 - 2.0 * cb * cy);
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const int p = 9 + 2 * k;
            const double lx = to_f64(lam[p * ps + node]), ly = to_f64(lam[(p + 1) * ps + node]);
            const double Cx = plane_cx(p), Cy = plane_cy(p), wk = k == 0 ? 1.0 / 3.0 : 1.0 / 6.0;
            const double Cu = Cx * u + Cy * v, CB = Cx * Bx + Cy * By;
            // g_x = wk (Bx + 3 (Cu Bx - CB u)), g_y = wk (By + 3 (Cu By - CB v))
            gu += wk * 3.0 * (lx * (Cx * Bx - CB) + ly * Cx * By);
            gv += wk * 3.0 * (lx * Cy * Bx + ly * (Cy * By - CB));
            gbx += wk * (lx * (1.0 + 3.0 * (Cu - Cx * u)) + ly * (-3.0 * Cx * v));
            gby += wk * (lx * (-3.0 * Cy * u) + ly * (1.0 + 3.0 * (Cu - Cy * v)));
        }
        if (dr) dr[node] = gr;
        if (dux) dux[node] = gu;
        if (duy) duy[node] = gv;
        if (dbx) dbx[node] = gbx;
        if (dby) dby[node] = gby;
    }
}

}  // namespace

// Tape of one recorded forward run (owned by the handle).
struct Tape {
    int nsteps, every, nseg;
    int64_t step_at_end;
    double* fields;  // 5 N: rho0, ux0, uy0, bx0, by0
    double* ckpt;    // nseg x 19 N FP64 checkpoints (unpadded planes)
};

void free_tape(lbmhd_t* h) {
    if (!h || !h->tape) return;
    Tape* t = (Tape*)h->tape;
    cudaFree(t->fields);
    cudaFree(t->ckpt);
    delete t;
    h->tape = nullptr;
}

}  // namespace lbmhd

using namespace lbmhd;

namespace {

int afail(int code, const std::string& m) {
    set_error(m);
    return code;
}

int acuda(lbmhd_t* h, cudaError_t e, const char* where) {
    if (h) h->failed = true;
    cudaGetLastError();
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return LBMHD_ECUDA;
}

#define LBMHD_ACK(h, call)                                 \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return acuda(h, e_, #call); \
    } while (0)

unsigned adj_grid(long long n) {
    long long b = (n + kAdjBlock - 1) / kAdjBlock;
    return (unsigned)(b < 1 ? 1 : (b > kAdjMaxBlocks ? kAdjMaxBlocks : b));
}

template <class R>
Coll<R> coll_t(const HostColl& h) {
    return make_coll_t<R>(h.tn, h.te, h.k18, h.k36, h.s5, h.s6, h.s7, h.s8, h.les, h.tie5, h.tie6);
}  // the adjoint supports unscaled formats only (FP64, FP32, FP32_DEV)

template <int P>
cudaError_t run_adj_step(const lbmhd_t* h, const void* x, const void* lin, void* lout,
                         double* partials) {
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    const long long n = (long long)h->geom.nx * h->geom.ny;
    const unsigned grid = adj_grid(n);
    adj_step_kernel<P><<<grid, kAdjBlock, 0, h->stream>>>(
        (const S*)x, (const R*)lin, (R*)lout, h->geom.nx, h->geom.ny, h->geom.ps,
        coll_t<R>(h->coll), h->coll.inv_scale, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

template <int P>
cudaError_t run_seed(const lbmhd_t* h, const void* x, const double* const* gin, void* lam) {
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    const long long n = (long long)h->geom.nx * h->geom.ny;
    adj_seed_kernel<P><<<adj_grid(n), kAdjBlock, 0, h->stream>>>(
        (const S*)x, gin[0], gin[1], gin[2], gin[3], gin[4], (R*)lam, h->geom.nx, h->geom.ny,
        h->geom.ps, h->coll.inv_scale);
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int lbmhd_adjoint_record(lbmhd_t* h, const double* rho0, const double* ux0, const double* uy0,
                         const double* bx0, const double* by0, int nsteps, int every) {
    TraceRange trace_("lbmhd_adjoint_record");
    if (!h) return afail(LBMHD_EINVAL, "handle is NULL");
    if (h->failed) return afail(LBMHD_ECUDA, "handle is unusable after a CUDA error");
    if (!rho0 || !ux0 || !uy0 || !bx0 || !by0) return afail(LBMHD_EINVAL, "NULL field");
    if (nsteps < 1 || every < 1) return afail(LBMHD_EINVAL, "nsteps and every must be >= 1");
    const int prec = h->p.precision;
    if (prec != LBMHD_FP64 && prec != LBMHD_FP32 && prec != LBMHD_FP32_DEV && prec != LBMHD_FF)
        return afail(LBMHD_EINVAL, "the adjoint supports FP64, FF, FP32 and FP32_DEV storage");
    if (h->p.les >= 2)
        return afail(LBMHD_EINVAL, "the adjoint supports les 0 and 1 (not les 2 or 3)");
    free_tape(h);
    const long long n = (long long)h->geom.nx * h->geom.ny;
    Tape* t = new (std::nothrow) Tape();
    if (!t) return afail(LBMHD_ENOMEM, "host allocation failed");
    t->nsteps = nsteps;
    t->every = every;
    t->nseg = (nsteps + every - 1) / every;
    cudaError_t e = cudaMalloc((void**)&t->fields, 5 * n * sizeof(double));
    if (e == cudaSuccess)
        e = cudaMalloc((void**)&t->ckpt, (size_t)t->nseg * kNumPlanes * n * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(t->fields);
        delete t;
        cudaGetLastError();
        return afail(LBMHD_ENOMEM, "device allocation for the adjoint tape failed");
    }
    h->tape = t;
    const double* src[5] = {rho0, ux0, uy0, bx0, by0};
    for (int i = 0; i < 5; ++i)
        LBMHD_ACK(h, cudaMemcpyAsync(t->fields + i * n, src[i], n * sizeof(double),
                                     cudaMemcpyDeviceToDevice, h->stream));
    int rc = lbmhd_init_device(h, t->fields, t->fields + n, t->fields + 2 * n, t->fields + 3 * n,
                               t->fields + 4 * n);
    if (rc) return rc;
    for (int s = 0; s < t->nseg; ++s) {
        LBMHD_ACK(h, launch_get_state(prec, h->buf[h->cur], t->ckpt + (size_t)s * kNumPlanes * n,
                                      h->geom, h->coll, h->stream));
        const int k = (s + 1) * every <= nsteps ? every : nsteps - s * every;
        rc = lbmhd_step(h, k);
        if (rc) return rc;
    }
    t->step_at_end = h->steps;
    return LBMHD_OK;
}

int lbmhd_adjoint_backward(lbmhd_t* h, const double* g_rho, const double* g_ux,
                           const double* g_uy, const double* g_bx, const double* g_by,
                           double* dtheta, double* d_rho0, double* d_ux0, double* d_uy0,
                           double* d_bx0, double* d_by0) {
    TraceRange trace_("lbmhd_adjoint_backward");
    if (!h) return afail(LBMHD_EINVAL, "handle is NULL");
    if (h->failed) return afail(LBMHD_ECUDA, "handle is unusable after a CUDA error");
    Tape* t = (Tape*)h->tape;
    if (!t) return afail(LBMHD_ESTATE, "no recorded forward run (lbmhd_adjoint_record)");
    if (h->steps != t->step_at_end)
        return afail(LBMHD_ESTATE, "the state moved since lbmhd_adjoint_record");
    const int prec = h->p.precision;
    const long long n = (long long)h->geom.nx * h->geom.ny;
    const size_t sb = storage_bytes(prec);
    const size_t rb = prec == LBMHD_FP64 || prec == LBMHD_FF ? 8 : sizeof(float);
    const size_t plane_bytes_s = (size_t)kNumPlanes * h->geom.ps * sb;
    const size_t plane_bytes_r = (size_t)kNumPlanes * h->geom.ps * rb;
    char* seg = nullptr;
    char* lam = nullptr;
    double* partials = nullptr;
    double* acc = nullptr;
    cudaError_t e = cudaMalloc((void**)&seg, (size_t)t->every * plane_bytes_s);
    if (e == cudaSuccess) e = cudaMalloc((void**)&lam, 2 * plane_bytes_r);
    if (e == cudaSuccess) e = cudaMalloc((void**)&partials, (size_t)kAdjMaxBlocks * 4 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc((void**)&acc, 4 * sizeof(double));
    if (e != cudaSuccess) {
        cudaFree(seg);
        cudaFree(lam);
        cudaFree(partials);
        cudaFree(acc);
        cudaGetLastError();
        return afail(LBMHD_ENOMEM, "device allocation for the adjoint sweep failed");
    }
    int rc = LBMHD_OK;
    auto fin = [&](int code) {
        cudaStreamSynchronize(h->stream);
        cudaFree(seg);
        cudaFree(lam);
        cudaFree(partials);
        cudaFree(acc);
        return code;
    };
    const double* gin[5] = {g_rho, g_ux, g_uy, g_bx, g_by};
    void* lcur = lam;
    void* lnext = lam + plane_bytes_r;
    e = cudaMemsetAsync(acc, 0, 4 * sizeof(double), h->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(partials, 0, (size_t)kAdjMaxBlocks * 4 * sizeof(double), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(lam, 0, 2 * plane_bytes_r, h->stream);
    if (e == cudaSuccess) {
        switch (prec) {
            case LBMHD_FP64: e = run_seed<P_FP64>(h, h->buf[h->cur], gin, lcur); break;
            case LBMHD_FF: e = run_seed<P_FF>(h, h->buf[h->cur], gin, lcur); break;
            case LBMHD_FP32: e = run_seed<P_FP32>(h, h->buf[h->cur], gin, lcur); break;
            default: e = run_seed<P_FP32_DEV>(h, h->buf[h->cur], gin, lcur); break;
        }
    }
    if (e != cudaSuccess) return fin(acuda(h, e, "adjoint seed"));
    for (int s = t->nseg - 1; s >= 0; --s) {
        const int len = (s + 1) * t->every <= t->nsteps ? t->every : t->nsteps - s * t->every;
        // restore the checkpoint and recompute the segment's states
        e = launch_set_state(prec, t->ckpt + (size_t)s * kNumPlanes * n, seg, h->geom, h->coll,
                             h->stream);
        for (int j = 1; j < len && e == cudaSuccess; ++j)
            e = launch_step(prec, h->vec, h->block, 0, seg + (size_t)(j - 1) * plane_bytes_s,
                            seg + (size_t)j * plane_bytes_s, h->geom, h->coll, h->stream);
        if (e != cudaSuccess) return fin(acuda(h, e, "adjoint recompute"));
        for (int j = len - 1; j >= 0; --j) {
            // every node of lnext is written by the scatter (a permutation)
            const void* x = seg + (size_t)j * plane_bytes_s;
            switch (prec) {
                case LBMHD_FP64: e = run_adj_step<P_FP64>(h, x, lcur, lnext, partials); break;
                case LBMHD_FF: e = run_adj_step<P_FF>(h, x, lcur, lnext, partials); break;
                case LBMHD_FP32: e = run_adj_step<P_FP32>(h, x, lcur, lnext, partials); break;
                default: e = run_adj_step<P_FP32_DEV>(h, x, lcur, lnext, partials); break;
            }
            if (e != cudaSuccess) return fin(acuda(h, e, "adjoint step"));
            void* tmp = lcur;
            lcur = lnext;
            lnext = tmp;
        }
    }
    if (d_rho0 || d_ux0 || d_uy0 || d_bx0 || d_by0) {
        if (prec == LBMHD_FP64)
            adj_init_kernel<double><<<adj_grid(n), kAdjBlock, 0, h->stream>>>(
                (const double*)lcur, t->fields, d_rho0, d_ux0, d_uy0, d_bx0, d_by0, h->geom.nx,
                h->geom.ny, h->geom.ps);
        else if (prec == LBMHD_FF)
            adj_init_kernel<ff><<<adj_grid(n), kAdjBlock, 0, h->stream>>>(
                (const ff*)lcur, t->fields, d_rho0, d_ux0, d_uy0, d_bx0, d_by0, h->geom.nx,
                h->geom.ny, h->geom.ps);
        else
            adj_init_kernel<float><<<adj_grid(n), kAdjBlock, 0, h->stream>>>(
                (const float*)lcur, t->fields, d_rho0, d_ux0, d_uy0, d_bx0, d_by0, h->geom.nx,
                h->geom.ny, h->geom.ps);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fin(acuda(h, e, "adjoint init Jacobian"));
    }
    // the per-block sums over all steps, combined in block order
    adj_reduce_kernel<<<1, kAdjBlock, 0, h->stream>>>(partials, (int)adj_grid(n), acc);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fin(acuda(h, e, "adjoint reduction"));
    double a[4] = {0, 0, 0, 0};
    e = cudaMemcpyAsync(a, acc, sizeof(a), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fin(acuda(h, e, "adjoint readback"));
    if (dtheta) {
        const double d2 = h->p.delta * h->p.delta;
        dtheta[0] = 18.0 * d2 * a[2] + 36.0 * d2 * a[3];  // d/dC_S
        dtheta[1] = a[0];                                  // d/dtau_nu
        dtheta[2] = a[1];                                  // d/dtau_eta
    }
    return fin(rc);
}

int lbmhd_adjoint_release(lbmhd_t* h) {
    if (!h) return afail(LBMHD_EINVAL, "handle is NULL");
    if (!h->failed) cudaStreamSynchronize(h->stream);
    free_tape(h);
    return LBMHD_OK;
}

}  // extern "C"
