// lbmhd_device.cuh -- device-side arithmetic of the filtered LB-MHD step
// (Flint & Vahala, arXiv:1607.08675): storage formats, the per-node MRT +
// local-LES collision of the D2Q9 density populations and the SRT
// collision of the D2Q5 vector magnetic populations, all in registers.
#pragma once

#include <cuda_fp16.h>
#include <stdint.h>

#include <type_traits>

#include "lbmhd_ff.cuh"

namespace lbmhd {

constexpr int kPlanes = 19;  // 9 f_i, then g_k (x, y) for k = 0..4

// Lattice (Sec. 3, explicit lists): c_x, c_y of the D2Q9 set and C_x, C_y
// of the D2Q5 set, expanded to the 19 storage planes.  Streaming pulls
// plane p at node x from x - c_p.
__host__ __device__ constexpr int plane_cx(int p) {
    return p < 9 ? (p == 1 || p == 5 || p == 8 ? 1 : (p == 3 || p == 6 || p == 7 ? -1 : 0))
                 : ((p - 9) / 2 == 1 ? 1 : ((p - 9) / 2 == 3 ? -1 : 0));
}
__host__ __device__ constexpr int plane_cy(int p) {
    return p < 9 ? (p == 2 || p == 5 || p == 6 ? 1 : (p == 4 || p == 7 || p == 8 ? -1 : 0))
                 : ((p - 9) / 2 == 2 ? 1 : ((p - 9) / 2 == 4 ? -1 : 0));
}
// Rest-state equilibrium (rho = 1, u = B = 0) of each plane: the D2Q9
// weights w_i = 4/9, 1/9, 1/36 (fixed by Eq. KinMomentEq); g has none.
template <class R>
__host__ __device__ constexpr R plane_rest(int p) {
    return p == 0 ? R(4) / R(9) : (p < 5 ? R(1) / R(9) : (p < 9 ? R(1) / R(36) : R(0)));
}

// Storage formats.  Every format is decoded to the deviation d = f - w
// (and g itself) in the arithmetic type R, and encoded back from it.
enum Prec { P_FP64 = 0, P_FP32 = 1, P_FP32_DEV = 2, P_FP16_DEV = 3, P_FF = 4 };

template <int P> struct Fmt;
template <> struct Fmt<P_FP64> {
    using S = double;
    using R = double;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ R dec(S v, int p, float) { return v - plane_rest<R>(p); }
    static __device__ __forceinline__ S enc(R d, int p, float) { return d + plane_rest<R>(p); }
};
template <> struct Fmt<P_FP32> {
    using S = float;
    using R = float;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ R dec(S v, int p, float) { return v - plane_rest<R>(p); }
    static __device__ __forceinline__ S enc(R d, int p, float) { return d + plane_rest<R>(p); }
};
template <> struct Fmt<P_FP32_DEV> {
    using S = float;
    using R = float;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ R dec(S v, int, float) { return v; }
    static __device__ __forceinline__ S enc(R d, int, float) { return d; }
};
// FP16: stored = d * scale.  The step kernels keep the scaled value through
// the collision (see collide<R, true>), so dec/enc here convert only.
template <> struct Fmt<P_FP16_DEV> {
    using S = unsigned short;  // raw binary16 bits
    using R = float;
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ R dec(S v, int, float) {
        return __half2float(__ushort_as_half(v));
    }
    static __device__ __forceinline__ S enc(R d, int, float) {
        return __half_as_ushort(__float2half_rn(d));
    }
};

// Double-word deviations: stored (hi, lo), arithmetic in double-word
// (lbmhd_ff.cuh); the stored pair is the normalised result of the collision.
template <> struct Fmt<P_FF> {
    using S = float2;
    using R = ff;
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ R dec(S v, int, float) { return ff(v.x, v.y); }
    static __device__ __forceinline__ S enc(R d, int, float) { return make_float2(d.hi, d.lo); }
};

// Reciprocal and square root in the arithmetic type.  FP64 keeps the
// IEEE-rounded operations (the parity mode); FP32 uses the single-
// instruction hardware approximations (relative error ~1e-7, far below
// the FP32/FP16 storage rounding the FP32 modes carry anyway).
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
__device__ __forceinline__ float rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float sqrt_(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// IEEE-rounded reciprocal and square root for float and double (the
// gradient closures use these); the double-word overloads of lbmhd_ff.cuh
// are its Newton reciprocal and Dekker square root.
template <class R>
__device__ __forceinline__ R recip(R x) {
    return R(1) / x;
}
__device__ __forceinline__ ff recip(ff x) { return rcp(x); }
template <class R>
__device__ __forceinline__ R root(R x) {
    return sqrt(x);
}
__device__ __forceinline__ ff root(ff x) { return sqrt_(x); }

// x times a small constant k (an integer or a power of two, exact in FP32):
// R(k) * x; the double-word overload (lbmhd_ff.cuh) scales cheaper.
template <class R>
__device__ __forceinline__ R kmul(float k, R x) {
    return R(k) * x;
}

// Collision parameters in the arithmetic type.
template <class R>
struct Coll {
    R tn, te;        // base tau_nu, tau_eta
    R tn2, te2;      // their squares
    R k18, k36;      // 18 C_S Delta^2, 36 C_S Delta^2
    R s5, s6;        // resolved energy-flux rates
    R s7, s8;        // fixed rates (used when > 0), else tied to s_nu
    int les;
    int tie5, tie6;  // s5 (s6) is the tied value 1/tau_nu
    R inv_s;         // scaled storage: 1 / scale (k18, k36 already divided by scale)
    R scl;           // scaled storage: the scale itself (1 otherwise)
    R d2;            // Delta^2 (filtered equilibria, les = 2)
    R cd2;           // C_S Delta^2 (cross-helicity closure, les = 3)
};

// Relaxation times of the cross-helicity closure of Carati et al. (Sec. 1.1,
// Eqs. CHClosureV/B): nu_t = C_S Delta^2 |S^v_ab S^b_ab|^(1/2) and
// eta_t = C_S Delta^2 sgn(j omega) |j omega|^(1/2), with S^v, S^b the
// symmetric gradients of u and B, omega and j the curls; tau = tau0 + 3 x
// (nu = (tau - 1/2)/3, Sec. 4.3); the total resistivity stays >= 0.
// gu / gb: d/dx, d/dy of (u_x, u_y) and (B_x, B_y): g[a][0] = d_x v_a.
template <class R>
__device__ __forceinline__ void carati_taus(const R (&gu)[2][2], const R (&gb)[2][2], R cd2,
                                            R tn, R te, R (&taus)[2]) {
    const R svxy = R(0.5) * (gu[0][1] + gu[1][0]);
    const R sbxy = R(0.5) * (gb[0][1] + gb[1][0]);
    const R ss = gu[0][0] * gb[0][0] + gu[1][1] * gb[1][1] + R(2) * svxy * sbxy;
    const R nu_t = cd2 * root(fabs(ss));
    const R om = gu[1][0] - gu[0][1], jz = gb[1][0] - gb[0][1];
    const R jw = jz * om;
    const R sg = jw > R(0) ? R(1) : (jw < R(0) ? R(-1) : R(0));
    const R eta_t = cd2 * sg * root(fabs(jw));
    taus[0] = tn + R(3) * nu_t;
    const R tm = te + R(3) * eta_t;
    taus[1] = tm < R(0.5) ? R(0.5) : tm;
}

// Filtered-equilibrium corrections of the paper's kinetic LES (Sec. 4.1):
// the filter rules for a product XY, (1/12) dX . dY (Eq. FilterExampleSmall),
// and for a ratio XY/Z, (1/(12 Z)) [dX . dY - (X dZ . dY + Y dZ . dX -
// X Y dZ . dZ / Z) / Z] (Eq. FilterExampleLarge), applied to the terms of
// Eqs. KinMomentEq and MagMomentEq.  fld = (rho, jx, jy, Bx, By) at the
// node, gx / gy their x / y derivatives; returns Delta^2 times the
// corrections of M_3, M_4, M_7 (= M_8) and N_y1 (= -N_x2).
template <class R>
__device__ __forceinline__ void filtered_shift(const R (&fld)[5], const R (&gx)[5],
                                               const R (&gy)[5], R d2, R (&sh)[4]) {
    const R ir = recip(fld[0]);
    constexpr R twelfth = R(1) / R(12);
    auto dot = [&](int a, int b) { return gx[a] * gx[b] + gy[a] * gy[b]; };
    // ratio rule with Z = rho for fields a, b
    auto ratio = [&](int a, int b) {
        return (dot(a, b) - (fld[a] * dot(0, b) + fld[b] * dot(0, a) - fld[a] * fld[b] * dot(0, 0) * ir) * ir) *
               (ir * twelfth);
    };
    const R rxx = ratio(1, 1), ryy = ratio(2, 2), rxy = ratio(1, 2);
    sh[0] = d2 * (rxy - twelfth * dot(3, 4));
    sh[1] = d2 * ((rxx - ryy) - twelfth * (dot(3, 3) - dot(4, 4)));
    sh[2] = d2 * (R(-3) * (rxx + ryy));
    sh[3] = d2 * (ratio(1, 4) - ratio(2, 3));
}

// Fused multiply-add in the arithmetic type: one rounding for FP32 and FP64,
// the double-word product and sum for FF.  kfma(k, x, y) = k x + y for a
// small constant k (kmul's exact or cheap scaling for FF).
template <class R>
__device__ __forceinline__ R fmad(R a, R b, R c) {
    return a * b + c;
}
template <>
__device__ __forceinline__ float fmad(float a, float b, float c) {
    return __fmaf_rn(a, b, c);
}
template <>
__device__ __forceinline__ double fmad(double a, double b, double c) {
    return __fma_rn(a, b, c);
}
template <class R>
__device__ __forceinline__ R kfma(float k, R x, R y) {
    return kmul(k, x) + y;
}
template <>
__device__ __forceinline__ float kfma(float k, float x, float y) {
    return __fmaf_rn(k, x, y);
}
template <>
__device__ __forceinline__ double kfma(float k, double x, double y) {
    return __fma_rn((double)k, x, y);
}

// One node: d[9] = streamed f_i - w_i, g[10] = streamed g_k (x, y);
// overwritten with the post-collision values.
//
// Density (Sec. 3): moments M_j = T_j . f for j = 3..8 (Eq. FluidTMatrix
// rows; the rest state contributes only to M_8, by 5/3), equilibria of
// Eq. KinMomentEq, n_j = M_j - M_j^eq.  Local eddy rate: Q = sqrt(n_4^2 +
// 4 n_3^2) gives |S| = 3 Q / (2 rho tau); tau_e = tau_nu + 3 C_S Delta^2 |S|
// solved as tau_e = (tau_nu + sqrt(tau_nu^2 + 18 C_S Delta^2 Q / rho)) / 2.
// Relaxation M_j <- M_j - s_j n_j and return through T^-1 = T^t diag(1/|T_j|^2)
// (the rows of T are orthogonal), i.e. f_i <- f_i - sum_j s_j n_j T_ji / |T_j|^2.
//
// Magnetic (Sec. 3, Eq. LBMagEqn): B = sum g_k, D2Q5 equilibrium
// g_k^eq = w'_k [B + 3((C_k.u) B - (C_k.B) u)], which with E = u_x B_y -
// u_y B_x is B/3 at rest and (B +- 3E e_perp)/6 on the axes.  The
// antisymmetric non-equilibrium first moment (N_y1 - N_x2)^neq =
// -(tau_m/3) j_z gives |j|; tau_m = (tau_eta + sqrt(tau_eta^2 +
// 36 C_S Delta^2 J)) / 2 with J = |N_y1 - N_x2 - 2E|.  g <- g - (g - g^eq)/tau_m.
//
// SCALED: d and g hold s times the deviations (FP16 storage scale s).  Every
// linear step is unchanged; the four quadratic terms get one factor 1/s,
// the density needs the unscaled sum, and 18 C_S Delta^2, 36 C_S Delta^2
// arrive divided by s (Q and J are scaled).  The outputs stay scaled.
//
// KIN: relax towards the filtered equilibria, sh = Delta^2 corrections of
// M_3, M_4, M_7 = M_8 and N_y1 (in the units of d and g).
//
// TAUS: use the relaxation times sh[0] (tau_e) and sh[1] (tau_m) given by
// the caller (cross-helicity closure) instead of the local Smagorinsky ones.
template <class R, bool SCALED = false, bool KIN = false, bool TAUS = false>
__device__ __forceinline__ void collide(R (&d)[9], R (&g)[10], const Coll<R>& c,
                                        const R* sh = nullptr) {
    // Rational constants, formed at compile time in the arithmetic type.
    constexpr R k1_3 = R(1) / R(3), k1_6 = R(1) / R(6), k5_3 = R(5) / R(3);
    constexpr R k1_12 = R(1) / R(12), k1_20 = R(1) / R(20), k1_180 = R(1) / R(180);
    // FP64 (its step is bound by the FP64 pipe) takes the moments and the
    // relaxation from shared pair sums -- a = d5 - d6, b = d8 - d7,
    // cc = d5 + d6, e = d7 + d8, p = d1 - d3, q = d2 - d4, r = d1 + d3,
    // t = d2 + d4: 22 sums for rho, j and M_3..M_8 instead of 43, 8% faster
    // at 8192^2.  The other types keep one sum tree per moment: the shared
    // form holds more values live (FP16 storage: 146 registers instead of
    // 128, 9% slower) and measured 2.7% slower for FF.
    constexpr bool SH = std::is_same<R, double>::value;
    const R a = d[5] - d[6], b = d[8] - d[7], cc = d[5] + d[6], e = d[7] + d[8];
    const R p = d[1] - d[3], q = d[2] - d[4], r = d[1] + d[3], t = d[2] + d[4];
    const R ab = a + b, ce = cc - e, rt = r + t, shd = cc + e, d0s = d[0] + shd;
    const R dsum9 = SH ? d0s + rt
                       : ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const R jx = SH ? p + ab : (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    const R jy = SH ? q + ce : (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    const R rho = R(1) + (SCALED ? dsum9 * c.inv_s : dsum9);
    const R irho = rcp(rho);
    const R ux = jx * irho, uy = jy * irho;
    const R bx = (g[0] + g[2]) + (g[4] + g[6]) + g[8];
    const R by = (g[1] + g[3]) + (g[5] + g[7]) + g[9];

    const R dsum = SH ? shd : (d[5] + d[6]) + (d[7] + d[8]);
    const R m3 = SH ? a - b : (d[5] - d[6]) + (d[7] - d[8]);
    const R m4 = SH ? r - t : (d[1] + d[3]) - (d[2] + d[4]);
    const R m5 = SH ? ab - kmul(2, p) : kmul(2, d[3] - d[1]) + (d[5] - d[6]) + (d[8] - d[7]);
    const R m6 = SH ? ce - kmul(2, q) : kmul(2, d[4] - d[2]) + (d[5] + d[6]) - (d[7] + d[8]);
    const R m7 = SH ? kmul(4, d0s) - kmul(5, rt)
                    : kmul(4, d[0]) - kmul(5, (d[1] + d[2]) + (d[3] + d[4])) + kmul(4, dsum);
    const R m8 = kmul(4, d[0]) - dsum;

    R j2i = (jx * jx + jy * jy) * irho;
    R q3 = jx * jy * irho - bx * by;
    R q4 = (jx * jx - jy * jy) * irho - bx * bx + by * by;
    // Ny1 = sum_k C_kx g_ky, Nx2 = sum_k C_ky g_kx; Ny1^eq = E = -Nx2^eq
    R E = ux * by - uy * bx;
    if (SCALED) {
        j2i *= c.inv_s;
        q3 *= c.inv_s;
        q4 *= c.inv_s;
        E *= c.inv_s;
    }
    R k7 = R(0);
    if (KIN) {
        q3 += sh[0];
        q4 += sh[1];
        k7 = sh[2];
        E += sh[3];
    }
    const R n3 = m3 - q3;
    const R n4 = m4 - q4;
    const R n5 = m5 + jx;
    const R n6 = m6 + jy;
    const R n7 = KIN ? (m7 + kmul(3, j2i)) - k7 : m7 + kmul(3, j2i);
    const R n8 = KIN ? m8 - ((k5_3 * dsum9 - kmul(3, j2i)) + k7)
                     : m8 - (k5_3 * dsum9 - kmul(3, j2i));

    R tau_e = c.tn, tau_m = c.te;
    if (c.les) {
        const R Q = sqrt_(n4 * n4 + kmul(4, n3 * n3));
        tau_e = kmul(0.5f, c.tn + sqrt_(c.tn2 + c.k18 * Q * irho));
        const R Ny1 = g[3] - g[7];
        const R Nx2 = g[4] - g[8];
        const R J = fabs(Ny1 - Nx2 - kmul(2, E));
        tau_m = kmul(0.5f, c.te + sqrt_(c.te2 + c.k36 * J));
    }
    if (TAUS) {
        tau_e = sh[0];
        tau_m = sh[1];
    }
    const R snu = rcp(tau_e);
    const R s7 = c.s7 > R(0) ? c.s7 : snu;
    const R s8 = c.s8 > R(0) ? c.s8 : snu;

    const R a3 = kmul(0.25f, snu * n3);
    const R a4 = kmul(0.25f, snu * n4);
    const R a5 = c.s5 * n5 * k1_12;
    const R a6 = c.s6 * n6 * k1_12;
    const R a7 = s7 * n7 * k1_180;
    const R a8 = s8 * n8 * k1_20;

    const R q78 = kmul(4, a7) - a8;
    d[0] -= kmul(4, a7 + a8);
    if constexpr (SH) {
        // the rows of T from shared partial sums: d1, d3 = (a4 - 5 a7) -+ 2 a5;
        // d2, d4 = -(a4 + 5 a7) -+ 2 a6; d5, d6 = (a6 + q78) +- (a3 + a5);
        // d7, d8 = (q78 - a6) +- (a3 - a5)
        const R w5 = kmul(5, a7);
        const R u13 = a4 - w5, u24 = -(a4 + w5);
        const R y5 = kmul(2, a5), y6 = kmul(2, a6);
        const R P = a3 + a5, M = a3 - a5, S = a6 + q78, D = q78 - a6;
        d[1] -= u13 - y5;
        d[2] -= u24 - y6;
        d[3] -= u13 + y5;
        d[4] -= u24 + y6;
        d[5] -= P + S;
        d[6] -= S - P;
        d[7] -= M + D;
        d[8] -= D - M;
    } else {
        d[1] -= a4 - kmul(2, a5) - kmul(5, a7);
        d[2] -= -a4 - kmul(2, a6) - kmul(5, a7);
        d[3] -= a4 + kmul(2, a5) - kmul(5, a7);
        d[4] -= -a4 + kmul(2, a6) - kmul(5, a7);
        d[5] -= (a3 + a5) + (a6 + q78);
        d[6] -= (a6 - a3) - (a5 - q78);
        d[7] -= (a3 - a5) - (a6 - q78);
        d[8] -= (a5 - a3) - (a6 - q78);
    }

    const R sm = rcp(tau_m);
    const R third = k1_3, sixth = k1_6;
    const R e3 = kmul(3, E);
    const R geq[10] = {third * bx,        third * by,          // k = 0
                       sixth * bx,        sixth * (by + e3),   // k = 1 (+x)
                       sixth * (bx - e3), sixth * by,          // k = 2 (+y)
                       sixth * bx,        sixth * (by - e3),   // k = 3 (-x)
                       sixth * (bx + e3), sixth * by};         // k = 4 (-y)
#pragma unroll
    for (int q = 0; q < 10; ++q) g[q] -= sm * (g[q] - geq[q]);
}

// The collision of collide() with its products and sums written as explicit
// fused multiply-adds (fmad, kfma), for kernels compiled without contraction
// (the kinetic closures' file): there the compiler fuses nothing by itself,
// so kernels of different shape that call this function round every
// operation the same way and give the same bits, and the explicit fusions
// save the instructions contraction would.  Same moments, equilibria,
// rates and relaxation as collide(), same template flags.
template <class R, bool SCALED = false, bool KIN = false, bool TAUS = false>
__device__ __forceinline__ void collide_xf(R (&d)[9], R (&g)[10], const Coll<R>& c,
                                           const R* sh = nullptr) {
    constexpr R k1_3 = R(1) / R(3), k1_6 = R(1) / R(6), k5_3 = R(5) / R(3);
    constexpr R k1_12 = R(1) / R(12), k1_20 = R(1) / R(20), k1_180 = R(1) / R(180);
    // FP64 takes the shared pair sums of collide(); the other types the
    // sum trees (same measurements).
    constexpr bool SH = std::is_same<R, double>::value;
    const R a = d[5] - d[6], b = d[8] - d[7], cc = d[5] + d[6], e = d[7] + d[8];
    const R p = d[1] - d[3], q = d[2] - d[4], r = d[1] + d[3], t = d[2] + d[4];
    const R ab = a + b, ce = cc - e, rt = r + t, shd = cc + e, d0s = d[0] + shd;
    const R dsum9 = SH ? d0s + rt
                       : ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    const R jx = SH ? p + ab : (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    const R jy = SH ? q + ce : (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    const R rho = SCALED ? fmad(dsum9, c.inv_s, R(1)) : R(1) + dsum9;
    const R irho = rcp(rho);
    const R ux = jx * irho, uy = jy * irho;
    const R bx = (g[0] + g[2]) + (g[4] + g[6]) + g[8];
    const R by = (g[1] + g[3]) + (g[5] + g[7]) + g[9];

    const R dsum = SH ? shd : (d[5] + d[6]) + (d[7] + d[8]);
    const R s1234 = SH ? rt : (d[1] + d[2]) + (d[3] + d[4]);
    const R m3 = SH ? a - b : (d[5] - d[6]) + (d[7] - d[8]);
    const R m4 = SH ? r - t : (d[1] + d[3]) - (d[2] + d[4]);
    const R m5 = SH ? kfma(-2, p, ab) : kfma(2, d[3] - d[1], (d[5] - d[6]) + (d[8] - d[7]));
    const R m6 = SH ? kfma(-2, q, ce) : kfma(2, d[4] - d[2], (d[5] + d[6]) - (d[7] + d[8]));
    const R m7 = kfma(-5, s1234, kmul(4, SH ? d0s : d[0] + dsum));
    const R m8 = kfma(4, d[0], -dsum);

    R j2i = fmad(jx, jx, jy * jy) * irho;
    R q3 = fmad(jx * jy, irho, -(bx * by));
    R q4 = fmad(fmad(jx, jx, -(jy * jy)), irho, fmad(by, by, -(bx * bx)));
    R E = fmad(ux, by, -(uy * bx));
    if (SCALED) {
        j2i *= c.inv_s;
        q3 *= c.inv_s;
        q4 *= c.inv_s;
        E *= c.inv_s;
    }
    R k7 = R(0);
    if (KIN) {
        q3 += sh[0];
        q4 += sh[1];
        k7 = sh[2];
        E += sh[3];
    }
    const R n3 = m3 - q3;
    const R n4 = m4 - q4;
    const R n5 = m5 + jx;
    const R n6 = m6 + jy;
    const R n7 = KIN ? kfma(3, j2i, m7) - k7 : kfma(3, j2i, m7);
    const R n8 = KIN ? m8 - (fmad(k5_3, dsum9, -kmul(3, j2i)) + k7)
                     : m8 - fmad(k5_3, dsum9, -kmul(3, j2i));

    R tau_e = c.tn, tau_m = c.te;
    if (c.les) {
        const R Q = sqrt_(fmad(n4, n4, kmul(4, n3 * n3)));
        tau_e = kmul(0.5f, c.tn + sqrt_(fmad(c.k18 * Q, irho, c.tn2)));
        const R Ny1 = g[3] - g[7];
        const R Nx2 = g[4] - g[8];
        const R J = fabs(Ny1 - Nx2 - kmul(2, E));
        tau_m = kmul(0.5f, c.te + sqrt_(fmad(c.k36, J, c.te2)));
    }
    if (TAUS) {
        tau_e = sh[0];
        tau_m = sh[1];
    }
    const R snu = rcp(tau_e);
    const R s7 = c.s7 > R(0) ? c.s7 : snu;
    const R s8 = c.s8 > R(0) ? c.s8 : snu;

    const R a3 = kmul(0.25f, snu * n3);
    const R a4 = kmul(0.25f, snu * n4);
    const R a5 = c.s5 * n5 * k1_12;
    const R a6 = c.s6 * n6 * k1_12;
    const R a7 = s7 * n7 * k1_180;
    const R a8 = s8 * n8 * k1_20;

    const R q78 = kfma(4, a7, -a8);
    d[0] -= kmul(4, a7 + a8);
    if constexpr (SH) {
        const R u13 = kfma(-5, a7, a4), u24 = kfma(-5, a7, -a4);
        const R P = a3 + a5, M = a3 - a5, S = a6 + q78, D = q78 - a6;
        d[1] -= kfma(-2, a5, u13);
        d[2] -= kfma(-2, a6, u24);
        d[3] -= kfma(2, a5, u13);
        d[4] -= kfma(2, a6, u24);
        d[5] -= P + S;
        d[6] -= S - P;
        d[7] -= M + D;
        d[8] -= D - M;
    } else {
        d[1] -= kfma(-5, a7, kfma(-2, a5, a4));
        d[2] -= kfma(-5, a7, kfma(-2, a6, -a4));
        d[3] -= kfma(-5, a7, kfma(2, a5, a4));
        d[4] -= kfma(-5, a7, kfma(2, a6, -a4));
        d[5] -= (a3 + a5) + (a6 + q78);
        d[6] -= (a6 - a3) - (a5 - q78);
        d[7] -= (a3 - a5) - (a6 - q78);
        d[8] -= (a5 - a3) - (a6 - q78);
    }

    const R sm = rcp(tau_m);
    const R third = k1_3, sixth = k1_6;
    const R e3 = kmul(3, E);
    const R geq[10] = {third * bx,        third * by,          // k = 0
                       sixth * bx,        sixth * (by + e3),   // k = 1 (+x)
                       sixth * (bx - e3), sixth * by,          // k = 2 (+y)
                       sixth * bx,        sixth * (by - e3),   // k = 3 (-x)
                       sixth * (bx + e3), sixth * by};         // k = 4 (-y)
#pragma unroll
    for (int q = 0; q < 10; ++q) g[q] = fmad(-sm, g[q] - geq[q], g[q]);
}

}  // namespace lbmhd
