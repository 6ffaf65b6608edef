// lbmhd3.cu -- the 3D extension of the LB-MHD step (Sec. 3 opening: the
// model extends to 3D with more lattice velocities; the Conclusion names
// D3Q27): D3Q27 density populations, D3Q7 vector magnetic populations (the
// six axes; the rest weight is zero), one fused pull-stream + collide kernel
// per step, and the handle behind the lbmhd3_* C ABI.
//
// Equilibria: the paper's D2Q9 expression with 3D vectors plus the 3D trace
// term -9/2 w |B|^2/6 (zero in 2D), and the paper's D2Q5 expression on the
// six axes with w' = 1/6.  Collision: BGK (the paper's MRT with every rate
// tied), magnetic SRT, with the local Smagorinsky rates of les = 1 from the
// traceless non-equilibrium stress and the axial vector of the magnetic
// non-equilibrium first moment.  The two gradient closures take two
// launches per step: a moments pass (rho - 1, j, B of the populations
// streamed into every node, seven planes), then the step, which forms
// central differences of those planes at the six neighbours and either
// relaxes towards the filtered equilibria (the paper's kinetic LES, Sec. 4.1,
// les = 2) or takes the cross-helicity closure's relaxation times
// (Eqs. CHClosureV/B, les = 3).
//
// This file is compiled without FMA contraction (-fmad=false) and writes its
// fused multiply-adds out (fmad), so the one- and two-node launch shapes,
// whose code the compiler shapes differently, round every operation alike
// and give the same bits.
//
// Layout: 45 SoA planes (27 f_i, then g_q (x, y, z) for q = +x, -x, +y, -y,
// +z, -z), node (x, y, z) at (z ny + y) nx + x, plane stride padded to 64
// elements.  f_i with i = 9 kz + 3 ky + kx, c = (v[kx], v[ky], v[kz]),
// v = {0, 1, -1}.  Arithmetic in deviations d = f - w (g itself).
#include <cuda_fp16.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <type_traits>

#include "lbmhd_bulk.cuh"
#include "lbmhd_device.cuh"
#include "lbmhd_internal.h"
#include "lbmhd_step_body.cuh"

namespace lbmhd {
namespace d3 {

constexpr int kQ = 27, kM = 6, kP = kQ + 3 * kM;  // 45 planes

__host__ __device__ constexpr int v1(int k) { return k == 0 ? 0 : (k == 1 ? 1 : -1); }
// velocity components of plane p (density planes, then the magnetic axes)
__host__ __device__ constexpr int pcx(int p) {
    return p < kQ ? v1(p % 3) : ((p - kQ) / 3 == 0 ? 1 : ((p - kQ) / 3 == 1 ? -1 : 0));
}
__host__ __device__ constexpr int pcy(int p) {
    return p < kQ ? v1((p / 3) % 3) : ((p - kQ) / 3 == 2 ? 1 : ((p - kQ) / 3 == 3 ? -1 : 0));
}
__host__ __device__ constexpr int pcz(int p) {
    return p < kQ ? v1(p / 9) : ((p - kQ) / 3 == 4 ? 1 : ((p - kQ) / 3 == 5 ? -1 : 0));
}
// D3Q27 weights: the product of the 1D weights {2/3, 1/6, 1/6}
template <class R>
__host__ __device__ constexpr R w1(int k) {
    return k == 0 ? R(2) / R(3) : R(1) / R(6);
}
template <class R>
__host__ __device__ constexpr R wq(int i) {
    return w1<R>(i % 3) * w1<R>((i / 3) % 3) * w1<R>(i / 9);
}
template <class R>
__host__ __device__ constexpr R plane_rest3(int p) {
    return p < kQ ? wq<R>(p) : R(0);
}
// The weight in the arithmetic type: FP32 and FP64 form the product in
// their own arithmetic, double-word takes the nearest double-word to the
// FP64 product (exact to 2^-48).
template <class R>
__device__ __forceinline__ R wqr(int i) {
    if constexpr (std::is_same<R, ff>::value)
        return ff(wq<double>(i));
    else
        return wq<R>(i);
}
__device__ __forceinline__ ff fmax(ff a, ff b) { return a > b ? a : b; }
using ::fmax;
// A read-only load of a value of the arithmetic type.
template <class R>
__device__ __forceinline__ R ldg_r(const R* p) {
    if constexpr (std::is_same<R, ff>::value) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(p));
        return ff(v.x, v.y);
    } else {
        return __ldg(p);
    }
}

// Storage formats: S stored, R arithmetic.  dec / enc convert a stored
// value of plane p to and from its deviation d = f - w_p (g itself); sc is
// the FP16 storage scale's inverse (dec) or the scale (enc), unused by the
// other formats.  to_f / from_f convert to and from the population value f
// in FP64 (initialisation and read-back).
template <int P> struct Fmt3;
template <> struct Fmt3<P_FP64> {
    using S = double;
    using R = double;
    static __device__ __forceinline__ R dec(S v, int p, float) { return v - plane_rest3<R>(p); }
    static __device__ __forceinline__ S enc(R d, int p, float) { return d + plane_rest3<R>(p); }
    static __device__ __forceinline__ double to_f(S v, int, double) { return v; }
    static __device__ __forceinline__ S from_f(double f, int, double) { return f; }
    // from the population f and its deviation d = f - w_p, both in FP64
    static __device__ __forceinline__ S from_fd(double f, double, int, double) { return f; }
};
template <> struct Fmt3<P_FP32> {
    using S = float;
    using R = float;
    static __device__ __forceinline__ R dec(S v, int p, float) { return v - plane_rest3<R>(p); }
    static __device__ __forceinline__ S enc(R d, int p, float) { return d + plane_rest3<R>(p); }
    static __device__ __forceinline__ double to_f(S v, int, double) { return (double)v; }
    static __device__ __forceinline__ S from_f(double f, int, double) { return (float)f; }
    static __device__ __forceinline__ S from_fd(double f, double, int, double) { return (float)f; }
};
// double-word deviations (hi, lo) of f - w_p (g itself), double-word
// arithmetic (the FP32 pipes)
template <> struct Fmt3<P_FF> {
    using S = float2;
    using R = ff;
    static __device__ __forceinline__ R dec(S v, int, float) { return ff(v.x, v.y); }
    static __device__ __forceinline__ S enc(R d, int, float) { return make_float2(d.hi, d.lo); }
    static __device__ __forceinline__ double to_f(S v, int p, double) {
        return ((double)v.x + (double)v.y) + plane_rest3<double>(p);
    }
    static __device__ __forceinline__ S from_f(double f, int p, double) {
        const ff d(f - plane_rest3<double>(p));
        return make_float2(d.hi, d.lo);
    }
    static __device__ __forceinline__ S from_fd(double, double d, int, double) {
        const ff v(d);
        return make_float2(v.hi, v.lo);
    }
};
// binary16 deviations times the storage scale (f - w_p, g itself), FP32
// arithmetic
template <> struct Fmt3<P_FP16_DEV> {
    using S = unsigned short;
    using R = float;
    static __device__ __forceinline__ R dec(S v, int, float inv_s) {
        return __half2float(__ushort_as_half(v)) * inv_s;
    }
    static __device__ __forceinline__ S enc(R d, int, float s) {
        return __half_as_ushort(__float2half_rn(d * s));
    }
    static __device__ __forceinline__ double to_f(S v, int p, double inv_s) {
        return (double)__half2float(__ushort_as_half(v)) * inv_s + plane_rest3<double>(p);
    }
    static __device__ __forceinline__ S from_f(double f, int p, double s) {
        return __half_as_ushort(__float2half_rn((float)((f - plane_rest3<double>(p)) * s)));
    }
    static __device__ __forceinline__ S from_fd(double, double d, int, double s) {
        return __half_as_ushort(__float2half_rn((float)(d * s)));
    }
};

template <class R>
struct Coll3 {
    R tn, te, tn2, te2, k18, k36;
    R d12;  // Delta^2 / 12 (les = 2)
    R cd2;  // C_S Delta^2 (les = 3)
    float s16, i16;  // FP16 storage scale and its inverse
    int les;
};

// Closure of a step: 0 = none or local rates (les 0, 1), 2 = filtered
// equilibria, 3 = cross-helicity relaxation times.
enum { K3_LOCAL = 0, K3_FILTER = 2, K3_CARATI = 3 };

// One node: d[27] = pulled f_i - w_i, g[18] = pulled g_q (x, y, z);
// overwritten with the post-collision values.  MODE K3_FILTER: gr[3 q + a]
// is the central difference along axis a of field q (rho - 1, j, B) of the
// streamed populations; MODE K3_CARATI: tau_e3, tau_m3 are the relaxation
// times.
template <class R, int MODE = K3_LOCAL>
__device__ __forceinline__ void collide3(R (&d)[kQ], R (&g)[3 * kM], const Coll3<R>& c,
                                         const R* gr = nullptr, R tau_e3 = R(0),
                                         R tau_m3 = R(0)) {
    // moments: rho - 1, j = rho u, B, and the second moment S = sum d c c
    R drho = R(0), jx = R(0), jy = R(0), jz = R(0);
    R sxx = R(0), syy = R(0), szz = R(0), sxy = R(0), sxz = R(0), syz = R(0);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int cx = v1(i % 3), cy = v1((i / 3) % 3), cz = v1(i / 9);
        drho += d[i];
        if (cx) jx += cx > 0 ? d[i] : -d[i];
        if (cy) jy += cy > 0 ? d[i] : -d[i];
        if (cz) jz += cz > 0 ? d[i] : -d[i];
        if (cx) sxx += d[i];
        if (cy) syy += d[i];
        if (cz) szz += d[i];
        if (cx && cy) sxy += cx * cy > 0 ? d[i] : -d[i];
        if (cx && cz) sxz += cx * cz > 0 ? d[i] : -d[i];
        if (cy && cz) syz += cy * cz > 0 ? d[i] : -d[i];
    }
    R bx = R(0), by = R(0), bz = R(0);
#pragma unroll
    for (int q = 0; q < kM; ++q) {
        bx += g[3 * q];
        by += g[3 * q + 1];
        bz += g[3 * q + 2];
    }
    const R rho = R(1) + drho;
    const R irho = rcp(rho);
    const R ux = jx * irho, uy = jy * irho, uz = jz * irho;
    const R bb = fmad(bz, bz, fmad(by, by, bx * bx));
    const R jj = fmad(jz, uz, fmad(jy, uy, jx * ux));  // |j|^2 / rho

    // non-equilibrium stress without its isotropic part: S - j j / rho + B B
    // (the equilibrium's rho/3 I and |B|^2/2 I drop out of the traceless part)
    R pxx = fmad(bx, bx, fmad(-jx, ux, sxx)), pyy = fmad(by, by, fmad(-jy, uy, syy)),
      pzz = fmad(bz, bz, fmad(-jz, uz, szz));
    const R pxy = fmad(bx, by, fmad(-jx, uy, sxy)), pxz = fmad(bx, bz, fmad(-jx, uz, sxz)),
            pyz = fmad(by, bz, fmad(-jy, uz, syz));
    const R tr = (pxx + pyy + pzz) * (R(1) / R(3));
    pxx -= tr;
    pyy -= tr;
    pzz -= tr;

    // magnetic non-equilibrium first moment: N_ab = (g_{+a,b} - g_{-a,b})
    // - (u_a B_b - B_a u_b); its axial vector
    const R ex = fmad(uy, bz, -(uz * by)), ey = fmad(uz, bx, -(ux * bz)),
            ez = fmad(ux, by, -(uy * bx));  // u x B
    const R ax = fmad(R(-2), ex, (g[3 * 2 + 2] - g[3 * 3 + 2]) - (g[3 * 4 + 1] - g[3 * 5 + 1]));
    const R ay = fmad(R(-2), ey, (g[3 * 4 + 0] - g[3 * 5 + 0]) - (g[3 * 0 + 2] - g[3 * 1 + 2]));
    const R az = fmad(R(-2), ez, (g[3 * 0 + 1] - g[3 * 1 + 1]) - (g[3 * 2 + 0] - g[3 * 3 + 0]));

    R tau_e = c.tn, tau_m = c.te;
    if constexpr (MODE == K3_CARATI) {
        tau_e = tau_e3;
        tau_m = tau_m3;
    }
    if (MODE == K3_LOCAL && c.les) {
        const R off = fmad(pyz, pyz, fmad(pxz, pxz, pxy * pxy));
        const R pp = fmad(R(2), off, fmad(pzz, pzz, fmad(pyy, pyy, pxx * pxx)));
        const R Q = sqrt_(R(2) * pp);
        tau_e = R(0.5) * (c.tn + sqrt_(fmad(c.k18 * Q, irho, c.tn2)));
        const R J = sqrt_(fmad(az, az, fmad(ay, ay, ax * ax)));
        tau_m = R(0.5) * (c.te + sqrt_(fmad(c.k36, J, c.te2)));
    }
    const R s = rcp(tau_e);
    const R sm = rcp(tau_m);
    const R sixth = R(1) / R(6);
    const R u3[3] = {ux, uy, uz}, b3[3] = {bx, by, bz};
    if constexpr (MODE == K3_FILTER) {
        const R j3[3] = {jx, jy, jz};
        // The filter rules of Sec. 2 applied to every nonlinear term of the
        // equilibria.  With G_a = d j_a - u_a d rho and H_b = d B_b - (B_b /
        // rho) d rho, the ratio rule (Eq. FilterExampleLarge) is
        // Rt(X_a, Y_b; rho) = G_a . H_b / (12 rho) and the product rule (Eq.
        // FilterExampleSmall) P(B_a, B_b) = d B_a . d B_b / 12; times Delta^2:
        //   (c.j)^2/rho -> c.R.c,  |j|^2/rho -> tr R,  (c.B)^2 -> c.P.c,
        //   |B|^2 -> tr P,  u_a B_b - B_a u_b -> + Rt(j_a, B_b) - Rt(j_b, B_a).
        R G[3][3], H[3][3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                G[a][k] = fmad(-u3[a], gr[k], gr[3 * (1 + a) + k]);
                H[a][k] = fmad(-b3[a] * irho, gr[k], gr[3 * (4 + a) + k]);
            }
        const R ci = c.d12 * irho;
        auto dotGG = [&](int a, int b) { return fmad(G[a][2], G[b][2], fmad(G[a][1], G[b][1], G[a][0] * G[b][0])); };
        auto dotBB = [&](int a, int b) {
            const R* A = gr + 3 * (4 + a);
            const R* B = gr + 3 * (4 + b);
            return fmad(A[2], B[2], fmad(A[1], B[1], A[0] * B[0]));
        };
        auto dotGH = [&](int a, int b) { return fmad(G[a][2], H[b][2], fmad(G[a][1], H[b][1], G[a][0] * H[b][0])); };
        // Q = j u - B B + Delta^2 (R - P), symmetric; the quadratic form of
        // the equilibrium's nonlinear part
        R Rd[3], Pd[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Rd[a] = ci * dotGG(a, a);
            Pd[a] = c.d12 * dotBB(a, a);
        }
        const R trR = Rd[0] + Rd[1] + Rd[2], trP = Pd[0] + Pd[1] + Pd[2];
        R qd[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) qd[a] = fmad(-b3[a], b3[a], fmad(j3[a], u3[a], Rd[a] - Pd[a]));
        // off-diagonal entries doubled: 2 Q_ab for (xy, xz, yz)
        R q2[3], em[3];
        {
            const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const int a = pa[k], b = pb[k];
                const R t = fmad(ci, dotGG(a, b), fmad(-c.d12, dotBB(a, b), fmad(j3[a], u3[b], -(b3[a] * b3[b]))));
                q2[k] = R(2) * t;
                em[k] = fmad(ci, dotGH(a, b) - dotGH(b, a), fmad(u3[a], b3[b], -(b3[a] * u3[b])));
            }
        }
        // sums of the diagonal over the non-zero axes of c
        const R sxy = qd[0] + qd[1], sxz = qd[0] + qd[2], syz = qd[1] + qd[2], sxyz = sxy + qd[2];
        const R base = fmad(R(-0.75), bb + trP, fmad(R(-1.5), jj + trR, drho));
        const R hh = R(2.25) * (bb + trP);
#pragma unroll
        for (int i = 0; i < kQ; ++i) {
            const int cx = v1(i % 3), cy = v1((i / 3) % 3), cz = v1(i / 9);
            R cj = R(0);
            if (cx) cj += cx > 0 ? jx : -jx;
            if (cy) cj += cy > 0 ? jy : -jy;
            if (cz) cj += cz > 0 ? jz : -jz;
            const int cc = cx * cx + cy * cy + cz * cz;
            R qf = R(0);
            if (cc == 1) qf = cx ? qd[0] : (cy ? qd[1] : qd[2]);
            if (cc == 2) qf = cz == 0 ? sxy : (cy == 0 ? sxz : syz);
            if (cc == 3) qf = sxyz;
            if (cx && cy) qf += cx * cy > 0 ? q2[0] : -q2[0];
            if (cx && cz) qf += cx * cz > 0 ? q2[1] : -q2[1];
            if (cy && cz) qf += cy * cz > 0 ? q2[2] : -q2[2];
            R t = fmad(R(3), cj, cc ? fmad(hh, R(cc), base) : base);
            t = fmad(R(4.5), qf, t);
            const R deq = wqr<R>(i) * t;
            d[i] = fmad(-s, d[i] - deq, d[i]);
        }
#pragma unroll
        for (int q = 0; q < kM; ++q) {
            const int a = q / 2;
            const R sg3 = q % 2 ? R(-3) : R(3);
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (b == a) {
                    g[3 * q + b] = fmad(-sm, g[3 * q + b] - sixth * b3[b], g[3 * q + b]);
                    continue;
                }
                // e(a, b) = -e(b, a); em holds (xy, xz, yz)
                const int k = a + b - 1;
                const R e = a < b ? em[k] : -em[k];
                const R geq = sixth * fmad(sg3, e, b3[b]);
                g[3 * q + b] = fmad(-sm, g[3 * q + b] - geq, g[3 * q + b]);
            }
        }
        return;
    }
    // equilibria in deviation form: w [(rho - 1) + 3 c.j + 9/2 (c.j)^2 / rho
    // - 3/2 j^2 / rho] + 9/2 w [|B|^2/2 |c|^2 - (c.B)^2 - |B|^2/6]
    const R base = fmad(R(-0.75), bb, fmad(R(-1.5), jj, drho));
    const R half_bb = R(2.25) * bb;
    const R k45 = R(4.5) * irho;
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int cx = v1(i % 3), cy = v1((i / 3) % 3), cz = v1(i / 9);
        R cj = R(0), cb = R(0);
        if (cx) {
            cj += cx > 0 ? jx : -jx;
            cb += cx > 0 ? bx : -bx;
        }
        if (cy) {
            cj += cy > 0 ? jy : -jy;
            cb += cy > 0 ? by : -by;
        }
        if (cz) {
            cj += cz > 0 ? jz : -jz;
            cb += cz > 0 ? bz : -bz;
        }
        const int cc = cx * cx + cy * cy + cz * cz;
        R t = fmad(R(3), cj, cc ? fmad(half_bb, R(cc), base) : base);
        t = fmad(k45 * cj, cj, fmad(R(-4.5) * cb, cb, t));
        const R deq = wqr<R>(i) * t;
        d[i] = fmad(-s, d[i] - deq, d[i]);
    }
    // magnetic: g_q^eq = (1/6) [B + 3 ((C.u) B - (C.B) u)]
#pragma unroll
    for (int q = 0; q < kM; ++q) {
        const int a = q / 2;           // axis
        const R sg3 = q % 2 ? R(-3) : R(3);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (b == a) {  // (C.u) B_a - (C.B) u_a = 0 along the axis itself
                g[3 * q + b] = fmad(-sm, g[3 * q + b] - sixth * b3[b], g[3 * q + b]);
                continue;
            }
            const R e = fmad(u3[a], b3[b], -(b3[a] * u3[b]));
            const R geq = sixth * fmad(sg3, e, b3[b]);
            g[3 * q + b] = fmad(-sm, g[3 * q + b] - geq, g[3 * q + b]);
        }
    }
}

// Lattice shape, plane stride, and the planes [zb, ze) a launch covers
// (zb may be -1 and ze nz + 1 for a moments pass around a plane range;
// planes wrap periodically).
struct Geom3 {
    int nx, ny, nz;
    long long ps;
    int zb, ze;
};

__host__ __device__ __forceinline__ int wrapz3(int z, int nz) { return z < 0 ? z + nz : (z >= nz ? z - nz : z); }

// The pull of one thread: V consecutive nodes along x of one (y, z) row;
// every plane one aligned vector load, the x-shifted planes completed from
// the neighbouring lane by a shuffle (lanes at a warp edge or the periodic
// wrap load the missing element).  tc < total (padding threads pass the
// last real index, so every address is valid).
template <int P, int V>
__device__ __forceinline__ void pull3(const typename Fmt3<P>::S* __restrict__ src, const Geom3 g,
                                      unsigned tc, typename Fmt3<P>::S (&raw)[kP][V], int& x0,
                                      int& y, int& z) {
    using S = typename Fmt3<P>::S;
    const int lane = threadIdx.x & 31;
    const unsigned nxv = (unsigned)(g.nx / V);
    const unsigned row = tc / nxv;  // y + ny (z - zb)
    x0 = (int)(tc - row * nxv) * V;
    y = (int)(row % (unsigned)g.ny);
    z = wrapz3(g.zb + (int)(row / (unsigned)g.ny), g.nz);
    const bool has_left = lane > 0 && x0 > 0;
    const bool has_right = lane < 31 && x0 + V < g.nx;
    const int xl = x0 == 0 ? g.nx - 1 : x0 - 1;
    const int xr = x0 + V == g.nx ? 0 : x0 + V;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
#pragma unroll
    for (int p = 0; p < kP; ++p) {
        const int cx = pcx(p), cy = pcy(p), cz = pcz(p);
        const int ry = cy == 0 ? y : (cy > 0 ? ym : yp);
        const int rz = cz == 0 ? z : (cz > 0 ? zm : zp);
        const S* base = src + p * g.ps + ((long long)rz * g.ny + ry) * g.nx;
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
}

// The seven fields rho - 1, j, B of decoded populations, summed in the
// order collide3 sums them.
template <class R>
__device__ __forceinline__ void fields3(const R (&d)[kQ], const R (&g)[3 * kM], R (&m)[7]) {
    R drho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int i = 0; i < kQ; ++i) {
        const int cx = v1(i % 3), cy = v1((i / 3) % 3), cz = v1(i / 9);
        drho += d[i];
        if (cx) jx += cx > 0 ? d[i] : -d[i];
        if (cy) jy += cy > 0 ? d[i] : -d[i];
        if (cz) jz += cz > 0 ? d[i] : -d[i];
    }
    R bx = R(0), by = R(0), bz = R(0);
#pragma unroll
    for (int q = 0; q < kM; ++q) {
        bx += g[3 * q];
        by += g[3 * q + 1];
        bz += g[3 * q + 2];
    }
    m[0] = drho;
    m[1] = jx;
    m[2] = jy;
    m[3] = jz;
    m[4] = bx;
    m[5] = by;
    m[6] = bz;
}

// The collision of one node under a gradient closure.  nbv(q, n): field q
// (rho - 1, jx, jy, jz, Bx, By, Bz of the streamed populations) at
// neighbour n (x+, x-, y+, y-, z+, z-).
template <class R, int MODE, class NB>
__device__ __forceinline__ void closure_collide3(R (&d)[kQ], R (&gg)[3 * kM], const Coll3<R>& c,
                                                 NB nbv) {
    if constexpr (MODE == K3_FILTER) {
        R gr[21];
#pragma unroll
        for (int q = 0; q < 7; ++q)
#pragma unroll
            for (int a = 0; a < 3; ++a) gr[3 * q + a] = R(0.5) * (nbv(q, 2 * a) - nbv(q, 2 * a + 1));
        collide3<R, K3_FILTER>(d, gg, c, gr);
    } else {
        // u = j / rho and B at the six neighbours, central differences
        R gu[3][3], gb[3][3];  // [component][axis]
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const R ip = rcp(R(1) + nbv(0, 2 * a)), im = rcp(R(1) + nbv(0, 2 * a + 1));
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                gu[b][a] = R(0.5) * fmad(nbv(1 + b, 2 * a), ip, -(nbv(1 + b, 2 * a + 1) * im));
                gb[b][a] = R(0.5) * (nbv(4 + b, 2 * a) - nbv(4 + b, 2 * a + 1));
            }
        }
        // S^v : S^b with S_ab = (d_b v_a + d_a v_b) / 2
        R ss = fmad(gu[2][2], gb[2][2], fmad(gu[1][1], gb[1][1], gu[0][0] * gb[0][0]));
        const int pa[3] = {0, 0, 1}, pb[3] = {1, 2, 2};
#pragma unroll
        for (int k2 = 0; k2 < 3; ++k2) {
            const int a = pa[k2], b = pb[k2];
            ss = fmad(R(0.5) * (gu[a][b] + gu[b][a]), gb[a][b] + gb[b][a], ss);
        }
        const R nu_t = c.cd2 * sqrt_(fabs(ss));
        const R om[3] = {gu[2][1] - gu[1][2], gu[0][2] - gu[2][0], gu[1][0] - gu[0][1]};
        const R jc[3] = {gb[2][1] - gb[1][2], gb[0][2] - gb[2][0], gb[1][0] - gb[0][1]};
        const R jw = fmad(jc[2], om[2], fmad(jc[1], om[1], jc[0] * om[0]));
        const R eta_t = c.cd2 * (jw > R(0) ? R(1) : (jw < R(0) ? R(-1) : R(0))) * sqrt_(fabs(jw));
        const R te = fmax(fmad(R(3), eta_t, c.te), R(0.5));
        collide3<R, K3_CARATI>(d, gg, c, nullptr, fmad(R(3), nu_t, c.tn), te);
    }
}

// Pull + collide + store of V nodes.  MODE K3_FILTER / K3_CARATI read the
// seven field planes mom (plane stride g.ps) at the six neighbours of each
// node.  t >= total: a padding thread (valid addresses, no store).
// FP16 storage, two nodes per thread: every plane is one 32-bit word per
// thread (node x0 in the low half, x0 + 1 in the high half), the x-shifted
// planes a funnel of half-words with the neighbouring lane's word
// (byte_perm).  The word holds the two nodes' inputs and, once a node is
// collided, its output in the same half, so the 45 planes take 45
// registers instead of 90.
template <int MODE>
__device__ __forceinline__ void step3_body_h(const unsigned short* __restrict__ src,
                                             unsigned short* __restrict__ dst, const Geom3 g,
                                             unsigned t, unsigned total, const Coll3<float>& c,
                                             const float* __restrict__ mom) {
    const int lane = threadIdx.x & 31;
    const bool live = t < total;
    const unsigned tc = live ? t : total - 1;
    const unsigned nxv = (unsigned)(g.nx / 2);
    const unsigned row = tc / nxv;  // y + ny (z - zb)
    const int x0 = (int)(tc - row * nxv) * 2;
    const int y = (int)(row % (unsigned)g.ny), z = wrapz3(g.zb + (int)(row / (unsigned)g.ny), g.nz);
    const bool has_left = lane > 0 && x0 > 0;
    const bool has_right = lane < 31 && x0 + 2 < g.nx;
    const int xl = x0 == 0 ? g.nx - 1 : x0 - 1;
    const int xr = x0 + 2 == g.nx ? 0 : x0 + 2;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
    unsigned w[kP];
#pragma unroll
    for (int p = 0; p < kP; ++p) {
        const int cx = pcx(p), cy = pcy(p), cz = pcz(p);
        const int ry = cy == 0 ? y : (cy > 0 ? ym : yp);
        const int rz = cz == 0 ? z : (cz > 0 ? zm : zp);
        const unsigned short* base = src + p * g.ps + ((long long)rz * g.ny + ry) * g.nx;
        const unsigned own = *reinterpret_cast<const unsigned*>(base + x0);
        if (cx == 0) {
            w[p] = own;
        } else if (cx > 0) {  // nodes x0 - 1, x0
            unsigned prev = __shfl_up_sync(0xffffffffu, own, 1);
            if (!has_left) prev = (unsigned)base[xl] << 16;
            w[p] = __byte_perm(prev, own, 0x5432);
        } else {  // nodes x0 + 1, x0 + 2
            unsigned next = __shfl_down_sync(0xffffffffu, own, 1);
            if (!has_right) next = (unsigned)base[xr];
            w[p] = __byte_perm(own, next, 0x5432);
        }
    }
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {
        const int sh = 16 * k;
        float d[kQ], gg[3 * kM];
#pragma unroll
        for (int i = 0; i < kQ; ++i)
            d[i] = Fmt3<P_FP16_DEV>::dec((unsigned short)(w[i] >> sh), i, c.i16);
#pragma unroll
        for (int q = 0; q < 3 * kM; ++q)
            gg[q] = Fmt3<P_FP16_DEV>::dec((unsigned short)(w[kQ + q] >> sh), kQ + q, c.i16);
        if constexpr (MODE == K3_LOCAL) {
            collide3<float>(d, gg, c);
        } else {
            const int x = x0 + k;
            const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
            const long long rowo = ((long long)z * g.ny + y) * g.nx;
            const long long nb[6] = {rowo + xp, rowo + xm, ((long long)z * g.ny + yp) * g.nx + x,
                                     ((long long)z * g.ny + ym) * g.nx + x,
                                     ((long long)zp * g.ny + y) * g.nx + x,
                                     ((long long)zm * g.ny + y) * g.nx + x};
            closure_collide3<float, MODE>(d, gg, c, [&](int q, int n) { return __ldg(mom + q * g.ps + nb[n]); });
        }
#pragma unroll
        for (int p = 0; p < kP; ++p) {
            const unsigned e = Fmt3<P_FP16_DEV>::enc(p < kQ ? d[p] : gg[p - kQ], p, c.s16);
            w[p] = (w[p] & ~(0xffffu << sh)) | (e << sh);
        }
    }
    if (live) {
        const long long node = ((long long)z * g.ny + y) * g.nx + x0;
#pragma unroll
        for (int p = 0; p < kP; ++p) *reinterpret_cast<unsigned*>(dst + p * g.ps + node) = w[p];
    }
}

template <int P, int V, int MODE>
__device__ __forceinline__ void step3_body(const typename Fmt3<P>::S* __restrict__ src,
                                           typename Fmt3<P>::S* __restrict__ dst, const Geom3 g,
                                           unsigned t, unsigned total,
                                           const Coll3<typename Fmt3<P>::R>& c,
                                           const typename Fmt3<P>::R* __restrict__ mom) {
    using S = typename Fmt3<P>::S;
    using R = typename Fmt3<P>::R;
    if constexpr (P == P_FP16_DEV && V == 2) {
        step3_body_h<MODE>(src, dst, g, t, total, c, mom);
        return;
    }
    const bool live = t < total;
    const unsigned tc = live ? t : total - 1;
    int x0, y, z;
    S raw[kP][V];
    pull3<P, V>(src, g, tc, raw, x0, y, z);
#pragma unroll
    for (int k = 0; k < V; ++k) {
        R d[kQ], gg[3 * kM];
#pragma unroll
        for (int i = 0; i < kQ; ++i) d[i] = Fmt3<P>::dec(raw[i][k], i, c.i16);
#pragma unroll
        for (int q = 0; q < 3 * kM; ++q) gg[q] = Fmt3<P>::dec(raw[kQ + q][k], kQ + q, c.i16);
        if constexpr (MODE == K3_LOCAL) {
            collide3<R>(d, gg, c);
        } else {
            const int x = x0 + k;
            const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
            const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
            const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
            const long long row = ((long long)z * g.ny + y) * g.nx;
            const long long nb[6] = {row + xp, row + xm, ((long long)z * g.ny + yp) * g.nx + x,
                                     ((long long)z * g.ny + ym) * g.nx + x,
                                     ((long long)zp * g.ny + y) * g.nx + x,
                                     ((long long)zm * g.ny + y) * g.nx + x};
            closure_collide3<R, MODE>(d, gg, c, [&](int q, int n) { return ldg_r(mom + q * g.ps + nb[n]); });
        }
#pragma unroll
        for (int i = 0; i < kQ; ++i) raw[i][k] = Fmt3<P>::enc(d[i], i, c.s16);
#pragma unroll
        for (int q = 0; q < 3 * kM; ++q) raw[kQ + q][k] = Fmt3<P>::enc(gg[q], kQ + q, c.s16);
    }
    if (live) {
        const long long node = ((long long)z * g.ny + y) * g.nx + x0;
#pragma unroll
        for (int p = 0; p < kP; ++p) {
            Pack<S, V> o;
#pragma unroll
            for (int k = 0; k < V; ++k) o.v[k] = raw[p][k];
            *reinterpret_cast<Pack<S, V>*>(dst + p * g.ps + node) = o;
        }
    }
}

// The moments pass of the gradient closures: rho - 1, j, B of the
// populations streamed into every node, into seven planes of R.
template <int P, int V>
__global__ void __launch_bounds__(256) mom3_kernel(const typename Fmt3<P>::S* __restrict__ src,
                                                   typename Fmt3<P>::R* __restrict__ mom, Geom3 g,
                                                   unsigned total, unsigned total_pad, float i16) {
    using S = typename Fmt3<P>::S;
    using R = typename Fmt3<P>::R;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total_pad; t += stride) {
        const bool live = t < total;
        int x0, y, z;
        S raw[kP][V];
        pull3<P, V>(src, g, live ? t : total - 1, raw, x0, y, z);
        R m[7][V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            R d[kQ], gg[3 * kM], mk[7];
#pragma unroll
            for (int i = 0; i < kQ; ++i) d[i] = Fmt3<P>::dec(raw[i][k], i, i16);
#pragma unroll
            for (int q = 0; q < 3 * kM; ++q) gg[q] = Fmt3<P>::dec(raw[kQ + q][k], kQ + q, i16);
            fields3<R>(d, gg, mk);
#pragma unroll
            for (int q = 0; q < 7; ++q) m[q][k] = mk[q];
        }
        if (live) {
            const long long node = ((long long)z * g.ny + y) * g.nx + x0;
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                Pack<R, V> o;
#pragma unroll
                for (int k = 0; k < V; ++k) o.v[k] = m[q][k];
                *reinterpret_cast<Pack<R, V>*>(mom + q * g.ps + node) = o;
            }
        }
    }
}

// ---- fused one-pass form of the gradient closures --------------------------
// A CTA owns a tile of kFX x kFTY columns (x, y) and a segment [z0, z1) of
// planes, and sweeps up it.  Shared memory holds the seven fields of the
// streamed populations of three consecutive planes over the tile and a
// one-node halo (a ring), and the 45 pulled values of the tile's nodes for
// two planes.  Per plane z: phase A pulls the populations of plane z + 1 at
// the tile and halo nodes, writes their fields into the ring and keeps the
// tile nodes' values; a barrier; phase B takes the values of plane z kept
// one plane earlier, the central differences from the ring, collides and
// stores; a barrier.  Every stored value is read once per step by phase A
// (halo pulls are neighbouring tiles' lines, from L2), so the step moves
// the 360 B/node of a plain FP32 step instead of the two-pass 416 + 180 B.
// The two barriers let phase A of plane z + 2 overwrite the ring slot of
// plane z - 1 and the kept values of plane z only after every thread has
// finished phase B of plane z.  Fields, differences and collision are those
// of the two-pass kernels, so both give the same bits.
// Measured on GB300, FP32, 256^3, les 2 (MLUPS, fraction of the measured copy
// bandwidth at 360 B/node): 10.2K (0.54); the two-pass kernels 8.8K (0.47),
// each of its passes latency-bound at 0.67-0.73 of copy bandwidth.  Earlier
// forms, measured slower: phase B pulling plane z again from L2 instead of
// keeping it (8-row tiles, 9.6K: ncu at 128^3 shows that re-pull missing L2
// for ~40% of its lines, DRAM reads 1.47x the stored state, 12 warps per SM
// at 139 registers, issue 51% busy; 16-row tiles 5.9K, re-reads 2.1x), an
// L1 prefetch of the next node's lines (8.0K), 4 and 5 CTAs per SM at 127
// and 96 registers (9.5K, 8.8K), 8-row tiles with kept values (one CTA per
// SM, 7.0K).  What remains is latency in phase A at 12 warps per SM.
constexpr int kFX = 32, kFTY = 4, kFThreads = 128, kFRing = 3;

constexpr int fused3_smem_floats() { return kFRing * 7 * (kFTY + 2) * (kFX + 2) + 2 * kP * kFTY * kFX; }

__device__ __forceinline__ int wrap3i(int a, int n) { return a < 0 ? a + n : (a >= n ? a - n : a); }

// The 45 populations streamed into node (x, y, z), decoded.
template <int P>
__device__ __forceinline__ void pull_node3(const typename Fmt3<P>::S* __restrict__ src, const Geom3& g,
                                           int x, int y, int z, typename Fmt3<P>::R (&d)[kQ],
                                           typename Fmt3<P>::R (&gg)[3 * kM], float i16) {
    const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
#pragma unroll
    for (int p = 0; p < kP; ++p) {
        const int cx = pcx(p), cy = pcy(p), cz = pcz(p);
        const int rx = cx == 0 ? x : (cx > 0 ? xm : xp);
        const int ry = cy == 0 ? y : (cy > 0 ? ym : yp);
        const int rz = cz == 0 ? z : (cz > 0 ? zm : zp);
        const unsigned off = ((unsigned)rz * (unsigned)g.ny + (unsigned)ry) * (unsigned)g.nx + (unsigned)rx;
        const auto v = __ldg(src + p * g.ps + off);
        if (p < kQ)
            d[p] = Fmt3<P>::dec(v, p, i16);
        else
            gg[p - kQ] = Fmt3<P>::dec(v, p, i16);
    }
}

template <int P, int MODE>
__global__ void __launch_bounds__(kFThreads, P == P_FP64 || P == P_FF ? 1 : 3)
    fused3_kernel(const typename Fmt3<P>::S* __restrict__ src, typename Fmt3<P>::S* __restrict__ dst,
                  Geom3 g, int tiles_x, int tiles_y, int seglen, Coll3<typename Fmt3<P>::R> c) {
    using R = typename Fmt3<P>::R;
    extern __shared__ __align__(16) unsigned char fused3_smem[];
    constexpr int HX = kFX + 2, HP = (kFTY + 2) * HX;  // halo row, halo plane
    constexpr int KP = kFTY * kFX;                     // one kept plane of a population
    R* ring = reinterpret_cast<R*>(fused3_smem);
    R* kept = ring + kFRing * 7 * HP;
    const int tile = (int)blockIdx.x % (tiles_x * tiles_y);
    const int seg = (int)blockIdx.x / (tiles_x * tiles_y);
    const int x0 = (tile % tiles_x) * kFX, y0 = (tile / tiles_x) * kFTY;
    const int tw = min(kFX, g.nx - x0), th = min(kFTY, g.ny - y0);
    const int z0 = g.zb + seg * seglen, z1 = min(z0 + seglen, g.ze);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int hw = tw + 2, hn = hw * (th + 2);

    // phase A: the fields of plane zz at the tile and halo nodes into its ring
    // slot, the tile nodes' pulled values into kept buffer zz mod 2
    auto phase_a = [&](int zz) {
        const int zw = wrap3i(zz, g.nz);
        R* slot = ring + (size_t)(((zz % kFRing) + kFRing) % kFRing) * 7 * HP;
        R* kz = kept + (size_t)(zz & 1) * kP * KP;
        for (int i = tid; i < hn; i += kFThreads) {
            const int hy = i / hw, hx = i - hy * hw;
            const int x = wrap3i(x0 - 1 + hx, g.nx), y = wrap3i(y0 - 1 + hy, g.ny);
            R d[kQ], gg[3 * kM], m[7];
            pull_node3<P>(src, g, x, y, zw, d, gg, c.i16);
            fields3<R>(d, gg, m);
#pragma unroll
            for (int q = 0; q < 7; ++q) slot[q * HP + hy * HX + hx] = m[q];
            if (hx >= 1 && hx <= tw && hy >= 1 && hy <= th) {
                R* k0 = kz + (hy - 1) * kFX + (hx - 1);
#pragma unroll
                for (int p = 0; p < kQ; ++p) k0[p * KP] = d[p];
#pragma unroll
                for (int q = 0; q < 3 * kM; ++q) k0[(kQ + q) * KP] = gg[q];
            }
        }
    };

    phase_a(z0 - 1);
    phase_a(z0);
    for (int z = z0; z < z1; ++z) {
        phase_a(z + 1);
        __syncthreads();
        const R* sm = ring + (size_t)(((z - 1) % kFRing + kFRing) % kFRing) * 7 * HP;
        const R* s0 = ring + (size_t)((z % kFRing)) * 7 * HP;
        const R* sp = ring + (size_t)(((z + 1) % kFRing)) * 7 * HP;
        // phase B: one tile node per thread (warp = row, lane = column)
        if (warp < th && lane < tw) {
            const int ly = warp;
            const int x = x0 + lane, y = y0 + ly;
            R d[kQ], gg[3 * kM];
            const R* k0 = kept + (size_t)(z & 1) * kP * KP + ly * kFX + lane;
#pragma unroll
            for (int p = 0; p < kQ; ++p) d[p] = k0[p * KP];
#pragma unroll
            for (int q = 0; q < 3 * kM; ++q) gg[q] = k0[(kQ + q) * KP];
            const int c0 = (ly + 1) * HX + lane + 1;
            closure_collide3<R, MODE>(d, gg, c, [&](int q, int n) {
                const int o = q * HP;
                return n == 0 ? s0[o + c0 + 1]
                     : n == 1 ? s0[o + c0 - 1]
                     : n == 2 ? s0[o + c0 + HX]
                     : n == 3 ? s0[o + c0 - HX]
                     : n == 4 ? sp[o + c0]
                              : sm[o + c0];
            });
            const unsigned node = ((unsigned)z * (unsigned)g.ny + (unsigned)y) * (unsigned)g.nx + (unsigned)x;
#pragma unroll
            for (int i = 0; i < kQ; ++i) dst[i * g.ps + node] = Fmt3<P>::enc(d[i], i, c.s16);
#pragma unroll
            for (int q = 0; q < 3 * kM; ++q) dst[(kQ + q) * g.ps + node] = Fmt3<P>::enc(gg[q], kQ + q, c.s16);
        }
        __syncthreads();
    }
}

// ---- warp-specialised fused form -------------------------------------------
// The same fields, differences and collision as fused3_kernel (and the
// two-pass kernels), so the same bits, with the pulls of the neighbourhood
// taken off the collision's critical path.  A CTA of 640 threads owns a tile
// of 32 x 8 columns.  Warps 8-19 are producers: one of the 34 x 10 tile and
// halo nodes per thread, they pull its 45 populations of plane z and write
// its seven fields into a ring of kWF plane slots in shared memory.  Warps
// 0-7 are consumers (warp = tile row, lane = column): for plane z each pulls
// its own node's 45 populations again (lines the producers pulled two
// planes earlier, from L2), issuing the loads before it waits for the
// fields of plane z + 1, then takes the central differences from the ring,
// collides and stores.  Keeping the pulled values of the tile in shared
// memory instead (a 138 KB ring) measured slower: shared memory takes L1's
// room, and L1 holds the loads in flight.  The register file is split by
// warpgroup (setmaxnreg): producers hold their pulled values in 64
// registers, consumers theirs and the collision in 144 (384 x 64 + 256 x 144
// = 640 x 96, the launch's registers, confirmed on the host from the
// compiled kernel before the first launch).  Producers and consumers hand
// slots over on shared-memory mbarriers, one arrival per warp after a warp
// barrier: full[K mod kWB] completes when every producer warp has written
// the fields of plane index K (each arrival a release, the waits acquire),
// empty[K mod kWF] when every consumer warp is done reading slot K.  With
// four slots the producers pull plane z + 3 while the consumers collide
// plane z (deeper rings measured slower); a producer issues its pulls before
// it waits for its slot.  A CTA is persistent over work
// units (tile, z-segment): unit u = blockIdx.x + i gridDim.x, each segment
// pulling one plane below and one above its own, and the counters run on
// across units, so a unit's first pulls overlap the previous unit's last
// collisions.  Every wait is bounded (~2 s); on expiry the warp sets bit 1
// of *status, and every warp leaves at its next check.
constexpr int kWX = 32, kWY = 8, kWF = 4, kWB = 4;
constexpr int kWsCons = kWX * kWY, kWsProd = 384, kWsThreads = kWsCons + kWsProd;
constexpr int kWsLaunchRegs = 96, kWsProdRegs = 64, kWsConsRegs = 144;
static_assert(kWsProd * kWsProdRegs + kWsCons * kWsConsRegs <= kWsThreads * kWsLaunchRegs,
              "the warpgroups' registers exceed the launch's");
static_assert(kWsThreads * kWsLaunchRegs <= 65536, "the launch's registers exceed an SM's");
constexpr int kWsHX = kWX + 2, kWsHP = kWsHX * (kWY + 2);  // halo row, halo plane (340)
static_assert(kWsHP <= kWsProd, "one tile or halo node per producer thread");
// A producer warp arriving for plane index K must find every producer warp
// past K - kWB.  It has waited for slot K - kWF to be handed back, and the
// consumers hand back a unit's last two slots after waiting only for its
// last plane, so all producers are known to be past K - kWF, no further:
// the barrier ring must be at least as long as the slot ring.
static_assert(kWB >= kWF && kWB >= 3, "full-barrier ring shorter than the slot ring");
constexpr size_t kWsSmem = (size_t)kWF * 7 * kWsHP * 4 + (kWB + kWF) * 8 + 16;

// The 45 populations streamed into node (x, y, z), stored values.
template <int P>
__device__ __forceinline__ void pull_raw3(const typename Fmt3<P>::S* __restrict__ src, const Geom3& g,
                                          int x, int y, int z, typename Fmt3<P>::S (&raw)[kP]) {
    const int xm = x == 0 ? g.nx - 1 : x - 1, xp = x == g.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? g.ny - 1 : y - 1, yp = y == g.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? g.nz - 1 : z - 1, zp = z == g.nz - 1 ? 0 : z + 1;
#pragma unroll
    for (int p = 0; p < kP; ++p) {
        const int cx = pcx(p), cy = pcy(p), cz = pcz(p);
        const int rx = cx == 0 ? x : (cx > 0 ? xm : xp);
        const int ry = cy == 0 ? y : (cy > 0 ? ym : yp);
        const int rz = cz == 0 ? z : (cz > 0 ? zm : zp);
        const unsigned off = ((unsigned)rz * (unsigned)g.ny + (unsigned)ry) * (unsigned)g.nx + (unsigned)rx;
        raw[p] = __ldg(src + p * g.ps + off);
    }
}

template <int P, int MODE>
__global__ void __launch_bounds__(kWsThreads, 1)
    ws3_kernel(const typename Fmt3<P>::S* __restrict__ src, typename Fmt3<P>::S* __restrict__ dst,
               Geom3 g, int tiles_x, int tiles_y, int seglen, int units,
               Coll3<typename Fmt3<P>::R> c, int* status, int debug) {
    using R = typename Fmt3<P>::R;
    using S = typename Fmt3<P>::S;
    static_assert(std::is_same<R, float>::value, "the warp-specialised kernel is for FP32 arithmetic");
    extern __shared__ __align__(16) unsigned char ws3_smem[];
    R* fring = reinterpret_cast<R*>(ws3_smem);
    unsigned long long* full = reinterpret_cast<unsigned long long*>(fring + kWF * 7 * kWsHP);
    unsigned long long* empty = full + kWB;
    int* abort_ = reinterpret_cast<int*>(empty + kWF);
    const int tid = threadIdx.x, lane = tid & 31;
    constexpr unsigned kAll = 0xffffffffu;
    if (tid == 0) {
        for (int b = 0; b < kWB; ++b) mbar_init(&full[b], kWsProd / 32);
        for (int b = 0; b < kWF; ++b) mbar_init(&empty[b], kWsCons / 32);
        *abort_ = 0;
    }
    __syncthreads();
    const int tiles = tiles_x * tiles_y;
    // Control flow stays warp-uniform: each lane waits (its own acquire), and
    // the warp goes on only if every lane's wait completed.
    auto wait_all = [&](unsigned long long* bar, unsigned parity) {
        const bool ok = __all_sync(kAll, mbar_wait_bounded(bar, parity));
        if (!ok && lane == 0) {
            atomicExch(abort_, 1);
            atomicOr(status, 2);
        }
        return ok;
    };
    auto stop = [&]() { return __any_sync(kAll, *(volatile int*)abort_ != 0); };
    auto failed = [&]() { return __any_sync(kAll, (*(volatile int*)status & 2) != 0); };

    if (tid < kWsCons) {
        asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;\n" ::"n"(kWsConsRegs));
        // ---- consumers: plane z0 + j of a unit reads the field slots of
        // producer indices Kb + j, + 1, + 2 (planes z - 1, z, z + 1)
        const int ly = tid >> 5, lx = lane;
        unsigned Kb = 0;
        for (int u = blockIdx.x; u < units; u += gridDim.x) {
            if (failed()) return;
            const int tile = u % tiles, seg = u / tiles;
            const int x0 = (tile % tiles_x) * kWX, y0 = (tile / tiles_x) * kWY;
            const int tw = min(kWX, g.nx - x0), th = min(kWY, g.ny - y0);
            const int z0 = g.zb + seg * seglen, n = min(z0 + seglen, g.ze) - z0;
            const bool live = lx < tw && ly < th;
            const int x = live ? x0 + lx : 0, y = live ? y0 + ly : 0;
            const int c0 = (ly + 1) * kWsHX + lx + 1;
            for (int j = 0; j < n; ++j) {
                if (stop()) return;
                const unsigned Kf = Kb + (unsigned)j + 2;
                S raw[kP];
                if (live) pull_raw3<P>(src, g, x, y, z0 + j, raw);
                if (!wait_all(&full[Kf % kWB], (Kf / kWB) & 1)) return;
                R d[kQ], gg[3 * kM];
                if (live) {
                    const R* sm = fring + (size_t)((Kb + j) % kWF) * 7 * kWsHP;
                    const R* s0 = fring + (size_t)((Kb + j + 1) % kWF) * 7 * kWsHP;
                    const R* sp = fring + (size_t)(Kf % kWF) * 7 * kWsHP;
#pragma unroll
                    for (int p = 0; p < kQ; ++p) d[p] = Fmt3<P>::dec(raw[p], p, c.i16);
#pragma unroll
                    for (int q = 0; q < 3 * kM; ++q) gg[q] = Fmt3<P>::dec(raw[kQ + q], kQ + q, c.i16);
                    closure_collide3<R, MODE>(d, gg, c, [&](int q, int nb) {
                        const int o = q * kWsHP;
                        return nb == 0 ? s0[o + c0 + 1]
                             : nb == 1 ? s0[o + c0 - 1]
                             : nb == 2 ? s0[o + c0 + kWsHX]
                             : nb == 3 ? s0[o + c0 - kWsHX]
                             : nb == 4 ? sp[o + c0]
                                       : sm[o + c0];
                    });
                }
                // slot Kb + j (plane z - 1) is read for the last time: hand it
                // back (after a warp barrier) before the stores
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[(Kb + j) % kWF]);
                if (live) {
                    const unsigned row = ((unsigned)z0 + (unsigned)j) * (unsigned)g.ny + (unsigned)y;
                    const unsigned o = row * (unsigned)g.nx + (unsigned)x;
#pragma unroll
                    for (int i = 0; i < kQ; ++i) dst[i * g.ps + o] = Fmt3<P>::enc(d[i], i, c.s16);
#pragma unroll
                    for (int q = 0; q < 3 * kM; ++q)
                        dst[(kQ + q) * g.ps + o] = Fmt3<P>::enc(gg[q], kQ + q, c.s16);
                }
            }
            // the unit's last two slots (its top plane and the one above)
            if (lane == 0) {
                mbar_arrive(&empty[(Kb + n) % kWF]);
                mbar_arrive(&empty[(Kb + n + 1) % kWF]);
            }
            Kb += (unsigned)n + 2;
        }
        return;
    }

    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;\n" ::"n"(kWsProdRegs));
    // ---- producers: plane index K (unit-local k = 0 .. n + 1, plane
    // z0 - 1 + k) into slot K mod kWF, once the consumers have handed back
    // slot K - kWF
    const int pt = tid - kWsCons;
    unsigned K = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        if (failed()) return;
        const int tile = u % tiles, seg = u / tiles;
        const int x0 = (tile % tiles_x) * kWX, y0 = (tile / tiles_x) * kWY;
        const int tw = min(kWX, g.nx - x0), th = min(kWY, g.ny - y0);
        const int z0 = g.zb + seg * seglen, n = min(z0 + seglen, g.ze) - z0;
        const int hw = tw + 2;
        const bool mine = pt < hw * (th + 2);
        const int hy = mine ? pt / hw : 0, hx = mine ? pt - hy * hw : 0;
        const int x = wrap3i(x0 - 1 + hx, g.nx), y = wrap3i(y0 - 1 + hy, g.ny);
        const int hi = hy * kWsHX + hx;
        for (int k = 0; k <= n + 1; ++k, ++K) {
            if (stop()) return;
            // the pulls go out before the wait for the slot, which only
            // guards the slot's writes
            S raw[kP];
            if (mine) pull_raw3<P>(src, g, x, y, wrap3i(z0 - 1 + k, g.nz), raw);
            if (K >= kWF && !wait_all(&empty[K % kWF], ((K / kWF) - 1) & 1)) return;
            if (mine) {
                R d[kQ], gg[3 * kM], m[7];
#pragma unroll
                for (int p = 0; p < kQ; ++p) d[p] = Fmt3<P>::dec(raw[p], p, c.i16);
#pragma unroll
                for (int q = 0; q < 3 * kM; ++q) gg[q] = Fmt3<P>::dec(raw[kQ + q], kQ + q, c.i16);
                fields3<R>(d, gg, m);
                R* slot = fring + (size_t)(K % kWF) * 7 * kWsHP;
#pragma unroll
                for (int q = 0; q < 7; ++q) slot[q * kWsHP + hi] = m[q];
            }
            __syncwarp();
            // (fault injection: announcements dropped, the consumers' waits expire)
            if (lane == 0 && !(debug & LBMHD_DEBUG_DROP_BARRIER_ARRIVAL)) mbar_arrive(&full[K % kWB]);
        }
    }
}

template <int P, int V, int MODE>
__global__ void __launch_bounds__(256) step3_kernel(const typename Fmt3<P>::S* __restrict__ src,
                                                    typename Fmt3<P>::S* __restrict__ dst,
                                                    Geom3 g, unsigned total, unsigned total_pad,
                                                    Coll3<typename Fmt3<P>::R> c,
                                                    const typename Fmt3<P>::R* __restrict__ mom) {
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total_pad; t += stride)
        step3_body<P, V, MODE>(src, dst, g, t, total, c, mom);
}

// The FP32 two-node step without a closure, held to 168 registers: left to
// itself ptxas takes 170, which the per-warp allocation rounds up to 176 per
// thread, leaving room for two CTAs of 128 threads per SM instead of three
// (measured 14.1K against 16.8K MLUPS at 256^3).
__global__ void __maxnreg__(168)
    step3f_kernel(const float* __restrict__ src, float* __restrict__ dst, Geom3 g, unsigned total,
                  unsigned total_pad, Coll3<float> c) {
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total_pad; t += stride)
        step3_body<P_FP32, 2, K3_LOCAL>(src, dst, g, t, total, c, nullptr);
}

// The FP16 two-node step without a closure, held to 128 registers (16 warps
// per SM instead of 12; 8 bytes of spill).
__global__ void __launch_bounds__(256, 2) step3h_kernel(const unsigned short* __restrict__ src,
                                                        unsigned short* __restrict__ dst, Geom3 g,
                                                        unsigned total, unsigned total_pad,
                                                        Coll3<float> c) {
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned t = blockIdx.x * blockDim.x + threadIdx.x; t < total_pad; t += stride)
        step3_body_h<K3_LOCAL>(src, dst, g, t, total, c, nullptr);
}

// Seven FP64 device fields: rho, ux, uy, uz, Bx, By, Bz.
struct Fields7 {
    double* f[7];
};

// Equilibrium initialisation from seven FP64 device fields.  f^eq = w [r -
// 3/2 r u^2 - 3/4 B^2 + 3 r c.u + 9/2 r (c.u)^2 + 9/4 B^2 |c|^2 - 9/2 (c.B)^2]
// with the node terms formed once (the kernel is bound by the FP64 rate);
// the deviation f^eq - w replaces r by r - 1, so the deviation formats take
// it without cancellation.  g_q^eq = (1/6) [B + 3 ((C_q.u) B - (C_q.B) u)]:
// the component along the axis is B_a / 6, the others carry +-3 E_ab with
// E_ab = u_a B_b - B_a u_b.
template <int P>
__global__ void init3_kernel(Fields7 in, long long n, typename Fmt3<P>::S* __restrict__ st,
                             long long ps, double s16) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double r = in.f[0][i], u[3] = {in.f[1][i], in.f[2][i], in.f[3][i]},
                     B[3] = {in.f[4][i], in.f[5][i], in.f[6][i]};
        const double bb = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
        const double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
        const double r3 = 3.0 * r, r45 = 4.5 * r, m225 = 2.25 * bb;
        const double common = -1.5 * r * uu - 0.75 * bb;
        const double a_abs = r + common, a_dev = (r - 1.0) + common;
#pragma unroll
        for (int p = 0; p < kQ; ++p) {
            const int cx = pcx(p), cy = pcy(p), cz = pcz(p);
            double cu = 0.0, cb = 0.0;
            if (cx) {
                cu += cx > 0 ? u[0] : -u[0];
                cb += cx > 0 ? B[0] : -B[0];
            }
            if (cy) {
                cu += cy > 0 ? u[1] : -u[1];
                cb += cy > 0 ? B[1] : -B[1];
            }
            if (cz) {
                cu += cz > 0 ? u[2] : -u[2];
                cb += cz > 0 ? B[2] : -B[2];
            }
            const int cc = cx * cx + cy * cy + cz * cz;
            double t = r3 * cu + r45 * cu * cu - 4.5 * cb * cb;
            if (cc) t += m225 * cc;
            const double w = wq<double>(p);
            st[p * ps + i] = Fmt3<P>::from_fd(w * (a_abs + t), w * (a_dev + t), p, s16);
        }
        const double E3[3] = {3.0 * (u[1] * B[2] - B[1] * u[2]), 3.0 * (u[0] * B[2] - B[0] * u[2]),
                              3.0 * (u[0] * B[1] - B[0] * u[1])};  // 3 E_yz, 3 E_xz, 3 E_xy
        const double sixth = 1.0 / 6.0;
#pragma unroll
        for (int q = 0; q < kM; ++q) {
            const int a = q / 2;
            const double sg = q % 2 ? -1.0 : 1.0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                double gv;
                if (b == a) {
                    gv = sixth * B[b];
                } else {
                    // E_ab = -E_ba; E3 is indexed by the axis not in {a, b}
                    const double e = (a < b ? 1.0 : -1.0) * E3[3 - a - b];
                    gv = sixth * (B[b] + sg * e);
                }
                st[(kQ + 3 * q + b) * ps + i] = Fmt3<P>::from_fd(gv, gv, kQ + 3 * q + b, s16);
            }
        }
    }
}

// rho, u (3), B (3) of the stored state into seven FP64 fields.
template <int P>
__global__ void moments3_kernel(const typename Fmt3<P>::S* __restrict__ st, long long ps,
                                long long n, Fields7 out, double i16) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int p = 0; p < kQ; ++p) {
            const double f = Fmt3<P>::to_f(st[p * ps + i], p, i16);
            rho += f;
            j[0] += pcx(p) * f;
            j[1] += pcy(p) * f;
            j[2] += pcz(p) * f;
        }
#pragma unroll
        for (int q = 0; q < kM; ++q)
#pragma unroll
            for (int b = 0; b < 3; ++b) B[b] += Fmt3<P>::to_f(st[(kQ + 3 * q + b) * ps + i], kQ + 3 * q + b, i16);
        out.f[0][i] = rho;
        for (int a = 0; a < 3; ++a) {
            out.f[1 + a][i] = j[a] / rho;
            out.f[4 + a][i] = B[a];
        }
    }
}

// Non-finite check: the rest population f_0 and the first magnetic plane
// of every node.  A non-finite value in any population of a node makes
// every post-collision population of the nodes that pull it non-finite,
// so a check after each step sees it at most one step after it appears.
template <int P>
__global__ void finite3_kernel(const typename Fmt3<P>::S* __restrict__ st, long long ps, long long n,
                               double i16, int* __restrict__ flag) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double a = Fmt3<P>::to_f(st[i], 0, i16), b = Fmt3<P>::to_f(st[kQ * ps + i], kQ, i16);
        if (!isfinite(a) || !isfinite(b)) atomicOr(flag, 1);
    }
}

// 45 FP64 planes of n encoded into the storage format.
template <int P>
__global__ void set3_kernel(const double* __restrict__ in, long long n,
                            typename Fmt3<P>::S* __restrict__ st, long long ps, double s16) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int p = 0; p < kP; ++p) st[p * ps + i] = Fmt3<P>::from_f(in[p * n + i], p, s16);
}

// The stored state decoded to 45 FP64 planes of n.
template <int P>
__global__ void get3_kernel(const typename Fmt3<P>::S* __restrict__ st, long long ps, long long n,
                            double* __restrict__ out, double i16) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
#pragma unroll
        for (int p = 0; p < kP; ++p) out[p * n + i] = Fmt3<P>::to_f(st[p * ps + i], p, i16);
}

// Diagnostics from the moment fields: per block, FP64 sums in a fixed order
// (thread sums over a grid-stride range, then a fixed tree), one row of 12
// per block; a single block then adds the rows in block order.
constexpr int kDiagBlock3 = 256, kDiagRows3 = 1024;
__global__ void __launch_bounds__(kDiagBlock3) diag3_kernel(const double* __restrict__ m7,
                                                            Geom3 g, double* __restrict__ rows) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    double s[12];
    for (int k = 0; k < 12; ++k) s[k] = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % g.nx), y = (int)((i / g.nx) % g.ny), z = (int)(i / ((long long)g.nx * g.ny));
        const double rho = m7[i];
        const double u[3] = {m7[n + i], m7[2 * n + i], m7[3 * n + i]};
        const double B[3] = {m7[4 * n + i], m7[5 * n + i], m7[6 * n + i]};
        s[0] += rho;
        for (int a = 0; a < 3; ++a) {
            s[1 + a] += rho * u[a];
            s[4 + a] += B[a];
        }
        s[7] += 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        s[8] += 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
        s[9] += u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
        const long long rowb = ((long long)z * g.ny + y) * g.nx;
        const long long xp = rowb + (x == g.nx - 1 ? 0 : x + 1), xm = rowb + (x == 0 ? g.nx - 1 : x - 1);
        const long long yp = ((long long)z * g.ny + (y == g.ny - 1 ? 0 : y + 1)) * g.nx + x;
        const long long ym = ((long long)z * g.ny + (y == 0 ? g.ny - 1 : y - 1)) * g.nx + x;
        const long long zp = ((long long)(z == g.nz - 1 ? 0 : z + 1) * g.ny + y) * g.nx + x;
        const long long zm = ((long long)(z == 0 ? g.nz - 1 : z - 1) * g.ny + y) * g.nx + x;
        const double div = 0.5 * (m7[4 * n + xp] - m7[4 * n + xm]) + 0.5 * (m7[5 * n + yp] - m7[5 * n + ym]) +
                           0.5 * (m7[6 * n + zp] - m7[6 * n + zm]);
        s[10] = fmax(s[10], fabs(div));
        s[11] += div * div;
    }
    __shared__ double red[12][kDiagBlock3];
    for (int k = 0; k < 12; ++k) red[k][threadIdx.x] = s[k];
    __syncthreads();
    for (int w = kDiagBlock3 / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 12; ++k)
                red[k][threadIdx.x] = k == 10 ? fmax(red[k][threadIdx.x], red[k][threadIdx.x + w])
                                              : red[k][threadIdx.x] + red[k][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 12) rows[blockIdx.x * 12 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void diag3_final_kernel(const double* __restrict__ rows, int nrows, long long n,
                                   double* __restrict__ out) {
    const int k = threadIdx.x;
    if (k >= 12) return;
    double a = 0.0;
    for (int r = 0; r < nrows; ++r) a = k == 10 ? fmax(a, rows[r * 12 + k]) : a + rows[r * 12 + k];
    if (k >= 7 && k <= 9) a /= (double)n;
    if (k == 11) a = sqrt(a / (double)n);
    out[k] = a;
}

unsigned grid3(long long n, int block) {
    long long b = (n + block - 1) / block;
    return (unsigned)(b < 1 ? 1 : (b > 65535LL * 64 ? 65535LL * 64 : b));
}

// One step: for les 2, 3 the moments pass into mom, then the step.
template <int P, int V>
cudaError_t launch3_pv(int block, const void* src, void* dst, const Geom3& g,
                       const Coll3<typename Fmt3<P>::R>& c, int les, void* mom, cudaStream_t st) {
    using S = typename Fmt3<P>::S;
    using R = typename Fmt3<P>::R;
    const unsigned total = (unsigned)((long long)g.nx / V * g.ny * (g.ze - g.zb));
    const unsigned total_pad = (total + 31u) / 32u * 32u;
    const unsigned blocks = (total_pad + block - 1) / block;
    if (les == 2 || les == 3) {
        // the fields of planes zb - 1 .. ze (all planes when that wraps round)
        Geom3 gm = g;
        if (g.ze - g.zb + 2 >= g.nz) {
            gm.zb = 0;
            gm.ze = g.nz;
        } else {
            gm.zb = g.zb - 1;
            gm.ze = g.ze + 1;
        }
        const unsigned mtotal = (unsigned)((long long)g.nx / V * g.ny * (gm.ze - gm.zb));
        const unsigned mpad = (mtotal + 31u) / 32u * 32u;
        mom3_kernel<P, V><<<(mpad + block - 1) / block, block, 0, st>>>((const S*)src, (R*)mom, gm, mtotal,
                                                                       mpad, c.i16);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        if (les == 2)
            step3_kernel<P, V, K3_FILTER><<<blocks, block, 0, st>>>((const S*)src, (S*)dst, g, total,
                                                                   total_pad, c, (const R*)mom);
        else
            step3_kernel<P, V, K3_CARATI><<<blocks, block, 0, st>>>((const S*)src, (S*)dst, g, total,
                                                                   total_pad, c, (const R*)mom);
        return cudaGetLastError();
    }
    if constexpr (P == P_FP16_DEV && V == 2)
        step3h_kernel<<<blocks, block, 0, st>>>((const S*)src, (S*)dst, g, total, total_pad, c);
    else if constexpr (P == P_FP32 && V == 2)
        step3f_kernel<<<blocks, block, 0, st>>>((const S*)src, (S*)dst, g, total, total_pad, c);
    else
        step3_kernel<P, V, K3_LOCAL><<<blocks, block, 0, st>>>((const S*)src, (S*)dst, g, total,
                                                               total_pad, c, nullptr);
    return cudaGetLastError();
}

// The fused form: tiles x segments work units, one CTA each.  The segment
// count makes the units fill whole waves of the resident CTAs where it can
// (each segment also pulls two planes of fields before its first plane).
template <int P, int MODE>
cudaError_t launch_fused3(const void* src, void* dst, const Geom3& g,
                          const Coll3<typename Fmt3<P>::R>& c, int resident, cudaStream_t st) {
    using S = typename Fmt3<P>::S;
    using R = typename Fmt3<P>::R;
    const int tiles_x = (g.nx + kFX - 1) / kFX, tiles_y = (g.ny + kFTY - 1) / kFTY;
    const long long tiles = (long long)tiles_x * tiles_y;
    const int nzr = g.ze - g.zb;  // planes this launch computes
    int best_seg = 1;
    double best = -1.0;
    for (int waves = 1; waves <= 8; ++waves) {
        long long nseg = (waves * (long long)resident + tiles / 2) / tiles;
        if (nseg < 1) nseg = 1;
        if (nseg > nzr) nseg = nzr;
        const int seglen = (int)((nzr + nseg - 1) / nseg);
        nseg = (nzr + seglen - 1) / seglen;
        const long long units = tiles * nseg;
        const long long slots = (units + resident - 1) / resident * resident;
        const double eff = (double)units / (double)slots * (double)seglen / (seglen + 1.0);
        if (eff > best + 1e-9) {
            best = eff;
            best_seg = seglen;
        }
    }
    const long long units = tiles * ((nzr + best_seg - 1) / best_seg);
    if (units > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)fused3_smem_floats() * sizeof(R);
    fused3_kernel<P, MODE><<<(unsigned)units, kFThreads, smem, st>>>((const S*)src, (S*)dst, g, tiles_x,
                                                                       tiles_y, best_seg, c);
    return cudaGetLastError();
}

// Opt the fused kernel of one precision and closure in to its shared memory
// (FP32 63 KB, FP64 126 KB); per_sm: its resident CTAs per SM.
template <int P, int MODE>
cudaError_t prepare_fused3_mode(int& per_sm) {
    using R = typename Fmt3<P>::R;
    const size_t smem = (size_t)fused3_smem_floats() * sizeof(R);
    cudaError_t e = cudaFuncSetAttribute(fused3_kernel<P, MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fused3_kernel<P, MODE>, kFThreads, smem);
    return e;
}

template <int P>
cudaError_t prepare_fused3(int les, int& per_sm) {
    return les == 2 ? prepare_fused3_mode<P, K3_FILTER>(per_sm) : prepare_fused3_mode<P, K3_CARATI>(per_sm);
}

template <int P>
cudaError_t launch_fused3_p(int les, const void* src, void* dst, const Geom3& g,
                            const Coll3<typename Fmt3<P>::R>& c, int resident, cudaStream_t st) {
    return les == 2 ? launch_fused3<P, K3_FILTER>(src, dst, g, c, resident, st)
                    : launch_fused3<P, K3_CARATI>(src, dst, g, c, resident, st);
}

// The warp-specialised form: a persistent grid of at most `resident` CTAs
// over tiles x segments work units.  The segment length balances the
// units over the CTAs against the two extra planes each segment pulls.
template <int P, int MODE>
cudaError_t launch_ws3(const void* src, void* dst, const Geom3& g, const Coll3<float>& c,
                       int resident, int* status, int debug, cudaStream_t st) {
    using S = typename Fmt3<P>::S;
    const int tiles_x = (g.nx + kWX - 1) / kWX, tiles_y = (g.ny + kWY - 1) / kWY;
    const long long tiles = (long long)tiles_x * tiles_y;
    const int nzr = g.ze - g.zb;
    int best_seg = nzr;
    double best = -1.0;
    for (int seglen = nzr; seglen >= 1; seglen = seglen > 8 ? seglen - (seglen + 7) / 8 : seglen - 1) {
        const long long units = tiles * ((nzr + seglen - 1) / seglen);
        const long long per_cta = (units + resident - 1) / resident;
        // planes computed over the busiest CTA's planes pulled
        const double eff = (double)tiles * nzr / ((double)per_cta * resident * (seglen + 1.0));
        if (eff > best + 1e-9) {
            best = eff;
            best_seg = seglen;
        }
        if (units > 64LL * resident) break;
    }
    const long long units = tiles * ((nzr + best_seg - 1) / best_seg);
    if (units > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    const int grid = (int)std::min<long long>(units, resident);
    ws3_kernel<P, MODE><<<grid, kWsThreads, kWsSmem, st>>>((const S*)src, (S*)dst, g, tiles_x, tiles_y,
                                                           best_seg, (int)units, c, status, debug);
    return cudaGetLastError();
}

// Resident CTAs per SM of the warp-specialised kernel (FP32 and FP16
// storage), 0 where it cannot run: its warpgroups' register split needs the
// launch to hold kWsLaunchRegs registers per thread, which the compiled
// kernel's register count must confirm.
template <int P, int MODE>
cudaError_t prepare_ws3_mode(int& per_sm) {
    per_sm = 0;
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, ws3_kernel<P, MODE>);
    if (e != cudaSuccess || a.numRegs < kWsLaunchRegs) return e;
    e = cudaFuncSetAttribute(ws3_kernel<P, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmem);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ws3_kernel<P, MODE>, kWsThreads, kWsSmem);
    return e;
}

template <int P>
cudaError_t prepare_ws3(int les, int& per_sm) {
    if constexpr (P == P_FP32 || P == P_FP16_DEV)
        return les == 2 ? prepare_ws3_mode<P, K3_FILTER>(per_sm) : prepare_ws3_mode<P, K3_CARATI>(per_sm);
    per_sm = 0;
    return cudaSuccess;
}

template <int P>
cudaError_t launch_ws3_p(int les, const void* src, void* dst, const Geom3& g,
                         const Coll3<typename Fmt3<P>::R>& c, int resident, int* status, int debug,
                         cudaStream_t st) {
    if constexpr (P == P_FP32 || P == P_FP16_DEV)
        return les == 2 ? launch_ws3<P, K3_FILTER>(src, dst, g, c, resident, status, debug, st)
                        : launch_ws3<P, K3_CARATI>(src, dst, g, c, resident, status, debug, st);
    return cudaErrorInvalidValue;
}

}  // namespace d3
}  // namespace lbmhd

using namespace lbmhd;
using namespace lbmhd::d3;

struct lbmhd3_t {
    Geom3 geom;
    lbmhd_params p;
    int device;
    cudaStream_t stream;
    bool own_stream;
    void* buf[2];
    int cur;
    bool initialised, failed;
    int vec, block;      // vec 0: the fused closure kernel (block unused)
    int fused_resident;  // resident fused CTAs on the device
    int ws_resident;     // resident warp-specialised CTAs on the device, 0 if unavailable
    int debug;           // fault-injection flags (lbmhd3_debug)
    int64_t steps, launches;
    void* mom;       // field planes of the gradient closures (les 2, 3)
    int* d_flag;     // bit 0: a non-finite value seen (check_finite_every)
    double* d_m7;    // moment fields for the diagnostics (allocated on first use)
    double* d_rows;  // diagnostics partial rows
    double* d_out;
};

namespace {

int fail3(int code, const std::string& m) {
    set_error(m);
    return code;
}

int cuda3(lbmhd3_t* h, cudaError_t e, const char* where) {
    if (h) h->failed = true;
    cudaGetLastError();
    set_error(std::string(where) + ": " + cudaGetErrorString(e));
    return LBMHD_ECUDA;
}

#define LBMHD3_CK(h, call)                                 \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda3(h, e_, #call); \
    } while (0)

int check3(lbmhd3_t* h) {
    if (!h) return fail3(LBMHD_EINVAL, "handle is NULL");
    if (h->failed) return fail3(LBMHD_ECUDA, "handle is unusable after a CUDA error");
    return LBMHD_OK;
}

// Calls f(std::integral_constant<int, P>{}) for the handle's storage format.
template <class F>
cudaError_t by_prec3(int prec, F f) {
    if (prec == LBMHD_FP64) return f(std::integral_constant<int, P_FP64>{});
    if (prec == LBMHD_FP32) return f(std::integral_constant<int, P_FP32>{});
    if (prec == LBMHD_FP16_DEV) return f(std::integral_constant<int, P_FP16_DEV>{});
    if (prec == LBMHD_FF) return f(std::integral_constant<int, P_FF>{});
    return cudaErrorInvalidValue;
}

// The pending non-finite report: ENONFINITE once the flag is set (until the
// next init or state write).  Synchronises.
int read_flag3(lbmhd3_t* h) {
    int flag = 0;
    LBMHD3_CK(h, cudaMemcpyAsync(&flag, h->d_flag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    LBMHD3_CK(h, cudaStreamSynchronize(h->stream));
    if (flag & 2) return fail3(LBMHD_ETIMEOUT, "a bounded wait of the closure kernel expired");
    if (flag & 1) return fail3(LBMHD_ENONFINITE, "non-finite value detected in the 3D state");
    return LBMHD_OK;
}

template <class R>
Coll3<R> coll3(const lbmhd_params& p) {
    Coll3<R> c;
    c.tn = (R)p.tau_nu;
    c.te = (R)p.tau_eta;
    c.tn2 = (R)(p.tau_nu * p.tau_nu);
    c.te2 = (R)(p.tau_eta * p.tau_eta);
    const double cd2 = p.C_S * p.delta * p.delta;
    c.k18 = (R)(18.0 * cd2);
    c.k36 = (R)(36.0 * cd2);
    c.d12 = (R)(p.delta * p.delta / 12.0);
    c.cd2 = (R)cd2;
    c.s16 = (float)p.fp16_scale;
    c.i16 = (float)(1.0 / p.fp16_scale);
    c.les = p.les == 1 ? 1 : 0;
    return c;
}

long long nodes3(const lbmhd3_t* h) { return (long long)h->geom.nx * h->geom.ny * h->geom.nz; }

// Planes [z0, z1) of the next state into the back buffer.
cudaError_t step3_planes(lbmhd3_t* h, int z0, int z1) {
    const void* src = h->buf[h->cur];
    void* dst = h->buf[1 - h->cur];
    const int les = h->p.les;
    Geom3 g = h->geom;
    g.zb = z0;
    g.ze = z1;
    const cudaError_t e = by_prec3(h->p.precision, [&](auto tag) {
        constexpr int P = decltype(tag)::value;
        using R = typename Fmt3<P>::R;
        const Coll3<R> c = coll3<R>(h->p);
        if (h->vec == 0) return launch_fused3_p<P>(les, src, dst, g, c, h->fused_resident, h->stream);
        if (h->vec == 3)
            return launch_ws3_p<P>(les, src, dst, g, c, h->ws_resident, h->d_flag, h->debug, h->stream);
        return h->vec == 2 ? launch3_pv<P, 2>(h->block, src, dst, g, c, les, h->mom, h->stream)
                           : launch3_pv<P, 1>(h->block, src, dst, g, c, les, h->mom, h->stream);
    });
    if (e == cudaSuccess) h->launches += les >= 2 && (h->vec == 1 || h->vec == 2) ? 2 : 1;
    return e;
}

cudaError_t one_step3(lbmhd3_t* h) {
    const cudaError_t e = step3_planes(h, 0, h->geom.nz);
    if (e == cudaSuccess) h->cur = 1 - h->cur;
    return e;
}

// Halo messages: the planes of a list, one z-plane each (nx ny stored
// values), gathered from a state into buf or scattered from buf, as raw
// values of the storage width: grid row k copies plane pl.p[k], in 16-byte
// words when a z-plane is a whole number of them (T = uint4), else in
// values.
struct PlaneList3 {
    int n;
    int p[kP];
};
template <class T>
__global__ void __launch_bounds__(256) move3_kernel(bool pack, T* __restrict__ st, long long ps_w,
                                                    long long off_w, int nw, PlaneList3 pl,
                                                    T* __restrict__ buf) {
    const int k = blockIdx.y;
    T* s = st + pl.p[k] * ps_w + off_w;
    T* b = buf + (long long)k * nw;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) {
        if (pack)
            b[i] = s[i];
        else
            s[i] = b[i];
    }
}

template <class T>
cudaError_t move3_planes(bool pack, void* st, long long ps, long long off, long long nxy,
                         const PlaneList3& pl, void* buf, cudaStream_t stream) {
    if (pl.n == 0 || nxy == 0) return cudaSuccess;
    const bool wide = (nxy * (long long)sizeof(T)) % 16 == 0 && (ps * (long long)sizeof(T)) % 16 == 0 &&
                      (uintptr_t)st % 16 == 0 && (uintptr_t)buf % 16 == 0;
    if (wide) {
        const long long r = 16 / (long long)sizeof(T);  // values per word
        const int nw = (int)(nxy / r);
        const dim3 grid((unsigned)std::min<long long>((nw + 255) / 256, 1024), (unsigned)pl.n);
        move3_kernel<uint4><<<grid, 256, 0, stream>>>(pack, (uint4*)st, ps / r, off / r, nw, pl, (uint4*)buf);
    } else {
        const dim3 grid((unsigned)std::min<long long>((nxy + 255) / 256, 1024), (unsigned)pl.n);
        move3_kernel<T><<<grid, 256, 0, stream>>>(pack, (T*)st, ps, off, (int)nxy, pl, (T*)buf);
    }
    return cudaGetLastError();
}

Fields7 contiguous7(double* base, long long n) {
    Fields7 f;
    for (int q = 0; q < 7; ++q) f.f[q] = base + q * n;
    return f;
}

// rho, u, B of the current state into seven FP64 device fields.
cudaError_t moments3_fields(lbmhd3_t* h, const Fields7& out) {
    const long long n = (long long)h->geom.nx * h->geom.ny * h->geom.nz;
    return by_prec3(h->p.precision, [&](auto tag) {
        constexpr int P = decltype(tag)::value;
        using S = typename Fmt3<P>::S;
        moments3_kernel<P><<<grid3(n, 256), 256, 0, h->stream>>>((const S*)h->buf[h->cur], h->geom.ps, n,
                                                                  out, 1.0 / h->p.fp16_scale);
        return cudaGetLastError();
    });
}

cudaError_t moments3_into(lbmhd3_t* h, double* m7) {
    return moments3_fields(h, contiguous7(m7, (long long)h->geom.nx * h->geom.ny * h->geom.nz));
}

// Equilibrium initialisation of the current buffer from device fields.
cudaError_t init3_fields(lbmhd3_t* h, const Fields7& in) {
    const long long n = (long long)h->geom.nx * h->geom.ny * h->geom.nz;
    return by_prec3(h->p.precision, [&](auto tag) {
        constexpr int P = decltype(tag)::value;
        init3_kernel<P><<<grid3(n, 256), 256, 0, h->stream>>>(in, n, (typename Fmt3<P>::S*)h->buf[h->cur],
                                                               h->geom.ps, h->p.fp16_scale);
        return cudaGetLastError();
    });
}

size_t value3_bytes(int prec) {
    return prec == LBMHD_FP64 || prec == LBMHD_FF ? 8
                                                  : (prec == LBMHD_FP32 ? 4 : (prec == LBMHD_FP16_DEV ? 2 : 0));
}

}  // namespace

extern "C" {

int lbmhd3_bytes_per_cell(int precision) { return (int)(2 * kP * value3_bytes(precision)); }

int lbmhd3_create(int nx, int ny, int nz, const lbmhd_params* p, lbmhd3_t** out) {
    if (!out || !p) return fail3(LBMHD_EINVAL, "NULL argument");
    *out = nullptr;
    if (p->abi_version != LBMHD_ABI_VERSION) return fail3(LBMHD_EVERSION, "ABI version mismatch");
    if (nx < 1 || ny < 1 || nz < 1 || (long long)nx * ny * nz > (1LL << 30))
        return fail3(LBMHD_EINVAL, "nx, ny, nz must be >= 1 with nx*ny*nz <= 2^30 nodes");
    if (value3_bytes(p->precision) == 0)
        return fail3(LBMHD_EINVAL, "3D lattices: FP64, FP32, FP16 deviation or double-word storage");
    if (p->precision == LBMHD_FP16_DEV && !(p->fp16_scale > 0.0 && p->fp16_scale < 1e30))
        return fail3(LBMHD_EINVAL, "fp16_scale must be positive and finite");
    if (p->les < 0 || p->les > 3)
        return fail3(LBMHD_EINVAL,
                     "les must be 0 (off), 1 (local rates), 2 (filtered equilibria) or 3 "
                     "(cross-helicity closure)");
    if (!(p->tau_nu > 0.5) || !(p->tau_eta > 0.5) || !(p->tau_nu < 1e6) || !(p->tau_eta < 1e6))
        return fail3(LBMHD_EINVAL, "tau_nu and tau_eta must be finite and > 1/2");
    if (!(p->C_S >= 0.0) || !(p->C_S < 1e6) || !(p->delta > 0.0) || !(p->delta < 1e6))
        return fail3(LBMHD_EINVAL, "C_S must be >= 0 and delta > 0, both finite");
    if (p->check_finite_every < 0) return fail3(LBMHD_EINVAL, "check_finite_every must be >= 0");
    lbmhd3_t* h = new (std::nothrow) lbmhd3_t();
    if (!h) return fail3(LBMHD_ENOMEM, "host allocation failed");
    std::memset((void*)h, 0, sizeof(*h));
    h->p = *p;
    h->geom.nx = nx;
    h->geom.ny = ny;
    h->geom.nz = nz;
    const long long n = (long long)nx * ny * nz;
    h->geom.ps = (n + 63) / 64 * 64;
    h->geom.zb = 0;
    h->geom.ze = nz;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) {
        delete h;
        return cuda3(nullptr, e, "cudaGetDevice");
    }
    if (p->stream) {
        h->stream = (cudaStream_t)p->stream;
    } else {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete h;
            return cuda3(nullptr, e, "cudaStreamCreateWithFlags");
        }
        h->own_stream = true;
    }
    const size_t bytes = (size_t)kP * h->geom.ps * value3_bytes(p->precision);
    // field planes in the arithmetic type: FP64, or FP32 for the FP32 and FP16 formats
    const size_t mbytes =
        p->les >= 2 ? (size_t)7 * h->geom.ps * (p->precision == LBMHD_FP64 || p->precision == LBMHD_FF ? 8 : 4) : 0;
    void** bufs[4] = {&h->buf[0], &h->buf[1], &h->mom, (void**)&h->d_flag};
    const size_t sizes[4] = {bytes, bytes, mbytes, sizeof(int)};
    for (int b = 0; b < 4; ++b) {
        if (!sizes[b]) continue;
        e = cudaMalloc(bufs[b], sizes[b]);
        if (e != cudaSuccess) {
            for (int k = 0; k < b; ++k) cudaFree(*bufs[k]);
            if (h->own_stream) cudaStreamDestroy(h->stream);
            delete h;
            cudaGetLastError();
            return fail3(e == cudaErrorMemoryAllocation ? LBMHD_ENOMEM : LBMHD_ECUDA,
                         std::string("device allocation failed: ") + cudaGetErrorString(e));
        }
    }
    // two nodes per thread where nx allows (8- or 16-byte loads), 128
    // threads.  Gradient closures: FP32 and FP16 storage take the
    // warp-specialised kernel (else the fused kernel), FP64 and FF (bound by
    // their arithmetic, where the one-pass kernels measured slower) the
    // two-pass kernels one node per thread (two nodes need more than 255
    // registers in FP64).
    h->vec = nx % 2 == 0 && p->les < 2 && p->precision != LBMHD_FF ? 2 : 1;
    h->block = 128;
    if (p->les >= 2 && p->precision != LBMHD_FP64 && p->precision != LBMHD_FF) {  // the fused kernel
        h->vec = 0;
        h->block = kFTY;
    }
    if (p->les >= 2) {
        int per_sm = 0, nsm = 0;
        e = by_prec3(p->precision, [&](auto tag) {
            return prepare_fused3<decltype(tag)::value>(p->les, per_sm);
        });
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
        if (e != cudaSuccess) {
            lbmhd3_destroy(h);
            return cuda3(nullptr, e, "fused closure kernel setup");
        }
        h->fused_resident = per_sm * nsm > 0 ? per_sm * nsm : 1;
        h->ws_resident = 0;
        if (p->precision == LBMHD_FP32 || p->precision == LBMHD_FP16_DEV) {
            int ws_sm = 0;
            e = by_prec3(p->precision, [&](auto tag) {
                return prepare_ws3<decltype(tag)::value>(p->les, ws_sm);
            });
            if (e != cudaSuccess) {
                lbmhd3_destroy(h);
                return cuda3(nullptr, e, "warp-specialised closure kernel setup");
            }
            h->ws_resident = ws_sm * nsm;
            if (h->ws_resident > 0) {
                h->vec = 3;
                h->block = kWY;
            }
        }
    }
    *out = h;
    return LBMHD_OK;
}

int lbmhd3_set_launch(lbmhd3_t* h, int vec, int block) {
    int rc = check3(h);
    if (rc) return rc;
    if (vec == 0) {
        if (h->p.les < 2) return fail3(LBMHD_EINVAL, "vec 0 (the fused kernel) is for les 2, 3");
        h->vec = 0;
        h->block = kFTY;
        return LBMHD_OK;
    }
    if (vec == 3) {
        if (h->p.les < 2 || (h->p.precision != LBMHD_FP32 && h->p.precision != LBMHD_FP16_DEV))
            return fail3(LBMHD_EINVAL, "vec 3 (the warp-specialised kernel) is for les 2, 3 in FP32 or FP16 storage");
        if (block != kWY) return fail3(LBMHD_EINVAL, "vec 3 takes block 8 (tile rows)");
        if (h->ws_resident < 1)
            return fail3(LBMHD_EINVAL, "the warp-specialised kernel cannot run on this device");
        h->vec = 3;
        h->block = block;
        return LBMHD_OK;
    }
    if ((vec != 1 && vec != 2) || h->geom.nx % vec)
        return fail3(LBMHD_EINVAL, "vec must be 0 (les 2, 3), 1 or 2 and divide nx");
    if (block < 32 || block > 256 || block % 32)
        return fail3(LBMHD_EINVAL, "block must be a multiple of 32 in [32, 256]");
    h->vec = vec;
    h->block = block;
    return LBMHD_OK;
}

int lbmhd3_get_launch(const lbmhd3_t* h, int* vec, int* block) {
    if (!h || !vec || !block) return fail3(LBMHD_EINVAL, "NULL argument");
    *vec = h->vec;
    *block = h->block;
    return LBMHD_OK;
}

int lbmhd3_init(lbmhd3_t* h, const double* rho, const double* ux, const double* uy,
                const double* uz, const double* bx, const double* by, const double* bz) {
    TraceRange trace_("lbmhd3_init");
    int rc = check3(h);
    if (rc) return rc;
    const double* f[7] = {rho, ux, uy, uz, bx, by, bz};
    for (int i = 0; i < 7; ++i)
        if (!f[i]) return fail3(LBMHD_EINVAL, "NULL field");
    const long long n = nodes3(h);
    for (long long i = 0; i < n; ++i)
        if (!(rho[i] > 0.0) || !(rho[i] < 1e300))
            return fail3(LBMHD_EINVAL, "rho must be positive and finite");
    double* tmp = nullptr;
    LBMHD3_CK(h, cudaMallocAsync((void**)&tmp, 7 * n * sizeof(double), h->stream));
    for (int i = 0; i < 7; ++i)
        LBMHD3_CK(h, cudaMemcpyAsync(tmp + i * n, f[i], n * sizeof(double), cudaMemcpyHostToDevice,
                                     h->stream));
    LBMHD3_CK(h, init3_fields(h, contiguous7(tmp, n)));
    LBMHD3_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    LBMHD3_CK(h, cudaFreeAsync(tmp, h->stream));
    LBMHD3_CK(h, cudaStreamSynchronize(h->stream));
    h->initialised = true;
    h->steps = 0;
    return LBMHD_OK;
}

int lbmhd3_init_device(lbmhd3_t* h, const double* rho, const double* ux, const double* uy,
                       const double* uz, const double* bx, const double* by, const double* bz) {
    int rc = check3(h);
    if (rc) return rc;
    const double* f[7] = {rho, ux, uy, uz, bx, by, bz};
    Fields7 in;
    for (int i = 0; i < 7; ++i) {
        if (!f[i]) return fail3(LBMHD_EINVAL, "NULL field");
        in.f[i] = const_cast<double*>(f[i]);
    }
    LBMHD3_CK(h, init3_fields(h, in));
    LBMHD3_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    h->initialised = true;
    h->steps = 0;
    return LBMHD_OK;
}

int lbmhd3_moments_device(lbmhd3_t* h, double* rho, double* ux, double* uy, double* uz,
                          double* bx, double* by, double* bz) {
    int rc = check3(h);
    if (rc) return rc;
    if (!h->initialised) return fail3(LBMHD_ESTATE, "moments before lbmhd3_init");
    double* f[7] = {rho, ux, uy, uz, bx, by, bz};
    Fields7 out;
    for (int i = 0; i < 7; ++i) {
        if (!f[i]) return fail3(LBMHD_EINVAL, "NULL field");
        out.f[i] = f[i];
    }
    LBMHD3_CK(h, moments3_fields(h, out));
    return LBMHD_OK;
}

int lbmhd3_set_state(lbmhd3_t* h, const double* state) {
    int rc = check3(h);
    if (rc) return rc;
    if (!state) return fail3(LBMHD_EINVAL, "NULL state");
    const long long n = nodes3(h);
    double* tmp = nullptr;
    LBMHD3_CK(h, cudaMallocAsync((void**)&tmp, (size_t)kP * n * sizeof(double), h->stream));
    LBMHD3_CK(h, cudaMemcpyAsync(tmp, state, (size_t)kP * n * sizeof(double), cudaMemcpyHostToDevice,
                                 h->stream));
    LBMHD3_CK(h, by_prec3(h->p.precision, [&](auto tag) {
                  constexpr int P = decltype(tag)::value;
                  set3_kernel<P><<<grid3(n, 256), 256, 0, h->stream>>>(
                      tmp, n, (typename Fmt3<P>::S*)h->buf[h->cur], h->geom.ps, h->p.fp16_scale);
                  return cudaGetLastError();
              }));
    LBMHD3_CK(h, cudaFreeAsync(tmp, h->stream));
    LBMHD3_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    LBMHD3_CK(h, cudaStreamSynchronize(h->stream));
    h->initialised = true;
    return LBMHD_OK;
}

static int raw3(lbmhd3_t* h, bool get, void* state, size_t bytes) {
    int rc = check3(h);
    if (rc) return rc;
    if (!state) return fail3(LBMHD_EINVAL, "NULL state");
    const size_t vb = value3_bytes(h->p.precision);
    const size_t row = (size_t)nodes3(h) * vb;
    if (bytes != (size_t)kP * row) return fail3(LBMHD_EINVAL, "byte count is not 45 * nodes * value size");
    if (get && !h->initialised) return fail3(LBMHD_ESTATE, "get_state_raw before lbmhd3_init");
    const size_t pitch = (size_t)h->geom.ps * vb;
    if (get)
        LBMHD3_CK(h, cudaMemcpy2DAsync(state, row, h->buf[h->cur], pitch, row, kP, cudaMemcpyDeviceToHost,
                                       h->stream));
    else {
        LBMHD3_CK(h, cudaMemcpy2DAsync(h->buf[h->cur], pitch, state, row, row, kP, cudaMemcpyHostToDevice,
                                       h->stream));
        LBMHD3_CK(h, cudaMemsetAsync(h->d_flag, 0, sizeof(int), h->stream));
    }
    LBMHD3_CK(h, cudaStreamSynchronize(h->stream));
    if (!get) h->initialised = true;
    return LBMHD_OK;
}

int lbmhd3_get_state_raw(lbmhd3_t* h, void* state, size_t bytes) { return raw3(h, true, state, bytes); }

int lbmhd3_set_state_raw(lbmhd3_t* h, const void* state, size_t bytes) {
    return raw3(h, false, const_cast<void*>(state), bytes);
}

int lbmhd3_step(lbmhd3_t* h, int n) {
    TraceRange trace_("lbmhd3_step");
    int rc = check3(h);
    if (rc) return rc;
    if (n < 0) return fail3(LBMHD_EINVAL, "n must be >= 0");
    if (!h->initialised) return fail3(LBMHD_ESTATE, "lbmhd3_step before lbmhd3_init");
    const int every = h->p.check_finite_every;
    const long long nn = nodes3(h);
    for (int s = 0; s < n; ++s) {
        LBMHD3_CK(h, one_step3(h));
        ++h->steps;
        if (every > 0 && h->steps % every == 0)
            LBMHD3_CK(h, by_prec3(h->p.precision, [&](auto tag) {
                          constexpr int P = decltype(tag)::value;
                          finite3_kernel<P><<<grid3(nn, 256), 256, 0, h->stream>>>(
                              (const typename Fmt3<P>::S*)h->buf[h->cur], h->geom.ps, nn,
                              1.0 / h->p.fp16_scale, h->d_flag);
                          return cudaGetLastError();
                      }));
    }
    return LBMHD_OK;
}

int lbmhd3_step_planes(lbmhd3_t* h, int z0, int z1) {
    TraceRange trace_("lbmhd3_step_planes");
    int rc = check3(h);
    if (rc) return rc;
    if (!(0 <= z0 && z0 < z1 && z1 <= h->geom.nz))
        return fail3(LBMHD_EINVAL, "planes: need 0 <= z0 < z1 <= nz");
    if (!h->initialised) return fail3(LBMHD_ESTATE, "lbmhd3_step_planes before lbmhd3_init");
    LBMHD3_CK(h, step3_planes(h, z0, z1));
    return LBMHD_OK;
}

int lbmhd3_step_commit(lbmhd3_t* h) {
    int rc = check3(h);
    if (rc) return rc;
    if (!h->initialised) return fail3(LBMHD_ESTATE, "lbmhd3_step_commit before lbmhd3_init");
    h->cur = 1 - h->cur;
    ++h->steps;
    return LBMHD_OK;
}

static int plane_move3(lbmhd3_t* h, bool pack, int z, uint64_t mask, void* buf, void* stream) {
    int rc = check3(h);
    if (rc) return rc;
    if (!buf) return fail3(LBMHD_EINVAL, "NULL buffer");
    if (z < 0 || z >= h->geom.nz) return fail3(LBMHD_EINVAL, "plane outside the lattice");
    if (mask >> kP) return fail3(LBMHD_EINVAL, "plane mask bits above 44");
    const size_t vb = value3_bytes(h->p.precision);
    if ((uintptr_t)buf % vb) return fail3(LBMHD_EINVAL, "buffer not aligned to the stored value size");
    if (pack && !h->initialised) return fail3(LBMHD_ESTATE, "pack before lbmhd3_init");
    PlaneList3 pl;
    pl.n = 0;
    for (int p = 0; p < kP; ++p)
        if (mask >> p & 1) pl.p[pl.n++] = p;
    const long long nxy = (long long)h->geom.nx * h->geom.ny;
    cudaStream_t st = stream ? (cudaStream_t)stream : h->stream;
    void* state = h->buf[h->cur];
    cudaError_t e;
    if (vb == 8)
        e = move3_planes<unsigned long long>(pack, state, h->geom.ps, z * nxy, nxy, pl, buf, st);
    else if (vb == 4)
        e = move3_planes<unsigned>(pack, state, h->geom.ps, z * nxy, nxy, pl, buf, st);
    else
        e = move3_planes<unsigned short>(pack, state, h->geom.ps, z * nxy, nxy, pl, buf, st);
    LBMHD3_CK(h, e);
    return LBMHD_OK;
}

int lbmhd3_pack_plane(lbmhd3_t* h, int z, uint64_t mask, void* buf, void* stream) {
    return plane_move3(h, true, z, mask, buf, stream);
}

int lbmhd3_unpack_plane(lbmhd3_t* h, int z, uint64_t mask, const void* buf, void* stream) {
    return plane_move3(h, false, z, mask, const_cast<void*>(buf), stream);
}

int lbmhd3_moments(lbmhd3_t* h, double* out7) {
    TraceRange trace_("lbmhd3_moments");
    int rc = check3(h);
    if (rc) return rc;
    if (!out7) return fail3(LBMHD_EINVAL, "NULL output");
    if (!h->initialised) return fail3(LBMHD_ESTATE, "moments before lbmhd3_init");
    const long long n = nodes3(h);
    double* tmp = nullptr;
    LBMHD3_CK(h, cudaMallocAsync((void**)&tmp, 7 * n * sizeof(double), h->stream));
    LBMHD3_CK(h, moments3_into(h, tmp));
    LBMHD3_CK(h, cudaMemcpyAsync(out7, tmp, 7 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LBMHD3_CK(h, cudaFreeAsync(tmp, h->stream));
    LBMHD3_CK(h, cudaStreamSynchronize(h->stream));
    return read_flag3(h);  // a pending non-finite report
}

int lbmhd3_get_state(lbmhd3_t* h, double* out) {
    int rc = check3(h);
    if (rc) return rc;
    if (!out) return fail3(LBMHD_EINVAL, "NULL output");
    if (!h->initialised) return fail3(LBMHD_ESTATE, "get_state before lbmhd3_init");
    const long long n = nodes3(h);
    double* tmp = nullptr;
    LBMHD3_CK(h, cudaMallocAsync((void**)&tmp, (size_t)kP * n * sizeof(double), h->stream));
    LBMHD3_CK(h, by_prec3(h->p.precision, [&](auto tag) {
                  constexpr int P = decltype(tag)::value;
                  get3_kernel<P><<<grid3(n, 256), 256, 0, h->stream>>>(
                      (const typename Fmt3<P>::S*)h->buf[h->cur], h->geom.ps, n, tmp, 1.0 / h->p.fp16_scale);
                  return cudaGetLastError();
              }));
    LBMHD3_CK(h, cudaMemcpyAsync(out, tmp, (size_t)kP * n * sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
    LBMHD3_CK(h, cudaFreeAsync(tmp, h->stream));
    LBMHD3_CK(h, cudaStreamSynchronize(h->stream));
    return read_flag3(h);  // a pending non-finite report
}

int lbmhd3_diagnostics(lbmhd3_t* h, double* out12) {
    TraceRange trace_("lbmhd3_diagnostics");
    int rc = check3(h);
    if (rc) return rc;
    if (!out12) return fail3(LBMHD_EINVAL, "NULL output");
    if (!h->initialised) return fail3(LBMHD_ESTATE, "diagnostics before lbmhd3_init");
    const long long n = nodes3(h);
    if (!h->d_m7) {
        LBMHD3_CK(h, cudaMalloc((void**)&h->d_m7, 7 * n * sizeof(double)));
        LBMHD3_CK(h, cudaMalloc((void**)&h->d_rows, kDiagRows3 * 12 * sizeof(double)));
        LBMHD3_CK(h, cudaMalloc((void**)&h->d_out, 12 * sizeof(double)));
    }
    LBMHD3_CK(h, moments3_into(h, h->d_m7));
    long long nb = (n + kDiagBlock3 - 1) / kDiagBlock3;
    if (nb > kDiagRows3) nb = kDiagRows3;
    diag3_kernel<<<(unsigned)nb, kDiagBlock3, 0, h->stream>>>(h->d_m7, h->geom, h->d_rows);
    LBMHD3_CK(h, cudaGetLastError());
    diag3_final_kernel<<<1, 32, 0, h->stream>>>(h->d_rows, (int)nb, n, h->d_out);
    LBMHD3_CK(h, cudaGetLastError());
    LBMHD3_CK(h, cudaMemcpyAsync(out12, h->d_out, 12 * sizeof(double), cudaMemcpyDeviceToHost,
                                 h->stream));
    LBMHD3_CK(h, cudaStreamSynchronize(h->stream));
    return read_flag3(h);  // a pending non-finite report
}

int lbmhd3_sync(lbmhd3_t* h) {
    int rc = check3(h);
    if (rc) return rc;
    LBMHD3_CK(h, cudaStreamSynchronize(h->stream));
    return h->initialised ? read_flag3(h) : LBMHD_OK;
}

int lbmhd3_debug(lbmhd3_t* h, int flags) {
    if (!h) return fail3(LBMHD_EINVAL, "handle is NULL");
    h->debug = flags;
    return LBMHD_OK;
}

int64_t lbmhd3_step_count(const lbmhd3_t* h) { return h ? h->steps : 0; }

int64_t lbmhd3_launch_count(const lbmhd3_t* h) { return h ? h->launches : 0; }

void lbmhd3_destroy(lbmhd3_t* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
    cudaFree(h->mom);
    cudaFree(h->d_flag);
    cudaFree(h->d_m7);
    cudaFree(h->d_rows);
    cudaFree(h->d_out);
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
}

}  // extern "C"
