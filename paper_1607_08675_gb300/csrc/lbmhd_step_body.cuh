// lbmhd_step_body.cuh -- the per-thread work of one fused stream-collide
// step over V consecutive nodes of a row, shared by the single-lattice
// kernel (lbmhd_step.cu) and the batched ensemble kernel (lbmhd_batch.cu)
// so that both compute bit-identical results.
//
// Layout: 19 SoA planes, x fastest.  Thread t of a lattice covers nodes
// (y, x0 .. x0 + V - 1) with y = t / (nx / V), x0 = (t mod (nx / V)) V; the
// 32 lanes of a warp hold consecutive t.  Each plane is read with one
// aligned vector load; an x-shifted plane gets its missing edge element
// from the neighbouring lane by a warp shuffle, and only a lane at a warp
// edge or at the periodic wrap loads it from memory.  The collision runs in
// registers.
#pragma once

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
template <>
__device__ __forceinline__ float2 shfl_up1(float2 v) {
    return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
template <class S>
__device__ __forceinline__ S shfl_down1(S v) {
    return __shfl_down_sync(0xffffffffu, v, 1);
}
template <>
__device__ __forceinline__ unsigned short shfl_down1(unsigned short v) {
    return (unsigned short)__shfl_down_sync(0xffffffffu, (unsigned)v, 1);
}
template <>
__device__ __forceinline__ float2 shfl_down1(float2 v) {
    return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1),
                       __shfl_down_sync(0xffffffffu, v.y, 1));
}

// FP16 storage with V = 2W nodes per thread: each plane row segment is W
// 32-bit words, two binary16 values per word (lower address in the low
// half).  The x-shift of a plane is a funnel of half-words (byte_perm), the
// two nodes of a word are decoded with one paired conversion and encoded
// with one (cvt.rn.f16x2.f32), and the collision runs on the scaled values.
template <int V>
__device__ __forceinline__ void step_body_h(const unsigned short* __restrict__ src,
                                            unsigned short* __restrict__ dst, int nx, int ny,
                                            long long ps, unsigned t, unsigned total,
                                            const Coll<float>& c, int y0) {
    constexpr int W = V / 2;
    using Word = unsigned int;
    const int lane = threadIdx.x & 31;
    const unsigned nxv = (unsigned)(nx / V);
    const bool live = t < total;
    const unsigned tc = live ? t : total - 1;
    const unsigned ty = tc / nxv;  // row within the launch
    const int y = y0 + (int)ty;
    const int x0 = (int)(tc - ty * nxv) * V;
    const int ym = y == 0 ? ny - 1 : y - 1;
    const int yp = y == ny - 1 ? 0 : y + 1;
    const bool has_left = lane > 0 && x0 > 0;
    const bool has_right = lane < 31 && x0 + V < nx;
    const int xl = x0 == 0 ? nx - 1 : x0 - 1;
    const int xr = x0 + V == nx ? 0 : x0 + V;

    Word raw[kPlanes][W];
#pragma unroll
    for (int p = 0; p < kPlanes; ++p) {
        const int cx = plane_cx(p), cy = plane_cy(p);
        const int row = cy == 0 ? y : (cy > 0 ? ym : yp);
        const unsigned short* base = src + p * ps + (long long)row * nx;
        const Pack<Word, W> pk = *reinterpret_cast<const Pack<Word, W>*>(base + x0);
        if (cx == 0) {
#pragma unroll
            for (int j = 0; j < W; ++j) raw[p][j] = pk.v[j];
        } else if (cx > 0) {  // node x0 - 1 in the high half of the left word
            Word prev = __shfl_up_sync(0xffffffffu, pk.v[W - 1], 1);
            if (!has_left) prev = (Word)base[xl] << 16;
            raw[p][0] = __byte_perm(prev, pk.v[0], 0x5432);
#pragma unroll
            for (int j = 1; j < W; ++j) raw[p][j] = __byte_perm(pk.v[j - 1], pk.v[j], 0x5432);
        } else {  // node x0 + V in the low half of the right word
            Word next = __shfl_down_sync(0xffffffffu, pk.v[0], 1);
            if (!has_right) next = (Word)base[xr];
#pragma unroll
            for (int j = 0; j < W - 1; ++j) raw[p][j] = __byte_perm(pk.v[j], pk.v[j + 1], 0x5432);
            raw[p][W - 1] = __byte_perm(pk.v[W - 1], next, 0x5432);
        }
    }

#pragma unroll
    for (int j = 0; j < W; ++j) {
        float d0[9], g0[10], d1[9], g1[10];
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const float2 f2 = __half22float2(*reinterpret_cast<const __half2*>(&raw[p][j]));
            if (p < 9) {
                d0[p] = f2.x;
                d1[p] = f2.y;
            } else {
                g0[p - 9] = f2.x;
                g1[p - 9] = f2.y;
            }
        }
        collide<float, true>(d0, g0, c);
        collide<float, true>(d1, g1, c);
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const __half2 h = p < 9 ? __floats2half2_rn(d0[p], d1[p])
                                    : __floats2half2_rn(g0[p - 9], g1[p - 9]);
            raw[p][j] = *reinterpret_cast<const Word*>(&h);
        }
    }

    if (live) {
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            Pack<Word, W> o;
#pragma unroll
            for (int j = 0; j < W; ++j) o.v[j] = raw[p][j];
            *reinterpret_cast<Pack<Word, W>*>(dst + p * ps + (long long)y * nx + x0) = o;
        }
    }
}

// One thread's step.  All 32 lanes of the warp must call it together
// (shuffles); t >= total marks a padding thread, which loads valid
// addresses (those of thread total - 1) and stores nothing.  Thread t of a
// launch over the rows y0 .. y0 + total / (nx / V) - 1 covers row
// y0 + t / (nx / V).
template <int P, int V>
__device__ __forceinline__ void step_body(const typename Fmt<P>::S* __restrict__ src,
                                          typename Fmt<P>::S* __restrict__ dst, int nx, int ny,
                                          long long ps, unsigned t, unsigned total,
                                          const Coll<typename Fmt<P>::R>& c, float scale,
                                          float inv_scale, int y0 = 0) {
    if constexpr (P == P_FP16_DEV && V % 2 == 0) {
        step_body_h<V>(src, dst, nx, ny, ps, t, total, c, y0);
        return;
    }
    using S = typename Fmt<P>::S;
    using R = typename Fmt<P>::R;
    const int lane = threadIdx.x & 31;
    const unsigned nxv = (unsigned)(nx / V);
    const bool live = t < total;
    const unsigned tc = live ? t : total - 1;
    const unsigned ty = tc / nxv;  // row within the launch
    const int y = y0 + (int)ty;
    const int x0 = (int)(tc - ty * nxv) * V;
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
        collide<R, Fmt<P>::kScaled>(d, g, c);
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

template <class R>
__host__ __device__ inline Coll<R> make_coll_t(double tn, double te, double k18, double k36,
                                               double s5, double s6, double s7, double s8,
                                               int les, int tie5 = 0, int tie6 = 0) {
    Coll<R> c;
    c.tn = (R)tn;
    c.te = (R)te;
    c.tn2 = (R)(tn * tn);
    c.te2 = (R)(te * te);
    c.k18 = (R)k18;
    c.k36 = (R)k36;
    c.s5 = (R)s5;
    c.s6 = (R)s6;
    c.s7 = (R)s7;
    c.s8 = (R)s8;
    c.les = les;
    c.tie5 = tie5;
    c.tie6 = tie6;
    c.inv_s = R(1);
    c.scl = R(1);
    c.d2 = R(0);
    c.cd2 = (R)(k18 / 18.0);
    return c;
}

// Collision parameters of a storage format: FP16 deviations keep their
// storage scale through the collision, so the LES constants are divided by
// it (see collide<R, true>).
template <class R>
inline Coll<R> coll_for_prec(const HostColl& h, int prec) {
    Coll<R> c = make_coll_t<R>(h.tn, h.te, h.k18, h.k36, h.s5, h.s6, h.s7, h.s8, h.les, h.tie5,
                               h.tie6);
    c.d2 = (R)h.d2;
    if (prec == P_FP16_DEV) {
        c.k18 = (R)(h.k18 / (double)h.scale);
        c.k36 = (R)(h.k36 / (double)h.scale);
        c.inv_s = (R)h.inv_scale;
        c.scl = (R)h.scale;
    }
    return c;
}

}  // namespace lbmhd
