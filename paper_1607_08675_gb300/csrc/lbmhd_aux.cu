// lbmhd_aux.cu -- equilibrium initialisation, moments, state transfer,
// the non-finite check and the FP64 diagnostics reduction.
#include "lbmhd_cp_async.cuh"
#include "lbmhd_device.cuh"
#include "lbmhd_diag_plan.h"
#include "lbmhd_internal.h"

#include <mutex>
#include <type_traits>

namespace lbmhd {

// ---- FP64 views of a stored value ---------------------------------------
// abs: the population itself; dev: its deviation from the rest state.
template <int P>
__device__ __forceinline__ double dev_of(typename Fmt<P>::S v, int p, float inv_scale) {
    if constexpr (P == P_FP64) return v - plane_rest<double>(p);
    else if constexpr (P == P_FP32) return (double)v - (double)plane_rest<float>(p);
    else if constexpr (P == P_FP32_DEV) return (double)v;
    else if constexpr (P == P_FF) return (double)v.x + (double)v.y;
    else return (double)__half2float(__ushort_as_half(v)) * (double)inv_scale;
}
// Rest value that dev_of subtracted (FP32 storage subtracts the FP32 weight).
template <int P>
__device__ __forceinline__ double rest_of(int p) {
    if constexpr (P == P_FP32) return (double)plane_rest<float>(p);
    else return plane_rest<double>(p);
}
template <int P>
__device__ __forceinline__ typename Fmt<P>::S enc_d(double absval, double devval, float scale) {
    if constexpr (P == P_FP64) return absval;
    else if constexpr (P == P_FP32) return (float)absval;
    else if constexpr (P == P_FP32_DEV) return (float)devval;
    else if constexpr (P == P_FF) {
        const float hi = (float)devval;
        return make_float2(hi, (float)(devval - (double)hi));
    } else return __half_as_ushort(__float2half_rn((float)(devval * (double)scale)));
}

// ---- equilibrium initialisation (Sec. 3 equilibria) ----------------------
template <int P>
__global__ void init_kernel(const double* __restrict__ rho, const double* __restrict__ ux,
                            const double* __restrict__ uy, const double* __restrict__ bx,
                            const double* __restrict__ by, typename Fmt<P>::S* __restrict__ st,
                            long long n, int nx, long long ps, float scale, int* bad) {
    (void)nx;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const double r = rho[c], u = ux[c], v = uy[c], Bx = bx[c], By = by[c];
        if (bad && !(r > 0.0 && isfinite(r))) atomicOr(bad, 8);
        const double u2 = u * u + v * v, b2 = Bx * Bx + By * By;
        // f^eq = w [r (1 - 3/2 u^2) + 3 r c.u + 9/2 r (c.u)^2 + 9/4 B^2 c^2
        //           - 9/2 (c.B)^2]; the deviation f^eq - w replaces r (1 - ...)
        // by (r - 1) - 3/2 r u^2.  The node terms are formed once (the init is
        // bound by GB300's FP64 rate).
        const double r3 = 3.0 * r, r45 = 4.5 * r, m225 = 2.25 * b2, ru2 = 1.5 * r * u2;
        const double a_abs = r - ru2, a_dev = (r - 1.0) - ru2;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int cx = plane_cx(i), cy = plane_cy(i);
            const double cu = cx * u + cy * v, cb = cx * Bx + cy * By;
            const int c2 = cx * cx + cy * cy;
            const double w = plane_rest<double>(i);
            double t = r3 * cu + r45 * cu * cu - 4.5 * cb * cb;
            if (c2) t += m225 * c2;
            st[i * ps + c] = enc_d<P>(w * (a_abs + t), w * (a_dev + t), scale);
        }
        // g_k^eq = w'_k [B + 3 ((C_k.u) B - (C_k.B) u)]: B/3 at rest; on an axis
        // the component along it is w' B exactly, the other one carries
        // +-3 E with E = u_x B_y - u_y B_x
        const double E3 = 3.0 * (u * By - v * Bx);
        const double third = 1.0 / 3.0, sixth = 1.0 / 6.0;
        const double gv[10] = {third * Bx,        third * By,          // k = 0
                               sixth * Bx,        sixth * (By + E3),   // +x
                               sixth * (Bx - E3), sixth * By,          // +y
                               sixth * Bx,        sixth * (By - E3),   // -x
                               sixth * (Bx + E3), sixth * By};         // -y
#pragma unroll
        for (int q = 0; q < 10; ++q) st[(9 + q) * ps + c] = enc_d<P>(gv[q], gv[q], scale);
    }
}

// ---- moments of a stored state ------------------------------------------
template <int P>
__device__ __forceinline__ void node_moments(const typename Fmt<P>::S* __restrict__ st,
                                             long long ps, long long o, float inv_scale,
                                             double& r, double& u, double& v, double& Bx,
                                             double& By) {
    double d[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = dev_of<P>(st[i * ps + o], i, inv_scale);
    double drho = 0.0;
#pragma unroll
    for (int i = 0; i < 9; ++i) drho += d[i];
    const double jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    const double jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    r = 1.0 + drho;  // the rest weights sum to one
    u = jx / r;
    v = jy / r;
    Bx = 0.0;
    By = 0.0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        Bx += dev_of<P>(st[(9 + 2 * k) * ps + o], 9 + 2 * k, inv_scale);
        By += dev_of<P>(st[(10 + 2 * k) * ps + o], 10 + 2 * k, inv_scale);
    }
}

template <int P>
__global__ void moments_kernel(const typename Fmt<P>::S* __restrict__ st, double* rho, double* ux,
                               double* uy, double* bx, double* by, long long n, long long ps,
                               float inv_scale) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        double r, u, v, Bx, By;
        node_moments<P>(st, ps, c, inv_scale, r, u, v, Bx, By);
        rho[c] = r;
        ux[c] = u;
        uy[c] = v;
        bx[c] = Bx;
        by[c] = By;
    }
}

template <int P>
__global__ void get_state_kernel(const typename Fmt<P>::S* __restrict__ st, double* out,
                                 long long n, long long ps, float inv_scale) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const auto v = st[p * ps + c];
            double a;
            if constexpr (P == P_FP64) a = v;
            else if constexpr (P == P_FP32) a = (double)v;
            else a = rest_of<P>(p) + dev_of<P>(v, p, inv_scale);
            out[p * n + c] = a;
        }
    }
}

template <int P>
__global__ void set_state_kernel(const double* __restrict__ in, typename Fmt<P>::S* st,
                                 long long n, long long ps, float scale) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int p = 0; p < kPlanes; ++p) {
            const double a = in[p * n + c];
            st[p * ps + c] = enc_d<P>(a, a - plane_rest<double>(p), scale);
        }
    }
}

template <int P>
__global__ void finite_kernel(const typename Fmt<P>::S* __restrict__ st, int* flag, long long n,
                              long long ps, float inv_scale) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
         c += (long long)gridDim.x * blockDim.x) {
        const double a = dev_of<P>(st[c], 0, inv_scale);
        const double b = dev_of<P>(st[9 * ps + c], 9, inv_scale);
        if (!isfinite(a) || !isfinite(b)) atomicOr(flag, 1);
    }
}

// ---- diagnostics ----------------------------------------------------------
// Warps sweep column strips down the lattice (the work split below), so the
// central differences of omega, j_z and div B take x-neighbours from lane
// shuffles and y-neighbours from the rows kept in registers.  The per-node
// arithmetic runs in the format's arithmetic type R,
// as in the step kernels: FP32 for the FP32 and FP16 storage forms, FP64
// for FP64 storage, double-word for FF.  Each thread sums its nodes in an
// accumulator type A -- FP64 for FP64 storage, double-word (48-bit
// significand, on the FP32 pipes) otherwise -- so that no per-node FP64
// instruction is issued for the FP32 forms (GB300's FP64 pipe is a small
// fraction of its FP32 pipes; with FP64 per-node arithmetic this pass was
// FP64-bound at ~10x its memory time).  The per-term FP32 rounding is
// unbiased, ~1e-7 of a term, and averages down to ~1e-7 / sqrt(N) of a sum.
// The thread sums then go to FP64: fixed warp-shuffle tree -> fixed
// cross-warp order -> one partial row per block; a single-block pass
// combines the rows in block order.  Same lattice, same result, bit for bit.
constexpr int kNQ = 12;  // kOwn, kDiagWarps, kDiagBlocks: lbmhd_diag_plan.h

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Per-thread accumulator: a += t and its FP64 value.
template <class R> struct DiagAcc { using A = ff; };
template <> struct DiagAcc<double> { using A = double; };
__device__ __forceinline__ void acc_add(double& a, double t) { a += t; }
__device__ __forceinline__ void acc_add(ff& a, ff t) { a += t; }
__device__ __forceinline__ void acc_add(ff& a, float t) { dw_accumulate(a, t); }
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ double acc_value(ff a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ double to_f64(float v) { return v; }
__device__ __forceinline__ double to_f64(double v) { return v; }
__device__ __forceinline__ double to_f64(ff v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ bool gt(float a, float b) { return a > b; }
__device__ __forceinline__ bool gt(double a, double b) { return a > b; }
__device__ __forceinline__ bool gt(ff a, ff b) { return a > b; }

// Moments of one stored node in the arithmetic type (the sums of the step
// kernels' collision, deviation form): m = (rho - 1, j_x, j_y, u_x, u_y,
// B_x, B_y).  rho - 1 and j are sums of the stored values themselves, so
// the mass and momentum sums carry no rounding of 1 + (rho - 1).
enum { kDrho = 0, kJx, kJy, kUx, kUy, kBx, kBy, kNM };
template <int P>
__device__ __forceinline__ void node_moments_raw(const typename Fmt<P>::S (&raw)[kPlanes],
                                                 float inv_scale,
                                                 typename Fmt<P>::R (&m)[kNM]) {
    using R = typename Fmt<P>::R;
    R d[9], g[10];
#pragma unroll
    for (int i = 0; i < 9; ++i) d[i] = Fmt<P>::dec(raw[i], i, inv_scale);
#pragma unroll
    for (int q = 0; q < 10; ++q) g[q] = Fmt<P>::dec(raw[9 + q], 9 + q, inv_scale);
    R dsum9 = ((d[0] + d[1]) + (d[2] + d[3])) + ((d[4] + d[5]) + (d[6] + d[7])) + d[8];
    R jx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
    R jy = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
    R Bx = (g[0] + g[2]) + (g[4] + g[6]) + g[8];
    R By = (g[1] + g[3]) + (g[5] + g[7]) + g[9];
    if (Fmt<P>::kScaled) {  // FP16 storage carries the storage scale
        const R is = (R)inv_scale;
        dsum9 *= is;
        jx *= is;
        jy *= is;
        Bx *= is;
        By *= is;
    }
    const R ir = rcp(R(1) + dsum9);
    m[kDrho] = dsum9;
    m[kJx] = jx;
    m[kJy] = jy;
    m[kUx] = jx * ir;
    m[kUy] = jy * ir;
    m[kBx] = Bx;
    m[kBy] = By;
}

// Lane shuffles of one value of the arithmetic type.
__device__ __forceinline__ float shfl_up_r(float v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ float shfl_dn_r(float v) { return __shfl_down_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_up_r(double v) { return __shfl_up_sync(0xffffffffu, v, 1); }
__device__ __forceinline__ double shfl_dn_r(double v) {
    return __shfl_down_sync(0xffffffffu, v, 1);
}
__device__ __forceinline__ ff shfl_up_r(ff v) { return ff(shfl_up_r(v.hi), shfl_up_r(v.lo)); }
__device__ __forceinline__ ff shfl_dn_r(ff v) { return ff(shfl_dn_r(v.hi), shfl_dn_r(v.lo)); }

// Work split: a warp sweeps a strip of kOwn columns down a segment of rows.
// Lane l holds column x0 - 1 + l (periodic): lanes 1..sw own the strip's
// columns, lanes 0 and sw + 1 the halo columns whose moments the owners'
// x-differences need; the moments of rows y - 1, y, y + 1 stay in
// registers as the warp moves down, so every node's moments are formed once
// (plus the halo columns and two rows per segment) from the 19 values
// stored at it.  No barrier: a warp's stored values pass through its own
// ring of rows (below).

// Rows of stored values in flight per warp.  4- and 8-byte values are
// staged by asynchronous copies (cp.async) into a per-warp ring of
// kDiagRing<P> rows in shared memory: the coming rows are in flight while a
// row is reduced, with no register set to hold them (a prefetch of the
// next row into registers took the kernel to 107 registers, two blocks per
// SM).  Three rows for 4-byte values (depths 2 to 6 measured within 2% of
// each other), two for 8-byte ones (the same bytes).  In the per-lane form
// lane l copies and later reads back only its own column, so its own
// wait_group is the only synchronisation the ring needs; the wide form (in
// the kernel) copies 16-byte granules and adds warp barriers.  Two-byte
// FP16 values are read straight into registers.
template <int P>
constexpr int kDiagRing = sizeof(typename Fmt<P>::S) == 2   ? 0
                          : sizeof(typename Fmt<P>::S) == 4 ? 3
                                                            : 2;
// Elements of one staged plane row: 32 (one per lane), or in the wide form
// (4-byte values) the 36 of a 16-byte aligned window over the warp's 32
// columns.
template <int P, bool WIDE>
constexpr int kDiagRowE = WIDE ? 36 : 32;
template <int P, bool WIDE>
constexpr size_t diag_smem_bytes() {
    return (size_t)kDiagWarps * kDiagRing<P> * kPlanes * kDiagRowE<P, WIDE> *
           sizeof(typename Fmt<P>::S);
}

// Blocks per SM the register budget is sized for.  FP16: three (80
// registers; 0.78 ms at 8192^2, against 0.99 ms at 96 registers and 1.45
// ms at the 64 ptxas picks with no minimum given).  FP32 forms: three as
// well (80 registers; 117 at one block, no faster).  FP64 and FF: one (FF
// loses 16% at three).
template <int P>
constexpr int kDiagMinBlocks = (P == P_FP64 || P == P_FF) ? 1 : 3;

template <int P, bool WIDE>
__global__ void __launch_bounds__(32 * kDiagWarps, kDiagMinBlocks<P>)
    diag_kernel(const typename Fmt<P>::S* __restrict__ st, int nx, int ny, long long ps,
                float inv_scale, int nstrips, int seglen, long long nunits, double* partials) {
    using R = typename Fmt<P>::R;
    using A = typename DiagAcc<R>::A;
    using S = typename Fmt<P>::S;
    constexpr int K = kDiagRing<P>;
    static_assert(K == 0 || K >= 2, "the ring holds rows y - 1 and y while y + 1 lands");
    static_assert(!WIDE || (K > 0 && sizeof(S) == 4), "wide rows: 4-byte values in the ring");
    extern __shared__ __align__(16) unsigned char diag_ring_smem[];
    __shared__ double red[kDiagWarps][kNQ];
    const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
    constexpr int RE = kDiagRowE<P, WIDE>;
    S* ring0 = reinterpret_cast<S*>(diag_ring_smem) + (size_t)warp * K * kPlanes * RE;
    S* ring = ring0 + lane;
    A acc[kNQ];
#pragma unroll
    for (int q = 0; q < kNQ; ++q) acc[q] = A(0);
    R dmax = R(0);
    const R half = R(0.5);
    const long long nwarps = (long long)gridDim.x * kDiagWarps;
    for (long long unit = (long long)blockIdx.x * kDiagWarps + warp; unit < nunits;
         unit += nwarps) {
        const int x0 = (int)(unit % nstrips) * kOwn;
        const int y0 = (int)(unit / nstrips) * seglen;
        const int y1 = min(y0 + seglen, ny);
        const int sw = min(kOwn, nx - x0);
        const bool own = lane >= 1 && lane <= sw;
        int col = x0 - 1 + (lane <= sw + 1 ? lane : 1);  // idle lanes shadow an owner
        col = col < 0 ? col + nx : (col >= nx ? col - nx : col);
        // Rows are fetched in order y0 - 1, y0, y0 + 1, ...; yf is the
        // stored row of the next one (periodic; y0 - 1 wraps more than once
        // when ny <= 2).
        int yf = (y0 - 1) % ny;
        if (yf < 0) yf += ny;
        auto fetch_ptr = [&]() {
            const S* src = st + ((long long)yf * nx + col);
            yf = yf + 1 == ny ? 0 : yf + 1;
            return src;
        };
        // The terms of row y from the moments of rows y - 1 (a), y (b) and
        // y + 1 (c), into partial sums g of a group of rows (assigned for
        // the group's first row); x-neighbours from lanes -1 and +1.
        auto row_terms = [&](const R (&a)[kNM], const R (&b)[kNM], const R (&c)[kNM],
                             R (&g)[kNQ], bool first) {
            const R vL = shfl_up_r(b[kUy]), vR = shfl_dn_r(b[kUy]);
            const R bxL = shfl_up_r(b[kBx]), bxR = shfl_dn_r(b[kBx]);
            const R byL = shfl_up_r(b[kBy]), byR = shfl_dn_r(b[kBy]);
            if (own) {
                const R u = b[kUx], v = b[kUy], Bx = b[kBx], By = b[kBy];
                const R om = half * (vR - vL) - half * (c[kUx] - a[kUx]);
                const R dv = half * (bxR - bxL) + half * (c[kBy] - a[kBy]);
                const R jz = half * (byR - byL) - half * (c[kBx] - a[kBx]);
                const R adv = fabs(dv);
                if (gt(adv, dmax)) dmax = adv;
                const R t[kNQ] = {b[kDrho],  // the node count is added at the end
                                  b[kJx],
                                  b[kJy],
                                  Bx,
                                  By,
                                  b[kJx] * u + b[kJy] * v,  // rho |u|^2
                                  Bx * Bx + By * By,
                                  om * om,
                                  u * Bx + v * By,
                                  R(0),  // slot 9 is the div B maximum
                                  dv * dv,
                                  jz * jz};
#pragma unroll
                for (int q = 0; q < kNQ; ++q)
                    if (q != 9) g[q] = first ? t[q] : g[q] + t[q];
            }
        };
        // FP32 arithmetic with the ring sweeps rows in groups of three: the
        // moments of three rows rotate through m0, m1, m2 with no copies,
        // and each group's terms (at most two FP32 roundings per term,
        // unbiased) are folded into the double-word accumulators once --
        // about a third of the instructions per row go to those folds.
        // FP64 and double-word arithmetic gain nothing from the grouping,
        // and the FP16 form, which loads straight into registers, loses the
        // overlap of one row's loads with the previous row's arithmetic: they
        // fold every row.
        constexpr int G = (std::is_same<R, float>::value && K > 0) ? 3 : 1;
        R m0[kNM], m1[kNM], m2[kNM];
        auto fold = [&](const R (&g)[kNQ]) {
            if (own) {
#pragma unroll
                for (int q = 0; q < kNQ; ++q)
                    if (q != 9) acc_add(acc[q], g[q]);
            }
        };
        auto sweep = [&](auto&& next) {
            next(m0);  // row y0 - 1
            next(m1);  // row y0
            if constexpr (G == 3) {
                for (int y = y0; y < y1; y += 3) {
                    R g[kNQ];
                    next(m2);  // row y + 1
                    row_terms(m0, m1, m2, g, true);
                    if (y + 1 < y1) {
                        next(m0);  // row y + 2
                        row_terms(m1, m2, m0, g, false);
                    }
                    if (y + 2 < y1) {
                        next(m1);  // row y + 3
                        row_terms(m2, m0, m1, g, false);
                    }
                    fold(g);
                }
            } else {
                for (int y = y0; y < y1; ++y) {
                    R g[kNQ];
                    next(m2);  // row y + 1
                    row_terms(m0, m1, m2, g, true);
                    fold(g);
#pragma unroll
                    for (int q = 0; q < kNM; ++q) {
                        m0[q] = m1[q];
                        m1[q] = m2[q];
                    }
                }
            }
        };
        if constexpr (K > 0) {
            // rows y0 - 1 .. y1 pass through the ring; row t (counted from
            // y0 - 1) sits in slot t % K.  One commit group per row, empty
            // past the last row, keeps "row t done" = "at most K - 1 groups
            // pending".
            const int nrows = y1 - y0 + 2;
            int tn = 0;  // the next row to take
            // Wide form (4-byte values, rows and planes 16-byte aligned, nx a
            // multiple of 4): plane i's columns [wx, wx + 36), wx = (x0 - 1)
            // rounded down to a multiple of 4, arrive as 9 copies of 16
            // bytes, each granule from its column modulo nx (the periodic
            // wrap at the row ends; nx is a multiple of 4, so a granule
            // never straddles it).  Lane l < 27 copies granule l % 9 of
            // planes l / 9, l / 9 + 3, ... (7 instructions per row instead
            // of 19), so lanes read one another's copies: a warp barrier
            // after the wait, and another before a slot is refilled.
            if constexpr (WIDE) {
                const int wx = (x0 - 1) & ~3;  // floor to a multiple of 4 (x0 - 1 >= -1)
                const int off = (x0 - 1) - wx + (lane <= sw + 1 ? lane : 1);
                const int grp = lane / 9, part = lane - 9 * (lane / 9);
                int gcol = (wx + 4 * part) % nx;  // this lane's granule, wrapped
                if (gcol < 0) gcol += nx;
                const long long ps3 = 3 * ps;
                auto issue_w = [&](int t) {
                    if (t < nrows) {
                        const S* src = fetch_ptr() - col + gcol + grp * ps;
                        S* dst = ring0 + (t % K) * (kPlanes * RE) + grp * RE + 4 * part;
                        if (lane < 27) {
#pragma unroll
                            for (int j = 0; j < 7; ++j) {
                                if (grp + 3 * j < kPlanes) cp_async_16(dst + 3 * j * RE, src);
                                src += ps3;
                            }
                        }
                    }
                    cp_async_commit();
                };
                auto take_w = [&](R (&m)[kNM]) {
                    cp_async_wait<K - 1>();
                    __syncwarp();
                    S raw[kPlanes];
                    const S* p = ring0 + (tn % K) * (kPlanes * RE) + off;
#pragma unroll
                    for (int i = 0; i < kPlanes; ++i) raw[i] = p[i * RE];
                    node_moments_raw<P>(raw, inv_scale, m);
                    __syncwarp();
                    issue_w(tn + K);
                    ++tn;
                };
#pragma unroll
                for (int t = 0; t < K; ++t) issue_w(t);
                sweep(take_w);
            } else {
                auto issue = [&](int t) {
                    if (t < nrows) {
                        const S* src = fetch_ptr();
                        S* dst = ring + (t % K) * (kPlanes * RE);
#pragma unroll
                        for (int i = 0; i < kPlanes; ++i)
                            cp_async_small<sizeof(S)>(dst + i * RE, src + i * ps);
                    }
                    cp_async_commit();
                };
                auto take = [&](R (&m)[kNM]) {
                    cp_async_wait<K - 1>();
                    S raw[kPlanes];
                    const S* p = ring + (tn % K) * (kPlanes * RE);
#pragma unroll
                    for (int i = 0; i < kPlanes; ++i) raw[i] = p[i * RE];
                    node_moments_raw<P>(raw, inv_scale, m);
                    issue(tn + K);  // the slot is free once its values are in registers
                    ++tn;
                };
#pragma unroll
                for (int t = 0; t < K; ++t) issue(t);
                sweep(take);
            }
            cp_async_wait<0>();
        } else {
            auto load = [&](R (&m)[kNM]) {
                const S* src = fetch_ptr();
                S raw[kPlanes];
#pragma unroll
                for (int i = 0; i < kPlanes; ++i) raw[i] = src[i * ps];
                node_moments_raw<P>(raw, inv_scale, m);
            };
            sweep(load);
        }
    }
#pragma unroll
    for (int q = 0; q < kNQ; ++q) {
        const double t = q == 9 ? to_f64(dmax) : acc_value(acc[q]);
        const double w = q == 9 ? warp_max(t) : warp_sum(t);
        if (lane == 0) red[warp][q] = w;
    }
    __syncthreads();
    if (threadIdx.x < kNQ) {
        const int q = threadIdx.x;
        double s = red[0][q];
        for (int w = 1; w < kDiagWarps; ++w) s = q == 9 ? fmax(s, red[w][q]) : s + red[w][q];
        partials[(long long)blockIdx.x * kNQ + q] = s;
    }
}

__global__ void diag_final_kernel(const double* __restrict__ partials, int nblocks, double ncell,
                                  double* out) {
    __shared__ double red[256 / 32][kNQ];
    double acc[kNQ];
#pragma unroll
    for (int q = 0; q < kNQ; ++q) acc[q] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < kNQ; ++q)
            acc[q] = q == 9 ? fmax(acc[q], partials[b * kNQ + q]) : acc[q] + partials[b * kNQ + q];
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll
    for (int q = 0; q < kNQ; ++q) {
        const double w = q == 9 ? warp_max(acc[q]) : warp_sum(acc[q]);
        if (lane == 0) red[warp][q] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s[kNQ];
        for (int q = 0; q < kNQ; ++q) {
            s[q] = red[0][q];
            for (int w = 1; w < 256 / 32; ++w) s[q] = q == 9 ? fmax(s[q], red[w][q]) : s[q] + red[w][q];
        }
        const double inv = 1.0 / ncell;
        out[0] = ncell + s[0];  // the threads summed rho - 1
        out[1] = s[1];
        out[2] = s[2];
        out[3] = s[3];
        out[4] = s[4];
        out[5] = 0.5 * s[5] * inv;
        out[6] = 0.5 * s[6] * inv;
        out[7] = 0.5 * s[7] * inv;
        out[8] = s[8] * inv;
        out[9] = s[9];
        out[10] = sqrt(s[10] * inv);
        out[11] = 0.5 * s[11] * inv;
    }
}

// ---- launchers ------------------------------------------------------------
static unsigned grid_for(long long n, int block) {
    long long b = (n + block - 1) / block;
    if (b > 65535LL * 8) b = 65535LL * 8;
    return (unsigned)(b < 1 ? 1 : b);
}

#define LBMHD_DISPATCH(prec, CALL)            \
    switch (prec) {                           \
        case P_FP64: { constexpr int P = P_FP64; CALL; } break;         \
        case P_FP32: { constexpr int P = P_FP32; CALL; } break;         \
        case P_FP32_DEV: { constexpr int P = P_FP32_DEV; CALL; } break; \
        case P_FP16_DEV: { constexpr int P = P_FP16_DEV; CALL; } break; \
        case P_FF: { constexpr int P = P_FF; CALL; } break;             \
        default: return cudaErrorInvalidValue;                          \
    }

cudaError_t launch_init(int prec, const double* rho, const double* ux, const double* uy,
                        const double* bx, const double* by, void* state, const Geom& g,
                        const HostColl& c, cudaStream_t st, int* bad) {
    const long long n = (long long)g.nx * g.ny;
    LBMHD_DISPATCH(prec, (init_kernel<P><<<grid_for(n, 256), 256, 0, st>>>(
                             rho, ux, uy, bx, by, (typename Fmt<P>::S*)state, n, g.nx, g.ps,
                             c.scale, bad)));
    return cudaGetLastError();
}

cudaError_t launch_moments(int prec, const void* state, double* rho, double* ux, double* uy,
                           double* bx, double* by, const Geom& g, const HostColl& c,
                           cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    LBMHD_DISPATCH(prec, (moments_kernel<P><<<grid_for(n, 256), 256, 0, st>>>(
                             (const typename Fmt<P>::S*)state, rho, ux, uy, bx, by, n, g.ps,
                             c.inv_scale)));
    return cudaGetLastError();
}

cudaError_t launch_get_state(int prec, const void* state, double* out, const Geom& g,
                             const HostColl& c, cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    LBMHD_DISPATCH(prec, (get_state_kernel<P><<<grid_for(n, 256), 256, 0, st>>>(
                             (const typename Fmt<P>::S*)state, out, n, g.ps, c.inv_scale)));
    return cudaGetLastError();
}

cudaError_t launch_set_state(int prec, const double* in, void* state, const Geom& g,
                             const HostColl& c, cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    LBMHD_DISPATCH(prec, (set_state_kernel<P><<<grid_for(n, 256), 256, 0, st>>>(
                             in, (typename Fmt<P>::S*)state, n, g.ps, c.scale)));
    return cudaGetLastError();
}

// Halo messages of a decomposed lattice: the selected planes of one row,
// gathered into (PACK) or scattered from a contiguous buffer, element j of
// plane slot q at buf[q * nx + j].  W: a stored value's size as an unsigned
// type of the same width (values are moved, not interpreted).
struct PlaneList {
    int p[kPlanes];
};
template <class W, bool PACK>
__global__ void row_planes_kernel(W* __restrict__ state, long long ps, int nx, int row,
                                  PlaneList pl, int nplanes, W* __restrict__ buf) {
    const long long n = (long long)nplanes * nx;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int q = (int)(i / nx);
        const long long e = pl.p[q] * ps + (long long)row * nx + (i - (long long)q * nx);
        if (PACK) buf[i] = state[e];
        else state[e] = buf[i];
    }
}

template <class W>
static cudaError_t row_planes_w(bool pack, void* state, const Geom& g, int row,
                                const PlaneList& pl, int nplanes, void* buf, cudaStream_t st) {
    const long long n = (long long)nplanes * g.nx;
    if (pack)
        row_planes_kernel<W, true><<<grid_for(n, 256), 256, 0, st>>>((W*)state, g.ps, g.nx, row,
                                                                     pl, nplanes, (W*)buf);
    else
        row_planes_kernel<W, false><<<grid_for(n, 256), 256, 0, st>>>((W*)state, g.ps, g.nx, row,
                                                                      pl, nplanes, (W*)buf);
    return cudaGetLastError();
}

cudaError_t launch_row_planes(int prec, bool pack, void* state, const Geom& g, int row,
                              const int* planes, int nplanes, void* buf, cudaStream_t st) {
    if (nplanes <= 0) return cudaSuccess;
    PlaneList pl;
    for (int q = 0; q < kPlanes; ++q) pl.p[q] = q < nplanes ? planes[q] : 0;
    switch (storage_bytes(prec)) {
        case 2: return row_planes_w<unsigned short>(pack, state, g, row, pl, nplanes, buf, st);
        case 4: return row_planes_w<unsigned int>(pack, state, g, row, pl, nplanes, buf, st);
        case 8: return row_planes_w<unsigned long long>(pack, state, g, row, pl, nplanes, buf, st);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_check_finite(int prec, const void* state, int* flag, const Geom& g,
                                const HostColl& c, cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    LBMHD_DISPATCH(prec, (finite_kernel<P><<<grid_for(n, 256), 256, 0, st>>>(
                             (const typename Fmt<P>::S*)state, flag, n, g.ps, c.inv_scale)));
    return cudaGetLastError();
}

// Warps of diag_kernel<P, WIDE> resident on the current device at once (the
// kernel's registers and ring bound its blocks per SM), found once per
// device: a process may drive GPUs with different SM counts.
struct DiagOcc {
    long long warps;  // resident warps of the kernel on the device
    int nsm;
};
constexpr int kOccDevices = 64;
template <int P, bool WIDE>
static DiagOcc diag_occupancy() {
    static std::mutex mu;
    static DiagOcc cache[kOccDevices];
    static bool have[kOccDevices] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    auto query = [dev] {
        constexpr size_t smem = diag_smem_bytes<P, WIDE>();
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(diag_kernel<P, WIDE>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        int nsm = 0, bps = 0;
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, diag_kernel<P, WIDE>,
                                                      32 * kDiagWarps, smem);
        cudaGetLastError();  // a failed query leaves the floors below
        nsm = nsm > 0 ? nsm : 1;
        return DiagOcc{(long long)nsm * (bps > 0 ? bps : 1) * kDiagWarps, nsm};
    };
    if (dev < 0 || dev >= kOccDevices) return query();
    std::lock_guard<std::mutex> lock(mu);
    if (!have[dev]) {
        cache[dev] = query();
        have[dev] = true;
    }
    return cache[dev];
}

// The 4-byte formats have two forms of the kernel; both take the plan of the
// form with fewer resident warps, so that one lattice is cut the same way,
// and gives the same bits, whichever form its layout selects.
template <int P>
static DiagOcc diag_occupancy_shared() {
    const DiagOcc a = diag_occupancy<P, true>(), b = diag_occupancy<P, false>();
    return a.warps < b.warps ? a : b;
}

// The wide form serves 4-byte storage whose rows and planes start on
// 16-byte boundaries.
static bool diag_wide(int prec, const Geom& g, const void* state) {
    return (prec == P_FP32 || prec == P_FP32_DEV) && g.nx % 4 == 0 && g.ps % 4 == 0 &&
           ((uintptr_t)state & 15) == 0;
}

static DiagPlan diag_plan_for(const Geom& g, int prec) {
    DiagOcc o{kDiagWarps, 1};
    switch (prec) {
        case P_FP64: o = diag_occupancy<P_FP64, false>(); break;
        case P_FP32: o = diag_occupancy_shared<P_FP32>(); break;
        case P_FP32_DEV: o = diag_occupancy_shared<P_FP32_DEV>(); break;
        case P_FP16_DEV: o = diag_occupancy<P_FP16_DEV, false>(); break;
        case P_FF: o = diag_occupancy<P_FF, false>(); break;
        default: break;
    }
    return diag_plan(g.nx, g.ny, o.warps, o.nsm);
}

// Partial rows a reduction of this lattice needs on the current device.
int diag_num_blocks(const Geom& g, int prec) { return diag_plan_for(g, prec).nblocks; }

template <int P, bool WIDE>
static cudaError_t diag_launch_p(const void* state, double* partials, const Geom& g,
                                 const HostColl& c, const DiagPlan& d, cudaStream_t st) {
    constexpr size_t smem = diag_smem_bytes<P, WIDE>();
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(
            diag_kernel<P, WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    diag_kernel<P, WIDE><<<d.nblocks, 32 * kDiagWarps, smem, st>>>(
        (const typename Fmt<P>::S*)state, g.nx, g.ny, g.ps, c.inv_scale, d.nstrips, d.seglen,
        d.nunits, partials);
    return cudaGetLastError();
}

cudaError_t launch_diag(int prec, const void* state, double* partials, double* out12,
                        const Geom& g, const HostColl& c, cudaStream_t st) {
    const bool wide = diag_wide(prec, g, state);
    const DiagPlan d = diag_plan_for(g, prec);
    const int nb = d.nblocks;
    cudaError_t e = cudaSuccess;
    if (wide && prec == P_FP32)
        e = diag_launch_p<P_FP32, true>(state, partials, g, c, d, st);
    else if (wide)
        e = diag_launch_p<P_FP32_DEV, true>(state, partials, g, c, d, st);
    else
        LBMHD_DISPATCH(prec, (e = diag_launch_p<P, false>(state, partials, g, c, d, st)));
    if (e != cudaSuccess) return e;
    diag_final_kernel<<<1, 256, 0, st>>>(partials, nb, (double)g.nx * g.ny, out12);
    return cudaGetLastError();
}

}  // namespace lbmhd

// ---- double-word arithmetic check -----------------------------------------
namespace lbmhd {

__global__ void ff_eval_kernel(int op, const double* __restrict__ x, const double* __restrict__ y,
                               double* __restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const ff a(x[i]), b(y[i]);
        ff r;
        switch (op) {
            case 0: r = a + b; break;
            case 1: r = a - b; break;
            case 2: r = a * b; break;
            case 3: r = rcp(a); break;
            case 4: r = sqrt_(a); break;
            case 5: r = kmul((float)y[i], a); break;
            default: {
                const ff s = a + b;
                const double ulp = s.hi == 0.0f ? 0.0
                                   : ldexp(1.0, ilogb((double)s.hi) - 23);
                out[i] = ulp > 0.0 ? fabs((double)s.lo) / ulp : (s.lo == 0.0f ? 0.0 : 1e30);
                continue;
            }
        }
        out[i] = (double)r.hi + (double)r.lo;
    }
}

}  // namespace lbmhd

extern "C" int lbmhd_ff_eval(int op, const double* x, const double* y, double* out, long long n) {
    using namespace lbmhd;
    if (!x || !y || !out || n < 0 || op < 0 || op > 6) {
        set_error("lbmhd_ff_eval: NULL array, n < 0 or unknown op");
        return LBMHD_EINVAL;
    }
    if (n == 0) return LBMHD_OK;
    double* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, 3 * (size_t)n * sizeof(double));
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("lbmhd_ff_eval: ") + cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? LBMHD_ENOMEM : LBMHD_ECUDA;
    }
    const size_t b = (size_t)n * sizeof(double);
    e = cudaMemcpy(d, x, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d + n, y, b, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        ff_eval_kernel<<<grid_for(n, 256), 256>>>(op, d, d + n, d + 2 * n, n);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, d + 2 * n, b, cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(std::string("lbmhd_ff_eval: ") + cudaGetErrorString(e));
        return LBMHD_ECUDA;
    }
    return LBMHD_OK;
}
