/*
 * lbmhd.h -- C ABI of the GB300 (sm_103a) filtered lattice Boltzmann MHD
 * library: a D2Q9 multi-relaxation-time density distribution and a D2Q5
 * vector magnetic distribution on a periodic 2D lattice, with a local
 * Smagorinsky-type eddy viscosity and eddy resistivity (Flint & Vahala,
 * "Lattice Boltzmann Large Eddy Simulation Model of MHD", arXiv:1607.08675).
 *
 * Conventions shared by every entry point:
 *  - All functions are extern "C"; those returning int return LBMHD_OK (0)
 *    or a negative LBMHD_E* code and never abort.  lbmhd_last_error() gives
 *    a message for the calling thread's last failure.
 *  - A field is nx*ny doubles, node (x, y) at index y*nx + x (x fastest).
 *  - Host pointers are owned by the caller and are not retained after the
 *    call returns.  Device pointers (the *_device variants) must be
 *    cudaMalloc'd (or torch) memory on the handle's device; they are read or
 *    written in stream order on the handle's stream and not retained.
 *  - The library owns all device memory of a handle; lbmhd_destroy frees it.
 *  - After LBMHD_ECUDA a handle may only be destroyed.  After any other
 *    error the handle is unchanged and stays usable.
 *  - Calls on one handle must not race each other (one host thread at a
 *    time); different handles are independent.
 *
 * Physics: streaming is the shift of Sec. 1.2 (pull form: f_i(x) <-
 * f*_i(x - c_i)); the density collision relaxes the moments M = T f of
 * Eq. FluidTMatrix towards Eq. KinMomentEq with diagonal rates s_j (Sec. 3);
 * the magnetic collision is single-relaxation towards the D2Q5 equilibrium
 * of Sec. 3 (Eq. LBMagEqn).  Transport coefficients follow Sec. 4.3:
 * nu = (1/s_3 - 1/2)/3, eta = (1/s_m - 1/2)/3.  With les != 0 each node
 * raises its relaxation times by the Smagorinsky increments
 * nu_t = C_S Delta^2 |S| and eta_t = C_S Delta^2 |j| of
 * Eqs. SmagorinskyMHDClosureV/B, with |S| and |j| taken from the node's own
 * non-equilibrium moments (Sec. 1.2: sum c_a c_b f^(1) = -(rho tau/3) 2 S_ab)
 * and the implicit dependence on tau solved exactly.  With les = 2 the
 * collision instead relaxes towards the paper's filtered equilibria
 * (Sec. 4.1): M_i^eq + Delta^2 M_i^(Delta), the corrections obtained by
 * applying the filter rules for products and ratios (Eqs.
 * FilterExampleSmall/Large) to Eqs. KinMomentEq and MagMomentEq (Eq.
 * DeltaEqEx is the M_3 case), with periodic central differences of the
 * streamed conserved moments; each step is then two launches (a moments
 * pass and the step) and needs 5 extra planes of device memory.  les = 3
 * uses the same moments pass for the cross-helicity closure of Carati et
 * al. quoted in Sec. 1.1 (Eqs. CHClosureV/B): nu_t = C_S Delta^2
 * |S^v_ab S^b_ab|^(1/2), eta_t = C_S Delta^2 sgn(j.omega) |j.omega|^(1/2)
 * from central differences of u and B, tau = tau0 + 3 x (backscatter
 * allowed, total resistivity kept >= 0).  les = 2 and 3 are not available
 * to the adjoint.
 */
#ifndef LBMHD_H
#define LBMHD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBMHD_ABI_VERSION 1u

/* Status codes. */
#define LBMHD_OK 0
#define LBMHD_EINVAL (-1)     /* bad argument or parameter */
#define LBMHD_ENOMEM (-2)     /* device or host allocation failed */
#define LBMHD_ECUDA (-3)      /* CUDA runtime error; handle unusable */
#define LBMHD_ENONFINITE (-4) /* a non-finite density was detected */
#define LBMHD_ETIMEOUT (-5)   /* a bounded device wait expired */
#define LBMHD_EVERSION (-6)   /* params.abi_version mismatch */
#define LBMHD_ESTATE (-7)     /* call out of order (e.g. step before init) */

/* Storage / arithmetic of a handle.  The populations are kept in HBM as
 * 19 planes (9 f_i, then g_k x/y for k = 0..4).  *_DEV formats store the
 * deviation from the rest equilibrium (f_i - w_i; g_k itself). */
typedef enum {
    LBMHD_FP64 = 0,     /* FP64 storage, FP64 arithmetic (parity mode) */
    LBMHD_FP32 = 1,     /* FP32 storage of f and g, FP32 arithmetic */
    LBMHD_FP32_DEV = 2, /* FP32 storage of deviations, FP32 arithmetic */
    LBMHD_FP16_DEV = 3, /* FP16 storage of scaled deviations, FP32 arithmetic */
    LBMHD_FF = 4        /* double-word deviations: each value an FP32 pair
                           (hi, lo), 8 bytes, 48-bit significand; arithmetic
                           in double-word on the FP32 units (unit roundoff
                           2^-48 against FP64's 2^-53).  TMA variant not
                           available. */
} lbmhd_precision;

typedef struct lbmhd_t lbmhd_t;

/* Run parameters.  Fill with lbmhd_params_default, then override. */
typedef struct {
    uint32_t abi_version;  /* must be LBMHD_ABI_VERSION */
    int32_t precision;     /* lbmhd_precision */
    double tau_nu;         /* base 1/s_3 = 1/s_4, > 1/2 (Sec. 4.3: nu) */
    double tau_eta;        /* base 1/s_m, > 1/2 (Sec. 4.3: eta) */
    double C_S;            /* Smagorinsky constant, >= 0, enters linearly */
    double delta;          /* filter width Delta in lattice units, > 0 */
    double s5, s6;         /* energy-flux rates; <= 0: tied to 1/tau_nu */
    double s7, s8;         /* energy rates; <= 0: tied to the local s_nu */
    int32_t les;           /* 0: none; 1: local Smagorinsky rates; 2: the paper's
                              filtered equilibria (kinetic LES); 3: the
                              cross-helicity closure (see below) */
    int32_t check_finite_every; /* 0: never; k: test rho every k steps */
    double fp16_scale;     /* LBMHD_FP16_DEV: stored = deviation * scale */
    void* stream;          /* cudaStream_t to run on; NULL: library stream */
} lbmhd_params;

/* FP64 diagnostics (sums over nodes in a fixed order, deterministic).
 * <.> is the mean over nodes; omega, j_z and div B use periodic central
 * differences of the node moments. */
typedef struct {
    double mass;           /* sum rho */
    double mom_x, mom_y;   /* sum rho u */
    double bsum_x, bsum_y; /* sum B */
    double E_kin;          /* <rho |u|^2> / 2 */
    double E_mag;          /* <|B|^2> / 2 */
    double enstrophy;      /* <omega^2> / 2 */
    double cross_helicity; /* <u . B> */
    double divB_max;       /* max |div B| (Sec. 1.2 claim: div B = 0) */
    double divB_rms;       /* sqrt <(div B)^2> */
    double current_sq;     /* <j_z^2> / 2 */
    int64_t step;          /* steps taken since init */
} lbmhd_diag;

/* Defaults: FP64, tau_nu = tau_eta = 0.6, C_S = 0.1, delta = 1, all of
 * s5..s8 tied, les = 1, no finite check, fp16_scale = 1024, stream NULL. */
void lbmhd_params_default(lbmhd_params* p);

/* Validate p and allocate the two population buffers of an nx x ny
 * periodic lattice on the current CUDA device.  Rejects (EINVAL) nx or
 * ny < 1, tau <= 1/2, non-finite values, C_S < 0, delta <= 0, a given
 * s5..s8 outside (0, 2), fp16_scale <= 0, and a non-positive bulk
 * viscosity xi = -1/9 - 1/(9 s_4) - 1/(15 s_7) + 2/(5 s_8) (Sec. 4.3) at
 * the base rates.  *out is set on success only. */
int lbmhd_create(int nx, int ny, const lbmhd_params* p, lbmhd_t** out);

/* Set the state to the local equilibria f^eq(rho, u, B), g^eq(u, B) of
 * Sec. 3 (the paper gives no initial condition; equilibrium is taken).
 * Arguments: five host fields of nx*ny doubles (x fastest; caller-owned,
 * not retained).  Pinned host arrays (cudaHostAlloc / cudaHostRegister) are
 * read by the kernel in place; pageable ones are staged through a
 * temporary device copy.  rho must be positive and finite: checked on the
 * device; on failure EINVAL and the handle is uninitialised (step and
 * moments return ESTATE) until a successful init.  Resets the step
 * counter.  Synchronises with the handle's stream before returning. */
int lbmhd_init(lbmhd_t* h, const double* rho, const double* ux, const double* uy,
               const double* bx, const double* by);

/* As lbmhd_init, from device fields; enqueued on the handle's stream.  The
 * fields are read in that stream's order: the caller completes them first
 * (produces them on the handle's stream, or synchronises), and keeps them
 * until the handle's stream has passed the call. */
int lbmhd_init_device(lbmhd_t* h, const double* rho, const double* ux, const double* uy,
                      const double* bx, const double* by);

/* Advance n >= 0 time steps: each is one fused launch of pull-stream and
 * collide (Sec. 1.2 and Sec. 3) over the whole lattice.  Asynchronous on
 * the handle's stream; long runs replay a captured CUDA graph.  Returns
 * ESTATE before init.  A pending non-finite report (check_finite_every)
 * is returned by the next synchronising call. */
int lbmhd_step(lbmhd_t* h, int n);

/* rho, u and B of the current state (conserved by the collision, so they
 * are the moments of Sec. 3 of the last streamed populations).  Host
 * output fields of nx*ny doubles (caller-owned); pinned ones are written by
 * the kernel in place, pageable ones through a temporary device copy.
 * Synchronises. */
int lbmhd_moments(lbmhd_t* h, double* rho, double* ux, double* uy, double* bx, double* by);

/* As lbmhd_moments, into device fields; enqueued, does not synchronise. */
int lbmhd_moments_device(lbmhd_t* h, double* rho, double* ux, double* uy, double* bx,
                         double* by);

/* FP64 diagnostics of the current state (see lbmhd_diag).  Synchronises. */
int lbmhd_diagnostics(lbmhd_t* h, lbmhd_diag* out);

/* Copy the 19 population planes out as FP64 (decoded from the storage
 * format): host array of 19*nx*ny doubles, plane p at p*nx*ny.  Planes
 * 0..8 are f_i in the order of the lattice lists of Sec. 3; plane 9+2k+a
 * is component a of g_k.  Synchronises. */
int lbmhd_get_state(lbmhd_t* h, double* state);

/* Replace the state with host FP64 planes (layout as lbmhd_get_state),
 * encoded to the storage format; the step counter is left unchanged.
 * Together with lbmhd_get_state this is checkpoint / resume, bit for bit
 * for FP64, FP32 and FP16 storage.  LBMHD_FF pairs are rounded to FP64 on
 * the way out (the stored deviation carries up to 48 bits), so an FF run
 * resumed from them continues from a state within FP64 rounding of the
 * original, not bit for bit (lbmhd_get_state_raw / lbmhd_set_state_raw are). */
int lbmhd_set_state(lbmhd_t* h, const double* state);

/* The stored state in the handle's own format, for bit-exact checkpoints of
 * every format (FF pairs included) at the storage size: a host buffer of
 * bytes = 19 * nx * ny * value size (8 for FP64 and FF, 4 for FP32 and
 * FP32_DEV, 2 for FP16_DEV; lbmhd_bytes_per_cell / 2 per node), plane p at
 * byte offset p * nx * ny * value size, node (x, y) at y * nx + x within a
 * plane.  Values: FP64 / FP32 populations f and g; FP32_DEV deviations
 * f - w (g itself); FP16_DEV binary16 deviations times fp16_scale; FF
 * (hi, lo) FP32 pairs of the deviations.  Caller-owned; synchronises.
 * EINVAL for NULL or a wrong byte count, ESTATE (get) before init.
 * set_state_raw leaves the step counter unchanged. */
int lbmhd_get_state_raw(lbmhd_t* h, void* state, size_t bytes);
int lbmhd_set_state_raw(lbmhd_t* h, const void* state, size_t bytes);

/* Copy rows [src_row, src_row + nrows) of every population plane of src's
 * current state into rows [dst_row, ...) of dst's (same nx and precision;
 * both on this GPU).  Enqueued on dst's stream after src's pending work.
 * This is the halo exchange of a y-slab domain decomposition (one ghost
 * row above and below each slab, refreshed after every step): the step
 * reads only rows y - 1, y, y + 1, so stepping each slab with ghost rows
 * and exchanging them reproduces the undivided lattice bit for bit.  (The
 * paper has no counterpart: it is the sharding of the lattice.)
 * EINVAL for mismatched handles or rows outside a lattice. */
int lbmhd_copy_rows(lbmhd_t* dst, int dst_row, lbmhd_t* src, int src_row, int nrows);

/* ---- one step in parts, and halo messages (domain decomposition) --------
 * The step of Sec. 1.2 / Sec. 3 pulls every population from a neighbour
 * (streaming is a shift) and collides locally, so a lattice cut into row
 * slabs can be advanced slab by slab, each slab with ghost rows that hold
 * copies of its neighbours' boundary rows.  These calls let one handle hold
 * a slab: the interior rows that need no ghost row are computed while the
 * halo is in flight, the rows next to the ghosts once it has arrived, and
 * ghost rows are never computed at all.  (The paper has no counterpart:
 * this is the sharding of the lattice.)
 *
 * lbmhd_step_rows: rows y0 <= y < y1 of the next state (periodic pull) into
 * the handle's back buffer; the current state is unchanged and stays
 * current.  Reads rows y0 - 1 .. y1 of the current state (y0 - 2 .. y1 + 1
 * with les 2, 3, whose moment gradients pull from two rows away).  Rows not
 * computed before the commit keep the back buffer's older contents.
 * Asynchronous on the handle's stream; no finite check.  EINVAL unless
 * 0 <= y0 < y1 <= ny; ESTATE before init.
 * lbmhd_step_commit: the back buffer becomes the current state and the step
 * counter advances by one (host only, nothing is enqueued). */
int lbmhd_step_rows(lbmhd_t* h, int y0, int y1);
int lbmhd_step_commit(lbmhd_t* h);

/* Halo messages: the planes selected by plane_mask (bit p = plane p of the
 * 19, in the order f_0..f_8, g_0x, g_0y, ..., g_4y) of row `row` of the
 * current state, gathered into (pack) or scattered from (unpack) buf: device
 * memory holding popcount(plane_mask) * nx stored values in the handle's
 * storage format (lbmhd_get_state_raw's value layout), plane after plane in
 * increasing plane order, x fastest.  buf is caller-owned, aligned to the
 * stored value size.  Enqueued on `stream` (cudaStream_t; NULL: the
 * handle's stream); ordering against the handle's stream is the caller's
 * (events).  Which planes a ghost row needs: with local rates (les 0, 1)
 * the ghost row below a slab needs the planes streaming upwards (c_y = +1:
 * f_2, f_5, f_6, g_2), the one above those streaming downwards; with
 * les 2, 3 the nearer ghost row also needs the planes with c_y = 0 and the
 * further one the planes streaming towards the slab.  EINVAL for NULL or
 * misaligned buf, a row outside the lattice or mask bits above 18; ESTATE
 * (pack) before init. */
int lbmhd_pack_row(lbmhd_t* h, int row, unsigned plane_mask, void* buf, void* stream);
int lbmhd_unpack_row(lbmhd_t* h, int row, unsigned plane_mask, const void* buf, void* stream);

/* Wait for the handle's stream; reports a pending non-finite density. */
int lbmhd_sync(lbmhd_t* h);

/* Steps taken since the last init (host counter, no synchronisation). */
int64_t lbmhd_step_count(const lbmhd_t* h);

/* Algorithmic HBM bytes per node update of a step (19 populations read and
 * 19 written): 304 (FP64), 152 (FP32, FP32_DEV), 76 (FP16_DEV); 0 for an
 * unknown precision. */
int lbmhd_bytes_per_cell(int precision);

/* Number of step-kernel launches issued by this handle since creation. */
int64_t lbmhd_launch_count(const lbmhd_t* h);

/* Launch shape of the step kernel.  vec >= 1 selects the register kernel:
 * vec nodes per thread along x (1, 2 or 4, dividing nx) and block threads
 * per block (multiple of 32, <= 256).  vec = 0 selects the TMA-staged
 * kernel (FP32, FP32_DEV, FP16_DEV): persistent CTAs of `block` threads
 * stream row tiles of `block` nodes (128, 256 or 512, dividing nx) through
 * a shared-memory ring filled by bulk asynchronous copies.  vec = 8 is
 * available for FP16 storage (16-byte loads).  Default: the register
 * kernel with 4 nodes per thread in 64-thread blocks (FP32 storage), 8
 * nodes in 32-thread blocks (FP16 storage) or 2 nodes in 128-thread blocks
 * (FP64), falling back to narrower vectors when nx is not a multiple.
 * Results do not depend on the shape (bit for bit).  EINVAL if the shape
 * is not available.
 * For les 2 and 3 (steps that need moment gradients): vec = 1 selects the
 * fused kernel (one launch per step; CTAs sweep column strips; `block`
 * ignored on input, reported as strip width + 32), vec = 0 the two-pass
 * kernels (a moments pass, then the step: two launches per step).  Both
 * give the same bits.  Default: fused for FP32, FP32_DEV, FP16_DEV and for
 * FF with les 3; two-pass for FP64 and for FF with les 2 (faster there). */
int lbmhd_set_launch(lbmhd_t* h, int vec, int block);
int lbmhd_get_launch(const lbmhd_t* h, int* vec, int* block);

/* Diagnostics of a caller-owned state buffer, allocating nothing.  The
 * paper has no counterpart: this serves callers that cannot call
 * cudaMalloc, e.g. a host application whose device memory all comes from
 * its own arena, or a latency-critical loop that cannot take the implicit
 * device synchronisation of cudaMalloc / cudaFree.
 * Arguments: state = device pointer to 19 planes in the storage format of
 * `precision` (lbmhd_precision), plane p at element offset p*plane_stride,
 * node (x, y) at y*nx + x within a plane (plane_stride >= nx*ny; an FP64
 * array from lbmhd_get_state qualifies with plane_stride = nx*ny);
 * fp16_scale = the scale of LBMHD_FP16_DEV storage (ignored otherwise);
 * out = device pointer to 12 doubles, written in the field order of
 * lbmhd_diag (mass ... current_sq); stream = cudaStream_t (NULL: legacy
 * default stream).  Enqueued on the stream; does not synchronise.
 * Alignment: state on a multiple of the stored value size (8 bytes for
 * FP64 and FF, 4 for FP32 and FP32_DEV, 2 for FP16_DEV), out on 8 bytes;
 * other pointers get EINVAL before anything is launched.
 * The per-block partial sums live in one static device array of 96 KiB
 * (1024 rows of 12 doubles), held by every GPU that loads the library
 * until the process exits; every lattice the library accepts
 * (nx*ny <= 2^30) fits, larger ones are rejected with EINVAL.  The first
 * call on a device looks up the array's device address (once per device)
 * and the first call for each precision queries the reduction kernel's
 * occupancy (the work split follows it), so make those first calls before
 * any stream capture.  All calls share the
 * array: calls that overlap on the GPU (other streams, other threads)
 * race and give wrong sums; serialise them.  Each call writes every
 * partial row it reads, so no clearing is needed between calls.
 * Errors: EINVAL for NULL or misaligned pointers, an unknown precision,
 * bad sizes or scale; ECUDA if the address lookup or the launch fails. */
int lbmhd_diagnostics_noalloc(const void* state, int precision, int nx, int ny,
                              long long plane_stride, double fp16_scale, double* out,
                              void* stream);

/* Free everything the handle owns.  NULL is accepted. */
void lbmhd_destroy(lbmhd_t* h);

/* One double-word (LBMHD_FF) operation, elementwise on the device, for
 * checking that arithmetic against its error bounds.  x, y, out: host
 * arrays of n doubles (caller-owned).  Each input is first rounded to the
 * nearest double-word (48-bit significand); out[i] = hi + lo of the
 * result, computed in FP64.  op: 0 x + y, 1 x - y, 2 x * y, 3 1 / x,
 * 4 sqrt(x), 5 (float)y * x (the constant-product path; y must hold FP32
 * values), 6 the normalisation excess |lo| / ulp(hi) of x + y (<= 0.5 for a
 * normalised pair).  Synchronises.  Errors: EINVAL for NULL pointers, n < 0
 * or an unknown op; ENOMEM; ECUDA. */
int lbmhd_ff_eval(int op, const double* x, const double* y, double* out, long long n);

/* ---- adjoint (discrete, hand-written) ------------------------------------
 * Gradients of a scalar function of the final moments with respect to
 * C_S, tau_nu, tau_eta and the initial fields, through the exact transpose
 * of the discrete step (pull-stream and the collision of Sec. 3 with the
 * local Smagorinsky rates).  Supported storage: FP64, FF, FP32, FP32_DEV.  The
 * derivative of |x| and of sqrt at 0 (local |S|, |j| of exactly zero) is
 * taken as 0. */

/* Initialise from five device fields (as lbmhd_init_device) and advance
 * nsteps steps, keeping an FP64 checkpoint of the state every `every`
 * steps in device memory owned by the handle (ceil(nsteps/every) * 19 *
 * nx*ny doubles, plus a copy of the five fields).  Afterwards the handle
 * holds the final state.  Replaces any earlier record. */
int lbmhd_adjoint_record(lbmhd_t* h, const double* rho0, const double* ux0, const double* uy0,
                         const double* bx0, const double* by0, int nsteps, int every);

/* Back-propagate dL/d(final rho, u_x, u_y, B_x, B_y) (device fields; NULL
 * means zero) through the recorded run: restore each checkpoint, recompute
 * the segment with the forward kernel (bit-identical), and apply the
 * adjoint step backwards.  Writes dtheta[0..2] = dL/dC_S, dL/dtau_nu,
 * dL/dtau_eta (host, FP64, accumulated in FP64) and, where not NULL, the
 * device fields dL/d(rho0, ux0, uy0, bx0, by0).  ESTATE without a record or
 * if the handle stepped since.  Temporary device memory: `every` states in
 * the storage format and two adjoint states.  Synchronises. */
int lbmhd_adjoint_backward(lbmhd_t* h, const double* g_rho, const double* g_ux,
                           const double* g_uy, const double* g_bx, const double* g_by,
                           double* dtheta, double* d_rho0, double* d_ux0, double* d_uy0,
                           double* d_bx0, double* d_by0);

/* Free the recorded checkpoints (also done by lbmhd_destroy). */
int lbmhd_adjoint_release(lbmhd_t* h);

/* ---- 3D lattices (D3Q27 density, D3Q7 vector magnetic populations) -------
 * The paper works in 2D and notes that the model extends to 3D with more
 * lattice velocities (Sec. 3 opening; the Conclusion names D3Q27).  The 3D
 * step: D3Q27 populations with the paper's D2Q9 equilibrium written with 3D
 * vectors plus the 3D trace term -9/2 w |B|^2/6 (zero in 2D), D3Q7 vector
 * populations with the paper's D2Q5 equilibrium on the six axes (weight
 * 1/6; the rest weight is zero, so six vector populations are stored), BGK
 * collision (the paper's MRT with all rates tied) and magnetic SRT, with the
 * local Smagorinsky rates (les 1) from the traceless non-equilibrium stress
 * and the axial vector of the magnetic non-equilibrium first moment.
 * Storage: FP64, FP32, FP16 deviations (binary16 (f - w_i) times
 * fp16_scale, g times fp16_scale; FP32 arithmetic) or double-word
 * deviations (FF: (hi, lo) FP32 pairs, double-word arithmetic), 45 planes
 * (27 f_i with i = 9 kz + 3 ky + kx,
 * c = (v[kx], v[ky], v[kz]), v = {0, 1, -1}; then g_q (x, y, z) for
 * q = +x, -x, +y, -y, +z, -z), node (x, y, z) at (z ny + y) nx + x.  Host
 * fields: FP64 arrays of nx*ny*nz, x fastest, caller-owned.  Periodic in
 * x, y and z.  The gradient closures take two launches per step (a pass
 * that writes rho - 1, j, B of the streamed populations into seven planes,
 * then the step with central differences of those planes at the six
 * neighbours): les 2 relaxes towards the paper's filtered equilibria
 * (Sec. 4.1; the product and ratio rules of Sec. 2 applied to every
 * nonlinear term of the 3D equilibria), les 3 takes the cross-helicity
 * closure's relaxation times (Eqs. CHClosureV/B with 3D strain and curl). */
typedef struct lbmhd3_t lbmhd3_t;

/* Uses precision (FP64, FP32, FP16_DEV with fp16_scale, or FF), check_finite_every (every k steps
 * the rest population f_0 and the first magnetic plane of every node are
 * tested; a non-finite value is seen at most one step after it appears and
 * reported as ENONFINITE by the next lbmhd3_sync, moments, get_state or
 * diagnostics call until the next init or state write), tau_nu, tau_eta, C_S, delta, les (0 off,
 * 1 local rates, 2 filtered equilibria, 3 cross-helicity closure) and stream
 * of p.  Allocates two state buffers, and for les 2, 3 seven field planes.
 * EINVAL for other precisions or closures, tau <= 1/2, more than 2^30
 * nodes; ENOMEM. */
int lbmhd3_create(int nx, int ny, int nz, const lbmhd_params* p, lbmhd3_t** out);
/* Equilibrium initialisation from seven host fields; synchronises.  EINVAL
 * for NULL or a density that is not positive and finite. */
int lbmhd3_init(lbmhd3_t* h, const double* rho, const double* ux, const double* uy,
                const double* uz, const double* bx, const double* by, const double* bz);
/* n fused stream-collide steps, asynchronous on the handle's stream. */
int lbmhd3_step(lbmhd3_t* h, int n);
/* As lbmhd3_init, from seven device fields of nx*ny*nz doubles; enqueued on
 * the handle's stream (no check of rho).  The fields are read in that
 * stream's order: the caller completes them first (produces them on the
 * handle's stream, or synchronises), and keeps them until the handle's
 * stream has passed the call. */
int lbmhd3_init_device(lbmhd3_t* h, const double* rho, const double* ux, const double* uy,
                       const double* uz, const double* bx, const double* by, const double* bz);
/* As lbmhd3_moments, into seven device fields; enqueued, does not
 * synchronise. */
int lbmhd3_moments_device(lbmhd3_t* h, double* rho, double* ux, double* uy, double* uz,
                          double* bx, double* by, double* bz);
/* Replace the state with host FP64 planes (layout as lbmhd3_get_state),
 * encoded to the storage format; the step counter is left unchanged.  With
 * lbmhd3_get_state this is checkpoint / resume, bit for bit for FP64, FP32
 * and FP16 storage (FF pairs are rounded to FP64 on the way out; the raw
 * pair below is exact for every format).  Synchronises. */
int lbmhd3_set_state(lbmhd3_t* h, const double* state);
/* The stored state in its own format: a host buffer of bytes = 45 * nodes
 * * value size (8 FP64 and FF, 4 FP32, 2 FP16), plane p at byte offset
 * p * nodes * value size, node (x, y, z) at (z ny + y) nx + x.  Values: FP64
 * / FP32 populations; FP16 binary16 deviations f - w (g itself) times
 * fp16_scale; FF (hi, lo) FP32 pairs of the deviations.  Caller-owned;
 * synchronises.  EINVAL for NULL or a wrong byte count; ESTATE (get) before
 * init.  set leaves the step counter unchanged. */
int lbmhd3_get_state_raw(lbmhd3_t* h, void* state, size_t bytes);
int lbmhd3_set_state_raw(lbmhd3_t* h, const void* state, size_t bytes);
/* rho, ux, uy, uz, bx, by, bz into out7 (host, 7 * nx*ny*nz doubles, field
 * after field); synchronises. */
int lbmhd3_moments(lbmhd3_t* h, double* out7);
/* The 45 populations as FP64 (host, 45 * nx*ny*nz doubles); synchronises. */
int lbmhd3_get_state(lbmhd3_t* h, double* out);
/* FP64 sums, deterministic: mass, momentum (3), sum of B (3), E_K =
 * <rho |u|^2>/2, E_M = <|B|^2>/2, cross helicity <u.B>, max and rms of the
 * periodic central-difference div B; synchronises.  The first call
 * allocates 7 * nx*ny*nz doubles of moment fields kept by the handle. */
int lbmhd3_diagnostics(lbmhd3_t* h, double* out12);
/* Work shape: vec nodes per thread along x (1, 2; must divide nx), block
 * threads (multiple of 32, <= 256).  vec 0 (les 2, 3 only; block ignored,
 * reported as 4): the fused one-pass kernel, in which a CTA sweeps a tile of
 * 32 x 4 columns along z keeping the fields of consecutive planes and the
 * tile's pulled values in shared memory; the default for FP32 closures.
 * vec 3 (les 2, 3 in FP32 or FP16 storage; block 8 = tile rows): the
 * warp-specialised one-pass kernel, in which producer warps pull the planes
 * ahead of the consumer warps that collide them, handing shared-memory
 * slots over on mbarriers with bounded waits; an expired wait makes the
 * next synchronising call return LBMHD_ETIMEOUT.  EINVAL for a shape the
 * handle's closure or format does not take.  Results do not depend on it. */
int lbmhd3_set_launch(lbmhd3_t* h, int vec, int block);
int lbmhd3_get_launch(const lbmhd3_t* h, int* vec, int* block);
int lbmhd3_sync(lbmhd3_t* h);
/* Fault injection for tests of failure detection (the paper has no
 * counterpart).  With LBMHD_DEBUG_DROP_BARRIER_ARRIVAL the producer warps
 * of the warp-specialised closure kernel (vec 3) stop announcing their
 * planes, so the consumer warps' bounded waits expire (~2 s), the kernel
 * returns and the next synchronising call returns LBMHD_ETIMEOUT (the GPU
 * context stays usable; lbmhd3_init or a state write clears the report).
 * 0 clears it.  EINVAL for a NULL handle. */
int lbmhd3_debug(lbmhd3_t* h, int flags);
int64_t lbmhd3_step_count(const lbmhd3_t* h);
int64_t lbmhd3_launch_count(const lbmhd3_t* h);

/* z-slab sharding of a 3D lattice (the step streams by a shift, Sec. 1.2,
 * and collides locally, Sec. 3, so planes are advanced independently given
 * their neighbours).
 * lbmhd3_step_planes: planes z0 <= z < z1 of the next state (periodic pull)
 * into the back buffer; the current state stays current.  Reads planes
 * z0 - 1 .. z1 of the current state (z0 - 2 .. z1 + 1 with les 2, 3).
 * Planes not computed before the commit keep the back buffer's older
 * contents.  Asynchronous on the handle's stream.  EINVAL unless
 * 0 <= z0 < z1 <= nz; ESTATE before init.
 * lbmhd3_step_commit: the back buffer becomes the current state and the
 * step counter advances (host only). */
int lbmhd3_step_planes(lbmhd3_t* h, int z0, int z1);
int lbmhd3_step_commit(lbmhd3_t* h);

/* Halo messages of the 3D state: the planes selected by plane_mask (bit p
 * = storage plane p of the 45) of z-plane z of the current state, gathered
 * into (pack) or scattered from (unpack) buf: device memory of
 * popcount(plane_mask) * nx * ny stored values in the storage format, plane
 * after plane in increasing order, x fastest then y.  buf is caller-owned,
 * aligned to the stored value size.  Enqueued on `stream` (cudaStream_t;
 * NULL: the handle's stream).  A ghost plane below a slab needs the planes
 * streaming upwards (c_z = +1: the 9 f_i with kz = 1 and g_{+z}); with les
 * 2, 3 the nearer ghost plane also needs the c_z = 0 planes and the second
 * ghost plane the upward ones.  EINVAL for NULL or misaligned buf, a plane
 * outside the lattice or mask bits above 44; ESTATE (pack) before init. */
int lbmhd3_pack_plane(lbmhd3_t* h, int z, uint64_t plane_mask, void* buf, void* stream);
int lbmhd3_unpack_plane(lbmhd3_t* h, int z, uint64_t plane_mask, const void* buf, void* stream);
/* Bytes a 3D step moves per node: 45 values read and written (0 for an
 * unsupported precision). */
int lbmhd3_bytes_per_cell(int precision);
void lbmhd3_destroy(lbmhd3_t* h);

/* ---- ensembles: many independent lattices advanced together ------------
 * A batch holds nruns periodic lattices of their own sizes, each with its
 * own tau_nu, tau_eta and C_S (every other parameter from `common`), and
 * advances all of them by the same step of Sec. 1.2 / Sec. 3 in one
 * persistent kernel: co-resident CTAs sweep the work units of every run,
 * meet at a grid barrier, and continue with the next step
 * (steps_per_launch steps per launch); long runs replay a captured CUDA
 * graph of such launches.  Each run evolves bit-identically to an lbmhd_t
 * with the same parameters.  The grid-barrier wait is bounded (about one
 * second); on expiry the step reports LBMHD_ETIMEOUT at the next
 * synchronising call and every run must be re-initialised.
 * With les = 2 or 3 (common->les) each step is one launch with no grid
 * barrier: the fused kinetic kernel over every run's strip-segments (one CTA
 * per segment of a column strip of a run; vec 1), or the moments pass and
 * the step over every run's nodes (vec 0, `block` nodes per unit); the batch
 * holds five moment planes per run for the latter.  The default is the
 * single lattice's choice: two-pass for FP64, and for FF with les 2. */
typedef struct lbmhd_batch_t lbmhd_batch_t;

/* Arrays of nruns entries (caller-owned, not retained).  Every run is
 * validated as lbmhd_create validates one lattice; the ensemble may hold
 * at most 2^31 nodes.  Allocates both population buffers. */
int lbmhd_batch_create(int nruns, const int* nx, const int* ny, const double* tau_nu,
                       const double* tau_eta, const double* C_S, const lbmhd_params* common,
                       lbmhd_batch_t** out);

/* Equilibrium initialisation of run `run` from five host fields (as
 * lbmhd_init).  Every run must be initialised before lbmhd_batch_step. */
int lbmhd_batch_init(lbmhd_batch_t* b, int run, const double* rho, const double* ux,
                     const double* uy, const double* bx, const double* by);

/* Advance every run by n steps (asynchronous on the batch's stream). */
int lbmhd_batch_step(lbmhd_batch_t* b, int n);

/* Host moments / FP64 populations of one run (layouts as lbmhd_moments and
 * lbmhd_get_state); synchronise. */
int lbmhd_batch_moments(lbmhd_batch_t* b, int run, double* rho, double* ux, double* uy,
                        double* bx, double* by);
int lbmhd_batch_get_state(lbmhd_batch_t* b, int run, double* state);

/* Wait for the batch's stream; reports ETIMEOUT / ENONFINITE. */
int lbmhd_batch_sync(lbmhd_batch_t* b);

/* Work shape: vec nodes per thread (1, 2, 4; must divide every run's nx),
 * block threads per work unit (multiple of 32, <= 256), steps per
 * persistent launch (1..4096).  Results do not depend on the shape.
 * Ensembles with les 2 or 3 take one step per launch and vec 1 (the fused
 * kernel; block is then not used) or vec 0 (the two-pass kernels). */
int lbmhd_batch_set_launch(lbmhd_batch_t* b, int vec, int block, int steps_per_launch);
int lbmhd_batch_get_launch(const lbmhd_batch_t* b, int* vec, int* block, int* steps_per_launch);

/* Autotuner: times every available (vec, block, steps_per_launch) for
 * trial_steps steps on a rest state and keeps the fastest.  Results are
 * cached in the JSON file cache_path (key: GPU name, precision, the
 * multiset of lattice shapes); a cached key is applied without timing.
 * cache_path may be NULL (no cache).  Must run before any
 * lbmhd_batch_init (ESTATE otherwise); best_mlups (may be NULL) receives
 * the winner's throughput. */
int lbmhd_batch_autotune(lbmhd_batch_t* b, const char* cache_path, int trial_steps,
                         double* best_mlups);

/* Counters (host, no synchronisation): steps since the last init, and
 * persistent-kernel launches since creation. */
int64_t lbmhd_batch_step_count(const lbmhd_batch_t* b);
int64_t lbmhd_batch_launch_count(const lbmhd_batch_t* b);

/* Fault injection for tests of failure detection.  With
 * LBMHD_DEBUG_DROP_BARRIER_ARRIVAL one CTA leaves the persistent kernel
 * before its first grid barrier, so the others' bounded waits expire and
 * the next synchronising call returns LBMHD_ETIMEOUT (the GPU context stays
 * usable).  0 clears it. */
#define LBMHD_DEBUG_DROP_BARRIER_ARRIVAL 1
int lbmhd_batch_debug(lbmhd_batch_t* b, int flags);

/* Free everything the batch owns.  NULL is accepted. */
void lbmhd_batch_destroy(lbmhd_batch_t* b);

/* Message of the calling thread's last failed call ("" if none). */
const char* lbmhd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LBMHD_H */
