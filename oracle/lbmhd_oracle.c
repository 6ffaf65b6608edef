/*
 * lbmhd_oracle.c -- plain, slow, FP64 CPU oracle for the filtered lattice
 * Boltzmann MHD time step of Flint & Vahala, "Lattice Boltzmann Large Eddy
 * Simulation Model of MHD" (arXiv:1607.08675).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA path is checked against.  Only the test suite, the package smoke check
 * and the CPU-baseline leg of the benchmark may build, load or call it.  It
 * shares no code, header, table or helper with the CUDA library.
 *
 * Written for readability, not speed: scalar loops, IEEE double, compiled
 * with -ffp-contract=off so that every product and sum is rounded on its own.
 *
 * Storage convention of a lattice state (shared with the CUDA path only as a
 * documented layout, never as code): 19 planes of nx*ny doubles, plane p at
 * offset p*nx*ny, cell (x, y) at y*nx + x.  Planes 0..8 are the D2Q9 density
 * populations f_i; plane 9 + 2k + a is component a (0 = x, 1 = y) of the
 * D2Q5 vector magnetic population g_k.  The state stored between steps is
 * the post-collision population at each node (streaming happens at the start
 * of the next step, by pulling from x - c_i).
 *
 * Readings of the paper taken here (where it is silent or garbled):
 *   - D2Q9 weights {4/9, 1/9, 1/36} and D2Q5 weights {1/3, 1/6}: not stated
 *     in Sec. 3; these are the only values for which T f^eq reproduces the
 *     equilibrium-moment table (Eq. KinMomentEq) and T_m g^eq reproduces
 *     Eq. MagMomentEq.
 *   - N_{a1}^eq, N_{a2}^eq use u (not rho*u): Eq. MagMomentEq prints rho*u
 *     but the D2Q5 equilibrium of Sec. 3 and the induction term of
 *     Eq. FinalMagnetic both give u_x B_a - u_a B_x.
 *   - Local LES relaxation (the paper gives no local rate; this is its
 *     MHD-Smagorinsky closure, Eqs. SmagorinskyMHDClosureV/B, applied as an
 *     eddy increment of the transport coefficients of Sec. 4.3):
 *       nu_eff  = nu  + C_S Delta^2 |S|,  |S| from the non-equilibrium
 *                 stress (Sec. 1.2: sum c_a c_b f^(1) = -(rho tau/3)(2 S_ab))
 *       eta_eff = eta + C_S Delta^2 |j|,  |j| from the antisymmetric part of
 *                 the non-equilibrium first moment of g, -(tau_m/3) j_z
 *     with nu = (tau - 1/2)/3 and eta = (tau_m - 1/2)/3 (Sec. 4.3).  The
 *     implicit dependence on tau is solved exactly (a quadratic in tau).
 *   - s_5, s_6 default to the base 1/tau_nu, s_7 = s_8 to the local s_nu; any
 *     positive value given overrides (the paper leaves them free, Sec. 3).
 *   - les = 2 is the paper's own kinetic LES (Sec. 4.1): the collision
 *     relaxes towards the filtered equilibria M_i^eq + Delta^2 M_i^(Delta),
 *     with M_i^(Delta) obtained by applying the filter rules for products
 *     (Eq. FilterExampleSmall) and ratios (Eq. FilterExampleLarge) to every
 *     term of Eqs. KinMomentEq and MagMomentEq (Eq. DeltaEqEx is the M_3
 *     case the paper prints; the others "are done similarly").  The fields
 *     in those rules are the resolved conserved moments of the streamed
 *     populations; their gradients are periodic central differences.  The
 *     local Smagorinsky rates of les = 1 are not applied in this mode.
 *   - les = 3 is the cross-helicity closure of Carati et al. quoted in
 *     Sec. 1.1 (Eqs. CHClosureV/B): nu_t = C_S Delta^2 |S^v_ab S^b_ab|^(1/2),
 *     eta_t = C_S Delta^2 sgn(j . omega) |j . omega|^(1/2), from periodic
 *     central differences of u = (rho u)/rho and B of the streamed
 *     populations; tau_e = tau_nu + 3 nu_t, tau_m = tau_eta + 3 eta_t
 *     (nu = (tau - 1/2)/3, Sec. 4.3).  eta_t < 0 (backscatter) is kept, but
 *     the total resistivity is not allowed below zero: tau_m >= 1/2.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Lattice vectors, Sec. 3 (explicit component lists). */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int MCX[5] = {0, 1, 0, -1, 0};
static const int MCY[5] = {0, 0, 1, 0, -1};

#define NF 9
#define NG 5
#define NPLANE 19

/* Parameter vector passed from the host wrapper (all doubles). */
enum { P_TAU_NU = 0, P_TAU_ETA, P_CS, P_DELTA, P_S5, P_S6, P_S7, P_S8, P_LES, P_COUNT };

static double w9(int i) {
    int c2 = CX[i] * CX[i] + CY[i] * CY[i];
    if (c2 == 0) return 4.0 / 9.0;
    if (c2 == 1) return 1.0 / 9.0;
    return 1.0 / 36.0;
}

static double w5(int k) { return k == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }

/* T of Eq. FluidTMatrix, built from its row formulas. */
static void build_T(double T[NF][NF]) {
    for (int i = 0; i < NF; ++i) {
        double cx = CX[i], cy = CY[i];
        double cx2 = cx * cx, cy2 = cy * cy;
        T[0][i] = 1.0;
        T[1][i] = cx;
        T[2][i] = cy;
        T[3][i] = cx * cy;
        T[4][i] = cx2 - cy2;
        T[5][i] = 3.0 * cx * cy2 - 2.0 * cx;
        T[6][i] = 3.0 * cy * cx2 - 2.0 * cy;
        T[7][i] = 4.0 - 9.0 * (cx2 + cy2 - 2.0 * cx2 * cy2);
        T[8][i] = 4.0 - 4.0 * (cx2 + cy2) + 3.0 * cx2 * cy2;
    }
}

/* T_m of Eq. MagTMatrix, from its row formulas. */
static void build_Tm(double Tm[NG][NG]) {
    for (int k = 0; k < NG; ++k) {
        double cx = MCX[k], cy = MCY[k];
        Tm[0][k] = 1.0;
        Tm[1][k] = cx;
        Tm[2][k] = cy;
        Tm[3][k] = cx * cx;
        Tm[4][k] = cy * cy;
    }
}

/* Gauss-Jordan inverse with partial pivoting; exported for the pins (the
 * step applies the exact orthogonal inverse instead, see orc_collide_cell). */
static int invert(int n, const double* A, double* Ainv) {
    double a[NF][2 * NF];
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < 2 * n; ++c)
            a[r][c] = c < n ? A[r * n + c] : (c - n == r ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int r = col + 1; r < n; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < 2 * n; ++c) {
                double t = a[col][c]; a[col][c] = a[piv][c]; a[piv][c] = t;
            }
        double d = a[col][col];
        for (int c = 0; c < 2 * n; ++c) a[col][c] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == col) continue;
            double m = a[r][col];
            if (m == 0.0) continue;
            for (int c = 0; c < 2 * n; ++c) a[r][c] -= m * a[col][c];
        }
    }
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) Ainv[r * n + c] = a[r][c + n];
    return 0;
}

static double g_T[NF][NF], g_Tinv[NF][NF], g_norm2[NF];
static int g_ready = 0;

static void setup(void) {
    if (g_ready) return;
    build_T(g_T);
    invert(NF, &g_T[0][0], &g_Tinv[0][0]);
    for (int j = 0; j < NF; ++j) {
        g_norm2[j] = 0.0;
        for (int i = 0; i < NF; ++i) g_norm2[j] += g_T[j][i] * g_T[j][i];
    }
    g_ready = 1;
}

/* ---- exported: lattice constants and matrices (for pins) --------------- */

void orc_lattice(int* cx, int* cy, int* mcx, int* mcy, double* w, double* wm) {
    for (int i = 0; i < NF; ++i) { cx[i] = CX[i]; cy[i] = CY[i]; w[i] = w9(i); }
    for (int k = 0; k < NG; ++k) { mcx[k] = MCX[k]; mcy[k] = MCY[k]; wm[k] = w5(k); }
}

void orc_tmatrix(double* T, double* Tinv, double* Tm) {
    setup();
    double tm[NG][NG];
    build_Tm(tm);
    memcpy(T, g_T, sizeof g_T);
    memcpy(Tinv, g_Tinv, sizeof g_Tinv);
    memcpy(Tm, tm, sizeof tm);
}

/* D2Q9 equilibrium, Sec. 3 (f_i^(eq) with the Maxwell-stress term). */
void orc_feq(double rho, double ux, double uy, double bx, double by, double* f) {
    double u2 = ux * ux + uy * uy;
    double b2 = bx * bx + by * by;
    for (int i = 0; i < NF; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        double cb = CX[i] * bx + CY[i] * by;
        double c2 = CX[i] * CX[i] + CY[i] * CY[i];
        double w = w9(i);
        f[i] = w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * u2)
             + 4.5 * w * (0.5 * b2 * c2 - cb * cb);
    }
}

/* D2Q5 vector equilibrium, Sec. 3; g[2k + a]. */
void orc_geq(double ux, double uy, double bx, double by, double* g) {
    double B[2] = {bx, by}, U[2] = {ux, uy};
    for (int k = 0; k < NG; ++k) {
        double Cu = MCX[k] * ux + MCY[k] * uy;
        double CB = MCX[k] * bx + MCY[k] * by;
        for (int a = 0; a < 2; ++a)
            g[2 * k + a] = w5(k) * (B[a] + 3.0 * (Cu * B[a] - CB * U[a]));
    }
}

/* ---- the collision at one node ------------------------------------------
 * z: the 19 streamed (pre-collision) populations of the node.
 * out: the 19 post-collision populations.
 * aux (optional, 4 doubles): tau_nu_eff, tau_m_eff, Q, J.
 */
static void collide_impl(const double* z, const double* p, const double* shift,
                         const double* taus, double* out, double* aux);

void orc_collide_cell(const double* z, const double* p, double* out, double* aux) {
    collide_impl(z, p, NULL, NULL, out, aux);
}

/* As orc_collide_cell, relaxing towards the filtered equilibria shifted by
 * shift = Delta^2 (M3, M4, M7 = M8, N_y1) corrections (les = 2). */
void orc_collide_cell_shift(const double* z, const double* p, const double* shift, double* out) {
    collide_impl(z, p, shift, NULL, out, NULL);
}

/* taus (les = 3, else NULL): the node's relaxation times tau_nu, tau_m
 * from the cross-helicity closure, used instead of the local rates. */
static void collide_impl(const double* z, const double* p, const double* shift,
                         const double* taus, double* out, double* aux) {
    setup();
    const double* f = z;
    const double* g = z + NF;
    double tau_nu = p[P_TAU_NU], tau_eta = p[P_TAU_ETA];
    double CS = p[P_CS], delta = p[P_DELTA];
    int les = p[P_LES] == 1.0;

    /* moments rho, rho u, B (Sec. 3) */
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < NF; ++i) {
        rho += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
    }
    double ux = jx / rho, uy = jy / rho;
    double bx = 0.0, by = 0.0;
    for (int k = 0; k < NG; ++k) { bx += g[2 * k]; by += g[2 * k + 1]; }

    /* M = T f (Eq. Transformation) */
    double M[NF];
    for (int j = 0; j < NF; ++j) {
        M[j] = 0.0;
        for (int i = 0; i < NF; ++i) M[j] += g_T[j][i] * f[i];
    }
    /* equilibrium moments, Eq. KinMomentEq (written in rho and rho u) */
    double Meq[NF];
    Meq[0] = rho;
    Meq[1] = jx;
    Meq[2] = jy;
    Meq[3] = jx * jy / rho - bx * by;
    Meq[4] = (jx * jx - jy * jy) / rho - bx * bx + by * by;
    Meq[5] = -jx;
    Meq[6] = -jy;
    Meq[7] = -3.0 * (jx * jx + jy * jy) / rho;
    Meq[8] = 5.0 / 3.0 * rho - 3.0 * (jx * jx + jy * jy) / rho;
    if (shift) { /* filtered equilibria (les = 2) */
        Meq[3] += shift[0];
        Meq[4] += shift[1];
        Meq[7] += shift[2];
        Meq[8] += shift[2];
    }

    double n[NF];
    for (int j = 0; j < NF; ++j) n[j] = M[j] - Meq[j];

    /* local eddy relaxation times (reading above) */
    double tau_e = tau_nu, tau_m = tau_eta, Q = 0.0, J = 0.0;
    if (les) {
        /* |S| = 3 Q / (2 rho tau_e), Q = sqrt(n_4^2 + 4 n_3^2);
         * tau_e = tau_nu + 3 C_S Delta^2 |S|  =>  quadratic in tau_e */
        Q = sqrt(n[4] * n[4] + 4.0 * n[3] * n[3]);
        tau_e = 0.5 * (tau_nu + sqrt(tau_nu * tau_nu + 18.0 * CS * delta * delta * Q / rho));
        /* N = T_m g (Eq. Transformation), rows C_x and C_y; equilibria of
         * Eq. MagMomentEq with u. |j| = 3 J / tau_m. */
        double Ny1 = 0.0, Nx2 = 0.0;
        for (int k = 0; k < NG; ++k) {
            Ny1 += MCX[k] * g[2 * k + 1];
            Nx2 += MCY[k] * g[2 * k];
        }
        double Ny1eq = ux * by - uy * bx;
        double Nx2eq = uy * bx - ux * by;
        J = fabs((Ny1 - Ny1eq) - (Nx2 - Nx2eq));
        tau_m = 0.5 * (tau_eta + sqrt(tau_eta * tau_eta + 36.0 * CS * delta * delta * J));
    }
    if (taus) { /* les = 3: rates from the resolved gradients */
        tau_e = taus[0];
        tau_m = taus[1];
    }
    double s_nu = 1.0 / tau_e;
    double s[NF];
    s[0] = s[1] = s[2] = 0.0; /* conserved: n_0 = n_1 = n_2 = 0 anyway */
    s[3] = s[4] = s_nu;
    s[5] = p[P_S5] > 0.0 ? p[P_S5] : 1.0 / tau_nu;
    s[6] = p[P_S6] > 0.0 ? p[P_S6] : 1.0 / tau_nu;
    s[7] = p[P_S7] > 0.0 ? p[P_S7] : s_nu;
    s[8] = p[P_S8] > 0.0 ? p[P_S8] : s_nu;

    /* relax in moment space, return with T^-1 (Sec. 3).  The rows of T are
     * mutually orthogonal, so T^-1 = T^t diag(1/|T_j|^2) exactly; each term is
     * divided by the exact integer |T_j|^2 (a numerically inverted T is off
     * by an ulp and biases the populations a little every step). */
    double Ms[NF];
    for (int j = 0; j < NF; ++j) Ms[j] = M[j] - s[j] * n[j];
    for (int i = 0; i < NF; ++i) {
        double acc = 0.0;
        for (int j = 0; j < NF; ++j) acc += g_T[j][i] * Ms[j] / g_norm2[j];
        out[i] = acc;
    }

    /* magnetic SRT collision in distribution space (Eq. LBMagEqn) */
    double geq[2 * NG];
    orc_geq(ux, uy, bx, by, geq);
    if (shift) {
        /* N_y1^eq -> N_y1^eq + D and N_x2^eq -> N_x2^eq - D enter g^eq through
         * its first-moment term 3 w'_k C_kb (u_b B_a - B_b u_a) */
        for (int k = 0; k < NG; ++k) {
            geq[2 * k + 1] += 3.0 * w5(k) * MCX[k] * shift[3];
            geq[2 * k] -= 3.0 * w5(k) * MCY[k] * shift[3];
        }
    }
    double sm = 1.0 / tau_m;
    for (int q = 0; q < 2 * NG; ++q) out[NF + q] = g[q] - sm * (g[q] - geq[q]);

    if (aux) { aux[0] = tau_e; aux[1] = tau_m; aux[2] = Q; aux[3] = J; }
}

/* ---- the paper's kinetic LES (les = 2) ------------------------------------
 * Filter rules of Sec. 2, summed over the direction beta:
 *   product (Eq. FilterExampleSmall):  P(X, Y) = (1/12) dX . dY
 *   ratio   (Eq. FilterExampleLarge):  Rt(X, Y; Z) = 1/(12 Z) [ dX . dY
 *            - (X dZ . dY + Y dZ . dX - X Y dZ . dZ / Z) / Z ]
 * The filtered equilibrium of a term XY (XY/Z) is its value in the filtered
 * fields plus Delta^2 P (Delta^2 Rt).  Applied to Eq. KinMomentEq (linear
 * terms have no correction):
 *   M3: Rt(jx, jy; rho) - P(Bx, By)
 *   M4: Rt(jx, jx; rho) - Rt(jy, jy; rho) - P(Bx, Bx) + P(By, By)
 *   M7 = M8: -3 (Rt(jx, jx; rho) + Rt(jy, jy; rho))
 * and to Eq. MagMomentEq with u (reading above), N_y1^eq = (jx By - jy Bx)/rho
 * = -N_x2^eq:
 *   N_y1: Rt(jx, By; rho) - Rt(jy, Bx; rho),  N_x2 the negative.
 * d[q][a]: derivative of field q (rho, jx, jy, Bx, By) along a (x, y).
 * out: Delta^2 times (M3, M4, M7 (= M8), N_y1) corrections. */
static double dotg(const double d[5][2], int a, int b) {
    return d[a][0] * d[b][0] + d[a][1] * d[b][1];
}

static double rt(double X, double Y, double Z, int ix, int iy, int iz, const double d[5][2]) {
    return (dotg(d, ix, iy) - (X * dotg(d, iz, iy) + Y * dotg(d, iz, ix) - X * Y * dotg(d, iz, iz) / Z) / Z) /
           (12.0 * Z);
}

void orc_kinetic_shift(const double* fld, const double* grad, double delta, double* out) {
    double d[5][2];
    for (int q = 0; q < 5; ++q) { d[q][0] = grad[2 * q]; d[q][1] = grad[2 * q + 1]; }
    double rho = fld[0], jx = fld[1], jy = fld[2], bx = fld[3], by = fld[4];
    double d2 = delta * delta;
    double Rxx = rt(jx, jx, rho, 1, 1, 0, d), Ryy = rt(jy, jy, rho, 2, 2, 0, d);
    double Rxy = rt(jx, jy, rho, 1, 2, 0, d);
    double Pxy = dotg(d, 3, 4) / 12.0, Pxx = dotg(d, 3, 3) / 12.0, Pyy = dotg(d, 4, 4) / 12.0;
    out[0] = d2 * (Rxy - Pxy);
    out[1] = d2 * (Rxx - Ryy - Pxx + Pyy);
    out[2] = d2 * (-3.0 * (Rxx + Ryy));
    out[3] = d2 * (rt(jx, by, rho, 1, 4, 0, d) - rt(jy, bx, rho, 2, 3, 0, d));
}

/* ---- lattice-wide operations --------------------------------------------- */

static long wrap(long a, long n) {
    long r = a % n;
    return r < 0 ? r + n : r;
}

static int plane_cx(int p) { return p < NF ? CX[p] : MCX[(p - NF) / 2]; }
static int plane_cy(int p) { return p < NF ? CY[p] : MCY[(p - NF) / 2]; }

/* Streaming, a pure shift (Sec. 1.2): dst_p(x) = src_p(x - c_p), periodic.
 * nthreads > 1 splits the rows (OpenMP builds only); each value is a copy,
 * so the result does not depend on it. */
static void stream_rows(int nx, int ny, const double* src, double* dst, int nthreads) {
    long N = (long)nx * ny;
    (void)nthreads;
    for (int p = 0; p < NPLANE; ++p) {
        int cx = plane_cx(p), cy = plane_cy(p);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x)
                dst[p * N + y * nx + x] =
                    src[p * N + wrap(y - cy, ny) * nx + wrap(x - cx, nx)];
    }
}

void orc_stream(int nx, int ny, const double* src, double* dst) {
    stream_rows(nx, ny, src, dst, 1);
}

/* Equilibrium initialisation: f = f^eq(rho, u, B), g = g^eq(u, B). */
void orc_init(int nx, int ny, const double* rho, const double* ux, const double* uy,
              const double* bx, const double* by, double* state) {
    long N = (long)nx * ny;
    double f[NF], g[2 * NG];
    for (long c = 0; c < N; ++c) {
        orc_feq(rho[c], ux[c], uy[c], bx[c], by[c], f);
        orc_geq(ux[c], uy[c], bx[c], by[c], g);
        for (int i = 0; i < NF; ++i) state[i * N + c] = f[i];
        for (int q = 0; q < 2 * NG; ++q) state[(NF + q) * N + c] = g[q];
    }
}

/* One or more full time steps: stream, then collide at every node.
 * state (19 planes) is advanced in place; work is a caller buffer of the
 * same size.  nthreads > 1 splits the streaming, moment and collision loops
 * over rows (OpenMP builds only); every node is computed by the same
 * operations whatever the split, so results do not depend on it. */
static void kinetic_collide_all(int nx, int ny, const double* p, const double* work,
                                double* state, int nthreads);

int orc_step(int nx, int ny, const double* p, double* state, double* work, int nsteps,
             int nthreads) {
    setup();
    long N = (long)nx * ny;
    (void)nthreads;
    for (int t = 0; t < nsteps; ++t) {
        stream_rows(nx, ny, state, work, nthreads);
        if (p[P_LES] == 2.0 || p[P_LES] == 3.0) {
            kinetic_collide_all(nx, ny, p, work, state, nthreads);
            continue;
        }
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
        for (long y = 0; y < ny; ++y) {
            double z[NPLANE], o[NPLANE];
            for (long x = 0; x < nx; ++x) {
                long c = y * nx + x;
                for (int q = 0; q < NPLANE; ++q) z[q] = work[q * N + c];
                orc_collide_cell(z, p, o, NULL);
                for (int q = 0; q < NPLANE; ++q) state[q * N + c] = o[q];
            }
        }
    }
    return 0;
}

/* les = 3: relaxation times from the cross-helicity closure, given the
 * fields (rho, jx, jy, Bx, By) at the node and its four neighbours
 * (xp, xm, yp, ym). */
void orc_carati_taus(const double* p, const double* c0, const double* xp, const double* xm,
                     const double* yp, const double* ym, double* taus) {
    double cd2 = p[P_CS] * p[P_DELTA] * p[P_DELTA];
    /* u = j / rho at each point, then central differences */
    double dux_dx = 0.5 * (xp[1] / xp[0] - xm[1] / xm[0]);
    double dux_dy = 0.5 * (yp[1] / yp[0] - ym[1] / ym[0]);
    double duy_dx = 0.5 * (xp[2] / xp[0] - xm[2] / xm[0]);
    double duy_dy = 0.5 * (yp[2] / yp[0] - ym[2] / ym[0]);
    double dbx_dx = 0.5 * (xp[3] - xm[3]), dbx_dy = 0.5 * (yp[3] - ym[3]);
    double dby_dx = 0.5 * (xp[4] - xm[4]), dby_dy = 0.5 * (yp[4] - ym[4]);
    (void)c0;
    /* S_ab = (d_b v_a + d_a v_b) / 2 for v = u and v = B */
    double svxx = dux_dx, svyy = duy_dy, svxy = 0.5 * (dux_dy + duy_dx);
    double sbxx = dbx_dx, sbyy = dby_dy, sbxy = 0.5 * (dbx_dy + dby_dx);
    double ss = svxx * sbxx + svyy * sbyy + 2.0 * svxy * sbxy;
    double nu_t = cd2 * sqrt(fabs(ss));
    double om = duy_dx - dux_dy, jz = dby_dx - dbx_dy;
    double jw = jz * om;
    double eta_t = cd2 * (jw > 0.0 ? 1.0 : (jw < 0.0 ? -1.0 : 0.0)) * sqrt(fabs(jw));
    taus[0] = p[P_TAU_NU] + 3.0 * nu_t;
    taus[1] = p[P_TAU_ETA] + 3.0 * eta_t;
    if (taus[1] < 0.5) taus[1] = 0.5;
}

/* les = 2: conserved moments of the streamed populations, their periodic
 * central differences, the filtered-equilibrium shifts, then the collision.
 * les = 3: the same moments give the cross-helicity closure's rates. */
static void kinetic_collide_all(int nx, int ny, const double* p, const double* work,
                                double* state, int nthreads) {
    long N = (long)nx * ny;
    double* m = (double*)malloc(sizeof(double) * 5 * N);
    (void)nthreads;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
    for (long c = 0; c < N; ++c) {
        double r = 0, jx = 0, jy = 0, bx = 0, by = 0;
        for (int i = 0; i < NF; ++i) {
            double fi = work[i * N + c];
            r += fi; jx += CX[i] * fi; jy += CY[i] * fi;
        }
        for (int k = 0; k < NG; ++k) {
            bx += work[(NF + 2 * k) * N + c];
            by += work[(NF + 2 * k + 1) * N + c];
        }
        m[c] = r; m[N + c] = jx; m[2 * N + c] = jy; m[3 * N + c] = bx; m[4 * N + c] = by;
    }
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x) {
            long c = y * nx + x;
            long xp = y * nx + wrap(x + 1, nx), xm = y * nx + wrap(x - 1, nx);
            long yp = wrap(y + 1, ny) * nx + x, ym = wrap(y - 1, ny) * nx + x;
            double fld[5], grad[10], z[NPLANE], o[NPLANE], sh[4];
            for (int q = 0; q < 5; ++q) {
                fld[q] = m[q * N + c];
                grad[2 * q] = 0.5 * (m[q * N + xp] - m[q * N + xm]);
                grad[2 * q + 1] = 0.5 * (m[q * N + yp] - m[q * N + ym]);
            }
            for (int q = 0; q < NPLANE; ++q) z[q] = work[q * N + c];
            if (p[P_LES] == 2.0) {
                orc_kinetic_shift(fld, grad, p[P_DELTA], sh);
                collide_impl(z, p, sh, NULL, o, NULL);
            } else {
                double a0[5], axp[5], axm[5], ayp[5], aym[5], taus[2];
                for (int q = 0; q < 5; ++q) {
                    a0[q] = m[q * N + c];
                    axp[q] = m[q * N + xp]; axm[q] = m[q * N + xm];
                    ayp[q] = m[q * N + yp]; aym[q] = m[q * N + ym];
                }
                orc_carati_taus(p, a0, axp, axm, ayp, aym, taus);
                collide_impl(z, p, NULL, taus, o, NULL);
            }
            for (int q = 0; q < NPLANE; ++q) state[q * N + c] = o[q];
        }
    free(m);
}

/* One step evaluated at selected nodes only: out[c*19 + q] is the
 * post-collision population q at node idx[c] after streaming from state. */
/* Conserved moments (rho, jx, jy, Bx, By) of the populations streamed into
 * node (x, y). */
static void streamed_moments(int nx, int ny, const double* state, long x, long y, double* m) {
    long N = (long)nx * ny;
    x = wrap(x, nx);
    y = wrap(y, ny);
    for (int q = 0; q < 5; ++q) m[q] = 0.0;
    for (int p = 0; p < NPLANE; ++p) {
        double v = state[p * N + wrap(y - plane_cy(p), ny) * nx + wrap(x - plane_cx(p), nx)];
        if (p < NF) { m[0] += v; m[1] += CX[p] * v; m[2] += CY[p] * v; }
        else if ((p - NF) % 2 == 0) m[3] += v;
        else m[4] += v;
    }
}

void orc_step_cells(int nx, int ny, const double* p, const double* state, long ncells,
                    const long* idx, double* out) {
    setup();
    long N = (long)nx * ny;
    for (long c = 0; c < ncells; ++c) {
        long x = idx[c] % nx, y = idx[c] / nx;
        double z[NPLANE];
        for (int q = 0; q < NPLANE; ++q)
            z[q] = state[q * N + wrap(y - plane_cy(q), ny) * nx + wrap(x - plane_cx(q), nx)];
        if (p[P_LES] == 3.0) {
            double m0[5], mxp[5], mxm[5], myp[5], mym[5], taus[2];
            streamed_moments(nx, ny, state, x, y, m0);
            streamed_moments(nx, ny, state, x + 1, y, mxp);
            streamed_moments(nx, ny, state, x - 1, y, mxm);
            streamed_moments(nx, ny, state, x, y + 1, myp);
            streamed_moments(nx, ny, state, x, y - 1, mym);
            orc_carati_taus(p, m0, mxp, mxm, myp, mym, taus);
            collide_impl(z, p, NULL, taus, out + c * NPLANE, NULL);
        } else if (p[P_LES] == 2.0) {
            double m0[5], mxp[5], mxm[5], myp[5], mym[5], grad[10], sh[4];
            streamed_moments(nx, ny, state, x, y, m0);
            streamed_moments(nx, ny, state, x + 1, y, mxp);
            streamed_moments(nx, ny, state, x - 1, y, mxm);
            streamed_moments(nx, ny, state, x, y + 1, myp);
            streamed_moments(nx, ny, state, x, y - 1, mym);
            for (int q = 0; q < 5; ++q) {
                grad[2 * q] = 0.5 * (mxp[q] - mxm[q]);
                grad[2 * q + 1] = 0.5 * (myp[q] - mym[q]);
            }
            orc_kinetic_shift(m0, grad, p[P_DELTA], sh);
            collide_impl(z, p, sh, NULL, out + c * NPLANE, NULL);
        } else {
            orc_collide_cell(z, p, out + c * NPLANE, NULL);
        }
    }
}

/* Per-node local LES quantities after streaming (tau_e, tau_m, Q, J). */
void orc_les_fields(int nx, int ny, const double* p, const double* state, double* aux) {
    setup();
    long N = (long)nx * ny;
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x) {
            double z[NPLANE], o[NPLANE], a[4];
            for (int q = 0; q < NPLANE; ++q)
                z[q] = state[q * N + wrap(y - plane_cy(q), ny) * nx + wrap(x - plane_cx(q), nx)];
            orc_collide_cell(z, p, o, a);
            for (int r = 0; r < 4; ++r) aux[r * N + y * nx + x] = a[r];
        }
}

/* Moments of a stored state: rho, u, B at every node (Sec. 3). The
 * collision conserves them, so they are those of the streamed populations
 * of the step that produced the state. */
void orc_moments(int nx, int ny, const double* state, double* rho, double* ux, double* uy,
                 double* bx, double* by) {
    long N = (long)nx * ny;
    for (long c = 0; c < N; ++c) {
        double r = 0.0, jx = 0.0, jy = 0.0, Bx = 0.0, By = 0.0;
        for (int i = 0; i < NF; ++i) {
            double fi = state[i * N + c];
            r += fi; jx += CX[i] * fi; jy += CY[i] * fi;
        }
        for (int k = 0; k < NG; ++k) {
            Bx += state[(NF + 2 * k) * N + c];
            By += state[(NF + 2 * k + 1) * N + c];
        }
        rho[c] = r; ux[c] = jx / r; uy[c] = jy / r; bx[c] = Bx; by[c] = By;
    }
}

/* Diagnostics.  out[0..11]:
 *  0 mass = sum rho            1,2 sum rho u_x, sum rho u_y
 *  3,4 sum B_x, sum B_y        5 E_K = <rho |u|^2>/2       6 E_M = <|B|^2>/2
 *  7 enstrophy <omega^2>/2     8 cross helicity <u.B>
 *  9 max |div B|               10 rms div B                11 <j_z^2>/2
 * <.> is the mean over nodes; omega, j_z and div B use periodic central
 * differences (the discrete operator under which the paper's div B = 0
 * statement is checked). */
void orc_diagnostics(int nx, int ny, const double* state, double* out) {
    long N = (long)nx * ny;
    double* rho = (double*)malloc(sizeof(double) * N * 5);
    double *ux = rho + N, *uy = rho + 2 * N, *bx = rho + 3 * N, *by = rho + 4 * N;
    orc_moments(nx, ny, state, rho, ux, uy, bx, by);
    double s[12];
    for (int r = 0; r < 12; ++r) s[r] = 0.0;
    double dmax = 0.0;
    for (long y = 0; y < ny; ++y)
        for (long x = 0; x < nx; ++x) {
            long c = y * nx + x;
            long xp = y * nx + wrap(x + 1, nx), xm = y * nx + wrap(x - 1, nx);
            long yp = wrap(y + 1, ny) * nx + x, ym = wrap(y - 1, ny) * nx + x;
            s[0] += rho[c];
            s[1] += rho[c] * ux[c];
            s[2] += rho[c] * uy[c];
            s[3] += bx[c];
            s[4] += by[c];
            s[5] += rho[c] * (ux[c] * ux[c] + uy[c] * uy[c]);
            s[6] += bx[c] * bx[c] + by[c] * by[c];
            double om = 0.5 * (uy[xp] - uy[xm]) - 0.5 * (ux[yp] - ux[ym]);
            s[7] += om * om;
            s[8] += ux[c] * bx[c] + uy[c] * by[c];
            double dv = 0.5 * (bx[xp] - bx[xm]) + 0.5 * (by[yp] - by[ym]);
            if (fabs(dv) > dmax) dmax = fabs(dv);
            s[10] += dv * dv;
            double jz = 0.5 * (by[xp] - by[xm]) - 0.5 * (bx[yp] - bx[ym]);
            s[11] += jz * jz;
        }
    double inv = 1.0 / (double)N;
    out[0] = s[0];
    out[1] = s[1];
    out[2] = s[2];
    out[3] = s[3];
    out[4] = s[4];
    out[5] = 0.5 * s[5] * inv;
    out[6] = 0.5 * s[6] * inv;
    out[7] = 0.5 * s[7] * inv;
    out[8] = s[8] * inv;
    out[9] = dmax;
    out[10] = sqrt(s[10] * inv);
    out[11] = 0.5 * s[11] * inv;
    free(rho);
}

/* ---- independent routes used only by pins --------------------------------- */

/* Plain BGK step in distribution space (Sec. 1.2), f and g with their own
 * single relaxation times and no LES: the special case the MRT step must
 * reduce to when every rate is tied (Sec. 4.3). */
int orc_step_bgk(int nx, int ny, double tau_nu, double tau_eta, double* state, double* work,
                 int nsteps) {
    long N = (long)nx * ny;
    for (int t = 0; t < nsteps; ++t) {
        orc_stream(nx, ny, state, work);
        for (long c = 0; c < N; ++c) {
            double f[NF], g[2 * NG], feq[NF], geq[2 * NG];
            for (int i = 0; i < NF; ++i) f[i] = work[i * N + c];
            for (int q = 0; q < 2 * NG; ++q) g[q] = work[(NF + q) * N + c];
            double rho = 0, jx = 0, jy = 0, bx = 0, by = 0;
            for (int i = 0; i < NF; ++i) { rho += f[i]; jx += CX[i] * f[i]; jy += CY[i] * f[i]; }
            for (int k = 0; k < NG; ++k) { bx += g[2 * k]; by += g[2 * k + 1]; }
            orc_feq(rho, jx / rho, jy / rho, bx, by, feq);
            orc_geq(jx / rho, jy / rho, bx, by, geq);
            for (int i = 0; i < NF; ++i) state[i * N + c] = f[i] - (f[i] - feq[i]) / tau_nu;
            for (int q = 0; q < 2 * NG; ++q)
                state[(NF + q) * N + c] = g[q] - (g[q] - geq[q]) / tau_eta;
        }
    }
    return 0;
}
