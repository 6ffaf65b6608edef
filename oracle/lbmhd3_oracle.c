/*
 * lbmhd3_oracle.c -- plain, slow, FP64 CPU oracle for the 3D extension of
 * the lattice Boltzmann MHD step of Flint & Vahala (arXiv:1607.08675).
 *
 * TEST INFRASTRUCTURE ONLY.  The independent reference the CUDA 3D path is
 * checked against; only the test suite, the package smoke check and the
 * CPU-baseline leg of the benchmark may build, load or call it.  It shares
 * no code, header, table or helper with the CUDA library (nor with the 2D
 * oracle).  Scalar loops, IEEE double, compiled with -ffp-contract=off.
 *
 * The paper works in 2D and states that the model extends to 3D with more
 * lattice velocities (Sec. 3 opening; the Conclusion names D3Q27).  The
 * readings taken for that extension:
 *   - Density lattice D3Q27, c in {-1, 0, 1}^3, weights the tensor product
 *     of the 1D weights {2/3, 1/6, 1/6} (the D2Q9 weights 4/9, 1/9, 1/36 are
 *     the same product in 2D).
 *   - Density equilibrium: the paper's D2Q9 expression (Sec. 3) with 3D
 *     vectors, w rho [1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u^2] + 9/2 w [1/2 B^2 c^2
 *     - (B.c)^2 - B^2/6].  The last term, the trace of 1/2 B^2 I - B B over
 *     3, is zero in 2D (so the 2D equilibrium is unchanged) and is what keeps
 *     mass conserved and gives the Maxwell stress 1/2 B^2 I - B B in 3D.
 *   - Magnetic lattice D3Q7 (rest, +-x, +-y, +-z) with the paper's D2Q5
 *     equilibrium w'_k [B + 3((C_k.u) B - (C_k.B) u)]; the factor 3 with
 *     sum_k w'_k C_k C_k = I/3 fixes w' = 1/6 on the six axes and 0 at rest,
 *     so the rest population stays zero and is not stored (six vector
 *     populations).  In a flow independent of z the +-z pair plays the
 *     D2Q5 rest population (weight 2/6 = 1/3).
 *   - Collision: the single relaxation (BGK) form, i.e. the paper's MRT
 *     with every non-conserved rate tied to s_nu (equal to BGK in 2D),
 *     f <- f - (f - f^eq)/tau_e; magnetic g <- g - (g - g^eq)/tau_m.
 *   - Local LES rates (les = 1) as in 2D: Q = sqrt(2 P:P) with P the
 *     traceless part of the non-equilibrium stress sum_i (f_i - f_i^eq) c c
 *     (in 2D exactly sqrt(n4^2 + 4 n3^2)); J = |a|, a the axial vector of
 *     the antisymmetric part of the non-equilibrium first moment
 *     N_ab = sum_k C_ka (g_kb - g_kb^eq) (in 2D |N_y1 - N_x2 - 2E|);
 *     tau_e = (tau_nu + sqrt(tau_nu^2 + 18 C_S Delta^2 Q / rho)) / 2,
 *     tau_m = (tau_eta + sqrt(tau_eta^2 + 36 C_S Delta^2 J)) / 2.
 *   - The paper's kinetic LES (les = 2, Sec. 4.1) in this BGK form: relax
 *     towards the filtered equilibria f^eq + Delta^2 f^(Delta),
 *     g^eq + Delta^2 g^(Delta), the corrections obtained by applying the
 *     product rule P(X, Y) = dX . dY / 12 (Eq. FilterExampleSmall) and the
 *     ratio rule Rt(X, Y; rho) (Eq. FilterExampleLarge) to every nonlinear
 *     term of the equilibria: (c.j)^2/rho -> sum_ab c_a c_b Rt(j_a, j_b),
 *     |j|^2/rho -> sum_a Rt(j_a, j_a), |B|^2 -> sum_a P(B_a, B_a),
 *     (c.B)^2 -> sum_ab c_a c_b P(B_a, B_b), j_a B_b/rho -> Rt(j_a, B_b).
 *     The fields are the conserved moments of the streamed populations,
 *     their gradients periodic central differences (as in 2D).  In 2D these
 *     are the moment-table corrections the 2D oracle applies (M_3, M_4,
 *     M_7 = M_8, N_y1); with every rate tied the 2D MRT relaxes towards the
 *     same shifted distribution.
 *   - The cross-helicity closure (les = 3, Eqs. CHClosureV/B) with 3D
 *     vectors: nu_t = C_S Delta^2 |S^v : S^b|^(1/2), eta_t = C_S Delta^2
 *     sgn(j . omega) |j . omega|^(1/2), omega = curl u, j = curl B, from the
 *     same central differences of u = j/rho and B; tau_e = tau_nu + 3 nu_t,
 *     tau_m = max(tau_eta + 3 eta_t, 1/2).
 *
 * State: 45 planes of nx*ny*nz doubles, plane p at offset p*N, node
 * (x, y, z) at (z*ny + y)*nx + x.  Planes 0..26: f_i with i = 9 kz + 3 ky + kx,
 * c = (v[kx], v[ky], v[kz]), v = {0, 1, -1}.  Plane 27 + 3q + a: component a
 * (x, y, z) of g_q, q = 0..5 for C = +x, -x, +y, -y, +z, -z.  The stored
 * state is post-collision; a step pulls from x - c, then collides.
 * Parameter vector p: tau_nu, tau_eta, C_S, Delta, les (0, 1, 2 or 3).
 */
#include <math.h>
#include <stdlib.h>

#define NQ 27
#define NM 6
#define NP3 (NQ + 3 * NM)

static const int V1[3] = {0, 1, -1};
static const double W1[3] = {2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0};
static const int CM[NM][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};

static void cvec(int i, int c[3]) {
    c[0] = V1[i % 3];
    c[1] = V1[(i / 3) % 3];
    c[2] = V1[i / 9];
}

static double wq(int i) { return W1[i % 3] * W1[(i / 3) % 3] * W1[i / 9]; }

static double wm(int q) {
    (void)q;
    return 1.0 / 6.0;
}

/* ---- exported: lattice constants (for pins) ---------------------------- */

void orc3_lattice(int* c, double* w, int* cm, double* wmag) {
    for (int i = 0; i < NQ; ++i) {
        int v[3];
        cvec(i, v);
        for (int a = 0; a < 3; ++a) c[3 * i + a] = v[a];
        w[i] = wq(i);
    }
    for (int q = 0; q < NM; ++q) {
        for (int a = 0; a < 3; ++a) cm[3 * q + a] = CM[q][a];
        wmag[q] = wm(q);
    }
}

/* Density equilibrium (the paper's D2Q9 form with 3D vectors and the 3D
 * trace term, see the header). */
void orc3_feq(double rho, const double* u, const double* B, double* f) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    double BB = B[0] * B[0] + B[1] * B[1] + B[2] * B[2];
    for (int i = 0; i < NQ; ++i) {
        int c[3];
        cvec(i, c);
        double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
        double cB = c[0] * B[0] + c[1] * B[1] + c[2] * B[2];
        double cc = (double)(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        double w = wq(i);
        f[i] = w * rho * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu) +
               4.5 * w * (0.5 * BB * cc - cB * cB - BB / 6.0);
    }
}

/* Magnetic equilibrium (the paper's D2Q5 form on the six D3Q7 axes):
 * g[3q + a] = w'_q [B_a + 3((C_q.u) B_a - (C_q.B) u_a)]. */
void orc3_geq(const double* u, const double* B, double* g) {
    for (int q = 0; q < NM; ++q) {
        double Cu = CM[q][0] * u[0] + CM[q][1] * u[1] + CM[q][2] * u[2];
        double CB = CM[q][0] * B[0] + CM[q][1] * B[1] + CM[q][2] * B[2];
        for (int a = 0; a < 3; ++a) g[3 * q + a] = wm(q) * (B[a] + 3.0 * (Cu * B[a] - CB * u[a]));
    }
}

static void collide3_impl(const double* z, const double* p, const double* fsh, const double* gsh,
                          const double* taus, double* out, double* aux);

/* One node: z = the 45 pulled populations; out = post-collision.
 * aux (optional, 4 doubles): tau_e, tau_m, Q, J. */
void orc3_collide_cell(const double* z, const double* p, double* out, double* aux) {
    collide3_impl(z, p, NULL, NULL, NULL, out, aux);
}

/* fsh (27) / gsh (18): Delta^2 corrections of the equilibria (les = 2) or
 * NULL; taus (2): relaxation times replacing tau_nu, tau_eta (les = 3) or
 * NULL. */
static void collide3_impl(const double* z, const double* p, const double* fsh, const double* gsh,
                          const double* taus, double* out, double* aux) {
    const double* f = z;
    const double* g = z + NQ;
    double tau_nu = p[0], tau_eta = p[1], CS = p[2], delta = p[3];
    int les = p[4] == 1.0;
    /* moments: rho, rho u, B */
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < NQ; ++i) {
        int c[3];
        cvec(i, c);
        rho += f[i];
        for (int a = 0; a < 3; ++a) j[a] += c[a] * f[i];
    }
    for (int q = 0; q < NM; ++q)
        for (int a = 0; a < 3; ++a) B[a] += g[3 * q + a];
    double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    double feq[NQ], geq[3 * NM];
    orc3_feq(rho, u, B, feq);
    orc3_geq(u, B, geq);
    if (fsh)
        for (int i = 0; i < NQ; ++i) feq[i] += fsh[i];
    if (gsh)
        for (int k = 0; k < 3 * NM; ++k) geq[k] += gsh[k];
    /* non-equilibrium stress and its traceless part */
    double P[3][3] = {{0.0}};
    for (int i = 0; i < NQ; ++i) {
        int c[3];
        cvec(i, c);
        double fn = f[i] - feq[i];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) P[a][b] += fn * c[a] * c[b];
    }
    double tr = (P[0][0] + P[1][1] + P[2][2]) / 3.0;
    for (int a = 0; a < 3; ++a) P[a][a] -= tr;
    double PP = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) PP += P[a][b] * P[a][b];
    double Q = sqrt(2.0 * PP);
    /* non-equilibrium first moment of g and its axial vector */
    double N[3][3] = {{0.0}};
    for (int q = 0; q < NM; ++q)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) N[a][b] += CM[q][a] * (g[3 * q + b] - geq[3 * q + b]);
    double ax = N[1][2] - N[2][1], ay = N[2][0] - N[0][2], az = N[0][1] - N[1][0];
    double J = sqrt(ax * ax + ay * ay + az * az);
    double tau_e = tau_nu, tau_m = tau_eta;
    if (taus) {
        tau_e = taus[0];
        tau_m = taus[1];
    } else if (les) {
        tau_e = 0.5 * (tau_nu + sqrt(tau_nu * tau_nu + 18.0 * CS * delta * delta * Q / rho));
        tau_m = 0.5 * (tau_eta + sqrt(tau_eta * tau_eta + 36.0 * CS * delta * delta * J));
    }
    for (int i = 0; i < NQ; ++i) out[i] = f[i] - (f[i] - feq[i]) / tau_e;
    for (int k = 0; k < 3 * NM; ++k) out[NQ + k] = g[k] - (g[k] - geq[k]) / tau_m;
    if (aux) {
        aux[0] = tau_e;
        aux[1] = tau_m;
        aux[2] = Q;
        aux[3] = J;
    }
}

/* ---- gradient closures (les = 2, 3) --------------------------------------
 * fld: rho, jx, jy, jz, Bx, By, Bz at the node; grad[3 q + g]: derivative of
 * field q along axis g (periodic central differences). */

static double dot3(const double* grad, int a, int b) {
    return grad[3 * a] * grad[3 * b] + grad[3 * a + 1] * grad[3 * b + 1] +
           grad[3 * a + 2] * grad[3 * b + 2];
}

/* product rule (Eq. FilterExampleSmall) without the Delta^2 */
static double pr3(const double* grad, int a, int b) { return dot3(grad, a, b) / 12.0; }

/* ratio rule (Eq. FilterExampleLarge) for X Y / rho, fields a, b */
static double rt3(const double* fld, const double* grad, int a, int b) {
    double X = fld[a], Y = fld[b], Z = fld[0];
    return (dot3(grad, a, b) - (X * dot3(grad, 0, b) + Y * dot3(grad, 0, a) -
                                X * Y * dot3(grad, 0, 0) / Z) / Z) / (12.0 * Z);
}

/* Delta^2 corrections of the equilibria (les = 2, see the header). */
void orc3_kinetic_shift(const double* fld, const double* grad, double delta, double* fsh,
                        double* gsh) {
    double d2 = delta * delta;
    double R[3][3], P[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            R[a][b] = rt3(fld, grad, 1 + a, 1 + b);
            P[a][b] = pr3(grad, 4 + a, 4 + b);
        }
    double trR = R[0][0] + R[1][1] + R[2][2], trP = P[0][0] + P[1][1] + P[2][2];
    for (int i = 0; i < NQ; ++i) {
        int c[3];
        cvec(i, c);
        double cRc = 0.0, cPc = 0.0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                cRc += c[a] * c[b] * R[a][b];
                cPc += c[a] * c[b] * P[a][b];
            }
        double cc = (double)(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        /* the nonlinear terms of orc3_feq, each replaced by its correction */
        fsh[i] = d2 * wq(i) * (4.5 * cRc - 1.5 * trR + 4.5 * (0.5 * trP * cc - cPc - trP / 6.0));
    }
    for (int q = 0; q < NM; ++q) {
        int a = q / 2;
        double sg = q % 2 ? -1.0 : 1.0;
        /* (C.u) B_b - (C.B) u_b = sg (j_a B_b - B_a j_b) / rho */
        for (int b = 0; b < 3; ++b)
            gsh[3 * q + b] = d2 * wm(q) * 3.0 * sg *
                             (rt3(fld, grad, 1 + a, 4 + b) - rt3(fld, grad, 1 + b, 4 + a));
    }
}

/* Relaxation times of the cross-helicity closure (les = 3) from the fields
 * at the six neighbours: f6[6][7] for x+, x-, y+, y-, z+, z-. */
void orc3_carati_taus(const double* p, const double* f6, double* taus) {
    double cd2 = p[2] * p[3] * p[3];
    double gu[3][3], gb[3][3]; /* g[a][c] = d_c v_a */
    for (int c = 0; c < 3; ++c) {
        const double* fp = f6 + 7 * (2 * c);
        const double* fm = f6 + 7 * (2 * c + 1);
        for (int a = 0; a < 3; ++a) {
            gu[a][c] = 0.5 * (fp[1 + a] / fp[0] - fm[1 + a] / fm[0]);
            gb[a][c] = 0.5 * (fp[4 + a] - fm[4 + a]);
        }
    }
    double ss = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            ss += 0.5 * (gu[a][b] + gu[b][a]) * 0.5 * (gb[a][b] + gb[b][a]);
    double nu_t = cd2 * sqrt(fabs(ss));
    double om[3] = {gu[2][1] - gu[1][2], gu[0][2] - gu[2][0], gu[1][0] - gu[0][1]};
    double jc[3] = {gb[2][1] - gb[1][2], gb[0][2] - gb[2][0], gb[1][0] - gb[0][1]};
    double jw = jc[0] * om[0] + jc[1] * om[1] + jc[2] * om[2];
    double eta_t = cd2 * (jw > 0.0 ? 1.0 : (jw < 0.0 ? -1.0 : 0.0)) * sqrt(fabs(jw));
    taus[0] = p[0] + 3.0 * nu_t;
    taus[1] = p[1] + 3.0 * eta_t;
    if (taus[1] < 0.5) taus[1] = 0.5;
}

/* ---- lattice-wide operations --------------------------------------------- */

static long wrap3(long a, long n) {
    long r = a % n;
    return r < 0 ? r + n : r;
}

static void plane_c(int p, int c[3]) {
    if (p < NQ) {
        cvec(p, c);
    } else {
        int q = (p - NQ) / 3;
        for (int a = 0; a < 3; ++a) c[a] = CM[q][a];
    }
}

/* Streaming, a pure shift: dst_p(x) = src_p(x - c_p), periodic. */
void orc3_stream(int nx, int ny, int nz, const double* src, double* dst) {
    long N = (long)nx * ny * nz;
    for (int p = 0; p < NP3; ++p) {
        int c[3];
        plane_c(p, c);
        for (long z = 0; z < nz; ++z)
            for (long y = 0; y < ny; ++y)
                for (long x = 0; x < nx; ++x)
                    dst[p * N + (z * ny + y) * nx + x] =
                        src[p * N + (wrap3(z - c[2], nz) * ny + wrap3(y - c[1], ny)) * nx +
                            wrap3(x - c[0], nx)];
    }
}

/* Equilibrium initialisation from seven fields of N doubles. */
void orc3_init(int nx, int ny, int nz, const double* rho, const double* ux, const double* uy,
               const double* uz, const double* bx, const double* by, const double* bz,
               double* state) {
    long N = (long)nx * ny * nz;
    for (long n = 0; n < N; ++n) {
        double u[3] = {ux[n], uy[n], uz[n]}, B[3] = {bx[n], by[n], bz[n]};
        double f[NQ], g[3 * NM];
        orc3_feq(rho[n], u, B, f);
        orc3_geq(u, B, g);
        for (int i = 0; i < NQ; ++i) state[i * N + n] = f[i];
        for (int k = 0; k < 3 * NM; ++k) state[(NQ + k) * N + n] = g[k];
    }
}

/* nsteps full steps in place (work: a caller buffer of the same size).
 * nthreads > 1 splits the collision over z planes (OpenMP builds only); the
 * bits do not depend on it. */
static void kinetic3_collide_all(int nx, int ny, int nz, const double* p, const double* work,
                                 double* state, int nthreads);

int orc3_step(int nx, int ny, int nz, const double* p, double* state, double* work, int nsteps,
              int nthreads) {
    long N = (long)nx * ny * nz;
    (void)nthreads;
    for (int t = 0; t < nsteps; ++t) {
        orc3_stream(nx, ny, nz, state, work);
        if (p[4] == 2.0 || p[4] == 3.0) {
            kinetic3_collide_all(nx, ny, nz, p, work, state, nthreads);
            continue;
        }
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
        for (long z = 0; z < nz; ++z) {
            double zz[NP3], o[NP3];
            for (long n = z * nx * ny; n < (z + 1) * nx * ny; ++n) {
                for (int q = 0; q < NP3; ++q) zz[q] = work[q * N + n];
                orc3_collide_cell(zz, p, o, NULL);
                for (int q = 0; q < NP3; ++q) state[q * N + n] = o[q];
            }
        }
    }
    return 0;
}

/* rho, j (3), B (3) of the populations streamed into every node (7 planes). */
static void streamed_fields3(long N, const double* work, double* m) {
    for (long n = 0; n < N; ++n) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < NQ; ++i) {
            int c[3];
            cvec(i, c);
            double fi = work[i * N + n];
            r += fi;
            for (int a = 0; a < 3; ++a) j[a] += c[a] * fi;
        }
        for (int q = 0; q < NM; ++q)
            for (int a = 0; a < 3; ++a) B[a] += work[(NQ + 3 * q + a) * N + n];
        m[n] = r;
        for (int a = 0; a < 3; ++a) {
            m[(1 + a) * N + n] = j[a];
            m[(4 + a) * N + n] = B[a];
        }
    }
}

/* les = 2, 3: the fields of the streamed populations, their central
 * differences, then the filtered-equilibrium collision or the closure's
 * relaxation times, node by node. */
static void kinetic3_collide_all(int nx, int ny, int nz, const double* p, const double* work,
                                 double* state, int nthreads) {
    long N = (long)nx * ny * nz;
    double* m = (double*)malloc(sizeof(double) * 7 * N);
    (void)nthreads;
    streamed_fields3(N, work, m);
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads > 0 ? nthreads : 1) schedule(static)
#endif
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long n = (z * ny + y) * nx + x;
                long nb[6] = {(z * ny + y) * nx + wrap3(x + 1, nx), (z * ny + y) * nx + wrap3(x - 1, nx),
                              (z * ny + wrap3(y + 1, ny)) * nx + x, (z * ny + wrap3(y - 1, ny)) * nx + x,
                              (wrap3(z + 1, nz) * ny + y) * nx + x, (wrap3(z - 1, nz) * ny + y) * nx + x};
                double zz[NP3], o[NP3], fld[7], grad[21];
                for (int q = 0; q < 7; ++q) {
                    fld[q] = m[q * N + n];
                    for (int g = 0; g < 3; ++g)
                        grad[3 * q + g] = 0.5 * (m[q * N + nb[2 * g]] - m[q * N + nb[2 * g + 1]]);
                }
                for (int q = 0; q < NP3; ++q) zz[q] = work[q * N + n];
                if (p[4] == 2.0) {
                    double fsh[NQ], gsh[3 * NM];
                    orc3_kinetic_shift(fld, grad, p[3], fsh, gsh);
                    collide3_impl(zz, p, fsh, gsh, NULL, o, NULL);
                } else {
                    double f6[42], taus[2];
                    for (int k = 0; k < 6; ++k)
                        for (int q = 0; q < 7; ++q) f6[7 * k + q] = m[q * N + nb[k]];
                    orc3_carati_taus(p, f6, taus);
                    collide3_impl(zz, p, NULL, NULL, taus, o, NULL);
                }
                for (int q = 0; q < NP3; ++q) state[q * N + n] = o[q];
            }
    free(m);
}

/* The 45 populations streamed into node (x, y, z) (periodic). */
static void pulled3(int nx, int ny, int nz, const double* state, long x, long y, long z,
                    double* zz) {
    long N = (long)nx * ny * nz;
    x = wrap3(x, nx);
    y = wrap3(y, ny);
    z = wrap3(z, nz);
    for (int q = 0; q < NP3; ++q) {
        int cv[3];
        plane_c(q, cv);
        zz[q] = state[q * N + (wrap3(z - cv[2], nz) * ny + wrap3(y - cv[1], ny)) * nx +
                      wrap3(x - cv[0], nx)];
    }
}

/* rho, j (3), B (3) of 45 pulled populations. */
static void fields_of(const double* zz, double* m) {
    for (int q = 0; q < 7; ++q) m[q] = 0.0;
    for (int i = 0; i < NQ; ++i) {
        int c[3];
        cvec(i, c);
        m[0] += zz[i];
        for (int a = 0; a < 3; ++a) m[1 + a] += c[a] * zz[i];
    }
    for (int q = 0; q < NM; ++q)
        for (int a = 0; a < 3; ++a) m[4 + a] += zz[NQ + 3 * q + a];
}

/* One step at selected nodes only: out[c * 45 + q] = post-collision
 * population q at node idx[c] after streaming from state. */
void orc3_step_cells(int nx, int ny, int nz, const double* p, const double* state, long ncells,
                     const long* idx, double* out) {
    static const int NB[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    for (long c = 0; c < ncells; ++c) {
        long n = idx[c];
        long x = n % nx, y = (n / nx) % ny, z = n / ((long)nx * ny);
        double zz[NP3];
        pulled3(nx, ny, nz, state, x, y, z, zz);
        if (p[4] == 2.0 || p[4] == 3.0) {
            double f6[42], fld[7], grad[21], nb[NP3];
            fields_of(zz, fld);
            for (int k = 0; k < 6; ++k) {
                pulled3(nx, ny, nz, state, x + NB[k][0], y + NB[k][1], z + NB[k][2], nb);
                fields_of(nb, f6 + 7 * k);
            }
            for (int q = 0; q < 7; ++q)
                for (int g = 0; g < 3; ++g)
                    grad[3 * q + g] = 0.5 * (f6[7 * (2 * g) + q] - f6[7 * (2 * g + 1) + q]);
            if (p[4] == 2.0) {
                double fsh[NQ], gsh[3 * NM];
                orc3_kinetic_shift(fld, grad, p[3], fsh, gsh);
                collide3_impl(zz, p, fsh, gsh, NULL, out + c * NP3, NULL);
            } else {
                double taus[2];
                orc3_carati_taus(p, f6, taus);
                collide3_impl(zz, p, NULL, NULL, taus, out + c * NP3, NULL);
            }
        } else {
            orc3_collide_cell(zz, p, out + c * NP3, NULL);
        }
    }
}

/* rho, u (3), B (3) of a state into out (7 planes of N). */
void orc3_moments(int nx, int ny, int nz, const double* state, double* out) {
    long N = (long)nx * ny * nz;
    for (long n = 0; n < N; ++n) {
        double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < NQ; ++i) {
            int c[3];
            cvec(i, c);
            double fi = state[i * N + n];
            rho += fi;
            for (int a = 0; a < 3; ++a) j[a] += c[a] * fi;
        }
        for (int q = 0; q < NM; ++q)
            for (int a = 0; a < 3; ++a) B[a] += state[(NQ + 3 * q + a) * N + n];
        out[n] = rho;
        for (int a = 0; a < 3; ++a) {
            out[(1 + a) * N + n] = j[a] / rho;
            out[(4 + a) * N + n] = B[a];
        }
    }
}

/* Diagnostics of a state, in row-major node order: out = mass, momentum
 * (3), sum of B (3), E_K = <rho |u|^2>/2, E_M = <|B|^2>/2, cross helicity
 * <u.B>, max and rms of the central-difference div B (periodic). */
void orc3_diagnostics(int nx, int ny, int nz, const double* state, double* out) {
    long N = (long)nx * ny * nz;
    double* m = (double*)malloc(sizeof(double) * 7 * N);
    orc3_moments(nx, ny, nz, state, m);
    for (int k = 0; k < 12; ++k) out[k] = 0.0;
    double dmax = 0.0, d2 = 0.0;
    for (long z = 0; z < nz; ++z)
        for (long y = 0; y < ny; ++y)
            for (long x = 0; x < nx; ++x) {
                long n = (z * ny + y) * nx + x;
                double rho = m[n], u[3], B[3];
                for (int a = 0; a < 3; ++a) {
                    u[a] = m[(1 + a) * N + n];
                    B[a] = m[(4 + a) * N + n];
                }
                out[0] += rho;
                for (int a = 0; a < 3; ++a) {
                    out[1 + a] += rho * u[a];
                    out[4 + a] += B[a];
                }
                out[7] += 0.5 * rho * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                out[8] += 0.5 * (B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
                out[9] += u[0] * B[0] + u[1] * B[1] + u[2] * B[2];
                long xp = (z * ny + y) * nx + wrap3(x + 1, nx), xm = (z * ny + y) * nx + wrap3(x - 1, nx);
                long yp = (z * ny + wrap3(y + 1, ny)) * nx + x, ym = (z * ny + wrap3(y - 1, ny)) * nx + x;
                long zp = (wrap3(z + 1, nz) * ny + y) * nx + x, zm = (wrap3(z - 1, nz) * ny + y) * nx + x;
                double div = 0.5 * (m[4 * N + xp] - m[4 * N + xm]) + 0.5 * (m[5 * N + yp] - m[5 * N + ym]) +
                             0.5 * (m[6 * N + zp] - m[6 * N + zm]);
                if (fabs(div) > dmax) dmax = fabs(div);
                d2 += div * div;
            }
    out[7] /= (double)N;
    out[8] /= (double)N;
    out[9] /= (double)N;
    out[10] = dmax;
    out[11] = sqrt(d2 / (double)N);
    free(m);
}
