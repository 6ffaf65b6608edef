"""Pins of the 3D oracle (oracle/lbmhd3_oracle.c) to what the paper and the
mathematics fix, none of them a retyping of its formulas:

- the lattices: D3Q27 weights isotropic to fourth order, the six-axis
  magnetic lattice isotropic to second order (the moment conditions the
  Chapman-Enskog limit of Sec. 3 needs);
- the equilibria's moments: mass, momentum and the MHD stress
  rho/3 I + rho u u + |B|^2/2 I - B B; the magnetic first moment u B - B u;
- the paper's printed 2D equilibria (Sec. 3, D2Q9 and D2Q5) are the
  c_z-marginals of the 3D ones for u_z = B_z = 0;
- dynamics: a flow independent of z (or of x, or of y) evolves, summed over
  the velocities along the idle axis, exactly as the 2D BGK oracle (the
  paper's MRT with tied rates) with LES off;
- conservation of mass, momentum and sum B with the local LES rates on;
- shear-wave and magnetic-diffusion decay along z at nu k^2, eta k^2 with
  nu = (tau_nu - 1/2)/3, eta = (tau_eta - 1/2)/3 (Sec. 4.3), converging at
  second order;
- the local |S| estimate 3 Q / (2 rho tau) against the analytic strain;
- div B at round-off for s_m = 1 (central differences commute in 3D too);
- the paper's kinetic LES (les = 2): the moments of the equilibrium
  corrections are the filtered MHD stress and EMF corrections, checked
  against brute-force Gaussian filtering (Eq. Gaussian) along an oblique
  direction to fourth order in Delta; a flow independent of one axis steps
  exactly as the 2D oracle's kinetic LES with tied rates; Delta -> 0 is LES
  off; conservation;
- the cross-helicity closure (les = 3): the energy drain of an Alfvenic
  shear along z is <(nu + nu_t) |du|^2> and <(eta + eta_t) |dB|^2> with the
  eddy coefficients of Eqs. CHClosureV/B, backscatter for B = -u;
  C_S = 0 is LES off; conservation.
"""
import numpy as np
import pytest

from paper_1607_08675_gb300 import inputs


@pytest.fixture(scope="module")
def o3():
    from oracle import oracle3

    oracle3.build()
    return oracle3


@pytest.fixture(scope="module")
def o2():
    from oracle import oracle

    oracle.build()
    return oracle


def test_lattice_isotropy(o3):
    c, w, cm, wm = o3.lattice()
    c = c.astype(float)
    I = np.eye(3)
    assert abs(w.sum() - 1) < 1e-15
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", w, c, c), I / 3, atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-16)
    four = np.einsum("i,ia,ib,ic,id->abcd", w, c, c, c, c)
    iso = (np.einsum("ab,cd->abcd", I, I) + np.einsum("ac,bd->abcd", I, I) +
           np.einsum("ad,bc->abcd", I, I)) / 9
    assert np.allclose(four, iso, atol=1e-16)
    assert sorted(map(tuple, c.astype(int))) == sorted(
        (a, b, d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1))
    cm = cm.astype(float)
    assert abs(wm.sum() - 1) < 1e-15  # the rest weight is zero
    assert np.allclose(np.einsum("k,ka,kb->ab", wm, cm, cm), I / 3, atol=1e-16)


@pytest.mark.parametrize("seed", range(4))
def test_equilibrium_moments_are_the_mhd_fluxes(o3, seed):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.2 * rng.random()
    u = 0.1 * rng.standard_normal(3)
    B = 0.1 * rng.standard_normal(3)
    c, w, cm, wm = o3.lattice()
    c, cm = c.astype(float), cm.astype(float)
    f = o3.feq(rho, u, B)
    assert abs(f.sum() - rho) < 1e-15
    assert np.allclose(c.T @ f, rho * u, atol=1e-16)
    stress = rho / 3 * np.eye(3) + rho * np.outer(u, u) + 0.5 * B @ B * np.eye(3) - np.outer(B, B)
    assert np.allclose(np.einsum("i,ia,ib->ab", f, c, c), stress, atol=1e-15)
    g = o3.geq(u, B).reshape(6, 3)
    assert np.allclose(g.sum(axis=0), B, atol=1e-16)
    N = np.einsum("ka,kb->ab", cm, g)
    assert np.allclose(N, np.outer(u, B) - np.outer(B, u), atol=1e-16)


def _index2d(o2):
    cx, cy, _, _, _, _ = o2.lattice()
    return {(int(a), int(b)): i for i, (a, b) in enumerate(zip(cx, cy))}


def marginal_f(o2, o3, f3, axis=2):
    """Sum the D3Q27 populations over the velocity component along `axis`,
    in the D2Q9 order of the 2D oracle (the other two axes in order)."""
    c, _, _, _ = o3.lattice()
    keep = [a for a in range(3) if a != axis]
    idx = _index2d(o2)
    out = np.zeros((9,) + f3.shape[1:])
    for i in range(27):
        out[idx[(int(c[i][keep[0]]), int(c[i][keep[1]]))]] += f3[i]
    return out


def marginal_g(o3, g3, axis=2):
    """The six axis populations to the D2Q5 layout of the 2D oracle: the
    pair along `axis` becomes the rest population; components of the other
    two axes, in order."""
    _, _, cm, _ = o3.lattice()
    keep = [a for a in range(3) if a != axis]
    g3 = g3.reshape((6, 3) + g3.shape[1:])
    out = np.zeros((5, 2) + g3.shape[2:])
    d2 = {(0, 0): 0, (1, 0): 1, (0, 1): 2, (-1, 0): 3, (0, -1): 4}
    for q in range(6):
        k = d2[(int(cm[q][keep[0]]), int(cm[q][keep[1]]))]
        for j, a in enumerate(keep):
            out[k, j] += g3[q, a]
    return out.reshape((10,) + g3.shape[2:])


@pytest.mark.parametrize("seed", range(3))
def test_2d_equilibria_are_the_marginals(o2, o3, seed):
    """The paper's D2Q9 and D2Q5 equilibria (as the 2D oracle computes them)
    are the 3D equilibria summed over c_z, for u_z = B_z = 0."""
    rng = np.random.default_rng(10 + seed)
    rho, (ux, uy), (bx, by) = 1 + 0.1 * rng.random(), 0.1 * rng.standard_normal(2), \
        0.1 * rng.standard_normal(2)
    f3 = o3.feq(rho, [ux, uy, 0.0], [bx, by, 0.0])
    assert np.allclose(marginal_f(o2, o3, f3), o2.feq(rho, ux, uy, bx, by), atol=2e-16)
    g3 = o3.geq([ux, uy, 0.0], [bx, by, 0.0])
    assert np.allclose(marginal_g(o3, g3), o2.geq(ux, uy, bx, by).reshape(-1), atol=2e-16)


def _fields2d(n1, n2, seed):
    rho, ux, uy, bx, by = inputs.orszag_tang(n1, n2, seed=seed, amp=1e-3)
    return rho, ux, uy, bx, by


@pytest.mark.parametrize("axis", [2, 0, 1])
def test_flow_independent_of_one_axis_is_the_2d_bgk_flow(o2, o3, axis):
    """A 3D Orszag-Tang flow that does not vary along `axis` (and has no
    velocity or field along it), stepped by the 3D oracle and summed over the
    velocities along that axis, equals the 2D oracle's BGK step (the paper's
    MRT with tied rates) of the same 2D flow -- with LES off, where the two
    models must agree exactly (up to rounding order)."""
    n1, n2, n3, steps = 12, 10, 3, 15
    tau, taum = 0.62, 0.71
    rho, ua, ub, ba, bb = _fields2d(n1, n2, seed=4)  # 2D arrays (n2, n1)
    keep = [a for a in range(3) if a != axis]  # the 2D x and y, in order
    sizes = {keep[0]: n1, keep[1]: n2, axis: n3}
    nx, ny, nz = sizes[0], sizes[1], sizes[2]

    def lift(a2):
        # a2[j, i]: i along keep[0], j along keep[1]; tile along `axis`
        out = np.zeros((nz, ny, nx))
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    pos = (x, y, z)
                    out[z, y, x] = a2[pos[keep[1]], pos[keep[0]]]
        return out

    zero = np.zeros((nz, ny, nx))
    u = [zero, zero, zero]
    B = [zero, zero, zero]
    u[keep[0]], u[keep[1]] = lift(ua), lift(ub)
    B[keep[0]], B[keep[1]] = lift(ba), lift(bb)
    st3 = o3.init(lift(rho), u[0], u[1], u[2], B[0], B[1], B[2])
    st3 = o3.step(st3, o3.params(tau_nu=tau, tau_eta=taum, C_S=0.0, les=0), steps)
    st2 = o2.step_bgk(o2.init(rho, ua, ub, ba, bb), tau, taum, steps)
    f2 = marginal_f(o2, o3, st3[:27], axis)
    g2 = marginal_g(o3, st3[27:], axis)
    got = np.concatenate([f2, g2])  # (19, nz, ny, nx)
    # every slice across the idle axis is the 2D state (19, n2, n1): the
    # array axes left after taking one are keep[1] then keep[0]
    arr_axis = 3 - axis  # array axis of `axis` in (plane, z, y, x)
    for s in range(sizes[axis]):
        sl = np.take(got, s, axis=arr_axis)
        assert sl.shape == st2.shape
        assert np.max(np.abs(sl - st2)) < 5e-15, (axis, s, np.max(np.abs(sl - st2)))


def _field3d(n, seed, amp=0.03):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    k = 2 * np.pi / n
    rho = 1 + 0.01 * np.cos(k * x + 0.3) * np.sin(k * z)
    ph = rng.random(6) * 2 * np.pi
    u = [amp * np.sin(k * y + ph[0]), amp * np.sin(k * z + ph[1]), amp * np.sin(k * x + ph[2])]
    B = [amp * np.cos(k * z + ph[3]), amp * np.cos(k * x + ph[4]), amp * np.cos(k * y + ph[5])]
    return rho, u, B


def test_conservation_with_les(o3):
    rho, u, B = _field3d(8, seed=2)
    st = o3.init(rho, *u, *B)
    p = o3.params(tau_nu=0.55, tau_eta=0.6, C_S=0.2, delta=2.0, les=1)
    d0 = o3.diagnostics(st)
    st = o3.step(st, p, 40)
    d1 = o3.diagnostics(st)
    for k in ("mass", "mom_x", "mom_y", "mom_z", "bsum_x", "bsum_y", "bsum_z"):
        assert abs(d1[k] - d0[k]) < 1e-12 * max(1.0, abs(d0[k])) * 10, (k, d0[k], d1[k])
    assert d1["E_kin"] < d0["E_kin"] and d1["E_mag"] < d0["E_mag"]


def _decay_rate(o3, n, tau, taum, kind, steps=40):
    z = np.arange(n)
    k = 2 * np.pi / n
    shp = (n, 2, 3)  # (nz, ny, nx): the wave varies along z only
    zz = np.broadcast_to(z[:, None, None], shp)
    zero = np.zeros(shp)
    rho = np.ones(shp)
    amp = 1e-6
    if kind == "shear":
        u = [amp * np.sin(k * zz), zero, zero]
        B = [zero, zero, zero]
    else:
        u = [zero, zero, zero]
        B = [amp * np.sin(k * zz), zero, zero]
    st = o3.init(rho, *u, *B)
    p = o3.params(tau_nu=tau, tau_eta=taum, C_S=0.0, les=0)
    a = []
    for _ in range(2):
        st = o3.step(st, p, steps)
        m = o3.moments(st)
        fld = m[1] if kind == "shear" else m[4]
        a.append(np.sum(fld[:, 0, 0] * np.sin(k * z)) / np.sum(np.sin(k * z) ** 2))
    return -np.log(a[1] / a[0]) / steps / k ** 2


@pytest.mark.parametrize("kind", ["shear", "magnetic"])
def test_decay_rates_along_z(o3, kind):
    """Shear wave u_x(z) and magnetic mode B_x(z): the measured diffusivity
    tends to nu = (tau - 1/2)/3 (eta for B) at second order in k."""
    tau, taum = 0.8, 0.9
    want = (tau - 0.5) / 3 if kind == "shear" else (taum - 0.5) / 3
    e = [abs(_decay_rate(o3, n, tau, taum, kind) / want - 1) for n in (16, 32)]
    assert e[1] < 3e-3 and e[1] < e[0] / 3, e


def test_local_strain_estimate(o3):
    """u_x = U sin(k z): once the non-equilibrium part has developed from the
    equilibrium start (20 steps), the local estimate 3 Q / (2 rho tau) at
    each node tracks |dU/dz| = U k |cos(k z)| (LES off, so tau is the base
    tau), to O(k^2)."""
    n, U = 32, 1e-4
    k = 2 * np.pi / n
    z = np.arange(n)
    shp = (n, 1, 1)
    zz = z.reshape(shp)
    zero = np.zeros(shp)
    tau = 0.7
    st = o3.init(np.ones(shp), U * np.sin(k * zz), zero, zero, zero, zero, zero)
    p = o3.params(tau_nu=tau, tau_eta=0.7, C_S=0.0, les=0)
    steps = 20
    st = o3.step(st, p, steps)
    pulled = o3.stream(st)
    nu = (tau - 0.5) / 3
    damp = np.exp(-nu * k * k * steps)
    for zi in (0, 3, 8, 13):
        _, aux = o3.collide_cell(pulled[:, zi, 0, 0], p)
        est = 3 * aux[2] / (2 * tau)
        want = U * k * abs(np.cos(k * zi)) * damp
        assert abs(est - want) < 0.01 * U * k, (zi, est, want)


def test_div_b_machine_zero_at_unit_magnetic_rate(o3):
    """B as the periodic central-difference curl of a potential (exactly
    divergence free under central differences), tau_eta = 1, LES off: div B
    stays at round-off over the run."""
    n = 8
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, n, n, n)) * 1e-2

    def d(f, axis):  # central difference along array axis (z=0, y=1, x=2)
        return 0.5 * (np.roll(f, -1, axis) - np.roll(f, 1, axis))

    Bx = d(A[2], 1) - d(A[1], 0)
    By = d(A[0], 0) - d(A[2], 2)
    Bz = d(A[1], 2) - d(A[0], 1)
    rho, u, _ = _field3d(n, seed=6, amp=0.02)
    st = o3.init(rho, *u, Bx, By, Bz)
    assert o3.diagnostics(st)["divB_max"] < 1e-16
    st = o3.step(st, o3.params(tau_nu=0.7, tau_eta=1.0, C_S=0.0, les=0), 30)
    diag = o3.diagnostics(st)
    assert diag["divB_max"] < 1e-15, diag["divB_max"]


def test_thread_count_does_not_change_the_bits(o3):
    rho, u, B = _field3d(6, seed=7)
    st = o3.init(rho, *u, *B)
    p = o3.params(tau_nu=0.55, tau_eta=0.6, C_S=0.15, les=1)
    one = o3.step(st, p, 5, nthreads=1)
    assert np.array_equal(o3.step(st, p, 5, nthreads=4), one)


def test_step_cells_equals_full_step(o3):
    rho, u, B = _field3d(6, seed=8)
    st = o3.init(rho, *u, *B)
    p = o3.params(tau_nu=0.55, tau_eta=0.6, C_S=0.15, les=1)
    st = o3.step(st, p, 3)
    full = o3.step(st, p, 1).reshape(45, -1)
    idx = np.array([0, 7, 35, 100, 215])
    assert np.array_equal(o3.step_cells(st, p, idx), full[:, idx].T)


# ---------------------------------------------------------------- the paper's kinetic LES (les = 2)


def _gauss_filter_1d(f, s, delta):
    """The paper's Gaussian filter (Eq. Gaussian, variance Delta^2/12 per
    axis) of a periodic profile f(s), by quadrature.  The 3D filter is the
    product of three such factors, so it is isotropic, and a field varying
    along one direction only is filtered by this 1D factor along it."""
    h = s[1] - s[0]
    r = np.arange(-len(s) // 2, len(s) // 2) * h
    G = np.sqrt(6.0 / (np.pi * delta ** 2)) * np.exp(-6.0 * r ** 2 / delta ** 2)
    out = np.zeros_like(f)
    for j, rj in enumerate(r):
        out += np.roll(f, int(round(rj / h))) * G[j] * h
    return out


def test_kinetic_shift_moments_match_gaussian_filtering(o3):
    """Fields varying along the oblique direction n = (1, 2, 3)/sqrt(14), so
    that every gradient component is non-zero.  The corrected equilibria
    must carry the filtered MHD stress (rho u u + |B|^2/2 I - B B filtered,
    the rho/3 I part being linear) and the filtered magnetic flux
    u B - B u: exact filtering minus the value in the filtered fields
    is the second moment of the f correction and the first moment of the
    g correction up to O(Delta^4) (the order Sec. 2 truncates at).  Their
    mass, momentum and sum of B stay zero."""
    c, _, cm, _ = o3.lattice()
    c, cm = c.astype(float), cm.astype(float)
    nvec = np.array([1.0, 2.0, 3.0]) / np.sqrt(14.0)
    L = 2 * np.pi
    s = np.linspace(0, L, 4096, endpoint=False)
    rho = 1.0 + 0.2 * np.sin(s + 0.3)
    j = np.stack([0.3 + 0.2 * np.sin(s) + 0.1 * np.cos(2 * s), 0.1 * np.cos(s) - 0.2 * np.sin(3 * s),
                  -0.15 * np.sin(2 * s + 1.0)])
    B = np.stack([0.2 * np.cos(s + 0.5), 0.1 + 0.1 * np.sin(2 * s), 0.25 * np.cos(3 * s - 0.2)])
    k = np.fft.fftfreq(len(s), L / len(s)) * 2 * np.pi
    deriv = lambda f: np.real(np.fft.ifft(1j * k * np.fft.fft(f)))

    def stress(r, jj, bb):
        out = np.einsum("a...,b...->ab...", jj, jj) / r
        out += 0.5 * np.einsum("a...,a...->...", bb, bb) * np.eye(3)[..., None]
        out -= np.einsum("a...,b...->ab...", bb, bb)
        return out

    def flux(r, jj, bb):  # sum_k C_ka g_kb^eq = u_a B_b - B_a u_b
        return (np.einsum("a...,b...->ab...", jj, bb) - np.einsum("a...,b...->ab...", bb, jj)) / r

    errs, plain, ferrs = [], [], []
    pick = slice(0, len(s), 128)
    for delta in (0.2, 0.1):
        F = lambda a: _gauss_filter_1d(a, s, delta)
        rb, jb, bb = F(rho), np.stack([F(a) for a in j]), np.stack([F(a) for a in B])
        exact = np.stack([[F(a) for a in row] for row in stress(rho, j, B)])
        exact_flux = np.stack([[F(a) for a in row] for row in flux(rho, j, B)])
        base, base_flux = stress(rb, jb, bb), flux(rb, jb, bb)
        fields = np.concatenate([[rb], jb, bb])  # (7, len(s))
        d = np.stack([deriv(a) for a in fields])
        e, ef, pl = 0.0, 0.0, 0.0
        for i in range(len(s))[pick]:
            fs, gs = o3.kinetic_shift(fields[:, i], np.outer(d[:, i], nvec), delta)
            assert abs(fs.sum()) < 1e-17 and np.allclose(c.T @ fs, 0, atol=1e-17)
            assert np.allclose(gs.reshape(6, 3).sum(axis=0), 0, atol=1e-17)
            got = base[:, :, i] + np.einsum("q,qa,qb->ab", fs, c, c)
            gotf = base_flux[:, :, i] + np.einsum("ka,kb->ab", cm, gs.reshape(6, 3))
            e = max(e, np.max(np.abs(got - exact[:, :, i])))
            ef = max(ef, np.max(np.abs(gotf - exact_flux[:, :, i])))
            pl = max(pl, np.max(np.abs(base[:, :, i] - exact[:, :, i])))
        errs.append(e)
        ferrs.append(ef)
        plain.append(pl)
    assert errs[1] < 3e-6 and ferrs[1] < 3e-6, (errs, ferrs, plain)
    assert 10.0 < errs[0] / errs[1] < 24.0, errs  # fourth order
    assert 10.0 < ferrs[0] / ferrs[1] < 24.0, ferrs
    assert plain[1] > 100 * errs[1]  # without the corrections: second order only


def _lift2d(arrays2d, axis, n3):
    """Tile 2D arrays a2[j, i] (i along the first kept axis, j along the
    second) along `axis`; returns arrays of shape (nz, ny, nx)."""
    keep = [a for a in range(3) if a != axis]
    n2, n1 = arrays2d[0].shape
    sizes = {keep[0]: n1, keep[1]: n2, axis: n3}
    z, y, x = np.meshgrid(np.arange(sizes[2]), np.arange(sizes[1]), np.arange(sizes[0]),
                          indexing="ij")
    pos = (x, y, z)
    return [a2[pos[keep[1]], pos[keep[0]]] for a2 in arrays2d], keep


@pytest.mark.parametrize("axis", [2, 0, 1])
def test_kinetic_les_flow_independent_of_one_axis_is_the_2d_kinetic_les(o2, o3, axis):
    """A flow that does not vary along `axis`, stepped with the filtered
    equilibria and summed over the velocities along that axis, equals the
    2D oracle's kinetic LES (the paper's MRT with every rate tied, where it
    relaxes towards the same shifted distribution)."""
    n1, n2, n3, steps = 12, 10, 3, 12
    tau, taum, delta = 0.62, 0.71, 2.5
    rho, ua, ub, ba, bb = inputs.orszag_tang(n1, n2, u0=0.08, b0=0.08, amp=1e-2, seed=9)
    (r3, a3, b3, ba3, bb3), keep = _lift2d([rho, ua, ub, ba, bb], axis, n3)
    zero = np.zeros_like(r3)
    u, B = [zero] * 3, [zero] * 3
    u[keep[0]], u[keep[1]] = a3, b3
    B[keep[0]], B[keep[1]] = ba3, bb3
    st3 = o3.step(o3.init(r3, *u, *B), o3.params(tau_nu=tau, tau_eta=taum, delta=delta, les=2), steps)
    st2 = o2.step(o2.init(rho, ua, ub, ba, bb),
                  o2.params(tau_nu=tau, tau_eta=taum, delta=delta, les=2), steps)
    plain = o2.step(o2.init(rho, ua, ub, ba, bb), o2.params(tau_nu=tau, tau_eta=taum, les=0), steps)
    assert np.max(np.abs(st2 - plain)) > 1e-6  # the corrections are visible
    got = np.concatenate([marginal_f(o2, o3, st3[:27], axis), marginal_g(o3, st3[27:], axis)])
    arr_axis = 3 - axis
    for sl in range(n3):
        d = np.max(np.abs(np.take(got, sl, axis=arr_axis) - st2))
        assert d < 1e-14, (axis, sl, d)


def test_kinetic_les_vanishing_width_is_les_off(o3):
    rho, u, B = _field3d(6, seed=11)
    st = o3.step(o3.init(rho, *u, *B), o3.params(les=0), 2)
    a = o3.step(st, o3.params(les=2, delta=1e-200), 4)
    b = o3.step(st, o3.params(les=0), 4)
    assert np.array_equal(a, b)


@pytest.mark.parametrize("les", [2, 3])
def test_gradient_closures_conserve(o3, les):
    rho, u, B = _field3d(8, seed=12, amp=0.05)
    st = o3.init(rho, *u, *B)
    p = o3.params(tau_nu=0.56, tau_eta=0.6, C_S=0.3, delta=2.5, les=les)
    d0 = o3.diagnostics(st)
    st = o3.step(st, p, 40)
    d1 = o3.diagnostics(st)
    assert abs(d1["mass"] - d0["mass"]) < 1e-13 * d0["mass"]
    for key in ("mom_x", "mom_y", "mom_z", "bsum_x", "bsum_y", "bsum_z"):
        assert abs(d1[key] - d0[key]) < 1e-13 * d0["mass"], key
    assert d1["E_kin"] < d0["E_kin"] and d1["E_mag"] < d0["E_mag"]


@pytest.mark.parametrize("les", [2, 3])
def test_gradient_closures_step_cells_and_threads(o3, les):
    rho, u, B = _field3d(6, seed=13, amp=0.05)
    p = o3.params(tau_nu=0.56, tau_eta=0.6, C_S=0.3, delta=2.5, les=les)
    st = o3.step(o3.init(rho, *u, *B), p, 3)
    full = o3.step(st, p, 1)
    idx = np.array([0, 5, 6, 35, 36, 107, 215])
    assert np.array_equal(o3.step_cells(st, p, idx), full.reshape(45, -1)[:, idx].T)
    assert np.array_equal(o3.step(st, p, 3, nthreads=4), o3.step(st, p, 3, nthreads=1))


# ---------------------------------------------------------------- cross-helicity closure (les = 3)


def _carati_rates_z(o3, n, sign, CS, delta, tn, te, amp=0.005, t0=40):
    """Shear u_x = U sin(k z) with B_x = sign u_x: the measured dE_K/dt and
    dE_M/dt against the closure's eddy viscosity and resistivity."""
    z = 2 * np.pi * np.arange(n) / n
    shp = (n, 1, 1)
    u = (amp * np.sin(z)).reshape(shp)
    zero = np.zeros(shp)
    st = o3.init(1 + zero, u, zero, zero, sign * u, zero, zero)
    p = o3.params(tau_nu=tn, tau_eta=te, C_S=CS, delta=delta, les=3)
    s0 = o3.step(st, p, t0 - 1)
    s1 = o3.step(s0, p, 1)
    s2 = o3.step(s1, p, 1)
    ek = lambda s: np.mean(0.5 * o3.moments(s)[0] * o3.moments(s)[1] ** 2)
    em = lambda s: np.mean(0.5 * o3.moments(s)[4] ** 2)
    dek, dem = (ek(s2) - ek(s0)) / 2, (em(s2) - em(s0)) / 2
    m = o3.moments(s1)
    k = np.fft.fftfreq(n, 1.0 / n) * 2 * np.pi / n
    du = np.real(np.fft.ifft(1j * k * np.fft.fft(m[1][:, 0, 0])))
    dbx = np.real(np.fft.ifft(1j * k * np.fft.fft(m[4][:, 0, 0])))
    cd2 = CS * delta ** 2
    nu, eta = (tn - 0.5) / 3, (te - 0.5) / 3
    # S^v:S^b = 2 (du/2)(dbx/2); omega = (0, du, 0), j = (0, dbx, 0)
    nu_t = cd2 * np.sqrt(np.abs(du * dbx) / 2)
    eta_t = cd2 * np.sign(du * dbx) * np.sqrt(np.abs(du * dbx))
    pk = -np.mean((nu + nu_t) * du ** 2)
    pm = -np.mean((eta + eta_t) * dbx ** 2)
    return dek / pk - 1, dem / pm - 1, -np.mean(nu * du ** 2), -np.mean(eta * dbx ** 2), dek, dem


@pytest.mark.parametrize("sign", [1.0, -1.0])
def test_cross_helicity_closure_dissipation_along_z(o3, sign):
    """Eqs. CHClosureV/B with 3D vectors, along the axis the 2D model does
    not have: an Alfvenic shear along z drains kinetic and magnetic energy
    at <(nu + nu_t) |du/dz|^2> and <(eta + eta_t) |dB/dz|^2>; for B = -u
    the eddy resistivity is negative (backscatter)."""
    ek, em, k0, m0, dek, dem = _carati_rates_z(o3, 64, sign, 1.0, 4.0, 0.6, 0.7)
    assert abs(ek) < 5e-3 and abs(em) < 5e-3, (ek, em)
    assert abs(dek / k0 - 1) > 0.05
    if sign > 0:
        assert dem / m0 - 1 > 0.05
    else:
        assert dem / m0 - 1 < -0.05


def test_cross_helicity_closure_vanishing_constant_is_les_off(o3):
    rho, u, B = _field3d(6, seed=14)
    st = o3.step(o3.init(rho, *u, *B), o3.params(les=0), 2)
    a = o3.step(st, o3.params(les=3, C_S=0.0), 4)
    b = o3.step(st, o3.params(les=0), 4)
    assert np.array_equal(a, b)
