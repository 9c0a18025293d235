"""Pins of the FP64 CPU oracle against what the paper and mathematics fix.

Each test checks one oracle function against something other than the
oracle itself: a value the paper states, a closed form, an independent
numerical route (quadrature, an ODE solve, a banded linear solve, a dense
matrix assembled face by face), or an invariant of the scheme.  Equation
numbers refer to Sun et al., arXiv 2303.14119.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, linalg, optimize, stats

import oracle
from paper_2303_14119_gb300 import synth
from oracle import EPS0, ME, QE, Oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def paper_defaults():
    with open(os.path.join(GOLDEN, "paper_defaults.json")) as fh:
        return json.load(fh)


# ---------------------------------------------------------------- Eqs. 8-11
def test_seey_peak_is_delta_max_at_A_max_for_normal_incidence():
    """Sec. 2 after Eq. 9: delta_max is the largest yield and A_max the normal
    incidence energy where it occurs.  Checked on the paper's defaults."""
    d = paper_defaults()
    dmax, amax = d["delta_max"], d["A_max_eV"]
    res = optimize.minimize_scalar(lambda A: -oracle.seey(A, 0.0, dmax, amax),
                                   bounds=(1.0, 10 * amax), method="bounded",
                                   options={"xatol": 1e-9})
    assert abs(-res.fun / dmax - 1.0) < 2e-4
    assert abs(res.x / amax - 1.0) < 2e-3


def test_seey_angle_scaling_identity():
    """Eqs. 8-9: the incidence angle rescales the energy axis by
    (1 + k alpha^2/pi) and the yield by (1 + k alpha^2/(2 pi))."""
    dmax, amax, ks = 3.0, 400.0, 1.0
    for alpha in (0.1, 0.5, 1.0, 1.5):
        for A in (5.0, 60.0, 400.0, 3000.0):
            lhs = oracle.seey(A * (1 + ks * alpha ** 2 / math.pi), alpha, dmax, amax, ks)
            rhs = (1 + ks * alpha ** 2 / (2 * math.pi)) * oracle.seey(A, 0.0, dmax, amax, ks)
            assert lhs == pytest.approx(rhs, rel=1e-13)


def test_seey_limits_and_monotonicity():
    assert oracle.seey(0.0, 0.0, 3.0, 400.0) == 0.0
    assert oracle.seey(1e-9, 0.0, 3.0, 400.0) < 1e-8
    A = np.linspace(1.0, 400.0, 200)
    y = [oracle.seey(a, 0.0, 3.0, 400.0) for a in A]
    assert np.all(np.diff(y) > 0)  # rising branch below A_max
    A = np.linspace(420.0, 5000.0, 200)
    y = [oracle.seey(a, 0.0, 3.0, 400.0) for a in A]
    assert np.all(np.diff(y) < 0)  # falling branch above A_max


def test_incident_energy_and_angle():
    """Eq. 10 in eV and Eq. 11 measured from the surface normal."""
    v = math.sqrt(2 * 100.0 * QE / ME)  # 100 eV electron
    assert oracle.incident_energy_eV(-v, 0.0) == pytest.approx(100.0, rel=1e-14)
    assert oracle.incident_energy_eV(-v / math.sqrt(2), v / math.sqrt(2)) == pytest.approx(100.0, rel=1e-14)
    assert oracle.incidence_angle(-1.0, 0.0) == 0.0
    assert oracle.incidence_angle(-2.0, 2.0) == pytest.approx(math.pi / 4, rel=1e-15)
    assert oracle.incidence_angle(-1e-3, 5.0) == pytest.approx(math.pi / 2, abs=1e-3)


def test_seey_matrix_layout():
    """Sec. 2: delta_e(i, j) over the (v1, v2) grid, only where v1 < 0."""
    o = Oracle(4, 6, 5, 20e-6, -6e7, 6e7, -3e7, 3e7)
    o.set_see(3.0, 400.0, 1.0, 2.0)
    delta, _, _ = o.tables()
    _, v1, v2 = o.grid()
    for i in range(6):
        for j in range(5):
            if v1[i] >= 0:
                assert delta[i, j] == 0.0
            else:
                A = 0.5 * ME * (v1[i] ** 2 + v2[j] ** 2) / QE
                al = math.atan(abs(v2[j] / v1[i]))
                assert delta[i, j] == pytest.approx(oracle.seey(A, al, 3.0, 400.0), rel=1e-14)
    # v2 -> -v2 symmetry (alpha uses |v2|) on a symmetric grid
    assert np.allclose(delta, delta[:, ::-1], rtol=1e-13, atol=0)


# ---------------------------------------------------------------- Eqs. 15-16
def test_emission_prefactor_gives_unit_flux():
    """Eq. 15's prefactor makes the flux integral of Eq. 16 equal Gamma_see."""
    for T in (1.0, 2.0, 5.0):
        vt = math.sqrt(T * QE / ME)
        val, err = integrate.dblquad(lambda v2, v1: v1 * oracle.emission_continuum(v1, v2, T),
                                     0.0, 12 * vt, -12 * vt, 12 * vt, epsabs=0, epsrel=1e-10)
        assert val == pytest.approx(1.0, rel=1e-8)


def test_emission_table_flux_and_temperature():
    """R5 reading: grid-normalised Eq. 15 carries unit flux; on a fine grid its
    flux-weighted mean of m v1^2/2 is T_se and its mean of m v2^2/2 is T_se/2
    (half-Maxwellian flux in v1, Maxwellian in v2)."""
    T = 2.0
    vt = math.sqrt(T * QE / ME)
    o = Oracle(2, 400, 300, 20e-6, -8 * vt, 8 * vt, -8 * vt, 8 * vt)
    o.set_see(3.0, 400.0, 1.0, T)
    _, gse, _ = o.tables()
    _, v1, v2 = o.grid()
    info = o.info()
    dv = info["dv1"] * info["dv2"]
    V1, V2 = np.meshgrid(v1, v2, indexing="ij")
    assert np.all(gse[V1 <= 0] == 0)
    flux = V1 * gse * dv
    assert flux.sum() == pytest.approx(1.0, rel=1e-13)
    e1 = (flux * 0.5 * ME * V1 ** 2).sum() / QE
    e2 = (flux * 0.5 * ME * V2 ** 2).sum() / QE
    assert e1 == pytest.approx(T, rel=1e-3)
    assert e2 == pytest.approx(T / 2, rel=1e-3)
    # ratio to the continuum form is one constant that tends to 1
    cont = np.vectorize(lambda a, b: oracle.emission_continuum(a, b, T))(V1, V2)
    m = V1 > 0
    r = gse[m] / cont[m]
    assert np.ptp(r) / r.mean() < 1e-10
    assert r.mean() == pytest.approx(1.0, rel=1e-4)


# ---------------------------------------------------------------- Eq. 7
def test_source_shape_density_and_moments():
    """R6 reading of Eq. 7: unit density, half Maxwellian on v2 > 0 (mean
    sqrt(2T/(pi m))), full Maxwellian in v1 (mean 0, <v1^2> = T/m)."""
    T = 4.0
    vt = math.sqrt(T * QE / ME)
    o = Oracle(8, 300, 400, 20e-6, -8 * vt, 8 * vt, -8 * vt, 8 * vt)
    o.set_source(1.0, 10e-6, 15e-6, T)
    _, _, gfe = o.tables()
    _, v1, v2 = o.grid()
    info = o.info()
    dv = info["dv1"] * info["dv2"]
    V1, V2 = np.meshgrid(v1, v2, indexing="ij")
    assert np.all(gfe[V2 <= 0] == 0)
    w = gfe * dv
    assert w.sum() == pytest.approx(1.0, rel=1e-13)
    assert (w * V1).sum() == pytest.approx(0.0, abs=1e-9 * vt)
    assert (w * V1 ** 2).sum() == pytest.approx(vt ** 2, rel=1e-3)
    assert (w * V2).sum() == pytest.approx(math.sqrt(2 / math.pi) * vt, rel=1e-3)
    # band: centres in [10, 15] um on 8 cells of 2.5 um -> centres 11.25, 13.75
    assert info["n_band"] == 2


# ---------------------------------------------------------------- Poisson
def _poisson_fd(ne, sigma, dx):
    """Independent route: second-order FD Poisson for the potential at cell
    centres, -phi'' = rho/eps0 with rho = -e n, E = sigma/(2 eps0) at the
    dielectric (Neumann) and phi = 0 at x = h_max (Dirichlet); E at centres
    is the mean of the two face fields -dphi/dx."""
    nx = len(ne)
    rho = -QE * np.asarray(ne)
    ab = np.zeros((3, nx))
    rhs = -rho / EPS0 * dx * dx
    ab[0, 1:] = 1.0
    ab[1, :] = -2.0
    ab[2, :-1] = 1.0
    # wall face: (phi_0 - phi_-1)/dx = -E_wall  ->  phi_-1 = phi_0 + dx E_wall
    ab[1, 0] = -1.0
    rhs[0] -= dx * sigma / (2 * EPS0)
    # vacuum face value zero: phi_nx = -phi_{nx-1}
    ab[1, -1] = -3.0
    phi = linalg.solve_banded((1, 1), ab, rhs)
    faces = np.empty(nx + 1)
    faces[0] = sigma / (2 * EPS0)
    faces[1:-1] = -(phi[1:] - phi[:-1]) / dx
    faces[-1] = -(0.0 - phi[-1]) / (dx / 2)
    return 0.5 * (faces[:-1] + faces[1:]), faces


def test_ex_matches_fd_poisson_solve():
    nx, nv1, nv2 = 40, 6, 6
    o = Oracle(nx, nv1, nv2, 20e-6, -6e7, 6e7, -3e7, 3e7)
    rng = np.random.default_rng(3)
    f = rng.uniform(0.0, 1.0, (nx, nv1, nv2)) * 1e6
    sigma = 2e-3
    o.set_state(f, sigma)
    ne, ex, _, _ = o.moments()
    info = o.info()
    assert ne == pytest.approx(f.sum(axis=(1, 2)) * info["dv1"] * info["dv2"], rel=1e-13)
    ref, faces = _poisson_fd(ne, sigma, info["dx"])
    scale = np.abs(ref).max()
    assert np.abs(ex - ref).max() < 1e-10 * scale
    assert ex[0] != pytest.approx(sigma / (2 * EPS0))  # centre, not the wall face
    # the vacuum-side face field equals the Gauss value: total charge balance
    assert faces[-1] == pytest.approx(sigma / (2 * EPS0) - QE / EPS0 * ne.sum() * info["dx"], rel=1e-9)


def test_external_field_mode():
    o = Oracle(8, 4, 4, 20e-6, -6e7, 6e7, -3e7, 3e7)
    o.set_fields(-1e6, self_consistent=False, Ex_ext=2.5e5)
    o.set_state(np.ones((8, 4, 4)), 1.0)
    _, ex, _, _ = o.moments()
    assert np.all(ex == 2.5e5)
    assert np.all(o.accel() == pytest.approx(-QE * 2.5e5 / ME, rel=1e-15))
    assert o.info()["a2"] == pytest.approx(QE * 1e6 / ME, rel=1e-15)


# ---------------------------------------------------------------- advection
def test_free_streaming_binomial_and_exact_shift():
    """With no forces the donor-cell x-update of a delta is a binomial kernel
    B(n, c) in the upwind direction; at c = 1 it is an exact shift."""
    nx, nv1, nv2 = 64, 8, 3
    h, V = 20e-6, 6e7
    dx, dv1 = h / nx, 2 * V / nv1
    vmax_c = V - dv1 / 2
    dt = dx / vmax_c  # c = 1 on the two outermost v1 rows
    o = Oracle(nx, nv1, nv2, h, -V, V, -3e7, 3e7, dt=dt)
    o.set_fields(0.0, self_consistent=False, Ex_ext=0.0)
    k0, n = 30, 15
    f0 = np.zeros((nx, nv1, nv2))
    f0[k0] = 1.0
    o.set_state(f0, 0.0)
    o.step(n)
    f = o.get_f()
    _, v1, _ = o.grid()
    for i in range(nv1):
        c = abs(v1[i]) * dt / dx
        s = 1 if v1[i] > 0 else -1
        m = np.arange(n + 1)
        expect = stats.binom.pmf(m, n, min(c, 1.0))
        got = f[k0 + s * m, i, :]
        assert np.allclose(got, expect[:, None], rtol=0, atol=1e-14)
        assert abs(f[:, i, :].sum() - nv2) < 1e-12  # nothing left the domain
    assert f[k0 + n, nv1 - 1, 0] == pytest.approx(1.0, abs=1e-14)
    assert f[k0 - n, 0, 0] == pytest.approx(1.0, abs=1e-14)


def _accel_for_courant(c, dv, dt):
    return c * dv / dt


@pytest.mark.parametrize("sign1", [1, -1])
def test_velocity_marginal_trinomial(sign1):
    """Constant forces: the x-marginal of a delta evolves by the unsplit
    donor-cell update in (v1, v2) alone, a trinomial kernel."""
    nx, nv1, nv2 = 64, 14, 12
    h, V1, V2 = 20e-6, 6e7, 3e7
    o = Oracle(nx, nv1, nv2, h, -V1, V1, -V2, V2, cfl=0.4)
    info = o.info()
    dt = info["dt"]
    c1, c2 = 0.2, 0.15
    a1 = sign1 * _accel_for_courant(c1, info["dv1"], dt)
    a2 = _accel_for_courant(c2, info["dv2"], dt)
    o.set_fields(-a2 * ME / QE, self_consistent=False, Ex_ext=-a1 * ME / QE)
    k0, i0, j0, n = 32, 7, 3, 6
    f0 = np.zeros((nx, nv1, nv2))
    f0[k0, i0, j0] = 1.0
    o.set_state(f0, 0.0)
    o.step(n)
    g = o.get_f().sum(axis=0)
    expect = np.zeros_like(g)
    for b in range(n + 1):
        for c in range(n + 1 - b):
            p = stats.multinomial.pmf([b, c, n - b - c], n, [c1, c2, 1 - c1 - c2])
            expect[i0 + sign1 * b, j0 + c] = p
    assert np.allclose(g, expect, rtol=0, atol=1e-13)


def test_x_v2_joint_trinomial():
    """No v1 force: at a fixed v1 row the delta spreads in (x, v2) as the
    trinomial of (c_x, c_2)."""
    nx, nv1, nv2 = 64, 10, 14
    o = Oracle(nx, nv1, nv2, 20e-6, -6e7, 6e7, -3e7, 3e7, cfl=0.4)
    info = o.info()
    dt, dx = info["dt"], info["dx"]
    c2 = 0.25
    a2 = _accel_for_courant(c2, info["dv2"], dt)
    o.set_fields(-a2 * ME / QE, self_consistent=False, Ex_ext=0.0)
    _, v1, _ = o.grid()
    i, k0, j0, n = 7, 20, 2, 7
    cx = v1[i] * dt / dx
    assert cx > 0
    f0 = np.zeros((nx, nv1, nv2))
    f0[k0, i, j0] = 1.0
    o.set_state(f0, 0.0)
    o.step(n)
    f = o.get_f()[:, i, :]
    expect = np.zeros_like(f)
    for a in range(n + 1):
        for b in range(n + 1 - a):
            expect[k0 + a, j0 + b] = stats.multinomial.pmf([a, b, n - a - b], n, [cx, c2, 1 - cx - c2])
    assert np.allclose(f, expect, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- dense matrix
def _dense_step(f, sigma, tabs, grid, p):
    """One step assembled face by face as an affine map f' = M f + b, with
    E_x from the FD Poisson solve above and sigma from Eq. 18."""
    nx, nv1, nv2 = f.shape
    x, v1, v2 = grid
    dx, dv1, dv2, dt = p["dx"], p["dv1"], p["dv2"], p["dt"]
    delta, gse, gfe = tabs
    N = f.size
    L = lambda k, i, j: (k * nv1 + i) * nv2 + j
    ne = f.sum(axis=(1, 2)) * dv1 * dv2
    ex, _ = _poisson_fd(ne, sigma, dx)
    a1 = -QE * ex / ME
    a2 = -QE * p["Ey"] / ME
    M = np.eye(N)
    b = np.zeros(N)
    # Gamma_see as a row vector on the x = 0 plane (Eqs. 12-14)
    r_see = np.zeros(N)
    for i in range(nv1):
        for j in range(nv2):
            if v1[i] < 0:
                r_see[L(0, i, j)] = delta[i, j] * (-v1[i]) * dv1 * dv2

    def add_face(lo, hi, row, scale):
        if lo is not None:
            M[lo] -= scale * row
        if hi is not None:
            M[hi] += scale * row

    for kf in range(nx + 1):
        for i in range(nv1):
            for j in range(nv2):
                row = np.zeros(N)
                v = v1[i]
                if v > 0:
                    row = v * gse[i, j] * r_see if kf == 0 else _unit(N, L(kf - 1, i, j)) * v
                elif v < 0 and kf < nx:
                    row = _unit(N, L(kf, i, j)) * v
                add_face(L(kf - 1, i, j) if kf > 0 else None, L(kf, i, j) if kf < nx else None,
                         row, dt / dx)
    for k in range(nx):
        for jf in range(nv2 + 1):
            for i in range(nv1):
                row = np.zeros(N)
                if a2 > 0 and jf > 0:
                    row = _unit(N, L(k, i, jf - 1)) * a2
                elif a2 < 0 and jf < nv2:
                    row = _unit(N, L(k, i, jf)) * a2
                add_face(L(k, i, jf - 1) if jf > 0 else None, L(k, i, jf) if jf < nv2 else None,
                         row, dt / dv2)
        for iface in range(nv1 + 1):
            for j in range(nv2):
                row = np.zeros(N)
                if a1[k] > 0 and iface > 0:
                    row = _unit(N, L(k, iface - 1, j)) * a1[k]
                elif a1[k] < 0 and iface < nv1:
                    row = _unit(N, L(k, iface, j)) * a1[k]
                add_face(L(k, iface - 1, j) if iface > 0 else None, L(k, iface, j) if iface < nv1 else None,
                         row, dt / dv1)
    band = [k for k in range(nx) if p["x_lo"] <= x[k] <= p["x_hi"]]
    for k in band:
        for i in range(nv1):
            for j in range(nv2):
                b[L(k, i, j)] += dt * p["J"] / QE / (len(band) * dx) * gfe[i, j]
    fn = (M @ f.ravel() + b).reshape(f.shape)
    dsig = 0.0
    for i in range(nv1):
        if v1[i] < 0:
            for j in range(nv2):
                dsig += (delta[i, j] - 1.0) * (-v1[i]) * f[0, i, j] * dv1 * dv2
    return fn, sigma + QE * dt * dsig


def _unit(N, idx):
    u = np.zeros(N)
    u[idx] = 1.0
    return u


def _strong_case(nx, nv1, nv2, seed=1):
    """A tiny grid with every term of the step active and large Courant
    numbers: self-consistent E_x that changes sign across x, large E_y, SEE
    with a spread emission shape, and a strong source."""
    h, V1, V2 = 20e-6, 6e7, 3e7
    o = Oracle(nx, nv1, nv2, h, -V1, V1, -V2, V2, cfl=0.4)
    info = o.info()
    a2 = _accel_for_courant(0.2, info["dv2"], info["dt"])
    p = dict(info, Ey=-a2 * ME / QE, J=1e7, x_lo=0.3 * h, x_hi=0.7 * h)
    o.set_fields(p["Ey"], True, 0.0)
    o.set_see(3.0, 400.0, 1.0, 400.0)
    o.set_source(p["J"], p["x_lo"], p["x_hi"], 300.0)
    # amplitude so the space-charge field is comparable to sigma/(2 eps0)
    emax = 0.25 * info["dv1"] / info["dt"] * ME / QE
    sigma = 2 * EPS0 * emax * 0.8
    n_tot = 1.6 * emax * EPS0 / QE  # areal density giving a field drop of 1.6 emax
    amp = 2 * n_tot / (h * 2 * V1 * 2 * V2)
    rng = np.random.default_rng(seed)
    f0 = rng.uniform(0.0, 1.0, (nx, nv1, nv2)) * amp
    return o, f0, sigma, p


def test_dense_matrix_brute_force():
    o, f0, sigma, p = _strong_case(4, 4, 5)
    o.set_state(f0, sigma)
    assert o.courant_sum() <= 1.0
    tabs = o.tables()
    grid = o.grid()
    a1 = o.accel()
    assert a1.max() > 0 > a1.min()  # both v1 directions exercised
    f, s = f0.copy(), sigma
    for _ in range(5):
        f, s = _dense_step(f, s, tabs, grid, p)
    o.step(5)
    got = o.get_f()
    assert np.abs(got - f).sum() / np.abs(f).sum() < 1e-13
    assert o.surface_charge() == pytest.approx(s, rel=1e-12)


# ---------------------------------------------------------------- invariants
def test_conservation_ledger():
    """Electron and charge balance to round-off (Eqs. 13-18 with R5, R9)."""
    o, f0, sigma, p = _strong_case(16, 12, 10, seed=5)
    o.set_state(f0, sigma)
    o.step(60)
    L = o.ledger()
    rhs = L["emit"] - L["pe"] - L["vac"] - L["lv"] + L["inj"]
    scale = max(abs(L["emit"]), abs(L["pe"]), abs(L["vac"]), abs(L["lv"]), abs(L["inj"]), L["N"])
    assert abs((L["N"] - L["N0"]) - rhs) < 1e-12 * scale
    assert L["emit"] == pytest.approx(L["see"], rel=1e-13)  # R5
    dsig = o.surface_charge() - L["sigma0"]
    assert dsig / QE == pytest.approx(L["see"] - L["pe"], rel=1e-12)  # Eq. 18
    assert L["inj"] == pytest.approx(60 * p["dt"] * p["J"] / QE, rel=1e-12)
    for key in ("emit", "pe", "vac", "lv"):
        assert L[key] > 0


def test_positivity_under_cfl():
    o, f0, sigma, p = _strong_case(12, 10, 8, seed=7)
    o.set_state(f0, sigma)
    for _ in range(20):
        assert o.courant_sum() <= 1.0
        o.step(1)
        f = o.get_f()
        assert f.min() >= -1e-14 * f.max()


def test_cfl_violation_is_reported():
    o = Oracle(8, 6, 6, 20e-6, -6e7, 6e7, -3e7, 3e7, dt=1e-12)
    assert o.step_status(1) == oracle.ECFL


def test_default_dt_from_cfl():
    o = Oracle(64, 48, 48, 20e-6, -6e7, 6e7, -3e7, 3e7, cfl=0.4)
    assert o.info()["dt"] == pytest.approx(0.4 * (20e-6 / 64) / 6e7, rel=1e-15)


def test_convergence_rule_degenerate_and_active():
    """End of Sec. 2: converged when sigma and both fluxes change by at most
    0.1 % over the window.  An empty domain is converged once the window has
    passed; a domain with a source switched on is not."""
    o = Oracle(8, 6, 6, 20e-6, -6e7, 6e7, -3e7, 3e7)
    o.set_convergence(5, 1e-3)
    o.step(4)
    assert o.info()["sat_step"] == -1
    o.step(1)
    assert o.info()["sat_step"] == 5
    o2 = Oracle(8, 6, 6, 20e-6, -6e7, 6e7, -3e7, 3e7)
    o2.set_see(3.0, 400.0, 1.0, 2.0)
    o2.set_source(1.0, 5e-6, 15e-6, 4.0)
    o2.set_convergence(5, 1e-3)
    o2.step(12)
    assert o2.info()["sat_step"] == -1
    h = o2.history()
    assert h.shape == (13, oracle.HIST_COLS)
    assert np.all(h[:, 0] == np.arange(13))


def test_see_disabled_means_no_secondaries():
    o, f0, sigma, p = _strong_case(6, 6, 6, seed=2)
    o.set_see(3.0, 400.0, 1.0, 400.0, enabled=False)
    o.set_state(f0, sigma)
    _, _, gpe, gsee = o.moments()
    assert gsee == 0.0 and gpe > 0
    o.step(1)
    # Eq. 18 with no SEE: every primary is deposited
    assert o.surface_charge() == pytest.approx(sigma - QE * p["dt"] * gpe, rel=1e-13)


# ---------------------------------------------------------------- Eqs. 19-20
def test_first_crossover_is_unit_yield():
    for dmax, amax in ((3.0, 400.0), (6.5, 650.0), (2.0, 250.0)):
        a1 = oracle.first_crossover(dmax, amax)
        ref = optimize.brentq(lambda A: oracle.seey(A, 0.0, dmax, amax) - 1.0, 1e-6, amax, xtol=1e-14)
        assert a1 == pytest.approx(ref, rel=1e-10)
        assert oracle.seey(a1, 0.0, dmax, amax) == pytest.approx(1.0, abs=1e-12)
    assert oracle.first_crossover(0.9, 400.0) < 0  # no crossover below unit yield


def test_time_of_flight_by_kinematics():
    """Sec. 3: a secondary leaving normally with energy A0 against a constant
    restoring acceleration returns after 2 v0/|a_x| (ODE with landing event)."""
    A0, ax = 2.0, 3e16
    v0 = math.sqrt(2 * A0 * QE / ME)
    ev = lambda t, y: y[0]
    ev.terminal, ev.direction = True, -1
    sol = integrate.solve_ivp(lambda t, y: [y[1], -ax], (0, 1e-6), [0.0, v0], events=ev,
                              rtol=1e-12, atol=1e-30, max_step=1e-12, first_step=1e-15)
    t_land = sol.t_events[0][0]
    assert oracle.time_of_flight(A0, ax) == pytest.approx(t_land, rel=1e-6)


def test_sigma_eq20_from_cosine_averaged_kinematics():
    """Eq. 20 is Eq. 19 with the squared normal emission speed averaged over
    the cosine law (<cos^2> = 1/2 by quadrature), E_x = sigma/(2 eps0) and
    a_x/a_y = E_x/E_y.  Solve Eq. 19 for sigma by root finding."""
    num, _ = integrate.quad(lambda t: math.cos(t) ** 2 * math.cos(t) * math.sin(t), 0, math.pi / 2)
    den, _ = integrate.quad(lambda t: math.cos(t) * math.sin(t), 0, math.pi / 2)
    c2 = num / den
    A0 = 2.0
    A1 = oracle.first_crossover(3.0, 400.0)
    for Ey in (-5e5, -1e6, -3e6):
        ay = QE * abs(Ey) / ME

        def residual(sig):
            ax = QE * sig / (2 * EPS0) / ME
            vn2 = 2 * A0 * QE / ME * c2  # averaged squared normal speed
            t = 2 * math.sqrt(vn2) / ax
            l_ef = 0.5 * ay * t * t
            return 2 / ME * (A1 - A0) * QE - 2 * ay * l_ef  # Eq. 19 in SI

        sig = optimize.brentq(residual, 1e-9, 1.0, xtol=1e-20, rtol=1e-14)
        assert oracle.sigma_eq20(Ey, A0, A1) == pytest.approx(sig, rel=1e-9)


def test_fowler_nordheim_matches_the_published_fn_constants():
    """Eq. 6 with W = e phi equals a E^2 / phi exp(-b phi^1.5 / E) with the
    first and second Fowler-Nordheim constants a = 1.541434e-6 A eV V^-2 and
    b = 6.830890e9 eV^-1.5 V m^-1 (Forbes and Deane, Proc. R. Soc. A 2007)."""
    a, b = 1.541434e-6, 6.830890e9
    for E in (1e6, 5e6, 1e9, 5e9, 2e10):
        for phi in (2.0, 4.08, 4.5, 5.5):
            ref = math.log(a) + 2 * math.log(E) - math.log(phi) - b * phi ** 1.5 / E
            got = oracle.fn_log_current(E, phi)
            assert abs(got - ref) <= 2e-6 * abs(b * phi ** 1.5 / E) + 1e-6, (E, phi, got, ref)


def test_fowler_nordheim_underflows_at_the_papers_field():
    """With E_CTJ = |E_y| = 5 MV/m and phi = 4.08 V the exponent is about
    -1.13e4: J = exp(ln J) is exactly 0 in FP64 (the reason a constant J
    stands in for Eq. 6)."""
    lj = oracle.fn_log_current(5e6, 4.08)
    assert -11300 < lj < -11200
    assert math.exp(lj) == 0.0


# ---- electron-electron BGK collisions (Eqs. 3-5)
def nrl_nu(n_m3, T_eV, ln_lambda):
    """The NRL Plasma Formulary's electron collision rate
    nu_e = 2.91e-6 n[cm^-3] lnL T_e[eV]^-1.5 / s; Eq. 4 is that rate divided
    by sqrt(2)."""
    return 2.91e-6 * (n_m3 * 1e-6) * ln_lambda * T_eV ** -1.5 / math.sqrt(2.0)


def test_nu_ee_matches_the_published_rate():
    for n in (1e12, 1e16, 3e19):
        for T in (0.5, 2.0, 40.0):
            for L in (5.0, 10.0):
                assert oracle.nu_ee(n, T, L) == pytest.approx(nrl_nu(n, T, L), rel=5e-3)


def maxwellian(v1, v2, T_eV, dv1, dv2):
    """Eq. 5 on the grid (no drift), scaled to unit density by its own sum."""
    T = T_eV * QE
    g = np.exp(-ME * (v1[:, None] ** 2 + v2[None, :] ** 2) / (2 * T))
    return g / (g.sum() * dv1 * dv2)


def bgk_pair(shape, f0, sigma, lnL, T_e=2.0):
    """One step with collisions and one without, from the same state."""
    nx, nv1, nv2 = shape
    out = []
    for on in (True, False):
        o = oracle.Oracle(nx, nv1, nv2, 20e-6, -6e7, 6e7, -3e7, 3e7, cfl=0.3)
        o.set_fields(-1e6)
        o.set_collisions(T_e, lnL, on)
        o.set_state(f0, sigma)
        assert o.courant_sum() <= 1.0
        ne_before, _, _, _ = o.moments()
        o.step(1)
        out.append((o.get_f(), o.moments()[0], ne_before, o.info()))
        o.close()
    return out


def grid_v(shape):
    nx, nv1, nv2 = shape
    dv1, dv2 = 12e7 / nv1, 6e7 / nv2
    v1 = -6e7 + (np.arange(nv1) + 0.5) * dv1
    v2 = -3e7 + (np.arange(nv2) + 0.5) * dv2
    return v1, v2, dv1, dv2


def test_bgk_keeps_every_plane_density():
    shape = (6, 20, 18)
    f0 = synth.random_f(shape, 3, 1e-2)
    (f_on, n_on, nb, info), (f_off, n_off, _, _) = bgk_pair(shape, f0, 0.0, lnL=1e10)
    dt = info["dt"]
    # the collision term is large enough to matter
    assert nrl_nu(nb.max(), 2.0, 1e10) * dt > 1e-3
    assert np.abs(f_on - f_off).max() > 1e-3 * np.abs(f_off).max()
    # but it moves no density between planes or out of them
    assert np.allclose(n_on, n_off, rtol=1e-12, atol=0)


def test_bgk_leaves_the_equilibrium_unchanged_and_relaxes_others():
    shape = (5, 24, 22)
    v1, v2, dv1, dv2 = grid_v(shape)
    M = maxwellian(v1, v2, 2.0, dv1, dv2)
    amp = np.array([1.0, 2.0, 0.5, 3.0, 1.5])[:, None, None] * 1e13
    f_eq = amp * M[None]
    (f_on, _, nb, info), (f_off, _, _, _) = bgk_pair(shape, f_eq, 0.0, lnL=1e9)
    scale = np.abs(f_off).max()
    assert np.abs(f_on - f_off).max() <= 1e-12 * scale
    # a Maxwellian at another temperature relaxes toward M at T_e, by
    # dt nu (n M - f) in one forward-Euler step
    M8 = maxwellian(v1, v2, 8.0, dv1, dv2)
    f_hot = amp * M8[None]
    (f_on, _, nb, info), (f_off, _, _, _) = bgk_pair(shape, f_hot, 0.0, lnL=1e9)
    dt = info["dt"]
    for k in range(shape[0]):
        expect = dt * nrl_nu(nb[k], 2.0, 1e9) * (nb[k] * M - f_hot[k])
        got = f_on[k] - f_off[k]
        assert np.abs(got - expect).max() <= 6e-3 * np.abs(expect).max()


# ---- electron reflection at the dielectric (R_f, Sec. 2 after Eq. 17)
def test_reflection_ledger_and_charge():
    """With R_f the wall returns R_f of each incident flux element at the
    mirrored velocity: the wall inflow equals the secondaries plus R_f times
    the primary flux, the electron ledger still closes, and only the absorbed
    part (1 - R_f) charges the surface."""
    Rf = 0.35
    o, f0, sigma, p = _strong_case(14, 12, 10, seed=8)
    o.set_reflection(Rf)
    o.set_state(f0, sigma)
    o.step(50)
    L = o.ledger()
    rhs = L["emit"] - L["pe"] - L["vac"] - L["lv"] + L["inj"]
    scale = max(abs(L["emit"]), abs(L["pe"]), abs(L["vac"]), abs(L["lv"]), abs(L["inj"]), L["N"])
    assert abs((L["N"] - L["N0"]) - rhs) < 1e-12 * scale
    assert L["emit"] == pytest.approx(L["see"] + Rf * L["pe"], rel=1e-12)
    dsig = o.surface_charge() - L["sigma0"]
    assert dsig / QE == pytest.approx(L["see"] - (1 - Rf) * L["pe"], rel=1e-11)


def test_full_reflection_leaves_the_charge_and_zero_reflection_changes_nothing():
    o, f0, sigma, p = _strong_case(10, 12, 8, seed=9)
    o.set_reflection(1.0)
    o.set_state(f0, sigma)
    o.step(20)
    assert o.surface_charge() == sigma
    L = o.ledger()
    assert L["see"] == 0.0 and L["emit"] == pytest.approx(L["pe"], rel=1e-12)
    a, _, _, _ = _strong_case(10, 12, 8, seed=9)
    b, _, _, _ = _strong_case(10, 12, 8, seed=9)
    b.set_reflection(0.0)
    for x in (a, b):
        x.set_state(f0, sigma)
        x.step(7)
    assert np.array_equal(a.get_f(), b.get_f())


def test_reflection_needs_a_symmetric_v1_grid():
    o = Oracle(8, 6, 6, 20e-6, -5e7, 6e7, -3e7, 3e7)
    with pytest.raises(oracle.OracleError):
        o.set_reflection(0.5)
    o.set_reflection(0.0)
    with pytest.raises(oracle.OracleError):
        Oracle(8, 6, 6, 20e-6, -6e7, 6e7, -3e7, 3e7).set_reflection(1.5)


# ---- Lie splitting (x, then velocity)
def test_lie_equals_unsplit_without_velocity_terms():
    h = 20e-6
    f0 = np.random.default_rng(3).uniform(size=(9, 10, 8)) * 1e10
    out = []
    for scheme in (0, 1):
        o = Oracle(9, 10, 8, h, -6e7, 6e7, -3e7, 3e7, cfl=0.4)
        o.set_fields(0.0, False, 0.0)          # no force: no v1 or v2 advection
        o.set_see(3.0, 400.0, 1.0, 400.0)     # wall inflow active
        o.set_scheme(scheme)
        o.set_state(f0, 0.0)
        o.step(3)
        out.append(o.get_f())
    assert np.array_equal(out[0], out[1])


def test_lie_splitting_error_is_second_order():
    """With X f = f - dt (A f + b) and V g = g - dt (B g - s), Lie gives
    V X f = (unsplit step) + dt^2 B (A f + b): the difference from the
    unsplit step scales exactly as dt^2."""
    nx, nv1, nv2 = 10, 12, 10
    o0, f0, sigma, p = _strong_case(nx, nv1, nv2, seed=21)
    diffs = []
    for scale in (1.0, 0.5):
        res = []
        for scheme in (0, 1):
            o = Oracle(nx, nv1, nv2, 20e-6, -6e7, 6e7, -3e7, 3e7, dt=p["dt"] * scale)
            o.set_fields(p["Ey"], True, 0.0)
            o.set_see(3.0, 400.0, 1.0, 400.0)
            o.set_source(p["J"], p["x_lo"], p["x_hi"], 300.0)
            o.set_scheme(scheme)
            o.set_state(f0, sigma)
            o.step(1)
            res.append(o.get_f())
        d = res[1] - res[0]
        assert np.abs(d).max() > 1e-6 * np.abs(res[0]).max()  # the schemes differ
        diffs.append(d)
    ratio = np.linalg.norm(diffs[0]) / np.linalg.norm(diffs[1])
    assert ratio == pytest.approx(4.0, rel=1e-8)
    assert np.allclose(diffs[0], 4.0 * diffs[1], rtol=1e-7, atol=1e-9 * np.abs(diffs[0]).max())


def test_lie_ledger_closes():
    o, f0, sigma, p = _strong_case(14, 12, 10, seed=22)
    o.set_scheme(1)
    o.set_state(f0, sigma)
    o.step(40)
    L = o.ledger()
    rhs = L["emit"] - L["pe"] - L["vac"] - L["lv"] + L["inj"]
    scale = max(abs(L["emit"]), abs(L["pe"]), abs(L["vac"]), abs(L["lv"]), abs(L["inj"]), L["N"])
    assert abs((L["N"] - L["N0"]) - rhs) < 1e-12 * scale
    dsig = o.surface_charge() - L["sigma0"]
    assert dsig / QE == pytest.approx(L["see"] - L["pe"], rel=1e-12)


# ---- Strang splitting (x over dt/2, velocity over dt, x over dt/2)
def test_strang_without_velocity_terms_is_two_half_steps():
    """With no force, source or collisions the velocity step is the
    identity, and a Strang step is two x-advection steps of dt/2, each with
    the wall fluxes of its own input: exactly two unsplit steps of dt/2."""
    h = 20e-6
    nx, nv1, nv2 = 9, 10, 8
    f0 = np.random.default_rng(4).uniform(size=(nx, nv1, nv2)) * 1e10
    ref = Oracle(nx, nv1, nv2, h, -6e7, 6e7, -3e7, 3e7, cfl=0.4)
    dt = ref.info()["dt"]
    out = []
    for scheme, step_dt, n in ((2, dt, 3), (0, 0.5 * dt, 6)):
        o = Oracle(nx, nv1, nv2, h, -6e7, 6e7, -3e7, 3e7, dt=step_dt)
        o.set_fields(0.0, False, 0.0)
        o.set_see(3.0, 400.0, 1.0, 400.0)
        o.set_reflection(0.3)
        o.set_scheme(scheme)
        o.set_state(f0, 1e-6)
        o.step(n)
        out.append((o.get_f(), o.surface_charge(), o.ledger()))
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    for key in ("emit", "see", "pe", "vac"):
        assert out[0][2][key] == out[1][2][key], key


def _dense_generators(f, sigma, tabs, grid, p):
    """Generators of the two sub-steps as matrices and a vector: the x pass
    over h is f + h Ax f (Eq. 15 inflow built from the pass's own input), the
    velocity pass over h is g + h (Av g + s) with the fields of f."""
    nx, nv1, nv2 = f.shape
    x, v1, v2 = grid
    dx, dv1, dv2 = p["dx"], p["dv1"], p["dv2"]
    delta, gse, gfe = tabs
    N = f.size
    L = lambda k, i, j: (k * nv1 + i) * nv2 + j
    ne = f.sum(axis=(1, 2)) * dv1 * dv2
    ex, _ = _poisson_fd(ne, sigma, dx)
    a1 = -QE * ex / ME
    a2 = -QE * p["Ey"] / ME
    Ax = np.zeros((N, N))
    Av = np.zeros((N, N))
    s = np.zeros(N)
    r_see = np.zeros(N)
    for i in range(nv1):
        for j in range(nv2):
            if v1[i] < 0:
                r_see[L(0, i, j)] = delta[i, j] * (-v1[i]) * dv1 * dv2

    def add_face(A, lo, hi, row, scale):
        if lo is not None:
            A[lo] -= scale * row
        if hi is not None:
            A[hi] += scale * row

    for kf in range(nx + 1):
        for i in range(nv1):
            for j in range(nv2):
                row = np.zeros(N)
                if v1[i] > 0:
                    row = v1[i] * gse[i, j] * r_see if kf == 0 else _unit(N, L(kf - 1, i, j)) * v1[i]
                elif v1[i] < 0 and kf < nx:
                    row = _unit(N, L(kf, i, j)) * v1[i]
                add_face(Ax, L(kf - 1, i, j) if kf > 0 else None, L(kf, i, j) if kf < nx else None,
                         row, 1.0 / dx)
    for k in range(nx):
        for jf in range(nv2 + 1):
            for i in range(nv1):
                row = np.zeros(N)
                if a2 > 0 and jf > 0:
                    row = _unit(N, L(k, i, jf - 1)) * a2
                elif a2 < 0 and jf < nv2:
                    row = _unit(N, L(k, i, jf)) * a2
                add_face(Av, L(k, i, jf - 1) if jf > 0 else None, L(k, i, jf) if jf < nv2 else None,
                         row, 1.0 / dv2)
        for iface in range(nv1 + 1):
            for j in range(nv2):
                row = np.zeros(N)
                if a1[k] > 0 and iface > 0:
                    row = _unit(N, L(k, iface - 1, j)) * a1[k]
                elif a1[k] < 0 and iface < nv1:
                    row = _unit(N, L(k, iface, j)) * a1[k]
                add_face(Av, L(k, iface - 1, j) if iface > 0 else None,
                         L(k, iface, j) if iface < nv1 else None, row, 1.0 / dv1)
    band = [k for k in range(nx) if p["x_lo"] <= x[k] <= p["x_hi"]]
    for k in band:
        for i in range(nv1):
            for j in range(nv2):
                s[L(k, i, j)] += p["J"] / QE / (len(band) * dx) * gfe[i, j]
    return Ax, Av, s


def _wall_charge_rate(f, tabs, grid, p):
    delta = tabs[0]
    v1 = grid[1]
    return sum((delta[i, j] - 1.0) * (-v1[i]) * f[0, i, j] * p["dv1"] * p["dv2"]
               for i in range(f.shape[1]) if v1[i] < 0 for j in range(f.shape[2]))


def test_strang_dense_matrix_brute_force():
    o, f0, sigma, p = _strong_case(4, 4, 5, seed=7)
    o.set_scheme(2)
    o.set_state(f0, sigma)
    assert o.courant_sum() <= 1.0
    tabs, grid = o.tables(), o.grid()
    dt = p["dt"]
    f, s = f0.copy(), sigma
    for _ in range(4):
        Ax, Av, src = _dense_generators(f, s, tabs, grid, p)
        f1 = f.ravel() + 0.5 * dt * (Ax @ f.ravel())
        f2 = f1 + dt * (Av @ f1 + src)
        f3 = f2 + 0.5 * dt * (Ax @ f2)
        s = s + QE * 0.5 * dt * (_wall_charge_rate(f, tabs, grid, p) +
                                 _wall_charge_rate(f2.reshape(f.shape), tabs, grid, p))
        f = f3.reshape(f.shape)
    o.step(4)
    assert np.abs(o.get_f() - f).sum() / np.abs(f).sum() < 1e-13
    assert o.surface_charge() == pytest.approx(s, rel=1e-12)
    # a step that differs from both the unsplit and the Lie step
    res = {}
    for scheme in (0, 1, 2):
        q = Oracle(4, 4, 5, 20e-6, -6e7, 6e7, -3e7, 3e7, cfl=0.4)
        q.set_fields(p["Ey"], True, 0.0)
        q.set_see(3.0, 400.0, 1.0, 400.0)
        q.set_source(p["J"], p["x_lo"], p["x_hi"], 300.0)
        q.set_scheme(scheme)
        q.set_state(f0, sigma)
        q.step(1)
        res[scheme] = q.get_f()
    for other in (0, 1):
        assert np.abs(res[2] - res[other]).max() > 1e-6 * np.abs(res[other]).max()


def test_strang_ledger_and_charge_close():
    """Without collisions (whose split form uses the density of f^n on the
    intermediate state, R13/R14) the electron and charge balance close."""
    o, f0, sigma, p = _strong_case(14, 12, 10, seed=23)
    o.set_reflection(0.25)
    o.set_scheme(2)
    o.set_state(f0, sigma)
    assert o.courant_sum() <= 1.0
    o.step(40)
    L = o.ledger()
    rhs = L["emit"] - L["pe"] - L["vac"] - L["lv"] + L["inj"]
    scale = max(abs(L["emit"]), abs(L["pe"]), abs(L["vac"]), abs(L["lv"]), abs(L["inj"]), L["N"])
    assert abs((L["N"] - L["N0"]) - rhs) < 1e-12 * scale
    dsig = o.surface_charge() - L["sigma0"]
    # R12: only the absorbed (1 - R_f) part of the incident flux deposits charge
    assert dsig / QE == pytest.approx(L["see"] - 0.75 * L["pe"], rel=1e-10)
    with pytest.raises(oracle.OracleError):
        o.set_scheme(3)


# ------------------------------------------------------- threaded oracle build
@pytest.mark.parametrize("scheme", [0, 1, 2])
def test_openmp_build_equals_serial_build_bitwise(scheme):
    """The OpenMP build runs the loops over x-planes on several threads and
    adds per-plane partials in plane order, as the serial build does: both
    give the same bits for f, sigma, the ledger and the history, for every
    time scheme, with every term of the step active."""
    shape = (12, 10, 12)
    f0 = synth.random_f(shape, 5, 1e3)
    # Coulomb logarithm scaled so that dt nu_ee is about 2 % on the densest plane
    probe = Oracle(*shape, 20e-6, -6e7, 6e7, -3e7, 3e7, cfl=0.4)
    probe.set_state(f0, 0.0)
    n_max, dt = probe.moments()[0].max(), probe.info()["dt"]
    ln_lambda = 10.0 * 0.02 / (dt * oracle.nu_ee(n_max, 2.0, 10.0))
    runs = []
    for th in (None, 3):
        o = Oracle(*shape, 20e-6, -6e7, 6e7, -3e7, 3e7, cfl=0.4, threads=th)
        o.set_fields(-1e6)
        o.set_see(3.0, 400.0, 1.0, 2.0)
        o.set_source(1e7, 10e-6, 15e-6, 4.0)
        o.set_collisions(2.0, ln_lambda, True)
        o.set_scheme(scheme)
        o.set_state(f0, 2e-6)
        o.step(25)
        runs.append((o.get_f(), o.surface_charge(), o.ledger(), o.history()))
        assert o.threads == (1 if th is None else 3)
    (fa, sa, la, ha), (fb, sb, lb, hb) = runs
    assert np.array_equal(fa, fb)
    assert sa == sb
    assert la == lb
    assert np.array_equal(ha, hb)


@pytest.mark.parametrize("scheme", [1, 2])
def test_split_schemes_agree_with_the_unsplit_step_to_first_order(scheme):
    """Lie (R13) and Strang (R14) splitting with the self-consistent field,
    SEE and the source on: one step differs from the unsplit step by O(dt^2)
    (halving dt quarters the difference) and a fixed time by O(dt) (halving
    dt halves it).  Every sub-step is a forward-Euler step, so all three
    schemes are first order in time; the velocity pass taking E_x from f^n
    does not lower that order."""
    shape = (12, 16, 14)
    f0 = synth.random_f(shape, 3, 1e4)

    def run(s, dt, n):
        o = Oracle(*shape, 20e-6, -6e7, 6e7, -3e7, 3e7, dt=dt)
        o.set_fields(-2e6, True, 0.0)
        o.set_see(3.0, 400.0, 1.0, 2.0)
        o.set_source(1e7, 4e-6, 14e-6, 4.0)
        o.set_scheme(s)
        o.set_state(f0, 2e-6)
        o.step(n)
        return o.get_f()

    dt0 = Oracle(*shape, 20e-6, -6e7, 6e7, -3e7, 3e7, cfl=0.4).info()["dt"]
    per_step, fixed_time = [], []
    for k in range(3):
        dt = dt0 / 2 ** k
        fs, fu = run(scheme, dt, 1), run(0, dt, 1)
        per_step.append(np.abs(fs - fu).sum() / np.abs(fu).sum())
        fs, fu = run(scheme, dt, 8 * 2 ** k), run(0, dt, 8 * 2 ** k)
        fixed_time.append(np.abs(fs - fu).sum() / np.abs(fu).sum())
    for a, b in zip(per_step, per_step[1:]):
        assert 3.6 < a / b < 4.4
    for a, b in zip(fixed_time, fixed_time[1:]):
        assert 1.8 < a / b < 2.4
