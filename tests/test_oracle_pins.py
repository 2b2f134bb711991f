"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test compares the oracle with something that is not the oracle: exact
solutions of the NLSE, closed-form discrete spectra, brute force over the
paper's printed stencil tables, polynomial exactness, numbers printed in the
paper, invariants.  Chosen so that a dropped term, a wrong sign or index or a
transposed operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1203_1263_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel_l2(x, ref):
    return float(np.linalg.norm(np.ravel(x - ref)) / np.linalg.norm(np.ravel(ref)))


def rk4_amplification(z):
    """Classic RK4 applied to y' = lambda y multiplies y by 1 + z + z^2/2 + z^3/6 + z^4/24, z = lambda dt."""
    return 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24


def cd_symbol(theta, h):
    """Eigenvalue of the 3-point second difference on exp(i theta j) or sin(theta j)."""
    return -(4.0 / (h * h)) * math.sin(theta / 2) ** 2


# ---------------------------------------------------------------------------
# P1, P2: exact solitons and spatial convergence orders
# ---------------------------------------------------------------------------

def _orders(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("order,expect,tol", [(2, 2.0, 0.15), (4, 4.0, 0.3)])
def test_bright_soliton_convergence(order, expect, tol):
    """Moving bright soliton (exact solution), Dirichlet walls far away."""
    errs = []
    for n in (501, 1001, 2001):
        p = W.bright_soliton_1d(order=order, n=n, t_end=2.0)
        out, _ = O.run_problem(p)
        exact = W.bright_soliton(p.extra["x"], p.extra["t_end"])
        errs.append(rel_l2(out, exact))
    for o in _orders(errs):
        assert abs(o - expect) < tol, (errs, _orders(errs))
    assert errs[-1] < (2e-3 if order == 2 else 3e-6)


@pytest.mark.parametrize("order,expect,tol", [(2, 2.0, 0.15), (4, 4.0, 0.3)])
def test_dark_soliton_msd_convergence(order, expect, tol):
    """The paper's co-moving dark soliton (Sec. 4, Eq. soliton) with the MSD wall."""
    errs = []
    for h in (0.2, 0.1, 0.05):
        p = W.dark_soliton_1d(order=order, h=h, L=30.0, t_end=2.0)
        out, _ = O.run_problem(p)
        exact = W.dark_soliton(p.extra["x"], p.extra["t_end"])
        errs.append(rel_l2(out, exact))
    for o in _orders(errs):
        assert abs(o - expect) < tol, (errs, _orders(errs))


def stationary_dark(x, a, s, kappa):
    """A tanh(kappa x) with A^2 = -2 a kappa^2 / s solves a psi'' - V0 psi + s|psi|^2 psi = 0
    for the constant potential V0 = -2 a kappa^2 (s < 0): a time-independent exact
    solution, so fixed (Dirichlet) walls are exact wherever they are placed."""
    return math.sqrt(-2.0 * a * kappa * kappa / s) * np.tanh(kappa * x)


@pytest.mark.parametrize("order,expect,tol", [(2, 2.0, 0.2), (4, 4.0, 0.35)])
@pytest.mark.parametrize("dims,axis", [(1, 0), (2, 0), (2, 1), (3, 2)])
def test_stationary_dark_soliton_dirichlet(order, expect, tol, dims, axis):
    """Walls at kappa x = -1.2 and 1.8, inside the core, so the Dirichlet
    Laplacian form (Eq. BCDlap) carries a non-zero Laplacian into 2SHOC."""
    a, s, kappa, T = 0.8, -1.0, 1.0, 0.5
    errs = []
    for h in (0.1, 0.05, 0.025):
        n = int(round(3.0 / h)) + 1
        x = -1.2 + h * np.arange(n)
        prof = stationary_dark(x, a, s, kappa)
        shape = [5] * dims
        shape[axis] = n
        sh = [1] * dims
        sh[axis] = n
        psi0 = np.ascontiguousarray(np.broadcast_to(prof.reshape(sh), shape)).astype(np.complex128)
        V = np.full(shape, -2.0 * a * kappa * kappa)
        dt = h * h / 8.0
        out = O.rk4(psi0, h, a, s, dt, int(round(T / dt)), V, W.BC_DIRICHLET, order)
        errs.append(rel_l2(out, psi0))
    # With 5-point transverse Dirichlet walls the interior is pinned hard, so
    # more than the scheme's order may show; never less.
    for o in _orders(errs):
        assert o > expect - tol, (errs, _orders(errs))
    assert errs[-1] < (1e-4 if order == 2 else 1e-7)


# ---------------------------------------------------------------------------
# P3: linear sine modes are exact discrete eigenfunctions
# ---------------------------------------------------------------------------

SINE_CASES = [((41,), (3,)), ((21, 17), (2, 5)), ((11, 13, 9), (2, 3, 1))]


@pytest.mark.parametrize("shape,modes", SINE_CASES)
@pytest.mark.parametrize("order", [2, 4])
def test_sine_modes_exact_rk4(shape, modes, order):
    """s = 0, V = 0, Dirichlet zero walls: Psi^n = R(i a dt lambda)^n Psi^0 where
    lambda = sum sigma (CD) or sum (sigma - h^2 sigma^2 / 12) (2SHOC)."""
    h, a, dt, n = 0.3, 0.7, 0.004, 25
    sig = [cd_symbol(math.pi * m / (N - 1), h) for N, m in zip(shape, modes)]
    lam = sum(sig) if order == 2 else sum(s_ - h * h * s_ * s_ / 12 for s_ in sig)
    psi0 = W.sine_mode(shape, modes)
    out = O.rk4(psi0, h, a, 0.0, dt, n, None, W.BC_DIRICHLET, order)
    expect = rk4_amplification(1j * a * dt * lam) ** n * psi0
    assert rel_l2(out, expect) < 1e-13


@pytest.mark.parametrize("shape,modes", SINE_CASES)
@pytest.mark.parametrize("order", [2, 4])
def test_sine_mode_laplacian_eigenvalue(shape, modes, order):
    h = 0.25
    sig = [cd_symbol(math.pi * m / (N - 1), h) for N, m in zip(shape, modes)]
    lam = sum(sig) if order == 2 else sum(s_ - h * h * s_ * s_ / 12 for s_ in sig)
    psi0 = W.sine_mode(shape, modes)
    D, L = O.laplacian(psi0, h, 1.0, 0.0, None, W.BC_DIRICHLET, order)
    inner = tuple(slice(1, -1) for _ in shape)
    assert np.max(np.abs(L[inner] - lam * psi0[inner])) < 1e-11 * abs(lam)


def test_temporal_order_four():
    """Global RK4 error against the semi-discrete solution exp(i a lambda t) falls as dt^4."""
    shape, modes, h, a, T = (33,), (5,), 0.2, 1.0, 0.5
    lam = cd_symbol(math.pi * modes[0] / (shape[0] - 1), h)
    psi0 = W.sine_mode(shape, modes)
    errs = []
    for nsteps in (40, 80, 160):
        dt = T / nsteps
        out = O.rk4(psi0, h, a, 0.0, dt, nsteps, None, W.BC_DIRICHLET, 2)
        errs.append(rel_l2(out, np.exp(1j * a * lam * T) * psi0))
    for o in _orders(errs):
        assert abs(o - 4.0) < 0.1, errs


# ---------------------------------------------------------------------------
# P4: stability bound (printed values) and its sharpness
# ---------------------------------------------------------------------------

def _golden_bounds():
    rows = []
    for line in open(os.path.join(GOLDEN, "stability_bounds.txt")):
        line = line.split("#")[0].split()
        if line:
            rows.append((int(line[0]), int(line[1]), float(line[2]), float(line[3]), float(line[4]),
                         float(line[5])))
    return rows


@pytest.mark.parametrize("row", _golden_bounds())
def test_stability_bound_printed(row):
    d, order, h, a, printed, tol = row
    got = O.stability_bound(d, h, a, order)
    assert abs(got - printed) <= tol * printed, (got, printed)


@pytest.mark.parametrize("order", [2, 4])
def test_stability_bound_is_sharp(order):
    """The highest sine mode grows just above the bound and does not just below it."""
    N, h, a = 101, 0.1, 1.0
    psi0 = W.sine_mode((N,), (N - 2,))
    bound = O.stability_bound(1, h, a, order)
    above = O.rk4(psi0, h, a, 0.0, 1.02 * bound, 200, None, W.BC_DIRICHLET, order)
    below = O.rk4(psi0, h, a, 0.0, 0.98 * bound, 200, None, W.BC_DIRICHLET, order)
    n0 = np.linalg.norm(psi0)
    assert np.linalg.norm(above) > 10 * n0
    assert np.linalg.norm(below) <= n0 * (1 + 1e-12)


# ---------------------------------------------------------------------------
# P5: uniform backgrounds and plane waves under MSD follow the scalar RK4 iterate
# ---------------------------------------------------------------------------

def scalar_rk4(z, dt, nsteps, rate):
    """Classic RK4 on z' = i rate(|z|^2) z."""
    f = lambda y: 1j * rate(abs(y) ** 2) * y
    for _ in range(nsteps):
        k1 = f(z); k2 = f(z + dt / 2 * k1); k3 = f(z + dt / 2 * k2); k4 = f(z + dt * k3)
        z = z + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return z


@pytest.mark.parametrize("shape", [(9,), (7, 8), (5, 6, 7)])
@pytest.mark.parametrize("order", [2, 4])
def test_uniform_background_msd(shape, order):
    rho, phi, s, a, dt, n = 1.3, 0.4, -1.0, 0.5, 0.01, 30
    z0 = math.sqrt(rho) * complex(math.cos(phi), math.sin(phi))
    psi0 = np.full(shape, z0, dtype=np.complex128)
    out = O.rk4(psi0, 0.2, a, s, dt, n, None, W.BC_MSD, order)
    z = scalar_rk4(z0, dt, n, lambda m2: s * m2)
    assert np.max(np.abs(out - z)) < 1e-13


@pytest.mark.parametrize("shape,k", [((12,), (0.9,)), ((10, 11), (0.7, -0.4)), ((8, 9, 10), (0.6, -0.5, 0.3))])
@pytest.mark.parametrize("order", [2, 4])
def test_plane_wave_msd(shape, k, order):
    """sqrt(rho) exp(i k.x) is an exact discrete solution under MSD: every site is
    z_n exp(i k.x) with z' = i(a lambda_k + s|z|^2) z.  Pins the MSD time-derivative
    form at faces, edges and corners and, for 2SHOC, the MSD Laplacian form."""
    h, rho, s, a, dt, n = 0.3, 0.8, 1.0, 0.6, 0.003, 40
    sig = [cd_symbol(kk * h, h) for kk in k]
    lam = sum(sig) if order == 2 else sum(s_ - h * h * s_ * s_ / 12 for s_ in sig)
    grids = np.meshgrid(*[np.arange(N) * h for N in shape], indexing="ij")
    phase = np.exp(1j * sum(kk * g for kk, g in zip(k, grids)))
    psi0 = math.sqrt(rho) * phase
    out = O.rk4(psi0, h, a, s, dt, n, None, W.BC_MSD, order)
    z = scalar_rk4(complex(math.sqrt(rho)), dt, n, lambda m2: a * lam + s * m2)
    assert np.max(np.abs(out - z * phase)) < 1e-12


# ---------------------------------------------------------------------------
# Laplacian-zero boundary (Sec. 3.3, Eqs. BCL0dt and BCL0lap)
# ---------------------------------------------------------------------------

def _boundary_mask(shape):
    m = np.zeros(shape, dtype=bool)
    for ax in range(len(shape)):
        idx = [slice(None)] * len(shape)
        idx[ax] = 0
        m[tuple(idx)] = True
        idx[ax] = -1
        m[tuple(idx)] = True
    return m


def scalar_rk4_array(z, dt, nsteps, rate):
    """scalar_rk4 applied elementwise to an array of initial values."""
    f = lambda y: 1j * rate(np.abs(y) ** 2) * y
    for _ in range(nsteps):
        k1 = f(z); k2 = f(z + dt / 2 * k1); k3 = f(z + dt / 2 * k2); k4 = f(z + dt * k3)
        z = z + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    return z


@pytest.mark.parametrize("shape", [(10,), (7, 9), (6, 7, 8)])
@pytest.mark.parametrize("order", [2, 4])
def test_l0_boundary_sites_follow_their_own_ode(shape, order):
    """Under L0 the time derivative at a boundary site involves that site alone
    (Eq. BCL0dt), so whatever the interior does, every boundary site is the
    scalar RK4 iterate of z' = i(s|z|^2 - V_b) z from its own initial value."""
    h, a, s, dt, n = 0.3, 0.7, 1.2, 0.002, 20
    psi = W.random_field(shape, seed=51)
    V = W.random_potential(shape, seed=52, scale=2.0)
    out = O.rk4(psi, h, a, s, dt, n, V, W.BC_L0, order)
    b = _boundary_mask(shape)
    Vb = V[b]
    expect = scalar_rk4_array(psi[b], dt, n, lambda m2: s * m2 - Vb)
    assert np.max(np.abs(out[b] - expect)) < 1e-13
    assert np.max(np.abs(out[~b] - psi[~b])) > 1e-3          # the interior moved


def _multilinear_field(shape, h, seed):
    """A complex combination of the monomials prod_{k in S} x_k (S any subset of
    the axes).  Each is harmonic, and every central second difference of it
    vanishes exactly, so the CD and 2SHOC Laplacians of it are 0 at every
    interior site, provided the boundary Laplacian is 0."""
    axes = [np.arange(N) * h - 0.5 * (N - 1) * h for N in shape]
    grids = np.meshgrid(*axes, indexing="ij")
    d = len(shape)
    c = W.random_field((2 ** d,), seed=seed)
    psi = np.zeros(shape, dtype=np.complex128)
    for m in range(2 ** d):
        term = np.ones(shape)
        for k in range(d):
            if m >> k & 1:
                term = term * grids[k]
        psi += c[m] * term
    return psi


@pytest.mark.parametrize("shape", [(11,), (8, 9), (6, 7, 8)])
@pytest.mark.parametrize("order", [2, 4])
def test_l0_harmonic_field_in_constant_potential(shape, order):
    """s = 0, V = V0: with D_b = 0 (Eq. BCL0lap) every Laplacian of a multilinear
    field is 0, so each site, boundary ones included (Eq. BCL0dt), is multiplied
    by R(-i V0 dt) per step.  Dirichlet's D_b = V0 Psi_b / a (and its F_b = 0)
    would not give this."""
    h, a, V0, dt, n = 0.25, 0.9, 0.7, 0.01, 25
    psi = _multilinear_field(shape, h, seed=53)
    V = np.full(shape, V0)
    out = O.rk4(psi, h, a, 0.0, dt, n, V, W.BC_L0, order)
    expect = psi * rk4_amplification(-1j * V0 * dt) ** n
    assert np.max(np.abs(out - expect)) < 1e-13 * np.max(np.abs(psi))
    assert np.max(np.abs(O.rk4(psi, h, a, 0.0, dt, n, V, W.BC_DIRICHLET, order) - expect)) > 1e-4
    # the energy density reduces to V0 |Psi|^2 on the interior
    inner = tuple(slice(1, -1) for _ in shape)
    e = h ** len(shape) * math.fsum((V0 * np.abs(psi[inner]) ** 2).ravel().tolist())
    assert abs(O.energy(psi, h, a, 0.0, V, W.BC_L0, order) - e) < 1e-12 * abs(e)


@pytest.mark.parametrize("shape", [(9,), (7, 8), (5, 6, 7)])
@pytest.mark.parametrize("order", [2, 4])
def test_uniform_background_l0(shape, order):
    rho, phi, s, a, dt, n = 0.9, -0.7, 1.0, 0.8, 0.01, 30
    z0 = math.sqrt(rho) * complex(math.cos(phi), math.sin(phi))
    out = O.rk4(np.full(shape, z0, dtype=np.complex128), 0.2, a, s, dt, n, None, W.BC_L0, order)
    assert np.max(np.abs(out - scalar_rk4(z0, dt, n, lambda m2: s * m2))) < 1e-13


@pytest.mark.parametrize("shape", [(12,), (8, 9), (5, 6, 7)])
@pytest.mark.parametrize("order", [2, 4])
def test_l0_is_dirichlet_for_the_free_linear_equation(shape, order):
    """With s = 0 and V = 0 both boundary forms reduce to F_b = 0 and D_b = 0."""
    psi = W.random_field(shape, seed=54)
    a1 = O.rk4(psi, 0.3, 0.8, 0.0, 0.003, 9, None, W.BC_L0, order)
    a2 = O.rk4(psi, 0.3, 0.8, 0.0, 0.003, 9, None, W.BC_DIRICHLET, order)
    assert np.array_equal(a1, a2)


# ---------------------------------------------------------------------------
# P6: brute force over the printed stencil tables; polynomial exactness
# ---------------------------------------------------------------------------

def _frac(x):
    if "/" in x:
        a, b = x.split("/")
        return float(a) / float(b)
    return float(x)


def _tables():
    t = {}
    for line in open(os.path.join(GOLDEN, "stencils_2shoc.txt")):
        f = line.split("#")[0].split()
        if not f:
            continue
        d, step, operand, scale = int(f[0]), int(f[1]), f[2], f[3]
        off = tuple(int(v) for v in f[4:4 + d])
        w = _frac(f[4 + d])
        t.setdefault((d, step), []).append((operand, scale, off, w))
    return t


def _apply(entries, fields, h, site):
    scales = {"inv_h2": 1 / h ** 2, "m1_12": -1 / 12, "one": 1.0, "inv_6h2": 1 / (6 * h * h)}
    acc = 0.0
    for operand, scale, off, w in entries:
        idx = tuple(s_ + o for s_, o in zip(site, off))
        acc += scales[scale] * w * fields[operand][idx]
    return acc


@pytest.mark.parametrize("shape", [(11,), (8, 9), (6, 7, 8)])
def test_stencil_tables_brute_force(shape):
    """D and the 2SHOC Laplacian equal a naive sum over the paper's tables at
    every site two or more cells from the walls."""
    tab = _tables()
    d = len(shape)
    h = 0.37
    psi = W.random_field(shape, seed=11)
    D_or, L_or = O.laplacian(psi, h, 1.0, 0.0, None, W.BC_DIRICHLET, 4)
    D_bf = np.zeros_like(psi)
    for site in np.ndindex(*shape):
        if all(0 < i < n - 1 for i, n in zip(site, shape)):
            D_bf[site] = _apply(tab[(d, 1)], {"psi": psi}, h, site)
    scale = np.max(np.abs(D_bf))
    for site in np.ndindex(*shape):
        if all(1 < i < n - 2 for i, n in zip(site, shape)):
            assert abs(D_or[site] - D_bf[site]) < 1e-13 * scale
            ref = _apply(tab[(d, 2)], {"psi": psi, "D": D_bf}, h, site)
            assert abs(L_or[site] - ref) < 1e-13 * scale, site


def _poly_field(shape, h, degree, seed):
    """Random polynomial of total degree <= degree and its exact Laplacian."""
    d = len(shape)
    u = W.uniform(seed, 64)
    coords = np.meshgrid(*[np.arange(n) * h - 0.4 for n in shape], indexing="ij")
    terms = [e for e in np.ndindex(*([degree + 1] * d)) if sum(e) <= degree]
    f = np.zeros(shape)
    lap = np.zeros(shape)
    for t_i, e in enumerate(terms):
        c = u[t_i % 64] - 0.5
        mono = np.ones(shape)
        for ax in range(d):
            mono = mono * coords[ax] ** e[ax]
        f += c * mono
        for ax in range(d):
            if e[ax] >= 2:
                m = np.ones(shape) * e[ax] * (e[ax] - 1)
                for bx in range(d):
                    m = m * coords[bx] ** (e[bx] - (2 if bx == ax else 0))
                lap += c * m
    return f, lap


@pytest.mark.parametrize("shape", [(13,), (9, 10), (7, 8, 7)])
@pytest.mark.parametrize("order,degree", [(2, 3), (4, 5)])
def test_polynomial_exactness(shape, order, degree):
    h = 0.11
    f, lap = _poly_field(shape, h, degree, seed=5)
    psi = (f + 0.5j * f).astype(np.complex128)
    _, L = O.laplacian(psi, h, 1.0, 0.0, None, W.BC_DIRICHLET, order)
    m = 2 if order == 4 else 1
    inner = tuple(slice(m, n - m) for n in shape)
    tol = 1e-9 * max(1.0, np.max(np.abs(f)) / h ** 2)
    assert np.max(np.abs(L[inner] - (lap + 0.5j * lap)[inner])) < tol
    # one degree higher is no longer exact (the test has teeth)
    f2, lap2 = _poly_field(shape, h, degree + 1, seed=6)
    _, L2 = O.laplacian(f2.astype(np.complex128), h, 1.0, 0.0, None, W.BC_DIRICHLET, order)
    assert np.max(np.abs(L2[inner].real - lap2[inner])) > 1e3 * tol


# ---------------------------------------------------------------------------
# P7, P8: mass and energy
# ---------------------------------------------------------------------------

def test_mass_closed_form_and_exact_sum():
    shape, h = (6, 7, 8), 0.3
    psi = np.full(shape, 0.5 + 0.25j)
    assert abs(O.mass(psi, h) - (0.3125 * h ** 3 * 336)) < 1e-15
    psi = W.random_field((40, 50), seed=3)
    exact = math.fsum((np.abs(psi) ** 2).ravel().tolist()) * h ** 2
    assert abs(O.mass(psi, h) - exact) <= 2e-16 * exact


@pytest.mark.parametrize("shape,modes", SINE_CASES)
@pytest.mark.parametrize("order", [2, 4])
def test_energy_closed_form(shape, modes, order):
    """For a sine mode with zero walls Lap Psi = lambda Psi, so
    E = h^d sum_interior [(-a lambda + V)|Psi|^2 - (s/2)|Psi|^4]."""
    h, a, s = 0.3, 0.7, -0.9
    sig = [cd_symbol(math.pi * m / (N - 1), h) for N, m in zip(shape, modes)]
    lam = sum(sig) if order == 2 else sum(s_ - h * h * s_ * s_ / 12 for s_ in sig)
    psi = 0.8 * W.sine_mode(shape, modes)
    V = W.random_potential(shape, seed=9, scale=2.0)
    inner = tuple(slice(1, -1) for _ in shape)
    m2 = np.abs(psi[inner]) ** 2
    terms = (-a * lam + V[inner]) * m2 - 0.5 * s * m2 * m2
    expect = h ** len(shape) * math.fsum(terms.ravel().tolist())
    got = O.energy(psi, h, a, s, V, W.BC_DIRICHLET, order)
    assert abs(got - expect) < 1e-12 * abs(expect)


@pytest.mark.parametrize("bc", [W.BC_DIRICHLET, W.BC_MSD, W.BC_L0])
def test_energy_counts_interior_sites_only(bc):
    """Every term of the energy density carries a factor of the site's own Psi,
    so a field that vanishes on the interior has zero energy whatever its walls hold."""
    shape = (6, 7, 5)
    psi = W.random_field(shape, seed=41)
    psi[1:-1, 1:-1, 1:-1] = 0
    V = W.random_potential(shape, seed=42, scale=2.0)
    assert O.energy(psi, 0.3, 0.7, 1.3, V, bc, 4) == 0.0
    assert O.energy(psi, 0.3, 0.7, 1.3, V, bc, 2) == 0.0


@pytest.mark.parametrize("order", [2, 4])
def test_mass_nonincreasing_linear_dirichlet(order):
    """s = 0, zero walls: RK4 has |R(iy)| <= 1 inside the bound, so the mass never grows."""
    shape, h, a = (12, 13), 0.2, 1.0
    psi = W.random_field(shape, seed=21)
    psi[0, :] = psi[-1, :] = psi[:, 0] = psi[:, -1] = 0
    V = W.random_potential(shape, seed=22, scale=3.0)
    dt = 0.8 * O.stability_bound(2, h, a, order, vmax=3.0)
    m_prev = O.mass(psi, h)
    for _ in range(20):
        psi = O.rk4(psi, h, a, 0.0, dt, 1, V, W.BC_DIRICHLET, order)
        m = O.mass(psi, h)
        assert m <= m_prev * (1 + 1e-14)
        m_prev = m


@pytest.mark.parametrize("order", [2, 4])
def test_bright_soliton_mass_energy_drift(order):
    """Bright soliton to t = 2 at h = 0.05, dt = h^2/8: |dM|/M <= 1e-9, |dE|/|E| <= 1e-8."""
    p = W.bright_soliton_1d(order=order, n=2001, t_end=2.0)
    out, _ = O.run_problem(p)
    M0, M1 = O.mass(p.psi0, p.h), O.mass(out, p.h)
    E0 = O.energy(p.psi0, p.h, p.a, p.s, None, p.bc, p.order)
    E1 = O.energy(out, p.h, p.a, p.s, None, p.bc, p.order)
    assert abs(M1 - M0) <= 1e-9 * M0
    assert abs(E1 - E0) <= 1e-8 * abs(E0)


# ---------------------------------------------------------------------------
# P9, P10: symmetry and split continuation
# ---------------------------------------------------------------------------

def test_vortex_rotation_symmetry():
    """Charge-1 vortex line in the axisymmetric trap on a square xy grid:
    Psi(-y, x, z) = i Psi(x, y, z) for all time."""
    p = W.trap_vortex_3d(shape=(11, 15, 15), h=0.6, noise=0.0)
    dt = 0.8 * O.stability_bound(3, p.h, p.a, 4, p.vmax(), abs(p.s) * np.max(np.abs(p.psi0)) ** 2)
    out = O.rk4(p.psi0, p.h, p.a, p.s, dt, 12, p.V, p.bc, p.order)
    n = 15
    jy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    lhs = out[:, ix, n - 1 - jy]
    rhs = 1j * out[:, jy, ix]
    assert np.max(np.abs(lhs - rhs)) < 1e-13
    assert np.max(np.abs(out - p.psi0)) > 1e-3      # it did evolve


@pytest.mark.parametrize("bc", [W.BC_DIRICHLET, W.BC_MSD, W.BC_L0, W.BC_PERIODIC])
def test_split_continuation_bitwise(bc):
    psi = W.random_field((9, 10), seed=31)
    V = W.random_potential((9, 10), seed=32)
    a1 = O.rk4(psi, 0.3, 0.8, 1.0, 0.002, 7, V, bc, 4)
    a2 = O.rk4(O.rk4(psi, 0.3, 0.8, 1.0, 0.002, 3, V, bc, 4), 0.3, 0.8, 1.0, 0.002, 4, V, bc, 4)
    assert np.array_equal(a1, a2)


# ---------------------------------------------------------------------------
# Periodic grids (the boundary of the stability analysis, Sec. 3.4): no
# boundary sites, every neighbour index taken modulo N.  Pinned by the
# discrete Fourier spectrum of both Laplacians (numpy's FFT), exact Fourier
# modes under RK4, plane waves of the cubic equation, shift invariance and
# closed-form mass and energy.
# ---------------------------------------------------------------------------

PERIODIC_SHAPES = [(16,), (9,), (8, 10), (7, 5), (6, 7, 5), (4, 6, 8)]


def fourier_symbol(shape, h, order):
    """lambda(k) of the periodic CD (order 2) or 2SHOC (order 4) Laplacian on
    the grid's discrete Fourier modes: sum_alpha sigma_alpha, or
    sum_alpha (sigma_alpha - h^2 sigma_alpha^2 / 12), sigma = -(4/h^2) sin^2(theta/2)."""
    lam = np.zeros(shape)
    for ax, n in enumerate(shape):
        theta = 2.0 * np.pi * np.fft.fftfreq(n)
        sig = -(4.0 / (h * h)) * np.sin(theta / 2) ** 2
        term = sig if order == 2 else sig - h * h * sig * sig / 12.0
        sh = [1] * len(shape)
        sh[ax] = n
        lam = lam + term.reshape(sh)
    return lam


@pytest.mark.parametrize("shape", PERIODIC_SHAPES)
@pytest.mark.parametrize("order", [2, 4])
def test_periodic_laplacian_is_its_fourier_symbol(shape, order):
    """On a random field, D (step 1) is the CD symbol and Lap the scheme's symbol, applied by FFT."""
    h = 0.3
    psi = W.random_field(shape, seed=61 + len(shape))
    D, L = O.laplacian(psi, h, 1.0, 0.0, None, W.BC_PERIODIC, order)
    fpsi = np.fft.fftn(psi)
    D_ref = np.fft.ifftn(fpsi * fourier_symbol(shape, h, 2))
    L_ref = np.fft.ifftn(fpsi * fourier_symbol(shape, h, order))
    scale = np.max(np.abs(L_ref))
    assert np.max(np.abs(D - D_ref)) < 1e-12 * scale
    assert np.max(np.abs(L - L_ref)) < 1e-12 * scale


def fourier_mode(shape, modes):
    """exp(i sum_alpha 2 pi m_alpha i_alpha / N_alpha)."""
    out = np.ones(shape, dtype=np.complex128)
    for ax, (n, m) in enumerate(zip(shape, modes)):
        v = np.exp(2j * np.pi * m * np.arange(n) / n)
        sh = [1] * len(shape)
        sh[ax] = n
        out = out * v.reshape(sh)
    return out


FOURIER_CASES = [((16,), (8,)), ((9,), (2,)), ((8, 10), (3, 5)), ((6, 7, 5), (1, 3, 2)), ((4, 6, 8), (2, 3, 4))]


@pytest.mark.parametrize("shape,modes", FOURIER_CASES)
@pytest.mark.parametrize("order", [2, 4])
def test_periodic_fourier_modes_exact_rk4(shape, modes, order):
    """s = 0, V = 0: a Fourier mode (Nyquist included) is multiplied by R(i a dt lambda) per step."""
    h, a, dt, n = 0.3, 0.7, 0.004, 25
    psi0 = fourier_mode(shape, modes)
    lam = fourier_symbol(shape, h, order)[tuple(m % N for m, N in zip(modes, shape))]
    out = O.rk4(psi0, h, a, 0.0, dt, n, None, W.BC_PERIODIC, order)
    assert rel_l2(out, rk4_amplification(1j * a * dt * lam) ** n * psi0) < 1e-13


@pytest.mark.parametrize("shape,modes", FOURIER_CASES[1:4])
@pytest.mark.parametrize("order", [2, 4])
def test_periodic_plane_wave_of_the_cubic_equation(shape, modes, order):
    """|Psi| is the same at every site of a plane wave, so each site is the
    scalar RK4 iterate of z' = i(a lambda + s|z|^2 - V0) z times the wave's phase."""
    h, a, s, V0, A, dt, n = 0.3, 0.7, -1.3, 0.4, 1.2, 0.003, 30
    phase = fourier_mode(shape, modes)
    lam = fourier_symbol(shape, h, order)[tuple(m % N for m, N in zip(modes, shape))]
    V = np.full(shape, V0)
    out = O.rk4(A * phase, h, a, s, dt, n, V, W.BC_PERIODIC, order)
    f = lambda z: 1j * (a * lam + s * abs(z) ** 2 - V0) * z
    z = complex(A)
    for _ in range(n):
        k1 = f(z); k2 = f(z + dt / 2 * k1); k3 = f(z + dt / 2 * k2); k4 = f(z + dt * k3)
        z = z + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
    assert np.max(np.abs(out - z * phase)) < 1e-13 * A


@pytest.mark.parametrize("shape", [(11,), (6, 9), (5, 4, 7)])
@pytest.mark.parametrize("order", [2, 4])
def test_periodic_grid_is_shift_invariant(shape, order):
    """A periodic grid has no distinguished site: shifting the state and the
    potential by any number of cells along any axis shifts the result, bit for bit."""
    psi = W.random_field(shape, seed=71)
    V = W.random_potential(shape, seed=72)
    out = O.rk4(psi, 0.4, 0.9, 1.1, 0.003, 6, V, W.BC_PERIODIC, order)
    for ax in range(len(shape)):
        for k in (1, 3):
            got = O.rk4(np.roll(psi, k, ax), 0.4, 0.9, 1.1, 0.003, 6, np.roll(V, k, ax), W.BC_PERIODIC, order)
            assert np.array_equal(got, np.roll(out, k, ax)), (ax, k)


@pytest.mark.parametrize("order", [2, 4])
def test_periodic_mass_and_energy_closed_form(order):
    """Every site of a plane wave counts (no boundary): M = h^d N A^2 and
    E = h^d N [-a lambda A^2 + V0 A^2 - (s/2) A^4]."""
    shape, modes, h, a, s, V0, A = (6, 7, 5), (1, 3, 2), 0.3, 0.7, -1.3, 0.4, 1.2
    psi = A * fourier_mode(shape, modes)
    lam = fourier_symbol(shape, h, order)[modes]
    n = np.prod(shape)
    assert abs(O.mass(psi, h) - h ** 3 * n * A * A) < 1e-13 * h ** 3 * n * A * A
    e = O.energy(psi, h, a, s, np.full(shape, V0), W.BC_PERIODIC, order)
    e_ref = h ** 3 * n * (-a * lam * A * A + V0 * A * A - 0.5 * s * A ** 4)
    assert abs(e - e_ref) < 1e-12 * abs(e_ref)


@pytest.mark.parametrize("order", [2, 4])
def test_periodic_linear_mass_nonincreasing(order):
    """RK4 on the imaginary axis has |R(iy)| <= 1 up to the bound, so the free
    linear flow on a periodic grid can only lose mass."""
    psi = W.random_field((12, 10), seed=81)
    h, a = 0.3, 1.0
    dt = 0.9 * O.stability_bound(2, h, a, order)
    m = [O.mass(psi, h)]
    for _ in range(5):
        psi = O.rk4(psi, h, a, 0.0, dt, 4, None, W.BC_PERIODIC, order)
        m.append(O.mass(psi, h))
    assert all(m[i + 1] <= m[i] * (1 + 1e-14) for i in range(5))
    assert m[-1] < m[0] * (1 - 1e-6)


def test_bad_arguments_rejected():
    with pytest.raises(ValueError):
        O.rk4(np.zeros((2, 5), np.complex128), 0.1, 1.0, 1.0, 0.001, 1)
    with pytest.raises(ValueError):
        O.rk4(np.zeros((5, 5), np.complex128), 0.1, 1.0, 1.0, 0.001, 1, order=3)
