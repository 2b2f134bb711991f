"""The plain-method workloads end to end on the GPU, against the oracle and
the exact solution.

  bright soliton 1D   N = 2001, h = 0.05, dt = h^2/8, 32000 steps to t = 10, CD and 2SHOC
  trap vortex 3D      87x87x203 (h = 0.2) and 256x256x512 (h = 17.2/255), 2SHOC, MSD,
                      dt = 0.8 x the potential-aware stability bound
  vortex rings 3D     512^3, h = 0.25, 2SHOC, MSD (the precision form's workload)

Tolerances are the method's end-time bars: relative L2 <= 1e-12 (FP64) and
<= 2e-5 (FP32 forms) against the FP64 oracle, at each workload's end time:
the 1D soliton over all 32,000 steps, 87x87x203 over all 3360 steps (the
oracle runs them on every host core, about a minute and a half on 16), the
vortex rings' 128^3 analogue over all 2000 steps against the oracle and the
512^3 grid over all 2000 steps FP32-with-FP64-accumulator against FP64.
The 256x256x512 and 512^3 grids are also checked over one step against the
oracle on every site.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1203_1263_gb300 import workloads as W
from paper_1203_1263_gb300.integrator import Integrator

pytestmark = pytest.mark.gpu


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def bound_dt(p):
    s_rho = abs(p.s) * float(np.max(np.abs(p.psi0))) ** 2
    return 0.8 * O.stability_bound(p.dims, p.h, p.a, p.order, p.vmax(), s_rho)


@pytest.mark.parametrize("order", [2, 4])
def test_bright_soliton_full_run(order):
    """32000 RK4 steps to t = 10: FP64 matches the oracle to 1e-12 and the
    exact soliton to the scheme's accuracy; the FP64-accumulator form stays
    within 2e-5 of the oracle."""
    p = W.bright_soliton_1d(order=order, n=2001, t_end=10.0)
    ref, _ = O.run_problem(p)
    exact = W.bright_soliton(p.extra["x"], p.extra["t_end"])
    ref_err = rel_l2(ref, exact)          # the scheme's own error at t = 10
    m0 = O.mass(p.psi0, p.h)
    for dtype, tol, mtol in (("c128", 1e-12, 1e-9), ("c64_acc64", 2e-5, 1e-6)):
        g = Integrator(p.psi0, p.h, p.a, p.s, None, "dirichlet", order, dtype)
        g.step(p.steps, p.dt)
        got = g.numpy()
        assert rel_l2(got, ref) <= tol, (dtype, rel_l2(got, ref))
        assert rel_l2(got, exact) <= ref_err + tol
        assert abs(g.mass() - m0) <= mtol * m0


# Pure FP32 (every stage array and Psi itself in FP32) over the full 32,000
# steps, against the oracle at t = 10.
@pytest.mark.parametrize("order", [2, 4])
def test_bright_soliton_plain_fp32_full_run(order):
    p = W.bright_soliton_1d(order=order, n=2001, t_end=10.0)
    ref, _ = O.run_problem(p)
    g = Integrator(p.psi0, p.h, p.a, p.s, None, "dirichlet", order, "c64")
    g.step(p.steps, p.dt)
    err = rel_l2(g.numpy(), ref)
    print(f"pure FP32, order {order}, 32000 steps: rel-L2 vs oracle {err:.3e}")
    assert err <= 2e-5


@pytest.fixture(scope="module")
def trap87():
    """The paper's headline grid in full: 87x87x203, 2SHOC, MSD, 3360 steps,
    run by the oracle on every host core."""
    p = W.trap_vortex_3d(shape=(203, 87, 87))
    dt = bound_dt(p)
    O.set_threads(os.cpu_count() or 1)
    ref = O.rk4(p.psi0, p.h, p.a, p.s, dt, p.steps, p.V, p.bc, p.order)
    return p, dt, ref


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 2e-5), ("c64_acc64", 2e-5)])
def test_trap_vortex_87x87x203_full_run(trap87, dtype, tol):
    """All 3360 steps (t = 23.2) against the oracle, every site; the mass
    against the oracle's.  Within the stability bound RK4 damps (|R(iy)| <= 1),
    so the mass may only decrease; it loses ~1e-3 here, the stiff content of
    the non-smooth Thomas-Fermi edge."""
    p, dt, ref = trap87
    g = Integrator(p.psi0, p.h, p.a, p.s, p.V, "msd", 4, dtype)
    g.step(p.steps, dt)
    err = rel_l2(g.numpy(), ref)
    m_ref, m0 = O.mass(ref, p.h), O.mass(p.psi0, p.h)
    print(f"87x87x203 {dtype}, 3360 steps: rel-L2 vs oracle {err:.3e}, "
          f"mass drift {abs(m_ref - m0) / m0:.3e}")
    assert err <= tol
    assert m_ref <= m0 * (1 + 1e-12)
    assert abs(g.mass() - m_ref) <= (1e-12 if dtype == "c128" else 2 * tol) * m_ref


def test_trap_vortex_256x256x512_one_step_full_size():
    """The benchmark's workload and launch configuration, one step, every site
    against the oracle."""
    p = W.trap_vortex_3d(shape=(512, 256, 256))
    dt = bound_dt(p)
    ref = O.rk4(p.psi0, p.h, p.a, p.s, dt, 1, p.V, p.bc, p.order)
    for dtype, tol in (("c128", 1e-12), ("c64", 2e-5)):
        g = Integrator(p.psi0, p.h, p.a, p.s, p.V, "msd", 4, dtype)
        g.step(1, dt)
        assert rel_l2(g.numpy(), ref) <= tol, dtype
        g.close()


def _boundary_mask(shape):
    m = np.zeros(shape, dtype=bool)
    for ax in range(len(shape)):
        idx = [slice(None)] * len(shape)
        idx[ax] = 0
        m[tuple(idx)] = True
        idx[ax] = -1
        m[tuple(idx)] = True
    return m


def test_256x256x512_laplacian_zero_boundary_full_size():
    """The benchmark's grid, potential and launch configuration with the
    Laplacian-zero boundary (Eqs. BCL0dt, BCL0lap), on the trap state plus a
    unit plane wave so that the walls carry a field: one step against the
    oracle on every site; then 16 more (one graph replay), after which every
    boundary site must be the scalar RK4 iterate of z' = i(s|z|^2 - V_b) z
    from its own initial value, since Eq. BCL0dt involves that site alone."""
    p = W.trap_vortex_3d(shape=(512, 256, 256))
    x = (np.arange(p.shape[2]) - 0.5 * (p.shape[2] - 1)) * p.h
    psi0 = p.psi0 + 0.5 * np.exp(0.4j * x)[None, None, :]
    s_rho = abs(p.s) * float(np.max(np.abs(psi0))) ** 2
    dt = 0.8 * O.stability_bound(3, p.h, p.a, 4, p.vmax(), s_rho)
    ref = O.rk4(psi0, p.h, p.a, p.s, dt, 1, p.V, W.BC_L0, 4)
    for dtype, tol in (("c128", 1e-12), ("c64", 2e-5)):
        g = Integrator(psi0, p.h, p.a, p.s, p.V, "l0", 4, dtype)
        g.step(1, dt)
        assert rel_l2(g.numpy(), ref) <= tol, dtype
        if dtype == "c128":
            g.step(16, dt)
            b = _boundary_mask(p.shape)
            z, Vb = psi0[b], p.V[b]
            f = lambda y: 1j * (p.s * np.abs(y) ** 2 - Vb) * y
            for _ in range(17):
                k1 = f(z); k2 = f(z + dt / 2 * k1); k3 = f(z + dt / 2 * k2); k4 = f(z + dt * k3)
                z = z + dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4)
            assert np.max(np.abs(g.numpy()[b] - z)) <= 1e-12 * np.max(np.abs(z))
        g.close()


def test_256x256x512_periodic_full_size():
    """The benchmark's grid, potential and launch configuration on a periodic
    grid (the boundary of the stability analysis, Sec. 3.4), on the trap
    state plus a unit plane wave (so that the wrap carries a field): one step
    against the oracle on every site, FP64 and FP32."""
    p = W.trap_vortex_3d(shape=(512, 256, 256))
    x = (np.arange(p.shape[2]) - 0.5 * (p.shape[2] - 1)) * p.h
    psi0 = p.psi0 + 0.5 * np.exp(0.4j * x)[None, None, :]
    s_rho = abs(p.s) * float(np.max(np.abs(psi0))) ** 2
    dt = 0.8 * O.stability_bound(3, p.h, p.a, 4, p.vmax(), s_rho)
    ref = O.rk4(psi0, p.h, p.a, p.s, dt, 1, p.V, W.BC_PERIODIC, 4)
    for dtype, tol in (("c128", 1e-12), ("c64", 2e-5)):
        g = Integrator(psi0, p.h, p.a, p.s, p.V, "periodic", 4, dtype)
        g.step(1, dt)
        assert rel_l2(g.numpy(), ref) <= tol, dtype
        g.close()


RINGS_DT = 0.8 * O.stability_bound(3, 0.25, 0.5, 4, 0.0, 1.0)   # the 512^3 grid's step (max|Psi0| = 1)


def test_vortex_rings_512cube_precision_form():
    """512^3, the precision form's workload: one step of the FP64 and the
    FP32-with-FP64-accumulator forms against the oracle on every site, then
    all 2000 steps of the two GPU forms against each other (relative L2, and
    the mass of each against the other)."""
    p = W.vortex_rings_3d(n=512)
    dt = bound_dt(p)
    assert abs(dt - RINGS_DT) <= 1e-15 * dt
    ref = O.rk4(p.psi0, p.h, p.a, p.s, dt, 1, None, p.bc, p.order)
    g64 = Integrator(p.psi0, p.h, p.a, p.s, None, "msd", 4, "c128")
    gmx = Integrator(p.psi0, p.h, p.a, p.s, None, "msd", 4, "c64_acc64")
    g64.step(1, dt)
    gmx.step(1, dt)
    assert rel_l2(g64.numpy(), ref) <= 1e-12
    assert rel_l2(gmx.numpy(), ref) <= 2e-5
    del ref
    m0, steps = O.mass(p.psi0, p.h), p.steps
    del p
    g64.step(steps - 1, dt)
    gmx.step(steps - 1, dt)
    a, b = g64.numpy(), gmx.numpy()
    err = rel_l2(b, a)
    m64, mmx = g64.mass(), gmx.mass()
    print(f"512^3, 2000 steps: c64_acc64 rel-L2 vs c128 {err:.3e}; mass drift c128 {abs(m64 - m0) / m0:.3e}, "
          f"c64_acc64 {abs(mmx - m0) / m0:.3e}, between forms {abs(mmx - m64) / m64:.3e}")
    assert err <= 2e-5
    # the MSD walls hold |Psi|^2 but not the phase, so mass crosses them (~1e-3 over the run); the two
    # forms must agree on it
    assert abs(mmx - m64) <= 1e-6 * m64


def test_vortex_rings_128cube_analogue_full_run():
    """The precision form's workload at 128^3 (h = 0.5: the same rings in
    half the box) with the 512^3 grid's step size, all 2000 steps, every site
    against the oracle (FP64 and FP32-with-FP64-accumulator)."""
    p = W.vortex_rings_3d(n=128, h=0.5)
    O.set_threads(os.cpu_count() or 1)
    ref = O.rk4(p.psi0, p.h, p.a, p.s, RINGS_DT, p.steps, None, p.bc, p.order)
    m0, m_ref = O.mass(p.psi0, p.h), O.mass(ref, p.h)
    for dtype, tol in (("c128", 1e-12), ("c64_acc64", 2e-5)):
        g = Integrator(p.psi0, p.h, p.a, p.s, None, "msd", 4, dtype)
        g.step(p.steps, RINGS_DT)
        err = rel_l2(g.numpy(), ref)
        print(f"128^3 rings {dtype}, 2000 steps: rel-L2 vs oracle {err:.3e}, mass drift {abs(m_ref - m0) / m0:.3e}")
        assert err <= tol
        assert abs(g.mass() - m_ref) <= (1e-12 if dtype == "c128" else 1e-6) * m_ref
        g.close()


@pytest.mark.parametrize("dims,total", [(1, 1000), (1, 10000), (2, 961), (2, 10000), (3, 9261), (3, 97336)])
@pytest.mark.parametrize("dtype,order", [("c64", 2), ("c128", 4), ("c128", 2), ("c64", 4)])
def test_paper_timing_workloads_match_oracle(dims, total, dtype, order):
    """The timing workloads of Sec. 7 at the tables' smaller sizes, 200 steps
    at k = 0.005, every site against the oracle."""
    p = W.paper_timing_problem(dims, total, order)
    n = 200
    ref = O.rk4(p.psi0, p.h, p.a, p.s, p.dt, n, None, p.bc, order)
    g = Integrator(p.psi0, p.h, p.a, p.s, None, "msd", order, dtype)
    g.step(n, p.dt)
    assert rel_l2(g.numpy(), ref) <= (1e-12 if dtype == "c128" else 2e-5)


def test_paper_dark_soliton_full_run():
    """The 1D timing run of Sec. 7 in full (N = 1000, 10,000 steps to t = 50,
    2SHOC, FP64): against the oracle, and against the exact moving dark
    soliton to within the scheme's own error."""
    p = W.paper_timing_problem(1, 1000, 4)
    ref = O.rk4(p.psi0, p.h, p.a, p.s, p.dt, p.steps, None, p.bc, 4)
    exact = W.dark_soliton(p.extra["x"], p.steps * p.dt)
    g = Integrator(p.psi0, p.h, p.a, p.s, None, "msd", 4, "c128")
    g.step(p.steps, p.dt)
    got = g.numpy()
    print(f"dark soliton 1D c128, 10000 steps: rel-L2 vs oracle {rel_l2(got, ref):.3e}, "
          f"oracle vs exact {rel_l2(ref, exact):.3e}")
    assert rel_l2(got, ref) <= 1e-12
    assert rel_l2(got, exact) <= rel_l2(ref, exact) + 1e-12
    assert rel_l2(ref, exact) < 1e-3
