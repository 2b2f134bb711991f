"""CUDA path vs the CPU oracle on seeded inputs, element by element.

Tolerances (the end-time bars of the method, applied to every comparison):
  FP64 (c128):            relative L2 <= 1e-12, max |diff| <= 1e-11 max|ref|
  FP32 (c64, c64_acc64):  relative L2 <= 2e-5,  max |diff| <= 2e-4 max|ref|
FP32 runs start from the FP64 inputs rounded to FP32 and are compared with
the FP64 oracle.  Grid shapes span several tiles of the tiled kernels with
ragged tails, and include the degenerate extents 3 and 4.
"""
import numpy as np
import pytest
import torch

import oracle as O
from paper_1203_1263_gb300 import workloads as W
from paper_1203_1263_gb300 import _lib as L
from paper_1203_1263_gb300.integrator import Integrator

pytestmark = pytest.mark.gpu

TOL = {"c128": (1e-12, 1e-11), "c64": (2e-5, 2e-4), "c64_acc64": (2e-5, 2e-4)}
BCS = {"dirichlet": W.BC_DIRICHLET, "msd": W.BC_MSD, "l0": W.BC_L0, "periodic": W.BC_PERIODIC}

SHAPES = {
    1: [(37,), (3,), (4,), (1000,)],
    2: [(19, 45), (3, 7), (4, 40), (70, 33)],
    3: [(9, 21, 70), (3, 4, 5), (13, 10, 37), (20, 17, 64)],
}


def _smooth(z, passes):
    for _ in range(passes):
        acc = z.copy()
        for ax in range(z.ndim):
            acc += np.roll(z, 1, ax) + np.roll(z, -1, ax)
        z = acc / (2 * z.ndim + 1)
    return z


def field(shape, seed):
    """Unit background with seeded, smoothed structure: density bumps of up to
    +-30 % that vanish at the walls, and a smooth phase of amplitude 1.
    MSD holds |Psi|^2 at the walls, which suits a near-constant background
    (the paper's use of it); on a rough random field the wall-adjacent density
    collapses and the wall ratio Im(F/Psi) blows up in the oracle as well."""
    r = _smooth(W.random_field(shape, seed), 3)
    r = r / np.max(np.abs(r))
    win = np.ones(shape)
    for ax, n in enumerate(shape):
        sh = [1] * len(shape)
        sh[ax] = n
        win = win * (np.sin(np.pi * np.arange(n) / (n - 1)) ** 2).reshape(sh)
    return ((1 + 0.3 * win * r.real) * np.exp(1j * r.imag)).astype(np.complex128)


def periodic_field(shape, seed):
    """Smooth periodic structure with no window: the values on either side of
    the wrap differ, so a wrong wrap shows."""
    r = _smooth(W.random_field(shape, seed), 3)
    r = r / np.max(np.abs(r))
    return ((1 + 0.3 * r.real) * np.exp(1j * r.imag)).astype(np.complex128)


def compare(got, ref, dtype):
    rl2, elem = TOL[dtype]
    got = np.asarray(got, dtype=np.complex128)
    err = np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel())
    emax = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err <= rl2 and emax <= elem, (err, emax)
    return err


def problem(shape, seed, with_v=True, bc="dirichlet"):
    psi = periodic_field(shape, seed) if bc == "periodic" else field(shape, seed)
    V = W.random_potential(shape, seed + 1, 0.5) if with_v else None
    return psi, V


def stable_dt(shape, h, a, s, order, V, frac=0.2):
    return frac * O.stability_bound(len(shape), h, a, order, 0.0 if V is None else float(np.max(V)), abs(s) * 1.7)


CASES = [(d, shp) for d in (1, 2, 3) for shp in SHAPES[d]]
_ORACLE_CACHE = {}


def oracle_rk4_cached(key, *args):
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = O.rk4(*args)
    return _ORACLE_CACHE[key]


@pytest.mark.parametrize("dims,shape", CASES)
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("bc", ["dirichlet", "msd", "l0", "periodic"])
@pytest.mark.parametrize("dtype", ["c128", "c64", "c64_acc64"])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_step_matches_oracle(dims, shape, order, bc, dtype, variant):
    h, a, s = 0.35, 0.8, -1.1
    psi, V = problem(shape, 100 + dims * 10 + order, bc=bc)
    dt = stable_dt(shape, h, a, s, order, V)
    nsteps = 21   # one graph replay of 16 steps + 5 single steps
    ref = oracle_rk4_cached((shape, order, bc), psi, h, a, s, dt, nsteps, V, BCS[bc], order)
    g = Integrator(psi, h, a, s, V, bc, order, dtype)
    g.set_kernel(variant)
    g.step(nsteps, dt)
    g.sync()
    compare(g.numpy(), ref, dtype)


@pytest.mark.parametrize("dims,shape", [(1, (37,)), (2, (19, 45)), (3, (9, 21, 70)), (3, (3, 4, 5))])
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("bc", ["dirichlet", "msd", "l0", "periodic"])
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_rhs_matches_oracle(dims, shape, order, bc, dtype):
    h, a, s = 0.3, 0.9, 1.3
    psi, V = problem(shape, 7 + dims, bc=bc)
    ref = O.evalF(psi, h, a, s, V, BCS[bc], order)
    g = Integrator(psi, h, a, s, V, bc, order, dtype)
    got = g.rhs().cpu().numpy()
    tol = 1e-13 if dtype == "c128" else 1e-5
    assert np.max(np.abs(got - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("dims,shape", [(1, (1000,)), (2, (70, 33)), (3, (20, 17, 64))])
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("bc", ["dirichlet", "msd", "l0", "periodic"])
@pytest.mark.parametrize("dtype", ["c128", "c64", "c64_acc64"])
def test_mass_energy_match_oracle(dims, shape, order, bc, dtype):
    h, a, s = 0.25, 0.7, -0.6
    psi, V = problem(shape, 55, bc=bc)
    g = Integrator(psi, h, a, s, V, bc, order, dtype)
    # the oracle sees exactly what the GPU holds (FP32 forms: the rounded state and potential)
    held = g.numpy().astype(np.complex128)
    Vh = V.astype(np.float32).astype(np.float64) if dtype != "c128" else V
    m_ref = O.mass(held, h)
    e_ref = O.energy(held, h, a, s, Vh, BCS[bc], order)
    assert abs(g.mass() - m_ref) <= 1e-13 * abs(m_ref)
    assert abs(g.energy() - e_ref) <= 1e-12 * abs(e_ref)


@pytest.mark.parametrize("dtype", ["c128", "c64", "c64_acc64"])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_split_continuation_and_determinism_bitwise(dtype, variant):
    psi, V = problem((11, 12, 40), 3)
    h, a, s, order = 0.3, 0.6, 1.0, 4
    dt = stable_dt(psi.shape, h, a, s, order, V)
    outs = []
    for split in ([7, 13], [20], [3, 17]):
        g = Integrator(psi, h, a, s, V, "msd", order, dtype)
        g.set_kernel(variant)
        for n in split:
            g.step(n, dt)
        outs.append(g.numpy())
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])


@pytest.mark.parametrize("dtype", ["c128", "c64", "c64_acc64"])
@pytest.mark.parametrize("dims,shape", [(2, (19, 45)), (3, (9, 21, 70)), (3, (20, 17, 64)), (3, (5, 40, 131)),
                                        (3, (70, 36, 75)), (3, (7, 7, 10)), (3, (12, 9, 9))])
@pytest.mark.parametrize("tile_cfg", [0, 1, 2, 3])
def test_tiled_kernel_equals_generic_bitwise(dtype, dims, shape, tile_cfg):
    """The tiled kernels perform the generic kernel's arithmetic in the same
    order; only where the operands come from differs."""
    for order in (2, 4):
        for bc in ("dirichlet", "msd", "l0", "periodic"):
            psi, V = problem(shape, 77, bc=bc)
            h, a, s = 0.3, 0.6, -1.0
            dt = stable_dt(shape, h, a, s, order, V)
            res = []
            for variant in (0, 1, 3, 2):
                g = Integrator(psi, h, a, s, V, bc, order, dtype)
                g.set_kernel(variant, tile_cfg)
                g.step(5, dt)
                res.append(g.numpy())
            assert np.array_equal(res[0], res[1]), (order, bc)
            assert np.array_equal(res[2], res[3]), (order, bc)


@pytest.mark.parametrize("n", [37, 1000, 2001, 5003, 60000])
@pytest.mark.parametrize("bc", ["dirichlet", "msd", "l0", "periodic"])
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("dtype,family", [("c128", "exact"), ("c128", "fp64"), ("c64", "fp32")])
def test_line_cluster_equals_per_site_bitwise(n, bc, order, dtype, family):
    """1D: the thread-block-cluster path (the whole call in one launch, the
    line in shared memory) gives the per-site kernel's bits, with either FP64
    stencil and also when the steps are split across calls; lines too long for
    shared memory (60,000 sites in FP64) take the per-site kernel."""
    psi, V = problem((n,), 65, bc=bc)
    h, a, s = 0.3, 0.6, -1.0
    dt = stable_dt((n,), h, a, s, order, V)
    per_site, line = (3, 2) if family == "exact" else (0, 1)
    res = []
    for variant, split in ((per_site, (21,)), (line, (21,)), (line, (5, 16))):
        g = Integrator(psi, h, a, s, V, bc, order, dtype)
        g.set_kernel(variant)
        fits = not (dtype == "c128" and n > 49152)
        assert g.kernel_in_use() == (line if variant == line and fits else per_site)
        if variant == line:
            d = Integrator(psi, h, a, s, V, bc, order, dtype)   # the default kernel for this length
            if dtype == "c128":   # the cluster up to 2500 sites, then one thread per site, FP64 stencil to 2^15
                assert d.kernel_in_use() == (1 if n <= 2500 else (0 if n <= 32768 else 3))
            else:
                assert d.kernel_in_use() == 1
            d.close()
        for k in split:
            g.step(k, dt)
        g.sync()
        res.append(g.numpy())
    assert np.array_equal(res[0], res[1]) and np.array_equal(res[1], res[2])


FUSED_SHAPES = [(16, 16, 16), (20, 24, 70), (33, 40, 64), (40, 37, 130), (18, 70, 66), (20, 24, 71)]


@pytest.mark.parametrize("shape", FUSED_SHAPES)
@pytest.mark.parametrize("bc", ["dirichlet", "msd", "l0", "periodic"])
@pytest.mark.parametrize("order", [2, 4])
@pytest.mark.parametrize("with_v", [True, False])
def test_fused_step_equals_stage_streaming_bitwise(shape, bc, order, with_v):
    """Two stages per pass (variant 4) against one pass per stage (variant 1),
    FP32: 37 steps (two graph-replayed chunks of 16 fused steps with the
    Psi ping-pong, then 5 single steps) give the same bits; odd Nx and
    periodic grids run the stage-streaming path."""
    psi, V = problem(shape, 61, with_v=with_v, bc=bc)
    h, a, s = 0.3, 0.6, -1.0
    dt = stable_dt(shape, h, a, s, order, V)
    res = []
    for variant in (1, 4):
        g = Integrator(psi, h, a, s, V, bc, order, "c64")
        g.set_kernel(variant)
        assert g.kernel_in_use() == (4 if variant == 4 and shape[2] % 2 == 0 and bc != "periodic" else 1)
        g.step(37, dt)
        g.sync()
        res.append(g.numpy())
    assert np.array_equal(res[0], res[1])
    compare(res[1], O.rk4(psi, h, a, s, dt, 37, V, BCS[bc], order), "c64")


@pytest.mark.parametrize("bc", ["dirichlet", "msd", "l0", "periodic"])
@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("dims,shape", [(1, (37,)), (2, (19, 45)), (3, (9, 21, 70))])
@pytest.mark.parametrize("factor", [1e2, 1e-4, 1e-8])
def test_exact_sum_scale_follows_the_state(variant, dims, shape, bc, factor):
    """The exact-sum stencil takes its fixed-point scale from the state before
    every step: a state written into psi after creation at 1e2, 1e-4 or 1e-8
    times the one the context was created with integrates to the FP64 bar."""
    psi, V = problem(shape, 91, bc=bc)
    h, a, s, order = 0.3, 0.6, -1.0, 4
    x = factor * psi
    dt = 0.2 * O.stability_bound(dims, h, a, order, float(np.max(V)), abs(s) * 1.7 * max(1.0, factor) ** 2)
    g = Integrator(psi, h, a, s, V, bc, order, "c128")
    g.set_kernel(variant)
    g.psi.copy_(torch.from_numpy(x).to(g.psi.device))
    g.step(21, dt)
    compare(g.numpy(), O.rk4(x, h, a, s, dt, 21, V, BCS[bc], order), "c128")


@pytest.mark.parametrize("dims,shape", [(1, (37,)), (2, (19, 45)), (3, (9, 21, 70))])
@pytest.mark.parametrize("variant", [2, 3])
def test_stiff_potential_keeps_the_exact_sum_stages(dims, shape, variant):
    """The exact-sum stencil's range depends on the state alone, not on the
    potential: with V 1e5 times the usual one the context keeps the exact-sum
    stages and meets the FP64 bar."""
    psi, V = problem(shape, 93)
    h, a, s, order = 0.3, 0.6, -1.0, 4
    Vs = V * 1e5
    dt = 0.2 * O.stability_bound(dims, h, a, order, float(np.max(Vs)), abs(s) * 1.7)
    g = Integrator(psi, h, a, s, Vs, "msd", order, "c128")
    g.set_kernel(variant)
    assert g.kernel_in_use() in (2, 3)
    g.step(21, dt)
    compare(g.numpy(), O.rk4(psi, h, a, s, dt, 21, Vs, W.BC_MSD, order), "c128")


@pytest.mark.parametrize("bc", ["dirichlet", "l0", "periodic"])
@pytest.mark.parametrize("variant", [2, 3])
@pytest.mark.parametrize("dims,shape", [(2, (19, 45)), (3, (9, 21, 70))])
def test_exact_sum_out_of_range_falls_back(variant, dims, shape, bc):
    """With the fixed-point range made 2^12 too small for the state (test
    hook), every site's stencil operands are out of range and every site
    takes the FP64 stencil: the result still meets the FP64 bar."""
    psi, V = problem(shape, 91, bc=bc)
    h, a, s, order = 0.3, 0.6, -1.0, 4
    dt = 0.2 * O.stability_bound(dims, h, a, order, float(np.max(V)), abs(s) * 1.7)
    g = Integrator(psi, h, a, s, V, bc, order, "c128")
    g.set_kernel(variant)
    g.debug_set(L.DEBUG_FIX_OFFSET, 12)
    g.step(4, dt)
    compare(g.numpy(), O.rk4(psi, h, a, s, dt, 4, V, BCS[bc], order), "c128")


@pytest.mark.parametrize("dtype,variant", [("c128", None), ("c128", 2), ("c64", None), ("c64_acc64", None)])
def test_refresh_potential_takes_new_values(dtype, variant):
    """V written after creation takes effect after nlse_refresh_potential, in
    every dtype alike (max|V| and, on the exact-sum stages, the scaled copy
    V / cLF are re-read)."""
    shape = (9, 21, 70)
    psi, V = problem(shape, 41)
    V2 = 2.0 * V + 0.1
    h, a, s, order = 0.3, 0.6, -1.0, 4
    dt = stable_dt(shape, h, a, s, order, V2)
    g = Integrator(psi, h, a, s, V, "msd", order, dtype)
    if variant is not None:
        g.set_kernel(variant)
    g.V.copy_(torch.from_numpy(V2).to(g.V.dtype).to(g.V.device))
    between = 0.5 * (O.stability_bound(3, h, a, order, float(np.max(V)), 0.0) +
                     O.stability_bound(3, h, a, order, float(np.max(V2)), 0.0))
    g.step(0, between)                       # within the bound of the potential the context read at creation
    g.refresh_potential()
    with pytest.raises(L.NLSEError) as e:    # above the bound of the new potential
        g.step(1, between)
    assert e.value.code == L.NLSE_EUNSTABLE
    g.step(17, dt)
    Vh = V2.astype(np.float32).astype(np.float64) if dtype != "c128" else V2
    compare(g.numpy(), O.rk4(psi, h, a, s, dt, 17, Vh, W.BC_MSD, order), dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_bounded_wait_times_out_and_context_recovers(dtype):
    """Every TMA barrier is made to expect 16 bytes its copy never delivers, so
    the kernel's bounded wait runs out (no fault, no hang); the host gets
    NLSE_ETIMEOUT once, and after the hook is removed the same context steps
    correctly again."""
    psi, V = problem((12, 10, 64), 17)
    h, a, s, order = 0.3, 0.6, -1.0, 4
    dt = stable_dt(psi.shape, h, a, s, order, V)
    g = Integrator(psi, h, a, s, V, "msd", order, dtype)
    g.set_kernel(1)
    g.debug_set(L.DEBUG_SPIN_LIMIT, 200000)       # ~0.1 ms per wait
    g.debug_set(L.DEBUG_EXTRA_TX, 16)
    g.step(1, dt)
    with pytest.raises(L.NLSEError) as e:
        g.sync()
    assert e.value.code == L.NLSE_ETIMEOUT
    g.debug_set(L.DEBUG_EXTRA_TX, 0)
    g.debug_set(L.DEBUG_SPIN_LIMIT, 2000000000)
    g.psi.copy_(torch.from_numpy(psi).to(g.psi.dtype).to(g.psi.device))
    g.step(3, dt)
    g.sync()
    compare(g.numpy(), O.rk4(psi, h, a, s, dt, 3, V, W.BC_MSD, order), dtype)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_autotune_picks_a_tile_and_keeps_results(dtype, tmp_path, monkeypatch):
    """The autotuner times the tile shapes on the context's own buffers without
    touching Psi, keeps one, and a second process-level lookup comes from the
    cache; the integration result is bit-for-bit the default's."""
    monkeypatch.setenv("NLSE_TUNE_CACHE", str(tmp_path / "tune.txt"))
    psi, V = problem((14, 30, 72), 23)
    h, a, s, order = 0.3, 0.6, -1.0, 4
    dt = stable_dt(psi.shape, h, a, s, order, V)
    tiled = 2 if dtype == "c128" else 1      # a grid this small defaults to the per-site kernel
    g0 = Integrator(psi, h, a, s, V, "msd", order, dtype)
    g0.set_kernel(tiled)
    g0.step(6, dt)
    ref = g0.numpy()
    g = Integrator(psi, h, a, s, V, "msd", order, dtype)
    g.set_kernel(tiled)
    before = g.numpy()
    cfg, ms = g.autotune()
    assert cfg in (0, 1, 2, 3) and ms > 0
    assert np.array_equal(before, g.numpy())          # Psi untouched by tuning
    g.step(6, dt)
    assert np.array_equal(ref, g.numpy())
    g2 = Integrator(psi, h, a, s, V, "msd", order, dtype)
    g2.set_kernel(tiled)
    cfg2, ms2 = g2.autotune()
    assert cfg2 == cfg and ms2 == 0.0                 # served from the cache
    assert (tmp_path / "tune.txt").read_text().count("=") >= 1


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_small_3d_grid_defaults_to_the_per_site_kernel(dtype):
    """A 3D grid small enough to be latency-bound (30,240 sites) defaults to
    the one-thread-per-site kernel with the plain stencil (nothing for the
    autotuner to time), with the same result as the tiled kernel of its
    arithmetic."""
    psi, V = problem((14, 30, 72), 23)
    h, a, s, order = 0.3, 0.6, -1.0, 4
    dt = stable_dt(psi.shape, h, a, s, order, V)
    g = Integrator(psi, h, a, s, V, "msd", order, dtype)
    assert g.autotune() == (-1, 0.0)
    g.step(6, dt)
    assert g.kernel_in_use() == 0
    t = Integrator(psi, h, a, s, V, "msd", order, dtype)
    t.set_kernel(1)
    t.step(6, dt)
    assert np.array_equal(g.numpy(), t.numpy())


def test_dt_above_bound_is_rejected():
    psi, V = problem((10, 10), 4)
    g = Integrator(psi, 0.2, 1.0, 1.0, V, "dirichlet", 4, "c128")
    bound = g.max_dt()
    with pytest.raises(L.NLSEError) as e:
        g.step(1, bound * 1.01)
    assert e.value.code == L.NLSE_EUNSTABLE
    g.step(1, bound * 0.99)
    g.sync()


@pytest.mark.parametrize("dtype", ["c128", "c64", "c64_acc64"])
def test_non_finite_is_reported(dtype):
    psi, V = problem((8, 9, 10), 5)
    psi[4, 4, 4] = np.nan
    g = Integrator(psi, 0.3, 1.0, 1.0, V, "msd", 4, dtype)
    g.step(2, 1e-4)
    with pytest.raises(L.NLSEError) as e:
        g.sync()
    assert e.value.code == L.NLSE_ENONFINITE
    with pytest.raises(L.NLSEError):
        g.mass()


def test_zero_steps_and_bad_dt():
    psi, V = problem((6, 7), 6)
    g = Integrator(psi, 0.3, 1.0, 1.0, V, "msd", 2, "c128")
    before = g.numpy()
    g.step(0, 1e-3)
    assert np.array_equal(before, g.numpy())
    for bad in (0.0, -1e-3, float("nan")):
        with pytest.raises(L.NLSEError) as e:
            g.step(1, bad)
        assert e.value.code == L.NLSE_EINVAL
