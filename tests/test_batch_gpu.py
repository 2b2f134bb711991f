"""Batched form: many uneven 2D runs advanced together.

Each run in a batch is computed with the same per-site arithmetic as a
single-run complex64 context using the tiled kernels, so the two must agree
bit for bit; a sample of runs is also checked against the FP64 oracle
(relative L2 <= 2e-5, the FP32 bar)."""
import numpy as np
import pytest

import oracle as O
from paper_1203_1263_gb300 import _lib as L
from paper_1203_1263_gb300 import workloads as W
from paper_1203_1263_gb300.integrator import BatchIntegrator, Integrator

pytestmark = pytest.mark.gpu
BCS = {"dirichlet": W.BC_DIRICHLET, "msd": W.BC_MSD, "l0": W.BC_L0}


def small_runs(seed=4, nruns=14):
    """Uneven runs with the batch workload's parameter recipe on smaller grids
    (sides 5..150, including the degenerate 3 and 4)."""
    runs = []
    for i, d in enumerate(W.batch_runs_2d(nruns=nruns, seed=seed, nmin=5, nmax=150, h=0.25)):
        if i == 0:
            d["n"] = 3
        if i == 1:
            d["n"] = 4
        p = W.batch_run_problem(d)
        s_rho = abs(p.s) * float(np.max(np.abs(p.psi0))) ** 2
        dt = 0.5 * O.stability_bound(2, p.h, p.a, p.order, p.vmax(), s_rho)
        runs.append(dict(psi0=p.psi0, h=p.h, a=p.a, s=p.s, dt=dt, V=p.V, bc=["dirichlet", "msd", "l0"][i % 3],
                         order=p.order))
    return runs


def test_batch_equals_single_runs_bitwise():
    runs = small_runs()
    b = BatchIntegrator(runs)
    b.step(21)     # one graph replay of 16 steps + 5 single steps
    b.sync()
    for i, r in enumerate(runs):
        g = Integrator(r["psi0"], r["h"], r["a"], r["s"], r["V"], r["bc"], r["order"], "c64")
        g.set_kernel(1)
        g.step(21, r["dt"])
        assert np.array_equal(b.numpy(i), g.numpy()), i


def test_batch_matches_oracle():
    runs = small_runs(seed=9, nruns=8)
    b = BatchIntegrator(runs)
    b.step(12)
    b.sync()
    for i, r in enumerate(runs):
        ref = O.rk4(r["psi0"], r["h"], r["a"], r["s"], r["dt"], 12, r["V"],
                    BCS[r["bc"]], r["order"])
        got = b.numpy(i).astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 2e-5, (i, err)


def test_batch_autotune_and_tiles_keep_results():
    runs = small_runs(seed=5, nruns=10)
    ref = BatchIntegrator(runs)
    ref.step(6)
    ref.sync()
    b = BatchIntegrator(runs)
    cfg, ms = b.autotune()
    assert cfg in (0, 1, 2, 3) and ms > 0
    b.step(6)
    b.sync()
    for t in (0, 1, 2):
        c = BatchIntegrator(runs)
        c.set_tile(t)
        c.step(6)
        c.sync()
        for i in range(len(runs)):
            assert np.array_equal(c.numpy(i), ref.numpy(i))
    for i in range(len(runs)):
        assert np.array_equal(b.numpy(i), ref.numpy(i))


def test_batch_rejects_bad_runs():
    runs = small_runs(nruns=3)
    runs[2] = dict(runs[2], dt=runs[2]["dt"] * 1e3)
    with pytest.raises(L.NLSEError) as e:
        BatchIntegrator(runs)
    assert e.value.code == L.NLSE_EUNSTABLE
    runs = small_runs(nruns=3)
    runs[1] = dict(runs[1], order=3)
    with pytest.raises(L.NLSEError):
        BatchIntegrator(runs)


def test_switching_tiles_on_one_batch_keeps_results():
    """The work lists (and the run fields after them) move when the tile shape
    changes; the status word must not, and every shape must continue the
    same integration."""
    runs = small_runs(seed=6, nruns=9)
    tiles = (1, 3, 0, 2)
    ref = BatchIntegrator(runs)
    ref.step(2 * len(tiles))
    ref.sync()
    b = BatchIntegrator(runs)
    for t in tiles:
        b.set_tile(t)
        b.step(2)
        b.sync()
    for i in range(len(runs)):
        assert np.array_equal(b.numpy(i), ref.numpy(i)), i


def workload_runs(nruns=512, seed=4):
    """The timed batch workload itself: 512 runs of sides 64..1024 (2.0e8
    sites), each at 0.8 of its own stability bound, Dirichlet walls."""
    runs = []
    for d in W.batch_runs_2d(nruns=nruns, seed=seed):
        p = W.batch_run_problem(d)
        s_rho = abs(p.s) * float(np.max(np.abs(p.psi0))) ** 2
        dt = 0.8 * O.stability_bound(2, p.h, p.a, p.order, p.vmax(), s_rho)
        runs.append(dict(psi0=p.psi0, h=p.h, a=p.a, s=p.s, dt=dt, V=p.V, bc="dirichlet", order=p.order))
    return runs


def test_full_batch_workload_matches_oracle():
    """Every run of the full 512-run workload (the benchmark's sides, launch
    configuration and tile autotuner) over 5 steps against the FP64 oracle."""
    runs = workload_runs()
    b = BatchIntegrator(runs)
    b.autotune()
    b.step(5)
    b.sync()
    worst = 0.0
    for i, r in enumerate(runs):
        ref = O.rk4(r["psi0"], r["h"], r["a"], r["s"], r["dt"], 5, r["V"], BCS[r["bc"]], r["order"])
        got = b.numpy(i).astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        worst = max(worst, err)
        assert err <= 2e-5, (i, r["psi0"].shape, err)
    print(f"512 runs, 5 steps: largest relative L2 {worst:.2e}")


def test_batch_workload_runs_full_length_match_oracle():
    """The four smallest runs of the workload's recipe and its largest one,
    batched together over the workload's full 1000 steps, against the FP64
    oracle."""
    runs = workload_runs()
    sides = np.array([r["psi0"].shape[0] for r in runs])
    pick = list(np.argsort(sides, kind="stable")[:4]) + [int(np.argmax(sides))]
    sub = [runs[i] for i in pick]
    b = BatchIntegrator(sub)
    b.step(1000)
    b.sync()
    for i, r in enumerate(sub):
        ref = O.rk4(r["psi0"], r["h"], r["a"], r["s"], r["dt"], 1000, r["V"], BCS[r["bc"]], r["order"])
        got = b.numpy(i).astype(np.complex128)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err <= 2e-5, (pick[i], r["psi0"].shape, err)
