"""Host-side logic of bench.py that needs no GPU: the workload's time step,
the HBM roofline arithmetic, the traffic figure's source check and the
config object both arms print."""
import math

import numpy as np
import pytest

import bench
import oracle as O
from paper_1203_1263_gb300 import workloads as W


@pytest.fixture(scope="module")
def small_problem():
    return W.trap_vortex_3d(shape=(24, 20, 40), h=0.45)


def test_workload_dt_is_the_oracles_bound(small_problem):
    p = small_problem
    s_rho = abs(p.s) * float(np.max(np.abs(p.psi0))) ** 2
    ref = 0.8 * O.stability_bound(3, p.h, p.a, p.order, p.vmax(), s_rho)
    assert bench.workload_dt(p) == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("dtype,with_v", [("c64", True), ("c64", False), ("c64_acc64", True)])
def test_roofline_fraction_is_algorithmic_bytes_over_time(dtype, with_v):
    sites, step_s = 33_554_432, 1.0e-3
    r = bench.roofline_for(dtype, sites, step_s, with_v)
    peak, _ = bench.peaks()
    b = bench.ALG_BYTES[dtype][0 if with_v else 1]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["alg_bytes_per_site_step"] == b
    assert r["achieved"] == pytest.approx(sites * b / step_s / 1e9, abs=0.05)
    assert r["frac"] == pytest.approx(r["achieved"] / peak, abs=1e-4)
    assert r["peak"] == peak


def test_stage_streaming_bytes_follow_from_the_arrays():
    """Bytes per site and step of one pass per stage (Eq. RK4_GPU), V present:
    stage 1 reads Psi^n and V and writes K_tot and Psi_tmp; stages 2 and 3
    read the stage input, Psi^n, K_tot and V and write K_tot and the stage
    output; stage 4 reads the stage input, Psi^n, K_tot and V and writes
    Psi^{n+1}."""
    def step_bytes(c, v, m):
        s1 = m + v + 2 * c
        s23 = 3 * c + v + 2 * c
        s4 = c + m + c + v + m
        return s1 + 2 * s23 + s4
    assert step_bytes(16, 8, 16) == bench.ALG_BYTES["c128"][0]
    assert step_bytes(16, 0, 16) == bench.ALG_BYTES["c128"][1]
    assert step_bytes(8, 4, 8) == bench.ALG_BYTES["c64"][0]
    assert step_bytes(8, 0, 8) == bench.ALG_BYTES["c64"][1]


def test_traffic_is_reported_only_for_the_captured_sources(monkeypatch):
    nbytes, at = bench.TRAFFIC_PER_STEP["c128"]
    monkeypatch.setattr(bench, "csrc_hash", lambda: at)
    assert bench.traffic_for("c128", "trap_vortex_3d_256x256x512") == nbytes
    assert bench.traffic_for("c128", "trap_vortex_3d_87x87x203") is None
    monkeypatch.setattr(bench, "csrc_hash", lambda: "0" * 16)
    assert bench.traffic_for("c128", "trap_vortex_3d_256x256x512") is None


def test_csrc_hash_covers_the_stage_sources():
    h = bench.csrc_hash()
    assert len(h) == 16 and int(h, 16) >= 0
    assert "stage_tma.cuh" in bench.STAGE3D_SOURCES and "stage_slab.cuh" in bench.STAGE3D_SOURCES


def test_config_object_is_the_same_for_both_arms(small_problem):
    p = small_problem
    dt = bench.workload_dt(p)
    a = bench.workload_config(p, dt, "c128", 1, "trap_vortex_3d_87x87x203")
    b = bench.workload_config(p, dt, "c128", 1, "trap_vortex_3d_87x87x203")
    assert a == b
    assert a["grid"] == list(p.shape) and a["dt"] == dt and a["parallelism"] == "single"
    assert bench.workload_config(p, dt, "c128", 2, "x")["parallelism"] == "replicas"
    assert not math.isnan(a["h"])
