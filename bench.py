#!/usr/bin/env python
"""RK4 NLSE benchmark: site-updates per second of the 3D Gross-Pitaevskii
trap-vortex problem (2SHOC Laplacian, MSD walls) on one GB300.

One bench step is one RK4 time step over the whole grid (four fused stage
kernels).  `value` is timed on the device with CUDA events around K steps
whose inputs are already resident in HBM; every array is larger than L2.
`e2e` is the same metric through the public API with Psi copied from and
back to pinned host memory around each chunk of steps (the paper's frames).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank integrates its own replica of the problem
on its own GPU (the method has no data exchange between problems); rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import platform
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1203_1263_gb300 import workloads as W  # noqa: E402

WORKLOADS = {
    "trap_vortex_3d_256x256x512": dict(shape=(512, 256, 256)),
    "trap_vortex_3d_87x87x203": dict(shape=(203, 87, 87)),
    "trap_vortex_3d_256x256x256": dict(shape=(256, 256, 256)),
}
METRIC = "RK4 site-updates/s (Gsite*step/s)"
UNIT = "Gsite*step/s"
# algorithmic HBM bytes per site per RK4 step of the stage-streaming form
# (stage 1 reads Psi, V and writes K_tot, Psi_tmp; stages 2/3 read Psi_stage,
# V, Psi^n, K_tot and write K_tot, Psi_next; stage 4 reads Psi_tmp, V, K_tot,
# Psi^n and writes Psi^{n+1}):
ALG_BYTES = {  # dtype -> (with V, without V)
    "c128": (304, 272),
    "c64": (152, 136),
    "c64_acc64": (176, 160),
}
# FP64 floating-point operations per site per RK4 step of the FP64 path (FMA = 2):
# per stage |Psi|^2 (3), N = s|Psi|^2 - V (2), a*Lap = cL x the exact integer
# sum (2; the kernels fold cL into the stage coefficients, the count keeps the
# method's multiply), F (4), and the stage update (stage 1: 4, stages 2 and 3:
# 8, stage 4: 6).  The Laplacian's stencil sums run on the integer pipe.
FP64_FLOPS_PER_SITE_STEP = 15 + 19 + 19 + 17
CHUNK = 56   # steps per frame in the end-to-end measurement (the 87x87x203 run's chunk size)


# Kernel launches per RK4 step of the 3D tiled path (every extent >= 7, x >= 10): per stage one
# deep-interior kernel and three wall-slab kernels; the FP64 exact-sum form adds the one-thread kernel
# that sets the next step's fixed-point scale.
LAUNCHES_PER_STEP = {"c128": 17, "c64": 16, "c64_acc64": 16}

# DRAM bytes (read + write) per RK4 step of the stage kernels on trap_vortex_3d_256x256x512, from one
# ncu capture (profiles/rk4_step_256x256x512_traffic_and_launches.md), with the hash of the 3D stage
# path's sources it was taken at: the figure is reported only while csrc_hash() still matches.
TRAFFIC_PER_STEP = {  # dtype -> (bytes per step, csrc hash of the capture)
    "c128": (10875.0e6, "ffb04f0babceec4d"),
    "c64": (5536.7e6, "ffb04f0babceec4d"),
    "c64_acc64": (6315.0e6, "ffb04f0babceec4d"),
}

# The sources the 3D stage path (deep kernels, wall slabs, scale update, step loop) is built from.
STAGE3D_SOURCES = ("api.cu", "reduce.cu", "nlse_device.cuh", "nlse_internal.h", "stage_3d_impl.cuh",
                   "stage_3d_p32_o2.cu", "stage_3d_p32_o4.cu", "stage_3d_p64_o2.cu", "stage_3d_p64_o4.cu",
                   "stage_3d_pmix_o2.cu", "stage_3d_pmix_o4.cu", "stage_generic.cuh", "stage_slab.cuh",
                   "stage_tiled.cuh", "stage_tma.cuh")


def workload_dt(p):
    """The bench workload's time step, the same in both arms: 0.8 x the RK4 stability bound with the
    potential and the nonlinearity, 2 sqrt(2) / (a rho_L + max|V| + |s| max|Psi|^2), rho_L = 4d/h^2 (CD)
    or 16d/(3h^2) (2SHOC)."""
    rho = 4.0 * p.dims / p.h ** 2 if p.order == 2 else 16.0 * p.dims / (3.0 * p.h ** 2)
    s_rho = abs(p.s) * float(np.max(np.abs(p.psi0))) ** 2
    return 0.8 * 2.0 * math.sqrt(2.0) / (p.a * rho + p.vmax() + s_rho)


def csrc_hash():
    """sha256 (first 16 hex digits) over the sources of the 3D stage path."""
    import hashlib
    h = hashlib.sha256()
    for name in STAGE3D_SOURCES:
        h.update(name.encode())
        h.update(open(os.path.join(ROOT, "paper_1203_1263_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(dtype, workload):
    """ncu bytes per step for the current kernels, or None (other workload, or kernels changed since)."""
    if workload != "trap_vortex_3d_256x256x512" or dtype not in TRAFFIC_PER_STEP:
        return None
    nbytes, at = TRAFFIC_PER_STEP[dtype]
    return nbytes if at is not None and at == csrc_hash() else None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def bf16_peak():
    """Dense bf16 tensor peak (TFLOP/s, burst) and where it came from."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]), "measured bf16 burst (cuBLAS)"
    return 1900.0, "fallback bf16 burst"


# FP64 peak of a GB300: 152 SMs x 2 FP64 FMA lanes per cycle x 2 flops at the
# 2070 MHz maximum clock = 1.26 TFLOP/s nominal.  The figure the FP64 view is
# taken against is measured live (fp64_peak) before the timed region.
FP64_PEAK_NOMINAL = 1.26
_FP64_PEAK = None


def fp64_peak():
    """Dense FP64 throughput of this GPU (TFLOP/s) and how it was obtained: cuBLAS DGEMM 4096^3
    (2 N^3 flops), best of 3 after one warm-up, timed with CUDA events; the nominal figure if no GPU."""
    global _FP64_PEAK
    if _FP64_PEAK is None:
        try:
            import torch
            n = 4096
            a = torch.randn(n, n, dtype=torch.float64, device="cuda")
            b = torch.randn(n, n, dtype=torch.float64, device="cuda")
            torch.matmul(a, b)
            best = None
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                e1.synchronize()
                t = e0.elapsed_time(e1) * 1e-3
                best = t if best is None else min(best, t)
            del a, b
            _FP64_PEAK = (2.0 * n ** 3 / best / 1e12, "measured live: cuBLAS DGEMM 4096^3, best of 3")
        except Exception:   # no GPU: the nominal figure
            _FP64_PEAK = (FP64_PEAK_NOMINAL, "nominal (152 SMs x 2 FP64 FMA lanes x 2 flops x 2070 MHz)")
    return _FP64_PEAK


def roofline_for(dtype, sites, step_s, with_v):
    """HBM roofline of one RK4 step on the stage-streaming bytes (304 B per site with V for FP64, 152 B
    for FP32, 176 B for FP32 stages with the FP64 master), and, for FP64, the FP64-pipe view (the pipe
    that binds that form on GB300) as a second figure."""
    hbm_peak, kind = peaks()
    bytes_site = ALG_BYTES[dtype][0 if with_v else 1]
    gbs = sites * bytes_site / step_s / 1e9
    hbm = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_peak, "unit": "GB/s",
           "frac": round(gbs / hbm_peak, 4), "peak_kind": kind + " (MEASURED_PEAKS.json copy bandwidth)",
           "alg_bytes_per_site_step": bytes_site}
    if dtype == "c128":
        tflops = sites * FP64_FLOPS_PER_SITE_STEP / step_s / 1e12
        pk, pk_kind = fp64_peak()
        hbm["fp64_pipe_view"] = {"achieved": round(tflops, 4), "peak": round(pk, 4), "unit": "TFLOP/s",
                                 "frac": round(tflops / pk, 4), "peak_kind": pk_kind,
                                 "flops_per_site_step": FP64_FLOPS_PER_SITE_STEP}
    return hbm


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples go to a temporary file, or to NLSE_CLOCKS_DIR when that is set
        out_dir = os.environ.get("NLSE_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"nlse_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def build_problem(name):
    spec = WORKLOADS[name]
    return W.trap_vortex_3d(shape=spec["shape"])


def slowest_rank(seconds, device, dist=None):
    """The job's time across replicas: the maximum of every rank's `seconds`
    (each rank integrates its own replica; nothing else is exchanged)."""
    import torch
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(site_steps_per_rank, seconds, device, world=1, dist=None):
    """Whole-job Gsite-step/s: all ranks' site-steps over the slowest rank's time."""
    return world * site_steps_per_rank / slowest_rank(seconds, device, dist) / 1e9


def workload_config(p, dt, precision, world, workload):
    """The `config` object of the JSON line (the same for both arms)."""
    big = p.sites * 16 > 129e6
    return {"workload": workload, "grid": list(p.shape), "h": p.h, "a": p.a, "s": p.s, "order": p.order,
            "bc": "msd", "dt": dt, "precision": precision,
            "l2": ("inputs larger than L2 (%.0f MB per state array)" % (p.sites * 16 / 1e6)) if big else
                  "state fits in L2",
            "parallelism": "replicas" if world > 1 else "single"}


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1203_1263_gb300.integrator import Integrator, max_dt

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    p = build_problem(args.workload)
    s_rho = abs(p.s) * float(np.max(np.abs(p.psi0))) ** 2
    dt = workload_dt(p)
    sites = p.sites
    stream = torch.cuda.Stream(dev)

    def timed(dtype, K, Wm, bc="msd", prob=None, dt_=None, repeats=1, sample_clocks=False):
        """K steps timed with CUDA events on the integrator's stream, `repeats` times; returns the
        integrator, the milliseconds of each repeat and the clock record."""
        prob = p if prob is None else prob
        dt_ = dt if dt_ is None else dt_
        with torch.cuda.stream(stream):
            g = Integrator(prob.psi0, prob.h, prob.a, prob.s, prob.V, bc, prob.order, dtype, device=dev, stream=stream)
            if args.variant is not None or args.tile != -1:
                g.set_kernel(args.variant if args.variant is not None else (2 if dtype == "c128" else 1), args.tile)
            g.step(Wm, dt_)
            g.sync()
            barrier()
            clk = ClockSampler(local_rank) if sample_clocks else None
            if clk:
                clk.start()
            ms = []
            for _ in range(repeats):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.step(K, dt_)
                e1.record(stream)
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            clocks = clk.stop() if clk else None
            g.sync()
            barrier()
        return g, ms, clocks

    K, Wm = args.steps, args.warmup
    # the timed region of the contract is the first repeat; the others give the median of the spread
    g64, ms_all, clocks = timed(args.dtype, K, Wm, repeats=max(1, args.repeats), sample_clocks=True)
    ms_max = slowest_rank(ms_all[0], dev, dist)
    value = world * sites * K / (ms_max * 1e-3) / 1e9

    result, details, forms = None, {}, {}
    if rank == 0:
        step_s = ms_max * 1e-3 / K
        roof = roofline_for(args.dtype, sites, step_s, p.V is not None)
        roof["traffic"] = traffic_for(args.dtype, args.workload)
        roof["traffic_unit"] = "bytes per RK4 step (ncu dram__bytes_read.sum + dram__bytes_write.sum)"
        roof["kernel"] = ("one RK4 step: 4 fused stage kernels (deep interior, TMA-fed) + 12 wall-slab kernels "
                          "(3 per stage, shared-memory staged)")
        med = statistics.median(ms_all) / K
        result = {
            "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": Wm,
            "ms_per_step": round(ms_max / K, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"c128": "f64", "c64": "f32", "c64_acc64": "f32+f64acc"}[args.dtype],
            "data": "synthetic (seeded trap-vortex IC, no dataset)",
            "config": workload_config(p, dt, args.dtype, world, args.workload),
            "roofline": roof, "clocks": clocks, "gpu_launches": LAUNCHES_PER_STEP[args.dtype] * K,
            "timing": {"repeats": len(ms_all), "ms_per_step": [round(m / K, 4) for m in ms_all],
                       "median_ms_per_step": round(med, 4),
                       "median_value": round(sites / (med * 1e-3) / 1e9, 4)},
        }

    # ---- other precision forms and boundaries on the same problem (speed-up over FP64 at a stated accuracy) ----
    if not args.no_forms and rank == 0:
        ref_state = g64.numpy()
        ref_steps = Wm + len(ms_all) * K   # steps the headline form has taken
        for dt_name in ("c64", "c64_acc64"):
            if dt_name == args.dtype:
                continue
            g2, ms2, _ = timed(dt_name, K, Wm)
            g2.step(ref_steps - (Wm + K), dt)   # (untimed) to the headline form's step count
            g2.sync()
            st = g2.numpy().astype(np.complex128)
            rl2 = float(np.linalg.norm((st - ref_state).ravel()) / np.linalg.norm(ref_state.ravel()))
            v2 = sites * K / (ms2[0] * 1e-3) / 1e9
            r2 = roofline_for(dt_name, sites, ms2[0] * 1e-3 / K, p.V is not None)
            r2["traffic"] = traffic_for(dt_name, args.workload)
            details[dt_name] = {"value": round(v2, 4), "unit": UNIT, "speedup_vs_f64": round(v2 / value, 3),
                                "rel_l2_vs_f64_gpu": rl2, "rel_l2_after_steps": ref_steps, "roofline": r2}
            forms[dt_name] = {"value": round(v2, 3), "x_f64": round(v2 / value, 3), "hbm_frac": r2["frac"],
                              "rel_l2_vs_f64": float("%.2e" % rl2)}
            g2.close()
        # the Laplacian-zero and periodic boundaries on the same grid: only the shell kernels differ
        for bc in ("l0", "periodic"):
            for dt_name in ("c128", "c64"):
                g3, ms3, _ = timed(dt_name, K, Wm, bc)
                v3 = sites * K / (ms3[0] * 1e-3) / 1e9
                r3 = roofline_for(dt_name, sites, ms3[0] * 1e-3 / K, p.V is not None)
                r3["traffic"] = None
                details[f"{dt_name}_{bc}"] = {"value": round(v3, 4), "unit": UNIT, "bc": bc, "roofline": r3}
                forms[f"{dt_name}_{bc}"] = {"value": round(v3, 3), "hbm_frac": r3["frac"]}
                g3.close()
        # the paper's headline grid (87 x 87 x 203; the state fits in L2) and the precision form's 512^3 grid
        p87 = W.trap_vortex_3d(shape=(203, 87, 87))
        dt87 = 0.8 * max_dt(3, p87.h, p87.a, 4, p87.vmax(), abs(p87.s) * float(np.max(np.abs(p87.psi0))) ** 2)
        for dt_name in ("c128", "c64_acc64"):
            g4, ms4, _ = timed(dt_name, 4 * K, Wm, prob=p87, dt_=dt87)
            v4 = p87.sites * 4 * K / (ms4[0] * 1e-3) / 1e9
            details[f"trap_87x87x203_{dt_name}"] = {"value": round(v4, 4), "unit": UNIT, "steps": 4 * K,
                                                    "ms_per_step": round(ms4[0] / (4 * K), 4)}
            forms[f"trap87_{dt_name}"] = {"value": round(v4, 3)}
            g4.close()
        del p87
        if args.rings:
            details["rings_512cube"] = rings_form(args, dev, timed, K, Wm)
            forms["rings512"] = {k: details["rings_512cube"][k] for k in ("c128", "c64_acc64", "x_f64",
                                                                         "rel_l2_after_steps")}
        details["soliton_1d_2001"] = soliton_form(dev)
        forms["soliton1d"] = {f"us_per_step_{k}": details["soliton_1d_2001"][k]["us_per_step"]
                              for k in ("c128", "c64")}

    if not args.no_batch and rank == 0:
        details["batch"] = batch_form(args, dev, min(K, 200), Wm)
        b = details["batch"]
        forms["batch"] = {"value": round(b["value"], 3), "x_f64": b["speedup_vs_f64"], "hbm_frac": b["roofline"]["frac"],
                          "rel_l2_vs_f64": float("%.2e" % b["max_rel_l2_vs_f64_gpu"])}

    if not args.no_surrogate and rank == 0:
        details["surrogate"] = surrogate_form(args, dev)
        su = details["surrogate"]
        forms["surrogate"] = {"train_tflops": su.get("train_tflops"), "bf16_frac": su["roofline"]["frac"]}
        if "rollout_t20" in su:
            sm = su["rollout_t20"]["summary"]
            forms["surrogate"].update({m: {"x_f64": sm[m]["mean_speedup_vs_f64"], "accepted": sm[m]["accepted_windows"],
                                           "final_rel_l2": float("%.2e" % sm[m]["max_final_rel_l2_vs_plain_f64"])}
                                       for m in ("parallel", "sampled")})

    if not args.no_paper_tables and rank == 0:
        result["paper_tables"] = paper_tables(dev)
    if args.chunk_study and rank == 0:
        result["chunk_study"] = chunk_study(dev)

    # ---- end to end through the public API: pinned host Psi in, CHUNK steps, Psi and mass out ----
    if not args.no_e2e:
        import torch
        host_np = p.psi0.astype(np.complex64) if args.dtype == "c64" else p.psi0
        host_in = torch.from_numpy(np.ascontiguousarray(host_np)).pin_memory()
        host_out = torch.empty_like(host_in).pin_memory()
        frames = max(3, K // CHUNK)
        with torch.cuda.stream(stream):
            g = Integrator(p.psi0, p.h, p.a, p.s, p.V, "msd", p.order, args.dtype, device=dev, stream=stream)
            if args.variant is not None or args.tile != -1:
                g.set_kernel(args.variant if args.variant is not None else (2 if args.dtype == "c128" else 1), args.tile)
            dev_psi = g.psi
            g.step(CHUNK, dt)        # untimed frame: builds the step graph
            g.sync()
            barrier()
            w0 = time.perf_counter()
            for _ in range(frames):
                dev_psi.copy_(host_in, non_blocking=True)
                g.step(CHUNK, dt)
                host_out.copy_(dev_psi, non_blocking=True)
                g.mass()          # synchronises the stream: the frame's result is on the host
            wall = time.perf_counter() - w0
            barrier()
        e2e_v = job_throughput(sites * CHUNK * frames, wall, dev, world, dist)
        if rank == 0:
            nbytes = host_in.numel() * host_in.element_size()
            result["e2e"] = {"value": round(e2e_v, 4), "unit": UNIT,
                             "h2d_bytes_per_step": nbytes // CHUNK, "d2h_bytes_per_step": (nbytes + 8) // CHUNK,
                             "chunk_steps": CHUNK, "frames": frames}

    # ---- CPU baseline: the oracle on a bounded sample of the same workload ----
    if rank == 0 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(p, dt, budget_s=args.cpu_budget)
    if rank == 0:
        if details:
            result["details"] = details
        if forms:      # last, so that the summary of every form is in the tail of the line
            result["forms"] = forms
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return result


def rings_form(args, dev, timed, K, Wm):
    """The precision form's workload: 512^3 vortex rings (h = 0.25, V = 0, MSD, 2SHOC), FP64 against FP32
    stages with the FP64 master and accumulator, K steps each, and their relative L2 after them."""
    pr = W.vortex_rings_3d(n=512)
    dtr = 0.8 * nlse_bound(pr)
    out = {"grid": list(pr.shape), "dt": dtr, "steps": K}
    states = {}
    for dt_name in ("c128", "c64_acc64"):
        g, ms, _ = timed(dt_name, K, Wm, prob=pr, dt_=dtr)
        v = pr.sites * K / (ms[0] * 1e-3) / 1e9
        r = roofline_for(dt_name, pr.sites, ms[0] * 1e-3 / K, False)
        out[dt_name] = round(v, 3)
        out[dt_name + "_roofline"] = r
        states[dt_name] = g.numpy()
        g.close()
    a, b = states["c128"], states["c64_acc64"]
    out["rel_l2_after_steps"] = float("%.2e" % (np.linalg.norm((b - a).ravel()) / np.linalg.norm(a.ravel())))
    out["x_f64"] = round(out["c64_acc64"] / out["c128"], 3)
    out["warmup_plus_steps"] = Wm + K
    return out


def nlse_bound(p):
    from paper_1203_1263_gb300.integrator import max_dt
    return max_dt(p.dims, p.h, p.a, p.order, p.vmax(), abs(p.s) * float(np.max(np.abs(p.psi0))) ** 2)


def soliton_form(dev, steps=32000):
    """The 1D bright soliton (N = 2001, h = 0.05, dt = h^2/8, Dirichlet, 2SHOC) over its 32,000 steps to
    t = 10 through one nlse_step call (CUDA events), FP64 and FP32: the line runs on one thread-block
    cluster; a tenth of the steps on the per-site kernel for comparison."""
    import torch
    from paper_1203_1263_gb300.integrator import Integrator
    p = W.bright_soliton_1d(order=4)
    out = {"grid": list(p.shape), "dt": p.dt, "steps": steps}
    stream = torch.cuda.Stream(dev)
    for dt_name, per_site in (("c128", 0), ("c64", 0)):   # the per-site kernel of the default's arithmetic
        row = {}
        for variant, n in ((None, steps), (per_site, steps // 10)):
            with torch.cuda.stream(stream):
                g = Integrator(p.psi0, p.h, p.a, p.s, None, "dirichlet", 4, dt_name, device=dev, stream=stream)
                if variant is not None:
                    g.set_kernel(variant)
                g.step(64, p.dt)
                g.sync()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.step(n, p.dt)
                e1.record(stream)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                key = "default" if variant is None else "per_site_kernel"
                row[key] = {"kernel": g.kernel_in_use(), "value": round(p.sites * n / (ms * 1e-3) / 1e9, 4),
                            "unit": UNIT, "us_per_step": round(ms * 1e3 / n, 3)}
                g.close()
        row["us_per_step"] = row["default"]["us_per_step"]
        row["seconds_for_32000_steps"] = round(row["default"]["us_per_step"] * 32000 / 1e6, 4)
        row["x_per_site_kernel"] = round(row["per_site_kernel"]["us_per_step"] / row["default"]["us_per_step"], 2)
        out[dt_name] = row
    return out


# The paper's GPU times (seconds) for its timing workloads, 10,000 steps, chunk
# 5000 (Sec. 7, Tables 1-3): (RK4+CD in FP32, RK4+2SHOC in FP64), GTX 580.
PAPER_TABLE_SECONDS = {
    1: {1000: (0.21, 0.49), 10000: (0.24, 0.67), 100000: (1.21, 4.52), 1000000: (9.41, 39.72),
        3000000: (27.65, 117.32)},
    2: {961: (0.29, 0.59), 10000: (0.34, 1.09), 99856: (1.76, 6.25), 1000000: (14.94, 54.65),
        2999824: (42.15, 162.79)},
    3: {9261: (0.59, 2.00), 97336: (2.90, 13.34), 970299: (31.85, 131.74), 2985984: (82.14, 365.47)},
}


def _timed_frames(p, dtype, order, dev, nsteps, chunk):
    """Wall seconds of the paper's usage through the public API: Psi from
    pinned host memory to the device, then nsteps in chunks of `chunk` with
    Psi copied back to pinned host memory after each chunk."""
    import torch
    from paper_1203_1263_gb300.integrator import Integrator
    host_np = p.psi0.astype(np.complex64) if dtype == "c64" else p.psi0
    host_in = torch.from_numpy(np.ascontiguousarray(host_np)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    stream = torch.cuda.Stream(dev)
    with torch.cuda.stream(stream):
        g = Integrator(p.psi0, p.h, p.a, p.s, p.V, "msd", order, dtype, device=dev, stream=stream)
        g.step(min(chunk, 16) + 1, p.dt)      # untimed: builds the step graph
        g.sync()
        w0 = time.perf_counter()
        g.psi.copy_(host_in, non_blocking=True)
        done = 0
        while done < nsteps:
            n = min(chunk, nsteps - done)
            g.step(n, p.dt)
            host_out.copy_(g.psi, non_blocking=True)
            stream.synchronize()
            done += n
        wall = time.perf_counter() - w0
        g.sync()
        g.close()
    return wall


def paper_tables(dev):
    """The timing runs of Sec. 7 (Tables 1-3) on this GPU: the dark soliton
    (1D), dark vortex (2D) and vortex ring (3D) workloads, 10,000 steps at
    k = 0.005 in chunks of 5000, RK4+CD in FP32 and RK4+2SHOC in FP64."""
    rows = []
    for dims, table in PAPER_TABLE_SECONDS.items():
        for total, (paper_cd, paper_2shoc) in table.items():
            row = {"dims": dims, "sites": total}
            for key, dtype, order, paper_s in (("cd_f32", "c64", 2, paper_cd), ("2shoc_f64", "c128", 4, paper_2shoc)):
                p = W.paper_timing_problem(dims, total, order)
                row["grid"] = list(p.shape)
                try:
                    sec = _timed_frames(p, dtype, order, dev, p.steps, 5000)
                except RuntimeError as e:      # e.g. NLSE_ENONFINITE: the run is reported, not timed
                    row[key] = {"error": str(e)[:200], "paper_seconds": paper_s}
                    continue
                row[key] = {"seconds": round(sec, 4), "Msite_step_s": round(p.sites * p.steps / sec / 1e6, 1),
                            "paper_seconds": paper_s, "speedup_vs_paper_gpu": round(paper_s / sec, 1)}
            rows.append(row)
    return {"workloads": "Sec. 4 dark soliton (1D, h=0.1), dark vortex (2D, h=0.25), vortex ring (3D, h=1.5); "
                         "MSD, k=0.005, 10,000 steps, chunks of 5000 with Psi to and from pinned host memory",
            "paper_gpu": "GeForce GTX 580 (Sec. 7)", "rows": rows}


def chunk_study(dev):
    """Slowdown against chunk size (Sec. 7, chunk-size figure): 1000 steps
    (t = 5) of the timing workloads at about 1e3 and 1e6 sites, Psi copied
    back to the host after every chunk; slowdown = time(chunk) / time(1000)."""
    out = []
    for dims, sizes in ((1, (1000, 1000000)), (2, (961, 1000000)), (3, (9261, 970299))):
        for total in sizes:
            for key, dtype, order in (("cd_f32", "c64", 2), ("2shoc_f64", "c128", 4)):
                p = W.paper_timing_problem(dims, total, order)
                t = {c: _timed_frames(p, dtype, order, dev, 1000, c) for c in (1000, 100, 10, 1)}
                out.append({"dims": dims, "sites": p.sites, "scheme": key, "seconds_chunk_1000": round(t[1000], 4),
                            "slowdown": {str(c): round(t[c] / t[1000], 2) for c in (100, 10, 1)}})
    return out


def batch_form(args, dev, K, Wm):
    """512 independent uneven 2D runs (sides 64..1024, mixed a, s, V, order,
    complex64) advanced together, against the plain FP64 GPU path (one
    context per run, run one after another) and single-run FP32 contexts."""
    import torch
    from paper_1203_1263_gb300.integrator import BatchIntegrator, Integrator, max_dt
    runs = []
    for d in W.batch_runs_2d(nruns=args.batch_runs, seed=4):
        p = W.batch_run_problem(d)
        s_rho = abs(p.s) * float(np.max(np.abs(p.psi0))) ** 2
        dt = 0.8 * max_dt(2, p.h, p.a, p.order, p.vmax(), s_rho)
        runs.append(dict(psi0=p.psi0, h=p.h, a=p.a, s=p.s, dt=dt, V=p.V, bc="dirichlet", order=p.order))
    sites = sum(r["psi0"].size for r in runs)
    stream = torch.cuda.Stream(dev)

    def timed(fn, steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn(steps)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3

    with torch.cuda.stream(stream):
        b = BatchIntegrator(runs, device=dev, stream=stream)
        if args.batch_tile is None:
            tile, _ = b.autotune()
        else:
            tile = args.batch_tile
            b.set_tile(tile)
        b.step(Wm)
        b.sync()
        t_batch = timed(b.step, K)
        b.sync()
        out = {}
        for dtype in ("c128", "c64"):
            gs = [Integrator(r["psi0"], r["h"], r["a"], r["s"], r["V"], "dirichlet", r["order"], dtype,
                             device=dev, stream=stream) for r in runs]
            for g, r in zip(gs, runs):
                g.step(Wm, r["dt"])
            torch.cuda.synchronize(dev)
            t = timed(lambda n: [g.step(n, r["dt"]) for g, r in zip(gs, runs)], K)
            out[dtype] = (t, gs)
        ref = out["c128"][1]
        errs = [float(np.linalg.norm(b.numpy(i).astype(np.complex128) - ref[i].numpy()) /
                      np.linalg.norm(ref[i].numpy())) for i in range(len(runs))]
    v_batch = sites * K / t_batch / 1e9
    v64 = sites * K / out["c128"][0] / 1e9
    v32 = sites * K / out["c64"][0] / 1e9
    return {"value": round(v_batch, 4), "unit": UNIT, "runs": len(runs), "sites": int(sites), "steps": K,
            "tile_cfg": tile, "speedup_vs_f64": round(v_batch / v64, 3),
            "f64_sequential": round(v64, 4), "f32_sequential": round(v32, 4),
            "speedup_vs_f32_sequential": round(v_batch / v32, 3),
            "max_rel_l2_vs_f64_gpu": max(errs), "dtype": "f32",
            "roofline": roofline_for("c64", sites, t_batch / K, True)}


def cpu_model():
    """The host CPU's model name (lscpu), for the record next to the oracle's timings."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def oracle_rate(p, dt, threads, budget_s, nsteps=2):
    """The oracle as it stands on `threads` host threads, on a z-slab of the workload sized to take about
    budget_s seconds: (Gsite*step/s, threads used, sample description)."""
    import oracle
    used = oracle.set_threads(threads)
    nz_probe = min(p.shape[0], 16 if threads > 1 else 5)
    sl = np.ascontiguousarray(p.psi0[:nz_probe])
    Vs = np.ascontiguousarray(p.V[:nz_probe]) if p.V is not None else None
    t0 = time.perf_counter()
    oracle.rk4(sl, p.h, p.a, p.s, dt, 1, Vs, p.bc, p.order)
    per_site = (time.perf_counter() - t0) / sl.size
    nz = int(max(5, min(p.shape[0], budget_s / (per_site * nsteps * sl[0].size))))
    sl = np.ascontiguousarray(p.psi0[:nz])
    Vs = np.ascontiguousarray(p.V[:nz]) if p.V is not None else None
    t0 = time.perf_counter()
    oracle.rk4(sl, p.h, p.a, p.s, dt, nsteps, Vs, p.bc, p.order)
    el = time.perf_counter() - t0
    return sl.size * nsteps / el / 1e9, used, (f"{nsteps} RK4 steps on a {nz}x{p.shape[1]}x{p.shape[2]} slab of the "
                                               f"workload ({el:.1f} s, FP64, {platform.machine()})")


def cpu_baseline(p, dt, budget_s=20.0):
    """The oracle as it stands on all host cores (the value) and on one core (the paper's serial baseline)."""
    v, cores, sample = oracle_rate(p, dt, os.cpu_count() or 1, budget_s)
    v1, _, sample1 = oracle_rate(p, dt, 1, budget_s / 2)
    return {"value": round(v, 6), "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
            "cpu_model": cpu_model(), "serial": {"value": round(v1, 6), "unit": UNIT, "cores": 1, "sample": sample1}}


# ---------------------------------------------------------------------------
# reference arm: the oracle (plain FP64 CPU program) on the same metric
# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    p = build_problem(args.workload)
    s_rho = abs(p.s) * float(np.max(np.abs(p.psi0))) ** 2
    dt = workload_dt(p)
    cores = oracle.set_threads(os.cpu_count() or 1)
    # one bench step = one RK4 step on a z-slab sized to ~budget / (K + W) seconds
    per_step_budget = max(0.5, args.ref_budget / max(1, args.steps + args.warmup))
    probe = np.ascontiguousarray(p.psi0[:8])
    Vp = np.ascontiguousarray(p.V[:8])
    t0 = time.perf_counter()
    oracle.rk4(probe, p.h, p.a, p.s, dt, 1, Vp, p.bc, p.order)
    per_plane = (time.perf_counter() - t0) / 8
    nz = int(max(5, min(p.shape[0], per_step_budget / per_plane)))
    psi = np.ascontiguousarray(p.psi0[:nz])
    V = np.ascontiguousarray(p.V[:nz])
    psi = oracle.rk4(psi, p.h, p.a, p.s, dt, args.warmup, V, p.bc, p.order)
    t0 = time.perf_counter()
    oracle.rk4(psi, p.h, p.a, p.s, dt, args.steps, V, p.bc, p.order)
    el = time.perf_counter() - t0
    v = psi.size * args.steps / el / 1e9
    sample = f"{args.steps} RK4 steps on a {nz}x{p.shape[1]}x{p.shape[2]} slab of the workload"
    return {"impl": "reference", "metric": METRIC, "value": round(v, 6), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded trap-vortex IC, no dataset)",
            "config": workload_config(p, dt, "c128", world, args.workload),
            "cpu_baseline": {"value": round(v, 6), "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu_model": cpu_model()},
            "e2e": {"value": round(v, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def surrogate_form(args, dev):
    """Learned surrogate on the 2D focusing workload (256 x 256, h = 0.2, one
    window = 32 RK4 steps of dt = 0.005): tensor-core throughput of training
    and inference, then a budgeted training run on FP64-integrator pairs and
    RK4-checked rollouts to t = 20 (125 windows) against plain FP64 RK4."""
    import torch
    from paper_1203_1263_gb300.integrator import Integrator
    from paper_1203_1263_gb300.surrogate import FOCUSING, Surrogate, generate_pairs, rollout, train
    n, C, nl, dil, nb = 256, 64, 6, (1, 2, 4, 8, 4, 1), 16
    h, dt, win = FOCUSING["h"], FOCUSING["dt"], FOCUSING["window"]
    stream = torch.cuda.current_stream(dev)
    out = {"grid": [n, n], "channels": C, "layers": nl, "dilations": list(dil), "batch": nb,
           "window_steps": win, "dt": dt, "dtype": "bf16 operands, f32 accumulate"}

    def ev_time(fn, reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) * 1e-3 / reps

    # ---- kernel throughput on seeded states (a separate instance: these steps move its weights) ----
    probe = Surrogate(n, n, channels=C, layers=nl, dilations=dil, max_batch=nb, seed=3)
    x = torch.as_tensor(np.stack([W.humps_2d(11, i, n=n, h=h) for i in range(nb)]), dtype=torch.complex64,
                        device=dev)
    y = x * np.exp(0.1j)
    for _ in range(3):
        probe.train_step(x, y, 1e-4, want_loss=False)
    t_train = ev_time(lambda: probe.train_step(x, y, 1e-4, want_loss=False), 20)
    t_fwd = ev_time(lambda: probe.forward(x, project=True), 20)
    x1 = x[:1].contiguous()
    t_fwd1 = ev_time(lambda: probe.forward(x1, project=True), 20)
    probe.close()
    peak_tf, peak_kind = bf16_peak()
    train_tf = probe.train_flops_per_state() * nb / t_train / 1e12
    fwd_tf = probe.flops_per_state() * nb / t_fwd / 1e12
    out["train_tflops"] = round(train_tf, 2)
    out["train_states_per_s"] = round(nb / t_train, 1)
    out["infer_tflops"] = round(fwd_tf, 2)
    out["infer_ms_per_window_batch16"] = round(t_fwd / nb * 1e3, 4)
    out["infer_ms_per_window_single"] = round(t_fwd1 * 1e3, 4)
    out["roofline"] = {"bound": "tensor", "achieved": round(train_tf, 2), "peak": peak_tf, "unit": "TFLOP/s",
                       "frac": round(train_tf / peak_tf, 4) if peak_tf else None, "traffic": None,
                       "kernel": "one training step (forward, backward-data, weight-gradient convolutions)",
                       "peak_kind": peak_kind}
    # ---- one window of plain RK4 on one 256 x 256 state ----
    psi_probe = W.humps_2d(11, 0, n=n, h=h)
    for dtype in ("c128", "c64"):
        g = Integrator(psi_probe, h, FOCUSING["a"], FOCUSING["s"], None, "dirichlet", 4, dtype, device=dev)
        g.step(win, dt)
        torch.cuda.synchronize(dev)
        out[f"rk4_ms_per_window_{dtype}"] = round(ev_time(lambda: g.step(win, dt), 10) * 1e3, 4)
        g.close()
    if args.surrogate_kernels_only:
        return out
    # ---- RK4 windows of 8 states at once on separate streams (the parallel checker's cost) ----
    from paper_1203_1263_gb300.surrogate import RK4Pool
    pool = RK4Pool(n, 8, device=dev)
    sts = [x[i] for i in range(8)]
    pool.advance(sts)
    torch.cuda.synchronize(dev)
    out["rk4_ms_per_window_c128_8_streams"] = round(ev_time(lambda: pool.advance(sts), 5) / 8 * 1e3, 4)
    pool.close()
    out["infer_speedup_vs_rk4_c128_unchecked"] = round(out["rk4_ms_per_window_c128"] / out["infer_ms_per_window_batch16"], 2)
    # ---- budgeted training on FP64-integrator pairs, then rollouts ----
    t0 = time.perf_counter()
    X, Y, kept = generate_pairs(args.sur_traj, 125, n=n, seed=5, device=dev)
    t_gen = time.perf_counter() - t0
    sur = Surrogate(n, n, channels=C, layers=nl, dilations=dil, max_batch=32, seed=7)
    t0 = time.perf_counter()
    hist = train(sur, X, Y, epochs=args.sur_epochs, batch=32, lr=5e-4, lr_end=1e-5, seed=0, noise=3e-3,
                 mass_weight=args.sur_mass_weight)
    torch.cuda.synchronize(dev)
    t_train_run = time.perf_counter() - t0
    del X, Y
    held = []
    for j in range(12):         # held-out initial states whose trajectories do not collapse
        Xh, _, k = generate_pairs(1, 125, n=n, seed=99 + j, device=dev)
        if k:
            held.append((99 + j, Xh[0].cpu().numpy().astype(np.complex128)))
        if len(held) == 3:
            break
    out["training"] = {"pairs": int(kept * 125), "trajectories": kept, "epochs": args.sur_epochs, "batch": 32,
                       "lr": "cosine 5e-4 -> 1e-5", "input_noise": 3e-3, "mass_weight": args.sur_mass_weight,
                       "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                       "data_seconds": round(t_gen, 2), "train_seconds": round(t_train_run, 2)}
    psi_w = held[0][1]
    rollout(None, psi_w, 2)                      # first calls load the kernels of the checks
    rollout(sur, psi_w, 2, mode="strict")
    rollout(sur, psi_w, 2, mode="parallel", width=8)
    per_state = []
    for seed, psi0 in held:
        ref, st_plain = rollout(None, psi0, 125)
        rolls = {"seed": seed, "plain_f64_seconds": round(st_plain.seconds, 4)}
        for mode in ("strict", "sampled", "parallel"):
            got, st = rollout(sur, psi0, 125, mode=mode, every=4, width=8)
            err = float(sur.compare(got[None], ref[None])[0])
            rolls[mode] = {"seconds": round(st.seconds, 4),
                           "speedup_vs_f64": round(st_plain.seconds / st.seconds, 3),
                           "accepted_windows": st.accepted, "rk4_windows": st.rk4_windows, "checked": st.checked,
                           "rejected_l2": st.rejected_l2, "rejected_mass": st.rejected_mass,
                           "max_raw_mass_drift_vs_m0": st.max_mass_drift,
                           "median_check_rel_l2": float(np.median(st.l2_errors)) if st.l2_errors else None,
                           "final_rel_l2_vs_plain_f64": err}
        per_state.append(rolls)
    summary = {m: {"mean_speedup_vs_f64": round(float(np.mean([r[m]["speedup_vs_f64"] for r in per_state])), 3),
                   "accepted_windows": [r[m]["accepted_windows"] for r in per_state],
                   "max_final_rel_l2_vs_plain_f64": max(r[m]["final_rel_l2_vs_plain_f64"] for r in per_state)}
               for m in ("strict", "sampled", "parallel")}
    out["rollout_t20"] = {"windows": 125, "every": 4, "parallel_width": 8,
                          "tolerances": {"rel_l2": 1e-2, "mass_drift_of_raw_output_vs_m0": 1e-4},
                          "summary": summary, "held_out": per_state}
    sur.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="trap_vortex_3d_256x256x512")
    ap.add_argument("--dtype", choices=["c128", "c64", "c64_acc64"], default="c128")
    ap.add_argument("--variant", type=int, default=None,
                    help="stage kernel (default: the library's per-precision default)")
    ap.add_argument("--tile", type=int, default=-1, help="tiled kernel CTA shape (-1 default)")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--batch-runs", type=int, default=512)
    ap.add_argument("--batch-tile", type=int, default=None,
                    help="batch deep-kernel tile shape (nlse_batch_set_tile 0..3; default: the autotuner's pick)")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--sur-traj", type=int, default=160, help="surrogate training trajectories (125 windows each)")
    ap.add_argument("--sur-epochs", type=int, default=60)
    ap.add_argument("--surrogate-kernels-only", action="store_true",
                    help="print only the surrogate's kernel throughput (training and inference steps) and exit")
    ap.add_argument("--no-paper-tables", action="store_true", help="skip the timing runs of the paper's Tables 1-3")
    ap.add_argument("--chunk-study", action="store_true", help="also time 1000 steps in chunks of 1..1000")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--repeats", type=int, default=5, help="timed repeats of K steps (the first is the value)")
    ap.add_argument("--no-rings", dest="rings", action="store_false",
                    help="skip the 512^3 precision-form leg")
    ap.add_argument("--sur-mass-weight", type=float, default=0.0,
                    help="weight of the mass-conservation term of the surrogate's training loss")
    ap.add_argument("--ref-budget", type=float, default=90.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.surrogate_kernels_only:
        import torch
        dev = torch.device("cuda", local_rank)
        torch.cuda.set_device(dev)
        res = {"surrogate_kernels": surrogate_form(args, dev)} if rank == 0 else None
    elif args.impl == "reference":
        res = run_reference(args, rank, world)
    else:
        res = run_ours(args, rank, world, local_rank)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
