"""Python front end of the CUDA integrator.

`Integrator` owns the device memory (torch tensors: Psi, V and the library's
workspace) and hands raw pointers and the CUDA stream to libnlse.  Every step
of the method runs in the library's kernels.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np
import torch

from . import _lib as L

_DTYPES = {"c128": L.C128, "c64": L.C64, "c64_acc64": L.C64_ACC64}
_BCS = {"dirichlet": L.BC_DIRICHLET, "msd": L.BC_MSD, "l0": L.BC_L0, "periodic": L.BC_PERIODIC}


def _code(table, v):
    return table[v] if isinstance(v, str) else int(v)


def max_dt(dims, h, a, order, vmax=0.0, s_rho_max=0.0) -> float:
    """RK4 linear stability bound (no safety factor)."""
    v = L.lib().nlse_max_dt(int(dims), float(h), float(a), int(order), float(vmax), float(s_rho_max))
    if v < 0:
        raise ValueError("invalid arguments to max_dt")
    return v


def workspace_bytes(shape, dtype="c128") -> int:
    n = L.int64_array(shape)
    return int(L.lib().nlse_workspace_bytes(len(shape), n, _code(_DTYPES, dtype)))


class Integrator:
    """RK4 integrator of i Psi_t + a Lap Psi - V Psi + s|Psi|^2 Psi = 0 on one GPU.

    psi0   complex array (numpy or torch), shape (N0[, N1[, N2]]), C order
    h, a, s, V (real array or None), bc ('dirichlet' | 'msd' | 'l0'), order (2 | 4)
    dtype  'c128' (FP64), 'c64' (FP32), 'c64_acc64' (FP32 stages, FP64 master and accumulator)
    """

    def __init__(self, psi0, h, a, s, V=None, bc="dirichlet", order=4, dtype="c128",
                 device: Optional[torch.device] = None, stream: Optional[torch.cuda.Stream] = None):
        self.lib = L.lib()
        self.device = torch.device(device if device is not None else "cuda", 0) if not isinstance(device, torch.device) \
            else device
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.dtype_code = _code(_DTYPES, dtype)
        self.bc = _code(_BCS, bc)
        self.order = int(order)
        self.h, self.a, self.s = float(h), float(a), float(s)
        cdt = torch.complex64 if self.dtype_code == L.C64 else torch.complex128
        vdt = torch.float64 if self.dtype_code == L.C128 else torch.float32
        self.psi = self._to_device(psi0, cdt)
        self.shape = tuple(self.psi.shape)
        self.dims = len(self.shape)
        self.V = None if V is None else self._to_device(V, vdt)
        if self.V is not None and tuple(self.V.shape) != self.shape:
            raise ValueError("V must have Psi's shape")
        n = L.int64_array(self.shape)
        nbytes = int(self.lib.nlse_workspace_bytes(self.dims, n, self.dtype_code))
        if nbytes == 0:
            raise ValueError(f"unsupported shape/dtype {self.shape} {dtype}")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        ctx = ctypes.c_void_p()
        L.check(self.lib.nlse_create(ctypes.byref(ctx), self.dims, n, self.h, self.a, self.s,
                                     None if self.V is None else self.V.data_ptr(), self.bc, self.order,
                                     self.dtype_code, self.psi.data_ptr(), self.workspace.data_ptr(), nbytes,
                                     self.stream.cuda_stream))
        self.ctx = ctx

    def _to_device(self, x, dt):
        if isinstance(x, np.ndarray):
            x = torch.from_numpy(np.ascontiguousarray(x))
        return x.to(device=self.device, dtype=dt).contiguous().clone()

    # ---- the C ABI, one call each ----
    def step(self, nsteps: int, dt: float) -> None:
        L.check(self.lib.nlse_step(self.ctx, int(nsteps), float(dt)))

    def refresh_potential(self) -> None:
        """Re-read self.V after writing new values into it (nlse_refresh_potential)."""
        L.check(self.lib.nlse_refresh_potential(self.ctx))

    def mass(self) -> float:
        out = ctypes.c_double()
        L.check(self.lib.nlse_mass(self.ctx, ctypes.byref(out)))
        return out.value

    def energy(self) -> float:
        out = ctypes.c_double()
        L.check(self.lib.nlse_energy(self.ctx, ctypes.byref(out)))
        return out.value

    def rhs(self, psi_in=None) -> torch.Tensor:
        """F(Psi) at every site (stage-precision complex tensor)."""
        sdt = torch.complex128 if self.dtype_code == L.C128 else torch.complex64
        x = self.psi.to(sdt) if psi_in is None else self._to_device(psi_in, sdt)
        out = torch.empty_like(x)
        L.check(self.lib.nlse_rhs(self.ctx, x.data_ptr(), out.data_ptr()))
        return out

    def sync(self) -> None:
        L.check(self.lib.nlse_sync(self.ctx))

    def set_kernel(self, variant: int, tile_cfg: int = -1) -> None:
        L.check(self.lib.nlse_set_kernel(self.ctx, int(variant), int(tile_cfg)))

    def kernel_in_use(self) -> int:
        """The stage kernel variant the graph-replayed steps run with (nlse_kernel_in_use)."""
        v = int(self.lib.nlse_kernel_in_use(self.ctx))
        L.check(min(v, 0))
        return v

    def autotune(self):
        """Pick the fastest tile shape for this problem (see nlse_autotune); returns (tile_cfg, ms)."""
        cfg = ctypes.c_int()
        ms = ctypes.c_float()
        L.check(self.lib.nlse_autotune(self.ctx, ctypes.byref(cfg), ctypes.byref(ms)))
        return cfg.value, ms.value

    def debug_set(self, key: int, value: int) -> None:
        """Test hook for the bounded device-side waits (see nlse_debug_set)."""
        L.check(self.lib.nlse_debug_set(self.ctx, int(key), int(value)))

    def max_dt(self, s_rho_max: float = 0.0, vmax: Optional[float] = None) -> float:
        if vmax is None:
            vmax = 0.0 if self.V is None else float(self.V.abs().max())
        return max_dt(self.dims, self.h, self.a, self.order, vmax, s_rho_max)

    def numpy(self) -> np.ndarray:
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return self.psi.detach().cpu().numpy()

    def close(self) -> None:
        if getattr(self, "ctx", None):
            self.lib.nlse_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchIntegrator:
    """Many independent 2D runs (complex64) advanced together (nlse_batch_*).

    runs: sequence of dicts with psi0 (complex array (Ny, Nx)), h, a, s, dt,
    V (real array or None), bc ('dirichlet' | 'msd' | 'l0'), order (2 | 4)."""

    def __init__(self, runs, device=None, stream=None):
        self.lib = L.lib()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.psi = []
        self.V = []
        descs = (L.RunDesc * len(runs))()
        for i, r in enumerate(runs):
            p = torch.from_numpy(np.array(r["psi0"], dtype=np.complex64)).to(self.device).contiguous()
            v = None if r.get("V") is None else \
                torch.from_numpy(np.array(r["V"], dtype=np.float32)).to(self.device).contiguous()
            self.psi.append(p)
            self.V.append(v)
            d = descs[i]
            d.n[0], d.n[1] = p.shape
            d.h, d.a, d.s, d.dt = float(r["h"]), float(r["a"]), float(r["s"]), float(r["dt"])
            d.bc = _code(_BCS, r.get("bc", "dirichlet"))
            d.order = int(r.get("order", 4))
            d.psi = p.data_ptr()
            d.V = None if v is None else v.data_ptr()
        self._descs = descs
        nbytes = int(self.lib.nlse_batch_workspace_bytes(len(runs), ctypes.byref(descs)))
        if nbytes == 0:   # invalid descriptors: let create report the reason
            b = ctypes.c_void_p()
            L.check(self.lib.nlse_batch_create(ctypes.byref(b), len(runs), ctypes.byref(descs), None, 0, None))
            raise L.NLSEError(L.NLSE_EINVAL, "invalid batch")
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        b = ctypes.c_void_p()
        L.check(self.lib.nlse_batch_create(ctypes.byref(b), len(runs), ctypes.byref(descs),
                                           self.workspace.data_ptr(), nbytes, self.stream.cuda_stream))
        self.b = b

    def step(self, nsteps: int) -> None:
        L.check(self.lib.nlse_batch_step(self.b, int(nsteps)))

    def sync(self) -> None:
        L.check(self.lib.nlse_batch_sync(self.b))

    def set_tile(self, tile_cfg: int) -> None:
        L.check(self.lib.nlse_batch_set_tile(self.b, int(tile_cfg)))

    def autotune(self):
        cfg = ctypes.c_int()
        ms = ctypes.c_float()
        L.check(self.lib.nlse_batch_autotune(self.b, ctypes.byref(cfg), ctypes.byref(ms)))
        return cfg.value, ms.value

    def numpy(self, i: int) -> np.ndarray:
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return self.psi[i].cpu().numpy()

    def close(self) -> None:
        if getattr(self, "b", None):
            self.lib.nlse_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
