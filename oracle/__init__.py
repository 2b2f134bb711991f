"""Plain FP64 CPU oracle for the NLSE RK4 integrator (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``nlse_oracle.c`` (compiled with gcc,
``-O2 -ffp-contract=off``) through ctypes and shares nothing with the CUDA
library.  Every function takes complex128 numpy arrays in C order and
returns new arrays; nothing is modified in place.

Parity status of each function (pins are in tests/test_oracle_pins.py):
  evalF, laplacian, rk4      pinned (closed forms, exact solitons, brute force;
                             the L0 boundary by its pointwise boundary ODE and
                             multilinear fields in a constant potential; the
                             periodic grid by the discrete Fourier spectrum of
                             both Laplacians, Fourier modes under RK4, plane
                             waves of the cubic equation and shift invariance)
  mass                       pinned (closed form, exact-sum comparison)
  energy                     pinned (conservation, closed form for sine modes)
  stability_bound            pinned (numbers printed in Sec. 4 and Sec. 3.4)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nlse_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_nlse.so")
_lock = threading.Lock()
_lib = None

BC_DIRICHLET = 0
BC_MSD = 1
BC_L0 = 2
BC_PERIODIC = 3


def build(force: bool = False) -> str:
    """Compile nlse_oracle.c into oracle/_build/liboracle_nlse.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c99", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)   # no OpenMP: serial build
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            I64P = ctypes.POINTER(ctypes.c_int64)
            DP = ctypes.c_void_p
            d_ = ctypes.c_double
            i_ = ctypes.c_int
            lib.oracle_evalF.argtypes = [i_, I64P, d_, d_, d_, DP, i_, i_, DP, DP]
            lib.oracle_laplacian.argtypes = [i_, I64P, d_, d_, d_, DP, i_, i_, DP, DP, DP]
            lib.oracle_rk4.argtypes = [i_, I64P, d_, d_, d_, DP, i_, i_, d_, ctypes.c_int64, DP]
            lib.oracle_mass.argtypes = [i_, I64P, d_, DP, ctypes.POINTER(d_)]
            lib.oracle_energy.argtypes = [i_, I64P, d_, d_, d_, DP, i_, i_, DP, ctypes.POINTER(d_)]
            lib.oracle_stability_bound.argtypes = [i_, d_, d_, i_, d_, d_]
            lib.oracle_stability_bound.restype = d_
            lib.oracle_set_threads.argtypes = [i_]
            for f in (lib.oracle_evalF, lib.oracle_laplacian, lib.oracle_rk4, lib.oracle_mass,
                      lib.oracle_energy, lib.oracle_set_threads):
                f.restype = i_
            _lib = lib
    return _lib


def _shape(psi):
    n = (ctypes.c_int64 * 3)(*(list(psi.shape) + [1] * (3 - psi.ndim)))
    return psi.ndim, n


def _c128(x):
    return np.ascontiguousarray(x, dtype=np.complex128)


def _vptr(V, shape):
    if V is None:
        return None, None
    V = np.ascontiguousarray(V, dtype=np.float64)
    assert V.shape == tuple(shape)
    return V, V.ctypes.data


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 = leave as is); returns the count in use."""
    return int(_load().oracle_set_threads(int(n)))


def evalF(psi, h, a, s, V=None, bc=BC_DIRICHLET, order=4):
    """F(Psi) = i[a Lap Psi + (s|Psi|^2 - V) Psi] with the boundary forms of Sec. 3.3."""
    lib = _load()
    psi = _c128(psi)
    d, n = _shape(psi)
    Vk, vp = _vptr(V, psi.shape)
    F = np.zeros_like(psi)
    _check(lib.oracle_evalF(d, n, h, a, s, vp, bc, order, psi.ctypes.data, F.ctypes.data), "evalF")
    return F


def laplacian(psi, h, a=1.0, s=0.0, V=None, bc=BC_DIRICHLET, order=4):
    """(D, Lap): step-1 D at every site (boundary sites: the BC Laplacian form
    when order == 4, else 0) and Lap at interior sites (0 on the boundary)."""
    lib = _load()
    psi = _c128(psi)
    d, n = _shape(psi)
    Vk, vp = _vptr(V, psi.shape)
    D = np.zeros_like(psi)
    L = np.zeros_like(psi)
    _check(lib.oracle_laplacian(d, n, h, a, s, vp, bc, order, psi.ctypes.data, D.ctypes.data, L.ctypes.data),
           "laplacian")
    return D, L


def rk4(psi, h, a, s, dt, nsteps, V=None, bc=BC_DIRICHLET, order=4):
    """Psi after nsteps RK4 steps (Eq. RK4, steps 1-10)."""
    lib = _load()
    out = _c128(psi).copy()
    d, n = _shape(out)
    Vk, vp = _vptr(V, out.shape)
    _check(lib.oracle_rk4(d, n, h, a, s, vp, bc, order, dt, int(nsteps), out.ctypes.data), "rk4")
    return out


def mass(psi, h):
    """h^d sum |Psi|^2 over all sites."""
    lib = _load()
    psi = _c128(psi)
    d, n = _shape(psi)
    out = ctypes.c_double()
    _check(lib.oracle_mass(d, n, h, psi.ctypes.data, ctypes.byref(out)), "mass")
    return out.value


def energy(psi, h, a, s, V=None, bc=BC_DIRICHLET, order=4):
    """h^d sum_interior [-a Re(conj Psi Lap Psi) + V|Psi|^2 - (s/2)|Psi|^4]."""
    lib = _load()
    psi = _c128(psi)
    d, n = _shape(psi)
    Vk, vp = _vptr(V, psi.shape)
    out = ctypes.c_double()
    _check(lib.oracle_energy(d, n, h, a, s, vp, bc, order, psi.ctypes.data, ctypes.byref(out)), "energy")
    return out.value


def stability_bound(d, h, a, order, vmax=0.0, s_rho_max=0.0):
    """RK4 linear stability bound on dt (no safety factor), Sec. 3.4."""
    return float(_load().oracle_stability_bound(int(d), float(h), float(a), int(order), float(vmax),
                                                float(s_rho_max)))


def run_problem(problem, nsteps=None, dt=None):
    """Integrate a workloads.Problem; dt defaults to the problem's dt, else
    0.8 x the stability bound with the potential and |s| max|Psi0|^2 terms."""
    if dt is None:
        dt = problem.dt if problem.dt is not None else 0.8 * stability_bound(
            problem.dims, problem.h, problem.a, problem.order, problem.vmax(),
            abs(problem.s) * float(np.max(np.abs(problem.psi0)) ** 2))
    if nsteps is None:
        nsteps = problem.steps
    return rk4(problem.psi0, problem.h, problem.a, problem.s, dt, nsteps, problem.V, problem.bc, problem.order), dt
