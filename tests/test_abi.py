"""The C ABI library loads and exports every entry point include/*.h declares;
host-only calls (no GPU needed) behave as documented."""
import ctypes
import glob
import os
import re

import pytest

from paper_1203_1263_gb300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(nlse_\w+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported():
    lib = L.lib()
    names = declared_symbols()
    assert "nlse_step" in names and "nlse_create" in names
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(L.SIGNATURES) | {"nlse_t"}


def test_max_dt_matches_printed_bounds():
    lib = L.lib()
    assert abs(lib.nlse_max_dt(1, 0.1, 1.0, 2, 0.0, 0.0) - 0.0070711) < 1e-7
    assert abs(lib.nlse_max_dt(1, 0.1, 1.0, 4, 0.0, 0.0) - 0.0053033) < 1e-7
    assert lib.nlse_max_dt(4, 0.1, 1.0, 4, 0.0, 0.0) < 0
    assert lib.nlse_max_dt(1, 0.1, 1.0, 3, 0.0, 0.0) < 0


def test_workspace_bytes():
    lib = L.lib()
    n = L.int64_array([512, 256, 256])
    sites = 512 * 256 * 256
    assert lib.nlse_workspace_bytes(3, n, L.C128) >= 3 * 16 * sites
    assert lib.nlse_workspace_bytes(3, n, L.C64) >= 3 * 8 * sites
    assert lib.nlse_workspace_bytes(3, n, L.C64_ACC64) >= 4 * 8 * sites
    assert lib.nlse_workspace_bytes(3, L.int64_array([2, 5, 5]), L.C128) == 0
    assert lib.nlse_workspace_bytes(2, L.int64_array([5, 5]), 7) == 0


@pytest.mark.parametrize("args,code", [
    (dict(dims=0), L.NLSE_EINVAL), (dict(N=[2, 5, 5]), L.NLSE_EINVAL), (dict(h=0.0), L.NLSE_EINVAL),
    (dict(a=-1.0), L.NLSE_EINVAL), (dict(order=3), L.NLSE_EINVAL), (dict(bc=5), L.NLSE_EINVAL), (dict(bc=4), L.NLSE_EINVAL),
    (dict(dtype=9), L.NLSE_EINVAL), (dict(psi=None), L.NLSE_EINVAL), (dict(ws=None), L.NLSE_EINVAL),
    (dict(ws_bytes=16), L.NLSE_ENOMEM), (dict(ws=4096 + 8), L.NLSE_EINVAL),
])
def test_create_rejects_bad_arguments_before_touching_the_gpu(args, code):
    lib = L.lib()
    a = dict(dims=3, N=[5, 5, 5], h=0.1, a=1.0, s=1.0, V=None, bc=0, order=4, dtype=0, psi=4096, ws=4096,
             ws_bytes=1 << 30)
    a.update(args)
    ctx = ctypes.c_void_p()
    rc = lib.nlse_create(ctypes.byref(ctx), a["dims"], L.int64_array(a["N"]), a["h"], a["a"], a["s"], a["V"],
                         a["bc"], a["order"], a["dtype"], a["psi"], a["ws"], a["ws_bytes"], None)
    assert rc == code
    assert ctx.value is None
    assert lib.nlse_last_error()


def _run(**kw):
    d = L.RunDesc()
    d.n[0], d.n[1] = kw.get("n", (64, 80))
    d.h, d.a, d.s = kw.get("h", 0.25), kw.get("a", 0.7), kw.get("s", -1.0)
    d.dt, d.bc, d.order = kw.get("dt", 0.005), kw.get("bc", L.BC_MSD), kw.get("order", 4)
    d.psi, d.V = kw.get("psi", 4096), None
    return d


@pytest.mark.parametrize("bc", [L.BC_DIRICHLET, L.BC_MSD, L.BC_L0])
def test_batch_workspace_accepts_every_boundary(bc):
    runs = (L.RunDesc * 2)(_run(bc=bc), _run(n=(33, 17), order=2, bc=bc))
    assert L.lib().nlse_batch_workspace_bytes(2, runs) >= 2 * (64 * 80 + 33 * 17) * 8


@pytest.mark.parametrize("bad", [dict(bc=3), dict(order=3), dict(n=(2, 40)), dict(h=0.0), dict(dt=1.0), dict(psi=4100)])
def test_batch_workspace_rejects_bad_runs(bad):
    runs = (L.RunDesc * 2)(_run(), _run(**bad))
    assert L.lib().nlse_batch_workspace_bytes(2, runs) == 0


@pytest.mark.parametrize("n", [[4, 2 ** 62 + 1], [512, 512, 129], [2 ** 31, 2 ** 31, 2 ** 31]])
def test_noalloc_rejects_oversized_grids_before_touching_the_gpu(n):
    """The site count is checked against the scratch limit before each
    multiplication, so extents whose product overflows int64 are rejected
    too, with the limit in the message."""
    lib = L.lib()
    rc = lib.nlse_mass_noalloc(len(n), L.int64_array(n), 0.1, L.C128, 4096, 4096, None)
    assert rc == L.NLSE_EINVAL
    assert b"maximum of 33554432 sites" in lib.nlse_last_error()
