"""nlse_mass_noalloc: the mass for callers that cannot allocate device memory.

Some callers may not call cudaMalloc (work issued while another component
captures the stream into a CUDA graph, plug-ins whose host application owns
all device memory, real-time loops that cannot take an allocation's
synchronisation).  nlse_mass_noalloc serves them with scratch kept inside
the library.  These tests call it through the C ABI and compare it with the
context entry point nlse_mass on the same data, twice in a row, with the
tolerance the other mass tests use (1e-13 relative).  This file is collected
last so that a run stopping at the first failure has run everything else.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1203_1263_gb300 import _lib as L
from paper_1203_1263_gb300 import workloads as W
from paper_1203_1263_gb300.integrator import Integrator

pytestmark = pytest.mark.gpu

DTYPES = {"c128": L.C128, "c64": L.C64, "c64_acc64": L.C64_ACC64}


def noalloc_mass(psi: torch.Tensor, h: float, dtype: str) -> float:
    lib = L.lib()
    out = torch.full((1,), float("nan"), dtype=torch.float64, device=psi.device)
    n = L.int64_array(psi.shape)
    stream = torch.cuda.current_stream(psi.device).cuda_stream
    L.check(lib.nlse_mass_noalloc(psi.dim(), n, float(h), DTYPES[dtype], psi.data_ptr(), out.data_ptr(), stream))
    torch.cuda.synchronize(psi.device)
    return float(out.item())


@pytest.mark.parametrize("dtype", ["c128", "c64", "c64_acc64"])
def test_noalloc_mass_matches_context_mass_on_consecutive_calls(dtype):
    h = 0.25
    fields = [W.random_field((33, 41, 70), seed=61), W.random_field((300, 257), seed=62)]
    refs, tensors = [], []
    for psi in fields:
        g = Integrator(psi, h, 0.7, -1.0, None, "dirichlet", 4, dtype)
        refs.append(g.mass())
        tensors.append(g.psi)
    # two calls in a row on different grids, then the first again: the shared
    # scratch keeps the previous call's contents and must not leak into the next
    for k in (0, 1, 0):
        got = noalloc_mass(tensors[k], h, dtype)
        assert abs(got - refs[k]) <= 1e-13 * abs(refs[k]), (k, got, refs[k])


def test_noalloc_rejects_grids_beyond_its_scratch():
    lib = L.lib()
    dev = torch.zeros(2, dtype=torch.float64, device="cuda")
    n = L.int64_array([512, 512, 129])   # 33,816,576 sites > 8192 blocks of 4096
    rc = lib.nlse_mass_noalloc(3, n, 0.1, L.C128, dev.data_ptr(), dev.data_ptr(), None)
    assert rc == L.NLSE_EINVAL
    assert b"maximum" in lib.nlse_last_error()
