"""The seeded input generators: shapes and structure of the workloads they
stand in for (no method arithmetic here, so nothing of the oracle)."""
import math

import numpy as np
import pytest

from paper_1203_1263_gb300 import workloads as W


@pytest.mark.parametrize("dims", [1, 2, 3])
def test_paper_timing_sizes_are_the_tables(dims):
    for total in W.PAPER_TABLE_SITES[dims]:
        p = W.paper_timing_problem(dims, total)
        assert p.sites == total and p.dims == dims
        assert p.bc == W.BC_MSD and p.V is None and p.s == -1.0 and p.a == 1.0
        assert p.dt == 0.005 and p.steps == 10000
        assert np.max(np.abs(p.psi0)) <= 1.0 + 1e-12


def test_paper_dark_soliton_is_eq_soliton_at_t0():
    p = W.paper_timing_problem(1, 1000)
    assert abs(p.h - 0.1) < 1e-15
    x = p.extra["x"]
    assert np.allclose(p.psi0, np.tanh(x / math.sqrt(2)) * np.exp(0.25j * x), atol=1e-14)


def _winding(phase_ring):
    d = np.diff(np.concatenate([phase_ring, phase_ring[:1]]))
    return int(round(np.sum((d + np.pi) % (2 * np.pi) - np.pi) / (2 * np.pi)))


def test_paper_vortex_2d_has_unit_charge():
    p = W.paper_timing_problem(2, 10000)
    n = p.shape[0]
    c = n // 2
    r = 20
    ring = np.concatenate([p.psi0[c - r, c - r:c + r], p.psi0[c - r:c + r, c + r],
                           p.psi0[c + r, c + r:c - r:-1], p.psi0[c + r:c - r:-1, c - r]])
    assert _winding(np.angle(ring)) == 1
    assert np.abs(p.psi0[0, 0]) > 0.99          # background density 1 at the walls


def test_paper_vortex_ring_3d_core_circle():
    """The ring's core: |Psi| is smallest near r = 5 in the z = 0 plane, and
    the phase winds once around the core in the x-z half-plane."""
    p = W.paper_timing_problem(3, 970299)
    n = p.shape[0]
    c = n // 2
    ax = W.centred_axis(n, p.h)
    plane = np.abs(p.psi0[c, c, :])              # z = 0, y = 0, along x
    j = int(np.argmin(plane[c:])) + c
    assert abs(ax[j] - 5.0) <= p.h
    jr = int(np.argmin(np.abs(ax - 5.0)))
    r = 3
    loop = np.concatenate([p.psi0[c - r, c, jr - r:jr + r], p.psi0[c - r:c + r, c, jr + r],
                           p.psi0[c + r, c, jr + r:jr - r:-1], p.psi0[c + r:c - r:-1, c, jr - r]])
    assert abs(_winding(np.angle(loop))) == 1


def test_paper_vortex_ring_back_flow_keeps_it_clear_of_the_walls():
    """Reading of Eq. 3dvr1: with the back-flow c the ring's core stays near
    z = 0 (without it the ring drifts about 0.5 per unit time into a wall),
    so the 10,000-step timing run stays finite.  Checked with the oracle over
    t = 5 on the smallest table grid (21^3)."""
    import oracle as O
    p = W.paper_timing_problem(3, 9261, 4)
    n = p.shape[0]
    ax = W.centred_axis(n, p.h)
    z = ax[:, None, None]
    rc = np.sqrt(ax[None, :, None] ** 2 + ax[None, None, :] ** 2)
    mask = (rc > 1.5) & (rc < 8.5) & (np.abs(z) < 12)

    def zbar(psi):
        w = np.clip(1 - np.abs(psi) ** 2, 0, None) * mask
        return float((w * z).sum() / w.sum())

    out = O.rk4(p.psi0, p.h, p.a, p.s, p.dt, 1000, None, p.bc, 4)
    still = O.rk4(p.psi0 * np.exp(-1j * p.extra["c"] * z / 2), p.h, p.a, p.s, p.dt, 1000, None, p.bc, 4)
    assert np.all(np.isfinite(out)) and np.max(np.abs(out)) < 1.5
    assert abs(zbar(out)) < 2.0
    assert abs(zbar(still)) > 2.0 * abs(zbar(out))
