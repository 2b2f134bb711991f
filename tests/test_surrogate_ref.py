"""Pins of the FP64 surrogate reference (CPU): central finite differences of
the loss, and closed-form cases of the network definition."""
import numpy as np

from oracle import surrogate_ref as S
from paper_1203_1263_gb300 import workloads as W


def _problem(C=3, L=3, dil=(1, 2, 1), shape=(2, 6, 7), seed=3):
    n = sum(co * 9 * ci + co for co, ci in S.layer_shapes(C, L))
    params = 0.4 * (2 * W.uniform(seed, n) - 1)
    psi = W.random_field(shape, seed + 1)
    target = W.random_field(shape, seed + 2)
    return params, psi, target, C, L, dil


def test_gradient_matches_finite_differences():
    params, psi, target, C, L, dil = _problem()
    loss, g = S.loss_and_grad(params, psi, target, C, L, dil)
    eps = 1e-6
    rng = np.random.default_rng(0)
    idx = rng.choice(params.size, 60, replace=False)
    for i in idx:
        p1, p2 = params.copy(), params.copy()
        p1[i] += eps
        p2[i] -= eps
        fd = (S.loss_and_grad(p1, psi, target, C, L, dil)[0] - S.loss_and_grad(p2, psi, target, C, L, dil)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_output_bias_only_network_adds_the_bias():
    params, psi, target, C, L, dil = _problem()
    params[:] = 0.0
    params[-2:] = [0.25, -0.5]          # b of the last layer
    out, _, _ = S.forward(params, psi, C, L, dil)
    assert np.allclose(out, psi + 0.25 - 0.5j, atol=0, rtol=1e-15)


def test_tap_convention_is_a_shift():
    """A single non-zero tap t = 5 (offset (0, +1)) reads the right neighbour."""
    x = W.random_field((1, 5, 6), 7)
    h = np.stack([x.real, x.imag], -1)
    Wl = np.zeros((2, 9, 2))
    Wl[0, 5, 0] = 1.0
    Wl[1, 5, 1] = 1.0
    z = S.conv(h, Wl, np.zeros(2), 1)
    assert np.array_equal(z[0, :, :-1, 0], x.real[0, :, 1:])
    assert np.all(z[0, :, -1, :] == 0)
