"""Pins of the FP64 surrogate reference (CPU): central finite differences of
the loss, and closed-form cases of the network definition."""
import numpy as np
import pytest

from oracle import surrogate_ref as S
from paper_1203_1263_gb300 import workloads as W


def _problem(C=3, L=3, dil=(1, 2, 1), shape=(2, 6, 7), seed=3):
    n = sum(co * 9 * ci + co for co, ci in S.layer_shapes(C, L))
    params = 0.4 * (2 * W.uniform(seed, n) - 1)
    psi = W.random_field(shape, seed + 1)
    target = W.random_field(shape, seed + 2)
    return params, psi, target, C, L, dil


@pytest.mark.parametrize("mass_weight", [0.0, 0.7])
def test_gradient_matches_finite_differences(mass_weight):
    params, psi, target, C, L, dil = _problem()
    loss, g = S.loss_and_grad(params, psi, target, C, L, dil, mass_weight)
    eps = 1e-6
    rng = np.random.default_rng(0)
    idx = rng.choice(params.size, 60, replace=False)
    for i in idx:
        p1, p2 = params.copy(), params.copy()
        p1[i] += eps
        p2[i] -= eps
        fd = (S.loss_and_grad(p1, psi, target, C, L, dil, mass_weight)[0] -
              S.loss_and_grad(p2, psi, target, C, L, dil, mass_weight)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_mass_term_closed_form_on_a_bias_only_network():
    """A network whose only non-zero parameter is the output bias b0 (real)
    maps psi to psi + b0 at every site, so with target = psi the MSE is b0^2/2
    and each state's relative mass change is (2 b0 sum Re psi + b0^2 HW) / M."""
    params, psi, _, C, L, dil = _problem()
    params[:] = 0.0
    b0 = 0.125
    params[-2] = b0
    mu = 3.0
    loss, _ = S.loss_and_grad(params, psi, psi, C, L, dil, mu)
    hw = psi.shape[1] * psi.shape[2]
    m = np.sum(np.abs(psi) ** 2, axis=(1, 2))
    delta = (2 * b0 * np.sum(psi.real, axis=(1, 2)) + b0 * b0 * hw) / m
    assert abs(loss - (0.5 * b0 * b0 + mu * np.mean(delta ** 2))) <= 1e-14


def test_project_mass_closed_form():
    """An output that is the input times a complex factor c_b per state is
    brought back to the input's mass: the result is psi_in c_b / |c_b|; a
    state whose output mass is zero is left as it is; projecting twice
    changes nothing."""
    psi = W.random_field((3, 6, 7), 21)
    c = np.array([2.0 - 1.5j, 0.25j, 0.0])
    out = psi * c[:, None, None]
    got = S.project_mass(psi, out)
    for b in range(2):
        assert np.allclose(got[b], psi[b] * c[b] / abs(c[b]), rtol=1e-14, atol=1e-15)
        assert abs(np.sum(np.abs(got[b]) ** 2) / np.sum(np.abs(psi[b]) ** 2) - 1) < 1e-14
    assert np.array_equal(got[2], out[2])
    assert np.allclose(S.project_mass(psi, got), got, rtol=1e-14, atol=1e-15)


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


def test_conv_equals_scipy_correlation_with_a_dilated_kernel():
    """A dilated 3x3 convolution with zero padding is scipy's 2D correlation
    ('same', zero fill) with the taps spread onto a (2d+1)^2 grid."""
    signal = __import__("pytest").importorskip("scipy.signal")
    rng = np.random.default_rng(11)
    nb, H, Wd, ci, co = 2, 9, 11, 3, 2
    x = rng.standard_normal((nb, H, Wd, ci))
    Wl = rng.standard_normal((co, 9, ci))
    bl = rng.standard_normal(co)
    for d in (1, 2, 3):
        z = S.conv(x, Wl, bl, d)
        for o in range(co):
            k = np.zeros((2 * d + 1, 2 * d + 1, ci))
            for t in range(9):
                k[d + d * (t // 3 - 1), d + d * (t % 3 - 1), :] = Wl[o, t, :]
            for n in range(nb):
                ref = bl[o] + sum(signal.correlate2d(x[n, :, :, c], k[:, :, c], mode="same", boundary="fill")
                                  for c in range(ci))
                assert np.allclose(z[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_single_layer_network_is_one_correlation_of_the_features():
    """layers = 1: psi_out = psi + z0 + i z1 with z the dilated correlation of
    the four input features (Re, Im, |psi|^2 Re, |psi|^2 Im) of psi."""
    signal = __import__("pytest").importorskip("scipy.signal")
    shapes = S.layer_shapes(8, 1)
    assert shapes == [(2, S.N_IN)]
    rng = np.random.default_rng(12)
    params = rng.standard_normal(2 * 9 * S.N_IN + 2)
    psi = W.random_field((1, 7, 8), 13)
    out, _, _ = S.forward(params, psi, 8, 1, (2,))
    Wl = params[:2 * 9 * S.N_IN].reshape(2, 9, S.N_IN)
    b = params[-2:]
    r = np.abs(psi[0]) ** 2
    feats = [psi[0].real, psi[0].imag, r * psi[0].real, r * psi[0].imag]
    d = 2
    z = []
    for o in range(2):
        acc = np.full(psi.shape[1:], b[o])
        for c in range(S.N_IN):
            k = np.zeros((2 * d + 1, 2 * d + 1))
            for t in range(9):
                k[d + d * (t // 3 - 1), d + d * (t % 3 - 1)] = Wl[o, t, c]
            acc = acc + signal.correlate2d(feats[c], k, mode="same", boundary="fill")
        z.append(acc)
    assert np.allclose(out[0], psi[0] + z[0] + 1j * z[1], rtol=1e-12, atol=1e-12)
