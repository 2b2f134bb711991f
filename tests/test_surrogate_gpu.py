"""The surrogate's tensor-core kernels against the FP64 CPU reference, its
training, its RK4 fallback, and what it gains over plain RK4."""
import math

import numpy as np
import pytest
import torch

from oracle import surrogate_ref as S
from paper_1203_1263_gb300 import _lib as L_
from paper_1203_1263_gb300 import workloads as W
from paper_1203_1263_gb300.surrogate import FOCUSING, Surrogate, generate_pairs, rollout, train

pytestmark = pytest.mark.gpu


def bf16_round(a):
    return torch.as_tensor(a).to(torch.bfloat16).to(torch.float64).numpy()


def small_net(C=16, L=4, dil=(1, 2, 3, 1), H=24, Wd=28, nb=2, seed=11):
    sur = Surrogate(H, Wd, channels=C, layers=L, dilations=dil, max_batch=nb, seed=seed)
    z = W.random_field((nb, H, Wd), seed + 1)
    psi = bf16_round(z.real) + 1j * bf16_round(z.imag)      # inputs exactly representable in BF16
    target = psi * np.exp(0.3j) + 0.05
    return sur, psi, target, C, L, dil


# (shape, kernel choice): C = 16 / 32 with the tcgen05 kernel (tc=1) on the inner
# forward and backward-data convolutions and the cp.async/ldmatrix mma.sync
# kernels elsewhere, or mma.sync everywhere (tc=0); C = 12: the generic kernel.
SHAPES = [(dict(C=16, L=4, dil=(1, 2, 3, 1)), 1), (dict(C=16, L=4, dil=(1, 2, 3, 1)), 0),
          (dict(C=32, L=4, dil=(1, 8, 5, 1), H=20, Wd=150, nb=3), 1), (dict(C=12, L=3, dil=(2, 1, 1)), 1),
          (dict(C=64, L=4, dil=(1, 3, 16, 1), H=18, Wd=140, nb=2), 1),
          (dict(C=64, L=4, dil=(1, 3, 16, 1), H=18, Wd=140, nb=2), 0)]
IDS = ["tc-16", "mma-16", "tc-32-wide", "generic-12", "tc-64-tma", "mma-64"]


def make(shape, tc):
    sur, psi, target, C, L, dil = small_net(**shape)
    sur.set_kernel(tc)
    return sur, psi, target, C, L, dil


@pytest.mark.parametrize("shape,tc", SHAPES, ids=IDS)
def test_forward_matches_reference(shape, tc):
    sur, psi, target, C, L, dil = make(shape, tc)
    params = bf16_round(sur.params.cpu().numpy())
    ref, _, _ = S.forward(params, psi, C, L, dil)
    x = torch.as_tensor(psi, dtype=torch.complex64).cuda()
    out = sur.forward(x).cpu().numpy()
    dy_ref, dy = ref - psi, out - psi
    assert np.linalg.norm(dy - dy_ref) <= 2e-2 * np.linalg.norm(dy_ref)
    # mass projection: each state carries its input's mass; the masses reported are the input's and
    # the raw output's (before the projection)
    masses = torch.zeros((x.shape[0], 2), dtype=torch.float64, device=x.device)
    outp = sur.forward(x, project=True, masses=masses).cpu().numpy().astype(np.complex128)
    refp = S.project_mass(psi, out.astype(np.complex128))
    assert np.max(np.abs(outp - refp)) <= 1e-6 * np.max(np.abs(refp))
    m_in = np.sum(np.abs(psi) ** 2, axis=(1, 2))
    m_out = np.sum(np.abs(outp) ** 2, axis=(1, 2))
    assert np.all(np.abs(m_out - m_in) <= 1e-6 * m_in)
    m = masses.cpu().numpy()
    assert np.allclose(m[:, 0], m_in, rtol=1e-12)
    assert np.allclose(m[:, 1], np.sum(np.abs(out.astype(np.complex128)) ** 2, axis=(1, 2)), rtol=1e-12)


def test_forward_rejects_bad_batches():
    sur, psi, target, C, L, dil = small_net()
    x = torch.as_tensor(psi, dtype=torch.complex64).cuda()
    with pytest.raises(L_.NLSEError) as e:
        L_.check(sur.lib.nlse_sur_forward(sur.s, sur.max_batch + 1, x.data_ptr(), x.data_ptr(), 0, None))
    assert e.value.code == L_.NLSE_EINVAL
    with pytest.raises(ValueError):
        sur.gradients(x, x[:1])
    with pytest.raises(L_.NLSEError):
        sur.set_mass_weight(-1.0)


def test_compare_is_the_relative_l2_per_state():
    sur, psi, target, C, L, dil = small_net(nb=2)
    a = torch.as_tensor(psi, dtype=torch.complex64).cuda()
    b = torch.as_tensor(target, dtype=torch.complex64).cuda()
    got = sur.compare(a, b)
    an, bn = a.cpu().numpy().astype(np.complex128), b.cpu().numpy().astype(np.complex128)
    ref = np.linalg.norm((an - bn).reshape(2, -1), axis=1) / np.linalg.norm(bn.reshape(2, -1), axis=1)
    assert np.allclose(got, ref, rtol=1e-12)


@pytest.mark.parametrize("mass_weight", [0.0, 0.5])
@pytest.mark.parametrize("shape,tc", SHAPES, ids=IDS)
def test_gradients_match_reference(shape, tc, mass_weight):
    """BF16 operands, FP32 accumulation: the gradient vector within 3 % (relative L2),
    with and without the loss's mass term."""
    sur, psi, target, C, L, dil = make(shape, tc)
    sur.set_mass_weight(mass_weight)
    params = bf16_round(sur.params.cpu().numpy())
    loss_ref, g_ref = S.loss_and_grad(params, psi, target, C, L, dil, mass_weight)
    x = torch.as_tensor(psi, dtype=torch.complex64).cuda()
    t = torch.as_tensor(target, dtype=torch.complex64).cuda()
    g, loss = sur.gradients(x, t)
    g = g.cpu().numpy().astype(np.float64)
    sur.sync()
    assert abs(loss - loss_ref) <= 2e-2 * loss_ref
    assert np.linalg.norm(g - g_ref) <= 3e-2 * np.linalg.norm(g_ref)
    # every layer's weight block individually
    off = 0
    for co, ci in S.layer_shapes(C, L):
        n = co * 9 * ci
        blk, ref = g[off:off + n], g_ref[off:off + n]
        assert np.linalg.norm(blk - ref) <= 5e-2 * np.linalg.norm(ref)
        off += n + co


def test_training_reduces_the_loss():
    sur, psi, target, C, L, dil = small_net(nb=4, seed=21)
    x = torch.as_tensor(psi, dtype=torch.complex64).cuda()
    t = torch.as_tensor(target, dtype=torch.complex64).cuda()
    first = sur.train_step(x, t, 3e-3)
    for _ in range(300):
        last = sur.train_step(x, t, 3e-3, want_loss=False)
    last = sur.train_step(x, t, 3e-3)
    assert last < 0.1 * first, (first, last)


def test_noisy_training_is_seeded_and_learns():
    """Input noise drawn in the kernel: the same seed gives the same run, and
    training with it still lowers the loss."""
    runs = []
    for _ in range(2):
        sur, psi, target, C, L, dil = small_net(C=64, L=4, dil=(1, 2, 2, 1), H=16, Wd=130, nb=2, seed=31)
        x = torch.as_tensor(psi, dtype=torch.complex64).cuda()
        t = torch.as_tensor(target, dtype=torch.complex64).cuda()
        first = sur.train_step(x, t, 1e-3, noise=3e-3)
        for _ in range(60):
            sur.train_step(x, t, 1e-3, want_loss=False, noise=3e-3)
        last = sur.train_step(x, t, 1e-3, noise=3e-3)
        sur.sync()
        runs.append((first, last, sur.params.clone()))
    assert runs[1][1] < 0.5 * runs[1][0]
    assert torch.allclose(runs[0][2], runs[1][2], rtol=0, atol=1e-6)
    with pytest.raises(L_.NLSEError):
        sur.train_step(x, t, 1e-3, noise=-1.0)


def test_fallback_takes_over_from_a_bad_network():
    """A network that is far off (large random weights) is rejected on every
    window, with or without the mass projection (the mass is judged on its
    raw output), so the rollout equals plain RK4 (up to the complex64
    hand-over between windows)."""
    n, windows = 48, 6
    psi0 = W.humps_2d(5, 0, n=n, h=FOCUSING["h"])
    sur = Surrogate(n, n, channels=16, layers=4, dilations=(1, 2, 2, 1), max_batch=4, seed=3)
    sur.load_params(sur.params * 40.0)
    ref, _ = rollout(None, psi0, windows)
    for mode, project in (("strict", False), ("sampled", False), ("strict", True), ("parallel", True)):
        got, st = rollout(sur, psi0, windows, mode=mode, every=3, project=project, width=4)
        assert st.accepted == 0 and st.rk4_windows == windows
        assert st.rejected_l2 + st.rejected_mass >= 1
        if mode == "strict":
            assert st.rejected_mass == windows and st.rejected_l2 == 0
        assert float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref)) <= 1e-5


@pytest.mark.parametrize("mode", ["strict", "sampled", "parallel"])
def test_mass_check_fires_with_projection_on(mode):
    """A network whose only output is a constant shift of 1e-3 on the real
    part, on a real Gaussian state (48 x 48, h = 0.2, width 1.5): the shift is
    within the relative-L2 tolerance of RK4 (~4e-3), but its raw output adds
    ~4e-3 of the mass.  With the mass projection on (the default) every window
    must still be rejected for mass, and the rollout equals plain RK4."""
    n, windows = 48, 6
    psi0, _ = W.gaussian_packet_2d(n, FOCUSING["h"], 1.0, 1.5, (0.0, 0.0), (0.0, 0.0), 1.0, 1.0)
    sur = Surrogate(n, n, channels=16, layers=4, dilations=(1, 2, 2, 1), max_batch=4, seed=3)
    p = torch.zeros_like(sur.params)
    p[-2] = 1e-3
    sur.load_params(p)
    ref, _ = rollout(None, psi0, windows)
    got, st = rollout(sur, psi0, windows, mode=mode, every=3, project=True, width=4)
    assert st.accepted == 0 and st.rk4_windows == windows
    assert st.rejected_mass >= 1 and st.rejected_l2 == 0
    assert st.max_mass_drift > 1e-3
    assert float(torch.linalg.vector_norm(got - ref) / torch.linalg.vector_norm(ref)) <= 1e-5


def test_gain_over_plain_rk4():
    """The focusing workload at its size (256 x 256, h = 0.2, windows of 32
    FP64 RK4 steps of dt = 0.005): trained on 80 FP64 trajectories of 125
    windows (30 epochs), the network advances a held-out state by one window
    at least 10x faster than one window of the FP64 integrator (states in
    batches of 16, the parallel rollout's use); and rolled out to t = 20 in
    the parallel mode with every window checked against FP64 RK4 from its own
    start (relative L2 <= 1e-2, mass of the unprojected output within 1e-4
    of the initial mass), every accepted window meets both bounds, the
    rejected ones are replaced by RK4, and the final state is within 2e-2 per
    accepted window of plain FP64 RK4 (a window's 1e-2, allowed to double
    under the dynamics over the rest of the run).  The checked rollout's
    wall-clock ratio to plain FP64 RK4 is printed: it depends on how many
    windows the network's unprojected mass passes (see the benchmark)."""
    n, win = 256, FOCUSING["window"]
    X, Y, kept = generate_pairs(80, 125, n=n, seed=5)
    sur = Surrogate(n, n, channels=64, layers=6, dilations=(1, 2, 4, 8, 4, 1), max_batch=32, seed=7)
    hist = train(sur, X, Y, epochs=30, batch=32, lr=5e-4, lr_end=1e-5, seed=0, noise=3e-3)
    del X, Y
    assert hist[-1] < 0.1 * hist[0]
    Xh, Yh, k = generate_pairs(1, 125, n=n, seed=101)
    assert k == 1
    # inference against one FP64 RK4 window
    from paper_1203_1263_gb300.integrator import Integrator
    g = Integrator(Xh[0].cpu().numpy().astype(np.complex128), FOCUSING["h"], FOCUSING["a"], FOCUSING["s"], None,
                   "dirichlet", 4, "c128")
    g.step(win, FOCUSING["dt"])
    x16 = Xh[:16].contiguous()
    sur.forward(x16)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    for _ in range(5):
        g.step(win, FOCUSING["dt"])
    e[1].record()
    e[2].record()
    for _ in range(5):
        sur.forward(x16)
    e[3].record()
    torch.cuda.synchronize()
    rk4_ms = e[0].elapsed_time(e[1]) / 5
    net_ms = e[2].elapsed_time(e[3]) / 5 / 16
    g.close()
    # the checked rollout
    psi0 = Xh[0].cpu().numpy().astype(np.complex128)
    ref, st_plain = rollout(None, psi0, 125)
    got, st = rollout(sur, psi0, 125, mode="parallel", width=8)
    err = float(sur.compare(got[None], ref[None])[0])
    print(f"\nkept {kept}; loss {hist[0]:.3e} -> {hist[-1]:.3e}; one window: FP64 RK4 {rk4_ms:.3f} ms, network "
          f"{net_ms:.4f} ms ({rk4_ms / net_ms:.1f}x); parallel rollout to t = 20: accepted {st.accepted}/125, "
          f"rejected l2 {st.rejected_l2} mass {st.rejected_mass}, max raw mass drift {st.max_mass_drift:.2e}, "
          f"final rel-L2 vs plain {err:.2e}, wall-clock {st_plain.seconds / st.seconds:.2f}x plain FP64 RK4")
    assert rk4_ms >= 10 * net_ms
    assert st.accepted + st.rk4_windows == 125
    assert st.checked >= st.accepted
    # each accepted window is within 1e-2 of RK4 from its own start; that error may grow under the focusing
    # dynamics over the rest of the run: allowed to double (2e-2 per accepted window); none accepted: RK4 alone
    assert err <= (2e-2 * st.accepted if st.accepted else 1e-5)


def test_concurrent_data_generation_matches_sequential_runs():
    """Trajectories advanced on separate streams equal one-at-a-time FP64 runs bit for bit."""
    from paper_1203_1263_gb300.integrator import Integrator
    n, windows = 40, 3
    X, Y, kept = generate_pairs(3, windows, n=n, seed=8, concurrent=2)
    assert kept == 3 and X.shape == (3 * windows, n, n)
    for k in range(3):
        g = Integrator(W.humps_2d(8, k, n=n, h=FOCUSING["h"]), FOCUSING["h"], FOCUSING["a"], FOCUSING["s"], None,
                       "dirichlet", 4, "c128")
        for w in range(windows):
            assert torch.equal(X[k * windows + w], g.psi.to(torch.complex64))
            g.step(FOCUSING["window"], FOCUSING["dt"])
            assert torch.equal(Y[k * windows + w], g.psi.to(torch.complex64))
        g.close()
