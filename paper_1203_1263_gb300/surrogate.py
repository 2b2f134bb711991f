"""Learned surrogate for the 2D NLSE: one network call advances a state by a
window of RK4 steps, re-checked against the plain RK4 path.

Everything numeric runs in libnlse's kernels: the network's forward and
backward passes and the Adam update (nlse_sur_*), the training data (the
FP64 integrator), the masses and relative L2 distances the checks judge by
(nlse_sur_forward's raw-output masses, nlse_sur_compare, nlse_mass_noalloc)
and the RK4 fallback.  This module only orchestrates.
"""
from __future__ import annotations

import ctypes
import math
import time
from dataclasses import dataclass, field
from typing import Optional

import numpy as np
import torch

from . import _lib as L
from . import workloads as W
from .integrator import Integrator, max_dt


class Surrogate:
    """Residual 3x3-convolution network on (Re, Im) of an H x W state."""

    def __init__(self, H: int, W_: int, channels: int = 64, layers: int = 6, dilations=(1, 2, 4, 8, 2, 1),
                 max_batch: int = 16, device=None, stream=None, seed: int = 5):
        self.lib = L.lib()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.H, self.W, self.C, self.L = H, W_, channels, layers
        assert len(dilations) == layers
        self.dilations = (ctypes.c_int * layers)(*dilations)
        self.max_batch = max_batch
        n = int(self.lib.nlse_sur_param_count(channels, layers))
        if n == 0:
            raise ValueError("bad surrogate shape")
        self.params = torch.zeros(n, dtype=torch.float32, device=self.device)
        nb = int(self.lib.nlse_sur_workspace_bytes(H, W_, channels, layers, max_batch))
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        s = ctypes.c_void_p()
        L.check(self.lib.nlse_sur_create(ctypes.byref(s), H, W_, channels, layers, self.dilations, max_batch,
                                         self.params.data_ptr(), self.workspace.data_ptr(), nb,
                                         self.stream.cuda_stream))
        self.s = s
        L.check(self.lib.nlse_sur_init(self.s, int(seed)))

    @property
    def nparams(self) -> int:
        return self.params.numel()

    def _layer_flops(self):
        out = []
        for l in range(self.L):
            ci = 4 if l == 0 else self.C
            co = 2 if l == self.L - 1 else self.C
            out.append(2.0 * self.H * self.W * 9 * ci * co)
        return out

    def flops_per_state(self) -> float:
        """Multiply-adds x 2 of one forward pass on one state."""
        return float(sum(self._layer_flops()))

    def train_flops_per_state(self) -> float:
        """Forward + weight-gradient of every layer + backward-data of layers 1.. (x 2 flops per multiply-add)."""
        f = self._layer_flops()
        return float(3 * sum(f) - f[0])

    def load_params(self, values) -> None:
        self.params.copy_(torch.as_tensor(values, dtype=torch.float32))
        L.check(self.lib.nlse_sur_sync_params(self.s))

    def forward(self, psi: torch.Tensor, project: bool = False, out: Optional[torch.Tensor] = None,
                masses: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Network output for [nb, H, W] states; project=True rescales each
        output to its input's mass.  masses: optional float64 device tensor
        [nb, 2] that receives each state's sum |psi_in|^2 and the sum |.|^2 of
        the network's raw output (before any projection)."""
        psi = psi.to(self.device, torch.complex64).contiguous()
        if out is None:
            out = torch.empty_like(psi)
        if masses is not None and (masses.dtype != torch.float64 or tuple(masses.shape) != (psi.shape[0], 2)):
            raise ValueError("masses must be a float64 tensor [nb, 2]")
        for i in range(0, psi.shape[0], self.max_batch):
            j = min(i + self.max_batch, psi.shape[0])
            L.check(self.lib.nlse_sur_forward(self.s, j - i, psi[i:j].data_ptr(), out[i:j].data_ptr(), int(project),
                                              None if masses is None else masses[i:j].data_ptr()))
        return out

    def set_mass_weight(self, mass_weight: float) -> None:
        """Weight of the mass-conservation term of the training loss (nlse_sur_set_mass_weight)."""
        L.check(self.lib.nlse_sur_set_mass_weight(self.s, float(mass_weight)))

    def compare(self, a: torch.Tensor, b: torch.Tensor) -> np.ndarray:
        """Per-state relative L2 distance ||a - b|| / ||b|| of [nb, H, W] complex64 states (nlse_sur_compare)."""
        a = a.to(self.device, torch.complex64).contiguous()
        b = b.to(self.device, torch.complex64).contiguous()
        if a.shape != b.shape:
            raise ValueError("a and b must have the same shape")
        out = np.zeros(a.shape[0], dtype=np.float64)
        for i in range(0, a.shape[0], self.max_batch):
            j = min(i + self.max_batch, a.shape[0])
            buf = (ctypes.c_double * (j - i))()
            L.check(self.lib.nlse_sur_compare(self.s, j - i, a[i:j].data_ptr(), b[i:j].data_ptr(), buf))
            out[i:j] = np.frombuffer(buf, dtype=np.float64)
        return out

    def _pair(self, psi: torch.Tensor, target: torch.Tensor):
        psi = psi.to(self.device, torch.complex64).contiguous()
        target = target.to(self.device, torch.complex64).contiguous()
        if psi.shape != target.shape or tuple(psi.shape[1:]) != (self.H, self.W):
            raise ValueError("psi and target must both be [nb, H, W]")
        return psi, target

    def gradients(self, psi: torch.Tensor, target: torch.Tensor):
        """Gradient of the mean squared error w.r.t. the parameters, and the loss."""
        psi, target = self._pair(psi, target)
        grad = torch.empty_like(self.params)
        loss = ctypes.c_double()
        L.check(self.lib.nlse_sur_gradients(self.s, psi.shape[0], psi.data_ptr(), target.data_ptr(),
                                             grad.data_ptr(), ctypes.byref(loss)))
        return grad, loss.value

    def train_step(self, psi: torch.Tensor, target: torch.Tensor, lr: float, want_loss: bool = True,
                   noise: float = 0.0):
        """One Adam step on the batch (psi, target); returns the loss before the
        step.  noise: relative input noise (see nlse_sur_train_step)."""
        psi, target = self._pair(psi, target)
        loss = ctypes.c_double()
        L.check(self.lib.nlse_sur_train_step(self.s, psi.shape[0], psi.data_ptr(), target.data_ptr(), float(lr),
                                             float(noise), ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def set_kernel(self, tensor_core_gen: int) -> None:
        """1: tcgen05 kernel for eligible forward / backward-data convolutions; 0: mma.sync only."""
        L.check(self.lib.nlse_sur_set_kernel(self.s, int(tensor_core_gen)))

    def sync(self) -> None:
        L.check(self.lib.nlse_sur_sync(self.s))

    def close(self):
        if getattr(self, "s", None):
            self.lib.nlse_sur_destroy(self.s)
            self.s = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# training data from the FP64 integrator
# ---------------------------------------------------------------------------
FOCUSING = dict(a=1.0, s=1.0, h=0.2, dt=0.005, window=32)


class RK4Pool:
    """`width` FP64 integrators of one n x n focusing problem, each on its own
    CUDA stream, so that independent windows of RK4 run concurrently."""

    def __init__(self, n: int, width: int, params=FOCUSING, device=None):
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.params = params
        zero = np.zeros((n, n), dtype=np.complex128)
        self.streams = [torch.cuda.Stream(self.device) for _ in range(width)]
        self.gs = [Integrator(zero, params["h"], params["a"], params["s"], None, "dirichlet", 4, "c128",
                              device=self.device, stream=st) for st in self.streams]

    def advance(self, starts, windows: int = 1):
        """RK4 from each state in `starts` (complex64 [n, n] tensors, at most
        `width`) by `windows` windows, concurrently; returns the complex64
        results, ordered after the current stream."""
        cur = torch.cuda.current_stream(self.device)
        outs = []
        for g, st, x in zip(self.gs, self.streams, starts):
            st.wait_stream(cur)
            with torch.cuda.stream(st):
                g.psi.copy_(x)
                g.step(self.params["window"] * windows, self.params["dt"])
                outs.append(g.psi.to(torch.complex64))
        for st in self.streams[:len(starts)]:
            cur.wait_stream(st)
        for o, st in zip(outs, self.streams):
            o.record_stream(cur)
        return outs

    def close(self):
        for g in self.gs:
            g.close()


def generate_pairs(n_traj: int, windows: int, n: int = 256, seed: int = 5, device=None, params=FOCUSING,
                   blowup: float = 10.0, concurrent: int = 16):
    """(psi_t, psi_{t+window}) pairs, complex64 [N, n, n], from FP64 RK4 runs of
    the focusing 2D NLSE with Dirichlet walls, 2SHOC, `concurrent` trajectories
    at a time on separate streams.  Initial states: 1-4 Gaussian humps
    (workloads.humps_2d).  Trajectories whose max|psi| exceeds `blowup` x its
    initial value (collapse) are dropped.  Returns (X, Y, trajectories kept)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    X, Y = [], []
    kept = 0
    width = max(1, min(concurrent, n_traj))
    pool = RK4Pool(n, width, params, dev)
    cur = torch.cuda.current_stream(dev)
    for k0 in range(0, n_traj, width):
        ks = list(range(k0, min(k0 + width, n_traj)))
        psi0 = [W.humps_2d(seed, k, n=n, h=params["h"]) for k in ks]
        snaps = [[] for _ in ks]
        for g, st, p0, sn in zip(pool.gs, pool.streams, psi0, snaps):
            st.wait_stream(cur)
            with torch.cuda.stream(st):      # one FP64 trajectory per stream, snapshots in complex64
                g.psi.copy_(torch.as_tensor(p0, dtype=torch.complex128).to(dev, non_blocking=False))
                sn.append(g.psi.to(torch.complex64))
                for _ in range(windows):
                    g.step(params["window"], params["dt"])
                    sn.append(g.psi.to(torch.complex64))
        torch.cuda.synchronize(dev)
        for p0, sn in zip(psi0, snaps):
            amp0 = float(np.max(np.abs(p0)))
            last = sn[-1]
            if float(last.abs().max()) > blowup * amp0 or not torch.isfinite(torch.view_as_real(last)).all():
                continue
            kept += 1
            X.extend(sn[:-1])
            Y.extend(sn[1:])
    pool.close()
    return torch.stack(X), torch.stack(Y), kept


def train(sur: Surrogate, X: torch.Tensor, Y: torch.Tensor, epochs: int, batch: int, lr: float, seed: int = 0,
          log_every: int = 0, lr_end: Optional[float] = None, noise: float = 0.0, mass_weight: float = 0.0):
    """Adam on shuffled mini-batches; returns the per-epoch mean loss.  With
    lr_end the rate follows a cosine from lr down to lr_end over the run;
    noise is the relative input noise of each step; mass_weight the weight of
    the loss's mass-conservation term."""
    sur.set_mass_weight(mass_weight)
    rng = np.random.default_rng(seed)
    hist = []
    per_epoch = max(1, X.shape[0] // batch)
    total = epochs * per_epoch
    it = 0
    for ep in range(epochs):
        order = torch.from_numpy(rng.permutation(X.shape[0])).to(X.device)
        tot, cnt = 0.0, 0
        for i in range(0, X.shape[0] - batch + 1, batch):
            idx = order[i:i + batch]
            xb, yb = X[idx].contiguous(), Y[idx].contiguous()
            rate = lr if lr_end is None else lr_end + 0.5 * (lr - lr_end) * (1 + math.cos(math.pi * it / total))
            it += 1
            loss = sur.train_step(xb, yb, rate, want_loss=(i // batch) % 8 == 0, noise=noise)
            if loss is not None:
                tot += loss
                cnt += 1
        hist.append(tot / max(cnt, 1))
        if log_every and (ep + 1) % log_every == 0:
            print(f"epoch {ep + 1}: loss {hist[-1]:.4e}")
    return hist


# ---------------------------------------------------------------------------
# rollout with the RK4 re-check and fallback
# ---------------------------------------------------------------------------
@dataclass
class RolloutStats:
    windows: int = 0
    accepted: int = 0          # windows taken from the network
    rk4_windows: int = 0       # windows advanced by RK4 after a rejection (or by plain RK4)
    rejected_l2: int = 0
    rejected_mass: int = 0
    checked: int = 0           # RK4 checks of a predicted window
    seconds: float = 0.0
    l2_errors: list = field(default_factory=list)
    max_mass_drift: float = 0.0   # largest |M(raw prediction) - M0| / M0 seen


def _mass(psi: torch.Tensor, h: float, out: torch.Tensor) -> float:
    """h^2 sum |psi|^2 of one complex64 [n, n] state (nlse_mass_noalloc)."""
    lib = L.lib()
    nn = L.int64_array(psi.shape)
    L.check(lib.nlse_mass_noalloc(2, nn, float(h), L.C64, psi.data_ptr(), out.data_ptr(),
                                  torch.cuda.current_stream(psi.device).cuda_stream))
    return float(out.item())


def rollout(sur: Optional[Surrogate], psi0, n_windows: int, params=FOCUSING, mode: str = "strict", every: int = 4,
            tol_l2: float = 1e-2, tol_mass: float = 1e-4, project: bool = True, device=None, width: int = 16):
    """Advance psi0 by n_windows windows of `window` RK4 steps.

    sur=None: plain FP64 RK4.  With a surrogate the rollout moves in spans of
    one window ("strict") or `every` windows ("sampled").  Within a span each
    window is predicted by the network from the previous prediction, and the
    mass of the network's raw output (before the optional projection) must
    stay within tol_mass of the trajectory's initial mass M0 (the NLSE
    conserves mass; plain RK4 changes it by ~1e-8 over t = 20 on this
    workload), so every window is judged on mass, against the start of the
    trajectory rather than the window, and the projection never hides a
    network that does not conserve it.  The span's last window is then re-run
    with FP64 RK4 from the same starting state and must agree within tol_l2
    (relative L2).  If either check fails the rollout returns to the span's
    verified starting state and advances the whole span with RK4.  With
    project=True an accepted prediction is rescaled to its input's mass.
    States pass between windows as complex64.

    "parallel" checks every window like "strict", but speculatively: the
    network predicts up to `width` windows ahead, an RK4Pool re-runs all of
    them at once (window j from predicted state j - 1, each on its own
    stream), the longest prefix that passes both checks is accepted, and at
    the first failing window the RK4 result from its (accepted) starting
    state takes over.  The depth adapts: twice the last round's progress
    after a failure, doubled after a clean round, between 2 and `width`."""
    if mode not in ("strict", "sampled", "parallel"):
        raise ValueError("mode must be 'strict', 'sampled' or 'parallel'")
    if mode == "parallel":
        return _rollout_parallel(sur, psi0, n_windows, params, width, tol_l2, tol_mass, project, device)
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    h, dt, steps = params["h"], params["dt"], params["window"]
    g = Integrator(np.asarray(psi0), h, params["a"], params["s"], None, "dirichlet", 4, "c128", device=dev)
    st = RolloutStats()
    mout = torch.zeros(1, dtype=torch.float64, device=dev)
    masses = torch.zeros((1, 2), dtype=torch.float64, device=dev)
    verified = torch.as_tensor(np.asarray(psi0), dtype=torch.complex64, device=dev)[None].contiguous()
    m0 = _mass(verified[0], 1.0, mout)          # sum |psi0|^2
    span_len = 1 if mode == "strict" else max(1, int(every))
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    if sur is None:
        g.step(steps * n_windows, dt)
        st.windows = st.rk4_windows = n_windows
        verified = g.psi.to(torch.complex64)[None]
    w = 0
    while sur is not None and w < n_windows:
        span = min(span_len, n_windows - w)
        cur, cand, ok = verified, None, True
        for j in range(span):
            if j:
                cur = cand
            cand = sur.forward(cur, project=project, masses=masses)
            drift = abs(float(masses[0, 1].item()) - m0) / m0
            st.max_mass_drift = max(st.max_mass_drift, drift) if drift == drift else float("inf")
            if not drift <= tol_mass:
                ok = False
                st.rejected_mass += 1
                break
        ref = None
        if ok:
            g.psi.copy_(cur[0].to(torch.complex128))
            g.step(steps, dt)
            ref = g.psi.to(torch.complex64)[None]
            err = float(sur.compare(cand, ref)[0])
            st.checked += 1
            st.l2_errors.append(err)
            if err <= tol_l2:
                st.accepted += span
                verified = cand
                w += span
                continue
            st.rejected_l2 += 1
        if span == 1 and ref is not None:
            verified = ref.contiguous()            # the check already advanced this window from `verified`
        else:
            g.psi.copy_(verified[0].to(torch.complex128))
            g.step(steps * span, dt)
            verified = g.psi.to(torch.complex64)[None].contiguous()
        st.rk4_windows += span
        w += span
    st.windows = max(st.windows, w)
    torch.cuda.synchronize(dev)
    st.seconds = time.perf_counter() - t0
    g.close()
    return verified[0], st


def _rollout_parallel(sur, psi0, n_windows, params, width, tol_l2, tol_mass, project, device):
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    n = int(np.asarray(psi0).shape[0])
    pool = RK4Pool(n, width, params, dev)
    st = RolloutStats()
    masses = torch.zeros((width, 2), dtype=torch.float64, device=dev)
    verified = torch.as_tensor(np.asarray(psi0), dtype=torch.complex64, device=dev)[None].contiguous()
    m0 = _mass(verified[0], 1.0, torch.zeros(1, dtype=torch.float64, device=dev))   # sum |psi0|^2
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    w = 0
    span = max(2, width // 4)         # speculation depth: doubled after a clean round, cut after a failure
    while w < n_windows:
        K = min(span, n_windows - w)
        preds = [verified]
        for j in range(K):          # raw-output masses of the chain, read back once for the round
            preds.append(sur.forward(preds[-1], project=project, masses=masses[j:j + 1]))
        refs = pool.advance([p[0] for p in preds[:K]])
        errs = sur.compare(torch.cat(preds[1:]), torch.stack(refs))
        drift = np.abs(masses[:K, 1].cpu().numpy() - m0) / m0
        st.checked += K
        st.l2_errors.extend(float(e) for e in errs)
        st.max_mass_drift = max(st.max_mass_drift, float(np.max(drift)))
        bad = np.nonzero(~((errs <= tol_l2) & (drift <= tol_mass)))[0]
        if bad.size == 0:
            st.accepted += K
            verified = preds[K]
            w += K
            span = min(width, 2 * span)
        else:
            j = int(bad[0])                  # windows 0..j-1 of this round accepted, window j from RK4
            span = max(2, min(width, 2 * (j + 1)))
            st.accepted += j
            st.rk4_windows += 1
            if drift[j] > tol_mass or not np.isfinite(drift[j]):
                st.rejected_mass += 1
            else:
                st.rejected_l2 += 1
            verified = refs[j][None].contiguous()
            w += j + 1
        st.windows = w
    torch.cuda.synchronize(dev)
    st.seconds = time.perf_counter() - t0
    pool.close()
    return verified[0], st
