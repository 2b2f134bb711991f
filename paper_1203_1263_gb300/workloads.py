"""Seeded synthetic inputs for the NLSE integrator: grids, potentials and
initial states.

This module holds no step of the integration method itself: it builds the
arrays that both the CUDA path and the CPU oracle are given (initial Psi,
the potential V, grid spacing), plus the closed-form solutions that the
tests compare against.  Every random draw comes from one counter-based
generator, SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), so a (seed, index) pair always gives the
same number on any machine.

Array convention: C order, last index fastest.  A 3D grid has shape
(Nz, Ny, Nx); a 2D grid (Ny, Nx); a 1D grid (Nx,).  Psi is complex128.
The grid is x_i = x_lo + i*h with one h on every axis (Sec. 3, Eq. disc).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

BC_DIRICHLET = 0
BC_MSD = 1
BC_L0 = 2
BC_PERIODIC = 3

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset..offset+n-1 of the SplitMix64 sequence started at `seed`."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, n: int) -> np.ndarray:
    """Standard normals by Box-Muller (cosine branch) on two uniform streams."""
    u1 = 1.0 - uniform(seed, n, 0)          # (0, 1]
    u2 = uniform(seed, n, n)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def centred_axis(n: int, h: float) -> np.ndarray:
    """x_i = (i - (n-1)/2) h."""
    return (np.arange(n, dtype=np.float64) - 0.5 * (n - 1)) * h


@dataclass
class Problem:
    """One integration problem: everything nlse_create and the oracle take."""
    name: str
    shape: tuple
    h: float
    a: float
    s: float
    bc: int
    order: int
    psi0: np.ndarray                  # complex128, `shape`
    V: Optional[np.ndarray] = None    # float64, `shape`, or None for V = 0
    steps: int = 0                    # the workload's step count
    dt: Optional[float] = None        # fixed dt; None => 0.8 x the stability bound
    extra: dict = field(default_factory=dict)

    @property
    def dims(self) -> int:
        return len(self.shape)

    @property
    def sites(self) -> int:
        return int(np.prod(self.shape))

    def vmax(self) -> float:
        return 0.0 if self.V is None else float(np.max(np.abs(self.V)))


# ---------------------------------------------------------------------------
# Closed-form solutions (pins)
# ---------------------------------------------------------------------------

def bright_soliton(x, t, a=1.0, s=1.0, omega=1.0, c=0.5):
    """Moving bright soliton of i psi_t + a psi_xx + s|psi|^2 psi = 0 (s > 0):
    sqrt(2 omega/s) sech(sqrt(omega/a)(x - c t)) exp(i(c x/(2a) + (omega - c^2/(4a)) t))."""
    amp = math.sqrt(2.0 * omega / s)
    env = amp / np.cosh(math.sqrt(omega / a) * (x - c * t))
    phase = c * x / (2.0 * a) + (omega - c * c / (4.0 * a)) * t
    return env * np.exp(1j * phase)


def dark_soliton(x, t, a=1.0, s=-1.0, Omega=-1.0, c=0.5):
    """Co-moving dark soliton of Sec. 4, Eq. soliton (s < 0, Omega < 0)."""
    amp = math.sqrt(abs(Omega / s))
    env = amp * np.tanh(math.sqrt(abs(Omega) / (2.0 * a)) * (x - c * t))
    phase = c * x / (2.0 * a) + (Omega - c * c / (4.0 * a)) * t
    return env * np.exp(1j * phase)


def sine_mode(shape, modes):
    """prod_alpha sin(pi m_alpha i_alpha / (N_alpha - 1)); zero on every face."""
    out = np.ones(shape, dtype=np.float64)
    for ax, (n, m) in enumerate(zip(shape, modes)):
        v = np.sin(math.pi * m * np.arange(n) / (n - 1))
        sh = [1] * len(shape)
        sh[ax] = n
        out = out * v.reshape(sh)
    return out.astype(np.complex128)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def bright_soliton_1d(order: int = 4, n: int = 2001, L: float = 50.0, t_end: float = 10.0,
                      a=1.0, s=1.0, omega=1.0, c=0.5) -> Problem:
    """1D bright soliton on x in [-L, L] with n points, Dirichlet walls,
    dt = h^2/8 to t_end (the 1D plain-method workload)."""
    h = 2.0 * L / (n - 1)
    x = -L + h * np.arange(n)
    dt = h * h / 8.0
    steps = int(round(t_end / dt))
    return Problem("bright_soliton_1d", (n,), h, a, s, BC_DIRICHLET, order,
                   bright_soliton(x, 0.0, a, s, omega, c), None, steps, dt,
                   extra=dict(x=x, omega=omega, c=c, t_end=steps * dt))


def dark_soliton_1d(order: int = 4, h: float = 0.1, L: float = 30.0, t_end: float = 2.0,
                    dt: Optional[float] = None) -> Problem:
    """Sec. 4 dark soliton (s=-1, a=1, c=0.5, Omega=-1) with the MSD wall."""
    n = int(round(2 * L / h)) + 1
    x = -L + h * np.arange(n)
    if dt is None:
        dt = h * h / 8.0
    steps = int(round(t_end / dt))
    return Problem("dark_soliton_1d", (n,), h, 1.0, -1.0, BC_MSD, order,
                   dark_soliton(x, 0.0), None, steps, dt,
                   extra=dict(x=x, t_end=steps * dt))


def trap_vortex_3d(shape=(203, 87, 87), h: Optional[float] = None, noise_seed: int = 2,
                   noise: float = 1e-3, mu: float = 4.0, a: float = 0.5, s: float = -1.0,
                   steps: int = 3360) -> Problem:
    """3D GPE in the trap V = (x^2 + y^2 + (z/2)^2)/2 with a straight charge-1
    vortex line along z: Thomas-Fermi background times a tanh core, times a
    seeded 1e-3 Gaussian phase noise.  MSD walls, 2SHOC.

    The xy box is x, y in [-8.6, 8.6] for every resolution (h = 17.2/(Nx-1)),
    so (203, 87, 87) has h = 0.2 and (512, 256, 256) has h = 17.2/255."""
    nz, ny, nx = shape
    if h is None:
        h = 17.2 / (nx - 1)
    z = centred_axis(nz, h)[:, None, None]
    y = centred_axis(ny, h)[None, :, None]
    x = centred_axis(nx, h)[None, None, :]
    V = 0.5 * (x * x + y * y + (z / 2.0) ** 2)
    V = np.broadcast_to(V, shape).astype(np.float64)
    r_perp = np.sqrt(x * x + y * y)
    theta = np.arctan2(y, x)
    tf = np.sqrt(np.maximum(mu - V, 0.0) / abs(s))
    core = np.tanh(r_perp * math.sqrt(mu / (2.0 * a)))
    psi = tf * core * np.exp(1j * theta)
    if noise > 0:
        xi = normal(noise_seed, int(np.prod(shape))).reshape(shape)
        psi = psi * np.exp(1j * noise * xi)
    return Problem(f"trap_vortex_3d_{nz}x{ny}x{nx}", tuple(shape), h, a, s, BC_MSD, 4,
                   np.ascontiguousarray(psi, dtype=np.complex128), np.ascontiguousarray(V), steps, None,
                   extra=dict(mu=mu))


def vortex_rings_3d(n: int = 512, h: float = 0.25, seed: int = 3, R: float = 8.0,
                    a: float = 0.5, s: float = -1.0, rho: float = 1.0, steps: int = 2000) -> Problem:
    """Two counter-propagating vortex rings of radius R (axes along z) in a
    uniform background, tanh cores; ring centres drawn from `seed`
    (x_j, y_j ~ U[-4, 4], z_1 ~ U[-20, -12], z_2 ~ U[12, 20]).  V = 0, MSD, 2SHOC."""
    u = uniform(seed, 6)
    cx = -4.0 + 8.0 * u[[0, 3]]
    cy = -4.0 + 8.0 * u[[1, 4]]
    cz = np.array([-20.0 + 8.0 * u[2], 12.0 + 8.0 * u[5]])
    sigma = [1.0, -1.0]
    ax = centred_axis(n, h)
    z = ax[:, None, None]
    y = ax[None, :, None]
    x = ax[None, None, :]
    kappa = math.sqrt(abs(s) * rho / (2.0 * a))
    psi = np.full((n, n, n), math.sqrt(rho), dtype=np.complex128)
    for j in range(2):
        rc = np.sqrt((x - cx[j]) ** 2 + (y - cy[j]) ** 2)
        zz = z - cz[j]
        dp = np.sqrt((rc - R) ** 2 + zz * zz)
        dm = np.sqrt((rc + R) ** 2 + zz * zz)
        tp = np.arctan2(zz, rc - R)
        tm = np.arctan2(zz, rc + R)
        psi *= np.tanh(kappa * dp) * np.tanh(kappa * dm) * np.exp(1j * sigma[j] * (tp - tm))
    return Problem(f"vortex_rings_3d_{n}^3", (n, n, n), h, a, s, BC_MSD, 4,
                   np.ascontiguousarray(psi), None, steps, None,
                   extra=dict(centres=np.stack([cx, cy, cz], 1)))


# Total grid sizes of the timing tables of Sec. 7 (Tables 1-3).
PAPER_TABLE_SITES = {1: (1000, 10000, 100000, 1000000, 3000000),
                     2: (961, 10000, 99856, 1000000, 2999824),
                     3: (9261, 97336, 970299, 2985984)}


def paper_timing_problem(dims: int, total: int, order: int = 4) -> Problem:
    """The timing workloads of Sec. 4 and Sec. 7: s = -1, a = 1, V = 0, MSD
    walls, k = 0.005 to t = 50 (10,000 steps).

      1D  the dark soliton of Eq. soliton (c = 0.5, Omega = -1) at h = 0.1
          (the step whose stability bounds Sec. 4 prints), N = total points
      2D  the dark vortex of Eq. exmp2Dvort with m = 1, its radial profile
          approximated, as in Sec. 4, by the c = 0 soliton profile
          tanh(r / sqrt 2); h = 0.25, N = M = floor(sqrt(total))
      3D  a dark vortex ring of radius d = 5 about the z axis: the 2D m = 1
          vortex placed at r = d in the r-z half-plane (tanh core, times its
          mirror at r = -d), h = 3/2, N = M = L = round(cbrt(total)), times
          the back-flow phase exp(i c z / (2a)) of Eq. 3dvr1.  The paper
          takes c from an asymptotic formula without printing it; here c is
          the large-ring speed of Roberts and Grant (1971),
          U = (ln(8R) - 0.615) / (2R) for i psi_t = -lap psi / 2 + |psi|^2 psi,
          rescaled to a = 1 (lengths x sqrt(2a)): c = sqrt(2) U(d / sqrt(2)).
          Without it the ring runs into a wall within the 10,000 steps and
          the MSD wall ratio diverges.
    Grids are centred on the origin."""
    a, s, dt, steps = 1.0, -1.0, 0.005, 10000
    if dims == 1:
        h = 0.1
        x = centred_axis(total, h)
        return Problem(f"paper_dark_soliton_1d_{total}", (total,), h, a, s, BC_MSD, order,
                       dark_soliton(x, 0.0), None, steps, dt, extra=dict(x=x))
    kappa = 1.0 / math.sqrt(2.0)      # sqrt(|Omega| / (2a)) with Omega = -1
    if dims == 2:
        n = int(math.isqrt(total))
        h = 0.25
        y = centred_axis(n, h)[:, None]
        x = centred_axis(n, h)[None, :]
        psi = np.tanh(kappa * np.sqrt(x * x + y * y)) * np.exp(1j * np.arctan2(y, x))
        return Problem(f"paper_dark_vortex_2d_{n}x{n}", (n, n), h, a, s, BC_MSD, order,
                       np.ascontiguousarray(psi, dtype=np.complex128), None, steps, dt)
    n = int(round(total ** (1.0 / 3.0)))
    h, d = 1.5, 5.0
    ax = centred_axis(n, h)
    z = ax[:, None, None]
    y = ax[None, :, None]
    x = ax[None, None, :]
    rc = np.sqrt(x * x + y * y)
    dp = np.sqrt((rc - d) ** 2 + z * z)
    dm = np.sqrt((rc + d) ** 2 + z * z)
    Rs = d / math.sqrt(2.0 * a)
    c = math.sqrt(2.0 * a) * (math.log(8.0 * Rs) - 0.615) / (2.0 * Rs)
    psi = np.tanh(kappa * dp) * np.tanh(kappa * dm) * np.exp(1j * (np.arctan2(z, rc - d) - np.arctan2(z, rc + d)))
    psi = psi * np.exp(1j * c * z / (2.0 * a))
    return Problem(f"paper_vortex_ring_3d_{n}^3", (n, n, n), h, a, s, BC_MSD, order,
                   np.ascontiguousarray(psi, dtype=np.complex128), None, steps, dt, extra=dict(c=c))


def gaussian_packet_2d(n: int, h: float, A: float, w: float, r0, p, a: float, s: float,
                       omega: float = 0.0):
    """A exp(-|r - r0|^2/(2 w^2)) exp(i p.r) on a centred n x n grid, and the
    trap V = omega^2 (x^2 + y^2)/2 (None when omega == 0)."""
    ax = centred_axis(n, h)
    y = ax[:, None]
    x = ax[None, :]
    psi = A * np.exp(-((x - r0[0]) ** 2 + (y - r0[1]) ** 2) / (2.0 * w * w)) * np.exp(1j * (p[0] * x + p[1] * y))
    V = None
    if omega > 0:
        V = np.ascontiguousarray(np.broadcast_to(0.5 * omega * omega * (x * x + y * y), (n, n)), dtype=np.float64)
    return np.ascontiguousarray(psi, dtype=np.complex128), V


TOWNES_MASS = 11.70   # critical mass of the 2D cubic NLSE for a = s = 1 (Townes soliton, 2*pi*1.8620)


def batch_runs_2d(nruns: int = 512, seed: int = 4, h: float = 0.25, nmin: int = 64, nmax: int = 1024,
                  steps: int = 1000):
    """Descriptors of `nruns` independent 2D runs with uneven sizes and parameters.

    Run r draws, from SplitMix64 stream (seed, 16 r ...): side ~ U{nmin..nmax},
    a ~ U[0.5, 1], s in {-1, +1}, trap omega ~ U[0.05, 0.2] with p = 1/2 else V = 0,
    order in {2, 4}, packet width w ~ U[2, 8], centre in the central half box,
    |p| ~ U[0, 1] in a uniform direction.  Focusing runs carry 0.8 of the
    critical mass so that none collapses; defocusing runs have A = 1.
    The initial state itself is built lazily by `batch_run_problem`."""
    runs = []
    for r in range(nruns):
        u = uniform(seed, 16, 16 * r)
        n = int(nmin + min(int(u[0] * (nmax - nmin + 1)), nmax - nmin))
        a = 0.5 + 0.5 * u[1]
        s = 1.0 if u[2] < 0.5 else -1.0
        omega = (0.05 + 0.15 * u[4]) if u[3] < 0.5 else 0.0
        order = 4 if u[5] < 0.5 else 2
        w = 2.0 + 6.0 * u[6]
        half = 0.25 * (n - 1) * h
        r0 = (-half + 2 * half * u[7], -half + 2 * half * u[8])
        pm = u[9]
        ang = 2.0 * math.pi * u[10]
        p = (pm * math.cos(ang), pm * math.sin(ang))
        if s > 0:
            A = math.sqrt(0.8 * TOWNES_MASS * a / (math.pi * w * w))
        else:
            A = 1.0
        runs.append(dict(n=n, h=h, a=a, s=s, omega=omega, order=order, w=w, r0=r0, p=p, A=A,
                         bc=BC_DIRICHLET, steps=steps))
    return runs


def batch_run_problem(run: dict) -> Problem:
    psi, V = gaussian_packet_2d(run["n"], run["h"], run["A"], run["w"], run["r0"], run["p"],
                                run["a"], run["s"], run["omega"])
    return Problem(f"batch_run_{run['n']}", (run["n"], run["n"]), run["h"], run["a"], run["s"],
                   run["bc"], run["order"], psi, V, run["steps"], None)


def humps_2d(seed: int, index: int, n: int = 256, h: float = 0.2):
    """1-4 bright Gaussian humps (amplitude ~ U[0.5, 1.5], width ~ U[0.7, 1.2],
    centres in the central 60 % of the box, phase slope |p| ~ U[0, 1]) for the
    focusing 2D surrogate workload.  Returns complex128 (n, n)."""
    u = uniform(seed, 32, 32 * index)
    k = 1 + min(int(u[0] * 4), 3)
    ax = centred_axis(n, h)
    y = ax[:, None]
    x = ax[None, :]
    half = 0.3 * (n - 1) * h
    psi = np.zeros((n, n), dtype=np.complex128)
    for j in range(k):
        o = 1 + 7 * j
        A = 0.5 + u[o]
        w = 0.7 + 0.5 * u[o + 1]
        x0 = -half + 2 * half * u[o + 2]
        y0 = -half + 2 * half * u[o + 3]
        pm = u[o + 4]
        ang = 2.0 * math.pi * u[o + 5]
        psi += A * np.exp(-((x - x0) ** 2 + (y - y0) ** 2) / (2 * w * w)) * \
            np.exp(1j * pm * (math.cos(ang) * x + math.sin(ang) * y))
    return psi


def random_field(shape, seed: int) -> np.ndarray:
    """Complex field with i.i.d. U[-1, 1) parts (parity tests on small grids)."""
    n = int(np.prod(shape))
    u = uniform(seed, 2 * n)
    z = (2.0 * u[:n] - 1.0) + 1j * (2.0 * u[n:] - 1.0)
    return z.reshape(shape).astype(np.complex128)


def random_potential(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    n = int(np.prod(shape))
    return (scale * uniform(seed, n)).reshape(shape).astype(np.float64)
