"""Seeded, synthetic inputs for the CDBM workloads of Sec. 3 of the paper.

This module holds only initial conditions and run parameters (grid, discrete
velocity set, I, tau, dt, dx, boundary kinds, step counts).  It contains none of
the method's arithmetic, so both the CUDA library's tests and the CPU oracle's
tests can take their inputs from it.

Every workload is deterministic; the ensemble draws its tube parameters from
``numpy.random.default_rng(seed)`` in a fixed order.

Velocity sets are the paper's per problem: Sod (Sec. 3.1), Lax (Sec. 3.2),
sound wave (Sec. 3.4) and Taylor-Green (Sec. 3.5).  Cell centres sit at
x_j = (j + 1/2) dx; a cell is "left" of an interface when its centre lies to the
left of it, so no centre falls on the interface.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
import math

import numpy as np

PERIODIC = 0
ZERO_GRADIENT = 1

# (v_a, v_b, v_c, v_d), (eta_a, eta_b, eta_c, eta_d)
VSET_SOD = ((2.5, 2.5, 1.2, 1.1), (0.0, 0.0, 0.0, 1.2))        # Sec. 3.1
VSET_LAX = ((4.4, 4.4, 3.0, 1.8), (0.0, 0.0, 5.0, 0.0))        # Sec. 3.2
VSET_SHOCK = ((21.8, 21.8, 17.8, 9.8), (18.8, 0.0, 0.0, 0.0))  # Sec. 3.3
VSET_SOUND = ((1.4, 1.1, 1.1, 1.0), (3.0, 0.0, 0.0, 0.0))      # Sec. 3.4
VSET_TGV = ((0.2, 0.2, 2.0, 2.0), (0.0, 5.0, 0.0, 2.6))        # Sec. 3.5


@dataclass
class Workload:
    """One run: parameters plus the initial rho, u_x, u_y, T fields ([ny][nx])."""
    name: str
    nx: int
    ny: int
    dx: float
    dy: float
    dt: float
    tau: float
    I: float
    vg: tuple
    eg: tuple
    bc_x: int
    bc_y: int
    steps: int
    rho: np.ndarray = field(repr=False)
    ux: np.ndarray = field(repr=False)
    uy: np.ndarray = field(repr=False)
    T: np.ndarray = field(repr=False)
    extra: dict = field(default_factory=dict)

    @property
    def cells(self) -> int:
        return self.nx * self.ny

    def with_steps(self, steps: int) -> "Workload":
        return replace(self, steps=int(steps))


def gamma_of(I: float, D: int = 2) -> float:
    """Specific heat ratio (D + I + 2) / (D + I), Sec. 2 after Eq. (5)."""
    return (D + I + 2.0) / (D + I)


def _centres(n: int, d: float, x0: float = 0.0) -> np.ndarray:
    return x0 + (np.arange(n) + 0.5) * d


def _riemann(name, nx, x_lo, x_hi, x_int, left, right, dt, tau, I, vset, steps):
    dx = (x_hi - x_lo) / nx
    x = _centres(nx, dx, x_lo)
    is_left = x < x_int
    fields = []
    for k in range(3):
        a = np.where(is_left, left[k], right[k]).astype(np.float64)
        fields.append(a.reshape(1, nx))
    rho, ux, T = fields
    return Workload(name=name, nx=nx, ny=1, dx=dx, dy=dx, dt=dt, tau=tau, I=float(I),
                    vg=vset[0], eg=vset[1], bc_x=ZERO_GRADIENT, bc_y=PERIODIC, steps=steps,
                    rho=rho, ux=ux, uy=np.zeros((1, nx)), T=T,
                    extra={"x_interface": x_int, "left": left, "right": right,
                           "x_lo": x_lo, "x_hi": x_hi})


def sod(nx: int = 500, I: float = 0.0, steps: int = 10000, dt: float = 2e-5,
        tau: float = 2e-5) -> Workload:
    """Sod tube on [0, 1], interface 0.5: (rho, u, T) = (1, 0, 1) | (0.125, 0, 0.8)."""
    return _riemann("sod", nx, 0.0, 1.0, 0.5, (1.0, 0.0, 1.0), (0.125, 0.0, 0.8),
                    dt, tau, I, VSET_SOD, steps)


def lax(nx: int = 2000, I: float = 0.0, steps: int = 10000, dt: float = 2e-5,
        tau: float = 1e-4) -> Workload:
    """Lax tube on [0, 2], interface 1: (0.445, 0.698, 7.928) | (0.5, 0, 1.142)."""
    return _riemann("lax", nx, 0.0, 2.0, 1.0, (0.445, 0.698, 7.928), (0.5, 0.0, 1.142),
                    dt, tau, I, VSET_LAX, steps)


def sound(n: int = 512, I: float = 0.0, steps: int = 2000, dt: float = 2e-5,
          tau: float = 1e-4, amp: float = 1e-3, ny: int | None = None) -> Workload:
    """Standing acoustic mode on the periodic unit square:
    rho = 1 + amp sin(2 pi x) sin(2 pi y), u = 0, T = 1 (ny = 1 gives the 1-D mode
    rho = 1 + amp sin(2 pi x))."""
    ny = n if ny is None else ny
    dx = 1.0 / n
    x = _centres(n, dx)
    if ny == 1:
        rho = (1.0 + amp * np.sin(2 * np.pi * x)).reshape(1, n)
    else:
        y = _centres(ny, 1.0 / ny)
        rho = 1.0 + amp * np.outer(np.sin(2 * np.pi * y), np.sin(2 * np.pi * x))
    z = np.zeros_like(rho)
    return Workload(name="sound", nx=n, ny=ny, dx=dx, dy=(1.0 / ny if ny > 1 else dx), dt=dt,
                    tau=tau, I=float(I), vg=VSET_SOUND[0], eg=VSET_SOUND[1], bc_x=PERIODIC,
                    bc_y=PERIODIC, steps=steps, rho=rho, ux=z.copy(), uy=z.copy(),
                    T=np.ones_like(rho), extra={"amp": amp})


def taylor_green(n: int = 4096, I: float = 3.0, steps: int = 2000, dt: float | None = None,
                 tau: float = 1e-4, U0: float = 0.01, L: float = 0.05, p0: float = 1.0,
                 rho0: float = 1.0, vset=VSET_TGV) -> Workload:
    """Taylor-Green vortex on the periodic square [0, 2L]^2 with k = pi / L:
    u = U0 sin(kx) cos(ky), v = -U0 cos(kx) sin(ky), rho = rho0,
    p = p0 + rho0 U0^2 / 4 (cos 2kx + cos 2ky), T = p / rho.
    The default dt is 5e-6 at n = 4096 (max(|v_x| + |v_y|) dt / dx = 0.82) and grows
    with the cell size on coarser grids, capped at tau / 2."""
    dx = 2 * L / n
    if dt is None:
        dt = min(5e-6 * 4096.0 / n, 0.5 * tau)
    k = math.pi / L
    x = _centres(n, dx)
    X, Y = np.meshgrid(x, x, indexing="xy")   # [ny][nx]
    ux = U0 * np.sin(k * X) * np.cos(k * Y)
    uy = -U0 * np.cos(k * X) * np.sin(k * Y)
    p = p0 + rho0 * U0 ** 2 / 4.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    rho = np.full_like(p, rho0)
    return Workload(name="taylor_green", nx=n, ny=n, dx=dx, dy=dx, dt=dt, tau=tau, I=float(I),
                    vg=vset[0], eg=vset[1], bc_x=PERIODIC, bc_y=PERIODIC, steps=steps,
                    rho=rho, ux=ux, uy=uy, T=p / rho,
                    extra={"U0": U0, "L": L, "k": k, "p0": p0, "rho0": rho0})


def random_smooth(nx: int, ny: int, seed: int = 0, vset=VSET_SOUND, I: float = 1.0,
                  dt: float = 2e-5, tau: float = 1e-4, amp: float = 0.05,
                  bc=(PERIODIC, PERIODIC), steps: int = 10) -> Workload:
    """Seeded smooth random fields (a few Fourier modes per field) for parity tests
    that need every velocity, axis and limiter branch exercised."""
    rng = np.random.default_rng(seed)
    x = _centres(nx, 1.0 / nx)
    y = _centres(ny, 1.0 / ny)
    X, Y = np.meshgrid(x, y, indexing="xy")
    out = []
    for base in (1.0, 0.0, 0.0, 1.0):
        a = np.full((ny, nx), base)
        for _ in range(3):
            kx, ky = rng.integers(0, 4, size=2)
            ph = rng.uniform(0, 2 * np.pi, size=2)
            c = rng.uniform(-amp, amp)
            a = a + c * np.cos(2 * np.pi * kx * X + ph[0]) * np.cos(2 * np.pi * ky * Y + ph[1])
        out.append(a)
    rho, ux, uy, T = out
    dx = 1.0 / nx
    return Workload(name="random_smooth", nx=nx, ny=ny, dx=dx, dy=1.0 / ny, dt=dt, tau=tau,
                    I=float(I), vg=vset[0], eg=vset[1], bc_x=bc[0], bc_y=bc[1], steps=steps,
                    rho=rho, ux=ux, uy=uy, T=T, extra={"seed": seed})


def random_blocks(nx: int, ny: int, seed: int = 0, vset=VSET_SOUND, I: float = 1.0,
                  dt: float = 2e-5, tau: float = 1e-4, bc=(PERIODIC, PERIODIC),
                  steps: int = 10) -> Workload:
    """Seeded piecewise-constant fields (jumps in x and y) that drive the limiter
    through its zero, left and right branches."""
    rng = np.random.default_rng(seed)
    bx = max(1, nx // 7)
    by = max(1, ny // 5)
    shape = ((ny + by - 1) // by, (nx + bx - 1) // bx)
    iy, ix = np.arange(ny)[:, None] // by, np.arange(nx)[None, :] // bx

    def blocks(lo, hi):              # each drawn value fills a by x bx block
        return rng.uniform(lo, hi, shape)[iy, ix]

    rho = blocks(0.5, 1.5)
    ux = blocks(-0.2, 0.2)
    uy = blocks(-0.2, 0.2)
    T = blocks(0.7, 1.3)
    dx = 1.0 / nx
    return Workload(name="random_blocks", nx=nx, ny=ny, dx=dx, dy=1.0 / ny, dt=dt, tau=tau,
                    I=float(I), vg=vset[0], eg=vset[1], bc_x=bc[0], bc_y=bc[1], steps=steps,
                    rho=np.ascontiguousarray(rho), ux=np.ascontiguousarray(ux),
                    uy=np.ascontiguousarray(uy), T=np.ascontiguousarray(T), extra={"seed": seed})


def ensemble_draw(n_tubes: int = 1024, seed: int = 0, nx_lo: int = 200, nx_hi: int = 4000):
    """Tube parameters of the shock-tube ensemble: Nx ~ U{nx_lo..nx_hi}, then per tube
    in order rho_L, rho_R ~ U[0.1, 1], T_L, T_R ~ U[0.5, 2], I ~ {0, 1, 2}; u = 0."""
    rng = np.random.default_rng(seed)
    nx = rng.integers(nx_lo, nx_hi + 1, n_tubes)
    tubes = []
    for t in range(n_tubes):
        rl, rr = rng.uniform(0.1, 1.0, 2)
        tl, tr = rng.uniform(0.5, 2.0, 2)
        I = float(rng.choice([0.0, 1.0, 2.0]))
        tubes.append({"nx": int(nx[t]), "rho": (rl, rr), "T": (tl, tr), "I": I})
    return tubes


def ensemble_tube(spec: dict, steps: int = 1000, dt: float = 2e-5, tau: float = 1e-4) -> Workload:
    """One tube of the ensemble on [0, 1], interface 0.5, Sod velocity set."""
    return _riemann("tube", spec["nx"], 0.0, 1.0, 0.5, (spec["rho"][0], 0.0, spec["T"][0]),
                    (spec["rho"][1], 0.0, spec["T"][1]), dt, tau, spec["I"], VSET_SOD, steps)


def sound_modes(n: int = 1024, seed: int = 0, kmax: int = 8, amp: float = 1e-3, I: float = 3.0,
                steps: int = 4000, dt: float = 2e-5, tau: float = 1e-4) -> Workload:
    """Periodic unit square with rho and T each perturbed by every Fourier mode
    (kx, ky) in [0..kmax]^2 with 0 < |k| <= kmax, amplitude amp and a uniform random
    phase per mode and field (drawn in the order rho modes, then T modes); u = 0.
    Sound-wave velocity set."""
    rng = np.random.default_rng(seed)
    x = _centres(n, 1.0 / n)
    X, Y = np.meshgrid(x, x, indexing="xy")
    modes = [(kx, ky) for kx in range(kmax + 1) for ky in range(kmax + 1)
             if 0 < kx * kx + ky * ky <= kmax * kmax]
    out = []
    for _ in range(2):
        a = np.ones((n, n))
        ph = rng.uniform(0.0, 2.0 * np.pi, len(modes))
        for (kx, ky), p in zip(modes, ph):
            a += amp * np.cos(2.0 * np.pi * (kx * X + ky * Y) + p)
        out.append(a)
    rho, T = out
    z = np.zeros((n, n))
    return Workload(name="sound_modes", nx=n, ny=n, dx=1.0 / n, dy=1.0 / n, dt=dt, tau=tau, I=float(I),
                    vg=VSET_SOUND[0], eg=VSET_SOUND[1], bc_x=PERIODIC, bc_y=PERIODIC, steps=steps,
                    rho=rho, ux=z, uy=z.copy(), T=T, extra={"seed": seed, "kmax": kmax, "amp": amp})


def paper_sod(steps: int = 400) -> Workload:
    """Sec. 3.1 as printed: 1500 x 1 cells on [0, 0.15] (dx = 1e-4), interface 0.075,
    dt = 2e-5, tau = 1e-4, gamma = 2 (I = 0)."""
    return _riemann("paper_sod", 1500, 0.0, 0.15, 0.075, (1.0, 0.0, 1.0), (0.125, 0.0, 0.8),
                    2e-5, 1e-4, 0.0, VSET_SOD, steps)


def paper_lax(steps: int = 10000) -> Workload:
    """Sec. 3.2 as printed: 1000 x 1 cells on [0, 2] (dx = 2e-3), interface 1, dt = 2e-5,
    tau = 1e-4, gamma = 1.4 (I = 3), t = 0.2."""
    return _riemann("paper_lax", 1000, 0.0, 2.0, 1.0, (0.445, 0.698, 7.928), (0.5, 0.0, 1.142),
                    2e-5, 1e-4, 3.0, VSET_LAX, steps)


def paper_shock(steps: int = 20000, tau: float = 1e-5) -> Workload:
    """Sec. 3.3: Ma = 15 shock into (1, 0, 1), post-shock state (5.8696, 14.7245, 44.6938)
    for x <= 0.02; 10000 x 1 cells with dx = 2e-4 (so the domain is [0, 2]; the text's
    x <= 1.5 does not match 10000 dx), dt = 2e-6, gamma = 1.4 (I = 3).  The paper
    gives no tau; 1e-5 keeps dt / tau = 0.2."""
    return _riemann("paper_shock", 10000, 0.0, 2.0, 0.02, (5.8696, 14.7245, 44.6938), (1.0, 0.0, 1.0),
                    2e-6, tau, 3.0, VSET_SHOCK, steps)


def paper_taylor_green(n: int, dt: float = 2e-5, tau: float = 5e-4) -> Workload:
    """Sec. 3.5: the vortex on [0, 0.1]^2 with tau = 5e-4, gamma = 1.4, velocity set
    (0.2, 0.2, 2, 2) / (0, 5, 0, 2.6) on an n x n grid."""
    return taylor_green(n=n, I=3.0, dt=dt, tau=tau)
