"""Synthetic workloads shaped like the paper's experiments.

Input generation only.  Each builder returns plain numpy arrays (initial data,
separable body-load tables, Dirichlet wall data) that both the oracle and the
CUDA library consume; nothing here evaluates the lattice Boltzmann scheme.

Workloads
---------
* ``periodic_mms``   -- periodic square with the moving manufactured solution of
  Eq. periodic_moving (any amplitude / wavenumbers), body load from the Navier form.
* ``dirichlet_mms``  -- same solution on a rectangle with u = u_hat on all edges.
* ``plane_wave_periodic`` -- periodic square with a body-force-free standing P or S wave.
* ``energy_box``     -- homogeneous Dirichlet, b = 0, the initial data of Sec. 6.2.
* ``grf_periodic``   -- periodic lattice at rest (u0 = 0) with a Gaussian random
  initial velocity (correlation length ell cells, given std), b = 0.
* ``batch_spec``     -- sizes, materials and boundary types of a ragged batch.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

from . import grf as _grf
from . import mms as _mms
from .material import lattice_speed, poisson_to_speeds


@dataclass
class Workload:
    """Everything needed to run one lattice from t = 0 for ``steps`` steps."""
    name: str
    nx: int
    ny: int
    dx: float
    dt: float
    cK: float
    cmu: float
    dirichlet: bool
    steps: int
    U0: np.ndarray                       # [5, ny, nx]
    dU0dx: np.ndarray                    # [5, ny, nx]
    dU0dy: np.ndarray                    # [5, ny, nx]
    u0: Optional[np.ndarray] = None      # [2, ny, nx]
    # separable body load b_c(x_k, y_l, t_m) = sum_r X[r,k] Y[r,l] T[m,c,r], m = 0..steps
    forcing: Optional[tuple] = None      # (X [R,nx], Y [R,ny], T [steps+1, 2, R])
    # d/dt u_D at the wall midpoints at t_m + dt/2, m = 0..steps-1: [steps, 2, 2(nx+ny)]
    wall: Optional[np.ndarray] = None
    exact: Optional[_mms.Manufactured] = None
    meta: dict = field(default_factory=dict)

    @property
    def c(self) -> float:
        return self.dx / self.dt

    def body_load(self, m: int) -> Optional[np.ndarray]:
        if self.forcing is None:
            return None
        X, Y, T = self.forcing
        return _mms.eval_tables(X, Y, T[m])

    def wall_data(self, m: int) -> Optional[np.ndarray]:
        return None if self.wall is None else self.wall[m]

    def exact_outputs(self, t: float) -> np.ndarray:
        """[v(2), j(3), u(2), sigma(3)] of the manufactured solution on the nodes."""
        sol = self.exact
        fields = sol.U_fields() + sol.displacement() + sol.stress()
        return _mms.dense_stack(fields, self.nx, self.ny, self.dx, t)


def _from_solution(name, sol, nx, ny, dx, dt, dirichlet, steps, with_forcing=True, with_wall=True):
    U0 = _mms.dense_stack(sol.U_fields(), nx, ny, dx, 0.0)
    dU0dx = _mms.dense_stack(sol.U_fields(p=1), nx, ny, dx, 0.0)
    dU0dy = _mms.dense_stack(sol.U_fields(r=1), nx, ny, dx, 0.0)
    u0 = _mms.dense_stack(sol.displacement(), nx, ny, dx, 0.0)
    forcing = None
    if with_forcing:
        times = np.arange(steps + 1) * dt
        forcing = _mms.separable_tables(sol.body_load(), nx, ny, dx, times)
    wall = None
    if dirichlet and with_wall:
        wall = np.stack([_mms.wall_velocity(sol, nx, ny, dx, (m + 0.5) * dt) for m in range(steps)])
    return Workload(name, nx, ny, dx, dt, sol.cK, sol.cmu, dirichlet, steps, U0, dU0dx, dU0dy,
                    u0, forcing, wall, sol)


def periodic_mms(n: int, cK2: float, cmu2: float, *, c: Optional[float] = None, cfl: float = 0.9,
                 steps: Optional[int] = None, t_final: float = 1.0, amp: float = 1.0,
                 kx: float = 4 * math.pi, ky: float = 2 * math.pi, w: float = 4 * math.pi,
                 length: float = 1.0) -> Workload:
    dx = length / n
    c = lattice_speed(cK2, cmu2, cfl) if c is None else c
    dt = dx / c
    if steps is None:
        steps = int(round(t_final / dt))
    sol = _mms.paper_moving_solution(math.sqrt(cK2), math.sqrt(cmu2), amp, kx, ky, w)
    return _from_solution(f"periodic_mms_{n}", sol, n, n, dx, dt, False, steps)


def dirichlet_mms(nx: int, ny: int, cK2: float, cmu2: float, *, c: Optional[float] = None,
                  cfl: float = 0.9, steps: Optional[int] = None, t_final: float = 1.0,
                  height: float = 1.0, amp: float = 1.0, kx: float = 4 * math.pi,
                  ky: float = 2 * math.pi, w: float = 4 * math.pi) -> Workload:
    dx = height / ny
    c = lattice_speed(cK2, cmu2, cfl) if c is None else c
    dt = dx / c
    if steps is None:
        steps = int(round(t_final / dt))
    sol = _mms.paper_moving_solution(math.sqrt(cK2), math.sqrt(cmu2), amp, kx, ky, w)
    return _from_solution(f"dirichlet_mms_{nx}x{ny}", sol, nx, ny, dx, dt, True, steps)


def plane_wave_periodic(n: int, cK2: float, cmu2: float, kind: str, *, cfl: float = 0.9,
                        steps: Optional[int] = None, t_final: float = 1.0, amp: float = 1e-2,
                        k: float = 2 * math.pi) -> Workload:
    """Periodic unit square with a body-force-free standing P wave (kind "P": u_x) or S wave
    (kind "S": u_y) along x, one wavelength per side for k = 2 pi; b = 0, so no forcing tables."""
    dx = 1.0 / n
    dt = dx / lattice_speed(cK2, cmu2, cfl)
    if steps is None:
        steps = int(round(t_final / dt))
    sol = _mms.plane_wave(math.sqrt(cK2), math.sqrt(cmu2), kind, amp, k)
    return _from_solution(f"plane_wave_{kind}_{n}", sol, n, n, dx, dt, False, steps, with_forcing=False)


def energy_box(n: int, cK2: float, cmu2: float, dt: float, steps: int) -> Workload:
    """Homogeneous Dirichlet on the unit square, b = 0, initial data of Sec. 6.2."""
    dx = 1.0 / n
    sol = _mms.paper_energy_initial(math.sqrt(cK2), math.sqrt(cmu2))
    wl = _from_solution(f"energy_box_{n}", sol, n, n, dx, dt, True, steps,
                        with_forcing=False, with_wall=False)
    wl.exact = None
    return wl


def grf_periodic(nx: int, ny: int, cK2: float, cmu2: float, *, cfl: float = 0.9, ell: float = 64.0,
                 std: float = 1e-3, seeds=(1, 2), steps: int = 100, dx: Optional[float] = None,
                 window: bool = False) -> Workload:
    """Lattice at rest with a Gaussian random initial velocity (u0 = 0, b = 0).

    U0 = [v0x, v0y, 0, 0, 0]; dU0 from spectral derivatives of the GRFs.  With
    ``window`` the velocity is multiplied by sin(pi x/Lx) sin(pi y/Ly), which
    vanishes on the edges (used for homogeneous Dirichlet lattices).
    """
    dx = 1.0 / max(nx, ny) if dx is None else dx
    c = lattice_speed(cK2, cmu2, cfl)
    dt = dx / c
    v = [_grf.gaussian_random_field(nx, ny, ell, std, s) for s in seeds]
    grads = [_grf.spectral_gradient(vi, dx) for vi in v]
    if window:
        xs = (np.arange(nx) + 0.5) / nx
        ys = (np.arange(ny) + 0.5) / ny
        wx, wy = np.sin(np.pi * xs)[None, :], np.sin(np.pi * ys)[:, None]
        dwx = (np.pi / (nx * dx)) * np.cos(np.pi * xs)[None, :]
        dwy = (np.pi / (ny * dx)) * np.cos(np.pi * ys)[:, None]
        win = wy * wx
        grads = [(g[0] * win + vi * wy * dwx, g[1] * win + vi * dwy * wx) for vi, g in zip(v, grads)]
        v = [vi * win for vi in v]
    U0 = np.zeros((5, ny, nx))
    dU0dx = np.zeros((5, ny, nx))
    dU0dy = np.zeros((5, ny, nx))
    U0[0], U0[1] = v
    dU0dx[0], dU0dy[0] = grads[0]
    dU0dx[1], dU0dy[1] = grads[1]
    return Workload(f"grf_periodic_{nx}x{ny}", nx, ny, dx, dt, math.sqrt(cK2), math.sqrt(cmu2),
                    window, steps, U0, dU0dx, dU0dy, np.zeros((2, ny, nx)),
                    meta={"ell": ell, "std": std, "seeds": list(seeds)})


@dataclass
class LatticeSpec:
    nx: int
    ny: int
    cK2: float
    cmu2: float
    nu: float
    dirichlet: bool
    ell: float
    seed: int


def batch_spec(count: int = 512, seed: int = 3, smin: int = 64, smax: int = 1024,
               amin: float = 1.0, amax: float = 4.0, numax: float = 0.49) -> List[LatticeSpec]:
    """Ragged batch: short side log-uniform in [smin, smax], aspect uniform in [amin, amax],
    random orientation, Poisson ratio uniform in [0, numax] with cK^2 + cmu^2 = 2,
    even index periodic, odd index homogeneous Dirichlet, GRF length s/16."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        s = int(round(math.exp(rng.uniform(math.log(smin), math.log(smax)))))
        a = rng.uniform(amin, amax)
        long = int(round(a * s))
        flip = bool(rng.integers(0, 2))
        nx, ny = (long, s) if flip else (s, long)
        nu = float(rng.uniform(0.0, numax))
        cK2, cmu2 = poisson_to_speeds(nu)
        out.append(LatticeSpec(nx, ny, cK2, cmu2, nu, i % 2 == 1, s / 16.0, 1000 + i))
    return out
