"""Manufactured solutions as separable trigonometric fields (Sec. 6.1).

Input generation only: this module knows the target PDE (Eqs. teq, cauchy and
the first-order variables of Eqs. vx-jxy) so it can produce the exact fields,
the body load b, the initial data and the Dirichlet data of a manufactured
displacement u_hat.  It contains none of the lattice Boltzmann scheme.

Every displacement component is one product

    u_hat_c = A_c * Fx(kx (x - ax t) + px) * Fy(ky (y - ay t) + py) * Ft(w t + pt),

with F in {sin, cos}; Eq. periodic_moving is of this form.  All derivatives
stay in that family, and at a fixed time every field is a sum of blocks

    field(x, y) = [sin kx x, cos kx x] C(t) [sin ky y, cos ky y]^T,

which gives exact dense values and exact separable tables
B(x_k, y_l, t) = sum_r X_r(x_k) Y_r(y_l) T_r(t).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Dict, List, Tuple

import numpy as np


@dataclass(frozen=True)
class Factor:
    kind: str      # "sin" or "cos"
    k: float       # wavenumber
    speed: float   # advection speed (argument k (s - speed t) + phase)
    phase: float

    def nth(self, n: int, theta):
        """n-th derivative of F with respect to its argument, at theta."""
        shift = n * math.pi / 2.0
        return np.sin(theta + shift) if self.kind == "sin" else np.cos(theta + shift)

    def basis_coeffs(self, n: int, t: float):
        """F^(n)(k s + psi(t)) = a sin(k s) + b cos(k s); returns (a, b)."""
        psi = -self.k * self.speed * t + self.phase + n * math.pi / 2.0
        if self.kind == "sin":
            return math.cos(psi), math.sin(psi)
        return -math.sin(psi), math.cos(psi)


@dataclass(frozen=True)
class DispComponent:
    amp: float
    fx: Factor
    fy: Factor
    ft: Factor     # speed must be 0; argument w t + phase


def _multinomial_splits(q: int):
    for q1 in range(q + 1):
        for q2 in range(q + 1 - q1):
            q3 = q - q1 - q2
            coef = math.factorial(q) // (math.factorial(q1) * math.factorial(q2) * math.factorial(q3))
            yield q1, q2, q3, coef


@dataclass
class SepField:
    """Sum of blocks {(kx, ky): C(t)} with C a 2x2 matrix function of t."""
    blocks: List[Tuple[float, float, Callable[[float], np.ndarray]]] = field(default_factory=list)

    def __add__(self, other: "SepField") -> "SepField":
        return SepField(self.blocks + other.blocks)

    def __sub__(self, other: "SepField") -> "SepField":
        return self + (-1.0) * other

    def __rmul__(self, s: float) -> "SepField":
        return SepField([(kx, ky, (lambda t, C=C, s=s: s * C(t))) for kx, ky, C in self.blocks])

    def merged(self, t: float) -> Dict[Tuple[float, float], np.ndarray]:
        out: Dict[Tuple[float, float], np.ndarray] = {}
        for kx, ky, C in self.blocks:
            key = (kx, ky)
            out[key] = out.get(key, np.zeros((2, 2))) + C(t)
        return out

    def keys(self):
        seen = []
        for kx, ky, _ in self.blocks:
            if (kx, ky) not in seen:
                seen.append((kx, ky))
        return seen

    def dense(self, xs, ys, t: float) -> np.ndarray:
        """Values on the tensor grid ys x xs -> array [len(ys), len(xs)]."""
        xs = np.asarray(xs, dtype=np.float64)
        ys = np.asarray(ys, dtype=np.float64)
        out = np.zeros((ys.size, xs.size))
        for (kx, ky), C in self.merged(t).items():
            bx = np.stack([np.sin(kx * xs), np.cos(kx * xs)])    # [2, nx]
            by = np.stack([np.sin(ky * ys), np.cos(ky * ys)])    # [2, ny]
            out += by.T @ C.T @ bx
        return out

    def points(self, xs, ys, t: float) -> np.ndarray:
        """Values at the point list (xs[i], ys[i])."""
        xs = np.asarray(xs, dtype=np.float64)
        ys = np.asarray(ys, dtype=np.float64)
        out = np.zeros(xs.shape)
        for (kx, ky), C in self.merged(t).items():
            bx = np.stack([np.sin(kx * xs), np.cos(kx * xs)])
            by = np.stack([np.sin(ky * ys), np.cos(ky * ys)])
            out += np.einsum("ip,ij,jp->p", bx, C, by)
        return out


def _deriv(comp: DispComponent, p: int, r: int, q: int) -> SepField:
    """d^p/dx^p d^r/dy^r d^q/dt^q of one displacement component."""
    fx, fy, ft = comp.fx, comp.fy, comp.ft

    def C(t, p=p, r=r, q=q):
        M = np.zeros((2, 2))
        for q1, q2, q3, coef in _multinomial_splits(q):
            sx = (fx.k ** p) * ((-fx.k * fx.speed) ** q1)
            sy = (fy.k ** r) * ((-fy.k * fy.speed) ** q2)
            st = (ft.k ** q3) * ft.nth(q3, ft.k * t + ft.phase)
            vx = np.array(fx.basis_coeffs(p + q1, t))
            vy = np.array(fy.basis_coeffs(r + q2, t))
            M += comp.amp * coef * sx * sy * st * np.outer(vx, vy)
        return M

    return SepField([(fx.k, fy.k, C)])


class Manufactured:
    """Exact fields of a manufactured displacement u_hat for wave speeds (cK, cmu)."""

    def __init__(self, ux: DispComponent, uy: DispComponent, cK: float, cmu: float):
        self.c = (ux, uy)
        self.cK, self.cmu = cK, cmu

    def D(self, comp: int, p: int = 0, r: int = 0, q: int = 0) -> SepField:
        return _deriv(self.c[comp], p, r, q)

    # first-order variables (Eqs. vx-jxy) with p extra x- and r extra y-derivatives
    def U_fields(self, p: int = 0, r: int = 0) -> List[SepField]:
        cK, cmu, D = self.cK, self.cmu, self.D
        vx = D(0, p, r, 1)
        vy = D(1, p, r, 1)
        dxux = D(0, p + 1, r)
        dyuy = D(1, p, r + 1)
        dxuy = D(1, p + 1, r)
        dyux = D(0, p, r + 1)
        js = (-cK) * (dxux + dyuy)
        jd = (-cmu) * (dxux - dyuy)
        jxy = (-cmu) * (dxuy + dyux)
        return [vx, vy, js, jd, jxy]

    def displacement(self) -> List[SepField]:
        return [self.D(0), self.D(1)]

    def stress(self) -> List[SepField]:
        """sigma = cK^2 div(u) I + cmu^2 (grad u + grad u^T - div(u) I), Eq. cauchy."""
        cK2, cmu2, D = self.cK ** 2, self.cmu ** 2, self.D
        div = D(0, 1, 0) + D(1, 0, 1)
        dif = D(0, 1, 0) - D(1, 0, 1)
        return [cK2 * div + cmu2 * dif, cK2 * div - cmu2 * dif, cmu2 * (D(1, 1, 0) + D(0, 0, 1))]

    def body_load(self) -> List[SepField]:
        """b = d2u/dt2 - cK^2 grad(div u) - cmu^2 lap(u) (Navier form of Eq. teq)."""
        cK2, cmu2, D = self.cK ** 2, self.cmu ** 2, self.D
        bx = D(0, 0, 0, 2) - cK2 * (D(0, 2, 0) + D(1, 1, 1)) - cmu2 * (D(0, 2, 0) + D(0, 0, 2))
        by = D(1, 0, 0, 2) - cK2 * (D(0, 1, 1) + D(1, 0, 2)) - cmu2 * (D(1, 2, 0) + D(1, 0, 2))
        return [bx, by]

    def velocity(self) -> List[SepField]:
        return [self.D(0, 0, 0, 1), self.D(1, 0, 0, 1)]


def paper_moving_solution(cK: float, cmu: float, amp: float = 1.0, kx: float = 4 * math.pi,
                          ky: float = 2 * math.pi, w: float = 4 * math.pi) -> Manufactured:
    """Eq. periodic_moving (amp = 1, kx = 4 pi, ky = 2 pi, w = 4 pi in the paper)."""
    ux = DispComponent(amp, Factor("sin", kx, 0.3, 0.0), Factor("cos", ky, 0.8, 0.0),
                       Factor("sin", w, 0.0, -0.1 * w))
    uy = DispComponent(amp, Factor("cos", kx, 0.7, 0.0), Factor("sin", ky, 0.1, 0.0),
                       Factor("cos", w, 0.0, 0.4 * w))
    return Manufactured(ux, uy, cK, cmu)


def paper_energy_initial(cK: float, cmu: float) -> Manufactured:
    """The initial data of the energy test (Sec. 6.2): u = sin(4 pi x) sin(2 pi y) [sin(4 pi (t-0.1)), sin(4 pi (t+0.4))].

    Zero on the boundary of the unit square for every t; u_0 and v_0 are taken at t = 0.
    """
    ux = DispComponent(1.0, Factor("sin", 4 * math.pi, 0.0, 0.0), Factor("sin", 2 * math.pi, 0.0, 0.0),
                       Factor("sin", 4 * math.pi, 0.0, -0.4 * math.pi))
    uy = DispComponent(1.0, Factor("sin", 4 * math.pi, 0.0, 0.0), Factor("sin", 2 * math.pi, 0.0, 0.0),
                       Factor("sin", 4 * math.pi, 0.0, 1.6 * math.pi))
    return Manufactured(ux, uy, cK, cmu)


def plane_wave(cK: float, cmu: float, kind: str, amp: float = 1e-2, k: float = 2 * math.pi) -> Manufactured:
    """Body-force-free standing waves along x: P wave (u_x) or S wave (u_y).

    u = amp sin(k x) cos(k c t) with c = sqrt(cK^2 + cmu^2) (P) or cmu (S).
    """
    cp = math.sqrt(cK ** 2 + cmu ** 2)
    zero = DispComponent(0.0, Factor("sin", k, 0.0, 0.0), Factor("cos", 0.0, 0.0, 0.0),
                         Factor("cos", 0.0, 0.0, 0.0))
    if kind == "P":
        ux = DispComponent(amp, Factor("sin", k, 0.0, 0.0), Factor("cos", 0.0, 0.0, 0.0),
                           Factor("cos", k * cp, 0.0, 0.0))
        return Manufactured(ux, zero, cK, cmu)
    uy = DispComponent(amp, Factor("sin", k, 0.0, 0.0), Factor("cos", 0.0, 0.0, 0.0),
                       Factor("cos", k * cmu, 0.0, 0.0))
    return Manufactured(zero, uy, cK, cmu)


# ---------------------------------------------------------------------------
# lattice sampling helpers (cell-centred nodes x_k = (k + 1/2) dx)
# ---------------------------------------------------------------------------

def node_coords(n: int, dx: float) -> np.ndarray:
    return (np.arange(n) + 0.5) * dx


def dense_stack(fields: List[SepField], nx: int, ny: int, dx: float, t: float) -> np.ndarray:
    xs, ys = node_coords(nx, dx), node_coords(ny, dx)
    return np.stack([f.dense(xs, ys, t) for f in fields])


def wall_points(nx: int, ny: int, dx: float):
    """Wall midpoints x_b in the edge order [left rows | right rows | bottom cols | top cols]."""
    xs, ys = node_coords(nx, dx), node_coords(ny, dx)
    Lx, Ly = nx * dx, ny * dx
    px = np.concatenate([np.zeros(ny), np.full(ny, Lx), xs, xs])
    py = np.concatenate([ys, ys, np.zeros(nx), np.full(nx, Ly)])
    return px, py


def wall_velocity(sol: Manufactured, nx: int, ny: int, dx: float, t: float) -> np.ndarray:
    """d/dt u_D at the wall midpoints at time t, [2, 2(nx+ny)]."""
    px, py = wall_points(nx, ny, dx)
    return np.stack([f.points(px, py, t) for f in sol.velocity()])


def separable_tables(fields: List[SepField], nx: int, ny: int, dx: float, times) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Exact separable form of a 2-component field on the lattice.

    Returns X [R, nx], Y [R, ny], T [len(times), 2, R] with
    field_c(x_k, y_l, t_m) = sum_r X[r, k] Y[r, l] T[m, c, r].
    """
    xs, ys = node_coords(nx, dx), node_coords(ny, dx)
    keys = []
    for f in fields:
        for key in f.keys():
            if key not in keys:
                keys.append(key)
    X, Y, index = [], [], []
    for (kx, ky) in keys:
        for a in range(2):
            for b in range(2):
                X.append(np.sin(kx * xs) if a == 0 else np.cos(kx * xs))
                Y.append(np.sin(ky * ys) if b == 0 else np.cos(ky * ys))
                index.append(((kx, ky), a, b))
    X = np.stack(X)
    Y = np.stack(Y)
    T = np.zeros((len(times), len(fields), len(index)))
    for m, t in enumerate(times):
        for c, f in enumerate(fields):
            merged = f.merged(float(t))
            for r, (key, a, b) in enumerate(index):
                if key in merged:
                    T[m, c, r] = merged[key][a, b]
    return X, Y, T


def eval_tables(X, Y, Tm) -> np.ndarray:
    """Dense [2, ny, nx] field from one time slice of separable tables."""
    return np.einsum("rx,ry,cr->cyx", X, Y, Tm)


def separable_wall_tables(fields: List[SepField], nx: int, ny: int, dx: float, times):
    """Separable form on the walls: Xn [R, nx] (node columns), Xw [R, 2] (x = 0, nx dx),
    Yn [R, ny] (node rows), Yw [R, 2] (y = 0, ny dx), T [len(times), 2, R]."""
    xs, ys = node_coords(nx, dx), node_coords(ny, dx)
    xw, yw = np.array([0.0, nx * dx]), np.array([0.0, ny * dx])
    keys = []
    for f in fields:
        for key in f.keys():
            if key not in keys:
                keys.append(key)
    Xn, Xw, Yn, Yw, index = [], [], [], [], []
    for (kx, ky) in keys:
        for a in range(2):
            for b in range(2):
                fx = np.sin if a == 0 else np.cos
                fy = np.sin if b == 0 else np.cos
                Xn.append(fx(kx * xs))
                Xw.append(fx(kx * xw))
                Yn.append(fy(ky * ys))
                Yw.append(fy(ky * yw))
                index.append(((kx, ky), a, b))
    T = np.zeros((len(times), len(fields), len(index)))
    for m, t in enumerate(times):
        for c, f in enumerate(fields):
            merged = f.merged(float(t))
            for r, (key, a, b) in enumerate(index):
                if key in merged:
                    T[m, c, r] = merged[key][a, b]
    return np.stack(Xn), np.stack(Xw), np.stack(Yn), np.stack(Yw), T
