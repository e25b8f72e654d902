"""Matrix form of one step of the scheme (Sec. 5.1), for tiny lattices.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

This is a second, independent statement of the same scheme: the C oracle
evaluates Eq. feq through the fluxes Phi_x, Phi_y, while this module assembles
the collision from the paper's matrices A_x, A_y and g_ij (Eq. stability_linear),
the streaming from an explicit permutation and the Dirichlet rule from D and
S_ij (Eqs. bc_ansatz-bc_q).  It is used to build the full one-step operator on
a 4x4 lattice (a 320x320 matrix plus an affine part) and the symmetrizer blocks
k_ij = g_ij^{-1} (Eq. def_symmetrizer).

State vector ordering: f[d, k, y, x] flattened (the C oracle's layout).
"""
from __future__ import annotations

import numpy as np

VEL = [(1, 0), (0, 1), (-1, 0), (0, -1)]  # Eq. index_vel
D_MAT = np.diag([-1.0, -1.0, 1.0, 1.0, 1.0])  # Eq. bc_d


def A_x(cK: float, cmu: float) -> np.ndarray:
    """Eq. stability_linear, A_x."""
    A = np.zeros((5, 5))
    A[0, 2] = A[2, 0] = cK
    A[0, 3] = A[3, 0] = cmu
    A[1, 4] = A[4, 1] = cmu
    return A


def A_y(cK: float, cmu: float) -> np.ndarray:
    """Eq. stability_linear, A_y."""
    A = np.zeros((5, 5))
    A[0, 4] = A[4, 0] = cmu
    A[1, 2] = A[2, 1] = cK
    A[1, 3] = A[3, 1] = -cmu
    return A


def g_block(d: int, cK: float, cmu: float, c: float) -> np.ndarray:
    """g_ij = 1/4 I + 1/(2c) (i A_x + j A_y)."""
    i, j = VEL[d]
    return 0.25 * np.eye(5) + (1.0 / (2.0 * c)) * (i * A_x(cK, cmu) + j * A_y(cK, cmu))


def G_matrix(cK: float, cmu: float, c: float) -> np.ndarray:
    """G = [g_10; g_01; g_-10; g_0-1] [I I I I] (20x20), population vector [f_10; f_01; f_-10; f_0-1]."""
    col = np.vstack([g_block(d, cK, cmu, c) for d in range(4)])
    row = np.hstack([np.eye(5)] * 4)
    return col @ row


def symmetrizer_blocks(cK: float, cmu: float, c: float) -> np.ndarray:
    """k_ij = g_ij^{-1}, shape [4, 5, 5] (Eq. def_symmetrizer)."""
    return np.stack([np.linalg.inv(g_block(d, cK, cmu, c)) for d in range(4)])


def K_matrix(cK: float, cmu: float, c: float) -> np.ndarray:
    k = symmetrizer_blocks(cK, cmu, c)
    K = np.zeros((20, 20))
    for d in range(4):
        K[5 * d:5 * d + 5, 5 * d:5 * d + 5] = k[d]
    return K


def S_matrix(d: int, cK: float, cmu: float, c: float) -> np.ndarray:
    """5x2 matrix mapping d/dt u_D to S_ij (Eq. bc_s).

    Rows 2..4 carry the factor 1/c that the equilibrium difference
    f^eq_ij - f^eq_{-i,-j} = (i Phi_x + j Phi_y)/c implies.
    """
    i, j = VEL[d]
    return np.array([
        [0.5, 0.0],
        [0.0, 0.5],
        [i * cK / c, j * cK / c],
        [i * cmu / c, -j * cmu / c],
        [j * cmu / c, i * cmu / c],
    ])


def _flat(d, k, y, x, nx, ny):
    return ((d * 5 + k) * ny + y) * nx + x


def one_step_operator(nx: int, ny: int, cK: float, cmu: float, c: float, dt: float,
                      dirichlet: bool, omega: float = 2.0, W: float = 0.125):
    """Return (M, F, Sg) with f(t+dt) = M f(t) + F b(t) + Sg g(t+dt/2).

    b is the flattened body load [2, ny, nx]; g the wall data [2, 2(nx+ny)].
    """
    n = 20 * nx * ny
    G = G_matrix(cK, cmu, c)
    C = np.eye(20) + omega * (G - np.eye(20))                 # Eq. collision_vector
    # forcing enters through U^num = sum f + dt/2 B and the W term (Eq. lbe)
    gcol = np.vstack([g_block(d, cK, cmu, c) for d in range(4)])   # f^eq = G f + g (dt/2) B
    Bsel = np.zeros((5, 2))
    Bsel[0, 0] = Bsel[1, 1] = 1.0
    Fnode = omega * gcol @ Bsel * (0.5 * dt) + dt * (2.0 - omega) * W * np.vstack([Bsel] * 4)

    # post-collision operator over the lattice (node-local blocks)
    Cl = np.zeros((n, n))
    Fl = np.zeros((n, 2 * nx * ny))
    for y in range(ny):
        for x in range(nx):
            rows = [_flat(d, k, y, x, nx, ny) for d in range(4) for k in range(5)]
            Cl[np.ix_(rows, rows)] = C
            bcols = [(comp * ny + y) * nx + x for comp in range(2)]
            Fl[np.ix_(rows, bcols)] = Fnode

    # streaming (+ boundary) as a matrix acting on post-collision values
    P = np.zeros((n, n))
    nw = 2 * (nx + ny)
    Sg = np.zeros((n, 2 * nw))
    for y in range(ny):
        for x in range(nx):
            for d, (i, j) in enumerate(VEL):
                xs, ys = x - i, y - j
                inside = 0 <= xs < nx and 0 <= ys < ny
                if inside or not dirichlet:
                    xs %= nx
                    ys %= ny
                    for k in range(5):
                        P[_flat(d, k, y, x, nx, ny), _flat(d, k, ys, xs, nx, ny)] = 1.0
                else:
                    dbar = (d + 2) % 4
                    for k in range(5):
                        P[_flat(d, k, y, x, nx, ny), _flat(dbar, k, y, x, nx, ny)] = D_MAT[k, k]
                    if d == 0:
                        w = y
                    elif d == 2:
                        w = ny + y
                    elif d == 1:
                        w = 2 * ny + x
                    else:
                        w = 2 * ny + nx + x
                    S = S_matrix(d, cK, cmu, c)
                    for k in range(5):
                        Sg[_flat(d, k, y, x, nx, ny), w] = S[k, 0]
                        Sg[_flat(d, k, y, x, nx, ny), nw + w] = S[k, 1]
    return P @ Cl, P @ Fl, Sg


def lattice_K(nx: int, ny: int, cK: float, cmu: float, c: float) -> np.ndarray:
    """Block-diagonal weight of ||f||_P^2 over the whole lattice, in the flat layout."""
    k = symmetrizer_blocks(cK, cmu, c)
    n = 20 * nx * ny
    K = np.zeros((n, n))
    for y in range(ny):
        for x in range(nx):
            for d in range(4):
                rows = [_flat(d, kk, y, x, nx, ny) for kk in range(5)]
                K[np.ix_(rows, rows)] = k[d]
    return K
