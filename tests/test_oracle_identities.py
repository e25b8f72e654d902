"""Pins of the FP64 oracle against exact statements of the paper (no GPU).

Each test checks the C oracle against something other than its own formula:
the moment conditions (Eq. cond_eq), the matrix form of Sec. 5.1, the
symmetrizer identities of Sec. 5.2/5.3, closed forms and symmetries.
"""
import math

import numpy as np
import pytest

from oracle import Oracle, Params
from oracle import matrix_form as mf

RNG = np.random.default_rng(12345)


def _oracle(nx, ny, cK=1.1 ** 0.5, cmu=0.4 ** 0.5, c=2.5, dirichlet=False, dx=0.1, omega=2.0):
    return Oracle(Params(nx, ny, dx, dx / c, cK, cmu, dirichlet, omega=omega))


def test_equilibrium_satisfies_moment_conditions():
    """Eq. feq fulfils every line of Eq. cond_eq (fluxes from A_x, A_y of Eq. stability_linear)."""
    for _ in range(20):
        cK, cmu, c = RNG.uniform(0.1, 1.5), RNG.uniform(0.0, 1.0), RNG.uniform(3.5, 6.0)
        o = _oracle(1, 1, cK, cmu, c)
        U = RNG.standard_normal(5)
        feq = np.stack([o.equilibrium(U, d) for d in range(4)])
        I = np.array([v[0] for v in mf.VEL], dtype=float)
        J = np.array([v[1] for v in mf.VEL], dtype=float)
        np.testing.assert_allclose(feq.sum(0), U, atol=1e-14)
        np.testing.assert_allclose((c * I[:, None] * feq).sum(0), mf.A_x(cK, cmu) @ U, atol=1e-13)
        np.testing.assert_allclose((c * J[:, None] * feq).sum(0), mf.A_y(cK, cmu) @ U, atol=1e-13)
        np.testing.assert_allclose((c * c * (I ** 2 - J ** 2)[:, None] * feq).sum(0), 0.0, atol=1e-12)


def _collision_from_oracle(o):
    """One step on a 1x1 periodic lattice streams every population back to its node,
    so the step is exactly the node collision matrix."""
    C = np.zeros((20, 20))
    for col in range(20):
        f = np.zeros((4, 5, 1, 1))
        f.reshape(20)[col] = 1.0
        o.set_state(f)
        o.step(track_displacement=False)
        C[:, col] = o.f.reshape(20)
    return C


def test_collision_matches_matrix_form_and_is_reflection():
    cK, cmu, c = 1.1 ** 0.5, 0.4 ** 0.5, 2.5
    o = _oracle(1, 1, cK, cmu, c)
    C = _collision_from_oracle(o)
    G = mf.G_matrix(cK, cmu, c)
    np.testing.assert_allclose(C, 2 * G - np.eye(20), atol=1e-15)
    # G is a projector with spectrum {0, 1} (Sec. 5.2), so 2G - I is an involution
    np.testing.assert_allclose(G @ G, G, atol=1e-15)
    np.testing.assert_allclose(C @ C, np.eye(20), atol=1e-14)
    ev = np.linalg.eigvals(G)
    assert np.all(np.minimum(np.abs(ev), np.abs(ev - 1)) < 1e-12)


def test_collision_is_isometry_in_weighted_norm():
    """K G symmetric and (2G - I)^T K (2G - I) = K with K = diag(g_ij^-1) (Eq. def_symmetrizer)."""
    for cK, cmu, c in [(1.1 ** 0.5, 0.4 ** 0.5, 2.5), (1.0, 0.3, 3.0), (1.2, 0.0, 2.5)]:
        C = _collision_from_oracle(_oracle(1, 1, cK, cmu, c))
        K = mf.K_matrix(cK, cmu, c)
        np.testing.assert_allclose(K @ mf.G_matrix(cK, cmu, c), (K @ mf.G_matrix(cK, cmu, c)).T, atol=1e-13)
        np.testing.assert_allclose(C.T @ K @ C, K, atol=1e-12)


def test_bounce_back_symmetrizer_identity():
    """k_{-i,-j} = D^T k_ij D (Sec. 5.3)."""
    k = mf.symmetrizer_blocks(1.1 ** 0.5, 0.4 ** 0.5, 2.5)
    D = mf.D_MAT
    for d in range(4):
        np.testing.assert_allclose(D.T @ k[d] @ D, k[(d + 2) % 4], atol=1e-13)


def test_cfl_condition_is_positive_definiteness():
    """All g_ij SPD iff 2 sqrt(cK^2 + cmu^2) < c (Eq. stab_cond)."""
    for _ in range(200):
        cK, cmu, c = RNG.uniform(0.05, 2), RNG.uniform(0.0, 2), RNG.uniform(0.5, 6)
        spd = all(np.linalg.eigvalsh(mf.g_block(d, cK, cmu, c)).min() > 0 for d in range(4))
        cond = 2 * math.sqrt(cK * cK + cmu * cmu) < c
        if abs(2 * math.sqrt(cK * cK + cmu * cmu) - c) > 1e-9:
            assert spd == cond


@pytest.mark.parametrize("dirichlet", [False, True])
def test_one_step_equals_brute_force_operator_4x4(dirichlet):
    """Whole step on a 4x4 lattice == the 320x320 operator assembled from G, the
    shift permutation, D and S (Sec. 5.1, Eqs. bc_ansatz-bc_q), with random body
    load and wall data."""
    nx = ny = 4
    cK, cmu, c, dx = 1.1 ** 0.5, 0.4 ** 0.5, 2.5, 0.25
    dt = dx / c
    o = _oracle(nx, ny, cK, cmu, c, dirichlet, dx)
    M, F, Sg = mf.one_step_operator(nx, ny, cK, cmu, c, dt, dirichlet)
    for _ in range(3):
        f = RNG.standard_normal((4, 5, ny, nx))
        B = RNG.standard_normal((2, ny, nx))
        g = RNG.standard_normal((2, 2 * (nx + ny)))
        o.set_state(f)
        o.step(B, g if dirichlet else None, track_displacement=False)
        expect = M @ f.reshape(-1) + F @ B.reshape(-1) + (Sg @ g.reshape(-1) if dirichlet else 0)
        np.testing.assert_allclose(o.f.reshape(-1), expect, atol=1e-13, rtol=0)


@pytest.mark.parametrize("dirichlet", [False, True])
def test_homogeneous_step_is_isometry(dirichlet):
    """M^T K M = K for b = 0 and homogeneous data (Props. 3 and 4)."""
    nx = ny = 4
    cK, cmu, c, dx = 1.1 ** 0.5, 0.4 ** 0.5, 2.5, 0.25
    M, _, _ = mf.one_step_operator(nx, ny, cK, cmu, c, dx / c, dirichlet)
    K = mf.lattice_K(nx, ny, cK, cmu, c)
    np.testing.assert_allclose(M.T @ K @ M, K, atol=1e-12)


def test_general_omega_matches_matrix_form():
    """The omega != 2 variant (first-order control, forcing weight W = 1/8) against the matrix form."""
    nx, ny, cK, cmu, c, dx = 3, 4, 1.0, 0.5, 3.0, 0.2
    o = _oracle(nx, ny, cK, cmu, c, False, dx, omega=1.6)
    M, F, _ = mf.one_step_operator(nx, ny, cK, cmu, c, dx / c, False, omega=1.6)
    f = RNG.standard_normal((4, 5, ny, nx))
    B = RNG.standard_normal((2, ny, nx))
    o.set_state(f)
    o.step(B, None, track_displacement=False)
    np.testing.assert_allclose(o.f.reshape(-1), M @ f.reshape(-1) + F @ B.reshape(-1), atol=1e-13)
    # the W weight makes the zeroth moment gain exactly dt * B per step
    o.set_state(f)
    U_before = o.moments(B)
    o.step(B, None, track_displacement=False)
    s_after = o.f.sum(axis=0)
    np.testing.assert_allclose(s_after[0:2].sum(axis=(1, 2)), (U_before[0:2] + 0.5 * o.p.dt * B).sum(axis=(1, 2)),
                               atol=1e-12)


def test_fourier_mode_closed_form():
    """Periodic, b = 0: a single Fourier mode evolves as (E(kappa) (2G - I))^n (derived from
    Eqs. collision_vector and streaming)."""
    nx, ny, cK, cmu, c, dx = 12, 10, 1.0, 0.6, 3.2, 0.1
    o = _oracle(nx, ny, cK, cmu, c, False, dx)
    kap = np.array([2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny])
    fhat = RNG.standard_normal(20) + 1j * RNG.standard_normal(20)
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    phase = np.exp(1j * (kap[0] * X + kap[1] * Y))
    f0 = np.real(fhat.reshape(4, 5)[:, :, None, None] * phase[None, None])
    o.set_state(np.ascontiguousarray(f0))
    nsteps = 37
    for _ in range(nsteps):
        o.step(track_displacement=False)
    E = np.zeros((20, 20), dtype=complex)
    for d, (i, j) in enumerate(mf.VEL):
        E[5 * d:5 * d + 5, 5 * d:5 * d + 5] = np.exp(-1j * (kap[0] * i + kap[1] * j)) * np.eye(5)
    Op = E @ (2 * mf.G_matrix(cK, cmu, c) - np.eye(20))
    fn = np.linalg.matrix_power(Op, nsteps) @ fhat
    expect = np.real(fn.reshape(4, 5)[:, :, None, None] * phase[None, None])
    np.testing.assert_allclose(o.f, expect, atol=1e-12)


def _run(o, f, n):
    o.set_state(f)
    for _ in range(n):
        o.step(track_displacement=False)
    return o.f.copy()


def test_mirror_and_transpose_symmetries():
    """Mirror x -> -x (P = diag(-1,1,1,1,-1), f'_{i,j} = P f_{-i,j}) and transpose
    x <-> y (Q: v_x <-> v_y, j_d -> -j_d, f'_{i,j} = Q f_{j,i}) commute with a periodic step."""
    n, cK, cmu, c, dx = 8, 1.1, 0.5, 3.0, 0.125
    o = _oracle(n, n, cK, cmu, c, False, dx)
    f = RNG.standard_normal((4, 5, n, n))
    P = np.array([-1, 1, 1, 1, -1.0])

    def mirror(g):
        out = np.empty_like(g)
        for d, (i, j) in enumerate(mf.VEL):
            src = mf.VEL.index((-i, j))
            out[d] = P[:, None, None] * g[src][:, :, ::-1]
        return np.ascontiguousarray(out)

    def transpose(g):
        out = np.empty_like(g)
        for d, (i, j) in enumerate(mf.VEL):
            src = g[mf.VEL.index((j, i))]
            t = np.transpose(src, (0, 2, 1))
            out[d] = np.stack([t[1], t[0], t[2], -t[3], t[4]])
        return np.ascontiguousarray(out)

    np.testing.assert_allclose(_run(o, mirror(f), 5), mirror(_run(o, f, 5)), atol=1e-13)
    np.testing.assert_allclose(_run(o, transpose(f), 5), transpose(_run(o, f, 5)), atol=1e-13)


def test_periodic_total_moment_conserved():
    """sum_x U is invariant for periodic lattices without body load (collision keeps U, streaming permutes)."""
    o = _oracle(7, 5)
    f = RNG.standard_normal((4, 5, 5, 7))
    o.set_state(f)
    s0 = o.moments().sum(axis=(1, 2))
    for _ in range(20):
        o.step(track_displacement=False)
    np.testing.assert_allclose(o.moments().sum(axis=(1, 2)), s0, atol=1e-12)


def test_init_zeroth_moment():
    """Eq. ic_second gives sum_ij f_ij(x, 0) = U0 - dt/2 B (the i, j and 2i^2-1 weights sum to 0)."""
    nx, ny = 6, 5
    o = _oracle(nx, ny)
    U0, dUx, dUy = (RNG.standard_normal((5, ny, nx)) for _ in range(3))
    B0 = RNG.standard_normal((2, ny, nx))
    o.init(U0, dUx, dUy, B0)
    expect = U0.copy()
    expect[0:2] -= 0.5 * o.p.dt * B0
    np.testing.assert_allclose(o.f.sum(axis=0), expect, atol=1e-14)
    # and U^num(0) = U0 exactly, so u^num(0) = u0 with u* = u0 - dt/2 v0
    np.testing.assert_allclose(o.moments(B0), U0, atol=1e-14)


def test_init_matches_asymptotic_first_order_form():
    """Eq. ic_second equals f^(0) + dt f^(1) of Eqs. asymp_ic0 / asymp_ic1 with U^(1) = 0 and
    d_t U0 = B - d_x Phi_x(U0) - d_y Phi_y(U0) (Eq. eqpde1), written here in matrix form."""
    cK, cmu, c, dx = 1.0, 0.5, 3.0, 0.1
    dt = dx / c
    o = _oracle(1, 1, cK, cmu, c, False, dx)
    Ax, Ay = mf.A_x(cK, cmu), mf.A_y(cK, cmu)
    U0, Ux, Uy = (RNG.standard_normal(5) for _ in range(3))
    B = np.zeros(5)
    B[0:2] = RNG.standard_normal(2)
    o.init(U0.reshape(5, 1, 1), Ux.reshape(5, 1, 1), Uy.reshape(5, 1, 1), B[0:2].reshape(2, 1, 1))
    dtU = B - Ax @ Ux - Ay @ Uy
    for d, (i, j) in enumerate(mf.VEL):
        g = mf.g_block(d, cK, cmu, c)
        f0 = g @ U0
        f1 = -0.5 * (g @ dtU) - 0.5 * c * (i * (g @ Ux) + j * (g @ Uy))
        np.testing.assert_allclose(o.f[d, :, 0, 0], f0 + dt * f1, atol=1e-14)


def test_dirichlet_rule_keeps_rigid_translation():
    """A uniform velocity g (u = g t, b = 0) is an exact equilibrium state; with the wall
    data d/dt u_D = g the boundary rule must reproduce the equilibrium populations, which
    requires S_ij = (1/2 g, (i Phi_x + j Phi_y)(g-state) / c) on the j rows."""
    nx, ny, cK, cmu, c, dx = 6, 5, 1.1 ** 0.5, 0.4 ** 0.5, 2.5, 0.2
    o = _oracle(nx, ny, cK, cmu, c, True, dx)
    gv = np.array([0.3, -0.7])
    U0 = np.zeros((5, ny, nx))
    U0[0], U0[1] = gv[0], gv[1]
    z = np.zeros((5, ny, nx))
    o.init(U0, z, z)
    wall = np.repeat(gv[:, None], 2 * (nx + ny), axis=1)
    for _ in range(25):
        o.step(None, wall)
    np.testing.assert_allclose(o.moments(), U0, atol=1e-14)
