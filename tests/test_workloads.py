"""Pins of the input generators (no GPU): manufactured-solution derivatives and
body load against finite differences, separable tables against dense values,
GRF statistics and spectral derivatives, material mapping."""
import math

import numpy as np

import workloads as W
from workloads import mms


def _fd4(f, h):
    return (-f(2 * h) + 8 * f(h) - 8 * f(-h) + f(-2 * h)) / (12 * h)


def test_mms_derivatives_and_body_load_against_finite_differences():
    cK, cmu = math.sqrt(1.1), math.sqrt(0.4)
    sol = mms.paper_moving_solution(cK, cmu)
    x = np.array([0.13, 0.71, 0.42])
    y = np.array([0.57, 0.08, 0.93])
    t = 0.37
    u = sol.displacement()

    def val(comp, dx=0.0, dy=0.0, dt=0.0):
        return u[comp].points(x + dx, y + dy, t + dt)

    h = 1e-3
    for c in range(2):
        np.testing.assert_allclose(sol.D(c, 1, 0, 0).points(x, y, t), _fd4(lambda s: val(c, dx=s), h), atol=1e-6)
        np.testing.assert_allclose(sol.D(c, 0, 1, 0).points(x, y, t), _fd4(lambda s: val(c, dy=s), h), atol=1e-6)
        np.testing.assert_allclose(sol.D(c, 0, 0, 1).points(x, y, t), _fd4(lambda s: val(c, dt=s), h), atol=1e-6)
    # body load from the Navier form against second differences of u
    h2 = 1e-3

    def d2(c, ax):
        def sh(s):
            kw = {ax: s}
            return val(c, **kw)
        return (-sh(2 * h2) + 16 * sh(h2) - 30 * sh(0) + 16 * sh(-h2) - sh(-2 * h2)) / (12 * h2 * h2)

    def dxy(c):
        return (val(c, dx=h2, dy=h2) - val(c, dx=h2, dy=-h2) - val(c, dx=-h2, dy=h2) + val(c, dx=-h2, dy=-h2)) / (4 * h2 * h2)

    bx = d2(0, "dt") - cK ** 2 * (d2(0, "dx") + dxy(1)) - cmu ** 2 * (d2(0, "dx") + d2(0, "dy"))
    by = d2(1, "dt") - cK ** 2 * (dxy(0) + d2(1, "dy")) - cmu ** 2 * (d2(1, "dx") + d2(1, "dy"))
    b = sol.body_load()
    np.testing.assert_allclose(b[0].points(x, y, t), bx, atol=2e-4 * np.max(np.abs(bx)))
    np.testing.assert_allclose(b[1].points(x, y, t), by, atol=2e-4 * np.max(np.abs(by)))


def test_separable_tables_reproduce_dense_fields():
    sol = mms.paper_moving_solution(1.0, 0.5)
    nx, ny, dx = 7, 5, 0.13
    times = [0.0, 0.21, 0.5]
    X, Y, T = mms.separable_tables(sol.body_load(), nx, ny, dx, times)
    for m, t in enumerate(times):
        dense = mms.dense_stack(sol.body_load(), nx, ny, dx, t)
        np.testing.assert_allclose(mms.eval_tables(X, Y, T[m]), dense, atol=1e-10)


def test_plane_wave_solves_homogeneous_equation():
    for kind in ("P", "S"):
        sol = mms.plane_wave(1.2, 0.7, kind)
        b = mms.dense_stack(sol.body_load(), 9, 4, 0.1, 0.3)
        assert np.max(np.abs(b)) < 1e-12


def test_grf_statistics_and_spectral_gradient():
    f = W.grf.gaussian_random_field(256, 128, 8.0, 1e-3, 7)
    assert abs(float(np.std(f)) - 1e-3) < 1e-12
    assert abs(float(np.mean(f))) < 1e-15
    gx, gy = W.grf.spectral_gradient(f, 0.5)
    fdx = (np.roll(f, -1, 1) - np.roll(f, 1, 1)) / (2 * 0.5)
    fdy = (np.roll(f, -1, 0) - np.roll(f, 1, 0)) / (2 * 0.5)
    assert np.max(np.abs(gx - fdx)) < 0.05 * np.max(np.abs(gx))
    assert np.max(np.abs(gy - fdy)) < 0.05 * np.max(np.abs(gy))
    # correlation length: the autocorrelation at lag ell is exp(-1/2)
    ac = np.fft.irfft2(np.abs(np.fft.rfft2(f)) ** 2, s=f.shape)
    assert abs(ac[0, 8] / ac[0, 0] - math.exp(-0.5)) < 0.1


def test_material_mapping():
    assert W.material.lame_to_speeds(1.0, 0.5) == (1.5, 0.5)
    for nu in (0.0, 0.25, 0.45, 0.49):
        cK2, cmu2 = W.material.poisson_to_speeds(nu)
        assert abs(cK2 + cmu2 - 2.0) < 1e-15
        lam = cK2 - cmu2
        assert abs(lam / (2 * (lam + cmu2)) - nu) < 1e-12
    c = W.material.lattice_speed(1.5, 0.5, 0.9)
    assert abs(W.material.cfl_ratio(1.5, 0.5, c) - 0.9) < 1e-15


def test_batch_spec_shape():
    spec = W.batch_spec()
    assert len(spec) == 512
    for i, s in enumerate(spec):
        short, long = min(s.nx, s.ny), max(s.nx, s.ny)
        assert 64 <= short <= 1024 and long <= 4 * short + 1
        assert s.dirichlet == (i % 2 == 1)
        assert 0.0 <= s.nu <= 0.49
