"""Pins of the FP64 oracle against the paper's numerical results (no GPU).

* second-order convergence on the moving manufactured solution, periodic
  (u and sigma, L2 and Linf), on force-free standing P and S waves, and Dirichlet (u in both norms, sigma in L2), with
  sigma in Linf degrading towards first order under Dirichlet (Sec. 6.1);
* conservation of ||f||_P to round-off on the energy set-up of Sec. 6.2
  (paper: max relative drift about 3.4e-15);
* bounded norm with data on two lattices (Sec. 6.2, Eq. stab_forcing);
* stable at CFL ratio 0.98, divergent within a few hundred steps at 1.01 (Sec. 6.2).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle, Params
from oracle.postprocess import SpaceTimeNorms


def _run_mms(wl):
    o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, wl.dirichlet))
    o.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
    nu, ns = SpaceTimeNorms(wl.dx, wl.dt), SpaceTimeNorms(wl.dx, wl.dt)
    for m in range(wl.steps):
        o.step(wl.body_load(m), wl.wall_data(m))
        out = o.outputs(wl.body_load(m + 1))
        ex = wl.exact_outputs((m + 1) * wl.dt)
        nu.add(out[5:7], ex[5:7])
        ns.add(out[7:10], ex[7:10])
    return (nu.L2rel, nu.Linfrel, ns.L2rel, ns.Linfrel)


def _slopes(a, b):
    return [math.log2(x / y) for x, y in zip(a, b)]


@pytest.mark.parametrize("mat", [(1.1, 0.4), (1.4, 0.1), (0.75, 0.75)])
def test_periodic_second_order(mat):
    errs = [_run_mms(W.periodic_mms(n, *mat, c=2.5, t_final=0.5)) for n in (40, 80)]
    for s in _slopes(*errs):
        assert 1.85 < s < 2.2, (errs, s)


@pytest.mark.parametrize("kind", ["P", "S"])
def test_plane_waves_are_force_free_and_converge_at_second_order(kind):
    """Config 1's forcing-free check: a standing P wave (c_P^2 = cK^2 + cmu^2) or S wave (cmu^2)
    along x solves Eq. teq with b = 0 (the Navier body load of the workload vanishes), and the
    oracle converges to it at second order in u and sigma, L2 and Linf, without any body load."""
    wl = W.plane_wave_periodic(32, 1.5, 0.5, kind, t_final=0.5)
    assert wl.forcing is None
    for t in (0.0, 0.3, 0.77):
        b = W.mms.dense_stack(wl.exact.body_load(), 32, 32, wl.dx, t)
        assert np.abs(b).max() < 1e-13, (t, np.abs(b).max())
    errs = [_run_mms(W.plane_wave_periodic(n, 1.5, 0.5, kind, t_final=0.5)) for n in (32, 64)]
    for s in _slopes(*errs):
        assert 1.85 < s < 2.2, (errs, s)


def test_dirichlet_second_order_u_and_first_order_sigma_linf():
    errs = [_run_mms(W.dirichlet_mms(n, n, 1.1, 0.4, c=2.5, t_final=0.5)) for n in (40, 80, 160)]
    s1, s2 = _slopes(errs[0], errs[1]), _slopes(errs[1], errs[2])
    # u: L2 and Linf second order; sigma: L2 about second order
    for s in (s1[0], s1[1], s2[0], s2[1]):
        assert 1.85 < s < 2.2
    assert s2[2] > 1.75
    # sigma in Linf: a boundary-localised first-order error takes over on fine lattices
    assert 0.8 < s2[3] < 1.5


def test_dirichlet_nonsquare_and_poisson_sweep():
    """Second-order u on a 2:1 rectangle for the Poisson-ratio sweep (cK^2 + cmu^2 = 2)."""
    for nu in (0.0, 0.25, 0.45, 0.49):
        cK2, cmu2 = W.material.poisson_to_speeds(nu)
        errs = [_run_mms(W.dirichlet_mms(2 * n, n, cK2, cmu2, cfl=0.9, t_final=0.25, amp=1e-2,
                                         kx=2 * math.pi, ky=2 * math.pi)) for n in (24, 48)]
        s = _slopes(*errs)
        assert 1.8 < s[0] < 2.3, (nu, errs)


def test_energy_conservation_homogeneous_dirichlet():
    """Sec. 6.2 set-up: 160^2, (cK^2, cmu^2) = (1.1, 0.4), dt = 1/400, b = 0, u_D = 0, t_f = 10 T."""
    wl = W.energy_box(160, 1.1, 0.4, 1.0 / 400.0, 4000)
    o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, True))
    o.init(wl.U0, wl.dU0dx, wl.dU0dy, None, wl.u0)
    e0 = math.sqrt(o.energy())
    drift = 0.0
    for m in range(wl.steps):
        o.step(None, None, track_displacement=False)
        if m % 50 == 49:
            drift = max(drift, abs(math.sqrt(o.energy()) - e0) / e0)
    # the paper prints 3.4e-15; the oracle must be within an order of magnitude of round-off
    assert drift < 3.4e-14, drift


def test_norm_bounded_with_data_on_two_lattices():
    """Sec. 6.2 / Eq. stab_forcing: MMS with b and inhomogeneous u_D, (1.4, 0.1); dx ||f||_P on
    (1/80, 1/200) and (1/160, 1/400) stays bounded and the two evolutions agree."""
    curves = []
    for n in (80, 160):
        wl = W.dirichlet_mms(n, n, 1.4, 0.1, c=2.5, t_final=1.0)
        o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, True))
        o.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
        stride = wl.steps // 20
        cur = [wl.dx * math.sqrt(o.energy())]
        for m in range(wl.steps):
            o.step(wl.body_load(m), wl.wall_data(m), track_displacement=False)
            if (m + 1) % stride == 0:
                cur.append(wl.dx * math.sqrt(o.energy()))
        curves.append(np.array(cur[:21]))
    a, b = curves
    assert np.max(a) < 5 * a[0] and np.max(b) < 5 * b[0]
    assert np.max(np.abs(a - b) / b) < 0.05


def test_stability_threshold():
    """(1.1, 0.4) at dx = 1/160, dt = 1/400 (ratio 0.98) stays bounded; (1.2, 0.4) (ratio 1.01)
    diverges within a few hundred steps (Sec. 6.2)."""
    # beyond the bound some k_ij is indefinite, so growth is measured by max |f|
    def growth(cK2, cmu2, steps):
        wl = W.periodic_mms(160, cK2, cmu2, c=2.5, steps=steps)
        o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, False))
        o.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
        f0 = float(np.max(np.abs(o.f)))
        for m in range(steps):
            o.step(wl.body_load(m), None, track_displacement=False)
        return float(np.max(np.abs(o.f))) / f0
    assert growth(1.1, 0.4, 600) < 3.0
    assert growth(1.2, 0.4, 600) > 1e6


def test_omega_below_two_is_first_order():
    """Sec. 4.1: second-order consistency needs omega = 2; with omega < 2 the scheme is
    dissipative and the displacement error converges at first order."""
    def err(n, omega):
        wl = W.periodic_mms(n, 1.1, 0.4, c=2.5, t_final=0.5)
        o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, False, omega=omega))
        o.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
        nrm = SpaceTimeNorms(wl.dx, wl.dt)
        for m in range(wl.steps):
            o.step(wl.body_load(m), None)
            nrm.add(o.outputs(wl.body_load(m + 1))[5:7], wl.exact_outputs((m + 1) * wl.dt)[5:7])
        return nrm.L2rel
    e = [err(n, 1.6) for n in (40, 80)]
    assert 0.85 < math.log2(e[0] / e[1]) < 1.2, e
