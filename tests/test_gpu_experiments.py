"""The paper's experiments through the CUDA library at sizes a test can afford:
Dirichlet convergence (second order for u in L2 and Linf and sigma in L2, first
order creeping into sigma Linf) for the Poisson-ratio sweep, and a 10^5-step run
on 512 x 256 with homogeneous data whose weighted norm stays constant (Sec. 6)."""
import pytest

from paper_2408_01081_gb300 import experiments as X

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nu", [0.0, 0.25, 0.45, 0.49])
def test_dirichlet_convergence_fp64(lbm, nu):
    res = X.dirichlet_convergence((32, 64, 128, 256), nus=(nu,), log=None)[str(nu)]
    for o in res["order_u_L2"] + res["order_u_Linf"]:
        assert 1.75 < o < 2.4, res
    # an O(dx) error in a boundary layer a few cells wide bounds the L2 order of sigma at 1.5
    # asymptotically (the interior converges at second order); Sec. 6.1's second order is the
    # pre-asymptotic range
    for o in res["order_sigma_L2"]:
        assert o > 1.45, res


def test_dirichlet_separable_wall_tables_match_dense(lbm):
    """The device expansion of separable wall data equals the per-step dense table."""
    import math
    import numpy as np
    import workloads as W
    from workloads import mms
    from tests.helpers import gpu_lattice
    wl = W.dirichlet_mms(40, 20, 1.1, 0.4, cfl=0.9, steps=30)
    a = gpu_lattice(lbm, wl)
    a.step(wl.steps)
    ra = a.moments()
    b = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=True, storage="f64")
    b.set_forcing(*wl.forcing)
    b.set_dirichlet_separable(*mms.separable_wall_tables(wl.exact.velocity(), wl.nx, wl.ny, wl.dx,
                                                         (np.arange(wl.steps) + 0.5) * wl.dt))
    b.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
    b.step(wl.steps)
    np.testing.assert_allclose(b.moments(), ra, rtol=0, atol=1e-13 * np.max(np.abs(ra)))
    del math


def test_long_run_energy_fp64(lbm):
    r = X.long_run(steps=100_000, nx=512, ny=256, every=10_000)
    assert r["finite"] and r["max_rel_energy_drift"] < 1e-12, r


def test_precision_errors_ordering(lbm):
    """Storage formats against the FP64 run on a small lattice: FP32 within its 1e-5 bar,
    FP16 and moment-space formats below BF16 (more mantissa bits or fewer rounded values),
    block floating point below FP16 deviations (15-bit mantissas sharing an exponent)."""
    res = X.precision_errors(n=256, steps=300, ell=16.0, every=100)
    assert res["checkpoints"] == [100, 200, 300]
    r = res["formats"]
    worst = {s: max(v["rel_l2_vs_f64"][300].values()) for s, v in r.items() if s != "f64"}
    assert worst["f32"] < 1e-5, worst
    assert worst["ms_f16"] < worst["f16"] < worst["bf16"], worst
    assert worst["ms_bf16"] < worst["bf16"], worst
    assert worst["ms_bfp"] < worst["ms_f16"], worst
