"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: 1e-12 relative L2 per output field for the FP64 path (the bound the
FP64 fused kernel is held to); the reduced-precision formats are compared with
their own stated bounds.  Sizes span several thread blocks and ragged row ends.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle, Params
from oracle import matrix_form as mf
from oracle.postprocess import rel_l2

from .helpers import field_errors, gpu_lattice, oracle_run

pytestmark = pytest.mark.gpu
TOL64 = 1e-12


def _config1(steps=1000):
    """Periodic 64x64, lambda = 1, mu = 0.5 (cK^2 = 1.5, cmu^2 = 0.5), 0.9 of the CFL bound,
    one wavelength per side, amplitude 1e-2."""
    return W.periodic_mms(64, 1.5, 0.5, cfl=0.9, steps=steps, amp=1e-2, kx=2 * math.pi, ky=2 * math.pi)


def test_config1_periodic_64_fp64_matches_oracle(lbm):
    wl = _config1()
    _, ref = oracle_run(wl)
    lat = gpu_lattice(lbm, wl)
    lat.step(wl.steps)
    out = lat.moments()
    errs = field_errors(out, ref)
    assert max(errs) < TOL64, errs
    # and the solution itself is second-order accurate against the manufactured one
    ex = wl.exact_outputs(wl.steps * wl.dt)
    assert rel_l2(out[5:7], ex[5:7]) < 2e-2


@pytest.mark.parametrize("kind", ["P", "S"])
def test_config1_force_free_plane_waves_fp64(lbm, kind):
    """Config 1's forcing-free check on the periodic 64^2 lattice, 1000 steps: a standing P or S
    wave with b = 0, so the default FP64 step (fixed-point node update) runs every step; it equals
    the oracle within the FP64 tolerance, and u stays within the scheme's second-order error of
    the exact wave."""
    wl = W.plane_wave_periodic(64, 1.5, 0.5, kind, steps=1000)
    _, ref = oracle_run(wl)
    lat = gpu_lattice(lbm, wl)
    lat.step(wl.steps)
    out = lat.moments()
    lat.close()
    errs = field_errors(out, ref)
    assert max(errs) < TOL64, errs
    ex = wl.exact_outputs(wl.steps * wl.dt)
    assert rel_l2(out[5:7], ex[5:7]) < 2e-3          # the oracle: 6.7e-4 (P wave)


@pytest.mark.parametrize("nx,ny", [(48, 24), (37, 23), (1100, 9)])
def test_dirichlet_mms_fp64_matches_oracle(lbm, nx, ny):
    wl = W.dirichlet_mms(nx, ny, 1.1, 0.4, cfl=0.9, steps=60, height=1.0)
    _, ref = oracle_run(wl)
    lat = gpu_lattice(lbm, wl)
    lat.step(wl.steps)
    errs = field_errors(lat.moments(), ref)
    assert max(errs) < TOL64, errs


@pytest.mark.parametrize("nx,ny", [(2, 2), (3, 5), (67, 45), (1031, 7), (520, 3)])
def test_periodic_ragged_sizes_fp64(lbm, nx, ny):
    rng = np.random.default_rng(nx * 100 + ny)
    wl = W.periodic_mms(max(nx, ny), 1.5, 0.5, steps=0)
    o = Oracle(Params(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, False))
    f = rng.standard_normal((4, 5, ny, nx))
    us = rng.standard_normal((2, ny, nx))
    o.set_state(f, us)
    lat = lbm.Lattice(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, dirichlet=False, storage="f64")
    lat.set_populations(f, us)
    for _ in range(7):
        o.step()
    lat.step(7)
    g, gu = lat.populations()
    np.testing.assert_allclose(g, o.f, rtol=0, atol=1e-13 * np.max(np.abs(o.f)))
    np.testing.assert_allclose(gu, o.ustar, rtol=0, atol=1e-13 * np.max(np.abs(o.ustar)))
    del wl


@pytest.mark.parametrize("dirichlet", [False, True])
def test_one_step_4x4_equals_brute_force_operator(lbm, dirichlet):
    """One GPU step on 4x4 == the 320x320 operator from G, the shift, D and S (Sec. 5.1)."""
    nx = ny = 4
    cK, cmu, c, dx = math.sqrt(1.1), math.sqrt(0.4), 2.5, 0.25
    dt = dx / c
    M, F, Sg = mf.one_step_operator(nx, ny, cK, cmu, c, dt, dirichlet)
    rng = np.random.default_rng(7)
    f = rng.standard_normal((4, 5, ny, nx))
    lat = lbm.Lattice(nx, ny, dx, dt, cK, cmu, dirichlet=dirichlet, storage="f64")
    expect = M @ f.reshape(-1)
    if dirichlet:
        g = rng.standard_normal((1, 2, 2 * (nx + ny)))
        lat.set_dirichlet(g)
        expect = expect + Sg @ g[0].reshape(-1)
    lat.set_populations(f)
    lat.step(1)
    out, _ = lat.populations()
    np.testing.assert_allclose(out.reshape(-1), expect, atol=1e-13, rtol=0)
    del F


def test_forcing_tables_match_oracle_4x4(lbm):
    """Body load enters through U^num (Eq. cond_eq): one step with random separable b."""
    nx = ny = 4
    cK, cmu, c, dx = math.sqrt(1.1), math.sqrt(0.4), 2.5, 0.25
    dt = dx / c
    M, F, _ = mf.one_step_operator(nx, ny, cK, cmu, c, dt, False)
    rng = np.random.default_rng(11)
    R = 3
    X, Y, T = rng.standard_normal((R, nx)), rng.standard_normal((R, ny)), rng.standard_normal((4, 2, R))
    lat = lbm.Lattice(nx, ny, dx, dt, cK, cmu, storage="f64")
    lat.set_forcing(X, Y, T)
    f = rng.standard_normal((4, 5, ny, nx))
    lat.set_populations(f, m=1)
    lat.step(1)
    out, _ = lat.populations()
    b1 = np.einsum("rx,ry,cr->cyx", X, Y, T[1])
    np.testing.assert_allclose(out.reshape(-1), M @ f.reshape(-1) + F @ b1.reshape(-1), atol=1e-13)


def test_energy_matches_oracle_and_is_conserved(lbm):
    """||f||_P on the GPU equals the oracle's; homogeneous Dirichlet, b = 0: conserved
    to round-off over 4000 steps (Sec. 6.2 set-up, paper: 3.4e-15)."""
    wl = W.energy_box(160, 1.1, 0.4, 1.0 / 400.0, 4000)
    o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, True))
    o.init(wl.U0, wl.dU0dx, wl.dU0dy, None, wl.u0)
    lat = gpu_lattice(lbm, wl, track=False)
    e0 = lat.energy()
    assert abs(e0 - o.energy()) < 1e-13 * o.energy()
    drift = 0.0
    for _ in range(40):
        lat.step(100)
        drift = max(drift, abs(math.sqrt(lat.energy()) - math.sqrt(e0)) / math.sqrt(e0))
    assert drift < 3.4e-14, drift


def test_error_sums_match_host_reduction(lbm):
    wl = _config1(steps=50)
    lat = gpu_lattice(lbm, wl)
    lat.step(wl.steps)
    out = lat.moments()
    ex = wl.exact_outputs(wl.steps * wl.dt)
    s = lat.error_sums(ex)
    e = out - ex
    np.testing.assert_allclose(s[0], np.sum(e * e, axis=(1, 2)), rtol=1e-12)
    np.testing.assert_allclose(s[1], np.sum(ex * ex, axis=(1, 2)), rtol=1e-12)
    np.testing.assert_allclose(s[2], np.max(np.abs(e), axis=(1, 2)), rtol=1e-12)


@pytest.mark.parametrize("storage", ["f64", "f32", "ms_bfp"])
def test_init_without_body_load_equals_zero_body_load(lbm, storage):
    """The initialisation skips every body-load term when no body load is given; with an
    explicit zero body load it evaluates them: the populations must agree exactly."""
    nx, ny = 133, 47
    rng = np.random.default_rng(17)
    U0, Ux, Uy = (rng.standard_normal((5, ny, nx)) * 1e-3 for _ in range(3))
    out = []
    for B0 in (None, np.zeros((2, ny, nx))):
        lat = lbm.Lattice(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, storage=storage, track_displacement=False)
        lat.init(U0, Ux, Uy, B0)
        out.append(lat.populations()[0])
        lat.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_checkpoint_resume_is_bit_exact(lbm):
    wl = _config1(steps=40)
    a = gpu_lattice(lbm, wl)
    a.step(20)
    blob = np.empty(lbm.lbm_state_bytes(a.ctx), dtype=np.uint8)
    lbm.lbm_save_state(a.ctx, blob)
    a.step(20)
    ref = a.moments()
    b = gpu_lattice(lbm, wl)
    lbm.lbm_load_state(b.ctx, blob, 20)
    b.step(20)
    np.testing.assert_array_equal(b.moments(), ref)


@pytest.mark.parametrize("storage,tol", [("f32", 1e-5), ("bf16", 5e-2), ("f16", 5e-3), ("ms_bf16", 1e-2),
                                         ("ms_f16", 1e-3), ("ms_bfp", 1e-3)])
def test_reduced_precision_against_oracle(lbm, storage, tol):
    """Populations stored in FP32 / BF16 / FP16 with FP32 arithmetic: relative L2 of the
    moment fields against the FP64 oracle after 200 steps of the config-1 problem."""
    wl = _config1(steps=200)
    _, ref = oracle_run(wl)
    lat = gpu_lattice(lbm, wl, storage=storage)
    lat.step(wl.steps)
    errs = field_errors(lat.moments(), ref, fields=range(5))
    assert max(errs) < tol, (storage, errs)


def test_api_errors(lbm):
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(8, 8, 0.1, 0.1 / 2.0, 1.0, 0.6)        # c = 2 < 2 sqrt(1.36)
    assert e.value.status == lbm.LBM_ERR_CFL
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(1, 8, 0.1, 0.01, 1.0, 0.6)
    assert e.value.status == lbm.LBM_ERR_ARG
    lat = lbm.Lattice(8, 8, 0.1, 0.01, 1.0, 0.6)
    with pytest.raises(lbm.LbmError) as e:
        lat.step(1)                                        # before init
    assert e.value.status == lbm.LBM_ERR_STATE
    lat.set_populations(np.zeros((4, 5, 8, 8)))
    lat.step(0)
    lat.set_forcing(np.ones((1, 8)), np.ones((1, 8)), np.ones((2, 2, 1)))
    lat.step(1)
    with pytest.raises(lbm.LbmError) as e:
        lat.step(1)                                        # table has rows for t = 0, 1 only
    assert e.value.status == lbm.LBM_ERR_STATE
    f = np.zeros((4, 5, 8, 8))
    f[1, 2, 3, 4] = np.nan
    lat.set_forcing()
    lat.set_populations(f)
    assert not lat.finite()


@pytest.mark.parametrize("dirichlet", [False, True])
def test_general_omega_matches_oracle(lbm, dirichlet):
    """omega != 2 (first-order control scheme with W = 1/8) against the oracle, with body load."""
    from oracle import Oracle, Params
    if dirichlet:
        wl = W.dirichlet_mms(40, 24, 1.1, 0.4, cfl=0.9, steps=50)
    else:
        wl = W.periodic_mms(48, 1.1, 0.4, cfl=0.9, steps=50)
    o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, wl.dirichlet, omega=1.7))
    o.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
    for m in range(wl.steps):
        o.step(wl.body_load(m), wl.wall_data(m))
    ref = o.outputs(wl.body_load(wl.steps))
    lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=wl.dirichlet, storage="f64")
    lat.set_relaxation(1.7)
    lat.set_forcing(*wl.forcing)
    if wl.dirichlet:
        lat.set_dirichlet(wl.wall)
    lat.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
    lat.step(wl.steps)
    errs = field_errors(lat.moments(), ref)
    assert max(errs) < TOL64, errs
    f, _ = lat.populations()
    np.testing.assert_allclose(f, o.f, atol=1e-12 * np.max(np.abs(o.f)))


@pytest.mark.parametrize("storage,tol", [("ms_bf16", 2e-2), ("ms_f16", 2e-3), ("ms_bfp", 2e-3)])
def test_moment_space_storage_dirichlet_with_forcing(lbm, storage, tol):
    """Moment-space storage (FP32 U, 16-bit non-equilibrium moments) on the Dirichlet
    manufactured solution with body load: every output field against the oracle."""
    wl = W.dirichlet_mms(64, 32, 1.1, 0.4, cfl=0.9, steps=120, amp=1e-2, kx=2 * math.pi, ky=2 * math.pi)
    _, ref = oracle_run(wl)
    lat = gpu_lattice(lbm, wl, storage=storage)
    lat.step(wl.steps)
    out = lat.moments()
    errs = field_errors(out, ref)
    assert max(errs) < tol, errs
    # the state round-trips through get/set populations and checkpoints
    blob = np.empty(lbm.lbm_state_bytes(lat.ctx), dtype=np.uint8)
    lbm.lbm_save_state(lat.ctx, blob)
    lbm.lbm_load_state(lat.ctx, blob, lat.m)
    np.testing.assert_array_equal(lat.moments(), out)
    assert lat.finite()


@pytest.mark.parametrize("dirichlet", [False, True])
@pytest.mark.parametrize("nx,ny", [(5, 3), (2, 2), (9, 2), (130, 2), (67, 45), (1031, 7), (130, 70), (31, 200),
                                   (241, 37), (360, 19), (121, 66)])
def test_two_step_fusion_fp32_is_bit_identical(lbm, dirichlet, nx, ny):
    """The fused kernels (two steps with rows staged by tensor copies or with register prefetch,
    three steps staged) equal single steps exactly in FP32 (tiles of 120 or 112 columns with a
    ragged last tile, the lattice's wrap columns, blocks of 16 rows or of the default 12 with a
    ragged last block, step counts that leave remainders)."""
    rng = np.random.default_rng(nx + 1000 * ny)
    f = rng.standard_normal((4, 5, ny, nx)) * 1e-3
    outs = []
    for fuse, staging, rows in ((1, 1, 16), (2, 0, 16), (2, 1, 16), (3, 1, 16), (3, 1, 0)):
        lat = lbm.Lattice(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, dirichlet=dirichlet, storage="f32",
                          track_displacement=False)
        lat.set_step_fusion(fuse, rows)
        lat.set_staging(staging)
        lat.set_populations(f)
        lat.step(9)
        lat.step(2)                         # three-step passes, then a remainder pair
        lat.synchronize()
        g, _ = lat.populations()
        outs.append(g)
        lat.close()
    for o in outs[1:]:
        np.testing.assert_array_equal(outs[0], o)


@pytest.mark.parametrize("storage", ["bf16", "f16"])
@pytest.mark.parametrize("dirichlet", [False, True])
@pytest.mark.parametrize("nx,ny", [(5, 3), (130, 70), (361, 41)])
def test_two_step_fusion_16bit_staged_equals_register_prefetch(lbm, storage, dirichlet, nx, ny):
    """16-bit populations: the staged and the register-prefetch two-step kernels do the same
    arithmetic (the intermediate step kept in FP32), so their states are identical."""
    rng = np.random.default_rng(7 * nx + ny)
    f = rng.standard_normal((4, 5, ny, nx)) * 1e-3
    outs = []
    for staging in (0, 1):
        lat = lbm.Lattice(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, dirichlet=dirichlet, storage=storage,
                          track_displacement=False)
        lat.set_step_fusion(2, 16)
        lat.set_staging(staging)
        lat.set_populations(f)
        lat.step(8)
        lat.synchronize()
        outs.append(lat.populations()[0])
        lat.close()
    np.testing.assert_array_equal(outs[0], outs[1])


@pytest.mark.parametrize("storage,tol", [("bf16", 5e-2), ("f16", 5e-3)])
def test_two_step_fusion_16bit_against_oracle(lbm, storage, tol):
    wl = W.grf_periodic(96, 64, 1.5, 0.5, ell=8.0, std=1e-3, seeds=(3, 4), steps=200)
    o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, False))
    o.init(wl.U0, wl.dU0dx, wl.dU0dy)
    for _ in range(200):
        o.step(track_displacement=False)
    ref = o.moments()
    errs = {}
    for fuse in (1, 2, 3):
        lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, storage=storage, track_displacement=False)
        lat.set_step_fusion(fuse, 64)
        lat.init(wl.U0, wl.dU0dx, wl.dU0dy)
        lat.step(200)
        errs[fuse] = max(field_errors(lat.moments(), ref, fields=range(5)))
        lat.close()
    for fuse in (2, 3):
        assert errs[fuse] < tol and errs[fuse] <= 1.2 * errs[1], errs


@pytest.mark.parametrize("storage,tol", [("ms_bf16", 1e-2), ("ms_f16", 1e-3), ("ms_bfp", 1e-3)])
@pytest.mark.parametrize("dirichlet", [False, True])
def test_two_step_fusion_moment_space_against_oracle(lbm, storage, tol, dirichlet):
    """Moment-space storage advanced two and three steps per pass by the staged kernels: the
    moment fields against the FP64 oracle (periodic GRF on 250 x 64, three tiles of 120 or 112
    columns with a ragged last one; Dirichlet: the homogeneous box of Sec. 6.2 on 96 x 96), no
    worse than one kernel per step."""
    if dirichlet:
        wl = W.energy_box(96, 1.1, 0.4, 1.0 / 240.0, 0)
    else:
        wl = W.grf_periodic(250, 64, 1.5, 0.5, ell=8.0, std=1e-3, seeds=(5, 6), steps=0)
    steps = 120
    o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet))
    o.init(wl.U0, wl.dU0dx, wl.dU0dy)
    for _ in range(steps):
        o.step(track_displacement=False)
    ref = o.moments()
    errs = {}
    for fuse in (1, 2, 3):
        lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=dirichlet, storage=storage,
                          track_displacement=False)
        lat.set_step_fusion(fuse, 16)
        lat.init(wl.U0, wl.dU0dx, wl.dU0dy)
        lat.step(steps - 1)                 # 119: the remainders of two- and three-step passes run too
        lat.step(1)
        lat.synchronize()
        errs[fuse] = max(field_errors(lat.moments(), ref, fields=range(5)))
        lat.close()
    for fuse in (2, 3):
        assert errs[fuse] < tol and errs[fuse] <= 1.2 * errs[1], errs


def _split_runs(lbm, nx, ny, f, us, steps, levels, dirichlet=False, wall=None, track=False, staging=1, rows=0):
    outs = {}
    for adds in levels:
        lat = lbm.Lattice(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, dirichlet=dirichlet, storage="f64",
                          track_displacement=track)
        lat.set_fp64_split(adds)
        lat.set_staging(staging)
        lat.set_step_fusion(1, rows)
        if wall is not None:
            lat.set_dirichlet(wall)
        lat.set_populations(f, us)
        lat.step(steps)
        outs[adds] = lat.populations()
        lat.close()
    return outs


@pytest.mark.parametrize("nx,ny", [(3, 5), (67, 45), (1031, 7), (130, 70)])
def test_fp64_split_is_bit_identical_periodic(lbm, nx, ny):
    """Additions moved to the integer pipes give the hardware FP64 results bit for bit."""
    rng = np.random.default_rng(7 * nx + ny)
    f = rng.standard_normal((4, 5, ny, nx))
    us = rng.standard_normal((2, ny, nx))
    outs = _split_runs(lbm, nx, ny, f, us, 11, [0, 1, 2, 5, 7], track=True)
    for adds in (1, 2, 5, 7):
        np.testing.assert_array_equal(outs[adds][0].view(np.int64), outs[0][0].view(np.int64))
        np.testing.assert_array_equal(outs[adds][1].view(np.int64), outs[0][1].view(np.int64))


@pytest.mark.parametrize("dirichlet", [False, True])
@pytest.mark.parametrize("nx,ny,rows", [(3, 5, 64), (127, 9, 4), (129, 33, 7), (300, 17, 1), (1031, 7, 3)])
def test_fp64_staged_step_equals_register_step(lbm, nx, ny, rows, dirichlet):
    """The FP64 step with its rows staged by asynchronous copies (split level 1, the IEEE sequence)
    gives the register kernel's populations and displacements bit for bit: ragged column
    blocks, row counts that do not divide ny, one row per block, wall data on Dirichlet edges."""
    steps = 9
    rng = np.random.default_rng(3 * nx + ny + rows)
    f = rng.standard_normal((4, 5, ny, nx))
    us = rng.standard_normal((2, ny, nx))
    wall = rng.standard_normal((steps, 2, 2 * (nx + ny))) * 1e-2 if dirichlet else None
    kw = dict(dirichlet=dirichlet, wall=wall, track=True, rows=rows)
    staged = _split_runs(lbm, nx, ny, f, us, steps, [1], staging=1, **kw)[1]
    plain = _split_runs(lbm, nx, ny, f, us, steps, [1], staging=0, **kw)[1]
    np.testing.assert_array_equal(staged[0].view(np.int64), plain[0].view(np.int64))
    np.testing.assert_array_equal(staged[1].view(np.int64), plain[1].view(np.int64))


def test_fp64_split_is_bit_identical_dirichlet_with_wall_data(lbm):
    nx, ny, steps = 150, 70, 25
    rng = np.random.default_rng(11)
    f = rng.standard_normal((4, 5, ny, nx)) * 1e-2
    us = rng.standard_normal((2, ny, nx))
    wall = rng.standard_normal((steps, 2, 2 * (nx + ny))) * 1e-2
    outs = _split_runs(lbm, nx, ny, f, us, steps, [0, 1, 6], dirichlet=True, wall=wall, track=True)
    for adds in (1, 6):
        np.testing.assert_array_equal(outs[adds][0].view(np.int64), outs[0][0].view(np.int64))
        np.testing.assert_array_equal(outs[adds][1].view(np.int64), outs[0][1].view(np.int64))


def test_fp64_split_handles_zeros_subnormals_and_wide_ranges(lbm):
    """Exact zeros, signed zeros, subnormals and operands 1e300 apart: the integer path
    either matches the hardware or hands the lane back to the FP64 pipe."""
    nx, ny = 96, 40
    rng = np.random.default_rng(5)
    f = rng.standard_normal((4, 5, ny, nx))
    pick = rng.integers(0, 6, size=f.shape)
    f[pick == 0] = 0.0
    f[pick == 1] = -0.0
    f[pick == 2] *= 1e-310                   # subnormal
    f[pick == 3] *= 1e-300
    f[pick == 4] *= 1e300
    f[:, :, :, :8] = 0.0                      # whole lanes of zeros (exact cancellations)
    outs = _split_runs(lbm, nx, ny, f, None, 5, [0, 1, 2, 3, 4, 5, 6, 7])
    for adds in range(1, 8):
        np.testing.assert_array_equal(outs[adds][0].view(np.int64), outs[0][0].view(np.int64))


def test_fp64_split_rejects_unsupported_counts(lbm):
    lat = lbm.Lattice(8, 8, 0.1, 0.1 / 3.2, 1.0, 0.6, storage="f64")
    for bad in (-1, 13, 100):
        with pytest.raises(lbm.LbmError):
            lat.set_fp64_split(bad)
    lat.set_fp64_split(11)
    lat.set_fp64_split(12)
    lat.close()
    # the fixed-point level needs cK / c at or above 2^-60
    lat = lbm.Lattice(8, 8, 1.0, 0.5, 1e-20, 0.0, storage="f64")
    with pytest.raises(lbm.LbmError):
        lat.set_fp64_split(12)
    lat.close()


FIXED = 12     # split level: the node update in exact fixed-point arithmetic


@pytest.mark.parametrize("case", ["grf_periodic", "energy_box", "ragged_periodic", "ragged_dirichlet"])
def test_fp64_fixed_point_level_matches_oracle(lbm, case):
    """Split level 12 (exact fixed-point node update, one rounding per output) against the
    FP64 oracle at the FP64 tolerance: periodic and homogeneous Dirichlet lattices without
    body load, ragged sizes, staged and register kernels."""
    if case == "grf_periodic":
        wl = W.grf_periodic(250, 64, 1.5, 0.5, ell=8.0, std=1e-3, seeds=(5, 6), steps=0)
        dirichlet, steps = False, 300
    elif case == "energy_box":
        wl = W.energy_box(96, 1.1, 0.4, 1.0 / 240.0, 0)
        dirichlet, steps = True, 300
    else:
        dirichlet = case == "ragged_dirichlet"
        wl = W.energy_box(37, 1.1, 0.4, 1.0 / 100.0, 0) if dirichlet else \
            W.grf_periodic(131, 29, 1.5, 0.5, ell=6.0, std=1e-3, seeds=(7, 8), steps=0)
        steps = 150
    o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet))
    o.init(wl.U0, wl.dU0dx, wl.dU0dy)
    for _ in range(steps):
        o.step(track_displacement=False)
    ref = o.moments()
    for staging in (1, 0):
        lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=dirichlet, storage="f64",
                          track_displacement=False)
        lat.set_fp64_split(FIXED)
        lat.set_staging(staging)
        lat.init(wl.U0, wl.dU0dx, wl.dU0dy)
        lat.step(steps)
        errs = field_errors(lat.moments(), ref, fields=range(5))
        lat.close()
        assert max(errs) < TOL64, (staging, errs)


@pytest.mark.parametrize("dirichlet", [False, True])
@pytest.mark.parametrize("nx,ny,rows", [(3, 5, 64), (129, 33, 7), (1031, 7, 3)])
def test_fp64_fixed_point_staged_equals_register_step(lbm, nx, ny, rows, dirichlet):
    """Level 12 computes the same bits in the staged and the register kernel (the same
    integer arithmetic per node), with wall data and displacement tracking; and it stays
    within FP64 accuracy of the FP64-pipe sequence (level 0)."""
    steps = 9
    rng = np.random.default_rng(5 * nx + ny + rows)
    f = rng.standard_normal((4, 5, ny, nx))
    us = rng.standard_normal((2, ny, nx))
    wall = rng.standard_normal((steps, 2, 2 * (nx + ny))) * 1e-2 if dirichlet else None
    kw = dict(dirichlet=dirichlet, wall=wall, track=True, rows=rows)
    staged = _split_runs(lbm, nx, ny, f, us, steps, [FIXED], staging=1, **kw)[FIXED]
    plain = _split_runs(lbm, nx, ny, f, us, steps, [FIXED], staging=0, **kw)[FIXED]
    ref = _split_runs(lbm, nx, ny, f, us, steps, [0], staging=0, **kw)[0]
    np.testing.assert_array_equal(staged[0].view(np.int64), plain[0].view(np.int64))
    np.testing.assert_array_equal(staged[1].view(np.int64), plain[1].view(np.int64))
    for part in (0, 1):
        rel = np.linalg.norm(staged[part] - ref[part]) / np.linalg.norm(ref[part])
        assert rel < 1e-14, (part, rel)


def test_fp64_fixed_point_conserves_energy(lbm):
    """Homogeneous Dirichlet, b = 0 (Sec. 6.2 set-up): ||f||_P conserved by the fixed-point
    level to the same bound as the FP64 path over 4000 steps."""
    wl = W.energy_box(160, 1.1, 0.4, 1.0 / 400.0, 4000)
    lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=True, storage="f64",
                      track_displacement=False)
    lat.set_fp64_split(FIXED)
    lat.init(wl.U0, wl.dU0dx, wl.dU0dy, None, wl.u0)
    e0 = lat.energy()
    drift = 0.0
    for _ in range(40):
        lat.step(100)
        drift = max(drift, abs(math.sqrt(lat.energy()) - math.sqrt(e0)) / math.sqrt(e0))
    lat.close()
    assert drift < 3.4e-14, drift


def test_fp64_fixed_point_handles_zeros_subnormals_and_wide_ranges(lbm):
    """Nodes outside the fixed-point range (all zero, tiny, near overflow) run the FP64
    sequence; the rest keep FP64 accuracy: finite where level 0 is finite, within FP64
    accuracy of level 0 over the whole field and over the band of tiny values."""
    nx, ny = 96, 40
    rng = np.random.default_rng(8)
    f = rng.standard_normal((4, 5, ny, nx))
    pick = rng.integers(0, 6, size=f.shape)
    f[pick == 0] = 0.0
    f[pick == 1] = -0.0
    f[pick == 2] *= 1e-310
    f[pick == 3] *= 1e-300
    f[pick == 4] *= 1e300
    f[:, :, :, :8] = 0.0
    f[:, :, 10:34, 40:90] = rng.standard_normal((4, 5, 24, 50)) * 1e-295   # below the fixed-point range
    outs = _split_runs(lbm, nx, ny, f, None, 5, [0, FIXED])
    def rel(a, b):
        sc = np.max(np.abs(b))
        return np.linalg.norm((a - b) / sc) / np.linalg.norm(b / sc)

    ref, got = outs[0][0], outs[FIXED][0]
    assert np.array_equal(np.isfinite(got), np.isfinite(ref))
    assert rel(got, ref) <= 1e-14, rel(got, ref)
    # nodes that only ever saw the tiny block ran the FP64 sequence: the same bits as level 0
    inner = (slice(None), slice(None), slice(16, 28), slice(46, 84))
    np.testing.assert_array_equal(got[inner].view(np.int64), ref[inner].view(np.int64))


@pytest.mark.parametrize("nx,ny,dirichlet", [(67, 45, False), (1031, 7, False), (150, 70, True)])
def test_fp64_faithful_split_levels_stay_at_fp64_accuracy(lbm, nx, ny, dirichlet):
    """Levels 8-11 round their integer-pipe additions faithfully (within 1/2 + 2^-9 ulp):
    after 40 steps every population stays within a few ulp-scale relative L2 of the
    all-FP64-pipe result, far inside the oracle tolerance."""
    rng = np.random.default_rng(3 * nx + ny)
    f = rng.standard_normal((4, 5, ny, nx)) * (1e-2 if dirichlet else 1.0)
    us = rng.standard_normal((2, ny, nx))
    wall = rng.standard_normal((40, 2, 2 * (nx + ny))) * 1e-2 if dirichlet else None
    outs = _split_runs(lbm, nx, ny, f, us, 40, [0, 8, 9, 10, 11], dirichlet=dirichlet, wall=wall, track=True)
    for level in (8, 9, 10, 11):
        for part in (0, 1):
            got, ref = outs[level][part], outs[0][part]
            rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
            assert rel < 1e-14, (level, part, rel)
        # the faithful path ran: it differs from the hardware sums in the last bit somewhere
        assert not np.array_equal(outs[level][0].view(np.int64), outs[0][0].view(np.int64)), level


def test_fp64_faithful_split_handles_zeros_subnormals_and_wide_ranges(lbm):
    """The faithful path hands subnormal, infinite or NaN results back to the FP64 pipe and
    handles exact zeros and operands 1e300 apart: finite where level 0 is finite, within FP64
    accuracy of level 0 over the whole field and over the band of tiny values."""
    nx, ny = 96, 40
    rng = np.random.default_rng(6)
    f = rng.standard_normal((4, 5, ny, nx))
    pick = rng.integers(0, 6, size=f.shape)
    f[pick == 0] = 0.0
    f[pick == 1] = -0.0
    f[pick == 2] *= 1e-310
    f[pick == 3] *= 1e-300
    f[pick == 4] *= 1e300
    f[:, :, :, :8] = 0.0
    outs = _split_runs(lbm, nx, ny, f, None, 5, [0, 8, 9, 10, 11])
    def rel(a, b):                      # relative L2, scaled first (values near 1e300 would overflow)
        sc = np.max(np.abs(b))
        return np.linalg.norm((a - b) / sc) / np.linalg.norm(b / sc)

    ref = outs[0][0]
    tiny = (np.abs(ref) < 1e-250) & (ref != 0.0)
    for level in (8, 9, 10, 11):
        got = outs[level][0]
        assert np.array_equal(np.isfinite(got), np.isfinite(ref)), level
        assert rel(got, ref) <= 1e-14, (level, rel(got, ref))
        if tiny.any():
            assert rel(got[tiny], ref[tiny]) <= 1e-12, (level, rel(got[tiny], ref[tiny]))


@pytest.mark.parametrize("dirichlet", [False, True])
def test_degenerate_material_without_shear_speed(lbm, dirichlet):
    """c_mu = 0 (no shear waves, the j_d / j_xy couplings vanish): still the oracle's result."""
    nx, ny, steps = 40, 24, 20
    rng = np.random.default_rng(17)
    f = rng.standard_normal((4, 5, ny, nx)) * 1e-2
    o = Oracle(Params(nx, ny, 0.1, 0.1 / 2.5, 1.0, 0.0, dirichlet))
    o.set_state(f, np.zeros((2, ny, nx)))
    for _ in range(steps):
        o.step(track_displacement=False)
    lat = lbm.Lattice(nx, ny, 0.1, 0.1 / 2.5, 1.0, 0.0, dirichlet=dirichlet, storage="f64", track_displacement=False)
    lat.set_populations(f)
    lat.step(steps)
    g, _ = lat.populations()
    lat.close()
    np.testing.assert_allclose(g, o.f, rtol=0, atol=1e-13 * np.max(np.abs(o.f)))


@pytest.mark.parametrize("storage,tol", [("f64", 1e-13), ("f32", 2e-6)])
def test_largest_row_count(lbm, storage, tol):
    """ny = 65535, the largest row count the library accepts, with a ragged 3-node row."""
    nx, ny, steps = 3, 65535, 4
    rng = np.random.default_rng(23)
    f = rng.standard_normal((4, 5, ny, nx)) * 1e-2
    o = Oracle(Params(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, False))
    o.set_state(f, np.zeros((2, ny, nx)))
    for _ in range(steps):
        o.step(track_displacement=False)
    lat = lbm.Lattice(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, storage=storage, track_displacement=False)
    lat.set_populations(f)
    lat.step(steps)
    g, _ = lat.populations()
    lat.close()
    np.testing.assert_allclose(g, o.f, rtol=0, atol=tol * np.max(np.abs(o.f)))


def test_staged_two_step_kernel_reports_a_wait_that_runs_out(lbm):
    """Test hook: the producer withholds one staged row, so every compute warp's bounded
    wait runs out (about 2 s); lbm_synchronize reports LBM_ERR_TIMEOUT once, the context
    stays usable, and a re-initialised lattice steps correctly afterwards."""
    nx, ny = 100, 12                        # one column tile, two blocks of 8 rows
    rng = np.random.default_rng(5)
    f = rng.standard_normal((4, 5, ny, nx)) * 1e-3
    lat = lbm.Lattice(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, storage="f32", track_displacement=False)
    lat.set_populations(f)
    lat.set_staging(2)
    for n in (2, 3):                        # the two-step and the three-step kernel
        lat.step(n)
        with pytest.raises(lbm.LbmError) as e:
            lat.synchronize()
        assert e.value.status == lbm.LBM_ERR_TIMEOUT
        lat.synchronize()                   # the flag was cleared
    lat.set_staging(1)
    lat.set_populations(f)
    lat.step(4)
    lat.synchronize()
    got = lat.populations()[0]
    ref = lbm.Lattice(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, storage="f32", track_displacement=False)
    ref.set_step_fusion(1, 64)
    ref.set_populations(f)
    ref.step(4)
    np.testing.assert_array_equal(got, ref.populations()[0])
    ref.close()
    lat.close()


def test_block_floating_point_saturation_is_reported(lbm):
    """LBM_MS_BFP: the deviation scale is fixed at initialisation; a body load that drives the
    deviations far beyond 8 times their initial size saturates blocks, which lbm_check_finite
    reports once as LBM_ERR_UNSTABLE.  A run within range reports nothing."""
    g = W.grf_periodic(64, 64, 1.5, 0.5, ell=8.0, std=1e-3, seeds=(3, 4), steps=0)
    ok = lbm.Lattice(g.nx, g.ny, g.dx, g.dt, g.cK, g.cmu, storage="ms_bfp", track_displacement=False)
    ok.init(g.U0, g.dU0dx, g.dU0dy)
    ok.step(300)
    assert ok.finite()
    ok.close()
    wl = W.periodic_mms(32, 1.5, 0.5, cfl=0.9, steps=60, amp=1e-2, kx=2 * math.pi, ky=2 * math.pi)
    lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, storage="ms_bfp", track_displacement=False)
    lat.set_forcing(*wl.forcing)
    tiny = 1e-7
    lat.init(wl.U0 * tiny, wl.dU0dx * tiny, wl.dU0dy * tiny, wl.body_load(0) * tiny)
    lat.step(wl.steps)
    assert not lat.finite()
    assert "block" in lbm.lbm_last_error(lat.ctx)
    assert lat.finite()                     # reported once, the flag is cleared
    lat.close()


def test_pinned_host_buffers_are_used_in_place(lbm):
    """Host arrays in pinned memory are read and written by the kernels in place; the
    results equal those through pageable host memory and through device memory."""
    import torch
    wl = _config1(steps=10)
    outs = []
    for kind in ("pageable", "pinned", "device"):
        lat = gpu_lattice(lbm, wl, storage="f64")        # forcing and init as in config 1
        if kind == "pageable":
            lat.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
        else:
            conv = (lambda a: torch.from_numpy(a).pin_memory()) if kind == "pinned" else \
                   (lambda a: torch.from_numpy(a).cuda())
            args = [conv(a) for a in (wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)]
            if kind == "pinned":
                lat.init(*[a.numpy() for a in args])
            else:
                torch.cuda.synchronize()
                lat.init(*args)
        lat.step(wl.steps)
        if kind == "pinned":
            out = torch.empty((10, wl.ny, wl.nx), dtype=torch.float64).pin_memory()
            lat.moments(out.numpy())
            outs.append(out.numpy().copy())
        elif kind == "device":
            out = torch.empty((10, wl.ny, wl.nx), dtype=torch.float64, device="cuda")
            lat.moments(out)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        else:
            outs.append(lat.moments())
        lat.close()
    np.testing.assert_array_equal(outs[0], outs[1])
    np.testing.assert_array_equal(outs[0], outs[2])


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_energy_monitor_is_quiet_and_changes_nothing_on_a_conserving_run(lbm, storage):
    """Homogeneous Dirichlet, b = 0: ||f||_P is conserved up to the storage format's rounding,
    so a monitor with growth 1 + 1e-9 (FP64) or 1 + 1e-5 (FP32), checked every 50 steps with the
    last check mid-run, reports nothing, and the state equals that of the same run without it
    bit for bit."""
    wl = W.energy_box(96, 1.1, 0.4, 1.0 / 240.0, 0)
    outs = []
    for every in (0, 50):
        lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=True, storage=storage,
                          track_displacement=False)
        lat.init(wl.U0, wl.dU0dx, wl.dU0dy)
        lat.set_energy_check(every, 1.0 + (1e-9 if storage == "f64" else 1e-5))
        lat.step(130)
        lat.step(290)
        lat.synchronize()
        outs.append(lat.moments())
        lat.close()
    np.testing.assert_array_equal(outs[0].view(np.int64), outs[1].view(np.int64))


def test_energy_monitor_reports_growth_beyond_its_bound(lbm):
    """A bound below the (conserved) energy: the first check sets the flag, the next
    lbm_synchronize reports LBM_ERR_UNSTABLE once and clears it; the context stays usable
    and turning the monitor off stops the reports.  Bad arguments and an uninitialised
    context are refused."""
    wl = W.energy_box(64, 1.1, 0.4, 1.0 / 170.0, 0)
    lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=True, storage="f64",
                      track_displacement=False)
    with pytest.raises(lbm.LbmError) as e:
        lat.set_energy_check(10, 2.0)                  # before lbm_init
    assert e.value.status == lbm.LBM_ERR_STATE
    lat.init(wl.U0, wl.dU0dx, wl.dU0dy)
    for every, growth in ((-1, 2.0), (10, 0.0), (10, float("nan")), (10, float("inf"))):
        with pytest.raises(lbm.LbmError) as e:
            lat.set_energy_check(every, growth)
        assert e.value.status == lbm.LBM_ERR_ARG
    lat.set_energy_check(10, 0.5)
    lat.step(9)
    lat.synchronize()                                  # no check has run yet
    lat.step(2)
    with pytest.raises(lbm.LbmError) as e:
        lat.synchronize()
    assert e.value.status == lbm.LBM_ERR_UNSTABLE
    lat.synchronize()                                  # reported once
    lat.set_energy_check(0, 0.5)
    lat.step(30)
    lat.synchronize()
    assert np.all(np.isfinite(lat.moments()))
    lat.close()


def test_refused_allocation_reports_oom_and_leaves_the_device_usable(lbm):
    """A lattice far beyond the GPU's memory (60000^2 FP64: two 576 GB state buffers, refused by
    the first allocation, before any launch): lbm_create returns LBM_ERR_OOM, and a lattice
    created next runs normally (the refused allocation does not leak into the launch checks
    of later calls)."""
    n = 60000
    with pytest.raises(lbm.LbmError) as e:
        lbm.Lattice(n, n, 1.0 / n, 1.0 / n / 3.2, 1.0, 0.6, storage="f64", track_displacement=False)
    assert e.value.status == lbm.LBM_ERR_OOM
    wl = W.energy_box(64, 1.1, 0.4, 1.0 / 170.0, 0)
    lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=True, storage="f64",
                      track_displacement=False)
    lat.init(wl.U0, wl.dU0dx, wl.dU0dy)
    e0 = lat.energy()
    lat.step(50)
    lat.synchronize()
    assert abs(lat.energy() - e0) <= 1e-13 * e0
    lat.close()


@pytest.mark.parametrize("storage,tol", [("ms_f16", 5e-3), ("ms_bfp", 5e-3)])
@pytest.mark.parametrize("nx", [9, 130])
def test_three_step_moment_space_on_two_rows(lbm, storage, tol, nx):
    """Periodic lattices of two rows: the staged rows of a three-step pass (three beyond each
    side) wrap more than once; every read stays inside the lattice and the result matches the
    oracle at the 16-bit format's accuracy on this rough field (about 1e-3 after 30 steps;
    a row read as zeros would be off by order one)."""
    ny = 2
    wl = W.grf_periodic(nx, ny, 1.5, 0.5, ell=3.0, std=1e-3, seeds=(5, 6), steps=0)
    o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, False))
    o.init(wl.U0, wl.dU0dx, wl.dU0dy)
    for _ in range(30):
        o.step(track_displacement=False)
    ref = o.moments()
    lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=False, storage=storage,
                      track_displacement=False)
    lat.init(wl.U0, wl.dU0dx, wl.dU0dy)
    lat.step(30)
    lat.synchronize()
    errs = field_errors(lat.moments(), ref, fields=range(5))
    lat.close()
    assert max(errs) < tol, errs


@pytest.mark.parametrize("dirichlet", [False, True])
def test_fp64_fixed_point_with_body_load(lbm, dirichlet):
    """The manufactured solutions of configs 1 and 2 carry a body load (and wall data on the
    rectangle): at split level 12 (the default) the body load enters the fixed-point update;
    the result equals the oracle within the FP64 tolerance and the all-FP64-pipe kernel
    (level 0) within rounding-level relative L2 (two different roundings of the same update
    over 80-120 steps), without being bit-identical to it."""
    if dirichlet:
        wl = W.dirichlet_mms(96, 48, 1.1, 0.4, cfl=0.9, steps=80, height=1.0)
    else:
        wl = W.periodic_mms(80, 1.5, 0.5, cfl=0.9, steps=120, amp=1e-2, kx=2 * math.pi, ky=2 * math.pi)
    _, ref = oracle_run(wl)
    outs = {}
    for level in (0, 12):
        lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=wl.dirichlet, storage="f64",
                          track_displacement=True)
        lat.set_fp64_split(level)
        if wl.forcing is not None:
            lat.set_forcing(*wl.forcing)
        if wl.dirichlet and wl.wall is not None:
            lat.set_dirichlet(wl.wall)
        lat.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
        lat.step(wl.steps)
        outs[level] = lat.moments()
        lat.close()
    assert max(field_errors(outs[12], ref)) < TOL64
    assert max(field_errors(outs[12], outs[0])) < 1e-13      # measured 1.6e-14 after 120 steps
    assert not np.array_equal(outs[12].view(np.int64), outs[0].view(np.int64))
