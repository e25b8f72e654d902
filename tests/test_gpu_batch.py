"""GPU tests of batched stepping: a ragged batch of periodic and Dirichlet
lattices with different materials follows, lattice by lattice, exactly the
single-lattice trajectory (bit-identical) and the FP64 oracle (1e-12); the
persistent mode equals the launch-per-step mode; the autotuner writes and reuses
its cache; a grid-barrier wait that cannot complete ends with LBM_ERR_TIMEOUT
and leaves the batch usable."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle, Params
from oracle.postprocess import rel_l2

pytestmark = pytest.mark.gpu

SIZES = [(5, 3, 0), (37, 23, 1), (130, 7, 0), (300, 9, 1), (64, 64, 0), (1031, 5, 1), (8, 200, 0), (2, 2, 1),
         (257, 33, 0), (96, 17, 1)]


def _descs(storage_nu_seed=0):
    rng = np.random.default_rng(5 + storage_nu_seed)
    out = []
    for i, (nx, ny, bc) in enumerate(SIZES):
        nu = float(rng.uniform(0, 0.49))
        cK2, cmu2 = W.material.poisson_to_speeds(nu)
        c = W.material.lattice_speed(cK2, cmu2, 0.9)
        dx = 1.0 / max(nx, ny)
        out.append((nx, ny, bc, dx, dx / c, math.sqrt(cK2), math.sqrt(cmu2)))
    return out


def _inputs(desc, seed):
    nx, ny, bc = desc[0], desc[1], desc[2]
    rng = np.random.default_rng(seed)
    U0 = rng.standard_normal((5, ny, nx)) * 1e-3
    Ux = rng.standard_normal((5, ny, nx)) * 1e-3
    Uy = rng.standard_normal((5, ny, nx)) * 1e-3
    return U0, Ux, Uy


def _run_batch(lbm, descs, storage, mode, steps, graph_steps=10):
    b = lbm.lbm_batch_create(descs, storage=lbm.STORAGE[storage])
    lbm.lbm_batch_set_mode(b, mode, graph_steps)
    for i, d in enumerate(descs):
        lbm.lbm_batch_init(b, i, *_inputs(d, 100 + i))
    lbm.lbm_batch_step(b, steps)
    lbm.lbm_batch_synchronize(b)
    outs = []
    for i, d in enumerate(descs):
        o = np.empty((10, d[1], d[0]))
        lbm.lbm_batch_moments(b, i, o)
        outs.append(o)
    en = [lbm.lbm_batch_energy(b, i) for i in range(len(descs))]
    lbm.lbm_batch_destroy(b)
    return outs, en


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_batch_equals_single_lattices_bitwise(lbm, storage):
    descs = _descs()
    outs, en = _run_batch(lbm, descs, storage, 0, 25)
    for i, d in enumerate(descs):
        nx, ny, bc, dx, dt, cK, cmu = d
        lat = lbm.Lattice(nx, ny, dx, dt, cK, cmu, dirichlet=bool(bc), storage=storage, track_displacement=False)
        lat.init(*_inputs(d, 100 + i))
        lat.step(25)
        ref = lat.moments()
        np.testing.assert_array_equal(outs[i][0:5], ref[0:5])
        assert en[i] == pytest.approx(lat.energy(), rel=1e-13)
        lat.close()


@pytest.mark.parametrize("mode", [0, 3])
def test_batch_matches_oracle_fp64(lbm, mode):
    descs = _descs()
    outs, _ = _run_batch(lbm, descs, "f64", mode, 25)
    for i, d in enumerate(descs):
        nx, ny, bc, dx, dt, cK, cmu = d
        o = Oracle(Params(nx, ny, dx, dt, cK, cmu, bool(bc)))
        o.init(*_inputs(d, 100 + i))
        for _ in range(25):
            o.step(None, None, track_displacement=False)
        ref = o.moments()
        for q in range(5):
            assert rel_l2(outs[i][q], ref[q]) < 1e-12, (i, q)


def test_persistent_mode_equals_launch_per_step(lbm):
    descs = _descs(1)
    a, _ = _run_batch(lbm, descs, "f64", 0, 37, graph_steps=8)
    b, _ = _run_batch(lbm, descs, "f64", 1, 37, graph_steps=8)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_tuner_writes_and_reuses_cache(lbm, tmp_path):
    descs = _descs(2)
    cache = tmp_path / "tune.txt"
    b = lbm.lbm_batch_create(descs, storage=lbm.LBM_F32)
    lbm.lbm_batch_tune(b, cache)
    widths = [lbm.lbm_batch_info(b, i)["tile_width"] for i in range(len(descs))]
    lbm.lbm_batch_destroy(b)
    text = cache.read_text()
    assert "|f32|class" in text and "|f32|mode|" in text
    b = lbm.lbm_batch_create(descs, storage=lbm.LBM_F32)
    lbm.lbm_batch_tune(b, cache)
    assert [lbm.lbm_batch_info(b, i)["tile_width"] for i in range(len(descs))] == widths
    # tuning after init is refused (it would advance the state)
    lbm.lbm_batch_init(b, 0, *_inputs(descs[0], 1))
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_tune(b, cache)
    assert e.value.status == lbm.LBM_ERR_STATE
    lbm.lbm_batch_destroy(b)


def test_barrier_timeout_is_reported_and_batch_stays_usable(lbm):
    descs = _descs(3)
    b = lbm.lbm_batch_create(descs, storage=lbm.LBM_F64)
    lbm.lbm_batch_set_mode(b, 1, 4)
    lbm.lbm_batch_set_barrier(b, 0.05, extra_arrivals=1)   # waits for an arrival that never comes
    for i, d in enumerate(descs):
        lbm.lbm_batch_init(b, i, *_inputs(d, 100 + i))
    lbm.lbm_batch_step(b, 4)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_synchronize(b)
    assert e.value.status == lbm.LBM_ERR_TIMEOUT
    lbm.lbm_batch_set_barrier(b, 2.0, 0)
    for i, d in enumerate(descs):
        lbm.lbm_batch_init(b, i, *_inputs(d, 100 + i))
    lbm.lbm_batch_step(b, 6)
    lbm.lbm_batch_synchronize(b)
    o = np.empty((10, descs[1][1], descs[1][0]))
    lbm.lbm_batch_moments(b, 1, o)
    assert np.all(np.isfinite(o))
    lbm.lbm_batch_destroy(b)


def test_torch_grf_inputs_match_numpy_recipe(lbm):
    """The GPU generator used for large batches reproduces the numpy GRF recipe."""
    from workloads.grf import batch_lattice_inputs_torch
    spec = W.batch_spec(count=4)
    for sp in spec[:2] + spec[3:4]:
        dx = 1.0 / max(sp.nx, sp.ny)
        U0, Ux, Uy = (t.cpu().numpy() for t in batch_lattice_inputs_torch(sp, dx))
        ref = W.grf_periodic(sp.nx, sp.ny, sp.cK2, sp.cmu2, ell=sp.ell, std=1e-3, seeds=(sp.seed, sp.seed + 7919),
                             dx=dx, window=sp.dirichlet)
        np.testing.assert_allclose(U0, ref.U0, atol=1e-15)
        np.testing.assert_allclose(Ux, ref.dU0dx, atol=1e-12 * np.max(np.abs(ref.dU0dx)))
        np.testing.assert_allclose(Uy, ref.dU0dy, atol=1e-12 * np.max(np.abs(ref.dU0dy)))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_three_step_mode_equals_the_other_modes_and_single_lattices(lbm, storage):
    """Mode 2 (three steps per pass over staged-row tiles of every lattice; steps beyond a
    multiple of three as single steps): in FP32 it equals mode 0 bit for bit at a step count
    that leaves remainders, inside and outside graphs; in BF16, after a multiple of three
    steps, it equals single-lattice runs (which also advance three steps per pass)."""
    descs = _descs(4)
    if storage == "f32":
        a, ea = _run_batch(lbm, descs, "f32", 0, 37, graph_steps=8)
        b, eb = _run_batch(lbm, descs, "f32", 2, 37, graph_steps=8)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)
        assert ea == eb
        return
    outs, _ = _run_batch(lbm, descs, "bf16", 2, 24, graph_steps=6)
    for i, d in enumerate(descs):
        nx, ny, bc, dx, dt, cK, cmu = d
        lat = lbm.Lattice(nx, ny, dx, dt, cK, cmu, dirichlet=bool(bc), storage="bf16", track_displacement=False)
        lat.init(*_inputs(d, 100 + i))
        lat.step(24)
        np.testing.assert_array_equal(outs[i][0:5], lat.moments()[0:5])
        lat.close()


def test_three_step_mode_is_refused_for_fp64_and_odd_graphs(lbm):
    descs = _descs(5)
    b = lbm.lbm_batch_create(descs, storage=lbm.LBM_F64)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_set_mode(b, 2, 10)
    assert e.value.status == lbm.LBM_ERR_ARG
    lbm.lbm_batch_destroy(b)
    b = lbm.lbm_batch_create(descs, storage=lbm.LBM_F32)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_set_mode(b, 2, 7)
    assert e.value.status == lbm.LBM_ERR_ARG
    lbm.lbm_batch_set_mode(b, 2, 10)
    lbm.lbm_batch_destroy(b)


def _descs_with_level1_lattices():
    """_descs(6) plus a periodic and a Dirichlet lattice whose cmu/c lies below 2^-60: the
    fixed-point update cannot take that multiplier, so these two run the IEEE sequence of split
    level 1 (a list of their own in mode 3)."""
    out = _descs(6)
    for nx, ny, bc in ((200, 13, 0), (131, 10, 1)):
        cK = 1.0
        c = W.material.lattice_speed(cK * cK, 0.0, 0.9)
        dx = 1.0 / max(nx, ny)
        out.append((nx, ny, bc, dx, dx / c, cK, 1e-25))
    return out


def test_staged_fp64_mode_equals_launch_per_step(lbm):
    """Mode 3 (FP64 on staged rows, 128 x 4 tiles on the fixed-point update and 128 x 2 on the
    level-1 sequence) equals mode 0 bit for bit, inside graphs (8 steps) and in the remainder
    steps (37 = 4 x 8 + 5), for ragged periodic and Dirichlet lattices of both node updates."""
    descs = _descs_with_level1_lattices()
    a, ea = _run_batch(lbm, descs, "f64", 0, 37, graph_steps=8)
    b, eb = _run_batch(lbm, descs, "f64", 3, 37, graph_steps=8)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    assert ea == eb


def test_staged_fp64_mode_is_refused_for_other_formats(lbm):
    descs = _descs(7)
    b = lbm.lbm_batch_create(descs, storage=lbm.LBM_F32)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_set_mode(b, 3, 10)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_batch_set_mode(b, 4, 10)
    assert e.value.status == lbm.LBM_ERR_ARG
    lbm.lbm_batch_destroy(b)


def test_tuned_fp64_batch_equals_launch_per_step(lbm, tmp_path):
    """The tuner times modes 0, 1 and 3 for an FP64 batch and keeps the fastest; whichever it
    keeps, the trajectory equals mode 0's bit for bit."""
    descs = _descs_with_level1_lattices()
    ref, _ = _run_batch(lbm, descs, "f64", 0, 12, graph_steps=4)
    cache = tmp_path / "tune.txt"
    b = lbm.lbm_batch_create(descs, storage=lbm.LBM_F64)
    lbm.lbm_batch_tune(b, cache)
    assert "|f64|mode|" in cache.read_text()
    for i, d in enumerate(descs):
        lbm.lbm_batch_init(b, i, *_inputs(d, 100 + i))
    lbm.lbm_batch_step(b, 12)
    lbm.lbm_batch_synchronize(b)
    for i, d in enumerate(descs):
        o = np.empty((10, d[1], d[0]))
        lbm.lbm_batch_moments(b, i, o)
        np.testing.assert_array_equal(o, ref[i])
    lbm.lbm_batch_destroy(b)
