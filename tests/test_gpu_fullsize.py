"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (periodic, no body load, no displacement tracking):

* periodic 8192^2 GRF, every storage format (the reduced ones two steps per pass,
  the library default): sampled nodes (edges, corners, interior)
  after 3 steps against the oracle run on a periodic patch around each sample
  (the domain of dependence of 3 steps is 3 nodes, the patch is 16 wide);
  properties that hold at any size: sum of U and ||f||_P conserved;
* Dirichlet 2048x1024 with the moving manufactured solution, FP64 and FP32,
  displacement tracked: every node after 20 steps against a full oracle run;
* the benchmark's batch of 512 ragged lattices (233 M nodes, FP32, tuned launch
  mode, 100-step graphs): sampled lattices bit-identical to single-lattice runs.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import Oracle, Params
from oracle.postprocess import rel_l2

from .helpers import field_errors, gpu_lattice, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def grf8192():
    return W.grf_periodic(8192, 8192, 1.5, 0.5, cfl=0.9, ell=64.0, std=1e-3, seeds=(1, 2), steps=3)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-5), ("bf16", 1e-2), ("f16", 1.5e-3),
                                         ("ms_bf16", 5e-3), ("ms_f16", 1e-3), ("ms_bfp", 1e-3)])
def test_periodic_8192_sampled_against_oracle_patches(lbm, grf8192, storage, tol):
    import torch
    wl = grf8192
    n, k, P = 8192, 3, 16
    lat = lbm.Lattice(n, n, wl.dx, wl.dt, wl.cK, wl.cmu, storage=storage, track_displacement=False)
    dev = torch.device("cuda")
    lat.init(torch.from_numpy(wl.U0).to(dev), torch.from_numpy(wl.dU0dx).to(dev), torch.from_numpy(wl.dU0dy).to(dev))
    e0 = lat.energy()
    s0 = None
    out = torch.empty((10, n, n), dtype=torch.float64, device=dev)
    lat.moments(out)
    s0 = out[0:5].sum(dim=(1, 2)).cpu().numpy()
    lat.step(k)
    lat.moments(out)
    s1 = out[0:5].sum(dim=(1, 2)).cpu().numpy()
    e1 = lat.energy()
    rng = np.random.default_rng(99)
    pts = [(0, 0), (n - 1, 0), (0, n - 1), (n - 1, n - 1), (0, 4097), (n - 1, 123), (77, 0), (5000, n - 1),
           (1, 1), (n - 2, n - 2)] + [tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(22)]
    xs = torch.tensor([p[0] for p in pts], device=dev)
    ys = torch.tensor([p[1] for p in pts], device=dev)
    got = out[:, ys, xs].cpu().numpy()                 # [10, samples]
    lat.close()
    del out
    ref = np.zeros_like(got)
    for s, (x, y) in enumerate(pts):
        ix = (np.arange(P) - P // 2 + x) % n
        iy = (np.arange(P) - P // 2 + y) % n
        sub = lambda a: np.ascontiguousarray(a[:, iy][:, :, ix])
        o = Oracle(Params(P, P, wl.dx, wl.dt, wl.cK, wl.cmu, False))
        o.init(sub(wl.U0), sub(wl.dU0dx), sub(wl.dU0dy))
        for _ in range(k):
            o.step(track_displacement=False)
        U = o.moments()
        ref[0:5, s] = U[:, P // 2, P // 2]
    if storage in ("f64", "f32"):
        for q in range(5):
            assert rel_l2(got[q], ref[q]) < tol, (storage, q, rel_l2(got[q], ref[q]))
    else:
        # 16-bit storage quantises every population to about 2^-9 (BF16) or 2^-12 (FP16) of its
        # size; after 3 steps the stress fields are still about 1 % of the velocities, so their
        # errors are measured against the velocity scale, the size the quantum is relative to
        vscale = np.linalg.norm(ref[0:2]) / math.sqrt(2)
        for q in range(5):
            err = np.linalg.norm(got[q] - ref[q]) / max(np.linalg.norm(ref[q]), vscale)
            assert err < tol, (storage, q, err)
    # properties at full size: sum of U and the weighted norm are invariants (periodic, b = 0), up
    # to the storage format's rounding (populations in 16 bits carry U in 16 bits; the moment
    # space keeps U itself in FP32)
    atol = {"f64": 1e-12, "f32": 1e-6, "ms_bf16": 1e-6, "ms_f16": 1e-6, "ms_bfp": 1e-6, "f16": 1e-3, "bf16": 1e-2}[storage]
    assert np.all(np.abs(s1 - s0) <= atol * (np.abs(s0) + np.sqrt(n * n) * 1e-3)), (storage, s1 - s0)
    etol = {"f64": 1e-13, "f32": 1e-5, "ms_bf16": 1e-3, "ms_f16": 1e-4, "ms_bfp": 1e-4, "f16": 1e-3, "bf16": 1e-2}[storage]
    assert abs(e1 - e0) <= etol * e0, (storage, (e1 - e0) / e0)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_dirichlet_2048x1024_against_full_oracle(lbm, storage, tol):
    cK2, cmu2 = W.material.poisson_to_speeds(0.25)
    wl = W.dirichlet_mms(2048, 1024, cK2, cmu2, cfl=0.9, steps=20, height=1.0, amp=1e-2,
                         kx=2 * math.pi, ky=2 * math.pi)
    _, ref = oracle_run(wl)
    lat = gpu_lattice(lbm, wl, storage=storage)
    lat.step(wl.steps)
    errs = field_errors(lat.moments(), ref)
    lat.close()
    assert max(errs) < tol, errs


def test_batch_512_lattices_sampled_against_single_lattices(lbm, tmp_path):
    """The benchmark's batch workload at full size and in its launch configuration (autotuned
    tiles and mode, graphs of 100 steps): the smallest, the largest and a spread of other
    lattices, periodic and Dirichlet, equal single-lattice runs bit for bit after 200 steps,
    and the smallest periodic and Dirichlet lattices equal the FP64 oracle within 1e-5."""
    import torch
    from workloads.grf import batch_lattice_inputs_torch
    spec = W.batch_spec(count=512)
    descs = []
    for sp in spec:
        c = W.material.lattice_speed(sp.cK2, sp.cmu2, 0.9)
        dx = 1.0 / max(sp.nx, sp.ny)
        descs.append((sp.nx, sp.ny, int(sp.dirichlet), dx, dx / c, sp.cK2 ** 0.5, sp.cmu2 ** 0.5))
    b = lbm.lbm_batch_create(descs, storage=lbm.LBM_F32)
    lbm.lbm_batch_tune(b, str(tmp_path / "tune.txt"))
    for i, (sp, d) in enumerate(zip(spec, descs)):
        lbm.lbm_batch_init(b, i, *batch_lattice_inputs_torch(sp, d[3], device="cuda"))
    mode = 0
    for line in open(tmp_path / "tune.txt"):
        if "|f32|mode|" in line:
            mode = int(line.rsplit("|", 1)[1])
    lbm.lbm_batch_set_mode(b, mode, 100)
    lbm.lbm_batch_step(b, 200)
    lbm.lbm_batch_synchronize(b)
    nodes = [d[0] * d[1] for d in descs]
    pick = {int(np.argmin(nodes)), int(np.argmax(nodes))} | set(range(0, 512, 73)) | {1, 511}
    for i in sorted(pick):
        sp, d = spec[i], descs[i]
        nx, ny, bc, dx, dt, cK, cmu = d
        got = torch.empty((10, ny, nx), dtype=torch.float64, device="cuda")
        lbm.lbm_batch_moments(b, i, got)
        lbm.lbm_batch_synchronize(b)
        lat = lbm.Lattice(nx, ny, dx, dt, cK, cmu, dirichlet=bool(bc), storage="f32", track_displacement=False)
        lat.init(*batch_lattice_inputs_torch(sp, dx, device="cuda"))
        lat.step(200)
        ref = torch.empty_like(got)
        lat.moments(ref)
        lat.synchronize()
        torch.cuda.synchronize()
        lat.close()
        assert torch.equal(got[0:5], ref[0:5]), (i, nx, ny, bc)
    # anchored to the FP64 oracle: the smallest periodic and the smallest Dirichlet lattice of the
    # batch, run by the oracle from the same inputs, agree with the batch's FP32 fields within the
    # FP32 storage bound
    for bc_want in (0, 1):
        i = min((j for j in range(512) if descs[j][2] == bc_want), key=lambda j: nodes[j])
        sp, (nx, ny, bc, dx, dt, cK, cmu) = spec[i], descs[i]
        got = torch.empty((10, ny, nx), dtype=torch.float64, device="cuda")
        lbm.lbm_batch_moments(b, i, got)
        lbm.lbm_batch_synchronize(b)
        U0, Ux, Uy = (t.cpu().numpy() for t in batch_lattice_inputs_torch(sp, dx, device="cuda"))
        o = Oracle(Params(nx, ny, dx, dt, cK, cmu, bool(bc)))
        o.init(U0, Ux, Uy)
        for _ in range(200):
            o.step(track_displacement=False)
        ref = o.outputs()
        errs = field_errors(got.cpu().numpy(), ref, range(5))
        assert max(errs) < 1e-5, (i, nx, ny, bc, errs)
    lbm.lbm_batch_destroy(b)
