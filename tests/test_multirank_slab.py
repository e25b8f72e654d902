"""Row-slab decomposition on CPU ranks: gloo processes split one lattice into slabs,
exchange halo rows every step through paper_2408_01081_gb300.slab.exchange (the code
the GPU ranks use with NCCL) and must reproduce the whole-lattice oracle run bit for
bit, periodic and Dirichlet, with two ranks (each the other's upper and lower
neighbour when periodic) and three.

Each rank's slab is held by the FP64 oracle on the slab's rows plus its halo rows.
The oracle stores pre-collision populations, so its halo messages carry the
neighbour's whole boundary node (20 values per column) where the CUDA slabs send the
5 values of one post-collision direction; the split, the neighbours, the message
order and the reassembly are the same code."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(dirichlet):
    import workloads as W
    if dirichlet:
        return W.energy_box(12, 1.1, 0.4, 1.0 / 30.0, 0)
    return W.grf_periodic(12, 11, 1.5, 0.5, ell=3.0, std=1e-3, seeds=(8, 9), steps=0)


def _rank(rank, world, dirichlet, steps, port, q):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    from oracle import Oracle, Params
    from paper_2408_01081_gb300.slab import exchange, neighbours, slab_rows
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        wl = _problem(dirichlet)
        nx, ny = wl.nx, wl.ny
        whole = Oracle(Params(nx, ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet))
        whole.init(wl.U0, wl.dU0dx, wl.dU0dy)
        y0, rows = slab_rows(ny, world, rank)
        lower, upper = neighbours(world, rank, not dirichlet)
        lo, hi = int(lower is not None), int(upper is not None)
        own = slice(lo, lo + rows)
        slab = Oracle(Params(nx, rows + lo + hi, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet))
        src_rows = [(y0 - lo + i) % ny for i in range(rows + lo + hi)]
        slab.set_state(np.ascontiguousarray(whole.f[:, :, src_rows, :]))
        buf = lambda: torch.empty((4, 5, nx), dtype=torch.float64)
        from_lower, from_upper = (buf() if lo else None), (buf() if hi else None)
        for _ in range(steps):
            to_lower = torch.from_numpy(slab.f[:, :, lo, :].copy()) if lo else None
            to_upper = torch.from_numpy(slab.f[:, :, lo + rows - 1, :].copy()) if hi else None
            exchange(dist, rank, world, not dirichlet, to_lower, to_upper, from_lower, from_upper)
            if lo:
                slab.f[:, :, 0, :] = from_lower.numpy()
            if hi:
                slab.f[:, :, lo + rows, :] = from_upper.numpy()
            slab.step(track_displacement=False)
            whole.step(track_displacement=False)
        same = bool(np.array_equal(slab.f[:, :, own, :], whole.f[:, :, y0:y0 + rows, :]))
        q.put((rank, same, float(np.max(np.abs(whole.f)))))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("dirichlet", [False, True])
@pytest.mark.parametrize("world", [2, 3])
def test_slabs_on_gloo_ranks_reproduce_the_whole_lattice(world, dirichlet):
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, dirichlet, 9, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[0] for r in res] == list(range(world))
    for rank, same, fmax in res:
        assert fmax > 0.0
        assert same, rank


def test_slab_rows_cover_the_lattice_once():
    sys.path.insert(0, ROOT)
    from paper_2408_01081_gb300.slab import neighbours, slab_rows
    for ny in (2, 7, 11, 64, 8192):
        for world in range(1, min(ny, 9) + 1):
            spans = [slab_rows(ny, world, r) for r in range(world)]
            assert spans[0][0] == 0 and all(s[1] >= 1 for s in spans)
            assert all(spans[i][0] + spans[i][1] == spans[i + 1][0] for i in range(world - 1))
            assert spans[-1][0] + spans[-1][1] == ny
            assert max(s[1] for s in spans) - min(s[1] for s in spans) <= 1
    assert neighbours(3, 0, True) == (2, 1) and neighbours(3, 0, False) == (None, 1)
    assert neighbours(3, 2, False) == (1, None) and neighbours(2, 1, True) == (0, 0)
    assert neighbours(1, 0, True) == (0, 0) and neighbours(1, 0, False) == (None, None)
    with pytest.raises(ValueError):
        slab_rows(4, 5, 0)


def test_slab_creation_is_validated_before_any_device_work():
    """lbm_create_slab checks the row range and the storage format on the host."""
    sys.path.insert(0, ROOT)
    from paper_2408_01081_gb300 import build, lbm
    build.build()
    for y0, rows in [(-1, 3), (0, 0), (5, 4), (8, 1)]:
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create_slab(8, 8, 0.1, 0.01, 1.0, 0.5, y0, rows)
        assert e.value.status == lbm.LBM_ERR_ARG, (y0, rows)
    for st in (lbm.LBM_MS_BF16, lbm.LBM_MS_F16, lbm.LBM_MS_BFP):
        with pytest.raises(lbm.LbmError) as e:
            lbm.lbm_create_slab(8, 8, 0.1, 0.01, 1.0, 0.5, 0, 4, storage=st)
        assert e.value.status == lbm.LBM_ERR_ARG
