"""lbm_energy_noalloc: the weighted-norm reduction for callers that cannot
allocate device memory (their pool belongs to another allocator, or cudaFree's
device-wide synchronisation is not acceptable where they run).  It must agree
with the context-based lbm_energy on two calls in a row, and reject lattices
with more rows than its static scratch holds.  Collected last on purpose."""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_energy_matches_lbm_energy_on_two_calls(lbm):
    import torch
    wl = W.energy_box(96, 1.1, 0.4, 1.0 / 240.0, 0)
    lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=True, storage="f64",
                      track_displacement=False)
    lat.init(wl.U0, wl.dU0dx, wl.dU0dy)
    f = torch.empty((4, 5, wl.ny, wl.nx), dtype=torch.float64, device="cuda")
    out_dev = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call in range(2):
        if call:
            lat.step(37)
        lbm.lbm_get_populations(lat.ctx, f)
        ref = lat.energy()
        got = lbm.lbm_energy_noalloc(f, wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu)
        assert abs(got - ref) <= 1e-12 * abs(ref), (call, got, ref)
        lbm.lbm_energy_noalloc(f, wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, out=out_dev)
        torch.cuda.synchronize()
        assert abs(out_dev.item() - ref) <= 1e-12 * abs(ref)
    lat.close()


def test_noalloc_rejects_too_many_rows(lbm):
    import torch
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_energy_noalloc(f, 4, 16385, 0.1, 0.01, 1.0, 0.5)
    assert e.value.status == lbm.LBM_ERR_ARG
    assert "16384" in lbm.lbm_last_error(None)
