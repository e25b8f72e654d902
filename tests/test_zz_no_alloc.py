"""lbm_energy_noalloc: the weighted-norm reduction for callers that cannot
allocate device memory (their pool belongs to another allocator, or cudaFree's
device-wide synchronisation is not acceptable where they run).  It must agree
with the context-based lbm_energy on two calls in a row, and reject lattices
with more rows than its static scratch holds.

The file name sorts last so that a run stopping at the first failure has
already run every other test; each test here also passes alone in a fresh
process (the scratch needs no clearing, every row partial is rewritten)."""
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


def test_noalloc_at_the_row_limit_on_a_side_stream(lbm):
    """ny = 16384 (every scratch row in use, the result slot right after them) with a
    small nx, on a non-default stream; compared with lbm_energy of the same state."""
    import numpy as np
    import torch
    nx, ny = 6, 16384
    dx = 1.0 / ny
    cK, cmu = 1.1 ** 0.5, 0.4 ** 0.5
    dt = dx / (2.0 * (cK * cK + cmu * cmu) ** 0.5 / 0.9)
    side = torch.cuda.Stream()
    lat = lbm.Lattice(nx, ny, dx, dt, cK, cmu, dirichlet=False, storage="f64", track_displacement=False,
                      stream=side.cuda_stream)
    rng = np.random.default_rng(7)
    f0 = torch.from_numpy(rng.standard_normal((4, 5, ny, nx))).cuda()
    torch.cuda.synchronize()          # the copy ran on torch's stream, the context uses `side`
    lbm.lbm_set_populations(lat.ctx, f0, None, 0)
    lat.step(3)
    f = torch.empty((4, 5, ny, nx), dtype=torch.float64, device="cuda")
    lbm.lbm_get_populations(lat.ctx, f)
    ref = lat.energy()
    out_dev = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()          # the fill ran on torch's stream
    for _ in range(2):
        got = lbm.lbm_energy_noalloc(f, nx, ny, dx, dt, cK, cmu, stream=side.cuda_stream)
        assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
        lbm.lbm_energy_noalloc(f, nx, ny, dx, dt, cK, cmu, out=out_dev, stream=side.cuda_stream)
        side.synchronize()
        assert abs(out_dev.item() - ref) <= 1e-12 * abs(ref)
    lat.close()


def test_noalloc_rejects_too_many_rows(lbm):
    """The C entry point itself rejects ny beyond its scratch (called through the raw
    ctypes symbol, below the binding's shape check; nothing is launched)."""
    import ctypes
    import torch
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    v = ctypes.c_double()
    st = lbm.load().lbm_energy_noalloc(ctypes.c_void_p(f.data_ptr()), 4, 16385, 0.1, 0.01, 1.0, 0.5,
                                       ctypes.cast(ctypes.byref(v), ctypes.c_void_p), 0, ctypes.c_void_p(0))
    assert st == lbm.LBM_ERR_ARG
    assert "16384" in lbm.lbm_last_error(None)


def test_noalloc_rejects_host_memory_for_f(lbm):
    """A host pointer given as f is refused before any launch."""
    import ctypes
    import numpy as np
    f = np.zeros((4, 5, 2, 2))
    v = ctypes.c_double()
    st = lbm.load().lbm_energy_noalloc(ctypes.c_void_p(f.ctypes.data), 2, 2, 0.1, 0.01, 1.0, 0.5,
                                       ctypes.cast(ctypes.byref(v), ctypes.c_void_p), 0, ctypes.c_void_p(0))
    assert st == lbm.LBM_ERR_ARG
    assert "device memory" in lbm.lbm_last_error(None)
