"""Row slabs on the GPU: one lattice split into slabs held by one process, halo rows
exchanged through lbm_halo_pack / lbm_halo_unpack every step (paper_2408_01081_gb300.slab),
must follow the single-lattice kernel bit for bit (the multi-rank exchange itself is
covered on CPU gloo ranks in test_multirank_slab.py)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _run_whole(lbm, nx, ny, f, steps, dirichlet, storage):
    lat = lbm.Lattice(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, dirichlet=dirichlet, storage=storage,
                      track_displacement=False)
    lat.set_step_fusion(1, 64)
    lat.set_populations(f)
    lat.step(steps)
    g = lat.populations()[0]
    e = lat.energy()
    lat.close()
    return g, e


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("dirichlet", [False, True])
@pytest.mark.parametrize("nslabs", [2, 3])
def test_slabs_follow_the_whole_lattice_bit_for_bit(lbm, storage, dirichlet, nslabs):
    from paper_2408_01081_gb300 import slab as S
    nx, ny, steps = 70, 23, 11
    rng = np.random.default_rng(nslabs * 10 + int(dirichlet))
    f = rng.standard_normal((4, 5, ny, nx)) * 1e-3
    ref, e_ref = _run_whole(lbm, nx, ny, f, steps, dirichlet, storage)
    slabs = []
    for r in range(nslabs):
        y0, rows = S.slab_rows(ny, nslabs, r)
        s = S.Slab(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, y0, rows, dirichlet=dirichlet, storage=storage)
        lbm.lbm_set_populations(s.ctx, np.ascontiguousarray(f[:, :, y0:y0 + rows, :]))
        slabs.append(s)
    S.step_local(slabs, steps)
    e_sum = 0.0
    for s in slabs:
        g = np.empty((4, 5, s.rows, nx))
        lbm.lbm_get_populations(s.ctx, g)
        np.testing.assert_array_equal(g, ref[:, :, s.y0:s.y0 + s.rows, :])
        e_sum += s.energy()
        s.close()
    assert abs(e_sum - e_ref) <= 1e-13 * abs(e_ref)


def test_slab_moments_and_message_rules(lbm):
    """Moments of a slab are its own rows of the lattice's moments; a message buffer is
    required exactly where the slab has a neighbour."""
    import torch
    from paper_2408_01081_gb300 import slab as S
    nx, ny = 40, 16
    rng = np.random.default_rng(3)
    f = rng.standard_normal((4, 5, ny, nx)) * 1e-3
    whole = lbm.Lattice(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, dirichlet=True, track_displacement=False)
    whole.set_populations(f)
    whole.step(5)
    ref = whole.moments()
    whole.close()
    slabs = [S.Slab(nx, ny, 0.1, 0.1 / 3.2, 1.0, 0.6, *S.slab_rows(ny, 2, r), dirichlet=True) for r in range(2)]
    for s in slabs:
        lbm.lbm_set_populations(s.ctx, np.ascontiguousarray(f[:, :, s.y0:s.y0 + s.rows, :]))
    S.step_local(slabs, 5)
    for s in slabs:
        np.testing.assert_array_equal(s.moments(), ref[:, s.y0:s.y0 + s.rows, :])
    bottom = slabs[0]
    assert bottom.to_lower is None and bottom.to_upper is not None
    assert lbm.lbm_halo_bytes(bottom.ctx) == 5 * nx * 8
    with pytest.raises(lbm.LbmError) as e:          # the bottom slab of a Dirichlet lattice has no lower neighbour
        lbm.lbm_halo_pack(bottom.ctx, torch.empty(5 * nx * 8, dtype=torch.uint8, device="cuda"), bottom.to_upper)
    assert e.value.status == lbm.LBM_ERR_ARG
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_halo_unpack(bottom.ctx, None, None)
    assert e.value.status == lbm.LBM_ERR_ARG
    for s in slabs:
        s.close()
