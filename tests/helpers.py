"""Shared test helpers: run a workload through the oracle or the CUDA library."""
from __future__ import annotations

import numpy as np

from oracle import Oracle, Params
from oracle.postprocess import rel_l2


def oracle_run(wl, steps=None, track=True):
    steps = wl.steps if steps is None else steps
    o = Oracle(Params(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, wl.dirichlet))
    o.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
    for m in range(steps):
        o.step(wl.body_load(m), wl.wall_data(m), track_displacement=track)
    return o, o.outputs(wl.body_load(steps))


def gpu_lattice(lbm, wl, storage="f64", track=True):
    lat = lbm.Lattice(wl.nx, wl.ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=wl.dirichlet, storage=storage,
                      track_displacement=track)
    if wl.forcing is not None:
        lat.set_forcing(*wl.forcing)
    if wl.dirichlet and wl.wall is not None:
        lat.set_dirichlet(wl.wall)
    lat.init(wl.U0, wl.dU0dx, wl.dU0dy, wl.body_load(0), wl.u0)
    return lat


def field_errors(a, b, fields=range(10)):
    return [rel_l2(a[q], b[q]) for q in fields]
