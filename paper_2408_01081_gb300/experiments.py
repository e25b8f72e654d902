"""The paper's numerical experiments (Sec. 6) run through the CUDA library.

* :func:`dirichlet_convergence` -- manufactured solution on (0, 2) x (0, 1) with
  u = u_hat on all edges and the body load of the Navier form, on lattices
  2N x N; spatial relative L2 / Linf errors of u and sigma at t_final and the
  observed orders between successive lattices.
* :func:`long_run` -- homogeneous Dirichlet, b = 0, the initial data of the
  energy test (Sec. 6.2) on a 2:1 rectangle; relative drift of ||f||_P.
* :func:`precision_errors` -- periodic lattice with a Gaussian-random initial
  velocity, every storage format run for the same number of steps; relative L2
  of each moment field against the FP64 run (which matches the CPU oracle to
  1e-12), and the step rate of each format.

Inputs come from :mod:`workloads` (exact separable tables for b and the wall
data, so nothing per step is built on the host); every step runs in the
library's kernels.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import lbm as L


def _exact_on_device(fields, nx, ny, dx, t, device):
    """Dense exact fields [len(fields), ny, nx] on the GPU from the separable form."""
    import torch
    xs = torch.tensor((np.arange(nx) + 0.5) * dx, dtype=torch.float64, device=device)
    ys = torch.tensor((np.arange(ny) + 0.5) * dx, dtype=torch.float64, device=device)
    out = torch.zeros((len(fields), ny, nx), dtype=torch.float64, device=device)
    for q, f in enumerate(fields):
        for (kx, ky), C in f.merged(t).items():
            bx = torch.stack([torch.sin(kx * xs), torch.cos(kx * xs)])
            by = torch.stack([torch.sin(ky * ys), torch.cos(ky * ys)])
            Ct = torch.tensor(C, dtype=torch.float64, device=device)
            out[q] += by.T @ Ct.T @ bx
    return out


def dirichlet_mms_run(ny, nu, storage="f64", t_final=0.5, cfl=0.9, amp=1e-2, kx=2 * math.pi, ky=2 * math.pi,
                      w=4 * math.pi, device="cuda"):
    """One lattice of the convergence sweep; returns errors at t_final and run statistics."""
    import torch
    from workloads import material, mms
    nx = 2 * ny
    dx = 1.0 / ny
    cK2, cmu2 = material.poisson_to_speeds(nu)
    c = material.lattice_speed(cK2, cmu2, cfl)
    dt = dx / c
    steps = int(round(t_final / dt))
    sol = mms.paper_moving_solution(math.sqrt(cK2), math.sqrt(cmu2), amp, kx, ky, w)
    dev = torch.device(device)
    U0 = _exact_on_device(sol.U_fields(), nx, ny, dx, 0.0, dev)
    Ux = _exact_on_device(sol.U_fields(p=1), nx, ny, dx, 0.0, dev)
    Uy = _exact_on_device(sol.U_fields(r=1), nx, ny, dx, 0.0, dev)
    u0 = _exact_on_device(sol.displacement(), nx, ny, dx, 0.0, dev)
    X, Y, T = mms.separable_tables(sol.body_load(), nx, ny, dx, np.arange(steps + 1) * dt)
    Xn, Xw, Yn, Yw, Tw = mms.separable_wall_tables(sol.velocity(), nx, ny, dx, (np.arange(steps) + 0.5) * dt)
    B0 = _exact_on_device(sol.body_load(), nx, ny, dx, 0.0, dev)
    lat = L.Lattice(nx, ny, dx, dt, math.sqrt(cK2), math.sqrt(cmu2), dirichlet=True, storage=storage,
                    track_displacement=True, stream=torch.cuda.current_stream().cuda_stream)
    try:
        lat.set_forcing(X, Y, T)
        lat.set_dirichlet_separable(Xn, Xw, Yn, Yw, Tw)
        lat.init(U0, Ux, Uy, B0, u0)
        del Ux, Uy, B0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat.step(steps)
        lat.synchronize()
        wall = time.perf_counter() - t0
        tf = steps * dt
        exact = _exact_on_device(sol.U_fields() + sol.displacement() + sol.stress(), nx, ny, dx, tf, dev)
        s = lat.error_sums(exact)
    finally:
        lat.close()
    sq_u, ref_u = s[0, 5:7].sum(), s[1, 5:7].sum()
    sq_s, ref_s = s[0, 7:10].sum(), s[1, 7:10].sum()
    return {"nx": nx, "ny": ny, "nu": nu, "storage": storage, "steps": steps, "t_final": tf,
            "u_L2rel": math.sqrt(sq_u / ref_u), "u_Linf": float(s[2, 5:7].max()),
            "sigma_L2rel": math.sqrt(sq_s / ref_s), "sigma_Linf": float(s[2, 7:10].max()),
            "wall_s": wall, "mlups": nx * ny * steps / wall / 1e6}


def orders(rows, key):
    return [math.log2(a[key] / b[key]) for a, b in zip(rows, rows[1:])]


def dirichlet_convergence(ny_list=(128, 256, 512, 1024, 2048, 4096), nus=(0.0, 0.25, 0.45, 0.49), storage="f64",
                          log=print, **kw):
    out = {}
    for nu in nus:
        rows = []
        for ny in ny_list:
            r = dirichlet_mms_run(ny, nu, storage, **kw)
            rows.append(r)
            if log:
                log(json.dumps(r))
        out[str(nu)] = {"rows": rows, "order_u_L2": orders(rows, "u_L2rel"), "order_u_Linf": orders(rows, "u_Linf"),
                        "order_sigma_L2": orders(rows, "sigma_L2rel"),
                        "order_sigma_Linf": orders(rows, "sigma_Linf")}
    return out


def long_run(steps=100_000, nx=512, ny=256, cK2=1.1, cmu2=0.4, cfl=None, dt=None, storage="f64", every=1000,
             device="cuda", split=None):
    """Homogeneous Dirichlet, b = 0, u0 = sin(4 pi x) sin(2 pi y) [sin(-0.4 pi), sin(1.6 pi)] on
    (0, nx dx) x (0, 1) with dx = 1/ny; max relative drift of ||f||_P over the run (FP64 at the
    library's default arithmetic, or at lbm_set_fp64_split level `split`)."""
    import torch
    from workloads import material, mms
    dx = 1.0 / ny
    if dt is None:
        dt = dx / material.lattice_speed(cK2, cmu2, cfl if cfl else 0.98)
    sol = mms.paper_energy_initial(math.sqrt(cK2), math.sqrt(cmu2))
    dev = torch.device(device)
    U0 = _exact_on_device(sol.U_fields(), nx, ny, dx, 0.0, dev)
    Ux = _exact_on_device(sol.U_fields(p=1), nx, ny, dx, 0.0, dev)
    Uy = _exact_on_device(sol.U_fields(r=1), nx, ny, dx, 0.0, dev)
    lat = L.Lattice(nx, ny, dx, dt, math.sqrt(cK2), math.sqrt(cmu2), dirichlet=True, storage=storage,
                    track_displacement=False, stream=torch.cuda.current_stream().cuda_stream)
    try:
        if split is not None:
            lat.set_fp64_split(split)
        lat.init(U0, Ux, Uy)
        e0 = math.sqrt(lat.energy())
        drift, done = 0.0, 0
        t0 = time.perf_counter()
        while done < steps:
            n = min(every, steps - done)
            lat.step(n)
            done += n
            drift = max(drift, abs(math.sqrt(lat.energy()) - e0) / e0)
        wall = time.perf_counter() - t0
        finite = lat.finite()
    finally:
        lat.close()
    return {"nx": nx, "ny": ny, "steps": steps, "storage": storage, "cK2": cK2, "cmu2": cmu2,
            "cfl_ratio": material.cfl_ratio(cK2, cmu2, dx / dt), "max_rel_energy_drift": drift, "finite": finite,
            "wall_s": wall}


def precision_errors(n=8192, steps=5000, formats=("f32", "bf16", "f16", "ms_bf16", "ms_f16", "ms_bfp"), seeds=(1, 2),
                     ell=64.0, std=1e-3, cK2=1.5, cmu2=0.5, cfl=0.9, every=1000, device="cuda", wl=None):
    """Relative L2 of v_x, v_y, j_s, j_d, j_xy at steps every, 2 every, ..., steps: each
    storage format against the FP64 run (kept as snapshots on the device).  ``wl``: the
    periodic GRF workload of size n x n if already generated."""
    import torch
    import workloads as W
    if wl is None:
        wl = W.grf_periodic(n, n, cK2, cmu2, cfl=cfl, ell=ell, std=std, seeds=seeds, steps=0)
    dev = torch.device(device)
    U0 = torch.from_numpy(wl.U0).to(dev)
    Ux = torch.from_numpy(wl.dU0dx).to(dev)
    Uy = torch.from_numpy(wl.dU0dy).to(dev)
    st = torch.cuda.current_stream()
    out = torch.empty((10, n, n), dtype=torch.float64, device=dev)
    checkpoints = list(range(every, steps + 1, every)) or [steps]
    names = ["v_x", "v_y", "j_s", "j_d", "j_xy"]
    res, ref = {}, {}
    for storage in ("f64",) + tuple(formats):
        lat = L.Lattice(n, n, wl.dx, wl.dt, wl.cK, wl.cmu, storage=storage, track_displacement=False,
                        stream=st.cuda_stream)
        lat.init(U0, Ux, Uy)
        row = {"rel_l2_vs_f64": {}}
        done, wall = 0, 0.0
        for cp in checkpoints:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            lat.step(cp - done)
            lat.synchronize()
            wall += time.perf_counter() - t0
            done = cp
            lat.moments(out)
            torch.cuda.synchronize()
            if storage == "f64":
                ref[cp] = out[0:5].clone()
            else:
                row["rel_l2_vs_f64"][cp] = {nm: float(torch.linalg.vector_norm(out[q] - ref[cp][q]) /
                                                      torch.linalg.vector_norm(ref[cp][q]))
                                            for q, nm in enumerate(names)}
        lat.close()
        row["mlups"] = n * n * done / wall / 1e6
        if storage == "f64":
            del row["rel_l2_vs_f64"]
        res[storage] = row
    return {"n": n, "steps": steps, "ell": ell, "std": std, "checkpoints": checkpoints, "formats": res}


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="convergence sweep and long run on the GPU")
    ap.add_argument("--what", default="all", choices=["all", "convergence", "longrun", "precision"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--every", type=int, default=1000)
    ap.add_argument("--storage", default="f64")
    ap.add_argument("--max-ny", type=int, default=4096)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = {}
    if a.what in ("all", "convergence"):
        nys = [n for n in (128, 256, 512, 1024, 2048, 4096) if n <= a.max_ny]
        res["convergence"] = dirichlet_convergence(nys, storage=a.storage)
    if a.what in ("all", "longrun"):
        res["longrun"] = [long_run(storage=a.storage)]
    if a.what == "precision":
        res["precision"] = precision_errors(n=a.n, steps=a.steps, every=a.every)
    txt = json.dumps(res, indent=1)
    if a.out:
        open(a.out, "w").write(txt)
    print(txt)
