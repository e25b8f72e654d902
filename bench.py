#!/usr/bin/env python3
"""Benchmark of the fused D2Q4^5 collide-stream step on GB300.

Workload (one step = one fused collide-stream kernel over the whole lattice):
periodic 8192 x 8192 lattice at rest with a Gaussian random initial velocity
(correlation length 64 cells, std 1e-3, seeds 1 and 2), cK^2 = 1.5, cmu^2 = 0.5
(lambda = 1, mu = 0.5), time step at 0.9 of the CFL-like bound, b = 0.

Main line: the FP64 path (MLUPS).  Also reported: the FP32 / BF16 / FP16
storage paths (MLUPS, speed-up over FP64, relative L2 error of every moment
field against the FP64 run after the same number of steps), the roofline of the
dominant kernel, an end-to-end figure through the C ABI with host buffers, the
SM clocks seen during the timed region, and the FP64 oracle timed on the host
cores on a bounded sample.

``--impl reference`` times the FP64 oracle (the only reference this paper has:
it ships no code) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = 8192
CK2, CMU2, CFL = 1.5, 0.5, 0.9
ELL, STD = 64.0, 1e-3
METRIC = "MLUPS and % of HBM roofline; mixed-precision vs FP64 at stated L2 error"
BYTES_PER_NODE = {"f64": 320, "f32": 160, "bf16": 80, "f16": 80,    # one read + one write of 20 values
                  "ms_bf16": 100, "ms_f16": 100, "ms_bfp": 100}    # 5 FP32 + 15 16-bit moments, read + write
FP64_OPS_PER_NODE = 47                                                # DADD/DFMA per node, no forcing
SPLIT_LEVEL = 12              # lbm_set_fp64_split default: the node update in exact fixed-point arithmetic
SPLIT_IEEE = 1                # the IEEE binary64 operation sequence with its 15 sums on the integer pipe
ARITHMETIC = ("binary64 state; per node exact 64-bit fixed-point arithmetic on the integer pipes (inputs as "
              "multiples of 2^-57 of the node's largest, 7 products rounded there) and one round-to-nearest-even "
              "conversion to binary64 per output (lbm_set_fp64_split level 12)")
# steps per launch of each format at the library's defaults (lbm_set_step_fusion)
STEPS_PER_PASS = {"f64": 1, "f32": 3, "bf16": 3, "f16": 3, "ms_bf16": 3, "ms_f16": 3, "ms_bfp": 3}
# DRAM bytes per node and launch of each step kernel (dram__bytes_read.sum + dram__bytes_write.sum
# from one ncu capture of this benchmark's own 8192^2 workload, averaged over its launches; no
# scaling), valid only while the kernel sources hash to "sha256".  "<fmt>_fused" is one launch of
# the two-step kernel (two steps), "<fmt>_fused3" of the three-step kernel, "f64_pipe" the FP64
# step with every operation on the FP64 pipe.
TRAFFIC_CAPTURE = {"sha256": "427275c0b852342612482484dcd6605f8b9ba6a8e2209f6534469d96ebb1a946",
                   "nodes": 8192 * 8192,
                   "bytes_per_node": {"f64": 319.23, "f64_ieee": 322.79, "f64_pipe": 319.26, "f32_fused3": 164.66,
                                      "bf16_fused3": 83.32, "f16_fused3": 83.33, "ms_bf16_fused3": 105.1,
                                      "ms_f16_fused3": 105.11, "ms_bfp_fused3": 105.2}}
KERNEL_SOURCES = ["paper_2408_01081_gb300/csrc/lbm_kernels.cuh", "paper_2408_01081_gb300/csrc/lbm_kind.cu",
                  "paper_2408_01081_gb300/csrc/lbm_tb.cuh", "paper_2408_01081_gb300/csrc/lbm_ms.cuh",
                  "paper_2408_01081_gb300/csrc/lbm_tbt.cuh", "paper_2408_01081_gb300/csrc/lbm_tma.cuh",
                  "paper_2408_01081_gb300/csrc/lbm_f64emu.cuh", "paper_2408_01081_gb300/csrc/lbm_mscodec.cuh",
                  "paper_2408_01081_gb300/csrc/lbm_f64stage.cuh", "paper_2408_01081_gb300/csrc/lbm_f64fx.cuh"]
# Pipe instruction counts of the default FP64 step kernel (step_f64_staged_kernel, split level 12) per node
# (thread instructions: 32 x smsp__inst_executed_pipe_{alu,fp64,fma}.sum / nodes from one ncu
# capture of 4096x2048),
# valid only while the kernel sources hash to "sha256".  Each SM issues 64 ALU-pipe and 2
# FP64-pipe thread instructions per clock, so one node needs at least
# max(alu / 64, fp64 / 2) SM clocks: the arithmetic roof of this kernel.
PIPE_CAPTURE = {"sha256": "427275c0b852342612482484dcd6605f8b9ba6a8e2209f6534469d96ebb1a946",
                "alu_per_node": 586.3, "fp64_per_node": 20.0, "fma_per_node": 188.4}
ALU_LANES_PER_SM, FP64_LANES_PER_SM, N_SM = 64, 2, 152


def kernel_digest():
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, rel), "rb").read())
    return h.hexdigest()


def pipe_counts():
    """(alu, fp64, fma) thread instructions per node of the FP64 step kernel, or None."""
    if PIPE_CAPTURE["sha256"] is None or PIPE_CAPTURE["sha256"] != kernel_digest():
        return None
    return PIPE_CAPTURE["alu_per_node"], PIPE_CAPTURE["fp64_per_node"], PIPE_CAPTURE["fma_per_node"]


def traffic_per_launch(fmt, nodes):
    """Measured DRAM bytes of one launch, or None when the sources changed since the capture or
    the lattice is not the captured one (traffic has a fixed L2-resident part, so it is not
    scaled to other sizes)."""
    if TRAFFIC_CAPTURE["sha256"] != kernel_digest() or nodes != TRAFFIC_CAPTURE["nodes"]:
        return None
    bpn = TRAFFIC_CAPTURE["bytes_per_node"].get(fmt)
    return None if bpn is None else round(bpn * nodes)


def _workload_desc(nx, ny):
    return (f"periodic {nx}x{ny} lattice at rest, Gaussian random initial velocity (ell={ELL:g} cells, "
            f"std={STD:g}, seeds 1,2), cK^2={CK2}, cmu^2={CMU2} (lambda=1, mu=0.5), dt at {CFL} of the CFL bound, b=0")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(v, dist=None, device="cpu"):
    """Largest value over the ranks of the process group (v itself without one)."""
    if dist is None:
        return v
    import torch
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, seconds_per_rank, dist=None, device="cpu"):
    """Units all ranks processed divided by the slowest rank's time (the job's wall time)."""
    ws = dist.get_world_size() if dist is not None else 1
    return units_per_rank * ws / reduce_max(seconds_per_rank, dist, device)


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            p = [s.strip() for s in line.split(",")]
            if len(p) >= 9:
                rows.append(p)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def make_inputs(nx, ny):
    import workloads as W
    wl = W.grf_periodic(nx, ny, CK2, CMU2, cfl=CFL, ell=ELL, std=STD, seeds=(1, 2), steps=0)
    return wl


def _cpu_oracle_mlups(nx, ny, steps, threads=None, warmup=1):
    """Time the FP64 oracle (as it stands) on the host cores: MLUPS, threads used."""
    import oracle
    from oracle import Oracle, Params
    oracle.build()
    if threads:
        oracle.set_threads(threads)
    wl = make_inputs(nx, ny)
    o = Oracle(Params(nx, ny, wl.dx, wl.dt, wl.cK, wl.cmu, False))
    o.init(wl.U0, wl.dU0dx, wl.dU0dy, None, wl.u0)
    for _ in range(max(1, warmup)):
        o.step(track_displacement=False)   # warm caches and thread pool, untimed
    t0 = time.perf_counter()
    for _ in range(steps):
        o.step(track_displacement=False)
    dt = time.perf_counter() - t0
    return nx * ny * steps / dt / 1e6, oracle.max_threads(), dt


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    # bounded sample of the same workload: a 512 x 512 periodic lattice of the same kind
    nx = ny = 512
    t0 = time.perf_counter()
    mlups, threads, _ = _cpu_oracle_mlups(nx, ny, args.steps, warmup=args.warmup)
    wall = time.perf_counter() - t0
    line = {"metric": METRIC, "value": round(mlups, 3), "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(1e3 * nx * ny / (mlups * 1e6), 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": _workload_desc(NX, NY), "sample": f"{nx}x{ny} lattice of the same workload"},
            "impl": "reference",
            "cpu_baseline": {"value": round(mlups, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
                             "sample": f"FP64 C oracle, {nx}x{ny} periodic GRF lattice, {args.steps} steps"},
            "e2e": {"value": round(mlups, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": round(wall, 2)}
    print(json.dumps(line), flush=True)


def batch_accounting(mode, storage, descs, steps, ntiles_one_step):
    """(algorithmic bytes per node and step, launches, tiles) of `steps` batch steps in `mode`
    for lattices descs = [(nx, ny, bc, ...)], graphs of 100 steps.

    Bytes: one read and one write of the state per launch (FP32 160 B per node, FP64 320); mode 2
    runs 33 three-step passes and one single step per 100 steps.  Launches: mode 1 one per graph,
    mode 2 two per pass (periodic and Dirichlet tiles) and one per single step, mode 3 one per step
    and boundary kind present (every lattice of the benchmark's workload has cK/c and cmu/c in
    [2^-60, 1/2), so all take the fixed-point update, whose lists are the two used).  Tiles: the
    library's one-step work-list (modes 0 and 1, `ntiles_one_step`), else the mode's own tiles,
    112 x 12 in mode 2 (FP32) and 128 x 4 in mode 3."""
    passes, singles = (steps // 3, steps % 3) if mode == 2 else (0, steps)
    bpn = (320 if storage == "f64" else 160) * (passes + singles) / steps
    kinds = len({d[2] for d in descs})
    launches = {1: steps // 100, 2: 2 * passes + singles, 3: kinds * steps}.get(mode, steps)
    tile_shape = {2: (112, 12), 3: (128, 4)}.get(mode)
    tiles = ntiles_one_step if tile_shape is None else sum(
        math.ceil(d[0] / tile_shape[0]) * math.ceil(d[1] / tile_shape[1]) for d in descs)
    return bpn, launches, tiles


def run_batch(args, lbm, torch, stream, dev, max_over_ranks, barrier, ws):
    """512 ragged lattices (config 4 of the workload set), FP32 (or FP64), graph of 100 steps per replay."""
    import workloads as W
    from workloads.grf import batch_lattice_inputs_torch
    spec = W.batch_spec(count=args.batch_count)
    descs = []
    for sp in spec:
        c = W.material.lattice_speed(sp.cK2, sp.cmu2, CFL)
        dx = 1.0 / max(sp.nx, sp.ny)
        descs.append((sp.nx, sp.ny, int(sp.dirichlet), dx, dx / c, sp.cK2 ** 0.5, sp.cmu2 ** 0.5))
    nodes = sum(d[0] * d[1] for d in descs)
    storage = args.batch_storage
    b = lbm.lbm_batch_create(descs, storage=lbm.STORAGE[storage], stream=stream.cuda_stream)
    cache = os.path.join(ROOT, "paper_2408_01081_gb300", "_build", "tune_cache.txt")
    t0 = time.perf_counter()
    if args.batch_mode < 0:
        lbm.lbm_batch_tune(b, cache)
    tune_s = time.perf_counter() - t0
    for i, (sp, d) in enumerate(zip(spec, descs)):
        U0, Ux, Uy = batch_lattice_inputs_torch(sp, d[3], device=dev)
        lbm.lbm_batch_init(b, i, U0, Ux, Uy)
    del U0, Ux, Uy
    mode = _batch_mode(cache, storage) if args.batch_mode < 0 else args.batch_mode
    lbm.lbm_batch_set_mode(b, mode, 100)
    lbm.lbm_batch_step(b, 100)
    lbm.lbm_batch_synchronize(b)
    barrier()
    steps = 200
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    lbm.lbm_batch_step(b, steps)
    e1.record(stream)
    lbm.lbm_batch_synchronize(b)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1)) / steps
    info = lbm.lbm_batch_info(b, 0)
    lbm.lbm_batch_destroy(b)
    peaks = _peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    bpn, launches, tiles = batch_accounting(mode, storage, descs, steps, info["ntiles"])
    ach = bpn * nodes / (ms * 1e-3) / 1e9
    label = {"f32": "FP32", "f64": "FP64"}[storage]
    return {"workload": f"{args.batch_count} lattices, short side log-uniform [64,1024], aspect U[1,4], nu U[0,0.49], "
                        "even periodic / odd homogeneous Dirichlet, GRF v0 (ell = short side/16, std 1e-3), "
                        f"{label} storage, CUDA graph of 100 steps per replay",
            "nodes": nodes, "steps": steps, "ms_per_step": round(ms, 4),
            "mlups": round(nodes * ws / (ms * 1e-3) / 1e6, 1),
            "mode": {0: "launch per step", 1: "persistent",
                     2: "three steps per pass (tiles with staged rows), one launch each for periodic and "
                        "Dirichlet tiles",
                     3: "FP64 tiles with staged rows, one launch per step each for periodic and Dirichlet "
                        "tiles"}[mode],
            "graph_replays": steps // 100, "gpu_launches": launches,
            "tiles": tiles, "tune_s": round(tune_s, 2),
            "hbm": {"achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s", "frac": round(ach / hbm_peak, 4),
                    "bytes_per_node_step": round(bpn, 2)}}


def run_surrogate(args):
    """U-Net jump of 32 steps on 256^2 periodic lattices: train within a time budget on fresh
    solver trajectories, then held-out error and wall-clock against the solver on this GPU."""
    import torch
    from paper_2408_01081_gb300 import surrogate as S
    t0 = time.perf_counter()
    chunks = lambda i: S.generate_chunk(256, 10_000 + i, H=256, W=256, k=32, J=4)
    sur, hist = S.train(chunks, 1000, batch=8, H=256, W=256, lr=1e-3, k=32, time_budget_s=args.surrogate_budget)
    train_s = time.perf_counter() - t0
    held = S.generate_chunk(64, 900_000, H=256, W=256, k=32, J=4)
    errs, pers = S.evaluate(sur, held, batch=16)
    errs_fast, _ = S.evaluate(sur, held, batch=16, act_bf16=True)
    tm = S.timing(sur, n=16, H=256, W=256)
    drv = S.driver_timing(sur, held, check_every=(1, 4, 16), tol=1e-3, storage="f32", n=16)
    for v in drv.values():
        v["net_gain_vs_f32"] = round(tm["lbm_f32_ms_per_lattice"] / v["ms_per_lattice_jump"], 3)
        v["net_gain_vs_f64"] = round(tm["lbm_f64_ms_per_lattice"] / v["ms_per_lattice_jump"], 3)
    del held
    torch.cuda.empty_cache()
    med = float(np.median(errs))
    return {"workload": "256^2 periodic lattices, GRF v0 (ell 16-64 cells), nu U[0,0.49], jump of 32 steps, "
                        "4-level U-Net (1.96 M params, BF16 weights, FP32 accumulate)",
            "train_s": round(train_s, 1), "iterations": sur.net.step_count, "batch": 8,
            "heldout_rel_l2_median": med, "heldout_rel_l2_max": float(np.max(errs)),
            "persistence_rel_l2_median": float(np.median(pers)),
            "fallback_tol": 1e-3, "falls_back": bool(med > 1e-3),
            "surrogate_ms_per_lattice": round(tm["surrogate_ms_per_lattice"], 4),
            "lbm_f64_ms_per_lattice": round(tm["lbm_f64_ms_per_lattice"], 4),
            "lbm_f32_ms_per_lattice": round(tm["lbm_f32_ms_per_lattice"], 4),
            "gain_vs_f64": round(tm["gain_vs_f64"], 3), "gain_vs_f32": round(tm["gain_vs_f32"], 3),
            "driver": {"what": "whole fallback-driver jumps per lattice (batch 16): inference + FP32 solver check "
                               "every N jumps + fallback copies, keyed by N; net gain = solver ms / driver ms",
                       "by_check_interval": drv},
            "bf16_activations": {"heldout_rel_l2_median": float(np.median(errs_fast)),
                                 "surrogate_ms_per_lattice": round(tm["surrogate_bf16_act_ms_per_lattice"], 4),
                                 "gain_vs_f64": round(tm["gain_bf16_act_vs_f64"], 3),
                                 "gain_vs_f32": round(tm["gain_bf16_act_vs_f32"], 3)}}


def _batch_mode(cache, storage="f32"):
    """Launch mode the tuner stored for this storage format on this GPU (0 if unknown)."""
    try:
        for line in open(cache):
            if f"|{storage}|mode|" in line:
                mode = int(line.rsplit("|", 1)[1])
        return mode
    except Exception:
        return 0


def run_ours(args):
    import torch
    from paper_2408_01081_gb300 import lbm

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    lbm.load()
    nx, ny = args.nx, args.ny
    wl = make_inputs(nx, ny)
    n_nodes = nx * ny
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)
    U0 = torch.from_numpy(wl.U0).to(dev)
    Ux = torch.from_numpy(wl.dU0dx).to(dev)
    Uy = torch.from_numpy(wl.dU0dy).to(dev)

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return reduce_max(v, dist, dev)

    results = {}
    finals = {}
    clocks = None
    for storage in args.formats:
        lat = lbm.Lattice(nx, ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=False, storage=storage,
                          track_displacement=False, stream=stream.cuda_stream)
        if args.no_fusion:
            lat.set_step_fusion(1)
        elif storage in args.fuse_formats:
            lat.set_step_fusion(2, args.rows_per_block)
        lat.set_staging(args.staging)
        lat.init(U0, Ux, Uy)
        lat.step(args.warmup)
        barrier()
        clk = Clocks(local) if storage == "f64" else None
        if clk:
            clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lat.step(args.steps)
        e1.record(stream)
        barrier()
        if clk:
            clocks = clk.stop()
        ms = max_over_ranks(e0.elapsed_time(e1))
        out = torch.empty((10, ny, nx), dtype=torch.float64, device=dev)
        lat.moments(out)
        torch.cuda.synchronize()
        finals[storage] = out[0:5].clone()
        del out
        lat.close()
        mlups_rank = n_nodes * args.steps / (ms * 1e-3) / 1e6
        spp = 1 if args.no_fusion else (2 if storage in args.fuse_formats else STEPS_PER_PASS[storage])
        if args.staging == 0 and spp > 1:
            # without staged rows the population formats pair steps in registers; moment space steps singly
            spp = 1 if storage.startswith("ms_") else 2
        results[storage] = {"ms_per_step": ms / args.steps, "mlups": mlups_rank * ws, "steps_per_pass": spp,
                            "launches": args.steps // spp + (1 if args.steps % spp else 0)}

    # N > 1: one lattice of nx x (N ny) rows split into row slabs, one per rank, with the halo
    # exchange of the streaming step (5 values per column and cut each way) over NCCL every
    # step; every rank's slab starts from the same periodic tile, so the global initial field
    # is the tile repeated N times along y (smooth and periodic, weak scaling)
    slabs = None
    if ws > 1 and args.multi == "slabs":
        from paper_2408_01081_gb300 import slab as SL
        sl = SL.DistributedSlab(dist, nx, ny * ws, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=False, storage="f64",
                                track_displacement=False)
        sl.init(U0, Ux, Uy)
        sl.step(args.warmup)
        barrier()
        clk = Clocks(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sl.step(args.steps)
        e1.record(stream)
        barrier()
        clocks = clk.stop()
        ms = max_over_ranks(e0.elapsed_time(e1))
        sl.close()
        slabs = {"ms_per_step": ms / args.steps, "mlups": n_nodes * ws * args.steps / (ms * 1e-3) / 1e6,
                 "global_lattice": f"{nx}x{ny * ws}", "rows_per_rank": ny,
                 "halo_bytes_per_step_per_cut_each_way": 5 * nx * 8,
                 "launches_per_step": 3, "exchange": "NCCL send/recv (torch.distributed.batch_isend_irecv)"}

    # for reference: the IEEE binary64 operation sequence of the node update with its 15 sums on
    # the integer pipe (split level 1, bit-identical to the FP64 pipe) and with every operation on
    # the FP64 pipe (split level 0)
    if "f64" in args.formats:
        k0 = min(args.steps, 100)
        for key, level in (("f64_ieee_sequence", SPLIT_IEEE), ("f64_pipe_only", 0)):
            lat = lbm.Lattice(nx, ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=False, storage="f64",
                              track_displacement=False, stream=stream.cuda_stream)
            lat.set_fp64_split(level)
            lat.set_staging(args.staging)
            lat.init(U0, Ux, Uy)
            lat.step(args.warmup)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            lat.step(k0)
            e1.record(stream)
            barrier()
            ms0 = max_over_ranks(e0.elapsed_time(e1))
            lat.close()
            results[key] = {"split_level": level, "mlups": round(n_nodes * k0 / (ms0 * 1e-3) / 1e6 * ws, 1),
                            "ms_per_step": round(ms0 / k0, 4), "steps": k0}

    # relative L2 of every moment field against the FP64 run after the same steps
    ref = finals.get("f64")
    names = ["v_x", "v_y", "j_s", "j_d", "j_xy"]
    for s in args.formats:
        if s == "f64" or ref is None:
            continue
        err = {}
        for q, nm in enumerate(names):
            num = torch.linalg.vector_norm(finals[s][q] - ref[q]).item()
            den = torch.linalg.vector_norm(ref[q]).item()
            err[nm] = num / den if den > 0 else num
        results[s]["rel_l2_vs_f64"] = err
        results[s]["speedup_vs_f64"] = results[s]["mlups"] / results["f64"]["mlups"]
    del finals

    # end to end through the C ABI with host buffers: H2D of the initial data from pinned
    # memory, init, K steps, D2H of the ten output fields, all inside the timed region
    e2e = None
    if not args.no_e2e:
        hU0 = torch.from_numpy(wl.U0).pin_memory()
        hUx = torch.from_numpy(wl.dU0dx).pin_memory()
        hUy = torch.from_numpy(wl.dU0dy).pin_memory()
        hout = torch.empty((10, ny, nx), dtype=torch.float64).pin_memory()
        lat = lbm.Lattice(nx, ny, wl.dx, wl.dt, wl.cK, wl.cmu, dirichlet=False, storage="f64",
                          track_displacement=False, stream=stream.cuda_stream)
        barrier()
        t0 = time.perf_counter()
        lat.init(hU0.numpy(), hUx.numpy(), hUy.numpy())
        lat.step(args.steps)
        lat.moments(hout.numpy())
        barrier()
        wall = max_over_ranks(time.perf_counter() - t0)
        lat.close()
        h2d = 3 * 5 * n_nodes * 8
        d2h = 10 * n_nodes * 8
        e2e = {"value": round(n_nodes * args.steps * ws / wall / 1e6, 2), "unit": "MLUPS",
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps,
               "wall_s": round(wall, 3)}
        del hU0, hUx, hUy, hout

    # untimed: every storage format against the FP64 run over the workload's 5000 steps, errors
    # of every moment field at each checkpoint (the precision configuration of the workload set)
    precision = None
    if args.precision_steps > 0 and len(args.formats) > 1:
        from paper_2408_01081_gb300 import experiments as X
        del U0, Ux, Uy
        torch.cuda.empty_cache()
        t0 = time.perf_counter()
        precision = X.precision_errors(n=nx, steps=args.precision_steps, every=args.precision_every,
                                       formats=tuple(s for s in args.formats if s != "f64"), ell=ELL, std=STD,
                                       cK2=CK2, cmu2=CMU2, cfl=CFL, wl=wl if nx == ny else None)
        precision["wall_s"] = round(time.perf_counter() - t0, 1)
        torch.cuda.empty_cache()

    batch = None
    if not args.no_batch:
        batch = run_batch(args, lbm, torch, stream, dev, max_over_ranks, barrier, ws)

    surrogate = None
    if not args.no_surrogate and rank == 0:
        surrogate = run_surrogate(args)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    peaks = _peaks()
    hbm_peak = peaks["hbm_gbs"] if peaks else 6800.0
    peak_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6.8 TB/s (of fallback)"
    r64 = results["f64"]
    nodes_per_s = n_nodes / (r64["ms_per_step"] * 1e-3)
    hbm_ach = BYTES_PER_NODE["f64"] * nodes_per_s / 1e9
    sm_mhz = (clocks or {}).get("sm_mhz") or 2032.0
    # FP64 pipe: 2 DFMA/DADD per SM per clock on GB300 (measured 601.6 G DFMA/s at ~1.98 GHz)
    fp64_peak = 152 * 2 * sm_mhz * 1e6 / 1e9
    hbm_part = {"bound": "hbm", "achieved": round(hbm_ach, 1), "peak": hbm_peak, "unit": "GB/s",
                "frac": round(hbm_ach / hbm_peak, 4), "bytes_per_node": BYTES_PER_NODE["f64"],
                "peak_source": peak_src}
    hbm_node_peak = hbm_peak * 1e9 / BYTES_PER_NODE["f64"]
    # the captured counts and traffic describe the default (staged) FP64 step kernel only
    pc = pipe_counts() if args.staging >= 1 else None
    arith = None
    if pc is not None:
        # arithmetic roof: SM clocks per node = max(ALU-pipe / 64, FP64-pipe / 2) thread instructions
        alu_pn, fp64_pn, fma_pn = pc
        clk_pn = max(alu_pn / ALU_LANES_PER_SM, fp64_pn / FP64_LANES_PER_SM)
        node_peak = N_SM * sm_mhz * 1e6 / clk_pn
        arith = {"alu_inst_per_node": alu_pn, "fp64_inst_per_node": fp64_pn, "fma_inst_per_node": fma_pn,
                 "sm_clocks_per_node": round(clk_pn, 3), "node_rate_peak_G_per_s": round(node_peak / 1e9, 3),
                 "node_rate_achieved_G_per_s": round(nodes_per_s / 1e9, 3),
                 "frac": round(nodes_per_s / node_peak, 4),
                 "hbm_node_rate_peak_G_per_s": round(hbm_node_peak / 1e9, 3),
                 "source": "ncu pipe instruction counts of this kernel x 152 SMs x median SM clock sampled in "
                           "the timed region"}
    if arith is not None and arith["node_rate_peak_G_per_s"] * 1e9 < hbm_node_peak:
        alu_bound = arith["alu_inst_per_node"] / ALU_LANES_PER_SM >= arith["fp64_inst_per_node"] / FP64_LANES_PER_SM
        inst_pn, lanes = ((arith["alu_inst_per_node"], ALU_LANES_PER_SM) if alu_bound else
                          (arith["fp64_inst_per_node"], FP64_LANES_PER_SM))
        roofline = {"bound": "alu", "achieved": round(inst_pn * nodes_per_s / 1e9, 1),
                    "peak": round(N_SM * lanes * sm_mhz * 1e6 / 1e9, 1),
                    "unit": "G ALU-pipe inst/s" if alu_bound else "G FP64-pipe inst/s",
                    "frac": arith["frac"], "model": arith, "hbm": hbm_part}
    else:
        roofline = dict(hbm_part)
        if arith is not None:
            roofline["arithmetic_roof"] = arith
    ieee = results.get("f64_ieee_sequence")
    if ieee is not None:
        ieee = dict(ieee, hbm_frac=round(BYTES_PER_NODE["f64"] * ieee["mlups"] * 1e6 / 1e9 / hbm_peak, 4),
                    note="the IEEE binary64 operation sequence (bit-identical to the FP64 pipe), its 15 sums "
                         "as exact binary64 additions on the integer pipe; bound by the FP64 and integer pipes")
    roofline.update({"traffic": args.traffic if args.traffic is not None else
                     (traffic_per_launch("f64", n_nodes) if args.staging >= 1 else None),
                     "kernel": (f"lbmk::step_f64_staged_kernel<periodic,split level {SPLIT_LEVEL}> (fixed-point "
                                f"node update; rows staged by asynchronous copies)" if args.staging >= 1 else
                                f"lbmk::step_kernel<F64,1,periodic,split level {SPLIT_LEVEL}>"),
                     "compute": {"arithmetic": ARITHMETIC,
                                 "fp64_pipe_ops_per_node": 20,
                                 "fp64_pipe_use": "the 20 conversions of the outputs to binary64",
                                 "fp64_pipe_peak": round(fp64_peak, 2), "unit": "GFP64op/s",
                                 "fp64_pipe_frac": round(20 * nodes_per_s / 1e9 / fp64_peak, 4),
                                 "fp64_pipe_peak_source": "152 SMs x 2 FP64 ops/clk x median SM clock sampled "
                                                          "in the timed region",
                                 "ieee_sequence": ieee, "fp64_pipe_only": results.get("f64_pipe_only")}})
    mixed = {}
    for s in args.formats:
        if s == "f64":
            continue
        r = results[s]
        nps = n_nodes / (r["ms_per_step"] * 1e-3)
        bpn = round(BYTES_PER_NODE[s] / r["steps_per_pass"], 3)   # algorithmic bytes per node and step
        ach = bpn * nps / 1e9
        mixed[s] = {"mlups": round(r["mlups"], 1), "ms_per_step": round(r["ms_per_step"], 4),
                    "speedup_vs_f64": round(r["speedup_vs_f64"], 3), "steps_per_pass": r["steps_per_pass"],
                    "launches": r["launches"],
                    "hbm": {"achieved": round(ach, 1), "peak": hbm_peak, "unit": "GB/s",
                            "frac": round(ach / hbm_peak, 4), "bytes_per_node_step": bpn,
                            "traffic": (traffic_per_launch({1: s, 2: s + "_fused", 3: s + "_fused3"}[r["steps_per_pass"]],
                                                           n_nodes) if args.staging >= 1 else None)},
                    "rel_l2_vs_f64_after_timed_run": {k: float(f"{v:.3e}") for k, v in r["rel_l2_vs_f64"].items()},
                    "timed_run_error_at_step": args.warmup + args.steps}
        if precision is not None and s in precision["formats"]:
            by_step = precision["formats"][s]["rel_l2_vs_f64"]
            mixed[s]["rel_l2_vs_f64"] = {str(cp): {k: float(f"{v:.3e}") for k, v in e.items()}
                                         for cp, e in by_step.items()}
            mixed[s]["max_rel_l2_vs_f64"] = {str(cp): float(f"{max(e.values()):.3e}") for cp, e in by_step.items()}
            last = max(by_step)
            mixed[s]["meets_1e-5_at_step"] = {str(last): bool(max(by_step[last].values()) <= 1e-5)}
    cpu = None
    if ws == 1 and not args.no_cpu:
        cx = cy = 1024
        mlups_cpu, threads, wall = _cpu_oracle_mlups(cx, cy, args.cpu_steps)
        cpu = {"value": round(mlups_cpu, 3), "unit": "MLUPS", "cores": threads, "kind": "oracle",
               "sample": f"FP64 C oracle, {cx}x{cy} periodic lattice of the same workload, "
                         f"{args.cpu_steps} steps ({wall:.1f} s)"}
    head = slabs if slabs is not None else r64
    line = {"metric": METRIC, "value": round(head["mlups"], 1), "unit": "MLUPS", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(head["ms_per_step"], 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "arithmetic": ARITHMETIC, "data": "synthetic",
            "config": {"workload": _workload_desc(nx, ny) + (
                           f"; {ws} row slabs of one {nx}x{ny * ws} lattice (the tile repeated along y)"
                           if slabs is not None else ""),
                       "nodes": n_nodes * (ws if slabs is not None else 1), "storage": "f64",
                       "parallelism": ("row slabs, NCCL halo exchange" if slabs is not None else
                                       "replicas" if ws > 1 else "single"),
                       "l2": f"inputs larger than L2: state {2 * 20 * n_nodes * 8 / 1e9:.1f} GB double-buffered"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": 3 * args.steps if slabs is not None else args.steps, "slabs": slabs,
            "clocks": clocks, "mixed_precision": mixed, "batch": batch, "surrogate": surrogate,
            "precision_run": None if precision is None else
            {"workload": _workload_desc(nx, ny), "steps": precision["steps"], "checkpoints": precision["checkpoints"],
             "reference": "FP64 GPU run of the same workload (tied to the oracle at <= 1e-12 by the parity tests)",
             "mlups_untimed": {k: round(v["mlups"], 1) for k, v in precision["formats"].items()},
             "wall_s": precision["wall_s"]}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=NX)
    ap.add_argument("--ny", type=int, default=NY)
    ap.add_argument("--formats", default="f64,f32,bf16,f16,ms_bf16,ms_f16,ms_bfp")
    ap.add_argument("--multi", default="slabs", choices=["slabs", "replicas"],
                    help="N > 1: FP64 line as row slabs of one lattice (halo exchange) or independent replicas")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-fusion", action="store_true", help="one kernel per step for every format")
    ap.add_argument("--fuse-formats", default="", help="formats advanced two steps per pass besides the default")
    ap.add_argument("--staging", type=int, default=1,
                    help="1: rows staged in shared memory (tensor copies for the multi-step kernels, asynchronous "
                         "copies for the FP64 step), 0: register loads")
    ap.add_argument("--rows-per-block", type=int, default=0, help="two-step kernel rows per block (0: library default)")
    ap.add_argument("--batch-count", type=int, default=512, help="lattices in the batch leg")
    ap.add_argument("--batch-mode", type=int, default=-1,
                    help="batch launch mode (0, 1, 2 for FP32, 3 for FP64); -1: the autotuner's choice")
    ap.add_argument("--batch-storage", default="f32", choices=["f32", "f64"],
                    help="storage of the batch leg (the workload's figure is FP32)")
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--surrogate-budget", type=float, default=60.0, help="surrogate training seconds")
    ap.add_argument("--cpu-steps", type=int, default=100)
    ap.add_argument("--precision-steps", type=int, default=5000,
                    help="untimed run of every format against FP64 (0: skip)")
    ap.add_argument("--precision-every", type=int, default=1000)
    ap.add_argument("--traffic", type=float, default=None,
                    help="DRAM bytes per launch of the step kernel from an ncu capture (null if unknown)")
    args = ap.parse_args()
    args.formats = [s for s in args.formats.split(",") if s]
    args.fuse_formats = [s for s in args.fuse_formats.split(",") if s]
    if "f64" not in args.formats:
        args.formats.insert(0, "f64")
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
