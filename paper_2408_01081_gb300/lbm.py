"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every function keeps the C name.  Array arguments may be numpy arrays (host
memory) or torch CUDA tensors (device memory, passed by ``data_ptr``); FP64,
C-contiguous, in the layouts the header documents.  All arithmetic runs in the
CUDA library; nothing here computes on the data.  If the library has not been
built, :func:`load` raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from .build import LIB

LBM_OK, LBM_ERR_ARG, LBM_ERR_CFL, LBM_ERR_OOM, LBM_ERR_CUDA, LBM_ERR_UNSTABLE, LBM_ERR_TIMEOUT, LBM_ERR_STATE = range(8)
LBM_PERIODIC, LBM_DIRICHLET = 0, 1
LBM_F64, LBM_F32, LBM_BF16, LBM_F16, LBM_MS_BF16, LBM_MS_F16, LBM_MS_BFP = 0, 1, 2, 3, 4, 5, 6
STORAGE = {"f64": LBM_F64, "f32": LBM_F32, "bf16": LBM_BF16, "f16": LBM_F16, "ms_bf16": LBM_MS_BF16,
           "ms_f16": LBM_MS_F16, "ms_bfp": LBM_MS_BFP}
STATUS_NAMES = ["LBM_OK", "LBM_ERR_ARG", "LBM_ERR_CFL", "LBM_ERR_OOM", "LBM_ERR_CUDA", "LBM_ERR_UNSTABLE",
                "LBM_ERR_TIMEOUT", "LBM_ERR_STATE"]

# every symbol declared in include/lbm.h
EXPORTS = ["lbm_create", "lbm_init", "lbm_set_relaxation", "lbm_set_step_fusion", "lbm_set_staging", "lbm_set_fp64_split", "lbm_set_energy_check", "lbm_set_forcing", "lbm_set_dirichlet", "lbm_set_dirichlet_separable", "lbm_step", "lbm_moments",
           "lbm_energy", "lbm_error_sums", "lbm_get_populations", "lbm_set_populations", "lbm_check_finite",
           "lbm_time_step", "lbm_synchronize", "lbm_destroy", "lbm_last_error", "lbm_state_bytes",
           "lbm_save_state", "lbm_load_state", "lbm_energy_noalloc", "lbm_create_slab", "lbm_halo_bytes",
           "lbm_halo_pack", "lbm_halo_unpack", "lbm_batch_create", "lbm_batch_init",
           "lbm_batch_tune", "lbm_batch_set_mode", "lbm_batch_step", "lbm_batch_synchronize", "lbm_batch_moments",
           "lbm_batch_energy", "lbm_batch_info", "lbm_batch_set_barrier", "lbm_batch_destroy",
           "lbm_batch_last_error"]


class LbmParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("bc", ctypes.c_int32), ("storage", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("cK", ctypes.c_double), ("cmu", ctypes.c_double),
        ("track_displacement", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
    ]


class LatticeDesc(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("bc", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double), ("cK", ctypes.c_double), ("cmu", ctypes.c_double),
    ]


class LbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


_lib = None


def load(path: Optional[str] = None):
    """Load ``liblbm.so``; raises if it is missing (no fallback of any kind)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
    sig = {
        "lbm_create": ([ctypes.POINTER(LbmParams), ctypes.POINTER(vp)], i32),
        "lbm_init": ([vp, dp, dp, dp, dp, dp, i32], i32),
        "lbm_set_forcing": ([vp, i32, dp, dp, dp, i64, i32], i32),
        "lbm_set_relaxation": ([vp, ctypes.c_double], i32),
        "lbm_set_step_fusion": ([vp, i32, i32], i32),
        "lbm_set_staging": ([vp, i32], i32),
        "lbm_set_fp64_split": ([vp, i32], i32),
        "lbm_set_energy_check": ([vp, i32, ctypes.c_double], i32),
        "lbm_set_dirichlet": ([vp, dp, i64, i32], i32),
        "lbm_set_dirichlet_separable": ([vp, i32, dp, dp, dp, dp, dp, i64, i32], i32),
        "lbm_step": ([vp, i64], i32),
        "lbm_moments": ([vp, dp, i32], i32),
        "lbm_energy": ([vp, dp], i32),
        "lbm_error_sums": ([vp, dp, i32, dp], i32),
        "lbm_get_populations": ([vp, dp, dp, i32], i32),
        "lbm_set_populations": ([vp, dp, dp, i64, i32], i32),
        "lbm_check_finite": ([vp], i32),
        "lbm_time_step": ([vp, ctypes.POINTER(i64)], i32),
        "lbm_synchronize": ([vp], i32),
        "lbm_destroy": ([vp], i32),
        "lbm_last_error": ([vp], ctypes.c_char_p),
        "lbm_state_bytes": ([vp, ctypes.POINTER(i64)], i32),
        "lbm_save_state": ([vp, vp, i32], i32),
        "lbm_load_state": ([vp, vp, i64, i32], i32),
        "lbm_energy_noalloc": ([dp, i32, i32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, dp, i32, vp], i32),
        "lbm_create_slab": ([ctypes.POINTER(LbmParams), i32, i32, ctypes.POINTER(vp)], i32),
        "lbm_halo_bytes": ([vp, ctypes.POINTER(i64)], i32),
        "lbm_halo_pack": ([vp, vp, vp], i32),
        "lbm_halo_unpack": ([vp, vp, vp], i32),
        "lbm_batch_create": ([i32, ctypes.POINTER(LatticeDesc), i32, vp, ctypes.POINTER(vp)], i32),
        "lbm_batch_init": ([vp, i32, dp, dp, dp, i32], i32),
        "lbm_batch_tune": ([vp, ctypes.c_char_p], i32),
        "lbm_batch_set_mode": ([vp, i32, i32], i32),
        "lbm_batch_step": ([vp, i64], i32),
        "lbm_batch_synchronize": ([vp], i32),
        "lbm_batch_moments": ([vp, i32, dp, i32], i32),
        "lbm_batch_energy": ([vp, i32, dp], i32),
        "lbm_batch_info": ([vp, i32, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i32),
                            ctypes.POINTER(i32)], i32),
        "lbm_batch_set_barrier": ([vp, ctypes.c_double, i32], i32),
        "lbm_batch_destroy": ([vp], i32),
        "lbm_batch_last_error": ([vp], ctypes.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and hasattr(x, "data_ptr") and bool(x.is_cuda)


def _arr(x, name: str):
    """(pointer, on_device, keepalive) for an FP64 array argument or None."""
    if x is None:
        return None, None, None
    if _is_torch_cuda(x):
        import torch
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise TypeError(f"{name}: CUDA tensor must be contiguous float64")
        return ctypes.c_void_p(x.data_ptr()), 1, x
    a = np.ascontiguousarray(x, dtype=np.float64) if not (isinstance(x, np.ndarray) and x.dtype == np.float64
                                                          and x.flags.c_contiguous) else x
    return ctypes.c_void_p(a.ctypes.data), 0, a


def _where(*flags):
    fl = {f for f in flags if f is not None}
    if len(fl) > 1:
        raise TypeError("mix of host and device arrays in one call")
    return fl.pop() if fl else 0


def _check(ctx, st):
    if st != LBM_OK:
        msg = load().lbm_last_error(ctx).decode(errors="replace")
        raise LbmError(st, msg)


# ---------------------------------------------------------------------------
# the C calls, one wrapper each
# ---------------------------------------------------------------------------

def lbm_create(nx, ny, dx, dt, cK, cmu, bc=LBM_PERIODIC, storage=LBM_F64, track_displacement=False, stream=None):
    p = LbmParams(int(nx), int(ny), int(bc), int(storage), float(dx), float(dt), float(cK), float(cmu),
                  int(bool(track_displacement)), 0, ctypes.c_void_p(stream or 0))
    ctx = ctypes.c_void_p()
    st = load().lbm_create(ctypes.byref(p), ctypes.byref(ctx))
    _check(None, st)
    return ctx


def lbm_create_slab(nx, ny, dx, dt, cK, cmu, y_begin, rows, bc=LBM_PERIODIC, storage=LBM_F64,
                    track_displacement=False, stream=None):
    """Context for rows [y_begin, y_begin + rows) of an nx x ny lattice (see include/lbm.h)."""
    p = LbmParams(int(nx), int(ny), int(bc), int(storage), float(dx), float(dt), float(cK), float(cmu),
                  int(bool(track_displacement)), 0, ctypes.c_void_p(stream or 0))
    ctx = ctypes.c_void_p()
    _check(None, load().lbm_create_slab(ctypes.byref(p), int(y_begin), int(rows), ctypes.byref(ctx)))
    return ctx


def lbm_halo_bytes(ctx) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().lbm_halo_bytes(ctx, ctypes.byref(n)))
    return int(n.value)


def _dev_ptr(t, name):
    if t is None:
        return None
    if not _is_torch_cuda(t) or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def lbm_halo_pack(ctx, to_lower, to_upper):
    """Device tensors of lbm_halo_bytes bytes (or None where the slab has no neighbour)."""
    _check(ctx, load().lbm_halo_pack(ctx, _dev_ptr(to_lower, "to_lower"), _dev_ptr(to_upper, "to_upper")))


def lbm_halo_unpack(ctx, from_lower, from_upper):
    _check(ctx, load().lbm_halo_unpack(ctx, _dev_ptr(from_lower, "from_lower"), _dev_ptr(from_upper, "from_upper")))


def lbm_init(ctx, U0, dU0dx, dU0dy, B0=None, u0=None):
    a = [_arr(U0, "U0"), _arr(dU0dx, "dU0dx"), _arr(dU0dy, "dU0dy"), _arr(B0, "B0"), _arr(u0, "u0")]
    on = _where(*[t[1] for t in a])
    _check(ctx, load().lbm_init(ctx, *[t[0] for t in a], on))


def lbm_set_step_fusion(ctx, steps_per_pass=2, rows_per_block=0):
    _check(ctx, load().lbm_set_step_fusion(ctx, int(steps_per_pass), int(rows_per_block)))


def lbm_set_staging(ctx, mode=1):
    _check(ctx, load().lbm_set_staging(ctx, int(mode)))


def lbm_set_fp64_split(ctx, level):
    _check(ctx, load().lbm_set_fp64_split(ctx, int(level)))


def lbm_set_energy_check(ctx, every, growth=1.0 + 1e-9):
    _check(ctx, load().lbm_set_energy_check(ctx, int(every), float(growth)))


def lbm_set_relaxation(ctx, omega):
    _check(ctx, load().lbm_set_relaxation(ctx, float(omega)))


def lbm_set_forcing(ctx, X=None, Y=None, T=None):
    if X is None:
        _check(ctx, load().lbm_set_forcing(ctx, 0, None, None, None, 0, 0))
        return
    R, nt = int(X.shape[0]), int(T.shape[0])
    a = [_arr(X, "X"), _arr(Y, "Y"), _arr(T, "T")]
    on = _where(*[t[1] for t in a])
    _check(ctx, load().lbm_set_forcing(ctx, R, a[0][0], a[1][0], a[2][0], nt, on))


def lbm_set_dirichlet(ctx, g=None):
    if g is None:
        _check(ctx, load().lbm_set_dirichlet(ctx, None, 0, 0))
        return
    p, on, _keep = _arr(g, "g")
    _check(ctx, load().lbm_set_dirichlet(ctx, p, int(g.shape[0]), on))


def lbm_set_dirichlet_separable(ctx, Xn, Xw, Yn, Yw, T):
    a = [_arr(v, n) for v, n in ((Xn, "Xn"), (Xw, "Xw"), (Yn, "Yn"), (Yw, "Yw"), (T, "T"))]
    on = _where(*[t[1] for t in a])
    _check(ctx, load().lbm_set_dirichlet_separable(ctx, int(Xn.shape[0]), *[t[0] for t in a], int(T.shape[0]), on))


def lbm_step(ctx, n=1):
    _check(ctx, load().lbm_step(ctx, int(n)))


def lbm_moments(ctx, out):
    p, on, _keep = _arr(out, "out")
    if on == 0 and p.value != out.ctypes.data:
        raise TypeError("out must be a C-contiguous float64 numpy array or CUDA tensor")
    _check(ctx, load().lbm_moments(ctx, p, on))
    return out


def lbm_energy(ctx) -> float:
    v = ctypes.c_double()
    _check(ctx, load().lbm_energy(ctx, ctypes.cast(ctypes.byref(v), ctypes.c_void_p)))
    return float(v.value)


def lbm_error_sums(ctx, exact):
    p, on, _keep = _arr(exact, "exact")
    out = np.zeros(30)
    _check(ctx, load().lbm_error_sums(ctx, p, on, ctypes.c_void_p(out.ctypes.data)))
    return out.reshape(3, 10)


def lbm_get_populations(ctx, f, ustar=None):
    a, b = _arr(f, "f"), _arr(ustar, "ustar")
    on = _where(a[1], b[1])
    _check(ctx, load().lbm_get_populations(ctx, a[0], b[0], on))


def lbm_set_populations(ctx, f, ustar=None, m=0):
    a, b = _arr(f, "f"), _arr(ustar, "ustar")
    on = _where(a[1], b[1])
    _check(ctx, load().lbm_set_populations(ctx, a[0], b[0], int(m), on))


def lbm_check_finite(ctx) -> bool:
    st = load().lbm_check_finite(ctx)
    if st == LBM_ERR_UNSTABLE:
        return False
    _check(ctx, st)
    return True


def lbm_time_step(ctx) -> int:
    m = ctypes.c_int64()
    _check(ctx, load().lbm_time_step(ctx, ctypes.byref(m)))
    return int(m.value)


def lbm_synchronize(ctx):
    _check(ctx, load().lbm_synchronize(ctx))


def lbm_destroy(ctx):
    load().lbm_destroy(ctx)


def lbm_last_error(ctx=None) -> str:
    return load().lbm_last_error(ctx).decode(errors="replace")


def lbm_state_bytes(ctx) -> int:
    n = ctypes.c_int64()
    _check(ctx, load().lbm_state_bytes(ctx, ctypes.byref(n)))
    return int(n.value)


def lbm_save_state(ctx, dst):
    if _is_torch_cuda(dst):
        _check(ctx, load().lbm_save_state(ctx, ctypes.c_void_p(dst.data_ptr()), 1))
    else:
        _check(ctx, load().lbm_save_state(ctx, ctypes.c_void_p(dst.ctypes.data), 0))


def lbm_load_state(ctx, src, m):
    if _is_torch_cuda(src):
        _check(ctx, load().lbm_load_state(ctx, ctypes.c_void_p(src.data_ptr()), int(m), 1))
    else:
        _check(ctx, load().lbm_load_state(ctx, ctypes.c_void_p(src.ctypes.data), int(m), 0))


def lbm_energy_noalloc(f, nx, ny, dx, dt, cK, cmu, out=None, stream=None) -> float:
    """||f||_P^2 of device populations f [4, 5, ny, nx] without any device allocation.

    ``out``: optional 1-element float64 CUDA tensor to receive the result on the
    device (no wait); otherwise the value is returned through host memory.

    The C call takes nx and ny apart from the pointer and cannot see how large the
    buffer is, so the shape of ``f`` is checked here against (4, 5, ny, nx) before
    anything reaches the library: a short buffer would otherwise be read past its end.
    The call runs with the device that holds ``f`` current."""
    nx, ny = int(nx), int(ny)
    shape = tuple(getattr(f, "shape", ()))
    if shape != (4, 5, ny, nx):
        raise ValueError(f"f must have shape (4, 5, ny, nx) = (4, 5, {ny}, {nx}), got {shape}")
    if out is not None and (getattr(out, "numel", lambda: 0)() < 1):
        raise ValueError("out must hold at least one element")
    if not _is_torch_cuda(f):
        raise TypeError("f must be a CUDA tensor (device memory)")
    p, _, _keep = _arr(f, "f")
    import torch
    with torch.cuda.device(f.device):
        if out is not None:
            po, on, _k2 = _arr(out, "out")
            if on != 1 or out.device != f.device:
                raise TypeError("out must be a CUDA tensor on the device of f")
            _check(None, load().lbm_energy_noalloc(p, nx, ny, float(dx), float(dt), float(cK), float(cmu),
                                                   po, 1, ctypes.c_void_p(stream or 0)))
            return None
        v = ctypes.c_double()
        _check(None, load().lbm_energy_noalloc(p, nx, ny, float(dx), float(dt), float(cK), float(cmu),
                                               ctypes.cast(ctypes.byref(v), ctypes.c_void_p), 0,
                                               ctypes.c_void_p(stream or 0)))
    return float(v.value)


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------

def _bcheck(b, st):
    if st != LBM_OK:
        raise LbmError(st, load().lbm_batch_last_error(b).decode(errors="replace"))


def lbm_batch_create(descs, storage=LBM_F64, stream=None):
    """descs: iterable of (nx, ny, bc, dx, dt, cK, cmu)."""
    arr = (LatticeDesc * len(descs))()
    for i, (nx, ny, bc, dx, dt, cK, cmu) in enumerate(descs):
        arr[i] = LatticeDesc(int(nx), int(ny), int(bc), 0, float(dx), float(dt), float(cK), float(cmu))
    h = ctypes.c_void_p()
    st = load().lbm_batch_create(len(descs), arr, int(storage), ctypes.c_void_p(stream or 0), ctypes.byref(h))
    _bcheck(None, st)
    return h


def lbm_batch_init(b, index, U0, dU0dx, dU0dy):
    a = [_arr(U0, "U0"), _arr(dU0dx, "dU0dx"), _arr(dU0dy, "dU0dy")]
    on = _where(*[t[1] for t in a])
    _bcheck(b, load().lbm_batch_init(b, int(index), a[0][0], a[1][0], a[2][0], on))


def lbm_batch_tune(b, cache_path=None):
    _bcheck(b, load().lbm_batch_tune(b, None if cache_path is None else str(cache_path).encode()))


def lbm_batch_set_mode(b, mode, graph_steps=100):
    _bcheck(b, load().lbm_batch_set_mode(b, int(mode), int(graph_steps)))


def lbm_batch_step(b, n=1):
    _bcheck(b, load().lbm_batch_step(b, int(n)))


def lbm_batch_synchronize(b):
    _bcheck(b, load().lbm_batch_synchronize(b))


def lbm_batch_moments(b, index, out):
    p, on, _keep = _arr(out, "out")
    _bcheck(b, load().lbm_batch_moments(b, int(index), p, on))
    return out


def lbm_batch_energy(b, index) -> float:
    v = ctypes.c_double()
    _bcheck(b, load().lbm_batch_energy(b, int(index), ctypes.cast(ctypes.byref(v), ctypes.c_void_p)))
    return float(v.value)


def lbm_batch_info(b, index=0):
    n, sb = ctypes.c_int64(), ctypes.c_int64()
    nt, tw = ctypes.c_int32(), ctypes.c_int32()
    _bcheck(b, load().lbm_batch_info(b, int(index), ctypes.byref(n), ctypes.byref(sb), ctypes.byref(nt),
                                     ctypes.byref(tw)))
    return {"nodes": n.value, "state_bytes": sb.value, "ntiles": nt.value, "tile_width": tw.value}


def lbm_batch_set_barrier(b, timeout_s, extra_arrivals=0):
    _bcheck(b, load().lbm_batch_set_barrier(b, float(timeout_s), int(extra_arrivals)))


def lbm_batch_destroy(b):
    load().lbm_batch_destroy(b)


def lbm_batch_last_error(b=None) -> str:
    return load().lbm_batch_last_error(b).decode(errors="replace")


class Lattice:
    """Owns one context; methods forward to the C calls above."""

    def __init__(self, nx, ny, dx, dt, cK, cmu, dirichlet=False, storage="f64", track_displacement=True,
                 stream=None):
        self.nx, self.ny = int(nx), int(ny)
        self.ctx = lbm_create(nx, ny, dx, dt, cK, cmu, LBM_DIRICHLET if dirichlet else LBM_PERIODIC,
                              STORAGE[storage] if isinstance(storage, str) else storage, track_displacement,
                              stream)

    def close(self):
        if self.ctx is not None:
            lbm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, U0, dU0dx, dU0dy, B0=None, u0=None):
        lbm_init(self.ctx, U0, dU0dx, dU0dy, B0, u0)

    def set_step_fusion(self, steps_per_pass=2, rows_per_block=0):
        lbm_set_step_fusion(self.ctx, steps_per_pass, rows_per_block)

    def set_staging(self, mode=1):
        lbm_set_staging(self.ctx, mode)

    def set_fp64_split(self, level):
        lbm_set_fp64_split(self.ctx, level)

    def set_energy_check(self, every, growth=1.0 + 1e-9):
        lbm_set_energy_check(self.ctx, every, growth)

    def set_relaxation(self, omega):
        lbm_set_relaxation(self.ctx, omega)

    def set_forcing(self, X=None, Y=None, T=None):
        lbm_set_forcing(self.ctx, X, Y, T)

    def set_dirichlet(self, g=None):
        lbm_set_dirichlet(self.ctx, g)

    def set_dirichlet_separable(self, Xn, Xw, Yn, Yw, T):
        lbm_set_dirichlet_separable(self.ctx, Xn, Xw, Yn, Yw, T)

    def step(self, n=1):
        lbm_step(self.ctx, n)

    def moments(self, out=None):
        if out is None:
            out = np.empty((10, self.ny, self.nx))
        return lbm_moments(self.ctx, out)

    def energy(self) -> float:
        return lbm_energy(self.ctx)

    def error_sums(self, exact):
        return lbm_error_sums(self.ctx, exact)

    def populations(self):
        f = np.empty((4, 5, self.ny, self.nx))
        us = np.empty((2, self.ny, self.nx))
        lbm_get_populations(self.ctx, f, us)
        return f, us

    def set_populations(self, f, ustar=None, m=0):
        lbm_set_populations(self.ctx, f, ustar, m)

    def finite(self) -> bool:
        return lbm_check_finite(self.ctx)

    @property
    def m(self) -> int:
        return lbm_time_step(self.ctx)

    def synchronize(self):
        lbm_synchronize(self.ctx)
