"""FP64 CPU oracle of the vectorial LBM for 2D linear elastodynamics (arXiv 2408.01081).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports, links or executes anything here, and
this package imports nothing from the CUDA library.

Contents
--------
* ``lbm_oracle.c`` -- the scheme itself in plain C (Sec. 3, summary in Sec. 3.6),
  loaded through ctypes by :class:`Oracle`.
* :mod:`oracle.matrix_form` -- the paper's matrix form of one step (Sec. 5.1,
  Eq. stability_linear; the Dirichlet rule Eqs. bc_ansatz-bc_q), used to build the
  brute-force one-step operator on tiny lattices and the symmetrizer k_ij.
* :mod:`oracle.postprocess` -- displacement, stress and the error norms (Sec. 3.5,
  Sec. 6.1).

Parity pins: see ``tests/test_oracle_*.py``.  Every oracle function is pinned
by at least one check that does not restate its own formula.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sysconfig
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "liblbm_oracle.so")


def build(force: bool = False) -> str:
    """Compile ``lbm_oracle.c`` with gcc (FP64, no FMA contraction, OpenMP if available)."""
    os.makedirs(_BUILD_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    cc = os.environ.get("CC", "gcc")
    base = [cc, "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    try:
        subprocess.run(base + ["-fopenmp", _SRC, "-o", tmp, "-lm"], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + [_SRC, "-o", tmp, "-lm"], check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
        ("dirichlet", ctypes.c_int32), ("pad_", ctypes.c_int32),
        ("dx", ctypes.c_double), ("dt", ctypes.c_double),
        ("cK", ctypes.c_double), ("cmu", ctypes.c_double),
        ("omega", ctypes.c_double), ("W", ctypes.c_double),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Params)
        lib.orc_step.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        lib.orc_step.restype = None
        lib.orc_init.argtypes = [pp, dp, dp, dp, dp, dp]
        lib.orc_init.restype = None
        lib.orc_moments.argtypes = [pp, dp, dp, dp]
        lib.orc_moments.restype = None
        lib.orc_equilibrium.argtypes = [pp, dp, ctypes.c_int, dp]
        lib.orc_equilibrium.restype = None
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        lib.orc_set_threads.restype = None
        lib.orc_max_threads.argtypes = []
        lib.orc_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


@dataclass
class Params:
    """Lattice and material parameters (dimensionless, Sec. 2.3 / 3.1)."""
    nx: int
    ny: int
    dx: float
    dt: float
    cK: float          # c~_K
    cmu: float         # c~_mu
    dirichlet: bool = False
    omega: float = 2.0
    W: float = 0.125   # forcing weight W_ij; enters only when omega != 2

    @property
    def c(self) -> float:
        return self.dx / self.dt

    def _c(self) -> _Params:
        return _Params(self.nx, self.ny, int(self.dirichlet), 0, self.dx, self.dt,
                       self.cK, self.cmu, self.omega, self.W)


class Oracle:
    """Holds one lattice's pre-collision populations f(x, t) and the helper u*.

    The time-dependent data are passed per step by the caller:
    ``B`` = body load [2, ny, nx] at the step's time t, ``g`` = d/dt u_D at the
    wall midpoints at t + dt/2 as [2, 2(nx+ny)] in the order
    [left rows | right rows | bottom columns | top columns].
    """

    def __init__(self, p: Params):
        self.p = p
        self._cp = p._c()
        n = p.nx * p.ny
        self.f = np.zeros((4, 5, p.ny, p.nx))
        self._f2 = np.zeros_like(self.f)
        self._fs = np.zeros_like(self.f)
        self.ustar = np.zeros((2, p.ny, p.nx))
        self.m = 0  # step counter, t = m dt
        del n

    # -- Eq. ic_second ---------------------------------------------------
    def init(self, U0, dU0dx, dU0dy, B0=None, u0=None):
        p = self.p
        U0 = np.ascontiguousarray(U0, dtype=np.float64)
        dU0dx = np.ascontiguousarray(dU0dx, dtype=np.float64)
        dU0dy = np.ascontiguousarray(dU0dy, dtype=np.float64)
        B0c = None if B0 is None else np.ascontiguousarray(B0, dtype=np.float64)
        _load().orc_init(ctypes.byref(self._cp), _ptr(U0), _ptr(dU0dx), _ptr(dU0dy),
                         _ptr(B0c), _ptr(self.f))
        # u*(0) = u0 - dt/2 v^num(0), so that u^num(0) = u0 (Eq. trapezoidal, step 1(b))
        U = self.moments(B0c)
        base = np.zeros((2, p.ny, p.nx)) if u0 is None else np.asarray(u0, dtype=np.float64)
        self.ustar = np.ascontiguousarray(base - 0.5 * p.dt * U[0:2])
        self.m = 0

    def set_state(self, f, ustar=None, m=0):
        self.f = np.ascontiguousarray(f, dtype=np.float64).copy()
        if ustar is not None:
            self.ustar = np.ascontiguousarray(ustar, dtype=np.float64).copy()
        self.m = m

    # -- one step (Sec. 3.6) ---------------------------------------------
    def step(self, B=None, g=None, track_displacement=True):
        Bc = None if B is None else np.ascontiguousarray(B, dtype=np.float64)
        gc = None if g is None else np.ascontiguousarray(g, dtype=np.float64)
        us = self.ustar if track_displacement else None
        _load().orc_step(ctypes.byref(self._cp), _ptr(self.f), _ptr(self._f2), _ptr(Bc),
                         _ptr(gc), _ptr(us), _ptr(self._fs))
        self.f, self._f2 = self._f2, self.f
        self.m += 1

    def moments(self, B=None):
        """U^num = sum f + dt/2 B at the current time, [5, ny, nx] (Eq. cond_eq)."""
        out = np.empty((5, self.p.ny, self.p.nx))
        Bc = None if B is None else np.ascontiguousarray(B, dtype=np.float64)
        _load().orc_moments(ctypes.byref(self._cp), _ptr(self.f), _ptr(Bc), _ptr(out))
        return out

    def energy(self) -> float:
        """||f||_P^2 = sum_x sum_ij f_ij^T k_ij f_ij with k_ij = g_ij^{-1}
        (Definition grid_norm, Eq. def_symmetrizer).  Node contributions are summed
        with an exactly rounded sum so the reduction adds no drift of its own."""
        from .matrix_form import symmetrizer_blocks
        k = symmetrizer_blocks(self.p.cK, self.p.cmu, self.p.c)
        per_node = np.einsum("dayx,dab,dbyx->yx", self.f, k, self.f, optimize=False)
        return math.fsum(per_node.ravel().tolist())

    def equilibrium(self, U, d):
        out = np.empty(5)
        U = np.ascontiguousarray(U, dtype=np.float64)
        _load().orc_equilibrium(ctypes.byref(self._cp), _ptr(U), int(d), _ptr(out))
        return out

    def outputs(self, B=None):
        """The ten output fields at the current time (Sec. 3.5).

        [v_x, v_y, j_s, j_d, j_xy, u_x, u_y, sigma_xx, sigma_yy, sigma_xy]
        """
        from .postprocess import outputs_from_moments
        U = self.moments(B)
        return outputs_from_moments(U, self.ustar, self.p.dt, self.p.cK, self.p.cmu)
