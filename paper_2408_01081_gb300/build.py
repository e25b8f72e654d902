"""Build the CUDA library ``liblbm.so`` in-tree for sm_103a (GB300).

One translation unit per storage format (FP64, FP32, BF16, FP16 and the three
moment-space formats) plus the host API, compiled in parallel with nvcc and linked into a shared library with the C
ABI of ``include/lbm.h``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include"), "-I", CSRC]


def _nvcc() -> str:
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cuh", ".h"))] + [os.path.join(ROOT, "include", "lbm.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force: bool = False, verbose: bool = False, out: str = None, defines=()) -> str:
    """Compile and link the library; ``out``/``defines`` build a tuning variant elsewhere."""
    lib = out or LIB
    if not force and out is None and up_to_date():
        return LIB
    build_dir = os.path.dirname(lib) if out else BUILD
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    dflags = [f"-D{d}" for d in defines]
    units = [(os.path.join(CSRC, "lbm_kind.cu"), os.path.join(build_dir, f"lbm_kind{k}.o"),
              [f"-DLBM_KIND={k}"] + dflags) for k in range(7)]
    extra = [f for f in sorted(os.listdir(CSRC)) if f.endswith(".cu") and f != "lbm_kind.cu"]
    units += [(os.path.join(CSRC, f), os.path.join(build_dir, f[:-3] + ".o"), dflags) for f in extra]
    procs = []
    for src, obj, defs in units:
        cmd = [nvcc] + ARCH + FLAGS + defs + ["-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((cmd, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join(" ".join(c) + "\n" + o for c, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    tmp = lib + f".tmp{os.getpid()}"
    link = [nvcc] + ARCH + ["-shared", "-o", tmp] + [obj for _, obj, _ in units] + ["-lcudart"]
    r = subprocess.run(link, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
