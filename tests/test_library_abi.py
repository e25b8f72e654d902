"""Host-side checks of the C ABI (no GPU): the library builds, loads and exports
every symbol that include/lbm.h declares, and argument validation in lbm_create
(which runs before any CUDA call) returns the documented status codes."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lbm\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2408_01081_gb300 import build, lbm
    build.build()
    return lbm


def test_library_exports_every_declared_symbol(lib):
    so = lib.load()
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(so, n)]
    assert not missing, missing
    assert set(lib.EXPORTS) <= declared | {"lbm_last_error"}


def test_create_validates_arguments_before_touching_the_gpu(lib):
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_create(1, 8, 0.1, 0.01, 1.0, 0.5)
    assert e.value.status == lib.LBM_ERR_ARG
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_create(8, 8, 0.1, 0.01, 1.0, 0.5, storage=9)
    assert e.value.status == lib.LBM_ERR_ARG
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_create(8, 8, 0.1, 0.1 / 2.5, 1.0, 0.8)          # 2 sqrt(1.64) = 2.56 >= 2.5
    assert e.value.status == lib.LBM_ERR_CFL
    assert "CFL" in lib.lbm_last_error(None)


def test_create_rejects_sizes_beyond_the_limits(lib):
    for nx, ny in [(8, 65536), ((1 << 24) + 1, 8), (8, 1), (0, 8)]:
        with pytest.raises(lib.LbmError) as e:
            lib.lbm_create(nx, ny, 0.1, 0.01, 1.0, 0.5)
        assert e.value.status == lib.LBM_ERR_ARG, (nx, ny)
    with pytest.raises(lib.LbmError) as e:
        lib.lbm_create(8, 8, 0.1, 0.01, 1.0, -0.1)           # negative shear speed
    assert e.value.status == lib.LBM_ERR_ARG
