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


def test_nn_host_side_validation_and_counters(lib):
    """Surrogate-layer calls reject invalid arguments before any CUDA call, and the launch
    counters are host values (four of them, none negative)."""
    import ctypes
    from paper_2408_01081_gb300 import nn as K
    counts = K.conv_counts()
    assert len(counts) == 4 and all(c >= 0 for c in counts)
    so = K._lib()
    assert so.lbm_nn_conv_counts(None) == lib.LBM_ERR_ARG
    fake = ctypes.c_void_p(16)            # never dereferenced: validation fails first
    # forward: unknown flag bit, channel counts off the 32 grid, a missing second output
    assert so.lbm_nn_conv_forward(fake, 32, None, 0, fake, None, fake, 32, None, 32, 1, 16, 16, 3, 64,
                                  None) == lib.LBM_ERR_ARG
    assert so.lbm_nn_conv_forward(fake, 48, None, 0, fake, None, fake, 32, None, 32, 1, 16, 16, 3, 0,
                                  None) == lib.LBM_ERR_ARG
    assert so.lbm_nn_conv_forward(fake, 32, None, 0, fake, None, fake, 16, None, 32, 1, 16, 16, 3, 0,
                                  None) == lib.LBM_ERR_ARG
    assert so.lbm_nn_conv_forward(None, 32, None, 0, fake, None, fake, 32, None, 32, 1, 16, 16, 3, 0,
                                  None) == lib.LBM_ERR_ARG
    # weight gradient: forward-only flags, too small a workspace
    ws = K.wgrad_workspace_bytes(32, 32, 1, 16, 16, 3)
    assert ws > 0
    assert so.lbm_nn_conv_backward_weight(fake, 32, fake, 32, None, 0, 1, 16, 16, 3, fake, K.ACT_BF16, fake, ws,
                                          None) == lib.LBM_ERR_ARG
    assert so.lbm_nn_conv_backward_weight(fake, 32, fake, 32, None, 0, 1, 16, 16, 3, fake, 0, fake, ws - 4,
                                          None) == lib.LBM_ERR_ARG


def test_wgrad_workspace_holds_whole_partials(lib):
    """The weight-gradient workspace is a whole number of [Cout][KS*KS][Cin] FP32 partial
    sums, grows with the pixel count up to a cap on the splits, and covers at least one
    split for every size."""
    from paper_2408_01081_gb300 import nn as K
    for Cin, Cout, B, H, W, KS in [(32, 32, 16, 256, 256, 3), (96, 32, 16, 256, 256, 3), (384, 128, 16, 64, 64, 3),
                                   (32, 48, 2, 32, 16, 3), (32, 32, 2, 8, 16, 3), (64, 32, 4, 64, 64, 1)]:
        unit = Cout * KS * KS * Cin * 4
        ws = K.wgrad_workspace_bytes(Cin, Cout, B, H, W, KS)
        assert ws % unit == 0 and ws >= unit, (Cin, Cout, B, H, W, KS)
        assert ws // unit <= 4 * 152 + B * H * W // 1024 + 1


def test_binding_constants_match_the_headers(lib):
    """Every enumerator of include/*.h that the Python bindings mirror has the same value there
    (status codes, boundary and storage kinds, convolution flags)."""
    from paper_2408_01081_gb300 import nn as K
    values = {}
    for fn in ("lbm.h", "lbm_nn.h"):
        src = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", fn)).read(), flags=re.S)
        for body in re.findall(r"enum\s*\{(.*?)\}", src, flags=re.S):
            for name, val in re.findall(r"(LBM_\w+)\s*=\s*(\d+)", body):
                values[name] = int(val)
    assert len(values) >= 20, values
    checked = 0
    for name, v in values.items():
        if hasattr(lib, name):
            assert getattr(lib, name) == v, name
            checked += 1
        short = name[len("LBM_NN_"):] if name.startswith("LBM_NN_") else None
        if short and hasattr(K, short):
            assert getattr(K, short) == v, name
            checked += 1
    assert checked == len(values), (checked, sorted(values))


def test_noalloc_binding_checks_the_shape_before_any_call(lib):
    """lbm_energy_noalloc takes nx, ny apart from the buffer; the binding refuses a
    buffer whose shape is not (4, 5, ny, nx) before the C call (so before any launch)."""
    import torch
    short = torch.zeros((4, 5, 3, 8), dtype=torch.float64)          # ny = 3 rows, 96 asked for
    with pytest.raises(ValueError):
        lib.lbm_energy_noalloc(short, 8, 96, 0.1, 0.01, 1.0, 0.5)
    with pytest.raises(ValueError):
        lib.lbm_energy_noalloc(torch.zeros(20 * 8 * 96, dtype=torch.float64), 8, 96, 0.1, 0.01, 1.0, 0.5)
    good = torch.zeros((4, 5, 96, 8), dtype=torch.float64)
    with pytest.raises(ValueError):
        lib.lbm_energy_noalloc(good, 8, 96, 0.1, 0.01, 1.0, 0.5, out=torch.zeros(0, dtype=torch.float64))
    with pytest.raises(TypeError):                                  # right shape, but host memory
        lib.lbm_energy_noalloc(good, 8, 96, 0.1, 0.01, 1.0, 0.5)
