"""ctypes binding of ``include/lbm_nn.h`` (argument marshalling only).

Buffers are torch CUDA tensors; every function forwards to the C call of the
same name with the tensors' device pointers and the current CUDA stream.
"""
from __future__ import annotations

import ctypes

from . import lbm as _lbm

EXPORTS = ["lbm_nn_conv_forward", "lbm_nn_check", "lbm_nn_conv_counts", "lbm_nn_wgrad_workspace_bytes", "lbm_nn_conv_backward_weight",
           "lbm_nn_bias_grad_workspace_bytes", "lbm_nn_bias_grad",
           "lbm_nn_weight_flip", "lbm_nn_relu_backward", "lbm_nn_pool", "lbm_nn_pool_backward", "lbm_nn_upsample",
           "lbm_nn_upsample_backward", "lbm_nn_mse", "lbm_nn_adam", "lbm_nn_to_bf16", "lbm_nn_pack_input",
           "lbm_nn_pack_target", "lbm_nn_residual_output", "lbm_nn_gradient"]

_done = False


def _lib():
    global _done
    lib = _lbm.load()
    if not _done:
        vp, i32, i64, f32, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
        sig = {
            "lbm_nn_conv_forward": [vp, i32, vp, i32, vp, vp, vp, i32, vp, i32, i32, i32, i32, i32, i32, vp],
            "lbm_nn_check": [vp],
            "lbm_nn_conv_counts": [vp],
            "lbm_nn_wgrad_workspace_bytes": [i32, i32, i32, i32, i32, i32],
            "lbm_nn_conv_backward_weight": [vp, i32, vp, i32, vp, i32, i32, i32, i32, i32, vp, i32, vp, i64, vp],
            "lbm_nn_bias_grad_workspace_bytes": [i64, i32],
            "lbm_nn_bias_grad": [vp, i64, i32, vp, vp, i64, vp],
            "lbm_nn_weight_flip": [vp, i32, i32, i32, vp, vp],
            "lbm_nn_relu_backward": [vp, vp, i64, vp],
            "lbm_nn_pool": [vp, i32, i32, i32, i32, vp, vp],
            "lbm_nn_pool_backward": [vp, i32, i32, i32, i32, vp, i32, vp],
            "lbm_nn_upsample": [vp, i32, i32, i32, i32, vp, vp],
            "lbm_nn_upsample_backward": [vp, i32, i32, i32, i32, vp, i32, vp],
            "lbm_nn_mse": [vp, vp, i64, i32, i32, f32, vp, vp, vp, vp],
            "lbm_nn_adam": [vp, vp, vp, vp, i64, f32, f32, f32, f32, i64, vp, vp],
            "lbm_nn_to_bf16": [vp, i64, vp, vp],
            "lbm_nn_pack_input": [vp, i64, i32, vp, vp, i32, i32, i32, i32, vp, vp],
            "lbm_nn_pack_target": [vp, vp, i64, i32, vp, i32, i32, i32, i32, vp, vp],
            "lbm_nn_residual_output": [vp, i64, vp, i32, vp, i32, i32, i32, i32, vp, i64, vp],
            "lbm_nn_gradient": [vp, i64, i32, i32, i32, i32, f64, vp, vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = i64 if name.endswith("_workspace_bytes") else i32
        _done = True
    return lib


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _s():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ok(name, st):
    if st != 0:
        raise _lbm.LbmError(st, f"{name} failed")


RELU, ACCUMULATE, X1_HALF, ACT_BF16, MMA_SYNC, WGRAD_PER_TAP = 1, 2, 4, 8, 16, 32     # flags of include/lbm_nn.h


_mma_sync_default = False


def use_mma_sync(on: bool) -> None:
    """Route 3x3 forward convolutions through the mma.sync kernels instead of the tcgen05
    kernel (same arithmetic, other summation order; for comparisons)."""
    global _mma_sync_default
    _mma_sync_default = bool(on)


def conv_forward(x1, C1, x2, C2, w_bf16, bias, y1, Co1, y2, Cout, B, H, W, KS, relu=False, beta=False,
                 x1_half=False, act_bf16=False, mma_sync=None):
    if mma_sync is None:
        mma_sync = _mma_sync_default
    flags = (RELU if relu else 0) | (ACCUMULATE if beta else 0) | (X1_HALF if x1_half else 0) | \
        (ACT_BF16 if act_bf16 else 0) | (MMA_SYNC if mma_sync else 0)
    _ok("lbm_nn_conv_forward", _lib().lbm_nn_conv_forward(_p(x1), C1, _p(x2), C2, _p(w_bf16), _p(bias), _p(y1), Co1,
                                                          _p(y2), Cout, B, H, W, KS, flags, _s()))


def check():
    """Synchronise the current stream; raises LbmError(LBM_ERR_TIMEOUT) if a bounded wait in a
    tcgen05 convolution ran out since the last check."""
    _ok("lbm_nn_check", _lib().lbm_nn_check(_s()))


def conv_counts():
    """Launches since the library was loaded: (forward tcgen05, forward mma.sync, weight gradient
    block-tiled, weight gradient per tap)."""
    out = (ctypes.c_int64 * 4)()
    _ok("lbm_nn_conv_counts", _lib().lbm_nn_conv_counts(ctypes.cast(out, ctypes.c_void_p)))
    return tuple(int(v) for v in out)


def wgrad_workspace_bytes(Cin, Cout, B, H, W, KS) -> int:
    return int(_lib().lbm_nn_wgrad_workspace_bytes(Cin, Cout, B, H, W, KS))


def conv_backward_weight(dy, Cout, x1, C1, x2, C2, B, H, W, KS, dw, workspace, beta=False, x1_half=False,
                         per_tap=False):
    flags = (ACCUMULATE if beta else 0) | (X1_HALF if x1_half else 0) | (WGRAD_PER_TAP if per_tap else 0)
    _ok("lbm_nn_conv_backward_weight",
        _lib().lbm_nn_conv_backward_weight(_p(dy), Cout, _p(x1), C1, _p(x2), C2, B, H, W, KS, _p(dw), flags,
                                           _p(workspace), workspace.numel() * workspace.element_size(), _s()))


def bias_grad_workspace_bytes(P, C) -> int:
    return int(_lib().lbm_nn_bias_grad_workspace_bytes(P, C))


def bias_grad(dy, P, C, db, workspace):
    _ok("lbm_nn_bias_grad", _lib().lbm_nn_bias_grad(_p(dy), P, C, _p(db), _p(workspace),
                                                    workspace.numel() * workspace.element_size(), _s()))


def weight_flip(w_bf16, Cout, Cin, KS, wt_bf16):
    _ok("lbm_nn_weight_flip", _lib().lbm_nn_weight_flip(_p(w_bf16), Cout, Cin, KS, _p(wt_bf16), _s()))


def relu_backward(dy, y):
    _ok("lbm_nn_relu_backward", _lib().lbm_nn_relu_backward(_p(dy), _p(y), dy.numel(), _s()))


def pool(x, B, H, W, C, y):
    _ok("lbm_nn_pool", _lib().lbm_nn_pool(_p(x), B, H, W, C, _p(y), _s()))


def pool_backward(dy, B, H, W, C, dx, beta=False):
    _ok("lbm_nn_pool_backward", _lib().lbm_nn_pool_backward(_p(dy), B, H, W, C, _p(dx), int(beta), _s()))


def upsample(x, B, H, W, C, y):
    _ok("lbm_nn_upsample", _lib().lbm_nn_upsample(_p(x), B, H, W, C, _p(y), _s()))


def upsample_backward(dy, B, H, W, C, dx, beta=False):
    _ok("lbm_nn_upsample_backward", _lib().lbm_nn_upsample_backward(_p(dy), B, H, W, C, _p(dx), int(beta), _s()))


def mse(out, tgt, P, C, cvalid, grad_scale, dout, workspace, loss_out):
    _ok("lbm_nn_mse", _lib().lbm_nn_mse(_p(out), _p(tgt), P, C, cvalid, float(grad_scale), _p(dout), _p(workspace),
                                        _p(loss_out), _s()))


def adam(w, g, m, v, lr, beta1, beta2, eps, step, w_bf16=None):
    _ok("lbm_nn_adam", _lib().lbm_nn_adam(_p(w), _p(g), _p(m), _p(v), w.numel(), float(lr), float(beta1),
                                          float(beta2), float(eps), int(step), _p(w_bf16), _s()))


def to_bf16(x, y):
    _ok("lbm_nn_to_bf16", _lib().lbm_nn_to_bf16(_p(x), x.numel(), _p(y), _s()))


def pack_input(U, sample_stride, nf, scale, extra, B, H, W, C, x):
    _ok("lbm_nn_pack_input", _lib().lbm_nn_pack_input(_p(U), sample_stride, nf, _p(scale), _p(extra), B, H, W, C,
                                                      _p(x), _s()))


def pack_target(Unow, Unext, sample_stride, nf, scale, B, H, W, C, t):
    _ok("lbm_nn_pack_target", _lib().lbm_nn_pack_target(_p(Unow), _p(Unext), sample_stride, nf, _p(scale), B, H, W,
                                                        C, _p(t), _s()))


def residual_output(Uin, in_stride, net, C, scale, nf, B, H, W, Uout, out_stride):
    _ok("lbm_nn_residual_output", _lib().lbm_nn_residual_output(_p(Uin), in_stride, _p(net), C, _p(scale), nf, B, H,
                                                                W, _p(Uout), out_stride, _s()))


def gradient(U, sample_stride, nf, B, H, W, dx, dUx, dUy):
    _ok("lbm_nn_gradient", _lib().lbm_nn_gradient(_p(U), sample_stride, nf, B, H, W, float(dx), _p(dUx), _p(dUy),
                                                  _s()))
