"""FP64 numpy reference of the surrogate's layers and of the whole U-Net, with
hand-derived backward passes, for checking the CUDA kernels and gradients.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Layouts follow the
library: activations [B, H, W, C], weights [Cout, KS, KS, Cin], circular padding.
The backward passes are pinned against central finite differences of the
forward passes (tests/test_oracle_nn.py).
"""
from __future__ import annotations

import numpy as np


def _shift(x, dy, dx):
    """x[b, (y + dy) % H, (x + dx) % W, c]."""
    return np.roll(x, shift=(-dy, -dx), axis=(1, 2))


def conv(x, w, b=None):
    """y[b,y,x,o] = sum_{ky,kx,c} w[o,ky,kx,c] x[b, y+ky-R, x+kx-R, c] + b[o] (circular)."""
    KS = w.shape[1]
    R = KS // 2
    y = np.zeros(x.shape[:3] + (w.shape[0],))
    for ky in range(KS):
        for kx in range(KS):
            y += np.einsum("bhwc,oc->bhwo", _shift(x, ky - R, kx - R), w[:, ky, kx, :])
    if b is not None:
        y += b
    return y


def conv_backward(dy, x, w):
    """Gradients of conv w.r.t. x, w and b for upstream gradient dy."""
    KS = w.shape[1]
    R = KS // 2
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for ky in range(KS):
        for kx in range(KS):
            dx += _shift(np.einsum("bhwo,oc->bhwc", dy, w[:, ky, kx, :]), -(ky - R), -(kx - R))
            dw[:, ky, kx, :] = np.einsum("bhwo,bhwc->oc", dy, _shift(x, ky - R, kx - R))
    return dx, dw, dy.sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def pool(x):
    B, H, W, C = x.shape
    return x.reshape(B, H // 2, 2, W // 2, 2, C).mean(axis=(2, 4))


def pool_backward(dy):
    return 0.25 * np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2)


def upsample(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample_backward(dy):
    B, H, W, C = dy.shape
    return dy.reshape(B, H // 2, 2, W // 2, 2, C).sum(axis=(2, 4))


class UNetRef:
    """Same wiring as the library's surrogate U-Net (4 levels, concatenated skips
    [up | skip], ReLU after every 3x3 convolution, linear 1x1 output)."""

    def __init__(self, params):
        # params: list of (w, b) in the library's layer order:
        # enc0a, enc0b, enc1a, enc1b, enc2a, enc2b, enc3a, enc3b, dec2a, dec2b, dec1a, dec1b, dec0a, dec0b, out
        self.p = [(np.asarray(w, np.float64), np.asarray(b, np.float64)) for w, b in params]

    def forward(self, x0):
        p = self.p
        cache = {"x0": x0}
        x = x0
        idx = 0
        for l in range(4):
            if l > 0:
                x = pool(cache[f"e{l - 1}"])
                cache[f"p{l}"] = x
            ea = relu(conv(x, *p[idx]))
            e = relu(conv(ea, *p[idx + 1]))
            cache[f"ea{l}"], cache[f"e{l}"] = ea, e
            idx += 2
        prev = cache["e3"]
        for l in (2, 1, 0):
            u = upsample(prev)
            cat = np.concatenate([u, cache[f"e{l}"]], axis=3)
            da = relu(conv(cat, *p[idx]))
            d = relu(conv(da, *p[idx + 1]))
            cache[f"u{l}"], cache[f"cat{l}"], cache[f"da{l}"], cache[f"d{l}"] = u, cat, da, d
            prev = d
            idx += 2
        out = conv(prev, *p[idx])
        cache["out"] = out
        self.cache = cache
        return out

    def backward(self, dout):
        """Gradients of all (w, b), in layer order, for upstream gradient dout."""
        p, c = self.p, self.cache
        grads = [None] * len(p)
        g_d, gw, gb = conv_backward(dout, c["d0"], p[14][0])
        grads[14] = (gw, gb)
        g_skip = {}
        idx = 12
        for l in (0, 1, 2):
            g_d = g_d * (c[f"d{l}"] > 0)
            g_da, gw, gb = conv_backward(g_d, c[f"da{l}"], p[idx + 1][0])
            grads[idx + 1] = (gw, gb)
            g_da = g_da * (c[f"da{l}"] > 0)
            g_cat, gw, gb = conv_backward(g_da, c[f"cat{l}"], p[idx][0])
            grads[idx] = (gw, gb)
            cu = c[f"u{l}"].shape[3]
            g_u, g_skip[l] = g_cat[..., :cu], g_cat[..., cu:]
            g_d = upsample_backward(g_u)
            idx -= 2
        g_e = g_d                      # gradient of e3
        for l in (3, 2, 1, 0):
            i = 2 * l
            g_e = g_e * (c[f"e{l}"] > 0)
            g_ea, gw, gb = conv_backward(g_e, c[f"ea{l}"], p[i + 1][0])
            grads[i + 1] = (gw, gb)
            g_ea = g_ea * (c[f"ea{l}"] > 0)
            x = c["x0"] if l == 0 else c[f"p{l}"]
            g_x, gw, gb = conv_backward(g_ea, x, p[i][0])
            grads[i] = (gw, gb)
            if l > 0:
                g_e = g_skip[l - 1] + pool_backward(g_x)
        return grads
