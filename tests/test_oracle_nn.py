"""Pins of the numpy layer reference (no GPU): the convolution against a direct
loop, and every backward pass (layers and the whole U-Net) against central
finite differences of the forward pass."""
import numpy as np

from oracle import nn_reference as R

RNG = np.random.default_rng(3)


def test_conv_matches_direct_loop():
    x = RNG.standard_normal((2, 4, 8, 3))
    w = RNG.standard_normal((5, 3, 3, 3))
    b = RNG.standard_normal(5)
    y = R.conv(x, w, b)
    B, H, W, C = x.shape
    ref = np.zeros((B, H, W, 5))
    for n in range(B):
        for i in range(H):
            for j in range(W):
                for o in range(5):
                    s = b[o]
                    for ky in range(3):
                        for kx in range(3):
                            s += np.dot(w[o, ky, kx], x[n, (i + ky - 1) % H, (j + kx - 1) % W])
                    ref[n, i, j, o] = s
    np.testing.assert_allclose(y, ref, atol=1e-12)


def _fd_check(f, x, g, n=12, h=1e-6):
    """compare <g, e_i> with (f(x + h e_i) - f(x - h e_i)) / 2h at random entries"""
    flat = x.reshape(-1)
    for idx in RNG.choice(flat.size, min(n, flat.size), replace=False):
        old = flat[idx]
        flat[idx] = old + h
        fp = f()
        flat[idx] = old - h
        fm = f()
        flat[idx] = old
        num = (fp - fm) / (2 * h)
        assert abs(num - g.reshape(-1)[idx]) <= 1e-6 * max(1.0, abs(num)), (idx, num, g.reshape(-1)[idx])


def test_layer_backward_against_finite_differences():
    x = RNG.standard_normal((2, 8, 8, 4))
    w = RNG.standard_normal((3, 3, 3, 4))
    b = RNG.standard_normal(3)
    up = RNG.standard_normal((2, 8, 8, 3))
    dx, dw, db = R.conv_backward(up, x, w)
    loss = lambda: float(np.sum(up * R.conv(x, w, b)))
    _fd_check(loss, x, dx)
    _fd_check(loss, w, dw)
    _fd_check(loss, b, db)
    up2 = RNG.standard_normal((2, 4, 4, 4))
    _fd_check(lambda: float(np.sum(up2 * R.pool(x))), x, R.pool_backward(up2))
    up3 = RNG.standard_normal((2, 16, 16, 4))
    _fd_check(lambda: float(np.sum(up3 * R.upsample(x))), x, R.upsample_backward(up3))


def small_unet_params(c=(4, 4, 4, 4), cin=3, cout=2, seed=0):
    rng = np.random.default_rng(seed)
    c0, c1, c2, c3 = c
    shapes = [(c0, 3, 3, cin), (c0, 3, 3, c0), (c1, 3, 3, c0), (c1, 3, 3, c1), (c2, 3, 3, c1), (c2, 3, 3, c2),
              (c3, 3, 3, c2), (c3, 3, 3, c3), (c2, 3, 3, c3 + c2), (c2, 3, 3, c2), (c1, 3, 3, c2 + c1),
              (c1, 3, 3, c1), (c0, 3, 3, c1 + c0), (c0, 3, 3, c0), (cout, 1, 1, c0)]
    return [(rng.standard_normal(s) * 0.3, rng.standard_normal(s[0]) * 0.1) for s in shapes]


def test_unet_backward_against_finite_differences():
    params = small_unet_params()
    net = R.UNetRef(params)
    x = RNG.standard_normal((1, 16, 16, 3))
    up = RNG.standard_normal((1, 16, 16, 2))
    net.forward(x)
    grads = net.backward(up)

    def loss():
        return float(np.sum(up * net.forward(x)))

    for i in (0, 3, 7, 8, 12, 14):
        _fd_check(loss, net.p[i][0], grads[i][0], n=6)
        _fd_check(loss, net.p[i][1], grads[i][1], n=2)
