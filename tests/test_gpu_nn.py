"""GPU tests of the surrogate's kernels against the FP64 numpy reference
(oracle/nn_reference.py): convolutions (forward, data and weight gradients,
two-input / two-output / accumulate forms), pooling, upsampling, loss, Adam,
packing, finite differences, and the whole U-Net's output and every parameter
gradient.  The reference uses the same BF16-rounded weights, so the remaining
differences are the BF16 split of the activations (about 2^-17 relative) and
FP32 accumulation."""
import numpy as np
import pytest

from oracle import nn_reference as R
from oracle.postprocess import rel_l2

pytestmark = pytest.mark.gpu
RNG = np.random.default_rng(21)


def _bf16(a):
    import torch
    return torch.from_numpy(np.asarray(a, np.float32)).to(torch.bfloat16).to(torch.float64).numpy()


def _t(a, dtype=None):
    import torch
    return torch.tensor(np.asarray(a), dtype=dtype or torch.float32, device="cuda")


def _wb(w):
    import torch
    return torch.tensor(np.asarray(w, np.float32), device="cuda").to(torch.bfloat16)


@pytest.mark.parametrize("KS,C1,C2,Cout,Co1", [(3, 32, 64, 48, 48), (3, 32, 0, 64, 16), (1, 64, 0, 32, 32),
                                               (3, 96, 32, 16, 8)])
def test_conv_forward(lbm, KS, C1, C2, Cout, Co1):
    import torch
    from paper_2408_01081_gb300 import nn as K
    B, H, W = 2, 16, 32
    x1 = RNG.standard_normal((B, H, W, C1)).astype(np.float32)
    x2 = RNG.standard_normal((B, H, W, C2)).astype(np.float32) if C2 else None
    w = _bf16(RNG.standard_normal((Cout, KS, KS, C1 + C2)) * 0.1)
    b = RNG.standard_normal(Cout).astype(np.float32)
    x = x1 if C2 == 0 else np.concatenate([x1, x2], axis=3)
    ref = np.maximum(R.conv(x.astype(np.float64), w, b), 0.0)
    prev = RNG.standard_normal((B, H, W, Cout)).astype(np.float32)
    y1 = _t(prev[..., :Co1].copy())
    y2 = _t(prev[..., Co1:].copy()) if Co1 < Cout else None
    K.conv_forward(_t(x1), C1, _t(x2) if C2 else None, C2, _wb(w), _t(b), y1, Co1, y2, Cout, B, H, W, KS,
                   relu=True, beta=True)
    got = y1.cpu().numpy() if y2 is None else np.concatenate([y1.cpu().numpy(), y2.cpu().numpy()], axis=3)
    assert rel_l2(got, ref + prev) < 2e-6 * 10, rel_l2(got, ref + prev)
    assert np.max(np.abs(got - (ref + prev))) < 1e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("H,W,C1,C2,Cout,Co1", [(8, 16, 32, 0, 32, 32), (16, 32, 32, 32, 32, 32),
                                               (32, 16, 64, 0, 128, 128), (16, 64, 128, 64, 192, 128),
                                               (64, 32, 32, 64, 64, 32)])
def test_conv3_halo_tile_forward(lbm, H, W, C1, C2, Cout, Co1):
    """The 8x16 halo-tiled 3x3 kernel (H >= 8, W >= 16, Cout a multiple of 32): single tiles
    whose halo wraps around the image, several tiles per image, two inputs, two outputs."""
    from paper_2408_01081_gb300 import nn as K
    B = 2
    x1 = RNG.standard_normal((B, H, W, C1)).astype(np.float32)
    x2 = RNG.standard_normal((B, H, W, C2)).astype(np.float32) if C2 else None
    w = _bf16(RNG.standard_normal((Cout, 3, 3, C1 + C2)) * 0.1)
    b = RNG.standard_normal(Cout).astype(np.float32)
    x = x1 if C2 == 0 else np.concatenate([x1, x2], axis=3)
    ref = R.conv(x.astype(np.float64), w, b)
    y1 = _t(np.zeros((B, H, W, Co1), np.float32))
    y2 = _t(np.zeros((B, H, W, Cout - Co1), np.float32)) if Co1 < Cout else None
    K.conv_forward(_t(x1), C1, _t(x2) if C2 else None, C2, _wb(w), _t(b), y1, Co1, y2, Cout, B, H, W, 3,
                   relu=False, beta=False)
    got = y1.cpu().numpy() if y2 is None else np.concatenate([y1.cpu().numpy(), y2.cpu().numpy()], axis=3)
    assert rel_l2(got, ref) < 2e-5, rel_l2(got, ref)
    assert np.max(np.abs(got - ref)) < 1e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("B,H,W,C1,C2,Cout,Co1,act_bf16,x1_half", [
    (8, 128, 128, 32, 0, 32, 32, False, False),     # 32 channels per CTA, two 128-pixel tiles
    (8, 128, 128, 32, 0, 32, 32, True, False),      # the same with single-BF16 activations
    (8, 128, 128, 64, 0, 64, 64, False, False),     # 64 channels, two tiles
    (8, 128, 128, 32, 32, 128, 128, True, False),   # 128 channels, two tiles, two inputs
    (4, 64, 64, 64, 64, 128, 64, False, False),     # one tile per CTA, two inputs, two outputs
    (2, 16, 8, 32, 0, 64, 64, False, False),        # one 16x8 tile per image: the halo wraps on every side
    (2, 32, 32, 256, 0, 256, 256, False, False),    # two CTAs along the output channels, 16 chunks
    (4, 64, 64, 64, 32, 96, 32, False, True),       # 96 channels (32 per CTA), x1 upsampled, accumulate
    (16, 256, 256, 32, 0, 32, 32, False, False),    # about nine blocks per persistent CTA, resident weights
    (16, 128, 128, 64, 64, 64, 64, False, False),   # several blocks per CTA, weights streamed per chunk
    (1, 16, 8, 32, 0, 32, 32, True, False),         # the smallest image the kernel takes: one block
    (1, 16, 16, 32, 0, 32, 16, False, True),        # x1 upsampled from 8x8, two outputs of 16 channels
    (2, 32, 32, 256, 256, 128, 128, False, False),  # 512 input channels: 32 chunks, weights streamed
])
def test_conv3_tcgen05(lbm, B, H, W, C1, C2, Cout, Co1, act_bf16, x1_half):
    """The tcgen05 3x3 kernel (persistent CTAs, two accumulators in tensor memory): against
    the reference on the first and last image, and against the mma.sync kernel (same
    products, other summation order) on every pixel; no bounded wait ran out."""
    from paper_2408_01081_gb300 import nn as K
    h1, w1 = (H // 2, W // 2) if x1_half else (H, W)
    x1 = RNG.standard_normal((B, h1, w1, C1)).astype(np.float32)
    x2 = RNG.standard_normal((B, H, W, C2)).astype(np.float32) if C2 else None
    w = _bf16(RNG.standard_normal((Cout, 3, 3, C1 + C2)) * 0.1)
    b = RNG.standard_normal(Cout).astype(np.float32)
    prev = RNG.standard_normal((B, H, W, Cout)).astype(np.float32)
    outs = []
    for mma_sync in (False, True):
        before = K.conv_counts()
        y1 = _t(prev[..., :Co1].copy())
        y2 = _t(prev[..., Co1:].copy()) if Co1 < Cout else None
        K.conv_forward(_t(x1), C1, _t(x2) if C2 else None, C2, _wb(w), _t(b), y1, Co1, y2, Cout, B, H, W, 3,
                       relu=True, beta=x1_half, x1_half=x1_half, act_bf16=act_bf16, mma_sync=mma_sync)
        K.check()
        after = K.conv_counts()
        # the launch went to the kernel asked for, not to a fallback
        assert (after[0] - before[0], after[1] - before[1]) == ((0, 1) if mma_sync else (1, 0)), (before, after)
        outs.append(y1.cpu().numpy() if y2 is None else np.concatenate([y1.cpu().numpy(), y2.cpu().numpy()], 3))
    got, legacy = outs
    assert rel_l2(got, legacy) < 2e-6, rel_l2(got, legacy)
    idx = [0, B - 1]
    xu = np.repeat(np.repeat(x1[idx], 2, axis=1), 2, axis=2) if x1_half else x1[idx]
    x = xu if C2 == 0 else np.concatenate([xu, x2[idx]], axis=3)
    if act_bf16:
        x = _bf16(x)
    ref = np.maximum(R.conv(x.astype(np.float64), w, b), 0.0) + (prev[idx] if x1_half else 0.0)
    assert rel_l2(got[idx], ref) < 2e-5, rel_l2(got[idx], ref)
    assert np.max(np.abs(got[idx] - ref)) < 1e-4 * np.max(np.abs(ref))


@pytest.mark.parametrize("H,W,Cout,Co1,KS,tc", [(16, 8, 32, 32, 3, True), (8, 16, 32, 32, 3, False),
                                                  (16, 16, 48, 48, 3, False), (16, 16, 32, 8, 3, False),
                                                  (16, 16, 32, 32, 1, False), (16, 4, 32, 32, 3, False)])
def test_conv_kernel_selection(lbm, H, W, Cout, Co1, KS, tc):
    """3x3 convolutions with H >= 16, W >= 8, Cout a multiple of 32 and Co1 a multiple of 16 run
    on the tcgen05 kernel, everything else on the mma.sync kernels; both give the reference."""
    from paper_2408_01081_gb300 import nn as K
    B, C1 = 2, 32
    x1 = RNG.standard_normal((B, H, W, C1)).astype(np.float32)
    w = _bf16(RNG.standard_normal((Cout, KS, KS, C1)) * 0.1)
    y1 = _t(np.zeros((B, H, W, Co1), np.float32))
    y2 = _t(np.zeros((B, H, W, Cout - Co1), np.float32)) if Co1 < Cout else None
    before = K.conv_counts()
    K.conv_forward(_t(x1), C1, None, 0, _wb(w), None, y1, Co1, y2, Cout, B, H, W, KS)
    K.check()
    after = K.conv_counts()
    assert (after[0] - before[0], after[1] - before[1]) == ((1, 0) if tc else (0, 1))
    got = y1.cpu().numpy() if y2 is None else np.concatenate([y1.cpu().numpy(), y2.cpu().numpy()], axis=3)
    ref = R.conv(x1.astype(np.float64), w)
    assert rel_l2(got, ref) < 2e-5, rel_l2(got, ref)


@pytest.mark.parametrize("P,C", [(1, 5), (100, 32), (70000, 64), (5000, 384), (1 << 21, 32)])
def test_bias_grad_sizes(lbm, P, C):
    """Channel counts below, at and above one block's 256 threads; one to many blocks."""
    import torch
    from paper_2408_01081_gb300 import nn as K
    dy = torch.randn((P, C), dtype=torch.float32, device="cuda")
    db = torch.empty(C, dtype=torch.float32, device="cuda")
    ws = torch.empty(K.bias_grad_workspace_bytes(P, C) // 4 + 1, dtype=torch.float32, device="cuda")
    K.bias_grad(dy, P, C, db, ws)
    ref = dy.double().sum(0)
    assert torch.max(torch.abs(db.double() - ref)).item() < 1e-5 * max(1.0, P ** 0.5)


@pytest.mark.parametrize("KS,C1,C2,Cout", [(3, 32, 0, 32), (3, 64, 32, 48), (1, 32, 0, 32)])
def test_conv_gradients(lbm, KS, C1, C2, Cout):
    import torch
    from paper_2408_01081_gb300 import nn as K
    B, H, W = 2, 32, 16
    x1 = RNG.standard_normal((B, H, W, C1)).astype(np.float32)
    x2 = RNG.standard_normal((B, H, W, C2)).astype(np.float32) if C2 else None
    x = x1 if C2 == 0 else np.concatenate([x1, x2], axis=3)
    w = _bf16(RNG.standard_normal((Cout, KS, KS, C1 + C2)) * 0.1)
    dy = RNG.standard_normal((B, H, W, Cout)).astype(np.float32)
    rdx, rdw, rdb = R.conv_backward(dy.astype(np.float64), x.astype(np.float64), w)
    ws = torch.empty(K.wgrad_workspace_bytes(C1 + C2, Cout, B, H, W, KS) // 4 + 1, dtype=torch.float32,
                     device="cuda")
    dw = torch.empty((Cout, KS, KS, C1 + C2), dtype=torch.float32, device="cuda")
    K.conv_backward_weight(_t(dy), Cout, _t(x1), C1, _t(x2) if C2 else None, C2, B, H, W, KS, dw, ws)
    assert rel_l2(dw.cpu().numpy(), rdw) < 2e-5, rel_l2(dw.cpu().numpy(), rdw)
    db = torch.empty(Cout, dtype=torch.float32, device="cuda")
    wsb = torch.empty(K.bias_grad_workspace_bytes(B * H * W, Cout) // 4 + 1, dtype=torch.float32, device="cuda")
    K.bias_grad(_t(dy), B * H * W, Cout, db, wsb)
    assert rel_l2(db.cpu().numpy(), rdb) < 1e-5
    wt = torch.empty((C1 + C2, KS, KS, Cout), dtype=torch.bfloat16, device="cuda")
    K.weight_flip(_wb(w), Cout, C1 + C2, KS, wt)
    dx1 = torch.empty((B, H, W, C1), dtype=torch.float32, device="cuda")
    dx2 = torch.empty((B, H, W, C2), dtype=torch.float32, device="cuda") if C2 else None
    if Cout % 32 == 0:
        K.conv_forward(_t(dy), Cout, None, 0, wt, None, dx1, C1, dx2, C1 + C2, B, H, W, KS)
        got = dx1.cpu().numpy() if not C2 else np.concatenate([dx1.cpu().numpy(), dx2.cpu().numpy()], axis=3)
        assert rel_l2(got, rdx) < 2e-5, rel_l2(got, rdx)


@pytest.mark.parametrize("B,H,W,C1,C2,Cout,x1_half,beta", [
    (2, 32, 16, 32, 0, 32, False, False),       # one 32x32 channel tile, 4 blocks
    (8, 64, 64, 32, 0, 32, False, True),        # 128 blocks over many splits, accumulate
    (4, 32, 32, 64, 32, 32, True, False),       # x1 half size + x2 (decoder), Cin 96
    (2, 32, 32, 64, 0, 128, False, False),      # 4 x 2 channel tiles
    (1, 16, 16, 256, 256, 64, False, False),    # 512 input channels, one block per image
])
def test_conv_wgrad_block_tiled(lbm, B, H, W, C1, C2, Cout, x1_half, beta):
    """The block-tiled 3x3 weight gradient (all nine taps per CTA, halo block staged once)
    against the FP64 reference and against the per-tap kernel; the launch went to it."""
    import torch
    from paper_2408_01081_gb300 import nn as K
    h1, w1 = (H // 2, W // 2) if x1_half else (H, W)
    x1 = RNG.standard_normal((B, h1, w1, C1)).astype(np.float32)
    x2 = RNG.standard_normal((B, H, W, C2)).astype(np.float32) if C2 else None
    xu = np.repeat(np.repeat(x1, 2, axis=1), 2, axis=2) if x1_half else x1
    x = xu if C2 == 0 else np.concatenate([xu, x2], axis=3)
    w = _bf16(RNG.standard_normal((Cout, 3, 3, C1 + C2)) * 0.1)
    dy = RNG.standard_normal((B, H, W, Cout)).astype(np.float32)
    _, rdw, _ = R.conv_backward(dy.astype(np.float64), x.astype(np.float64), w)
    prev = RNG.standard_normal((Cout, 3, 3, C1 + C2)).astype(np.float32)
    ws = torch.empty(K.wgrad_workspace_bytes(C1 + C2, Cout, B, H, W, 3) // 4 + 1, dtype=torch.float32,
                     device="cuda")
    outs = []
    for per_tap in (False, True):
        dw = _t(prev.copy())
        before = K.conv_counts()
        K.conv_backward_weight(_t(dy), Cout, _t(x1), C1, _t(x2) if C2 else None, C2, B, H, W, 3, dw, ws,
                               beta=beta, x1_half=x1_half, per_tap=per_tap)
        K.check()
        after = K.conv_counts()
        assert (after[2] - before[2], after[3] - before[3]) == ((0, 1) if per_tap else (1, 0)), (before, after)
        outs.append(dw.cpu().numpy() - (prev if beta else 0.0))
    got, per_tap_result = outs
    assert rel_l2(got, rdw) < 2e-5, rel_l2(got, rdw)
    # same products, FP32 sums over the pixels in another order
    assert rel_l2(got, per_tap_result) < 1e-5, rel_l2(got, per_tap_result)


def test_pool_upsample_mse_adam_pack(lbm):
    import torch
    from paper_2408_01081_gb300 import nn as K
    B, H, W, C = 2, 8, 16, 32
    x = RNG.standard_normal((B, H, W, C)).astype(np.float32)
    y = torch.empty((B, H // 2, W // 2, C), device="cuda")
    K.pool(_t(x), B, H, W, C, y)
    np.testing.assert_allclose(y.cpu().numpy(), R.pool(x.astype(np.float64)), atol=1e-6)
    dy = RNG.standard_normal((B, H // 2, W // 2, C)).astype(np.float32)
    dx = _t(np.ones((B, H, W, C)))
    K.pool_backward(_t(dy), B, H, W, C, dx, beta=True)
    np.testing.assert_allclose(dx.cpu().numpy(), 1.0 + R.pool_backward(dy), atol=1e-6)
    u = torch.empty((B, 2 * H, 2 * W, C), device="cuda")
    K.upsample(_t(x), B, H, W, C, u)
    np.testing.assert_allclose(u.cpu().numpy(), R.upsample(x), atol=0)
    du = RNG.standard_normal((B, 2 * H, 2 * W, C)).astype(np.float32)
    dxu = torch.empty((B, H, W, C), device="cuda")
    K.upsample_backward(_t(du), B, H, W, C, dxu)
    np.testing.assert_allclose(dxu.cpu().numpy(), R.upsample_backward(du.astype(np.float64)), atol=1e-5)
    # loss and its gradient over the first 5 channels
    out, tgt = (RNG.standard_normal((B, H, W, C)).astype(np.float32) for _ in range(2))
    dout = torch.empty((B, H, W, C), device="cuda")
    ws = torch.empty(512, dtype=torch.float64, device="cuda")
    loss = torch.empty(1, dtype=torch.float64, device="cuda")
    K.mse(_t(out), _t(tgt), B * H * W, C, 5, 0.5, dout, ws, loss)
    d = (out - tgt).astype(np.float64)
    assert abs(loss.item() - np.sum(d[..., :5] ** 2)) < 1e-6 * np.sum(d[..., :5] ** 2)
    ref = np.zeros_like(d)
    ref[..., :5] = 2 * d[..., :5] * 0.5
    np.testing.assert_allclose(dout.cpu().numpy(), ref, atol=1e-5)
    # Adam, first step: w - lr * g / (|g| + eps)
    w0, g0 = RNG.standard_normal(1000).astype(np.float32), RNG.standard_normal(1000).astype(np.float32)
    w, m, v = _t(w0), _t(np.zeros(1000)), _t(np.zeros(1000))
    wb = torch.empty(1000, dtype=torch.bfloat16, device="cuda")
    K.adam(w, _t(g0), m, v, 1e-2, 0.9, 0.999, 1e-8, 1, wb)
    np.testing.assert_allclose(w.cpu().numpy(), w0 - 1e-2 * g0 / (np.abs(g0) + 1e-8), atol=1e-6)
    np.testing.assert_allclose(wb.float().cpu().numpy(), _bf16(w.cpu().numpy()), atol=0)
    # input / target packing, residual output, periodic gradient
    U = RNG.standard_normal((B, 10, H, W))
    U2 = RNG.standard_normal((B, 10, H, W))
    scale = np.array([1.0, 2.0, 0.5, 4.0, 0.25])
    nu = np.array([0.3, -1.0], np.float32)
    xin = torch.empty((B, H, W, 32), device="cuda")
    K.pack_input(_t(U, torch.float64), 10 * H * W, 5, _t(scale, torch.float64), _t(nu), B, H, W, 32, xin)
    ref = np.zeros((B, H, W, 32))
    ref[..., :5] = np.transpose(U[:, :5], (0, 2, 3, 1)) / scale
    ref[..., 5] = nu[:, None, None]
    np.testing.assert_allclose(xin.cpu().numpy(), ref, rtol=1e-6, atol=1e-7)
    tg = torch.empty((B, H, W, 32), device="cuda")
    K.pack_target(_t(U, torch.float64), _t(U2, torch.float64), 10 * H * W, 5, _t(scale, torch.float64), B, H, W, 32, tg)
    reft = np.zeros((B, H, W, 32))
    reft[..., :5] = np.transpose((U2 - U)[:, :5], (0, 2, 3, 1)) / scale
    np.testing.assert_allclose(tg.cpu().numpy(), reft, rtol=1e-6, atol=1e-6)
    Uo = torch.zeros((B, 10, H, W), dtype=torch.float64, device="cuda")
    K.residual_output(_t(U, torch.float64), 10 * H * W, xin, 32, _t(scale, torch.float64), 5, B, H, W, Uo, 10 * H * W)
    np.testing.assert_allclose(Uo.cpu().numpy()[:, :5], U[:, :5] + scale[None, :, None, None] *
                               np.transpose(xin.cpu().numpy()[..., :5].astype(np.float64), (0, 3, 1, 2)), atol=1e-12)
    gx = torch.empty((B, 10, H, W), dtype=torch.float64, device="cuda")
    gy = torch.empty_like(gx)
    K.gradient(_t(U, torch.float64), 10 * H * W, 5, B, H, W, 0.1, gx, gy)
    np.testing.assert_allclose(gx.cpu().numpy()[:, :5], (np.roll(U, -1, 3) - np.roll(U, 1, 3))[:, :5] / 0.2, atol=1e-12)
    np.testing.assert_allclose(gy.cpu().numpy()[:, :5], (np.roll(U, -1, 2) - np.roll(U, 1, 2))[:, :5] / 0.2, atol=1e-12)


def test_unet_output_and_gradients_match_reference(lbm):
    """Whole U-Net (channels 32 at every level, 16x16, batch 2): output and every
    parameter gradient against the FP64 reference network with the same BF16 weights."""
    import torch
    from paper_2408_01081_gb300 import surrogate as S
    net = S.UNet((32, 32, 32, 32), seed=4)
    B, H, W = 2, 16, 16
    net._alloc(B, H, W)
    rng = np.random.default_rng(8)
    params = []
    for layer in net.layers:
        w = _bf16(rng.standard_normal(tuple(layer.w.shape)) * np.sqrt(2.0 / np.prod(layer.w.shape[1:])))
        b = rng.standard_normal(layer.cout) * 0.05
        params.append((w, b))
        layer.w.copy_(torch.tensor(w, dtype=torch.float32))
        layer.b.copy_(torch.tensor(b, dtype=torch.float32))
        layer.wb.copy_(layer.w.to(torch.bfloat16))
    x0 = rng.standard_normal((B, H, W, 32)).astype(np.float32)
    net.A["x0"].copy_(torch.tensor(x0))
    net.forward(B, H, W)
    ref_net = R.UNetRef([(w, b) for w, b in params])
    ref = ref_net.forward(x0.astype(np.float64))
    assert rel_l2(net.A["out"].cpu().numpy(), ref) < 1e-4, rel_l2(net.A["out"].cpu().numpy(), ref)
    dout = rng.standard_normal((B, H, W, 32)).astype(np.float32)
    net.G["out"].copy_(torch.tensor(dout))
    net.backward(B, H, W)
    grads = ref_net.backward(dout.astype(np.float64))
    for i, layer in enumerate(net.layers):
        e_w = rel_l2(layer.gw.cpu().numpy(), grads[i][0])
        e_b = rel_l2(layer.gb.cpu().numpy(), grads[i][1])
        assert e_w < 1e-3 and e_b < 1e-3, (i, e_w, e_b)


@pytest.mark.parametrize("H,W,KS", [(16, 32, 3), (8, 8, 3), (16, 16, 1)])
def test_conv_half_resolution_input_and_bf16_activations(lbm, H, W, KS):
    """x1 read nearest-upsampled from (H/2, W/2) equals the convolution of the materialised
    upsampled tensor; single-BF16 activations stay within BF16 rounding of the exact result."""
    import torch
    from paper_2408_01081_gb300 import nn as K
    B, C1, C2, Cout = 2, 64, 32, 64
    xc = RNG.standard_normal((B, H // 2, W // 2, C1)).astype(np.float32)
    xu = np.repeat(np.repeat(xc, 2, axis=1), 2, axis=2)
    x2 = RNG.standard_normal((B, H, W, C2)).astype(np.float32)
    w = _bf16(RNG.standard_normal((Cout, KS, KS, C1 + C2)) * 0.1)
    b = RNG.standard_normal(Cout).astype(np.float32)
    ref = R.conv(np.concatenate([xu, x2], axis=3).astype(np.float64), w, b)
    y = _t(np.zeros((B, H, W, Cout), np.float32))
    K.conv_forward(_t(xc), C1, _t(x2), C2, _wb(w), _t(b), y, Cout, None, Cout, B, H, W, KS, x1_half=True)
    assert rel_l2(y.cpu().numpy(), ref) < 2e-5, rel_l2(y.cpu().numpy(), ref)
    y2 = _t(np.zeros((B, H, W, Cout), np.float32))
    K.conv_forward(_t(xu), C1, _t(x2), C2, _wb(w), _t(b), y2, Cout, None, Cout, B, H, W, KS, act_bf16=True)
    e = rel_l2(y2.cpu().numpy(), ref)
    assert 1e-5 < e < 1e-2, e           # BF16 rounding of the activations, and only that
    # weight gradient with the half-resolution x1 equals the one of the upsampled tensor
    dy = RNG.standard_normal((B, H, W, Cout)).astype(np.float32)
    ws = torch.empty(K.wgrad_workspace_bytes(C1 + C2, Cout, B, H, W, KS) // 4 + 1, dtype=torch.float32,
                     device="cuda")
    dwh = torch.empty((Cout, KS, KS, C1 + C2), dtype=torch.float32, device="cuda")
    dwf = torch.empty_like(dwh)
    K.conv_backward_weight(_t(dy), Cout, _t(xc), C1, _t(x2), C2, B, H, W, KS, dwh, ws, x1_half=True)
    K.conv_backward_weight(_t(dy), Cout, _t(xu), C1, _t(x2), C2, B, H, W, KS, dwf, ws)
    torch.testing.assert_close(dwh, dwf, rtol=0, atol=0)
