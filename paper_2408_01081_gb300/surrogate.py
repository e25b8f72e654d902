"""Learned surrogate: a convolutional U-Net neural operator that jumps k steps
of the lattice Boltzmann solver on periodic lattices, trained on trajectories
the solver itself generates, with the solver as fallback and as the check of its error.

Model (channels-last, circular padding, ReLU):
    input  x0 = [U(t) / scale (5 fields), (nu - 0.245) / 0.1415, zero padding] -> 32 channels
    encoder level l = 0..3: two 3x3 convolutions to c_l channels, 2x2 average pooling between levels
    decoder level l = 2..0: nearest 2x upsampling, 3x3 convolution of [up | skip_l] to c_l, 3x3 c_l -> c_l
    output 1x1 convolution c_0 -> 32 (5 used): U(t + k dt) = U(t) + scale * out
With c = (32, 64, 128, 256) the network has 1.95 M parameters.

Every layer runs in the library's kernels (include/lbm_nn.h): tensor-core
implicit-GEMM convolutions with BF16 weights and FP32 accumulation, their
weight and data gradients, pooling, upsampling, the loss and Adam.  This module
only allocates buffers (torch tensors) and calls them in order.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass
from typing import List, Optional, Sequence

import numpy as np

from . import lbm as L
from . import nn as K

NU_MEAN, NU_STD = 0.245, 0.1415
CIN_PAD = 32          # input channels after padding
COUT_PAD = 32         # output channels (5 used)
NF = 5                # predicted fields: v_x, v_y, j_s, j_d, j_xy


class Conv:
    """One convolution: FP32 master weights, BF16 working and flipped copies, Adam state."""

    def __init__(self, cin1, cin2, cout, ks, relu, rng, device, zero=False):
        import torch
        self.cin1, self.cin2, self.cout, self.ks, self.relu = cin1, cin2, cout, ks, relu
        cin = cin1 + cin2
        std = math.sqrt(2.0 / (cin * ks * ks)) if relu else math.sqrt(1.0 / (cin * ks * ks))
        w = np.zeros((cout, ks, ks, cin), np.float32) if zero else rng.normal(0.0, std, (cout, ks, ks, cin))
        self.w = torch.tensor(w, dtype=torch.float32, device=device)
        self.b = torch.zeros(cout, dtype=torch.float32, device=device)
        self.wb = torch.empty((cout, ks, ks, cin), dtype=torch.bfloat16, device=device)
        self.wt = torch.empty((cin, ks, ks, cout), dtype=torch.bfloat16, device=device)
        self.gw = torch.zeros_like(self.w)
        self.gb = torch.zeros_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        K.to_bf16(self.w, self.wb)

    @property
    def nparams(self):
        return self.w.numel() + self.b.numel()

    def forward(self, x1, x2, y, B, H, W, x1_half=False, act_bf16=False):
        """x1_half: x1 is at (H/2, W/2), read nearest-upsampled (the decoder's upsampling)."""
        K.conv_forward(x1, self.cin1, x2, self.cin2, self.wb, self.b, y, self.cout, None, self.cout, B, H, W,
                       self.ks, relu=self.relu, x1_half=x1_half, act_bf16=act_bf16)

    def backward(self, dy, y, x1, x2, B, H, W, dx1, dx2, workspace, need_dx=True, x1_half=False):
        """dy: gradient w.r.t. this layer's output (overwritten by the ReLU mask); with x1_half
        the data gradient dx1 is at full resolution (the caller folds it back to (H/2, W/2))."""
        if self.relu:
            K.relu_backward(dy, y)
        K.conv_backward_weight(dy, self.cout, x1, self.cin1, x2, self.cin2, B, H, W, self.ks, self.gw, workspace,
                               x1_half=x1_half)
        K.bias_grad(dy, B * H * W, self.cout, self.gb, workspace)
        if need_dx:
            K.weight_flip(self.wb, self.cout, self.cin1 + self.cin2, self.ks, self.wt)
            K.conv_forward(dy, self.cout, None, 0, self.wt, None, dx1, self.cin1, dx2, self.cin1 + self.cin2,
                           B, H, W, self.ks, relu=False)

    def adam(self, lr, step, b1=0.9, b2=0.999, eps=1e-8):
        K.adam(self.w, self.gw, self.mw, self.vw, lr, b1, b2, eps, step, self.wb)
        K.adam(self.b, self.gb, self.mb, self.vb, lr, b1, b2, eps, step, None)


class UNet:
    def __init__(self, chans: Sequence[int] = (32, 64, 128, 256), seed: int = 0, device="cuda"):
        import torch
        self.torch = torch
        self.dev = torch.device(device)
        self.c = list(chans)
        assert len(self.c) == 4
        rng = np.random.default_rng(seed)
        c0, c1, c2, c3 = self.c
        d = self.dev
        self.enc = [
            (Conv(CIN_PAD, 0, c0, 3, True, rng, d), Conv(c0, 0, c0, 3, True, rng, d)),
            (Conv(c0, 0, c1, 3, True, rng, d), Conv(c1, 0, c1, 3, True, rng, d)),
            (Conv(c1, 0, c2, 3, True, rng, d), Conv(c2, 0, c2, 3, True, rng, d)),
            (Conv(c2, 0, c3, 3, True, rng, d), Conv(c3, 0, c3, 3, True, rng, d)),
        ]
        self.dec = {
            2: (Conv(c3, c2, c2, 3, True, rng, d), Conv(c2, 0, c2, 3, True, rng, d)),
            1: (Conv(c2, c1, c1, 3, True, rng, d), Conv(c1, 0, c1, 3, True, rng, d)),
            0: (Conv(c1, c0, c0, 3, True, rng, d), Conv(c0, 0, c0, 3, True, rng, d)),
        }
        # zero-initialised output: the untrained model predicts persistence U(t + k dt) = U(t)
        self.out = Conv(c0, 0, COUT_PAD, 1, False, rng, d, zero=True)
        self.layers: List[Conv] = [c for pair in self.enc for c in pair] + \
            [c for l in (2, 1, 0) for c in self.dec[l]] + [self.out]
        self.shape = None
        self.step_count = 0

    @property
    def nparams(self) -> int:
        return sum(l.nparams for l in self.layers)

    # -- buffers ---------------------------------------------------------
    def _alloc(self, B, H, W):
        if self.shape == (B, H, W):
            return
        t = self.torch
        f32 = dict(dtype=t.float32, device=self.dev)
        c0, c1, c2, c3 = self.c
        hw = [(H >> l, W >> l) for l in range(4)]
        A = {}
        for l, ch in enumerate(self.c):
            h, w = hw[l]
            A[f"ea{l}"] = t.empty((B, h, w, ch), **f32)
            A[f"e{l}"] = t.empty((B, h, w, ch), **f32)
            if l > 0:
                A[f"p{l}"] = t.empty((B, h, w, self.c[l - 1]), **f32)
        for l in (2, 1, 0):
            h, w = hw[l]
            A[f"u{l}"] = t.empty((B, h, w, self.c[l + 1]), **f32)     # shape only: G[u] is the upsampled gradient
            A[f"da{l}"] = t.empty((B, h, w, self.c[l]), **f32)
            A[f"d{l}"] = t.empty((B, h, w, self.c[l]), **f32)
        A["x0"] = t.empty((B, H, W, CIN_PAD), **f32)
        A["out"] = t.empty((B, H, W, COUT_PAD), **f32)
        A["tgt"] = t.empty((B, H, W, COUT_PAD), **f32)
        # gradient buffers (same shapes), reused
        G = {k: t.empty_like(v) for k, v in A.items() if k not in ("x0", "tgt")}
        ws = max(max(K.wgrad_workspace_bytes(l.cin1 + l.cin2, l.cout, B, H, W, l.ks) for l in self.layers),
                 max(K.bias_grad_workspace_bytes(B * H * W, l.cout) for l in self.layers))
        self.ws = t.empty(ws // 4 + 1, **f32)
        self.mse_ws = t.empty(512, dtype=t.float64, device=self.dev)
        self.loss = t.zeros(1, dtype=t.float64, device=self.dev)
        self.A, self.G = A, G
        self.shape = (B, H, W)

    # -- forward / backward ---------------------------------------------
    def forward(self, B, H, W, act_bf16=False):
        """x0 must already hold the packed input; result in self.A['out'].  The decoder's
        nearest upsampling is folded into the next convolution (it reads the coarse tensor).
        act_bf16: activations as one BF16 value (inference only; training uses the hi/lo pair)."""
        A = self.A
        x = A["x0"]
        for l in range(4):
            h, w = H >> l, W >> l
            if l > 0:
                K.pool(A[f"e{l - 1}"], B, 2 * h, 2 * w, self.c[l - 1], A[f"p{l}"])
                x = A[f"p{l}"]
            ca, cb = self.enc[l]
            ca.forward(x, None, A[f"ea{l}"], B, h, w, act_bf16=act_bf16)
            cb.forward(A[f"ea{l}"], None, A[f"e{l}"], B, h, w, act_bf16=act_bf16)
        prev = A["e3"]
        for l in (2, 1, 0):
            h, w = H >> l, W >> l
            ca, cb = self.dec[l]
            ca.forward(prev, A[f"e{l}"], A[f"da{l}"], B, h, w, x1_half=True, act_bf16=act_bf16)
            cb.forward(A[f"da{l}"], None, A[f"d{l}"], B, h, w, act_bf16=act_bf16)
            prev = A[f"d{l}"]
        self.out.forward(A["d0"], None, A["out"], B, H, W, act_bf16=act_bf16)

    def backward(self, B, H, W):
        """G['out'] must hold dLoss/dout; fills every layer's gw, gb."""
        A, G, ws = self.A, self.G, self.ws
        self.out.backward(G["out"], A["out"], A["d0"], None, B, H, W, G["d0"], None, ws)
        for l in (0, 1, 2):
            h, w = H >> l, W >> l
            ca, cb = self.dec[l]
            cb.backward(G[f"d{l}"], A[f"d{l}"], A[f"da{l}"], None, B, h, w, G[f"da{l}"], None, ws)
            # data gradient of [up | skip]: up part -> G[u], skip part -> G[e] (initialised here)
            coarse = A["e3"] if l == 2 else A[f"d{l + 1}"]
            ca.backward(G[f"da{l}"], A[f"da{l}"], coarse, A[f"e{l}"], B, h, w, G[f"u{l}"], G[f"e{l}"], ws,
                        x1_half=True)
            src = G["e3"] if l == 2 else G[f"d{l + 1}"]
            K.upsample_backward(G[f"u{l}"], B, h // 2, w // 2, self.c[l + 1], src)
        for l in (3, 2, 1, 0):
            h, w = H >> l, W >> l
            ca, cb = self.enc[l]
            cb.backward(G[f"e{l}"], A[f"e{l}"], A[f"ea{l}"], None, B, h, w, G[f"ea{l}"], None, ws)
            x = A["x0"] if l == 0 else A[f"p{l}"]
            ca.backward(G[f"ea{l}"], A[f"ea{l}"], x, None, B, h, w, G[f"p{l}"] if l > 0 else None, None, ws,
                        need_dx=l > 0)
            if l > 0:
                # skip gradient of level l-1 already holds the decoder part; add the pooling path
                K.pool_backward(G[f"p{l}"], B, 2 * h, 2 * w, self.c[l - 1], G[f"e{l - 1}"], beta=True)

    def adam_step(self, lr):
        self.step_count += 1
        for layer in self.layers:
            layer.adam(lr, self.step_count)

    def train_step(self, B, H, W, lr) -> float:
        """x0 and tgt packed; one forward, MSE over the 5 used channels, backward, Adam."""
        A = self.A
        self.forward(B, H, W)
        P = B * H * W
        K.mse(A["out"], A["tgt"], P, COUT_PAD, NF, 1.0 / (P * NF), self.G["out"], self.mse_ws, self.loss)
        self.backward(B, H, W)
        self.adam_step(lr)
        return self.loss  # device scalar (sum of squares), read lazily

    # -- state -------------------------------------------------------------
    def state_dict(self):
        return {f"w{i}": l.w.cpu().numpy() for i, l in enumerate(self.layers)} | \
               {f"b{i}": l.b.cpu().numpy() for i, l in enumerate(self.layers)}

    def load_state_dict(self, sd):
        t = self.torch
        for i, l in enumerate(self.layers):
            l.w.copy_(t.from_numpy(sd[f"w{i}"]))
            l.b.copy_(t.from_numpy(sd[f"b{i}"]))
            K.to_bf16(l.w, l.wb)


# ---------------------------------------------------------------------------
# data: trajectories of the batched solver
# ---------------------------------------------------------------------------

@dataclass
class Chunk:
    U: "object"          # [J+1, n, 10, H, W] FP64 snapshots every k steps (moment-field layout)
    nu: np.ndarray       # [n]
    nu_norm: "object"    # [n] float32 tensor, (nu - NU_MEAN) / NU_STD
    n: int
    J: int


def generate_chunk(n, seed, H=256, W=256, k=32, J=4, storage="f64", device="cuda", cfl=0.9,
                   ell_range=(16.0, 64.0), numax=0.49, std=1e-3, relift=True):
    """n periodic H x W lattices, random Poisson ratio and GRF initial velocity, J+1 snapshots
    of the moment fields every k steps, from the batched lattice Boltzmann solver.

    relift=True: before each k-step segment the populations are re-initialised from the
    moment fields (Eq. ic_second, periodic central differences), so every pair
    (U_j, U_{j+1}) is the same function of U_j that the fallback driver's check evaluates.
    A continuing run also carries non-equilibrium populations that U does not determine,
    so its k-step map is not a function of U alone."""
    import torch
    import workloads as Wk
    from workloads.grf import batch_lattice_inputs_torch
    rng = np.random.default_rng(seed)
    nu = rng.uniform(0.0, numax, n)
    ells = rng.uniform(*ell_range, n)
    descs, specs = [], []
    for i in range(n):
        cK2, cmu2 = Wk.material.poisson_to_speeds(float(nu[i]))
        c = Wk.material.lattice_speed(cK2, cmu2, cfl)
        dx = 1.0 / max(H, W)
        descs.append((W, H, 0, dx, dx / c, math.sqrt(cK2), math.sqrt(cmu2)))
        specs.append(Wk.LatticeSpec(W, H, cK2, cmu2, float(nu[i]), False, float(ells[i]), int(seed * 100003 + 2 * i)))
    dev = torch.device(device)
    stream = torch.cuda.current_stream().cuda_stream
    b = L.lbm_batch_create(descs, storage=L.STORAGE[storage], stream=stream)
    try:
        if storage == "f64":
            L.lbm_batch_set_mode(b, 3)      # staged rows: the same bits as one launch per step
        for i, sp in enumerate(specs):
            U0, Ux, Uy = batch_lattice_inputs_torch(sp, descs[i][3], std=std, device=dev)
            L.lbm_batch_init(b, i, U0, Ux, Uy)
        U = torch.empty((J + 1, n, 10, H, W), dtype=torch.float64, device=dev)
        dx = descs[0][3]
        for j in range(J + 1):
            if j:
                if relift:
                    dUx = torch.zeros((n, 10, H, W), dtype=torch.float64, device=dev)
                    dUy = torch.zeros_like(dUx)
                    K.gradient(U[j - 1], 10 * H * W, NF, n, H, W, dx, dUx, dUy)
                    for i in range(n):
                        L.lbm_batch_init(b, i, U[j - 1, i, :5].contiguous(), dUx[i, :5].contiguous(),
                                         dUy[i, :5].contiguous())
                    del dUx, dUy
                L.lbm_batch_step(b, k)
            for i in range(n):
                L.lbm_batch_moments(b, i, U[j, i])
        L.lbm_batch_synchronize(b)
    finally:
        L.lbm_batch_destroy(b)
    nu_norm = torch.tensor((nu - NU_MEAN) / NU_STD, dtype=torch.float32, device=dev)
    return Chunk(U, nu, nu_norm, n, J)


def field_scales(chunk) -> np.ndarray:
    """Per-field RMS of the moment fields over a chunk (network units)."""
    U = chunk.U[1:, :, :NF]
    return np.sqrt((U * U).mean(dim=(0, 1, 3, 4)).cpu().numpy())


class Surrogate:
    """The trained operator plus the normalisation it was trained with."""

    def __init__(self, net: UNet, scale: np.ndarray, k: int):
        import torch
        self.net = net
        self.k = k
        self.scale_np = np.asarray(scale, dtype=np.float64)
        self.scale = torch.tensor(self.scale_np, dtype=torch.float64, device=net.dev)

    def pack(self, U, stride, nu_norm, B, H, W):
        K.pack_input(U, stride, NF, self.scale, nu_norm, B, H, W, CIN_PAD, self.net.A["x0"])

    def predict(self, U, stride, nu_norm, B, H, W, Uout, out_stride, act_bf16=False):
        """Uout = U + scale * net(U): the moment fields k steps later (FP64).  act_bf16 runs
        the network with single-BF16 activations (half the tensor-core work)."""
        self.net._alloc(B, H, W)
        self.pack(U, stride, nu_norm, B, H, W)
        self.net.forward(B, H, W, act_bf16=act_bf16)
        K.residual_output(U, stride, self.net.A["out"], COUT_PAD, self.scale, NF, B, H, W, Uout, out_stride)


def train(chunks_fn, n_chunks, batch=8, H=256, W=256, lr=1e-3, lr_min=1e-5, epochs_per_chunk=1, seed=0,
          chans=(32, 64, 128, 256), k=32, log=None, scale=None, time_budget_s=None, eval_fn=None, eval_every=0,
          curve=None):
    """Train on chunks produced by chunks_fn(i) (fresh trajectories per chunk, or a fixed set
    cycled over).  Cosine learning-rate decay over all iterations.  With eval_fn and
    eval_every, after every eval_every chunks (and at the end) (iteration, seconds,
    eval_fn(surrogate)) is appended to the list `curve`.  Returns (Surrogate, history)."""
    import torch
    net = UNet(chans, seed=seed)
    first = chunks_fn(0)
    scale = field_scales(first) if scale is None else np.asarray(scale)
    sur = Surrogate(net, scale, k)
    iters_per_chunk = epochs_per_chunk * (first.n // batch) * first.J
    total = max(1, n_chunks * iters_per_chunk)
    net._alloc(batch, H, W)
    hist = []
    it = 0
    t0 = time.time()
    rng = np.random.default_rng(seed + 1)
    chunk = first
    for ci in range(n_chunks):
        if ci:
            chunk = chunks_fn(ci)
        stride = 10 * H * W
        for _ in range(epochs_per_chunk):
            blocks = [(j, i0) for j in range(chunk.J) for i0 in range(0, chunk.n - batch + 1, batch)]
            rng.shuffle(blocks)
            for j, i0 in blocks:
                lr_t = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * it / total))
                Unow = chunk.U[j, i0]
                Unext = chunk.U[j + 1, i0]
                sur.pack(Unow, stride, chunk.nu_norm[i0:], batch, H, W)
                K.pack_target(Unow, Unext, stride, NF, sur.scale, batch, H, W, COUT_PAD, net.A["tgt"])
                loss = net.train_step(batch, H, W, lr_t)
                it += 1
                if it % 20 == 0 or it == total:
                    lv = float(loss.item()) / (batch * H * W * NF)
                    hist.append((it, lv, time.time() - t0))
                    if log:
                        log(f"iter {it}/{total} loss {lv:.3e} lr {lr_t:.2e} {time.time() - t0:.1f}s")
                if time_budget_s and time.time() - t0 > time_budget_s:
                    if eval_fn is not None and curve is not None:
                        curve.append((it, round(time.time() - t0, 1), eval_fn(sur)))
                    return sur, hist
        del chunk
        torch.cuda.empty_cache()
        if eval_fn is not None and curve is not None and eval_every and (ci + 1) % eval_every == 0:
            curve.append((it, round(time.time() - t0, 1), eval_fn(sur)))
            if log:
                log(f"chunk {ci + 1}: held-out median {curve[-1][2]:.3e}")
    if eval_fn is not None and curve is not None and (not curve or curve[-1][0] != it):
        curve.append((it, round(time.time() - t0, 1), eval_fn(sur)))
    return sur, hist


def relative_error(sur, Upred, Uref, stride, B, H, W):
    """Relative L2 error over the 5 fields in network units (each field divided by its scale),
    reduced on the GPU; returns one value per sample."""
    import torch
    net = sur.net
    out = torch.empty((1, H, W, COUT_PAD), dtype=torch.float32, device=net.dev)
    ref = torch.empty_like(out)
    zero = torch.zeros_like(out)
    ws = torch.empty(512, dtype=torch.float64, device=net.dev)
    num = torch.empty(1, dtype=torch.float64, device=net.dev)
    den = torch.empty(1, dtype=torch.float64, device=net.dev)
    errs = []
    for b in range(B):
        K.pack_input(Upred[b], stride, NF, sur.scale, None, 1, H, W, COUT_PAD, out)
        K.pack_input(Uref[b], stride, NF, sur.scale, None, 1, H, W, COUT_PAD, ref)
        K.mse(out, ref, H * W, COUT_PAD, NF, 1.0, None, ws, num)
        K.mse(ref, zero, H * W, COUT_PAD, NF, 1.0, None, ws, den)
        errs.append(math.sqrt(float(num.item()) / float(den.item())))
    return np.array(errs)


# ---------------------------------------------------------------------------
# evaluation, timing and the fallback driver
# ---------------------------------------------------------------------------

def evaluate(sur, chunk, batch=16, act_bf16=False):
    """One-jump relative errors on a chunk: surrogate vs the solver's own next snapshot,
    and the persistence baseline U(t + k dt) ~ U(t)."""
    import torch
    H, W = chunk.U.shape[-2:]
    stride = 10 * H * W
    pred = torch.empty((batch, 10, H, W), dtype=torch.float64, device=sur.net.dev)
    errs, pers = [], []
    for j in range(chunk.J):
        for i0 in range(0, chunk.n - batch + 1, batch):
            sur.predict(chunk.U[j, i0], stride, chunk.nu_norm[i0:], batch, H, W, pred, stride, act_bf16=act_bf16)
            errs.extend(relative_error(sur, pred, chunk.U[j + 1, i0:i0 + batch], stride, batch, H, W))
            pers.extend(relative_error(sur, chunk.U[j, i0:i0 + batch], chunk.U[j + 1, i0:i0 + batch], stride, batch,
                                       H, W))
    return np.array(errs), np.array(pers)


def _solver_mode(storage):
    """The fastest batch mode of a storage format: three steps per pass (mode 2) for the
    population formats in FP32 / 16 bits (bit-identical to single steps in FP32), one step per
    launch on staged rows (mode 3) for FP64."""
    return 2 if storage in ("f32", "bf16", "f16") else 3 if storage == "f64" else 0


def _descs_for(nu, H, W, cfl=0.9):
    import workloads as Wk
    out = []
    for v in nu:
        cK2, cmu2 = Wk.material.poisson_to_speeds(float(v))
        c = Wk.material.lattice_speed(cK2, cmu2, cfl)
        dx = 1.0 / max(H, W)
        out.append((W, H, 0, dx, dx / c, math.sqrt(cK2), math.sqrt(cmu2)))
    return out


def relift_and_step(U, nu, k, storage="f64", batch=None):
    """The solver as reference: re-initialise populations from U (Eq. ic_second with periodic
    central-difference derivatives) and run k steps.  U: [n, 10, H, W] FP64 device tensor.
    ``batch``: a lattice batch made for these lattices (lbm_batch_create), reused across
    calls; without it one is created and destroyed here."""
    import torch
    n, _, H, W = U.shape
    descs = _descs_for(nu, H, W)
    dx = descs[0][3]
    stride = 10 * H * W
    dUx = torch.zeros_like(U)
    dUy = torch.zeros_like(U)
    K.gradient(U, stride, NF, n, H, W, dx, dUx, dUy)
    if batch is None:
        b = L.lbm_batch_create(descs, storage=L.STORAGE[storage], stream=torch.cuda.current_stream().cuda_stream)
        L.lbm_batch_set_mode(b, _solver_mode(storage))
    else:
        b = batch
    out = torch.empty_like(U)
    try:
        for i in range(n):
            L.lbm_batch_init(b, i, U[i, :5].contiguous(), dUx[i, :5].contiguous(), dUy[i, :5].contiguous())
        L.lbm_batch_step(b, k)
        for i in range(n):
            L.lbm_batch_moments(b, i, out[i])
        L.lbm_batch_synchronize(b)
    finally:
        if batch is None:
            L.lbm_batch_destroy(b)
    return out


class FallbackDriver:
    """Advances lattices by surrogate jumps of k steps.  Every `check_every`-th jump the
    solver re-runs the jump from the same state and checks the surrogate: a lattice whose
    relative error exceeds `tol` takes the solver's result instead (fallback)."""

    def __init__(self, sur, tol=1e-3, check_every=1, storage="f64"):
        self.sur, self.tol, self.check_every, self.storage = sur, tol, check_every, storage
        self.jumps = 0
        self.fallbacks = 0
        self.checked = 0
        self._batch, self._key = None, None

    def close(self):
        if self._batch is not None:
            L.lbm_batch_destroy(self._batch)
            self._batch, self._key = None, None

    def _solver(self, nu, H, W):
        """The solver batch for these lattices, made once and reused by later checks."""
        import torch
        key = (tuple(float(v) for v in nu), H, W)
        if key != self._key:
            self.close()
            self._batch = L.lbm_batch_create(_descs_for(nu, H, W), storage=L.STORAGE[self.storage],
                                             stream=torch.cuda.current_stream().cuda_stream)
            L.lbm_batch_set_mode(self._batch, _solver_mode(self.storage))
            self._key = key
        return self._batch

    def jump(self, U, nu):
        import torch
        n, _, H, W = U.shape
        stride = 10 * H * W
        nu_norm = torch.tensor((np.asarray(nu) - NU_MEAN) / NU_STD, dtype=torch.float32, device=U.device)
        pred = torch.empty_like(U)
        for i0 in range(0, n, 16):
            bsz = min(16, n - i0)
            self.sur.predict(U[i0], stride, nu_norm[i0:], bsz, H, W, pred[i0], stride)
        self.jumps += 1
        try:
            K.check()                   # a convolution whose bounded wait ran out left invalid output
        except L.LbmError as e:
            if e.status != L.LBM_ERR_TIMEOUT:
                raise
            ref = relift_and_step(U, nu, self.sur.k, self.storage, self._solver(nu, H, W))
            self.fallbacks += n
            return ref, None
        errs = None
        if self.check_every and self.jumps % self.check_every == 0:
            ref = relift_and_step(U, nu, self.sur.k, self.storage, self._solver(nu, H, W))
            errs = relative_error(self.sur, pred, ref, stride, n, H, W)
            self.checked += n
            for i, e in enumerate(errs):
                if not e <= self.tol:
                    pred[i].copy_(ref[i])
                    self.fallbacks += 1
        return pred, errs


def driver_timing(sur, chunk, check_every=(1, 4, 16), tol=1e-3, storage="f32", n=16):
    """Wall-clock of whole fallback-driver jumps on held-out lattices, per lattice and jump,
    everything included: inference, the solver's check every `check_every` jumps and the
    fallback copies.  Each jump starts from the solver's snapshot of the chunk.  Returns, per
    check interval, ms per lattice and jump, the fraction of checked lattices that fell back,
    and the median checked error."""
    import time
    import torch
    H, W = chunk.U.shape[-2:]
    n = min(n, chunk.n)
    nu = chunk.nu[:n]
    out = {}
    for ce in check_every:
        drv = FallbackDriver(sur, tol=tol, check_every=ce, storage=storage)
        drv.jump(chunk.U[0, :n].contiguous(), nu)           # warm-up: builds the solver batch
        drv.jumps = drv.fallbacks = drv.checked = 0
        errs = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in range(chunk.J):
            for _ in range(ce):
                _, e = drv.jump(chunk.U[j, :n], nu)
                if e is not None:
                    errs.extend(e)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[str(ce)] = {"ms_per_lattice_jump": 1e3 * dt / (drv.jumps * n), "jumps": drv.jumps,
                        "checked_lattices": drv.checked, "fallback_fraction": drv.fallbacks / max(1, drv.checked),
                        "median_checked_error": float(np.median(errs)) if errs else None}
        drv.close()
    return out


def timing(sur, n=16, H=256, W=256, reps=5):
    """ms per lattice for one jump: surrogate inference (batch n; hi/lo activations and
    single-BF16 activations) vs k solver steps on a batch of n lattices (FP64, FP32 storage),
    the solver started from the same random moment fields (populations of zero would send the
    FP64 fixed-point update to its fallback for every node)."""
    import torch
    k = sur.k
    stride = 10 * H * W
    rng = np.random.default_rng(5)
    nu = rng.uniform(0, 0.49, n)
    U = torch.zeros((n, 10, H, W), dtype=torch.float64, device=sur.net.dev)
    U[:, :5].normal_(0.0, 1e-3)
    nu_norm = torch.tensor((nu - NU_MEAN) / NU_STD, dtype=torch.float32, device=sur.net.dev)
    out = torch.empty_like(U)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t = {}
    for fast in (False, True):
        sur.predict(U[0], stride, nu_norm, n, H, W, out[0], stride, act_bf16=fast)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            sur.predict(U[0], stride, nu_norm, n, H, W, out[0], stride, act_bf16=fast)
        e1.record()
        torch.cuda.synchronize()
        t[fast] = e0.elapsed_time(e1) / reps / n
    t_sur = t[False]
    res = {"surrogate_ms_per_lattice": t_sur, "surrogate_bf16_act_ms_per_lattice": t[True], "batch": n, "H": H,
           "W": W, "k": k}
    for storage in ("f64", "f32"):
        b = L.lbm_batch_create(_descs_for(nu, H, W), storage=L.STORAGE[storage],
                               stream=torch.cuda.current_stream().cuda_stream)
        zero = torch.zeros((5, H, W), dtype=torch.float64, device=sur.net.dev)
        for i in range(n):
            L.lbm_batch_init(b, i, U[i, :5].contiguous(), zero, zero)
        L.lbm_batch_set_mode(b, _solver_mode(storage), 2 * k)
        L.lbm_batch_step(b, 2 * k)
        L.lbm_batch_synchronize(b)
        e0.record()
        L.lbm_batch_step(b, k * reps)
        e1.record()
        L.lbm_batch_synchronize(b)
        res[f"lbm_{storage}_ms_per_lattice"] = e0.elapsed_time(e1) / reps / n
        L.lbm_batch_destroy(b)
        res[f"gain_vs_{storage}"] = res[f"lbm_{storage}_ms_per_lattice"] / t_sur
        res[f"gain_bf16_act_vs_{storage}"] = res[f"lbm_{storage}_ms_per_lattice"] / t[True]
    return res


def run(out_dir, n_chunks=20, lattices=256, H=256, W=256, k=32, J=4, batch=8, lr=1e-3, time_budget_s=None,
        eval_lattices=64, chans=(32, 64, 128, 256), log=print, distinct_chunks=0, eval_every=0):
    """Generate trajectories, train, evaluate on held-out seeds, time; write report.json.
    distinct_chunks > 0 trains on that many chunks of `lattices` trajectories (seeds
    10000 + i), cycled over for n_chunks chunks (epochs); 0 draws fresh trajectories for
    every chunk.  eval_every > 0 records the held-out error every eval_every chunks on the
    first 16 held-out lattices (the learning curve)."""
    import json
    import os
    import torch
    os.makedirs(out_dir, exist_ok=True)
    if distinct_chunks > 0:
        chunks = lambda i: generate_chunk(lattices, 10_000 + i % distinct_chunks, H=H, W=W, k=k, J=J)
    else:
        chunks = lambda i: generate_chunk(lattices, 10_000 + i, H=H, W=W, k=k, J=J)
    held = generate_chunk(eval_lattices, 900_000, H=H, W=W, k=k, J=J)
    curve = []
    probe = Chunk(held.U[:, :16], held.nu[:16], held.nu_norm[:16], 16, held.J)
    eval_fn = (lambda s: float(np.median(evaluate(s, probe, batch=16)[0]))) if eval_every else None
    t0 = time.time()
    sur, hist = train(chunks, n_chunks, batch=batch, H=H, W=W, lr=lr, chans=chans, k=k, log=log,
                      time_budget_s=time_budget_s, eval_fn=eval_fn, eval_every=eval_every, curve=curve)
    t_train = time.time() - t0
    errs, pers = evaluate(sur, held, batch=16)
    errs_fast, _ = evaluate(sur, held, batch=16, act_bf16=True)
    tm = timing(sur, n=16, H=H, W=W)
    drv = FallbackDriver(sur, tol=1e-3, check_every=1)
    _, derr = drv.jump(held.U[0, :16].contiguous(), held.nu[:16])
    report = {
        "params": sur.net.nparams, "lattice": [H, W], "k": k, "train_chunks": n_chunks, "lattices_per_chunk": lattices,
        "pairs_seen": sur.net.step_count * batch, "iterations": sur.net.step_count, "train_s": round(t_train, 1),
        "final_loss": hist[-1][1] if hist else None,
        "heldout_rel_l2": {"median": float(np.median(errs)), "mean": float(np.mean(errs)), "max": float(np.max(errs))},
        "heldout_rel_l2_bf16_activations": {"median": float(np.median(errs_fast)), "max": float(np.max(errs_fast))},
        "persistence_rel_l2": {"median": float(np.median(pers)), "mean": float(np.mean(pers))},
        "fallback_tol": 1e-3, "fallback_fraction": drv.fallbacks / max(1, drv.checked),
        "check_errors_after_relift": [float(e) for e in derr],
        "timing": tm, "scale": sur.scale_np.tolist(), "history": hist[-50:],
        "distinct_trajectories": (distinct_chunks * lattices) if distinct_chunks > 0 else None,
        "curve": [{"iteration": c[0], "train_s": c[1], "heldout16_rel_l2_median": c[2]} for c in curve],
    }
    json.dump(report, open(os.path.join(out_dir, "report.json"), "w"), indent=1)
    np.savez(os.path.join(out_dir, "weights.npz"), **sur.net.state_dict(), scale=sur.scale_np)
    return sur, report


def kernel_workload(what, batch=16, H=256, W=256, repeats=3, act_bf16=False):
    """A fixed launch sequence for profiling the layer kernels with an untrained network:
    what = "infer" runs `repeats` inferences of `batch` lattices, "train" runs `repeats` + 1
    training steps of `batch` lattices on random inputs and targets."""
    import torch
    net = UNet((32, 64, 128, 256), seed=0)
    if what == "infer":
        sur = Surrogate(net, np.ones(NF), 32)
        stride = 10 * H * W
        U = torch.zeros((batch, 10, H, W), dtype=torch.float64, device=net.dev)
        U[:, :NF].normal_(0.0, 1e-3)
        nu = torch.zeros(batch, dtype=torch.float32, device=net.dev)
        out = torch.empty_like(U)
        for _ in range(repeats):
            sur.predict(U[0], stride, nu, batch, H, W, out[0], stride, act_bf16=act_bf16)
    elif what == "train":
        net._alloc(batch, H, W)
        net.A["x0"].normal_()
        net.A["tgt"].normal_()
        for _ in range(repeats + 1):
            net.train_step(batch, H, W, 1e-4)
    else:
        raise ValueError(what)
    torch.cuda.synchronize()


def layer_timing(batch=16, H=256, W=256, reps=20, chans=(32, 64, 128, 256)):
    """Microseconds per launch of every 3x3 convolution of the U-Net (random inputs and
    weights, ReLU, the decoder's first convolution reading its upsampled input at half
    size), tcgen05 kernel vs mma.sync kernels, hi/lo and single-BF16 activations, and of
    its weight gradient (block-tiled vs per-tap kernel); then inference (ms per lattice,
    `timing`) and one training step (batch 8) with each forward kernel family."""
    import torch
    c = list(chans)
    shapes = []
    for l in range(4):
        shapes += [(f"enc{l}a", H >> l, c[l - 1] if l else CIN_PAD, 0, c[l], False),
                   (f"enc{l}b", H >> l, c[l], 0, c[l], False)]
    for l in (2, 1, 0):
        shapes += [(f"dec{l}a", H >> l, c[l + 1], c[l], c[l], True), (f"dec{l}b", H >> l, c[l], 0, c[l], False)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    gen = torch.Generator(device="cuda").manual_seed(3)
    layers = []
    for name, h, C1, C2, Co, half in shapes:
        w_ = h * W // H
        h1, w1 = (h // 2, w_ // 2) if half else (h, w_)
        x1 = torch.randn(batch, h1, w1, C1, device="cuda", generator=gen)
        x2 = torch.randn(batch, h, w_, C2, device="cuda", generator=gen) if C2 else None
        wt = (torch.randn(Co, 3, 3, C1 + C2, device="cuda", generator=gen) * 0.05).to(torch.bfloat16)
        bias = torch.randn(Co, device="cuda", generator=gen)
        y = torch.empty(batch, h, w_, Co, device="cuda")
        flop = 2.0 * batch * h * w_ * 9 * (C1 + C2) * Co
        r = {"layer": name, "H": h, "W": w_, "Cin": C1 + C2, "Cout": Co}
        for act in (False, True):
            for ms in (False, True):
                def f():
                    K.conv_forward(x1, C1, x2, C2, wt, bias, y, Co, None, Co, batch, h, w_, 3, relu=True,
                                   x1_half=half, act_bf16=act, mma_sync=ms)
                for _ in range(3):
                    f()
                torch.cuda.synchronize()
                e0.record()
                for _ in range(reps):
                    f()
                e1.record()
                torch.cuda.synchronize()
                us = e0.elapsed_time(e1) / reps * 1e3
                key = ("bf16_act_" if act else "") + ("mma_sync" if ms else "tcgen05")
                r[key + "_us"] = round(us, 1)
                r[key + "_tflops"] = round(flop / us / 1e6, 1)
        # weight gradient of the same layer (dY = y), block-tiled vs per-tap kernel
        ws_w = torch.empty(K.wgrad_workspace_bytes(C1 + C2, Co, batch, h, w_, 3) // 4 + 1, device="cuda")
        dw = torch.empty(Co, 3, 3, C1 + C2, device="cuda")
        for per_tap in (False, True):
            def fw():
                K.conv_backward_weight(y, Co, x1, C1, x2, C2, batch, h, w_, 3, dw, ws_w, x1_half=half,
                                       per_tap=per_tap)
            for _ in range(2):
                fw()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(max(1, reps // 4)):
                fw()
            e1.record()
            torch.cuda.synchronize()
            r["wgrad_" + ("per_tap" if per_tap else "tiled") + "_us"] = round(
                e0.elapsed_time(e1) / max(1, reps // 4) * 1e3, 1)
        K.check()
        layers.append(r)
    out = {"batch": batch, "layers": layers,
           "sum_us": {k: round(sum(r[k] for r in layers), 1) for k in layers[0] if k.endswith("_us")}}
    net = UNet(chans, seed=0)
    sur = Surrogate(net, np.ones(NF), 32)
    for ms in (False, True):
        K.use_mma_sync(ms)
        try:
            t = timing(sur, n=batch, H=H, W=W)
            net._alloc(8, H, W)
            net.A["x0"].normal_(generator=gen)
            net.A["tgt"].normal_(generator=gen)
            for _ in range(2):
                net.train_step(8, H, W, 1e-4)
            torch.cuda.synchronize()
            e0.record()
            for _ in range(5):
                net.train_step(8, H, W, 1e-4)
            e1.record()
            torch.cuda.synchronize()
            t["train_step_ms_batch8"] = e0.elapsed_time(e1) / 5
            K.check()
        finally:
            K.use_mma_sync(False)
        out["mma_sync" if ms else "tcgen05"] = t
    return out


if __name__ == "__main__":
    import argparse
    ap = argparse.ArgumentParser(description="train and evaluate the surrogate on solver trajectories")
    ap.add_argument("--out", default="surrogate_run")
    ap.add_argument("--chunks", type=int, default=20)
    ap.add_argument("--lattices", type=int, default=256)
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--budget", type=float, default=None, help="training time budget in seconds")
    ap.add_argument("--distinct-chunks", type=int, default=0,
                    help="train on this many chunks of trajectories, cycled over (0: fresh trajectories per chunk)")
    ap.add_argument("--eval-every", type=int, default=0, help="record the held-out error every N chunks")
    ap.add_argument("--kernels", choices=["infer", "train"], default=None,
                    help="only run a fixed launch sequence of the layer kernels (for profiling)")
    ap.add_argument("--layer-timing", action="store_true",
                    help="time every 3x3 convolution, inference and a training step (tcgen05 vs mma.sync)")
    a = ap.parse_args()
    if a.layer_timing:
        import json
        print(json.dumps(layer_timing(batch=a.batch, H=a.size, W=a.size), indent=1))
    elif a.kernels:
        kernel_workload(a.kernels, batch=a.batch, H=a.size, W=a.size)
        print("done")
    else:
        _, rep = run(a.out, a.chunks, a.lattices, a.size, a.size, a.k, batch=a.batch, lr=a.lr,
                     time_budget_s=a.budget, distinct_chunks=a.distinct_chunks, eval_every=a.eval_every)
        import json
        print(json.dumps({k: v for k, v in rep.items() if k != "history"}, indent=1))
