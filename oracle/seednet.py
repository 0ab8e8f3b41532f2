"""CPU oracle of the learned seed proposal network -- TEST INFRASTRUCTURE ONLY.

The learned proposal of the GB300 build (not in the paper: the paper's block
recursive search seeds from neighbour and temporal vectors, Sec. 3.1) is a
5-layer 3x3 convolutional network with 32 channels on a quarter-resolution
grid (one cell = 4x4 pixels, one MB = 4x4 cells) that predicts one (dx, dy)
seed in pixels per MB.  This module restates its forward pass, its loss and
its backward pass in float64 numpy, rounding to bfloat16 exactly where the
GPU kernels store bfloat16 (inputs, weights, hidden activations, gradients
fed to the convolutions), so the GPU results can be compared within the
accumulation-order tolerance.  Only tests/ and bench.py's reference legs use
it; it shares no code with the CUDA path.

Layout: activations [N, Hc, Wc, C] (channels last); weights [Cout, 3, 3, Cin].
Layers: 16 -> 32 -> 32 -> 32 -> 32 -> 16 channels (the last layer's first two
channels are the cell's (dx, dy) / 8 px; its other outputs are padding),
ReLU after the first four.
"""
from __future__ import annotations

import numpy as np

CHANNELS = [16, 32, 32, 32, 32, 16]
SEED_SCALE = 8.0  # cell output 1.0 = 8 px
HUBER = 1.0       # px


def bf16(x):
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    f = np.asarray(x, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def features(ref, cur, temporal, subpel):
    """Input grid of one frame pair: per 4x4 cell the current and reference
    mean luma (/255 - 0.5), their difference, and the temporal candidate of
    the cell's MB (in pixels / 16); 16 channels, the rest zero; bfloat16."""
    H, W = cur.shape
    Hc, Wc = H // 4, W // 4
    c = cur.astype(np.float64).reshape(Hc, 4, Wc, 4).mean(axis=(1, 3))
    r = ref.astype(np.float64).reshape(Hc, 4, Wc, 4).mean(axis=(1, 3))
    x = np.zeros((Hc, Wc, 16))
    x[..., 0] = c / 255.0 - 0.5
    x[..., 1] = r / 255.0 - 0.5
    x[..., 2] = (c - r) / 255.0
    if temporal is not None:
        t = np.asarray(temporal, np.float64).reshape(H // 16, W // 16, 2) / (16.0 * subpel)
        x[..., 3] = np.repeat(np.repeat(t[..., 0], 4, 0), 4, 1)
        x[..., 4] = np.repeat(np.repeat(t[..., 1], 4, 0), 4, 1)
    return bf16(x)


def conv3x3(x, w, b):
    """y[n,i,j,o] = b[o] + sum_{dy,dx,c} x[n,i+dy-1,j+dx-1,c] w[o,dy,dx,c], zero padding."""
    N, H, W, C = x.shape
    xp = np.zeros((N, H + 2, W + 2, C))
    xp[:, 1:-1, 1:-1] = x
    y = np.zeros((N, H, W, w.shape[0])) + b
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("nhwc,oc->nhwo", xp[:, dy:dy + H, dx:dx + W], w[:, dy, dx])
    return y


def conv3x3_grad(x, w, dy_):
    """Gradients of conv3x3 w.r.t. its input, weights and bias."""
    N, H, W, C = x.shape
    xp = np.zeros((N, H + 2, W + 2, C))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            dw[:, dy, dx] = np.einsum("nhwo,nhwc->oc", dy_, xp[:, dy:dy + H, dx:dx + W])
            dxp[:, dy:dy + H, dx:dx + W] += np.einsum("nhwo,oc->nhwc", dy_, w[:, dy, dx])
    return dxp[:, 1:-1, 1:-1], dw, dy_.sum(axis=(0, 1, 2))


def forward(x, params, round_bf16=True):
    """Returns the list of layer outputs (post-activation); hidden outputs are
    rounded to bfloat16, the last layer stays in full precision."""
    acts = [x]
    for li, (w, b) in enumerate(params):
        wq = bf16(w) if round_bf16 else w
        y = conv3x3(acts[-1], wq, b)
        if li < len(params) - 1:
            y = np.maximum(y, 0.0)
            if round_bf16:
                y = bf16(y)
        acts.append(y)
    return acts


def pool_seeds(out):
    """Per-MB seed in pixels: SEED_SCALE x mean over the MB's 4x4 cells of
    output channels 0, 1.  out [N, Hc, Wc, C] -> [N, Hc/4 * Wc/4, 2]."""
    N, Hc, Wc, _ = out.shape
    s = out[..., :2].reshape(N, Hc // 4, 4, Wc // 4, 4, 2).mean(axis=(2, 4))
    return SEED_SCALE * s.reshape(N, -1, 2)


def loss_and_grad(out, labels, mask):
    """Huber loss (threshold HUBER px) between the pooled seeds and the labels
    (pixels) over the MBs with mask != 0, averaged over those MBs; returns the
    loss and d loss / d out."""
    N, Hc, Wc, C = out.shape
    seeds = pool_seeds(out)
    r = seeds - labels
    m = (np.asarray(mask) != 0)[..., None].astype(np.float64)
    n = max(float(m.sum()), 1.0)
    a = np.abs(r)
    loss = float((np.where(a <= HUBER, 0.5 * r * r, HUBER * (a - 0.5 * HUBER)) * m).sum() / n)
    gs = np.clip(r, -HUBER, HUBER) * m / n  # d loss / d seed
    g = gs.reshape(N, Hc // 4, 1, Wc // 4, 1, 2) * (SEED_SCALE / 16.0)
    d = np.zeros_like(out)
    d[..., :2] = np.broadcast_to(g, (N, Hc // 4, 4, Wc // 4, 4, 2)).reshape(N, Hc, Wc, 2)
    return loss, d


def backward(acts, params, dout, round_bf16=True):
    """Weight and bias gradients of every layer.  The gradient entering each
    convolution is rounded to bfloat16 (as the GPU feeds it to tensor cores)."""
    grads = [None] * len(params)
    g = dout
    for li in range(len(params) - 1, -1, -1):
        w, b = params[li]
        wq = bf16(w) if round_bf16 else w
        gq = bf16(g) if round_bf16 else g
        dx, dw, db = conv3x3_grad(acts[li], wq, gq)
        grads[li] = (dw, db)
        if li > 0:
            g = dx * (acts[li] > 0)
    return grads


ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def adam_step(p, g, m, v, t, lr):
    """One Adam update of the flat FP32 master parameters (Kingma and Ba,
    "Adam: A Method for Stochastic Optimization", Algorithm 1, with
    bias-corrected moments), every operation in float32 as the GPU applies it:
        m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
        p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps).
    t counts the updates from 1.  Returns the new (p, m, v)."""
    f32 = np.float32
    p, g, m, v = (np.asarray(a, f32) for a in (p, g, m, v))
    b1, b2, eps, lr = f32(ADAM_B1), f32(ADAM_B2), f32(ADAM_EPS), f32(lr)
    m = b1 * m + (f32(1) - b1) * g
    v = b2 * v + (f32(1) - b2) * g * g
    c1 = f32(1) - b1 ** f32(t)
    c2 = f32(1) - b2 ** f32(t)
    p = p - lr * (m / c1) / (np.sqrt(v / c2) + eps)
    return p, m, v


def init_params(seed):
    """He-normal weights and zero biases from numpy PCG64; the last layer starts
    at one tenth of that scale."""
    rng = np.random.default_rng(seed)
    params = []
    for li in range(5):
        cin, cout = CHANNELS[li], CHANNELS[li + 1]
        std = np.sqrt(2.0 / (9 * cin)) * (0.1 if li == 4 else 1.0)
        params.append((rng.normal(0.0, std, (cout, 3, 3, cin)), np.zeros(cout)))
    return params
