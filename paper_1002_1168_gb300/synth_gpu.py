"""Seeded synthetic VOP sequences rendered on the GPU, for the large
workloads (1920x1088 x 300 frames with 4 objects; 16 sequences of 3840x2160 x
60 frames with 8 objects) whose CPU rendering would take many minutes.

The scene model and its parameters are those of synth.make_sequence (drawn by
synth.draw_scene from the same numpy PCG64 seed): sinusoid textures evaluated
analytically at the objects' rotated and scaled coordinates, blobby ellipses,
a translating background.  The images are evaluated in FP32 with PyTorch on
the device and the per-frame Gaussian noise comes from a torch CUDA generator
seeded from the sequence seed, so frames are not bit-identical to the CPU
renderer's (nothing compares them); both the CUDA path and the oracle
receive the same arrays.  Holds none of the motion-estimation arithmetic.
"""
from __future__ import annotations

import numpy as np

from . import synth


def _texture_grid(torch, tex, xs, ys, ca=1.0, sa=0.0, scale=1.0):
    """tex at q = R(-angle) p / scale over the grid p = (xs[j], ys[i]), built
    from 1-D tables as in synth.Texture.grid; FP32 [len(ys), len(xs)]."""
    dev = xs.device
    al = torch.tensor((tex.kx * ca + tex.ky * sa) / scale, dtype=torch.float32, device=dev)
    be = torch.tensor((tex.ky * ca - tex.kx * sa) / scale, dtype=torch.float32, device=dev)
    ph = torch.tensor(tex.phase, dtype=torch.float32, device=dev)
    amp = torch.tensor(tex.amp, dtype=torch.float32, device=dev)
    ax = al[:, None] * xs[None, :] + ph[:, None]          # [n, W]
    by = be[:, None] * ys[None, :]                         # [n, H]
    left = torch.cat([(amp[:, None] * torch.cos(by)).T, (amp[:, None] * torch.sin(by)).T], dim=1)
    right = torch.cat([torch.sin(ax), torch.cos(ax)], dim=0)
    return 127.5 + (127.5 / float(tex.amp.sum())) * (left @ right)


def render_gpu(W, H, F, background, bg_offsets, objects, noise_sigma, seed, device="cuda"):
    """luma [F, H, W] u8 and alpha [n_obj, F, H, W] u8 (0/255) on the device."""
    import torch

    xs = torch.arange(W, dtype=torch.float32, device=device)
    ys = torch.arange(H, dtype=torch.float32, device=device)
    luma = torch.empty((F, H, W), dtype=torch.uint8, device=device)
    alpha = torch.zeros((len(objects), F, H, W), dtype=torch.uint8, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    for t in range(F):
        ox, oy = bg_offsets[t]
        img = _texture_grid(torch, background, xs - float(ox), ys - float(oy))
        for i, ob in enumerate(objects):
            cx, cy = ob.centers[t]
            ang, sc = ob.angles[t], ob.scales[t]
            rad = max(ob.a, ob.b) * (1.0 + float(np.abs(ob.harm_c).sum())) * sc + 2.0
            x0, x1 = max(0, int(np.floor(cx - rad))), min(W, int(np.ceil(cx + rad)) + 1)
            y0, y1 = max(0, int(np.floor(cy - rad))), min(H, int(np.ceil(cy + rad)) + 1)
            if x0 >= x1 or y0 >= y1:
                continue
            bx, by = xs[x0:x1] - float(cx), ys[y0:y1] - float(cy)
            ca, sa = float(np.cos(-ang)), float(np.sin(-ang))
            qx = (ca * bx[None, :] - sa * by[:, None]) / sc
            qy = (sa * bx[None, :] + ca * by[:, None]) / sc
            ex, ey = qx / ob.a, qy / ob.b
            rho = torch.hypot(ex, ey)
            th = torch.atan2(ey, ex)
            r = torch.ones_like(rho)
            for k, (c, psi) in enumerate(zip(ob.harm_c, ob.harm_psi)):
                r = r + float(c) * torch.cos((k + 2) * th + float(psi))
            m = rho <= r
            tex = _texture_grid(torch, ob.texture, bx, by, ca, sa, sc)
            img[y0:y1, x0:x1] = torch.where(m, tex, img[y0:y1, x0:x1])
            alpha[i, t, y0:y1, x0:x1] = m.to(torch.uint8) * 255
        if noise_sigma > 0:
            img = img + noise_sigma * torch.randn((H, W), generator=gen, device=device, dtype=torch.float32)
        luma[t] = torch.clamp(torch.round(img), 0, 255).to(torch.uint8)
    return luma, alpha


def make_sequence_gpu(W, H, F, seed, n_objects=1, vmax=8.0, bg_step=(1.0, 0.5), noise_sigma=3.0, blobby=True,
                      change_every=10, max_rot_deg=0.0, scale_range=(1.0, 1.0), obj_frac=0.30, device="cuda",
                      render_frames=None):
    """synth.make_sequence's scene, rendered on the device: (luma, alpha, meta).
    render_frames: only the first frames of the F-frame scene (identical to
    those of the whole rendering: the scene is drawn for F frames and the
    noise is drawn frame after frame)."""
    background, bg_offsets, objects, _ = synth.draw_scene(W, H, F, seed, n_objects, vmax, bg_step, blobby,
                                                          change_every, max_rot_deg, scale_range, obj_frac)
    Fr = F if render_frames is None else min(F, render_frames)
    luma, alpha = render_gpu(W, H, Fr, background, bg_offsets, objects, noise_sigma, seed, device)
    meta = dict(width=W, height=H, frames=F, n_objects=n_objects, vmax=vmax, noise_sigma=noise_sigma,
                seed=seed, generator="numpy PCG64 scene, torch CUDA noise, FP32 device rendering")
    return luma, alpha, meta


def hd_learned_eval(seed=1004, frames=300, device="cuda"):
    """1920x1088, 300 frames, 4 objects (4 VOPs) with translation |v| <= 8,
    rotation <= 5 deg and scale 0.95-1.05 over the sequence, noise sigma 2;
    search range 16, half-pel: the evaluation workload of the learned
    proposal."""
    return make_sequence_gpu(1920, 1088, frames, seed, n_objects=4, vmax=8.0, bg_step=(1.0, -0.5), noise_sigma=2.0,
                             change_every=30, max_rot_deg=5.0, scale_range=(0.95, 1.05), obj_frac=0.30,
                             device=device)


def uhd_batch(seed=1005, n_seq=16, frames=60, device="cuda"):
    """16 sequences of 3840x2160, 60 frames, 8 objects each (8 VOPs) with
    translation |v| <= 32 px/frame and rotation <= 3 deg, noise sigma 2;
    object radii chosen to cover about 2-5 % of the frame each; search range
    32, half-pel.  Returns [(luma, alpha, meta)] on the device."""
    out = []
    rng = np.random.default_rng(seed)
    for i in range(n_seq):
        out.append(make_sequence_gpu(3840, 2160, frames, seed * 1000 + i, n_objects=8, vmax=32.0,
                                     bg_step=tuple(rng.uniform(-4, 4, 2)), noise_sigma=2.0, change_every=20,
                                     max_rot_deg=3.0, scale_range=(1.0, 1.0), obj_frac=0.35, device=device))
    return out
