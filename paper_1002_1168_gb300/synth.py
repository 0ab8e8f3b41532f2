"""Seeded synthetic VOP sequences (8-bit luma + binary alpha per object).

This module only draws inputs: it holds none of the motion-estimation
arithmetic.  Textures are sums of sinusoids evaluated analytically at the
(sub-pixel, rotated, scaled) source coordinates, so no interpolation enters the
ground truth.  Objects are ellipses whose contour may be perturbed by a few
Fourier harmonics; each object is its own video object plane (VOP) with its own
alpha plane over the frame grid, painted over a translating background, with
Gaussian noise added per frame, rounded and clamped to 0..255.

The paper evaluates on four QCIF MPEG-4 test sequences (Sec. 4) that are not
available here; the named workloads below stand in for them with the frame
sizes, motion ranges and object structure of the workloads being measured.
All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Texture:
    """Sum of sinusoids; value range scaled to [0, 255] at its extremes."""
    kx: np.ndarray
    ky: np.ndarray
    phase: np.ndarray
    amp: np.ndarray

    @staticmethod
    def random(rng, n=8, period=(16.0, 128.0)):
        theta = rng.uniform(0.0, 2.0 * np.pi, n)
        per = rng.uniform(period[0], period[1], n)
        k = 2.0 * np.pi / per
        return Texture(k * np.cos(theta), k * np.sin(theta), rng.uniform(0, 2 * np.pi, n),
                       rng.uniform(0.2, 1.0, n))

    def __call__(self, x, y):
        s = np.zeros(np.broadcast(x, y).shape, np.float64)
        for i in range(len(self.amp)):
            s += self.amp[i] * np.sin(self.kx[i] * x + self.ky[i] * y + self.phase[i])
        return 127.5 + 127.5 * s / self.amp.sum()

    def grid(self, xs, ys, ca=1.0, sa=0.0, scale=1.0):
        """The texture at local coordinates q = R(-angle) (p - origin) / scale
        for the grid p = (xs[i], ys[j]) given relative to the origin; each
        wave sin(kx qx + ky qy + phase) = sin(al x + ph) cos(be y) +
        cos(al x + ph) sin(be y) is built from 1-D tables."""
        al = (self.kx * ca + self.ky * sa) / scale
        be = (self.ky * ca - self.kx * sa) / scale
        ax = np.outer(al, xs) + self.phase[:, None]           # [n, W]
        by = np.outer(be, ys)                                 # [n, H]
        left = np.concatenate([(self.amp[:, None] * np.cos(by)).T, (self.amp[:, None] * np.sin(by)).T], axis=1)
        right = np.concatenate([np.sin(ax), np.cos(ax)], axis=0)
        return 127.5 + (127.5 / self.amp.sum()) * (left @ right)


@dataclass
class MovingObject:
    """An elliptical (optionally blobby) object with its own texture.

    ``centers[t]`` is the object centre in frame t; ``angles[t]`` (radians)
    and ``scales[t]`` give its rotation and scale.  The contour in polar form is
    r(th) = 1 + sum_k c_k cos(k th + psi_k) on the unit ellipse with semi-axes
    (a, b)."""
    a: float
    b: float
    texture: Texture
    centers: np.ndarray
    angles: np.ndarray
    scales: np.ndarray
    harm_c: np.ndarray = field(default_factory=lambda: np.zeros(0))
    harm_psi: np.ndarray = field(default_factory=lambda: np.zeros(0))

    def local(self, t, X, Y):
        cx, cy = self.centers[t]
        ang, sc = self.angles[t], self.scales[t]
        dx, dy = X - cx, Y - cy
        ca, sa = np.cos(-ang), np.sin(-ang)
        return (ca * dx - sa * dy) / sc, (sa * dx + ca * dy) / sc

    def inside(self, qx, qy):
        ex, ey = qx / self.a, qy / self.b
        rho = np.hypot(ex, ey)
        th = np.arctan2(ey, ex)
        r = np.ones_like(rho)
        for k, (c, psi) in enumerate(zip(self.harm_c, self.harm_psi)):
            r += c * np.cos((k + 2) * th + psi)
        return rho <= r


@dataclass
class Sequence:
    """luma [F,H,W] u8 (composited), alpha [n_obj,F,H,W] u8 (0/255)."""
    luma: np.ndarray
    alpha: np.ndarray
    seed: int
    meta: dict

    @property
    def frames(self):
        return self.luma.shape[0]

    @property
    def height(self):
        return self.luma.shape[1]

    @property
    def width(self):
        return self.luma.shape[2]


def render(W, H, F, background: Texture, bg_offsets, objects, noise_sigma, rng) -> tuple:
    """Composite background + objects per frame, add noise, return (luma, alpha).
    Object masks and textures are evaluated inside each object's bounding box."""
    xs, ys = np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64)
    luma = np.empty((F, H, W), np.uint8)
    alpha = np.zeros((len(objects), F, H, W), np.uint8)
    for t in range(F):
        ox, oy = bg_offsets[t]
        img = background.grid(xs - ox, ys - oy)
        for i, ob in enumerate(objects):
            cx, cy = ob.centers[t]
            ang, sc = ob.angles[t], ob.scales[t]
            rad = max(ob.a, ob.b) * (1.0 + float(np.abs(ob.harm_c).sum())) * sc + 2.0
            x0, x1 = max(0, int(np.floor(cx - rad))), min(W, int(np.ceil(cx + rad)) + 1)
            y0, y1 = max(0, int(np.floor(cy - rad))), min(H, int(np.ceil(cy + rad)) + 1)
            if x0 >= x1 or y0 >= y1:
                continue
            bx, by = xs[x0:x1] - cx, ys[y0:y1] - cy
            ca, sa = np.cos(-ang), np.sin(-ang)
            qx = (ca * bx[None, :] - sa * by[:, None]) / sc
            qy = (sa * bx[None, :] + ca * by[:, None]) / sc
            m = ob.inside(qx, qy)
            tex = ob.texture.grid(bx, by, ca, sa, sc)
            sub = img[y0:y1, x0:x1]
            img[y0:y1, x0:x1] = np.where(m, tex, sub)
            alpha[i, t, y0:y1, x0:x1] = np.where(m, 255, 0).astype(np.uint8)
        if noise_sigma > 0:
            img = img + rng.normal(0.0, noise_sigma, img.shape)
        luma[t] = np.clip(np.rint(img), 0, 255).astype(np.uint8)
    return luma, alpha


def _bounce_path(rng, start, F, vmax, half_extent, W, H, change_every, integer=False, vmin=1.0):
    """Piecewise-constant velocity path kept inside the frame by reflection."""
    pos = np.array(start, np.float64)
    path = np.zeros((F, 2))
    v = None
    for t in range(F):
        if t % change_every == 0:
            mag = rng.uniform(vmin, vmax)
            ang = rng.uniform(0, 2 * np.pi)
            v = np.array([mag * np.cos(ang), mag * np.sin(ang)])
            if integer:
                v = np.rint(v)
        path[t] = pos
        nxt = pos + v
        for ax, lim in ((0, W), (1, H)):
            lo, hi = half_extent[ax] + 2, lim - half_extent[ax] - 2
            if nxt[ax] < lo or nxt[ax] > hi:
                v[ax] = -v[ax]
                nxt[ax] = pos[ax] + v[ax]
        pos = np.clip(nxt, [half_extent[0], half_extent[1]], [W - half_extent[0], H - half_extent[1]])
    return path


def draw_scene(W, H, F, seed, n_objects=1, vmax=8.0, bg_step=(1.0, 0.5), blobby=True, change_every=10,
               max_rot_deg=0.0, scale_range=(1.0, 1.0), obj_frac=0.30, integer_motion=False):
    """Scene parameters of make_sequence (background texture and offsets, the
    objects with their paths) and the generator, positioned for the noise."""
    rng = np.random.default_rng(seed)
    background = Texture.random(rng)
    bstep = np.array(bg_step, np.float64)
    bg_offsets = np.array([bstep * t for t in range(F)])
    objects = []
    for i in range(n_objects):
        a = obj_frac * min(W, H) * rng.uniform(0.8, 1.2) / np.sqrt(n_objects)
        b = a * rng.uniform(0.6, 0.9)
        ext = (min(a * 1.5, 0.45 * W), min(a * 1.5, 0.45 * H))
        start = (rng.uniform(ext[0], W - ext[0]), rng.uniform(ext[1], H - ext[1]))
        centers = _bounce_path(rng, start, F, vmax, ext, W, H, change_every, integer_motion)
        rot_rate = np.deg2rad(rng.uniform(-max_rot_deg, max_rot_deg))
        angles = rng.uniform(0, np.pi) + rot_rate * np.arange(F)
        s_end = rng.uniform(*scale_range)
        scales = np.linspace(1.0, s_end, F) if F > 1 else np.ones(1)
        if blobby:
            hc = rng.uniform(0.0, 0.15, 4)
            hp = rng.uniform(0, 2 * np.pi, 4)
        else:
            hc, hp = np.zeros(0), np.zeros(0)
        objects.append(MovingObject(a, b, Texture.random(rng), centers, angles, scales, hc, hp))
    return background, bg_offsets, objects, rng


def make_sequence(W, H, F, seed, n_objects=1, vmax=8.0, bg_step=(1.0, 0.5), noise_sigma=3.0,
                  blobby=True, change_every=10, max_rot_deg=0.0, scale_range=(1.0, 1.0),
                  obj_frac=0.30, integer_motion=False):
    """Generic sequence: n_objects moving objects over a translating background."""
    background, bg_offsets, objects, rng = draw_scene(W, H, F, seed, n_objects, vmax, bg_step, blobby, change_every,
                                                      max_rot_deg, scale_range, obj_frac, integer_motion)
    bstep = np.array(bg_step, np.float64)
    luma, alpha = render(W, H, F, background, bg_offsets, objects, noise_sigma, rng)
    meta = dict(width=W, height=H, frames=F, n_objects=n_objects, vmax=vmax, noise_sigma=noise_sigma,
                bg_step=list(bstep), seed=seed, generator="numpy PCG64")
    return Sequence(luma, alpha, seed, meta)


def qcif_pair(seed=1001, shift=None, bg_shift=None, noise_sigma=2.0):
    """QCIF 176x144 single pair: an ellipse with its own texture translated by an
    integer (dx, dy) in [-7, 7]^2 over a background moved by another integer
    vector; noise sigma 2.  Search range 16, full-pel."""
    W, H = 176, 144
    rng = np.random.default_rng(seed)
    background = Texture.random(rng)
    if shift is None:
        shift = rng.integers(-7, 8, 2)
    if bg_shift is None:
        while True:
            bg_shift = rng.integers(-4, 5, 2)
            if tuple(bg_shift) != tuple(shift):
                break
    a, b = 52.0, 38.0
    c0 = np.array([W / 2 + rng.uniform(-6, 6), H / 2 + rng.uniform(-6, 6)])
    centers = np.array([c0, c0 + np.asarray(shift, np.float64)])
    ob = MovingObject(a, b, Texture.random(rng), centers, np.array([0.0, 0.0]), np.ones(2))
    bg_offsets = np.array([[0.0, 0.0], np.asarray(bg_shift, np.float64)])
    luma, alpha = render(W, H, 2, background, bg_offsets, [ob], noise_sigma, rng)
    meta = dict(width=W, height=H, frames=2, shift=[int(s) for s in shift],
                bg_shift=[int(s) for s in bg_shift], noise_sigma=noise_sigma, seed=seed,
                search_range=16, subpel=1)
    return Sequence(luma, alpha, seed, meta)


def cif_sequence(seed=1002, frames=30):
    """CIF 352x288, 30 frames: one blobby object (Fourier-perturbed ellipse)
    under piecewise-constant sub-pixel translation |v| <= 8 px/frame (changing
    every 10 frames) over a globally translating background, noise sigma 3.
    Search range 16, half-pel."""
    seq = make_sequence(352, 288, frames, seed, n_objects=1, vmax=8.0, bg_step=(1.25, -0.5),
                        noise_sigma=3.0, blobby=True, change_every=10, obj_frac=0.33)
    seq.meta.update(search_range=16, subpel=2)
    return seq


BATCH_SIZES = [(176, 144)] * 16 + [(352, 288)] * 24 + [(704, 576)] * 16 + [(1920, 1088)] * 8


def batch_sequences(seed=1003, frames=10, sizes=None):
    """64 independent sequences of uneven size (16 QCIF, 24 CIF, 16 4CIF,
    8 1920x1088), 10 frames each, 1-4 objects with |v| <= 16 px/frame.
    Search range 16, half-pel."""
    sizes = BATCH_SIZES if sizes is None else sizes
    rng = np.random.default_rng(seed)
    out = []
    for i, (W, H) in enumerate(sizes):
        n_obj = int(rng.integers(1, 5))
        seq = make_sequence(W, H, frames, seed * 1000 + i, n_objects=n_obj, vmax=16.0,
                            bg_step=tuple(rng.uniform(-2, 2, 2)), noise_sigma=2.0,
                            blobby=True, change_every=5, obj_frac=0.30)
        seq.meta.update(search_range=16, subpel=2)
        out.append(seq)
    return out


def translated_pair(W, H, shift, seed=7, period=(32.0, 128.0), noise_sigma=0.0, subpel_shift=False):
    """A textured frame and its copy translated by `shift` pixels (content moves
    by +shift), fully opaque alpha.  Low-frequency texture, optional noise."""
    rng = np.random.default_rng(seed)
    tex = Texture.random(rng, period=period)
    Y, X = np.mgrid[0:H, 0:W].astype(np.float64)
    f0 = tex(X, Y)
    f1 = tex(X - shift[0], Y - shift[1])
    if noise_sigma > 0:
        f0 = f0 + rng.normal(0, noise_sigma, f0.shape)
        f1 = f1 + rng.normal(0, noise_sigma, f1.shape)
    luma = np.stack([f0, f1])
    luma = np.clip(np.rint(luma), 0, 255).astype(np.uint8)
    alpha = np.full((2, H, W), 255, np.uint8)
    return luma, alpha


def random_frames(W, H, F, seed, alpha_density=0.5, alpha_blobs=True):
    """Unstructured random luma (uniform 0..255) and alpha (random blobs or
    i.i.d. pixels) -- stresses edge cases rather than realism."""
    rng = np.random.default_rng(seed)
    luma = rng.integers(0, 256, (F, H, W), dtype=np.uint8)
    if alpha_blobs:
        Y, X = np.mgrid[0:H, 0:W]
        alpha = np.zeros((F, H, W), np.uint8)
        for t in range(F):
            for _ in range(3):
                cx, cy = rng.uniform(0, W), rng.uniform(0, H)
                r = rng.uniform(8, max(W, H) / 2)
                alpha[t][(X - cx) ** 2 + (Y - cy) ** 2 <= r * r] = 255
    else:
        alpha = np.where(rng.random((F, H, W)) < alpha_density, 255, 0).astype(np.uint8)
    return luma, alpha


def seednet_init(seed, channels=(16, 32, 32, 32, 32, 16)):
    """Initial weights of the seed network: He-normal (std sqrt(2 / (9 cin))),
    the last layer at a tenth of that, zero biases; numpy PCG64."""
    rng = np.random.default_rng(seed)
    out = []
    for li in range(5):
        cin, cout = channels[li], channels[li + 1]
        std = np.sqrt(2.0 / (9 * cin)) * (0.1 if li == 4 else 1.0)
        out.append((rng.normal(0.0, std, (cout, 3, 3, cin)), np.zeros(cout)))
    return out
