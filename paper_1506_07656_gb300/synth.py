"""Seeded synthetic image pairs with known ground-truth flow.

The paper evaluates on MPI-Sintel (1024x436), Kitti (1242x375), Mikolajczyk and
Middlebury (Sec. 5.1); none of them ship with this library, so every input is
generated here from a seed.  The generators reproduce the sizes of those
datasets and displacement statistics of the kind the paper reports for them
(Sec. 5.1: large displacements of tens of pixels), not their content.

This module holds no arithmetic of the matching method itself: it only makes
gray images in [0, 1] (value noise, repeated motifs), warps them with smooth
displacement fields by bilinear resampling, and returns the flow that maps each
pixel of the first image into the second.  Both the CUDA path and the CPU
oracle consume its outputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def _smoothstep(t: np.ndarray) -> np.ndarray:
    return t * t * (3.0 - 2.0 * t)


def _lattice_interp(lat: np.ndarray, W: int, H: int, cell: float) -> np.ndarray:
    """Smoothstep interpolation of a random lattice onto a W x H grid."""
    ys = np.arange(H, dtype=np.float64) / cell
    xs = np.arange(W, dtype=np.float64) / cell
    y0 = np.floor(ys).astype(np.int64)
    x0 = np.floor(xs).astype(np.int64)
    ty = _smoothstep(ys - y0)[:, None]
    tx = _smoothstep(xs - x0)[None, :]
    a = lat[y0][:, x0]
    b = lat[y0][:, x0 + 1]
    c = lat[y0 + 1][:, x0]
    d = lat[y0 + 1][:, x0 + 1]
    top = a + (b - a) * tx
    bot = c + (d - c) * tx
    return top + (bot - top) * ty


def value_noise(W: int, H: int, rng: np.random.Generator, octaves: int = 4,
                base_cell: float = 16.0, persistence: float = 0.5) -> np.ndarray:
    """Multi-octave value noise, min-max normalised to [0, 1] (float64 [H][W])."""
    out = np.zeros((H, W), dtype=np.float64)
    amp = 1.0
    cell = base_cell
    for _ in range(octaves):
        ny = int(math.ceil(H / cell)) + 2
        nx = int(math.ceil(W / cell)) + 2
        lat = rng.random((ny, nx))
        out += amp * _lattice_interp(lat, W, H, cell)
        amp *= persistence
        cell = max(cell / 2.0, 1.0)
    lo, hi = out.min(), out.max()
    return (out - lo) / max(hi - lo, 1e-12)


def bilinear(img: np.ndarray, x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """Sample img (float64 [H][W]) at real coordinates with border clamping."""
    H, W = img.shape
    x = np.clip(x, 0.0, W - 1.0)
    y = np.clip(y, 0.0, H - 1.0)
    x0 = np.minimum(np.floor(x).astype(np.int64), W - 2) if W > 1 else np.zeros_like(x, dtype=np.int64)
    y0 = np.minimum(np.floor(y).astype(np.int64), H - 2) if H > 1 else np.zeros_like(y, dtype=np.int64)
    x1 = np.minimum(x0 + 1, W - 1)
    y1 = np.minimum(y0 + 1, H - 1)
    fx = x - x0
    fy = y - y0
    a = img[y0, x0]
    b = img[y0, x1]
    c = img[y1, x0]
    d = img[y1, x1]
    return (a * (1 - fx) + b * fx) * (1 - fy) + (c * (1 - fx) + d * fx) * fy


@dataclass
class Pair:
    img1: np.ndarray      # float32 [H1][W1] in [0, 1]
    img2: np.ndarray      # float32 [H2][W2] in [0, 1]
    flow: np.ndarray      # float32 [H1][W1][2]: (dx, dy) taking a pixel of img1 into img2
    seed: int
    recipe: str


def _invert_backward_map(bx, by, W, H, iters=30):
    """Given I2(x') = I1(B(x')), find for each pixel x of I1 the x' with B(x') = x.

    bx, by: callables (x', y') -> source coordinates in I1.  Fixed-point
    iteration x' <- x' + (x - B(x')), which converges for the smooth,
    near-identity maps generated here.
    """
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    px, py = xs.copy(), ys.copy()
    for _ in range(iters):
        sx, sy = bx(px, py), by(px, py)
        px = px + (xs - sx)
        py = py + (ys - sy)
    return np.stack([px - xs, py - ys], axis=-1)


def _smooth_field(W, H, rng, max_disp, cell):
    fx = value_noise(W, H, rng, octaves=2, base_cell=cell) * 2.0 - 1.0
    fy = value_noise(W, H, rng, octaves=2, base_cell=cell) * 2.0 - 1.0
    mag = np.sqrt(fx * fx + fy * fy).max()
    s = max_disp / max(mag, 1e-12)
    return fx * s, fy * s


def make_pair_smooth(W: int, H: int, seed: int, max_disp: float = 6.0,
                     gain: float = 1.05, noise_sigma: float = 0.01, with_flow: bool = True) -> Pair:
    """Value-noise image warped by a seeded smooth displacement field.

    I1 = 4-octave value noise in [0,1].  I2(x') = gain * I1(x' - d(x')) + N(0, sigma^2),
    d a low-frequency field scaled to max |d| = max_disp, bilinear resampling.
    """
    rng = np.random.default_rng(seed)
    img1 = value_noise(W, H, rng, octaves=4, base_cell=16.0)
    dx, dy = _smooth_field(W, H, rng, max_disp, cell=max(W, H) / 2.0)

    def d_at(x, y):
        return bilinear(dx, x, y), bilinear(dy, x, y)

    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    src = d_at(xs, ys)
    img2 = gain * bilinear(img1, xs - src[0], ys - src[1])
    img2 = img2 + rng.normal(0.0, noise_sigma, size=img2.shape)
    img2 = np.clip(img2, 0.0, 1.0)
    if with_flow:
        flow = _invert_backward_map(lambda x, y: x - d_at(x, y)[0],
                                    lambda x, y: y - d_at(x, y)[1], W, H)
    else:
        flow = np.zeros((H, W, 2))
    return Pair(img1.astype(np.float32), img2.astype(np.float32), flow.astype(np.float32), seed,
                f"value-noise {W}x{H}, smooth warp max {max_disp}px, gain {gain}, noise {noise_sigma}")


def make_pair_motif(W: int, H: int, seed: int, max_disp: float = 40.0) -> Pair:
    """Noise image with 30% of its area tiled by a 16x16 motif, non-rigidly warped.

    Warp: x = c + R(-theta)(x' - c)/s - b(x'), with b a sum of 3 seeded Gaussian
    bumps scaled to max |b| = max_disp, s ~ U[0.9, 1.1], theta ~ U[-10, 10] deg.
    """
    rng = np.random.default_rng(seed)
    img1 = value_noise(W, H, rng, octaves=5, base_cell=32.0)
    motif = value_noise(16, 16, rng, octaves=3, base_cell=4.0)
    area = 0.3 * W * H
    rw = int(min(W, max(16, round(math.sqrt(area * W / H)))))
    rh = int(min(H, max(16, round(area / rw))))
    x0 = int(rng.integers(0, W - rw + 1))
    y0 = int(rng.integers(0, H - rh + 1))
    tiled = np.tile(motif, (rh // 16 + 1, rw // 16 + 1))[:rh, :rw]
    img1[y0:y0 + rh, x0:x0 + rw] = tiled

    cx, cy = (W - 1) / 2.0, (H - 1) / 2.0
    s = rng.uniform(0.9, 1.1)
    th = math.radians(rng.uniform(-10.0, 10.0))
    bumps = []
    for _ in range(3):
        bumps.append((rng.uniform(0, W), rng.uniform(0, H), rng.uniform(0.1, 0.25) * max(W, H),
                      rng.normal(size=2)))
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)

    def braw(x, y):
        bx = np.zeros_like(x)
        by = np.zeros_like(y)
        for (ux, uy, sg, v) in bumps:
            g = np.exp(-((x - ux) ** 2 + (y - uy) ** 2) / (2 * sg * sg))
            bx += v[0] * g
            by += v[1] * g
        return bx, by

    bx0, by0 = braw(xs, ys)
    scale = max_disp / max(np.sqrt(bx0 ** 2 + by0 ** 2).max(), 1e-12)
    ct, st = math.cos(-th), math.sin(-th)

    def src(x, y):
        bx, by = braw(x, y)
        ux = (ct * (x - cx) - st * (y - cy)) / s + cx - scale * bx
        uy = (st * (x - cx) + ct * (y - cy)) / s + cy - scale * by
        return ux, uy

    sx, sy = src(xs, ys)
    img2 = bilinear(img1, sx, sy)
    img2 = np.clip(img2 + rng.normal(0.0, 0.01, size=img2.shape), 0.0, 1.0)
    flow = _invert_backward_map(lambda x, y: src(x, y)[0], lambda x, y: src(x, y)[1], W, H)
    return Pair(img1.astype(np.float32), img2.astype(np.float32), flow.astype(np.float32), seed,
                f"noise {W}x{H} with 30% 16x16 motif, 3-bump warp max {max_disp}px, "
                f"similarity s={s:.3f} rot={math.degrees(th):.2f}deg")


def random_descriptor_field(W: int, H: int, seed: int) -> np.ndarray:
    """Random non-negative unit 9-vectors per pixel (float64 [H][W][9]).

    Used where a test needs pixel descriptors that are not produced by the
    descriptor step (translation and equivariance pins).
    """
    rng = np.random.default_rng(seed)
    v = rng.random((H, W, 9))
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def accuracy_at(matches: np.ndarray, flow: np.ndarray, T: float = 10.0) -> float:
    """Fraction of matches whose endpoint is within T px of the ground truth (Sec. 5.1).

    matches: [n][5] rows (x1, y1, x2, y2, score) with (x1, y1) a pixel of image 1.
    """
    if len(matches) == 0:
        return 0.0
    x1 = matches[:, 0].astype(np.int64)
    y1 = matches[:, 1].astype(np.int64)
    gt = flow[y1, x1]
    ex = matches[:, 2] - (matches[:, 0] + gt[:, 0])
    ey = matches[:, 3] - (matches[:, 1] + gt[:, 1])
    return float(np.mean(np.sqrt(ex * ex + ey * ey) <= T))
