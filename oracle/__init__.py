"""DeepMatching CPU oracle (test infrastructure only).

A plain CPU implementation of the method, written from the paper, that the
GPU path is checked against.  Only the tests, the smoke check and the bench's
CPU-baseline leg use it; the library never imports it.

Two builds of one C source (``dm_oracle.c``):
  * ``prec="f64"`` -- FP64, the paper's order of operations (Algorithm 1).
  * ``prec="f32"`` -- FP32 canonical mirror: a fixed operation order, own
    exp/log/pow, compensated (or plain) 4-child sums in child order, exact
    fixed-point path scores; the bit-exact target of the FP32
    GPU path.

Functions and the passages they follow:
  descriptors()   Sec. 3.2 "Pixel descriptor"; defaults of Sec. 5.2
  level0()        Eq. 3-4 (unpooled, unrectified bottom-level maps)
  level1_pooled() Eq. 3-12 for sampled lattice patches of level 1
  levels_sampled() Eq. 3-12 for sampled patches of any level below the top
  valid_flags()   Eq. 7 with the boundary rule: patch existence per level
  pyramid()       Algorithm 1 with Eq. 5-12 and the boundary rule of Sec. 3.2
  backtrack()     Eq. 13-15 (merge by highest score)
  reciprocal()    Eq. 16
  match()         the whole chain
  patch_vectors() the atomic patches of image 1 as 144-vectors (Eq. 3-4 window)
  kmeans_sphere() Sec. 4.1: k-means of the atomic patches with the centroids
                  projected back on the hypersphere after every update
  approx_match()  Sec. 4.1: the chain with every atomic patch replaced by its
                  closest prototype
  warp()          Algorithm 2: image downsized by sigma and rotated by -k pi/4
  invariant_match() Algorithm 2: the chain over 9 scales x 8 rotations, the
                  atomic correspondences mapped back and pooled, then Eq. 16
"""
from __future__ import annotations

import ctypes as C
import os
import platform
import subprocess
from dataclasses import dataclass, field

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "dm_oracle.c")
DF_SRC = os.path.join(HERE, "df_oracle.c")      # included by dm_oracle.c

DEFAULT_CFG = dict(nu1=1.0, nu2=1.0, nu3=1.0, slope=0.2, mu=0.3, image_scale=255.0, lam=1.4)


def _lib_path(prec: str) -> str:
    return os.path.join(HERE, f"liboracle_{prec}.so")


def build(force: bool = False) -> None:
    """Compile both oracle builds with gcc (no fp contraction; OpenMP)."""
    for prec, flag in (("f64", "0"), ("f32", "1")):
        out = _lib_path(prec)
        newest = max(os.path.getmtime(SRC), os.path.getmtime(DF_SRC))
        if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
            continue
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               f"-DORC_F32={flag}", SRC, "-o", out, "-lm"]
        if platform.machine() in ("x86_64", "AMD64"):
            cmd.insert(1, "-mfma")   # hardware fused multiply-add; same results as libm fmaf
        subprocess.check_call(cmd)


_LIBS: dict = {}


def _lib(prec: str):
    if prec not in _LIBS:
        build()
        lib = C.CDLL(_lib_path(prec))
        _LIBS[prec] = lib
    return _LIBS[prec]


def _dtype(prec: str):
    return np.float32 if prec == "f32" else np.float64


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


@dataclass
class Geometry:
    W1: int
    H1: int
    W2: int
    H2: int
    L: int
    P0x: int
    P0y: int
    Lx: int
    Ly: int
    dw: list
    dh: list

    def npatch(self, level: int) -> int:
        return self.P0x * self.P0y if level == 0 else self.Lx * self.Ly


def geometry(W1: int, H1: int, W2: int, H2: int) -> Geometry:
    out = np.zeros(5 + 2 * 34, dtype=np.int32)
    rc = _lib("f64").orc_geometry(W1, H1, W2, H2, _ptr(out))
    if rc != 0:
        raise ValueError(f"unsupported sizes {W1}x{H1} / {W2}x{H2}")
    L = int(out[0])
    dw = [int(v) for v in out[5:5 + L + 2]]
    dh = [int(v) for v in out[5 + L + 2:5 + 2 * (L + 2)]]
    return Geometry(W1, H1, W2, H2, L, int(out[1]), int(out[2]), int(out[3]), int(out[4]), dw, dh)


def descriptors(img: np.ndarray, prec: str = "f64", **cfg) -> np.ndarray:
    c = dict(DEFAULT_CFG, **cfg)
    img = np.ascontiguousarray(img, dtype=np.float32)
    H, W = img.shape
    out = np.zeros((H, W, 9), dtype=_dtype(prec))
    arr = np.array([c["nu1"], c["nu2"], c["nu3"], c["slope"], c["mu"], c["image_scale"]], dtype=np.float64)
    rc = _lib(prec).orc_descriptors(_ptr(img), W, H, _ptr(arr), _ptr(out))
    if rc != 0:
        raise ValueError("descriptor oracle failed")
    return out


def level0(d1: np.ndarray, d2: np.ndarray, prec: str = "f64", p0: int = 0, p1: int | None = None) -> np.ndarray:
    dt = _dtype(prec)
    d1 = np.ascontiguousarray(d1, dtype=dt)
    d2 = np.ascontiguousarray(d2, dtype=dt)
    H1, W1, _ = d1.shape
    H2, W2, _ = d2.shape
    g = geometry(W1, H1, W2, H2)
    if p1 is None:
        p1 = g.P0x * g.P0y
    out = np.zeros((p1 - p0, H2, W2), dtype=dt)
    rc = _lib(prec).orc_level0(_ptr(d1), W1, H1, _ptr(d2), W2, H2, p0, p1, _ptr(out))
    if rc != 0:
        raise ValueError("level0 oracle failed")
    return out


def level0_pooled(d1: np.ndarray, d2: np.ndarray, patches, prec: str = "f32", lam: float = DEFAULT_CFG["lam"]):
    """Level-0 pooled, rectified maps and argmax codes of the listed atomic patches."""
    dt = _dtype(prec)
    d1 = np.ascontiguousarray(d1, dtype=dt)
    d2 = np.ascontiguousarray(d2, dtype=dt)
    H1, W1, _ = d1.shape
    H2, W2, _ = d2.shape
    g = geometry(W1, H1, W2, H2)
    pl = np.ascontiguousarray(np.asarray(patches, dtype=np.int32))
    out = np.zeros((len(pl), g.dh[1], g.dw[1]), dtype=dt)
    am = np.zeros((len(pl), g.dh[1], g.dw[1]), dtype=np.uint8)
    lib = _lib(prec)
    lib.orc_level0_pooled.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                      C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]
    rc = lib.orc_level0_pooled(_ptr(d1), W1, H1, _ptr(d2), W2, H2, float(lam), _ptr(pl), len(pl), _ptr(out), _ptr(am))
    if rc != 0:
        raise ValueError("level0_pooled oracle failed")
    return out, am


def level1_pooled(d1: np.ndarray, d2: np.ndarray, patches, prec: str = "f32", lam: float = DEFAULT_CFG["lam"],
                  compensated: bool = True):
    """Level-1 pooled, rectified maps, argmax codes and existence of the listed
    lattice patches (for sampled checks of pairs too large for pyramid())."""
    dt = _dtype(prec)
    d1 = np.ascontiguousarray(d1, dtype=dt)
    d2 = np.ascontiguousarray(d2, dtype=dt)
    H1, W1, _ = d1.shape
    H2, W2, _ = d2.shape
    g = geometry(W1, H1, W2, H2)
    pl = np.ascontiguousarray(np.asarray(patches, dtype=np.int32))
    out = np.zeros((len(pl), g.dh[2], g.dw[2]), dtype=dt)
    am = np.zeros((len(pl), g.dh[2], g.dw[2]), dtype=np.uint8)
    ex = np.zeros(len(pl), dtype=np.uint8)
    lib = _lib(prec)
    lib.orc_level1_pooled.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int,
                                      C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    rc = lib.orc_level1_pooled(_ptr(d1), W1, H1, _ptr(d2), W2, H2, float(lam), int(bool(compensated)), _ptr(pl),
                               len(pl), _ptr(out), _ptr(am), _ptr(ex))
    if rc != 0:
        raise ValueError("level1_pooled oracle failed")
    return out, am, ex


def valid_flags(W1: int, H1: int, W2: int, H2: int) -> list:
    """Existence of every patch at every level l = 0..L (Eq. 7 with the
    boundary rule of Sec. 3.2): a list of uint8 arrays [npatch(l)]."""
    g = geometry(W1, H1, W2, H2)
    out = [np.zeros(g.npatch(l), dtype=np.uint8) for l in range(g.L + 1)]
    vv = (C.c_void_p * (g.L + 1))(*[a.ctypes.data for a in out])
    lib = _lib("f64")
    lib.orc_valid.argtypes = [C.c_int] * 4 + [C.c_void_p]
    if lib.orc_valid(W1, H1, W2, H2, vv) != 0:
        raise ValueError("valid oracle failed")
    return out


def levels_sampled(d1: np.ndarray, d2: np.ndarray, level: int, patches, prec: str = "f32",
                   lam: float = DEFAULT_CFG["lam"], compensated: bool = True):
    """Pooled, rectified maps, argmax codes and existence of the listed
    patches of one level l < L, computed from their atomic descendants only
    (the same arithmetic as pyramid(); for sampled checks of pairs too large
    for the whole pyramid).  Returns (maps [n][dh[l+1]][dw[l+1]], codes, exists)."""
    dt = _dtype(prec)
    d1 = np.ascontiguousarray(d1, dtype=dt)
    d2 = np.ascontiguousarray(d2, dtype=dt)
    H1, W1, _ = d1.shape
    H2, W2, _ = d2.shape
    g = geometry(W1, H1, W2, H2)
    pl = np.ascontiguousarray(np.asarray(patches, dtype=np.int32))
    out = np.zeros((len(pl), g.dh[level + 1], g.dw[level + 1]), dtype=dt)
    am = np.zeros(out.shape, dtype=np.uint8)
    ex = np.zeros(len(pl), dtype=np.uint8)
    lib = _lib(prec)
    lib.orc_levels_sampled.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                       C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    rc = lib.orc_levels_sampled(_ptr(d1), W1, H1, _ptr(d2), W2, H2, float(lam), int(bool(compensated)), int(level),
                                _ptr(pl), len(pl), _ptr(out), _ptr(am), _ptr(ex))
    if rc != 0:
        raise ValueError("levels_sampled oracle failed")
    return out, am, ex


@dataclass
class Pyramid:
    geom: Geometry
    prec: str
    pooled: list = field(default_factory=list)   # l = 0..L-1: [npatch(l)][dh[l+1]][dw[l+1]]
    argmax: list = field(default_factory=list)   # same shapes, uint8 codes (my+1)*3 + (mx+1)
    top: np.ndarray | None = None                # [npatch(L)][dh[L]][dw[L]]
    valid: list = field(default_factory=list)    # l = 0..L: [npatch(l)] uint8
    gap: list | None = None                      # optional, like pooled: relative top-two gap of each argmax
    cmaps: list | None = None                    # optional, l = 1..L: [npatch(l)][dh[l]][dw[l]] maps before pooling


def pyramid(d1: np.ndarray, d2: np.ndarray, prec: str = "f64", lam: float = DEFAULT_CFG["lam"],
            compensated: bool = True, gaps: bool = False, patches: np.ndarray | None = None,
            maps: bool = False) -> Pyramid:
    """Level maps of Algorithm 1.  `compensated` selects the FP32 mirror's
    child sum (TwoSum-compensated or plain, both in child order); FP64 ignores it.
    `gaps`: also the relative top-two gap of every pooling decision.
    `maps`: also each level's maps before pooling (pyr.cmaps[l], l = 1..L):
    FP64 the rectified C_l; FP32 the unrectified averages (C_l is their power).
    `patches`: [P0][144] vectors that replace image 1's atomic patches (the
    approximate form, Sec. 4.1); d1 then only gives the size of image 1."""
    dt = _dtype(prec)
    d1 = np.ascontiguousarray(d1, dtype=dt)
    d2 = np.ascontiguousarray(d2, dtype=dt)
    H1, W1, _ = d1.shape
    H2, W2, _ = d2.shape
    g = geometry(W1, H1, W2, H2)
    pyr = Pyramid(g, prec)
    for l in range(g.L):
        shape = (g.npatch(l), g.dh[l + 1], g.dw[l + 1])
        pyr.pooled.append(np.zeros(shape, dtype=dt))
        pyr.argmax.append(np.zeros(shape, dtype=np.uint8))
    pyr.top = np.zeros((g.npatch(g.L), g.dh[g.L], g.dw[g.L]), dtype=dt)
    pyr.valid = [np.zeros(g.npatch(l), dtype=np.uint8) for l in range(g.L + 1)]
    pp = (C.c_void_p * g.L)(*[a.ctypes.data for a in pyr.pooled])
    aa = (C.c_void_p * g.L)(*[a.ctypes.data for a in pyr.argmax])
    vv = (C.c_void_p * (g.L + 1))(*[a.ctypes.data for a in pyr.valid])
    gg = None
    if gaps:
        pyr.gap = [np.zeros(a.shape, dtype=np.float64) for a in pyr.pooled]
        gg = (C.c_void_p * g.L)(*[a.ctypes.data for a in pyr.gap])
    cc = None
    if maps:
        pyr.cmaps = [None] + [np.zeros((g.npatch(l), g.dh[l], g.dw[l]), dtype=dt) for l in range(1, g.L + 1)]
        cc = (C.c_void_p * (g.L + 1))(None, *[a.ctypes.data for a in pyr.cmaps[1:]])
    lib = _lib(prec)
    fn = lib.orc_pyramid if patches is None else lib.orc_pyramid_vec
    fn.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int,
                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    if patches is not None:
        src = np.ascontiguousarray(patches, dtype=dt)
        if src.shape != (g.npatch(0), 144):
            raise ValueError(f"patches must be [{g.npatch(0)}][144]")
    else:
        src = d1
    rc = fn(_ptr(src), W1, H1, _ptr(d2), W2, H2, float(lam), int(bool(compensated)), pp, aa, _ptr(pyr.top), vv, gg,
            cc)
    if rc != 0:
        raise ValueError("pyramid oracle failed")
    return pyr


@dataclass
class Backtrack:
    bestP_s: np.ndarray    # [P0] best score of each atomic patch (-inf: none)
    bestP_i: np.ndarray    # [P0] its pixel index ty*W2 + tx (-1: none)
    bestQ_s: np.ndarray    # [cells] best score per 4x4 cell of I'
    bestQ_i: np.ndarray    # [cells] its (patch*16 + offset in cell)
    leaf: np.ndarray | None  # [P0][H2][W2] merged atomic scores (optional)
    reached: np.ndarray    # [L+1] distinct tuples per level
    gap: np.ndarray | None = None   # [P0] smallest relative top-two gap of the decisions behind BestAt(p)
    leaf_raw: np.ndarray | None = None   # [P0][H2][W2] unrounded merged scores (FP32: fixed-point integers), -1 = none


def backtrack(pyr: Pyramid, dense_leaf: bool = False, leaf_raw: bool = False) -> Backtrack:
    g = pyr.geom
    dt = _dtype(pyr.prec)
    n0 = g.npatch(0)
    ncell = ((g.W2 + 3) // 4) * ((g.H2 + 3) // 4)
    bt = Backtrack(np.zeros(n0, dt), np.zeros(n0, np.int64), np.zeros(ncell, dt), np.zeros(ncell, np.int64),
                   np.zeros((n0, g.H2, g.W2), dt) if dense_leaf else None, np.zeros(g.L + 1, np.int64))
    pp = (C.c_void_p * g.L)(*[a.ctypes.data for a in pyr.pooled])
    aa = (C.c_void_p * g.L)(*[a.ctypes.data for a in pyr.argmax])
    vv = (C.c_void_p * (g.L + 1))(*[a.ctypes.data for a in pyr.valid])
    gg = None
    if pyr.gap is not None:
        bt.gap = np.zeros(n0, np.float64)
        gg = (C.c_void_p * g.L)(*[a.ctypes.data for a in pyr.gap])
    if leaf_raw:
        bt.leaf_raw = np.zeros((n0, g.H2, g.W2), np.float64)
    lib = _lib(pyr.prec)
    lib.orc_backtrack.argtypes = [C.c_int] * 4 + [C.c_void_p] * 13
    rc = lib.orc_backtrack(g.W1, g.H1, g.W2, g.H2, pp, aa, _ptr(pyr.top), vv,
                           _ptr(bt.bestP_s), _ptr(bt.bestP_i), _ptr(bt.bestQ_s), _ptr(bt.bestQ_i),
                           _ptr(bt.leaf) if dense_leaf else None, _ptr(bt.reached), gg,
                           _ptr(bt.gap) if bt.gap is not None else None,
                           _ptr(bt.leaf_raw) if leaf_raw else None)
    if rc != 0:
        raise ValueError("backtrack oracle failed")
    return bt


def reciprocal(pyr: Pyramid, bt: Backtrack) -> np.ndarray:
    """Rows (x1, y1, x2, y2, score), one per surviving atomic patch, in patch order."""
    g = pyr.geom
    out = np.zeros((g.npatch(0), 5), dtype=np.float64)
    lib = _lib(pyr.prec)
    lib.orc_reciprocal.argtypes = [C.c_int] * 4 + [C.c_void_p] * 5
    n = lib.orc_reciprocal(g.W1, g.H1, g.W2, g.H2, _ptr(bt.bestP_s), _ptr(bt.bestP_i),
                           _ptr(bt.bestQ_s), _ptr(bt.bestQ_i), _ptr(out))
    if n < 0:
        raise ValueError("reciprocal oracle failed")
    return out[:n]


def match(img1: np.ndarray, img2: np.ndarray, prec: str = "f64", compensated: bool = True, gaps: bool = False,
          **cfg):
    """Descriptors -> pyramid -> backtracking -> reciprocal matches (with the
    per-patch decision gaps in bt.gap when `gaps`)."""
    c = dict(DEFAULT_CFG, **cfg)
    lam = c.pop("lam")
    d1 = descriptors(img1, prec, **c)
    d2 = descriptors(img2, prec, **c)
    pyr = pyramid(d1, d2, prec, lam, compensated, gaps)
    bt = backtrack(pyr)
    return reciprocal(pyr, bt), pyr, bt


def patch_vectors(d1: np.ndarray) -> np.ndarray:
    """Image 1's atomic patches as vectors [P0][144] in d1's dtype: patch p
    (centre (4 (p % P0x) + 2, 4 (p // P0x) + 2), Eq. 3-4 window [x-2, x+1] x
    [y-2, y+1]) has a[(dy*4 + dx)*9 + c] = d1[y-2+dy][x-2+dx][c], zero for
    pixels outside image 1 (partial patches)."""
    H1, W1, _ = d1.shape
    P0x, P0y = (W1 + 1) // 4, (H1 + 1) // 4
    g = geometry(W1, H1, W1, H1)
    assert (g.P0x, g.P0y) == (P0x, P0y)
    pad = np.zeros((4 * P0y, 4 * P0x, 9), dtype=d1.dtype)
    h, w = min(H1, 4 * P0y), min(W1, 4 * P0x)
    pad[:h, :w] = d1[:h, :w]
    # [P0y][dy][P0x][dx][c] -> [P0y][P0x][dy][dx][c]
    a = pad.reshape(P0y, 4, P0x, 4, 9).transpose(0, 2, 1, 3, 4)
    return np.ascontiguousarray(a.reshape(P0y * P0x, 144))


def kmeans_sphere(A: np.ndarray, init: np.ndarray, iters: int, radius: float = 4.0):
    """Sec. 4.1 in FP64: Lloyd's k-means of the rows of A ([P0][144]) from the
    initial centroids `init` ([D][144]), each centroid rescaled to norm
    `radius` (the norm of a full atomic patch: 16 unit pixel descriptors)
    after every update.  One iteration = assignment to the closest centroid
    (the largest dot product, as all centroids have the same norm; ties to the
    lower index), then each centroid = the mean of its members projected on
    the sphere (a centroid without members keeps its value).  Returns the
    centroids and the assignment to them."""
    A = np.asarray(A, dtype=np.float64)

    def project(C):
        n = np.linalg.norm(C, axis=1, keepdims=True)
        return np.where(n > 0, C * (radius / np.where(n > 0, n, 1.0)), C)

    C = project(np.array(init, dtype=np.float64, copy=True))
    for _ in range(iters):
        assign = np.argmax(A @ C.T, axis=1)
        for d in range(C.shape[0]):
            members = A[assign == d]
            if len(members):
                C[d] = members.sum(axis=0)
        C = project(C)
    return C, np.argmax(A @ C.T, axis=1).astype(np.int32)


def approx_match(img1: np.ndarray, img2: np.ndarray, protos: np.ndarray, assign: np.ndarray, prec: str = "f64",
                 compensated: bool = True, **cfg):
    """Sec. 4.1: the chain with atomic patch p of image 1 replaced by the
    prototype protos[assign[p]] (given, e.g. from kmeans_sphere)."""
    c = dict(DEFAULT_CFG, **cfg)
    lam = c.pop("lam")
    d1 = descriptors(img1, prec, **c)
    d2 = descriptors(img2, prec, **c)
    q = np.asarray(protos, dtype=_dtype(prec))[np.asarray(assign)]
    pyr = pyramid(d1, d2, prec, lam, compensated, patches=q)
    bt = backtrack(pyr)
    return reciprocal(pyr, bt), pyr, bt


# --------------------------------------------------------------------------- #
# Scale and rotation invariant form (Algorithm 2)                              #
# --------------------------------------------------------------------------- #
# Scale factors 2^(|sigma|) for sigma = 0, 0.5, .., 2 and the rotation table
# cos / sin of k pi/4 (k = 0..7): definitions, rounded to the working precision.
INV_SCALES = (1.0, 1.4142135623730951, 2.0, 2.8284271247461903, 4.0)
_H = 0.70710678118654752440
ROT_C = (1.0, _H, 0.0, -_H, -1.0, -_H, 0.0, _H)
ROT_S = (0.0, _H, 1.0, _H, 0.0, -_H, -1.0, -_H)


def invariant_transforms():
    """Algorithm 2's loop order: sigma = -2, -1.5, .., 2 (outer), theta = k pi/4,
    k = 0..7 (inner); sigma1 = max(1, 2^sigma) downsizes image 1, sigma2 =
    max(1, 2^-sigma) image 2.  Entries (sigma1, sigma2, k)."""
    out = []
    for j in range(9):
        a = abs(j - 4)
        s1 = INV_SCALES[a] if j >= 4 else 1.0
        s2 = INV_SCALES[a] if j < 4 else 1.0
        for k in range(8):
            out.append((s1, s2, k))
    return out


def canvas_size(W: int, H: int, sigma: float, k: int):
    """Size of image W x H downsized by sigma and rotated by k pi/4 (the
    bounding box, so nothing is cropped), computed in double precision."""
    c, s = abs(ROT_C[k]), abs(ROT_S[k])
    Wr = max(1, int(np.floor((W * c + H * s) / sigma + 0.5)))
    Hr = max(1, int(np.floor((W * s + H * c) / sigma + 0.5)))
    return Wr, Hr


def _to_source(u, v, W, H, Wr, Hr, sigma, k, dt):
    """Canvas pixel (u, v) -> point of the original W x H image: the offset from
    the canvas centre rotated by +k pi/4 and scaled by sigma, about the image
    centre (fixed order of rounded operations in dtype dt)."""
    c, s, sg = dt(ROT_C[k]), dt(ROT_S[k]), dt(sigma)
    cu, cv = dt((Wr - 1) * 0.5), dt((Hr - 1) * 0.5)
    cx, cy = dt((W - 1) * 0.5), dt((H - 1) * 0.5)
    du = np.asarray(u, dtype=dt) - cu
    dv = np.asarray(v, dtype=dt) - cv
    rx = (c * du) - (s * dv)
    ry = (s * du) + (c * dv)
    return cx + sg * rx, cy + sg * ry


def warp(img: np.ndarray, sigma: float, k: int, prec: str = "f64") -> np.ndarray:
    """Algorithm 2's R_{-theta} * I_sigma: image downsized by sigma and rotated
    by -k pi/4 on the canvas of canvas_size(); bilinear interpolation (reading:
    the paper does not state the resampling; no prefilter -- the descriptor's
    own smoothing follows), zero outside the image."""
    dt = np.float32 if prec == "f32" else np.float64
    H, W = img.shape
    Wr, Hr = canvas_size(W, H, sigma, k)
    v, u = np.mgrid[0:Hr, 0:Wr]
    x, y = _to_source(u, v, W, H, Wr, Hr, sigma, k, dt)
    x0, y0 = np.floor(x), np.floor(y)
    fx, fy = x - x0, y - y0
    I = np.asarray(img, dtype=dt)
    xi, yi = x0.astype(np.int64), y0.astype(np.int64)

    def px(yy, xx):
        ok = (xx >= 0) & (yy >= 0) & (xx < W) & (yy < H)
        return np.where(ok, I[np.clip(yy, 0, H - 1), np.clip(xx, 0, W - 1)], dt(0))

    p00, p10, p01, p11 = px(yi, xi), px(yi, xi + 1), px(yi + 1, xi), px(yi + 1, xi + 1)
    top = p00 + fx * (p10 - p00)
    bot = p01 + fx * (p11 - p01)
    return (top + fy * (bot - top)).astype(dt)


def _round_px(x, n):
    """Nearest pixel index (floor(x + 1/2)) clamped to [0, n)."""
    return np.clip(np.floor(x + x.dtype.type(0.5)).astype(np.int64), 0, n - 1)


def _reciprocal_union(C1, T, S, W2: int, H2: int, P0x: int, prec: str) -> np.ndarray:
    """Eq. 16 over a set of atomic tuples (patch C1 of I, pixel T = y*W2 + x of
    I', raw score S; a tuple may appear several times): BestAt per patch of I
    (higher score, then lower T), BestAt' per 4x4 cell of I' (higher score,
    then lower C1*16 + offset in the cell); a patch's best tuple is kept iff it
    also wins its cell.  FP32: raw scores are fixed-point integers, rounded to
    FP32 once here.  Rows (x1, y1, x2, y2, score) in patch order."""
    C1 = np.asarray(C1, dtype=np.int64)
    T = np.asarray(T, dtype=np.int64)
    S = np.asarray(S, dtype=np.float64)
    CW2 = (W2 + 3) // 4
    tx, ty = T % W2, T // W2
    Q = C1 * 16 + (ty & 3) * 4 + (tx & 3)
    cell2 = (ty >> 2) * CW2 + (tx >> 2)
    o = np.lexsort((T, -S, C1))
    first = np.ones(len(o), bool)
    first[1:] = C1[o][1:] != C1[o][:-1]
    bestP = {int(C1[i]): (S[i], int(T[i])) for i in o[first]}
    o = np.lexsort((Q, -S, cell2))
    first = np.ones(len(o), bool)
    first[1:] = cell2[o][1:] != cell2[o][:-1]
    bestQ = {int(cell2[i]): (S[i], int(Q[i])) for i in o[first]}
    out = []
    for c1 in sorted(bestP):
        s, t = bestP[c1]
        tx_, ty_ = t % W2, t // W2
        q = bestQ.get((ty_ >> 2) * CW2 + (tx_ >> 2))
        if q is not None and q[0] == s and q[1] == c1 * 16 + (ty_ & 3) * 4 + (tx_ & 3):
            score = float(np.float32(s) * np.float32(1.0 / 268435456.0)) if prec == "f32" else float(s)
            out.append((4 * (c1 % P0x) + 2, 4 * (c1 // P0x) + 2, tx_, ty_, score))
    return np.array(out, dtype=np.float64).reshape(-1, 5)


def invariant_match(img1: np.ndarray, img2: np.ndarray, prec: str = "f64", transforms=None, **cfg):
    """Algorithm 2: DeepMatching of I downsized by sigma1 against I' downsized by
    sigma2 and rotated by -theta, for every transform; every atomic
    correspondence (the merged leaf tuples, Eq. 15) is mapped back to the input
    images (p -> sigma1 p, p' -> sigma2 R_theta p', here about the image
    centres, rounded to the nearest pixel) and pooled; Eq. 16 then keeps the
    tuples that are the best of their 4x4 cell of I (an atomic patch of I) and
    of I'.  Transforms whose images are too small for
    the pyramid are skipped.  Rows (x1, y1, x2, y2, score) in patch order."""
    c = dict(DEFAULT_CFG, **cfg)
    lam = c.pop("lam")
    dt = np.float32 if prec == "f32" else np.float64
    H1, W1 = img1.shape
    H2, W2 = img2.shape
    go = geometry(W1, H1, W2, H2)
    P0x, P0y = go.P0x, go.P0y
    cells1, tpix, scores = [], [], []
    for (s1, s2, k) in (transforms or invariant_transforms()):
        i1 = warp(img1, s1, 0, prec)
        i2 = warp(img2, s2, k, prec)
        h1, w1 = i1.shape
        h2, w2 = i2.shape
        if min(w1, h1) < 4 or max(w1, h1) < 5 or min(w2, h2) < 1:
            continue
        d1 = descriptors(i1, prec, **c)
        d2 = descriptors(i2, prec, **c)
        pyr = pyramid(d1, d2, prec, lam)
        bt = backtrack(pyr, leaf_raw=True)
        p, ty, tx = np.nonzero(bt.leaf_raw >= 0)
        if len(p) == 0:
            continue
        sc = bt.leaf_raw[p, ty, tx]
        g = pyr.geom
        # image 1: patch centre (rotation 0) -> original cell (atomic patch)
        x1, y1 = _to_source(4 * (p % g.P0x) + 2, 4 * (p // g.P0x) + 2, W1, H1, w1, h1, s1, 0, dt)
        X1, Y1 = _round_px(x1, W1), _round_px(y1, H1)
        C1 = np.minimum(Y1 >> 2, P0y - 1) * P0x + np.minimum(X1 >> 2, P0x - 1)
        # image 2: canvas pixel -> original pixel
        x2, y2 = _to_source(tx, ty, W2, H2, w2, h2, s2, k, dt)
        X2, Y2 = _round_px(x2, W2), _round_px(y2, H2)
        cells1.append(C1)
        tpix.append(Y2 * W2 + X2)
        scores.append(sc)
    if not cells1:
        return np.zeros((0, 5), dtype=np.float64)
    return _reciprocal_union(np.concatenate(cells1), np.concatenate(tpix), np.concatenate(scores), W2, H2, P0x, prec)


# --------------------------------------------------------------------------- #
# DM*: the earlier backtracking variant (Sec. 5.3, Table "oldvsnew")           #
# --------------------------------------------------------------------------- #
def local_maxima(m: np.ndarray) -> np.ndarray:
    """Mask of the local maxima of one correlation map (reading: the paper
    names them without a tie rule): q is one iff m[q] > 0 and, over its 8
    neighbours r inside the map, m[q] > m[r] for r before q in row-major order
    and m[q] >= m[r] for r after q -- so a plateau gives its first point and
    two maxima are never neighbours."""
    m = np.asarray(m)
    H, W = m.shape
    pad = np.full((H + 2, W + 2), -np.inf)
    pad[1:-1, 1:-1] = m
    mask = m > 0
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            if dy == 0 and dx == 0:
                continue
            nb = pad[1 + dy:H + 1 + dy, 1 + dx:W + 1 + dx]
            mask &= (m > nb) if (dy < 0 or (dy == 0 and dx < 0)) else (m >= nb)
    return mask


def pow_vec(x: np.ndarray, lam: float, prec: str) -> np.ndarray:
    """x^lam element by element in the working precision (Eq. 11)."""
    dt = _dtype(prec)
    x = np.ascontiguousarray(x, dtype=dt)
    out = np.empty_like(x)
    lib = _lib(prec)
    lib.orc_pow_vec.argtypes = [C.c_void_p, C.c_longlong, C.c_double, C.c_void_p]
    lib.orc_pow_vec(_ptr(x), x.size, float(lam), _ptr(out))
    return out


def _child(g: Geometry, l: int, ix: int, iy: int, i: int) -> int:
    """Child i of lattice patch (ix, iy) at level l (Eq. 5: offsets o_i =
    (-1,-1), (-1,+1), (+1,-1), (+1,+1) as (x, y), 2^l o_i pixels), as an index
    at level l-1, or -1 outside the grid."""
    ox = 1 if i >= 2 else -1
    oy = 1 if i & 1 else -1
    if l == 1:
        cx, cy = ix + (ox - 1) // 2, iy + (oy - 1) // 2
        return cy * g.P0x + cx if 0 <= cx < g.P0x and 0 <= cy < g.P0y else -1
    st = 1 << (l - 2)
    cx, cy = ix + ox * st, iy + oy * st
    return cy * g.Lx + cx if 0 <= cx < g.Lx and 0 <= cy < g.Ly else -1


def _ps_term(prec: str):
    """Score term of a map value: FP64 the value; FP32 the nearest multiple of
    2^-28 as a fixed-point integer (ties to even), as for the path scores."""
    if prec == "f32":
        return lambda v: int(np.rint(np.float32(v) * np.float32(268435456.0)))
    return float


def dmstar_entries(pyr: Pyramid, l: int, lam: float = DEFAULT_CFG["lam"]) -> dict:
    """Entry points of DM* at level l >= 1: the local maxima of the maps C_l of
    the existing patches, {(p, qy, qx): score term of C_l(p, q)} (needs
    pyramid(..., maps=True); FP32 detects on the unrectified averages, whose
    order is C_l's, and raises the value to lam for the score)."""
    g = pyr.geom
    term = _ps_term(pyr.prec)
    out = {}
    for p in range(g.npatch(l)):
        if not pyr.valid[l][p]:
            continue
        m = pyr.cmaps[l][p]
        ys, xs = np.nonzero(local_maxima(m))
        if len(ys) == 0:
            continue
        v = m[ys, xs]
        if pyr.prec == "f32":
            v = pow_vec(v, lam, "f32")
        for y, x, val in zip(ys.tolist(), xs.tolist(), v.tolist()):
            out[(p, y, x)] = term(val)
    return out


def dmstar_backtrack(pyr: Pyramid, lam: float = DEFAULT_CFG["lam"], entries: str = "maxima") -> dict:
    """DM*'s backtracking: tuples (l, p, q, s) start at the entry points of every
    level (entries="maxima") -- or, for comparison, at every position of the
    top level with the new form's entry set (entries="top") -- and carry their
    start score unchanged down the path (Eq. 13 children, merged by the highest
    start); an atomic tuple's score is its start plus the rectified atomic
    correlation at its end, P_0 at the last step (reading: "start and end
    point").  Returns {(c, ty, tx): raw score} of the atomic tuples."""
    g = pyr.geom
    L = g.L
    term = _ps_term(pyr.prec)
    if entries == "maxima":
        F = dmstar_entries(pyr, L, lam)
    else:
        F = {}
        for p in range(g.npatch(L)):
            if pyr.valid[L][p]:
                for (y, x), v in np.ndenumerate(pyr.top[p]):
                    F[(p, y, x)] = term(v)
    leaves = {}
    for l in range(L, 0, -1):
        nxt = dmstar_entries(pyr, l - 1, lam) if (l - 1 >= 1 and entries == "maxima") else {}
        P, A = pyr.pooled[l - 1], pyr.argmax[l - 1]
        mw, mh = g.dw[l], g.dh[l]
        for (p, qy, qx), s in F.items():
            ix, iy = p % g.Lx, p // g.Lx
            for i in range(4):
                c = _child(g, l, ix, iy, i)
                if c < 0 or not pyr.valid[l - 1][c]:
                    continue
                rx, ry = qx + (1 if i >= 2 else -1), qy + (1 if i & 1 else -1)
                if not (0 <= rx < mw and 0 <= ry < mh):
                    continue
                code = int(A[c, ry, rx])
                key = (c, 2 * ry + code // 3 - 1, 2 * rx + code % 3 - 1)
                v = s if l - 1 >= 1 else s + term(P[c, ry, rx])
                tgt = nxt if l - 1 >= 1 else leaves
                if key not in tgt or v > tgt[key]:
                    tgt[key] = v
        F = nxt
    return leaves


def dmstar_match(img1: np.ndarray, img2: np.ndarray, prec: str = "f64", entries: str = "maxima", **cfg) -> np.ndarray:
    """DM* (Sec. 5.3): entry points at the local maxima of every level >= 1,
    start + end scoring, then Eq. 16 as in the new form.  Rows (x1, y1, x2,
    y2, score) in patch order."""
    c = dict(DEFAULT_CFG, **cfg)
    lam = c.pop("lam")
    compensated = c.pop("compensated", True)
    d1 = descriptors(img1, prec, **c)
    d2 = descriptors(img2, prec, **c)
    pyr = pyramid(d1, d2, prec, lam, compensated=compensated, maps=True)
    leaves = dmstar_backtrack(pyr, lam, entries)
    g = pyr.geom
    if not leaves:
        return np.zeros((0, 5), dtype=np.float64)
    keys = np.array(list(leaves.keys()), dtype=np.int64)
    S = np.array(list(leaves.values()), dtype=np.float64)
    return _reciprocal_union(keys[:, 0], keys[:, 1] * g.W2 + keys[:, 2], S, g.W2, g.H2, g.P0x, prec)


# --------------------------------------------------------------------------- #
# DeepFlow (Sec. 4.3): variational refinement with the matches as a term      #
# --------------------------------------------------------------------------- #
DF_DEFAULT = dict(sigma=0.5, eta=0.95, gamma=0.8, delta=0.0, beta=300.0, b=0.6, kappa=5.0, zeta=0.1, eps=0.001,
                  sigma_m=50.0, omega=1.6, image_scale=255.0, n_fixed=5, n_sor=25, min_size=16)
_DF_KEYS = ("sigma", "eta", "gamma", "delta", "beta", "b", "kappa", "zeta", "eps", "sigma_m", "omega",
            "image_scale", "n_fixed", "n_sor", "min_size")


def df_params(**kw) -> np.ndarray:
    """The parameter vector of the DeepFlow oracle (defaults: the paper's
    values, Sec. 4.3 and Sec. 5.4, plus the readings' omega and min_size)."""
    bad = set(kw) - set(DF_DEFAULT)
    if bad:
        raise KeyError(f"unknown DeepFlow parameters {sorted(bad)}")
    c = dict(DF_DEFAULT, **kw)
    return np.array([float(c[k]) for k in _DF_KEYS], dtype=np.float64)


def df_levels(W: int, H: int, **kw):
    """Sizes of the coarse-to-fine pyramid, finest first."""
    ws = np.zeros(256, np.int32)
    hs = np.zeros(256, np.int32)
    lib = _lib("f64")
    lib.orc_df_levels.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]
    prm = df_params(**kw)
    n = lib.orc_df_levels(W, H, _ptr(prm), _ptr(ws), _ptr(hs), 256)
    return list(zip(ws[:n].tolist(), hs[:n].tolist()))


def df_resample(src: np.ndarray, Wd: int, Hd: int, s: float, down: bool, mul: float = 1.0, prec: str = "f64"):
    dt = _dtype(prec)
    src = np.ascontiguousarray(src, dtype=dt)
    dst = np.zeros((Hd, Wd), dtype=dt)
    lib = _lib(prec)
    lib.orc_df_resample.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int,
                                    C.c_double]
    lib.orc_df_resample(_ptr(src), src.shape[1], src.shape[0], _ptr(dst), Wd, Hd, float(s), int(bool(down)),
                        float(mul))
    return dst


def df_sor(A: np.ndarray, ps: np.ndarray, u: np.ndarray, v: np.ndarray, du: np.ndarray, dv: np.ndarray,
           omega: float, n_sor: int, prec: str = "f64"):
    """n_sor red-black SOR sweeps of one fixed-point step's linear system;
    A [h][w][5] = (A11, A12, A22, b1, b2), ps [h][w] smoothness weights.
    Returns (du, dv)."""
    dt = _dtype(prec)
    A, ps, u, v = (np.ascontiguousarray(a, dtype=dt) for a in (A, ps, u, v))
    du = np.array(du, dtype=dt)
    dv = np.array(dv, dtype=dt)
    h, w = ps.shape
    lib = _lib(prec)
    lib.orc_df_sor.argtypes = [C.c_void_p] * 6 + [C.c_int, C.c_int, C.c_double, C.c_int]
    lib.orc_df_sor(_ptr(A), _ptr(ps), _ptr(u), _ptr(v), _ptr(du), _ptr(dv), w, h, float(omega), int(n_sor))
    return du, dv


def df_phi(I1: np.ndarray, I2: np.ndarray, x1: int, y1: int, x2: int, y2: int, sigma_m: float = 50.0,
           prec: str = "f64") -> float:
    dt = _dtype(prec)
    I1 = np.ascontiguousarray(I1, dtype=dt)
    I2 = np.ascontiguousarray(I2, dtype=dt)
    lib = _lib(prec)
    lib.orc_df_phi.restype = C.c_double
    lib.orc_df_phi.argtypes = [C.c_void_p, C.c_void_p] + [C.c_int] * 8 + [C.c_double]
    return lib.orc_df_phi(_ptr(I1), _ptr(I2), I1.shape[1], I1.shape[0], I2.shape[1], I2.shape[0], x1, y1, x2, y2,
                          float(sigma_m))


def deepflow(img1: np.ndarray, img2: np.ndarray, matches: np.ndarray | None = None, prec: str = "f64", **kw):
    """DeepFlow (Sec. 4.3) of two images in [0, 1] (H x W) with DeepMatching
    matches rows (x1, y1, x2, y2, score) (may be empty).  Returns (u, v)."""
    dt = _dtype(prec)
    i1 = np.ascontiguousarray(img1, dtype=np.float32)
    i2 = np.ascontiguousarray(img2, dtype=np.float32)
    if i1.shape != i2.shape:
        raise ValueError("DeepFlow needs two images of the same size")
    H, W = i1.shape
    m = np.ascontiguousarray(np.zeros((0, 5)) if matches is None else matches, dtype=np.float32).reshape(-1, 5)
    u = np.zeros((H, W), dtype=dt)
    v = np.zeros((H, W), dtype=dt)
    prm = df_params(**kw)
    lib = _lib(prec)
    lib.orc_deepflow.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_void_p,
                                 C.c_void_p, C.c_void_p]
    rc = lib.orc_deepflow(_ptr(i1), _ptr(i2), W, H, _ptr(m), len(m), _ptr(prm), _ptr(u), _ptr(v))
    if rc != 0:
        raise ValueError("DeepFlow oracle failed")
    return u, v


def loss_grad(d1: np.ndarray, d2: np.ndarray, prec: str = "f64", lam: float = DEFAULT_CFG["lam"]):
    """Differentiable form: loss = sum over existing top patches of max_q C_L, and
    its gradients with respect to both descriptor fields (small inputs only)."""
    dt = _dtype(prec)
    d1 = np.ascontiguousarray(d1, dtype=dt)
    d2 = np.ascontiguousarray(d2, dtype=dt)
    H1, W1, _ = d1.shape
    H2, W2, _ = d2.shape
    g1 = np.zeros_like(d1)
    g2 = np.zeros_like(d2)
    loss = C.c_double()
    lib = _lib(prec)
    lib.orc_loss_grad.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_int, C.c_int, C.c_double,
                                  C.c_void_p, C.c_void_p, C.c_void_p]
    rc = lib.orc_loss_grad(_ptr(d1), W1, H1, _ptr(d2), W2, H2, float(lam), C.byref(loss), _ptr(g1), _ptr(g2))
    if rc != 0:
        raise ValueError("loss_grad oracle failed")
    return loss.value, g1, g2


def pow_r(x: float, lam: float, prec: str = "f32") -> float:
    lib = _lib(prec)
    lib.orc_pow_r.restype = C.c_double
    lib.orc_pow_r.argtypes = [C.c_double, C.c_double]
    return lib.orc_pow_r(float(x), float(lam))


def exp_r(z: float, prec: str = "f32") -> float:
    lib = _lib(prec)
    lib.orc_exp_r.restype = C.c_double
    lib.orc_exp_r.argtypes = [C.c_double]
    return lib.orc_exp_r(float(z))
