"""Pins of the DeepFlow oracle (Sec. 4.3).

* identical images and no matches: the flow is exactly zero (every data
  residual vanishes);
* an analytic texture translated by (1.5, -0.7) px: the flow recovers the
  translation inside the image;
* the matching term alone (no data term, beta at every level): the flow
  converges to a constant match field;
* SOR: many red-black sweeps solve the fixed-point step's linear system, the
  same solution as a direct sparse solve of the system assembled from the
  energy's normal equations;
* phi: zero on a linear ramp (rank-one structure tensor); on a texture with an
  exact integer shift (Delta = 0) it is sqrt(10 lambda_min) / (sigma_M
  sqrt(2 pi)) with lambda_min from a library eigen-solver;
* pyramid sizes follow floor(eta W + 1/2) down to the minimum side, and the
  bilinear resampling reproduces affine functions inside the image.
"""
import numpy as np
import pytest

import oracle

scipy_sparse = pytest.importorskip("scipy.sparse")
from scipy.sparse.linalg import spsolve  # noqa: E402


def _tex(x, y):
    return 0.5 + 0.2 * np.sin(0.31 * x + 0.17 * y) + 0.15 * np.cos(0.23 * y - 0.11 * x) + 0.1 * np.sin(0.05 * x * y / 8)


def _grid(W, H):
    y, x = np.mgrid[0:H, 0:W].astype(np.float64)
    return x, y


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_identical_images_give_zero_flow(prec):
    x, y = _grid(64, 48)
    I = _tex(x, y)
    u, v = oracle.deepflow(I, I, None, prec)
    assert np.all(u == 0) and np.all(v == 0)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_translation_is_recovered(prec):
    x, y = _grid(64, 48)
    t = (1.5, -0.7)
    u, v = oracle.deepflow(_tex(x, y), _tex(x - t[0], y - t[1]), None, prec)
    iu, iv = u[10:-10, 10:-10], v[10:-10, 10:-10]
    assert abs(iu.mean() - t[0]) < 0.01 and abs(iv.mean() - t[1]) < 0.01
    assert np.abs(iu - t[0]).max() < 0.1 and np.abs(iv - t[1]).max() < 0.1


def test_matching_term_alone_follows_the_matches():
    W, H = 48, 40
    x, y = _grid(W, H)
    t = (2, -1)
    I1 = _tex(x, y)
    I2 = _tex(x - t[0], y - t[1])
    m = [(xx, yy, xx + t[0], yy + t[1], 1.0) for yy in range(H) for xx in range(W)
         if 0 <= xx + t[0] < W and 0 <= yy + t[1] < H]
    u, v = oracle.deepflow(I1, I2, np.array(m), "f64", gamma=0.0, delta=0.0, b=0.0, n_fixed=10, n_sor=50)
    assert np.median(np.abs(u - t[0])) < 1e-3 and np.median(np.abs(v - t[1])) < 1e-3


def _assemble(A, ps, u, v):
    h, w = ps.shape
    n = w * h
    rows, cols, vals = [], [], []
    rhs = np.zeros(2 * n)
    for yy in range(h):
        for xx in range(w):
            o = yy * w + xx
            a = A[yy, xx]
            diag = 0.0
            ru, rv = a[3], a[4]
            for (px, py) in ((xx - 1, yy), (xx + 1, yy), (xx, yy - 1), (xx, yy + 1)):
                if 0 <= px < w and 0 <= py < h:
                    p = py * w + px
                    we = 0.5 * (ps[yy, xx] + ps[py, px])
                    diag += we
                    rows += [o, n + o]
                    cols += [p, n + p]
                    vals += [-we, -we]
                    ru += we * (u[py, px] - u[yy, xx])
                    rv += we * (v[py, px] - v[yy, xx])
            rows += [o, o, n + o, n + o]
            cols += [o, n + o, o, n + o]
            vals += [a[0] + diag, a[1], a[1], a[2] + diag]
            rhs[o], rhs[n + o] = ru, rv
    K = scipy_sparse.csr_matrix((vals, (rows, cols)), shape=(2 * n, 2 * n))
    return K, rhs


def test_sor_solves_the_linear_system():
    rng = np.random.default_rng(5)
    h, w = 7, 9
    A = np.zeros((h, w, 5))
    A[..., 0] = rng.uniform(1, 2, (h, w))
    A[..., 2] = rng.uniform(1, 2, (h, w))
    A[..., 1] = rng.uniform(-0.5, 0.5, (h, w))
    A[..., 3:] = rng.uniform(-1, 1, (h, w, 2))
    ps = rng.uniform(0.2, 1.0, (h, w))
    u, v = rng.normal(size=(h, w)), rng.normal(size=(h, w))
    du, dv = oracle.df_sor(A, ps, u, v, np.zeros((h, w)), np.zeros((h, w)), 1.6, 2000)
    K, rhs = _assemble(A, ps, u, v)
    sol = spsolve(K.tocsc(), rhs)
    np.testing.assert_allclose(du.ravel(), sol[:h * w], rtol=0, atol=1e-10)
    np.testing.assert_allclose(dv.ravel(), sol[h * w:], rtol=0, atol=1e-10)


def _cgrad(I):
    gx = 0.5 * (np.concatenate([I[:, 1:], I[:, -1:]], 1) - np.concatenate([I[:, :1], I[:, :-1]], 1))
    gy = 0.5 * (np.concatenate([I[1:], I[-1:]], 0) - np.concatenate([I[:1], I[:-1]], 0))
    return gx, gy


def test_phi_closed_forms():
    x, y = _grid(40, 30)
    ramp = 3.0 * x + 2.0 * y
    assert oracle.df_phi(ramp, ramp, 20, 15, 20, 15) < 1e-5
    I1 = 255.0 * _tex(x, y)
    I2 = np.zeros_like(I1)
    I2[:, 3:] = I1[:, :-3]                              # I2(x + 3) = I1(x): an exact integer shift
    gx, gy = _cgrad(I1)
    x1, y1 = 17, 12
    M = np.zeros((2, 2))
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            g = np.array([gx[y1 + dy, x1 + dx], gy[y1 + dy, x1 + dx]])
            M += np.outer(g, g)
    lmin = np.linalg.eigvalsh(M)[0]
    want = np.sqrt(10.0 * lmin) / (50.0 * np.sqrt(2.0 * np.pi))
    got = oracle.df_phi(I1, I2, x1, y1, x1 + 3, y1)
    assert got == pytest.approx(want, rel=1e-9)


def test_pyramid_sizes_and_affine_resampling():
    lv = oracle.df_levels(100, 60)
    assert lv[0] == (100, 60)
    for (w0, h0), (w1, h1) in zip(lv, lv[1:]):
        assert (w1, h1) == (int(np.floor(0.95 * w0 + 0.5)), int(np.floor(0.95 * h0 + 0.5)))
        assert min(w1, h1) >= 16
    wl, hl = lv[-1]
    assert min(int(np.floor(0.95 * wl + 0.5)), int(np.floor(0.95 * hl + 0.5))) < 16
    x, y = _grid(50, 40)
    f = 0.3 * x - 0.7 * y + 2.0
    Wd, Hd = 48, 38
    d = oracle.df_resample(f, Wd, Hd, 0.95, True)
    xd, yd = _grid(Wd, Hd)
    xs, ys = (xd + 0.5) / 0.95 - 0.5, (yd + 0.5) / 0.95 - 0.5
    inside = (xs <= 49) & (ys <= 39)
    np.testing.assert_allclose(d[inside], (0.3 * xs - 0.7 * ys + 2.0)[inside], rtol=0, atol=1e-12)
    up = oracle.df_resample(d, 50, 40, 0.95, False, 2.0)
    xs, ys = (x + 0.5) * 0.95 - 0.5, (y + 0.5) * 0.95 - 0.5
    inside = (xs >= 0) & (ys >= 0) & (xs <= Wd - 1) & (ys <= Hd - 1)
    want = 2.0 * (0.3 * ((xs + 0.5) / 0.95 - 0.5) - 0.7 * ((ys + 0.5) / 0.95 - 0.5) + 2.0)
    # d is affine where its own samples were not clamped: columns <= 46, rows <= 36
    inner = inside & (xs <= 45) & (ys <= 35)
    np.testing.assert_allclose(up[inner], want[inner], rtol=0, atol=1e-9)


def test_fp32_mirror_close_to_fp64():
    """The FP32 mirror follows the FP64 definition closely on a translated texture
    (the two differ only by rounding)."""
    x, y = _grid(48, 40)
    I1, I2 = _tex(x, y), _tex(x - 0.8, y + 0.4)
    u64, v64 = oracle.deepflow(I1, I2, None, "f64")
    u32, v32 = oracle.deepflow(I1, I2, None, "f32")
    assert np.abs(u64 - u32).max() < 1e-3 and np.abs(v64 - v32).max() < 1e-3
