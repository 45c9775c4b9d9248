"""Pins of the oracle's scale and rotation invariant form (Algorithm 2).

* the transform list is Algorithm 2's: 9 scale steps x 8 rotations, one of
  the two images downsized by 2^|sigma|;
* the warp: the identity is exact, right-angle rotations are exact array
  rotations, and downsizing by 2 is the mean of each 2x2 block (a closed
  form of bilinear sampling at the block centres);
* the chain restricted to the identity transform is the exact chain;
* a pair whose second image is the first rotated by 90 degrees is matched
  consistently with that rotation, which the exact form alone does not do.
"""
import numpy as np
import pytest

import oracle
from paper_1506_07656_gb300 import synth


def test_transform_list_follows_algorithm_2():
    t = oracle.invariant_transforms()
    assert len(t) == 72
    sig = [-2 + 0.5 * j for j in range(9)]
    for j, s in enumerate(sig):
        for k in range(8):
            s1, s2, kk = t[j * 8 + k]
            assert kk == k
            assert s1 == pytest.approx(max(1.0, 2.0 ** s), rel=1e-15)
            assert s2 == pytest.approx(max(1.0, 2.0 ** -s), rel=1e-15)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_warp_identity_and_right_angles(prec):
    rng = np.random.default_rng(3)
    img = rng.random((13, 18))
    dt = np.float32 if prec == "f32" else np.float64
    np.testing.assert_array_equal(oracle.warp(img, 1.0, 0, prec), img.astype(dt))
    for k, quarter in ((2, 1), (4, 2), (6, 3)):
        np.testing.assert_array_equal(oracle.warp(img, 1.0, k, prec), np.rot90(img, quarter).astype(dt))


def test_warp_downsize_by_two_is_the_block_mean():
    rng = np.random.default_rng(4)
    img = rng.random((12, 16))
    w = oracle.warp(img, 2.0, 0, "f64")
    want = img.reshape(6, 2, 8, 2).mean(axis=(1, 3))
    np.testing.assert_allclose(w, want, rtol=0, atol=1e-15)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_identity_transform_alone_is_the_exact_chain(prec):
    pr = synth.make_pair_smooth(40, 32, seed=5, max_disp=3.0)
    exact, _, _ = oracle.match(pr.img1, pr.img2, prec)
    inv = oracle.invariant_match(pr.img1, pr.img2, prec, transforms=[(1.0, 1.0, 0)])
    np.testing.assert_array_equal(inv, exact)


def _consistent_with_quarter_turn(m, W1, tol=3.0):
    # np.rot90(A)[i, j] = A[j, W-1-i]: pixel (x1, y1) of A appears at (x2, y2) = (y1, W-1-x1)
    if len(m) == 0:
        return 0.0
    return float(np.mean((np.abs(m[:, 2] - m[:, 1]) <= tol) & (np.abs(m[:, 3] - (W1 - 1 - m[:, 0])) <= tol)))


def test_quarter_turn_is_recovered():
    W, H = 48, 40
    img1 = synth.make_pair_smooth(W, H, seed=9, max_disp=1.0).img1
    img2 = np.ascontiguousarray(np.rot90(img1, 1))
    exact, _, _ = oracle.match(img1, img2, "f32")
    inv = oracle.invariant_match(img1, img2, "f32")
    assert _consistent_with_quarter_turn(inv, W) >= 0.7
    assert _consistent_with_quarter_turn(exact, W) <= 0.3


def test_fp32_mirror_agrees_with_fp64():
    """The invariant chain in the FP32 mirror and in FP64 choose the same matches
    on most patches (FP32 rounds the warp coordinates, so a few rectified pixels
    may move by one)."""
    W, H = 40, 32
    img1 = synth.make_pair_smooth(W, H, seed=23, max_disp=1.0).img1
    img2 = np.ascontiguousarray(np.rot90(img1, 1))
    m64 = oracle.invariant_match(img1, img2, "f64")
    m32 = oracle.invariant_match(img1, img2, "f32")
    k64 = {(r[0], r[1]): tuple(r[2:4]) for r in m64}
    agree = np.mean([k64.get((r[0], r[1])) == tuple(r[2:4]) for r in m32])
    assert agree >= 0.85, agree
