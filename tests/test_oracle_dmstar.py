"""Pins of the oracle's DM* variant (Sec. 5.3: local-maxima entry points at
every level, start + end scoring).

* local_maxima: a constant map has exactly its first point; a strictly
  increasing ramp has only its last point; separated planted bumps give
  exactly their centres; maxima are never neighbours and the global maximum
  is one of them; non-positive maps have none.
* the level maps kept by the pyramid are the maps it pools: pooling them
  (3x3, stride 2, first maximum) and rectifying gives the stored pooled maps
  and argmax codes, and C_L equals the stored top level.
* the traversal: started at every top position, the atomic tuples reached are
  exactly those of the new form's backtracking (its leaf set).
* the merge: for every atomic tuple, the merged score equals the best over an
  explicit enumeration of every path from every entry point (no merging).
* the end term: an atomic tuple's score minus its start is the rectified
  level-0 correlation at its pixel, taken from the unpooled level-0 maps.
"""
import numpy as np
import pytest

import oracle
from paper_1506_07656_gb300 import synth


def test_local_maxima_closed_cases():
    m = np.full((5, 7), 0.25)
    mask = oracle.local_maxima(m)
    assert mask.sum() == 1 and mask[0, 0]
    ramp = np.arange(1, 36, dtype=np.float64).reshape(5, 7)
    mask = oracle.local_maxima(ramp)
    assert mask.sum() == 1 and mask[4, 6]
    assert oracle.local_maxima(np.zeros((4, 4))).sum() == 0
    assert oracle.local_maxima(-np.ones((4, 4))).sum() == 0


def test_local_maxima_planted_bumps():
    H, W = 40, 50
    y, x = np.mgrid[0:H, 0:W]
    centres = [(5, 7), (20, 30), (33, 12), (8, 44)]
    m = sum(np.exp(-((y - cy) ** 2 + (x - cx) ** 2) / 8.0) * (1.0 + 0.1 * k) for k, (cy, cx) in enumerate(centres))
    ys, xs = np.nonzero(oracle.local_maxima(m))
    assert sorted(zip(ys.tolist(), xs.tolist())) == sorted(centres)


def test_local_maxima_invariants_random():
    rng = np.random.default_rng(3)
    for _ in range(20):
        m = rng.random((9, 11))
        m[rng.random(m.shape) < 0.2] = 0.5          # plateaus of equal values
        mask = oracle.local_maxima(m)
        ys, xs = np.nonzero(mask)
        pts = set(zip(ys.tolist(), xs.tolist()))
        assert np.unravel_index(np.argmax(m), m.shape) in pts
        for (a, b) in pts:
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if (dy or dx) and (a + dy, b + dx) in pts:
                        raise AssertionError("neighbouring maxima")


def _pool_rectify(A, mw, mh, lam, prec):
    """3x3 max over the window centred at 2r (in-map points only), first maximum
    in scan order, then rectification (FP32 pools the raw average)."""
    H, W = A.shape
    val = np.zeros((mh, mw))
    code = np.zeros((mh, mw), np.uint8)
    for ry in range(mh):
        for rx in range(mw):
            best, bc = -np.inf, 0
            for k, (my, mx) in enumerate((a, b) for a in (-1, 0, 1) for b in (-1, 0, 1)):
                y, x = 2 * ry + my, 2 * rx + mx
                if 0 <= y < H and 0 <= x < W and A[y, x] > best:
                    best, bc = A[y, x], k
            val[ry, rx], code[ry, rx] = best, bc
    if prec == "f32":
        val = oracle.pow_vec(val.astype(np.float32), lam, "f32")
    return val, code


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_level_maps_pool_to_the_stored_pyramid(prec):
    pr = synth.make_pair_smooth(37, 29, seed=2, max_disp=3.0)
    d1, d2 = oracle.descriptors(pr.img1, prec), oracle.descriptors(pr.img2, prec)
    pyr = oracle.pyramid(d1, d2, prec, maps=True)
    g = pyr.geom
    lam = oracle.DEFAULT_CFG["lam"]
    for l in range(1, g.L):
        for p in np.flatnonzero(pyr.valid[l])[:6]:
            v, c = _pool_rectify(pyr.cmaps[l][p], g.dw[l + 1], g.dh[l + 1], lam, prec)
            np.testing.assert_array_equal(c, pyr.argmax[l][p])
            np.testing.assert_array_equal(v.astype(pyr.pooled[l].dtype), pyr.pooled[l][p])
    top = pyr.cmaps[g.L] if prec == "f64" else oracle.pow_vec(pyr.cmaps[g.L], lam, "f32")
    ok = pyr.valid[g.L].astype(bool)
    np.testing.assert_array_equal(top[ok], pyr.top[ok])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_all_top_entries_reach_the_new_forms_leaves(prec):
    pr = synth.make_pair_smooth(40, 32, seed=7, max_disp=3.0)
    d1, d2 = oracle.descriptors(pr.img1, prec), oracle.descriptors(pr.img2, prec)
    pyr = oracle.pyramid(d1, d2, prec, maps=True)
    leaves = oracle.dmstar_backtrack(pyr, entries="top")
    bt = oracle.backtrack(pyr, leaf_raw=True)
    want = set(map(tuple, np.argwhere(bt.leaf_raw >= 0).tolist()))
    assert set(leaves) == want


def _enumerate(pyr, lam):
    """Every path from every entry point, no merging: best start + end per tuple."""
    g = pyr.geom
    term = oracle._ps_term(pyr.prec)
    best = {}

    def down(l, p, qy, qx, s):
        ix, iy = p % g.Lx, p // g.Lx
        for i in range(4):
            c = oracle._child(g, l, ix, iy, i)
            if c < 0 or not pyr.valid[l - 1][c]:
                continue
            rx, ry = qx + (1 if i >= 2 else -1), qy + (1 if i & 1 else -1)
            if not (0 <= rx < g.dw[l] and 0 <= ry < g.dh[l]):
                continue
            code = int(pyr.argmax[l - 1][c, ry, rx])
            ty, tx = 2 * ry + code // 3 - 1, 2 * rx + code % 3 - 1
            if l - 1 >= 1:
                down(l - 1, c, ty, tx, s)
            else:
                v = s + term(pyr.pooled[0][c, ry, rx])
                if (c, ty, tx) not in best or v > best[(c, ty, tx)]:
                    best[(c, ty, tx)] = v

    for l in range(1, g.L + 1):
        for (p, qy, qx), s in oracle.dmstar_entries(pyr, l, lam).items():
            down(l, p, qy, qx, s)
    return best


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_merge_equals_path_enumeration(prec):
    pr = synth.make_pair_smooth(40, 32, seed=11, max_disp=3.0)
    d1, d2 = oracle.descriptors(pr.img1, prec), oracle.descriptors(pr.img2, prec)
    pyr = oracle.pyramid(d1, d2, prec, maps=True)
    lam = oracle.DEFAULT_CFG["lam"]
    assert oracle.dmstar_backtrack(pyr, lam) == _enumerate(pyr, lam)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_end_term_is_the_rectified_atomic_correlation(prec):
    pr = synth.make_pair_smooth(40, 32, seed=13, max_disp=3.0)
    d1, d2 = oracle.descriptors(pr.img1, prec), oracle.descriptors(pr.img2, prec)
    pyr = oracle.pyramid(d1, d2, prec, maps=True)
    lam = oracle.DEFAULT_CFG["lam"]
    g = pyr.geom
    leaves = oracle.dmstar_backtrack(pyr, lam)
    starts = set()
    for l in range(1, g.L + 1):
        starts |= set(oracle.dmstar_entries(pyr, l, lam).values())
    C0 = oracle.level0(d1, d2, prec)                  # unpooled atomic correlations [P0][H2][W2]
    term = oracle._ps_term(prec)
    keys = list(leaves)[:400]
    ends = oracle.pow_vec(np.array([C0[c, ty, tx] for c, ty, tx in keys]), lam, prec)
    if prec == "f32":                                 # fixed-point integers: exact
        for (c, ty, tx), e in zip(keys, ends):
            assert leaves[(c, ty, tx)] - term(e) in starts
    else:                                             # FP64 sums: one rounding
        st = np.array(sorted(starts))
        for (c, ty, tx), e in zip(keys, ends):
            assert np.min(np.abs(st - (leaves[(c, ty, tx)] - e))) <= 1e-12


def test_fp32_mirror_agrees_with_fp64():
    """DM* in the FP32 mirror and in FP64 choose the same matches on most patches
    (they differ only where rounding flips a decision) with close scores."""
    pr = synth.make_pair_smooth(48, 40, seed=17, max_disp=3.0)
    m64 = oracle.dmstar_match(pr.img1, pr.img2, "f64")
    m32 = oracle.dmstar_match(pr.img1, pr.img2, "f32")
    k64 = {(r[0], r[1]): r for r in m64}
    same = [r for r in m32 if (r[0], r[1]) in k64 and tuple(k64[(r[0], r[1])][2:4]) == tuple(r[2:4])]
    assert len(same) >= 0.9 * len(m64)
    for r in same:
        assert abs(r[4] - k64[(r[0], r[1])][4]) < 1e-5
