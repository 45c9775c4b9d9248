"""Pins of the approximate form of the oracle (Sec. 4.1: atomic patches of
image 1 replaced by their closest prototype from a spherical k-means).

What fixes each part:
  * patch_vectors / the vector pyramid: the pyramid built from image 1's
    patches given as vectors equals, bit for bit, the one built from the
    descriptor field (a layout or order mistake in the vectors breaks it).
  * kmeans_sphere: planted, well-separated clusters on the sphere are
    recovered; every centroid has norm 4; the assignment is the brute-force
    closest centroid; a centroid is the projected mean of its members.
  * approx_match: with every patch its own prototype (D = P0, no iteration)
    the approximate chain is the exact one; level-1 patches whose children
    carry the same prototypes have the same maps (the sharing Sec. 4.1 notes).
"""
import numpy as np
import pytest

import oracle
from paper_1506_07656_gb300 import synth


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("size", [(48, 40), (47, 39)])
def test_vector_pyramid_equals_image_pyramid(prec, size):
    W, H = size
    pr = synth.make_pair_smooth(W, H, seed=31, max_disp=4.0)
    d1 = oracle.descriptors(pr.img1, prec)
    d2 = oracle.descriptors(pr.img2, prec)
    A = oracle.patch_vectors(d1)
    g = oracle.geometry(W, H, W, H)
    assert A.shape == (g.npatch(0), 144)
    ref = oracle.pyramid(d1, d2, prec)
    got = oracle.pyramid(d1, d2, prec, patches=A)
    for l in range(g.L):
        np.testing.assert_array_equal(got.pooled[l], ref.pooled[l])
        np.testing.assert_array_equal(got.argmax[l], ref.argmax[l])
    np.testing.assert_array_equal(got.top, ref.top)


def test_patch_vector_layout_by_hand():
    # one patch, element by element: a[(dy*4 + dx)*9 + c] = d1[y-2+dy][x-2+dx][c]
    rng = np.random.default_rng(5)
    d1 = rng.random((11, 9, 9))
    A = oracle.patch_vectors(d1)
    P0x = (9 + 1) // 4
    p = 1 * P0x + 1                      # centre (6, 6)
    for dy in range(4):
        for dx in range(4):
            for c in range(9):
                x, y = 6 - 2 + dx, 6 - 2 + dy
                want = d1[y, x, c] if x < 9 and y < 11 else 0.0
                assert A[p, (dy * 4 + dx) * 9 + c] == want
    # a partial patch: centre x = 6 of a 7-wide image, pixel column 7 is outside
    d1b = rng.random((8, 7, 9))
    Ab = oracle.patch_vectors(d1b)
    assert np.all(Ab[1].reshape(4, 4, 9)[:, 3, :] == 0.0)


def _planted(K=6, per=40, noise=0.02, seed=7):
    rng = np.random.default_rng(seed)
    centers = rng.standard_normal((K, 144))
    centers *= 4.0 / np.linalg.norm(centers, axis=1, keepdims=True)
    labels = np.repeat(np.arange(K), per)
    X = centers[labels] + noise * rng.standard_normal((K * per, 144))
    X *= 4.0 / np.linalg.norm(X, axis=1, keepdims=True)
    perm = rng.permutation(len(X))
    return centers, X[perm], labels[perm]


def test_kmeans_sphere_recovers_planted_clusters():
    centers, X, labels = _planted()
    # start from one member of each cluster, in cluster order
    init = np.stack([X[np.flatnonzero(labels == k)[0]] for k in range(len(centers))])
    C, assign = oracle.kmeans_sphere(X, init, iters=5)
    np.testing.assert_array_equal(assign, labels)
    # the centroid of a cluster is the projected mean of its members, close to the planted centre
    for k in range(len(centers)):
        assert np.linalg.norm(C[k] - centers[k]) < 0.05


def test_kmeans_sphere_invariants_brute_force():
    rng = np.random.default_rng(11)
    X = rng.random((60, 144))                          # non-negative, like descriptors
    X[:40] *= 4.0 / np.linalg.norm(X[:40], axis=1, keepdims=True)
    init = X[[3, 17, 29, 41, 55]]
    C, assign = oracle.kmeans_sphere(X, init, iters=3)
    np.testing.assert_allclose(np.linalg.norm(C, axis=1), 4.0, rtol=0, atol=1e-12)
    # assignment: the closest centroid by Euclidean distance, ties to the lower index
    for i in range(len(X)):
        d2 = [float(np.sum((X[i] - C[k]) ** 2)) for k in range(len(C))]
        assert assign[i] == int(np.argmin(d2))
    # one more update from these centroids reproduces the projected member means
    C2, _ = oracle.kmeans_sphere(X, C, iters=1)
    for k in range(len(C)):
        m = X[assign == k]
        if len(m):
            s = m.sum(axis=0)
            np.testing.assert_allclose(C2[k], 4.0 * s / np.linalg.norm(s), rtol=0, atol=1e-12)


def test_approx_with_each_patch_its_own_prototype_is_exact():
    W, H = 48, 40                                      # whole atomic patches only: every vector has norm 4
    pr = synth.make_pair_smooth(W, H, seed=41, max_disp=4.0)
    d1 = oracle.descriptors(pr.img1, "f64")
    A = oracle.patch_vectors(d1)
    np.testing.assert_allclose(np.linalg.norm(A, axis=1), 4.0, rtol=0, atol=1e-12)
    protos, assign = oracle.kmeans_sphere(A, A, iters=0)
    np.testing.assert_array_equal(assign, np.arange(len(A)))
    m_approx, p_approx, _ = oracle.approx_match(pr.img1, pr.img2, protos, assign, "f64")
    m_exact, p_exact, _ = oracle.match(pr.img1, pr.img2, "f64")
    for a, b in zip(p_approx.pooled, p_exact.pooled):
        np.testing.assert_allclose(a, b, rtol=0, atol=1e-12)
    np.testing.assert_array_equal(m_approx[:, :4], m_exact[:, :4])
    np.testing.assert_allclose(m_approx[:, 4], m_exact[:, 4], rtol=0, atol=1e-12)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_same_child_prototypes_give_the_same_level1_map(prec):
    W, H = 48, 40
    pr = synth.make_pair_smooth(W, H, seed=43, max_disp=4.0)
    d1 = oracle.descriptors(pr.img1, prec)
    d2 = oracle.descriptors(pr.img2, prec)
    A = oracle.patch_vectors(d1).astype(np.float64)
    protos, assign = oracle.kmeans_sphere(A, A[[0, 50]], iters=2)   # D = 2: repeated child tuples
    g = oracle.geometry(W, H, W, H)
    pyr = oracle.pyramid(d1, d2, prec, patches=protos.astype(d1.dtype)[assign])
    # level-1 lattice patch (ix, iy) has atomic children (ix-1 | ix, iy-1 | iy)
    seen = {}
    pairs = 0
    for iy in range(1, g.P0y):
        for ix in range(1, g.P0x):
            kids = tuple(int(assign[cy * g.P0x + cx]) for cx in (ix - 1, ix) for cy in (iy - 1, iy))
            p = iy * g.Lx + ix
            if kids in seen:
                np.testing.assert_array_equal(pyr.pooled[1][p], pyr.pooled[1][seen[kids]])
                pairs += 1
            else:
                seen[kids] = p
    assert pairs > 0
