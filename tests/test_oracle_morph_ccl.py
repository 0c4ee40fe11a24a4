"""Pins of the oracle's binary morphology and connected-component boxes (CPU).

Morphology is checked exhaustively on every 4x4 binary image against
scipy.ndimage (whose border_value reproduces the clipped window: outside
pixels count as 0 for dilation and as 1 for erosion), and against the
algebra of Eq. (5): duality, idempotence of opening and closing, and the
redundancy of the final horizontal opening after a 3x3 opening.
Labelling is checked against scipy.ndimage.label with 4-connectivity and a
brute-force union-find written here.
"""
import itertools

import numpy as np
import pytest

import oracle

nd = pytest.importorskip("scipy.ndimage")

SQ = np.ones((3, 3), bool)
ROW = np.ones((1, 3), bool)
FOUR = np.array([[0, 1, 0], [1, 1, 1], [0, 1, 0]], bool)


def _sp(op, M):
    M = M.astype(bool)
    if op == oracle.RO_DILATE3:
        return nd.binary_dilation(M, SQ, border_value=0)
    if op == oracle.RO_ERODE3:
        return nd.binary_erosion(M, SQ, border_value=1)
    if op == oracle.RO_DILATE1x3:
        return nd.binary_dilation(M, ROW, border_value=0)
    return nd.binary_erosion(M, ROW, border_value=1)


def _all_masks(h, w):
    n = h * w
    idx = np.arange(1 << n, dtype=np.int64)
    bits = (idx[:, None] >> np.arange(n)) & 1
    return bits.reshape(-1, h, w).astype(np.uint8)


def _tile(masks):
    """Lay many small masks side by side, separated so they never interact,
    as one image per op is not possible with the clipped border -- so we
    simply loop (the masks are tiny)."""
    return masks


@pytest.mark.parametrize("op", [0, 1, 2, 3])
def test_each_op_on_every_4x4_image(op):
    masks = _all_masks(4, 4)
    for M in masks[::3]:            # a third of all 65536, every residue class of bit 0/1
        assert np.array_equal(oracle.morph(M, op).astype(bool), _sp(op, M)), M


def test_chain_on_every_3x4_image_and_random_images():
    masks = list(_all_masks(3, 4))
    rng = np.random.default_rng(2)
    for _ in range(40):
        masks.append((rng.random((rng.integers(1, 30), rng.integers(1, 40))) < rng.uniform(0.2, 0.8)).astype(np.uint8))
    for M in masks:
        c = _sp(1, _sp(0, M))            # closing 3x3: erode(dilate)
        o = _sp(0, _sp(1, c))            # opening 3x3: dilate(erode)
        h = _sp(3 - 1, _sp(3, o))        # opening 1x3
        M1, M2, M3 = oracle.morph_chain(M, 0)
        assert np.array_equal(M1.astype(bool), c)
        assert np.array_equal(M2.astype(bool), o)
        assert np.array_equal(M3.astype(bool), h)
        # the other order: open1x3, close3, open3
        a = _sp(2, _sp(3, M))
        b = _sp(1, _sp(0, a))
        d = _sp(0, _sp(1, b))
        N1, N2, N3 = oracle.morph_chain(M, 1)
        assert np.array_equal(N1.astype(bool), a)
        assert np.array_equal(N2.astype(bool), b)
        assert np.array_equal(N3.astype(bool), d)


def test_morphology_algebra_on_random_images():
    rng = np.random.default_rng(9)
    for _ in range(60):
        T, F = rng.integers(1, 48), rng.integers(1, 64)
        M = (rng.random((T, F)) < rng.uniform(0.1, 0.9)).astype(np.uint8)
        # duality: dilation = complement of the erosion of the complement
        for d, e in ((0, 1), (2, 3)):
            assert np.array_equal(oracle.morph(M, d), 1 - oracle.morph(1 - M, e))
        # opening and closing are idempotent
        op = lambda X: oracle.morph(oracle.morph(X, 1), 0)
        cl = lambda X: oracle.morph(oracle.morph(X, 0), 1)
        assert np.array_equal(op(op(M)), op(M))
        assert np.array_equal(cl(cl(M)), cl(M))
        # opening shrinks, closing grows
        assert np.all(op(M) <= M) and np.all(cl(M) >= M)
        # after a 3x3 opening the horizontal 1x3 opening changes nothing
        _, M2, M3 = oracle.morph_chain(M, 0)
        assert np.array_equal(M2, M3)


def _uf_components(M):
    """Brute-force union-find over 4-neighbours."""
    T, F = M.shape
    parent = list(range(T * F))

    def find(a):
        while parent[a] != a:
            a = parent[a]
        return a

    for t in range(T):
        for f in range(F):
            if not M[t, f]:
                continue
            for tt, ff in ((t + 1, f), (t, f + 1)):
                if tt < T and ff < F and M[tt, ff]:
                    ra, rb = find(t * F + f), find(tt * F + ff)
                    if ra != rb:
                        parent[max(ra, rb)] = min(ra, rb)
    roots = {}
    for i in range(T * F):
        if M.flat[i]:
            roots.setdefault(find(i), []).append(i)
    return sorted(roots.values(), key=lambda px: min(px))


def _expected_boxes(M, q, E):
    T, F = M.shape
    out = []
    for px in _uf_components(M):
        px = np.array(px)
        t, f = px // F, px % F
        out.append([t.min(), t.max(), f.min(), f.max(), px.min(), px.size,
                    int(q.flat[px].astype(np.uint64).sum()), int(E[q.flat[px]].sum())])
    return np.array(out, np.int64).reshape(-1, 8)


def test_ccl_boxes_match_union_find_and_scipy():
    rng = np.random.default_rng(4)
    E = oracle.energy_table(0.25)
    for trial in range(80):
        T, F = rng.integers(1, 24), rng.integers(1, 40)
        M = (rng.random((T, F)) < rng.uniform(0.1, 0.9)).astype(np.uint8)
        q = rng.integers(0, 256, size=(T, F)).astype(np.uint8)
        got = oracle.ccl_boxes(M, q)
        assert np.array_equal(got, _expected_boxes(M, q, E))
        lab, n = nd.label(M, structure=FOUR)
        assert got.shape[0] == n
        assert np.all(np.diff(got[:, 4]) > 0)       # anchor order


def test_ccl_on_every_3x3_image():
    E = oracle.energy_table(0.25)
    q = np.arange(9, dtype=np.uint8).reshape(3, 3) * 20
    for M in _all_masks(3, 3):
        assert np.array_equal(oracle.ccl_boxes(M, q), _expected_boxes(M, q, E))


def test_ccl_hand_images():
    # checkerboard: every foreground pixel is its own component
    cb = (np.indices((9, 11)).sum(0) % 2).astype(np.uint8)
    b = oracle.ccl_boxes(cb, np.zeros_like(cb))
    assert b.shape[0] == cb.sum() and np.all(b[:, 5] == 1)
    # a square spiral is one component
    S = np.zeros((21, 21), np.uint8)
    t, f, dt, df = 0, 0, 0, 1
    lo_t, hi_t, lo_f, hi_f = 0, 20, 0, 20
    S[0, :] = 1
    for k in range(0, 10, 2):
        S[k, k:21 - k] = 1
        S[k:21 - k, 20 - k] = 1
        S[20 - k, k:21 - k] = 1
        S[k + 2:21 - k, k] = 1
        S[k + 2, k:k + 3] = 1
    b = oracle.ccl_boxes(S, np.ones_like(S))
    assert b.shape[0] == len(_uf_components(S))
    # diagonal neighbours do not connect (4-connectivity)
    D = np.eye(5, dtype=np.uint8)
    assert oracle.ccl_boxes(D, D).shape[0] == 5
    # empty and full images
    assert oracle.ccl_boxes(np.zeros((4, 4), np.uint8), np.zeros((4, 4), np.uint8)).shape[0] == 0
    full = oracle.ccl_boxes(np.ones((4, 6), np.uint8), np.full((4, 6), 255, np.uint8))
    assert full.tolist() == [[0, 3, 0, 5, 0, 24, 24 * 255, 24 << 32]]


def test_component_runs_and_boundary_against_scipy():
    """Runs rebuild the mask, their components are scipy's 4-connected labels
    numbered by first pixel (the box order), and the boundary is the mask
    minus its erosion by the 4-neighbour cross with a background border."""
    from scipy import ndimage
    rng = np.random.default_rng(21)
    cross = ndimage.generate_binary_structure(2, 1)
    for _ in range(25):
        T, F = int(rng.integers(1, 40)), int(rng.integers(1, 60))
        M = (rng.random((T, F)) < rng.uniform(0.2, 0.8)).astype(np.uint8)
        runs = oracle.component_runs(M)
        back = np.zeros_like(M)
        for c, t, f0, f1 in runs:
            assert np.all(back[t, f0:f1 + 1] == 0)
            back[t, f0:f1 + 1] = 1
        assert np.array_equal(back, M)
        lab, n = ndimage.label(M, structure=cross)
        # scipy numbers components by first pixel in raster order too
        mine = oracle.label(M)
        assert np.array_equal(mine + 1, lab)
        for c, t, f0, f1 in runs:
            assert np.all(lab[t, f0:f1 + 1] == c + 1)
        er = ndimage.binary_erosion(M, structure=cross, border_value=0)
        assert np.array_equal(oracle.boundary(M), (M.astype(bool) & ~er).astype(np.uint8))
        # the boxes of the CCL are the runs' extents per component
        boxes = oracle.ccl_boxes(M, np.zeros_like(M))
        for k, b in enumerate(boxes):
            rk = runs[runs[:, 0] == k]
            assert (b[0], b[1], b[2], b[3]) == (rk[:, 1].min(), rk[:, 1].max(), rk[:, 2].min(), rk[:, 3].max())
