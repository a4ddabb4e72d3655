"""Pins for the oracle's LBVH reference (Morton codes, sort, radix tree, boxes).

Morton codes are checked against hand-built bit strings; the radix tree
against the defining properties of a binary radix tree over sorted,
index-augmented keys with Karras's node numbering (HPG 2012); child boxes
against brute-force min/max over the triangles under each child.
"""
import numpy as np
import pytest

from paper_2503_12174_gb300 import scenes


def _interleave_str(qx, qy, qz):
    bx, by, bz = (format(q, "010b") for q in (qx, qy, qz))
    return int("".join(x + y + z for x, y, z in zip(bx, by, bz)), 2)


def _tri_at(c, s=0.01):
    """A small triangle whose FP32 centroid is (close to) c."""
    c = np.asarray(c, np.float32)
    return np.stack([c + np.float32([s, 0, 0]), c + np.float32([-s, s, 0]), c + np.float32([0, -s, 0])])


def test_morton_hand_computed(orc):
    # centroids at the bounds corners and at known fractions of the extent
    pts = [(0, 0, 0), (1, 1, 1), (0.5, 0.25, 0.75), (0.125, 0.999, 0.0)]
    verts, tris = [], []
    for i, p in enumerate(pts):
        verts.append(_tri_at(p, s=0.0))
        tris.append([3 * i, 3 * i + 1, 3 * i + 2])
    verts = np.concatenate(verts).astype(np.float32)
    tris = np.asarray(tris, np.int32)
    codes = orc.morton(verts, tris)
    assert codes[0] == 0
    assert codes[1] == (1 << 30) - 1
    assert codes[2] == _interleave_str(512, 256, 768)
    assert codes[3] == _interleave_str(128, 1022, 0)
    # x owns the highest bit of every triple
    assert _interleave_str(1, 0, 0) == 4 and _interleave_str(0, 1, 0) == 2 and _interleave_str(0, 0, 1) == 1


def _leaves(child, ref):
    if ref < 0:
        return [~ref]
    return _leaves(child, child[ref, 0]) + _leaves(child, child[ref, 1])


def _delta(keys, i, j):
    x = int(keys[i]) ^ int(keys[j])
    return 64 if x == 0 else 64 - x.bit_length()


def _check_radix_tree(codes_sorted, child):
    T = len(codes_sorted)
    keys = [(int(c) << 32) | i for i, c in enumerate(codes_sorted)]
    assert child.shape == (T - 1, 2)
    assert sorted(_leaves(child, 0)) == list(range(T))       # every leaf exactly once, root covers all
    internal_refs = child[child >= 0]
    assert sorted(internal_refs.tolist()) == list(range(1, T - 1))  # every non-root node has one parent
    for n in range(T - 1):
        lv = _leaves(child, n)
        a, b = min(lv), max(lv)
        assert sorted(lv) == list(range(a, b + 1))           # contiguous key range
        assert n in (a, b)                                   # Karras numbering
        L = _leaves(child, child[n, 0])
        s = max(L)
        assert min(L) == a
        d = _delta(keys, a, b)
        # the split is where the highest differing bit of the range flips
        assert _delta(keys, a, s) > d and _delta(keys, s + 1, b) > d
        assert _delta(keys, s, s + 1) == d
        # left child numbered by its last key, right child by its first key
        if child[n, 0] >= 0:
            assert child[n, 0] == s
        if child[n, 1] >= 0:
            assert child[n, 1] == s + 1


def _check_boxes(verts, tris, order, child, box):
    tv = verts[tris]                              # (T, 3, 3)
    tlo, thi = tv.min(1), tv.max(1)
    for n in range(len(child)):
        for s in range(2):
            lv = np.asarray(_leaves(child, child[n, s]))
            ids = order[lv]
            np.testing.assert_array_equal(box[n, s, :3], tlo[ids].min(0))
            np.testing.assert_array_equal(box[n, s, 3:], thi[ids].max(0))


@pytest.mark.parametrize("which", ["plane", "corner", "random", "duplicates"])
def test_lbvh_structure(orc, which):
    rng = np.random.default_rng(3)
    if which == "plane":
        sc = scenes.plane()
        verts, tris = sc.verts, sc.tris
    elif which == "corner":
        verts, tris, _ = scenes.corner_mesh()
    elif which == "random":
        verts = rng.random((300, 3)).astype(np.float32)
        tris = rng.integers(0, 300, (257, 3)).astype(np.int32)
    else:  # many identical centroids -> equal codes, tie broken by index
        base = rng.random((40, 3)).astype(np.float32)
        verts = np.concatenate([base, base, base]).astype(np.float32)
        tris = np.asarray([[i % 40, (i % 40) + 40, (i % 40) + 80] for i in range(200)], np.int32)
    codes = orc.morton(verts, tris)
    sc_codes, order, child, box = orc.lbvh(verts, tris)
    # sort of (code, index)
    ref_order = np.lexsort((np.arange(len(codes)), codes))
    np.testing.assert_array_equal(order, ref_order)
    np.testing.assert_array_equal(sc_codes, codes[ref_order])
    _check_radix_tree(sc_codes, child)
    _check_boxes(np.asarray(verts, np.float32), np.asarray(tris), order, child, box)
