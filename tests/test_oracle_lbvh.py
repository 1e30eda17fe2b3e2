"""Pins of the oracle's LBVH twin (CPU only): hand-derived Morton codes, an
independent quantise-and-deinterleave check, an independent top-down
binary-radix-tree builder (the tree of unique keys is unique, so Karras'
per-node construction must reproduce it exactly), structural invariants, and
the exactness of the K-sigma leaf boxes."""
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
LEAF = np.int64(0x80000000)


def test_morton_golden(orc):
    rows = np.loadtxt(os.path.join(GOLDEN, "morton_small.txt"))
    codes, lo, hi = orc.morton(rows[:, :3].astype(np.float32))
    np.testing.assert_array_equal(codes.astype(np.int64), rows[:, 3].astype(np.int64))


def _deinterleave(code, shift):
    v = np.zeros_like(code)
    for b in range(10):
        v |= ((code >> (3 * b + shift)) & 1) << b
    return v


def test_morton_quantisation_independent(orc):
    rng = np.random.default_rng(0)
    pts = rng.uniform(-3, 2, size=(5000, 3)).astype(np.float32)
    pts[:7] = pts[7]  # duplicates
    codes, lo, hi = orc.morton(pts)
    np.testing.assert_array_equal(lo, pts.min(0))
    np.testing.assert_array_equal(hi, pts.max(0))
    ext = (hi - lo).astype(np.float32)
    u = ((pts - lo).astype(np.float32) / ext).astype(np.float32)
    q = np.clip(np.floor((u * np.float32(1024)).astype(np.float32)), 0, 1023).astype(np.int64)
    c = codes.astype(np.int64)
    for ax, shift in ((0, 2), (1, 1), (2, 0)):
        np.testing.assert_array_equal(_deinterleave(c, shift), q[:, ax])
    assert c.max() < 2 ** 30


def _topdown(keys):
    """Recursive binary radix tree: a range splits after the last key that
    shares the range's longest common prefix plus a 0 bit.  Node numbering as
    in Karras 2012: a node's index is its split position (left child) or
    split+1 (right child); the root is 0."""
    n = len(keys)
    left = np.full(n - 1, -1, np.int64)
    right = np.full(n - 1, -1, np.int64)
    keys = [int(k) for k in keys]
    stack = [(0, n - 1, 0)]
    while stack:
        first, last, node = stack.pop()
        x = keys[first] ^ keys[last]
        bit = x.bit_length() - 1  # highest differing bit
        split = first
        while split + 1 <= last and not (keys[split + 1] >> bit) & 1:
            split += 1
        lc = (LEAF | split) if split == first else split
        rc = (LEAF | (split + 1)) if split + 1 == last else split + 1
        left[node], right[node] = lc, rc
        if split != first:
            stack.append((first, split, split))
        if split + 1 != last:
            stack.append((split + 1, last, split + 1))
    return left, right


@pytest.mark.parametrize("n,grid", [(2, None), (3, None), (17, None), (1000, None), (3000, 4), (777, 1)])
def test_lbvh_matches_topdown_builder(orc, n, grid):
    rng = np.random.default_rng(n)
    pts = rng.uniform(-1, 1, size=(n, 3))
    if grid:  # many equal Morton codes: ties resolved by the index half of the key
        pts = np.round(pts * grid) / grid
    pts = pts.astype(np.float32)
    t = orc.lbvh(pts)
    codes, _, _ = orc.morton(pts)
    want_keys = np.sort((codes.astype(np.uint64) << np.uint64(32)) | np.arange(n, dtype=np.uint64))
    np.testing.assert_array_equal(t["keys"], want_keys)
    L, R = _topdown(t["keys"])
    np.testing.assert_array_equal(t["left"].astype(np.int64) & 0xFFFFFFFF, L)
    np.testing.assert_array_equal(t["right"].astype(np.int64) & 0xFFFFFFFF, R)


def test_lbvh_structure(orc):
    n = 2000
    pts = np.random.default_rng(3).uniform(-1, 1, size=(n, 3)).astype(np.float32)
    t = orc.lbvh(pts)
    left = t["left"].astype(np.int64) & 0xFFFFFFFF
    right = t["right"].astype(np.int64) & 0xFFFFFFFF
    par = t["parent"]
    seen_leaf = np.zeros(n, int)
    seen_int = np.zeros(n - 1, int)
    depth_max = 0
    stack = [(0, 1)]
    while stack:
        node, depth = stack.pop()
        seen_int[node] += 1
        depth_max = max(depth_max, depth)
        for c in (left[node], right[node]):
            if c & LEAF:
                seen_leaf[c & 0x7FFFFFFF] += 1
                assert par[n - 1 + (c & 0x7FFFFFFF)] == node
            else:
                assert par[c] == node
                stack.append((c, depth + 1))
    assert np.all(seen_leaf == 1) and np.all(seen_int == 1)
    assert par[0] == -1
    assert depth_max <= 64


def test_single_and_empty(orc):
    t = orc.lbvh(np.zeros((1, 3), np.float32))
    assert t["keys"].shape == (1,) and t["parent"][0] == -1
    t = orc.lbvh(np.zeros((0, 3), np.float32))
    assert t["keys"].shape == (0,)


@pytest.mark.parametrize("box_mode", [0, 1])
def test_leaf_boxes_are_exact_extents(orc, box_mode):
    """The box of {m^2 <= K^2} touches the ellipsoid: the support point along
    world axis i is mu + K * Sigma e_i / sqrt(Sigma_ii)."""
    import scenes
    from scipy.spatial.transform import Rotation
    sc = scenes.uniform_scene(64, 5)
    sc["opacity"][:8] = np.float32(0.003)  # below 1/255: empty in mode 1
    sc["opacity"][8:16] = np.float32(0.02)  # shrunken radius in mode 1
    box = orc.leaf_boxes(sc, box_mode=box_mode)
    for j in range(64):
        q = sc["quat"][j].astype(np.float64)
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S = R @ np.diag(sc["scale"][j].astype(np.float64) ** 2) @ R.T
        K = 3.0
        o = float(sc["opacity"][j])
        if box_mode == 1:
            if o < 1 / 255:
                assert np.all(box[j, :3] > box[j, 3:])
                continue
            K = min(3.0, np.sqrt(2 * np.log(o * 255)))
        for i in range(3):
            p = sc["mean"][j].astype(np.float64) + K * S[:, i] / np.sqrt(S[i, i])
            e = p - sc["mean"][j]
            assert e @ np.linalg.inv(S) @ e == pytest.approx(K * K, rel=1e-9)
            assert box[j, 3 + i] == pytest.approx(p[i], abs=1e-12)
            assert box[j, i] == pytest.approx(2 * sc["mean"][j][i] - p[i], abs=1e-12)
