"""GPU parity of the LBVH builder against the oracle's CPU twin: sorted keys
and topology bit-exact, node boxes conservative and tight."""
import numpy as np
import pytest
import torch

import scenes

pytestmark = pytest.mark.gpu


def _dev(sc):
    return {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in sc.items()}


def _build(sc, **kw):
    from paper_2311_16043_gb300 import rt
    d = _dev(sc)
    return rt.rt_build_bvh(d["mean"], d["scale"], d["quat"], d["opacity"], rt.params(**kw)), d


def _export(bvh):
    from paper_2311_16043_gb300 import rt
    ex = rt.rt_bvh_export(bvh)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in ex.items()}


@pytest.mark.parametrize("n,seed,grid", [(1, 0, None), (2, 1, None), (3, 2, None), (4096, 1, None),
                                         (10001, 3, None), (5000, 4, 8), (300_000, 2, None),
                                         (2_000_000, 2, None)])
def test_topology_bit_exact(orc, n, seed, grid):
    """Sorted keys, children and parents equal the CPU twin's, up to the
    bench's 2M-Gaussian object scene."""
    sc = scenes.object_scene(n, seed) if n >= 300_000 else scenes.uniform_scene(n, seed)
    if grid:  # many equal Morton codes
        sc["mean"] = (np.round(sc["mean"] * grid) / grid).astype(np.float32)
    bvh, _ = _build(sc)
    ex = _export(bvh)
    ref = orc.lbvh(sc["mean"])
    np.testing.assert_array_equal(ex["keys"].view(np.uint64), ref["keys"])
    np.testing.assert_array_equal(ex["left"], ref["left"])
    np.testing.assert_array_equal(ex["right"], ref["right"])
    np.testing.assert_array_equal(ex["parent"], ref["parent"])
    info = bvh.info()
    np.testing.assert_array_equal(np.array(info["lo"], np.float32), sc["mean"].min(0))
    np.testing.assert_array_equal(np.array(info["hi"], np.float32), sc["mean"].max(0))


def test_degenerate_all_equal_means(orc):
    sc = scenes.uniform_scene(777, 9)
    sc["mean"][:] = np.float32(0.25)
    bvh, _ = _build(sc)
    ex = _export(bvh)
    ref = orc.lbvh(sc["mean"])
    np.testing.assert_array_equal(ex["keys"].view(np.uint64), ref["keys"])
    np.testing.assert_array_equal(ex["left"], ref["left"])


def _node_boxes(ref, leaf, n):
    """FP64 union boxes of the oracle topology: (lo, hi) per internal node."""
    left = ref["left"].astype(np.int64) & 0xFFFFFFFF
    right = ref["right"].astype(np.int64) & 0xFFFFFFFF
    perm = (ref["keys"] & np.uint64(0xFFFFFFFF)).astype(np.int64)
    box = np.zeros((n - 1, 6))
    order = []
    stack = [0]
    while stack:
        i = stack.pop()
        order.append(i)
        for c in (left[i], right[i]):
            if not c & 0x80000000:
                stack.append(c)

    def child_box(c):
        if c & 0x80000000:
            return leaf[perm[c & 0x7FFFFFFF]]
        return box[c]
    for i in reversed(order):
        a, b = child_box(left[i]), child_box(right[i])
        box[i] = np.concatenate([np.minimum(a[:3], b[:3]), np.maximum(a[3:], b[3:])])
    return box, left, right, perm


@pytest.mark.parametrize("box_mode", [0, 1])
def test_child_boxes_conservative_and_tight(orc, box_mode):
    n = 4096
    sc = scenes.uniform_scene(n, 1)
    sc["opacity"][:50] = np.float32(0.002)  # below the cutoff: empty boxes in mode 1
    sc["opacity"][1000:1040] = np.float32(0.002)  # a run of neighbours in Morton order
    bvh, _ = _build(sc, box_mode=box_mode)
    ex = _export(bvh)
    ref = orc.lbvh(sc["mean"])
    leaf = orc.leaf_boxes(sc, box_mode=box_mode)
    box, left, right, perm = _node_boxes(ref, leaf, n)
    for side, refs in ((0, left), (1, right)):
        g = ex["boxes"][:, 6 * side:6 * side + 6].astype(np.float64)
        exact = np.array([leaf[perm[c & 0x7FFFFFFF]] if c & 0x80000000 else box[c] for c in refs])
        nonempty = exact[:, 0] <= exact[:, 3]
        ext = (exact[:, 3:] - exact[:, :3])[nonempty]
        # contains the exact support ...
        assert np.all(g[nonempty, :3] <= exact[nonempty, :3])
        assert np.all(g[nonempty, 3:] >= exact[nonempty, 3:])
        # ... and is no more than the stated margin larger
        slack = np.maximum(exact[nonempty, :3] - g[nonempty, :3], g[nonempty, 3:] - exact[nonempty, 3:])
        assert np.all(slack <= 2e-4 * ext + 1e-5)
        if box_mode == 1:  # empty supports are NaN boxes, which no ray hits
            assert np.all(np.isnan(g[~nonempty]))
