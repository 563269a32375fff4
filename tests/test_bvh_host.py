"""Host-side checks of the scene hierarchy (binned SAH tree collapsed to
4-wide nodes) through ddgi_bvh_check: no GPU needed.  Every triangle must be
reachable exactly once, every child box must lie inside its parent's, every
triangle inside its leaf's box, and the walk's stack must stay within the
traversal's fixed stack."""
import numpy as np
import pytest

import synth

STACK4 = 128   # entries of the 4-wide traversal stack


@pytest.fixture(scope="module")
def g():
    import paper_2009_10796_gb300 as pkg
    pkg.load()
    return pkg


def _check(g, verts, tris):
    st = g.bvh_check(verts, tris)
    assert st["violations"] == 0, st
    assert st["tris"] == len(tris)
    if len(tris):
        assert st["max_stack"] <= STACK4
        assert st["depth4"] <= st["depth"] + 1
        assert 0 < st["nodes4"] <= st["nodes"]
    return st


@pytest.mark.parametrize("name", ["room", "city", "interior"])
def test_workload_scenes(g, name):
    sc = {"room": synth.room_scene, "city": synth.city_scene,
          "interior": lambda: synth.interior_scene()[0]}[name]()
    st = _check(g, sc.verts, sc.tris)
    # the 4-wide form needs about half the visits' worth of nodes
    assert st["nodes4"] < 0.6 * st["nodes"]
    print(f"[bvh] {name}: {st}")


def test_random_soup(g):
    rng = np.random.default_rng(7)
    c = rng.uniform(-100, 100, (5000, 1, 3))
    v = (c + rng.normal(0, 2.0, (5000, 3, 3))).reshape(-1, 3)
    t = np.arange(len(v), dtype=np.int32).reshape(-1, 3)
    _check(g, v, t)


def test_identical_triangles_fall_back_to_median_splits(g):
    # equal centroids: no SAH split exists; the builder must still cap leaves
    v = np.tile(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0]], np.float32), (1000, 1))
    t = np.arange(3000, dtype=np.int32).reshape(-1, 3)
    st = _check(g, v, t)
    assert st["leaves"] >= 1000 // 8


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 9])
def test_tiny_scenes(g, n):
    rng = np.random.default_rng(n)
    v = rng.uniform(-1, 1, (3 * n, 3)).astype(np.float32)
    t = np.arange(3 * n, dtype=np.int32).reshape(-1, 3)
    st = _check(g, v, t)
    if n == 0:
        assert st["nodes"] == 0 and st["nodes4"] == 0


def test_far_from_origin_and_flat(g):
    # large coordinates and a zero-thickness (flat) axis
    rng = np.random.default_rng(3)
    xy = rng.uniform(1e5, 1e5 + 50, (3000, 2))
    v = np.stack([xy[:, 0], xy[:, 1], np.full(3000, 7.0)], axis=1)
    t = np.arange(3000, dtype=np.int32).reshape(-1, 3)
    _check(g, v, t)


def test_bad_index_rejected(g):
    v = np.zeros((3, 3), np.float32)
    t = np.array([[0, 1, 5]], np.int32)
    with pytest.raises(g.DDGIError):
        g.bvh_check(v, t)


def test_deep_nested_scales_keep_the_stack_bound(g):
    """Triangles at geometrically shrinking scales around one point drive the
    SAH tree to its depth limits; the 4-wide walk's stack (which the trace
    kernels push without a bound test) must stay within its fixed size."""
    rng = np.random.default_rng(11)
    tris, verts = [], []
    for k in range(3000):
        s = 0.97 ** k
        c = rng.normal(0.0, 1.0, 3) * s
        for q in range(3):
            verts.append(c + rng.normal(0.0, 0.1, 3) * s)
        tris.append([3 * k, 3 * k + 1, 3 * k + 2])
    st = _check(g, np.asarray(verts, np.float32), np.asarray(tris, np.int32))
    print(f"[bvh] nested: {st}")
    assert st["depth"] > 20
