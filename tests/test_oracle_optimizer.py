"""Pins of the oracle's probe position optimizer (Sec. 5 and its listing),
against closed forms computed here from analytic ray/box distances."""
import numpy as np

import oracle
import synth

LIMIT = 0.45


def _desc(**kw):
    d = dict(origin=(0.0, 0.0, 0.0), spacing=(1.0, 1.0, 1.0), counts=(2, 2, 2), rays_per_probe=64,
             seed=77, optimizer_iters=1, offset_limit=LIMIT)
    d.update(kw)
    return synth.VolumeDesc(**d)


def _box_exit(x, dirs, lo, hi):
    """Distance from x (inside [lo, hi]) to the box's boundary along each dir."""
    t = np.full(len(dirs), np.inf)
    for a in range(3):
        with np.errstate(divide="ignore"):
            ta = np.where(dirs[:, a] > 0, (hi[a] - x[a]) / dirs[:, a],
                          np.where(dirs[:, a] < 0, (lo[a] - x[a]) / dirs[:, a], np.inf))
        t = np.minimum(t, ta)
    return t


def test_probe_inside_a_solid_moves_through_the_closest_backface():
    h = 0.2
    sc = synth.solid_box((-h, -h, -h), (h, h, h))
    desc = _desc()
    off = oracle.new_offsets(desc)
    oracle.optimize(oracle.SceneHandle(sc), desc, 3, [0], off)
    dirs = oracle.frame_dirs(desc.seed, 3, desc.rays_per_probe)
    t = _box_exit(np.zeros(3), dirs, -h * np.ones(3), h * np.ones(3))   # every ray hits a backface
    i = int(np.argmin(t))
    vec = t[i] * dirs[i]
    with np.errstate(divide="ignore"):
        comb = np.maximum(LIMIT / vec, -LIMIT / vec)
    scale = comb.min() - 1e-3
    assert scale > 1.0
    assert np.allclose(off[0], vec * scale, rtol=1e-10, atol=1e-12)
    assert abs(np.abs(off[0]).max() - (LIMIT - 1e-3 * np.abs(vec).max())) < 1e-9   # traced vs analytic t
    assert np.all(off[1:] == 0)


def test_backface_move_needs_room_beyond_the_backface():
    # a thick solid: the backface is farther than the offset limit allows -> no move
    sc = synth.solid_box((-2.0, -2.0, -2.0), (2.0, 2.0, 2.0))
    desc = _desc()
    off = oracle.new_offsets(desc)
    oracle.optimize(oracle.SceneHandle(sc), desc, 0, [0], off)
    assert np.all(off == 0)


def test_close_frontfaces_push_the_probe_toward_the_farthest_one():
    lo, hi = -np.ones(3), np.ones(3)
    sc = synth.box_room(lo, hi)
    desc = _desc()
    x0 = np.array([0.3, 0.1, -0.05])
    off = oracle.new_offsets(desc)
    off[0] = x0
    oracle.optimize(oracle.SceneHandle(sc), desc, 5, [0], off)
    dirs = oracle.frame_dirs(desc.seed, 5, desc.rays_per_probe)
    t = _box_exit(x0, dirs, lo, hi)                       # inward walls: all front faces
    ic = int(np.argmin(t))                                # closest, ties to the smaller index
    jf = len(t) - 1 - int(np.argmax(t[::-1]))             # farthest, ties to the larger index
    assert not np.dot(dirs[jf], dirs[ic]) > 0.5
    want = np.clip(x0 + min(0.2, t[jf]) * dirs[jf], -LIMIT, LIMIT)
    assert np.allclose(off[0], want, rtol=1e-12, atol=1e-14)


def test_single_visible_surface_does_not_move():
    # a small quad 1 m below: every front hit lies in a narrow cone
    b = synth._Builder()
    b.quad([(-0.1, -1.0, -0.1), (0.1, -1.0, -0.1), (0.1, -1.0, 0.1), (-0.1, -1.0, 0.1)], (0.0, 1.0, 0.0), obj=0)
    sc = b.finish(np.full((1, 3), 0.5), [1], np.zeros((0, 3)), "quad")
    desc = _desc(rays_per_probe=4096, optimizer_iters=3)
    off = oracle.new_offsets(desc)
    h = oracle.SceneHandle(sc)
    t, tri, bf = oracle.trace(h, np.zeros((desc.rays_per_probe, 3)),
                              oracle.frame_dirs(desc.seed, 0, desc.rays_per_probe))
    assert np.sum(tri >= 0) >= 2 and np.all(bf[tri >= 0] == 0)    # it is seen, from the front
    oracle.optimize(h, desc, 0, [0], off)
    assert np.all(off == 0)


def test_offsets_stay_within_the_limit_over_iterations():
    sc = synth.room_scene()
    desc = synth.room_volume(optimizer_iters=5, offset_limit=LIMIT)
    off = oracle.new_offsets(desc)
    oracle.optimize(oracle.SceneHandle(sc), desc, 0, np.arange(desc.n_probes), off)
    lim = LIMIT * np.asarray(desc.spacing)
    assert np.all(np.abs(off) <= lim * (1 + 1e-12))
    moved = np.any(off != 0, axis=1)
    assert 0 < moved.sum() < desc.n_probes


def test_optimizer_turns_a_buried_probe_on():
    # probe 0 sits inside a thin solid slab: OFF without the optimizer,
    # moved out of it (and no longer OFF) with it
    sc = synth.solid_box((-1.5, -0.1, -1.5), (1.5, 0.1, 1.5))
    h = oracle.SceneHandle(sc)
    for iters, want_off in ((0, True), (5, False)):
        desc = _desc(optimizer_iters=iters)
        st, irr, dist = oracle.new_state(desc)
        off = oracle.new_offsets(desc)
        oracle.update(h, synth.Lights(), desc, 0, st, irr, dist, offsets=off)
        assert (st[0] == oracle.OFF) == want_off, (iters, st[0], off[0])
        if iters:
            assert abs(off[0, 1]) > 0.1       # out of the slab


def test_optimizer_reduces_off_probes_in_the_room():
    """Moving buried probes out of the room's boxes turns some of them on."""
    sc = synth.room_scene()
    h = oracle.SceneHandle(sc)
    n_off = []
    for iters in (0, 5):
        desc = synth.room_volume(optimizer_iters=iters)
        st, irr, dist = oracle.new_state(desc)
        oracle.update(h, synth.room_lights(), desc, 0, st, irr, dist, offsets=oracle.new_offsets(desc))
        n_off.append(int((st == oracle.OFF).sum()))
    assert n_off[1] < n_off[0], n_off
