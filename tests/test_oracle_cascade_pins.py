"""Pins of the oracle's tracking window (Sec. 7.2) and cascade update (Sec. 7.3)."""
import numpy as np

import oracle
import synth


def _tagged_volume(desc):
    st, irr, dist = oracle.new_state(desc, initial=oracle.VIGILANT)
    v = oracle.make_volume(desc)
    return v, st, irr, dist


def _world_tags(v, desc, irr):
    """world position of every stored probe -> its tag (irr texel [1,1,0])."""
    out = {}
    cx, cy, cz = desc.counts
    for k in range(cz):
        for j in range(cy):
            for i in range(cx):
                p = oracle.lib().or_probe_phys(oracle.C.byref(v), i, j, k)
                pos = (round(v.origin[0] + i * v.spacing[0], 6), round(v.origin[1] + j * v.spacing[1], 6),
                       round(v.origin[2] + k * v.spacing[2], 6))
                out[pos] = (p, irr[p, 1, 1, 0])
    return out


def test_tracking_window_data_follows_world_positions():
    desc = synth.VolumeDesc(origin=(-3.5, -2.5, -2.0), spacing=(1.0, 1.0, 1.0), counts=(8, 6, 5),
                            state_machine=1)
    v, st, irr, dist = _tagged_volume(desc)
    # tag every probe with a function of its world position
    tags = _world_tags(v, desc, irr)
    for pos, (p, _) in tags.items():
        irr[p] = 1.0 + 0.01 * pos[0] + 0.1 * pos[1] + 0.37 * pos[2]
    rng = synth.Rng(5)
    cam = np.array([0.0, 0.0, 0.0])
    total = 0
    for step in range(60):
        cam = cam + rng.uniform(3, -1.7, 1.7)
        before = _world_tags(v, desc, irr)
        moved = oracle.tracking_scroll(v, cam, st, irr, dist)
        total += moved
        after = _world_tags(v, desc, irr)
        centre = np.array(v.origin) + 0.5 * (np.array(desc.counts) - 1) * np.array(desc.spacing)
        assert np.all(np.abs(cam - centre) <= np.array(desc.spacing) + 1e-12)
        for pos, (p, val) in after.items():
            if pos in before:
                # a probe that stayed in the window keeps its data
                assert val == before[pos][1]
                assert st[p] == oracle.VIGILANT
            else:
                # a plane that leapfrogged is reset
                assert val == 0.0 and st[p] == oracle.UNINIT and not dist[p].any()
                # newly covered world positions get fresh tags for later steps
                irr[p] = 1.0 + 0.01 * pos[0] + 0.1 * pos[1] + 0.37 * pos[2]
                st[p] = oracle.VIGILANT
    assert total > 20


def test_tracking_moves_count_planes():
    desc = synth.VolumeDesc(origin=(0, 0, 0), spacing=(2.0, 1.0, 1.0), counts=(4, 4, 4))
    v, st, irr, dist = _tagged_volume(desc)
    # centre at x = 3; the camera 7.5 m ahead moves the window 3 planes (centre 9, |7.5 + 3 - 9| <= 2)
    moved = oracle.tracking_scroll(v, [10.5, 1.5, 1.5], st, irr, dist)
    assert moved == 3 and v.origin[0] == 6.0 and v.shift[0] == 3
    assert np.sum(st == oracle.UNINIT) == 3 * 16


def test_cascade_of_one_volume_is_the_single_volume_update():
    sc = synth.room_scene(n_boxes=6)
    L = synth.room_lights()
    desc = synth.room_volume(counts=(4, 4, 4), spacing=(2.5, 2.5, 2.5), origin=(1.25, 1.25, 1.25),
                             hysteresis_irr=0.8, hysteresis_vis=0.7)
    h = oracle.SceneHandle(sc)
    a = oracle.new_state(desc)
    b = oracle.new_state(desc)
    for f in range(3):
        oracle.update(h, L, desc, f, *a)
        oracle.update_cascade(h, L, [oracle.make_volume(desc)], f, [b[0]], [b[1]], [b[2]])
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_cascade_furnace_exact():
    # two nested volumes in an emitting room: hit shading blends both volumes,
    # all probes agree, so M_t = Le (1 - rho^(t+1)) / (1 - rho) exactly
    Le, rho = 0.7, 0.5
    sc = synth.box_room((-6, -6, -6), (6, 6, 6), albedo=rho, emit=[Le, Le, Le])
    fine = synth.VolumeDesc(origin=(-2, -2, -2), spacing=(1, 1, 1), counts=(5, 5, 5), rays_per_probe=32,
                            hysteresis_irr=0, hysteresis_vis=0, state_machine=0, seed=3)
    coarse = synth.VolumeDesc(origin=(-4.5, -4.5, -4.5), spacing=(3, 3, 3), counts=(4, 4, 4),
                              rays_per_probe=32, hysteresis_irr=0, hysteresis_vis=0, state_machine=0,
                              seed=3)
    vf = oracle.make_volume(fine)
    # the coarse volume's fall-off box covers the room, so every hit has weight 1
    vc = oracle.make_volume(coarse, blend_lo=(-20, -20, -20), blend_hi=(20, 20, 20))
    sf, irf, df = oracle.new_state(fine)
    scs, irc, dc = oracle.new_state(coarse)
    h = oracle.SceneHandle(sc)
    for t in range(4):
        _, w = None, None
        oracle.update_cascade(h, synth.Lights(), [vf, vc], t, [sf, scs], [irf, irc], [df, dc])
        want = Le * (1 - rho ** (t + 1)) / (1 - rho)
        assert np.allclose(irf[:, 1:-1, 1:-1] ** 5, want, rtol=1e-12)
        assert np.allclose(irc[:, 1:-1, 1:-1] ** 5, want, rtol=1e-12)
    # both volumes contribute to hit shading in the fall-off region
    pos = np.array([[1.5, 0.0, 0.0]])    # inside the fine volume's last cell
    E, w = oracle.query_cascade([vf, vc], [sf, scs], [irf, irc], [df, dc], pos, np.array([[0, 1.0, 0]]),
                                np.zeros(3), want_weights=True)
    assert 0 < w[0, 0] < 1 and np.isclose(w.sum(), 1.0)
