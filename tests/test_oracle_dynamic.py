"""Pins of the oracle's dynamic-object wake-up (Sec. 6.3): sleeping probes in
an object's box extended by one cell plus the self-shadow bias are woken,
traced with hysteresis 0, become Awake, and go back to sleep once no object
is near; other states are untouched."""
import numpy as np

import oracle
import synth

SPACING = 1.0
B = 0.3


def _setup(states=None):
    sc = synth.room_scene(n_boxes=4)
    desc = synth.VolumeDesc(origin=(3.0, 3.0, 3.0), spacing=(SPACING,) * 3, counts=(4, 4, 4), rays_per_probe=32,
                            hysteresis_irr=0.9, hysteresis_vis=0.9, self_shadow_bias=B, seed=5)
    st, irr, dist = oracle.new_state(desc)
    st[:] = oracle.SLEEPING if states is None else states
    return oracle.SceneHandle(sc), desc, st, irr, dist


def _probe(desc, i, j, k):
    return i + desc.counts[0] * (j + desc.counts[1] * k)


def test_extension_is_one_cell_plus_the_bias():
    h, desc, st, irr, dist = _setup()
    ext = SPACING + 0.75 * SPACING * B
    x = np.asarray(desc.origin) + np.array([1, 1, 1]) * SPACING       # probe (1,1,1)
    # a point-like object just within / just beyond the extension along +x
    for gap, woken in ((ext - 1e-6, True), (ext + 1e-6, False)):
        s = st.copy()
        box = np.array([[x[0] + gap, x[1], x[2], x[0] + gap, x[1], x[2]]])
        oracle.update(h, synth.Lights(), desc, 0, s, irr.copy(), dist.copy(), dyn_boxes=box)
        p = _probe(desc, 1, 1, 1)
        assert (s[p] == oracle.AWAKE) == woken, (gap, s[p])


def test_wake_trace_converge_and_sleep_again():
    states = np.full(64, oracle.SLEEPING, np.uint8)
    states[0] = oracle.OFF
    states[63] = oracle.VIGILANT
    h, desc, st, irr, dist = _setup(states)
    x0 = np.asarray(desc.origin)
    box = np.array([[x0[0] - 0.1, x0[1] - 0.1, x0[2] - 0.1, x0[0] + 0.1, x0[1] + 0.1, x0[2] + 0.1]])
    rays = oracle.update(h, synth.room_lights(), desc, 0, st, irr, dist, dyn_boxes=box, want_rays=True)
    grid = np.stack(np.meshgrid(*[np.arange(4)] * 3, indexing="ij"), -1).reshape(-1, 3)
    ijk = np.array([[p % 4, (p // 4) % 4, p // 16] for p in range(64)])
    near = np.all(ijk <= 1, axis=1)        # within one cell + bias of the box around probe 0
    assert st[0] == oracle.OFF and st[63] == oracle.VIGILANT
    assert np.all(st[near & (np.arange(64) != 0)] == oracle.AWAKE)
    assert np.all(st[~near & (np.arange(64) != 63)] == oracle.SLEEPING)
    traced = ~np.isnan(rays[:, 0, 0])
    assert np.array_equal(traced, (st == oracle.AWAKE) | (st == oracle.VIGILANT))
    # newly woken probes blend with hysteresis 0: from the same zero atlas,
    # hysteresis 0.9 and hysteresis 0 give them the same texels, while the
    # already-vigilant probe 63 keeps 90% of its old (zero) value
    d0 = synth.VolumeDesc(**{**desc.__dict__, "hysteresis_irr": 0.0, "hysteresis_vis": 0.0})
    _, _, s2, i2, t2 = _setup(states)
    oracle.update(h, synth.room_lights(), d0, 0, s2, i2, t2, dyn_boxes=box)
    awake = st == oracle.AWAKE
    assert np.array_equal(i2[awake], irr[awake]) and np.array_equal(t2[awake], dist[awake])
    assert not np.allclose(i2[63], irr[63])
    # the object leaves: awake probes go back to sleep and are not traced
    rays = oracle.update(h, synth.room_lights(), desc, 1, st, irr, dist, dyn_boxes=None, want_rays=True)
    assert np.all(st[near & (np.arange(64) != 0)] == oracle.SLEEPING)
    assert np.array_equal(~np.isnan(rays[:, 0, 0]), st == oracle.VIGILANT)


def test_awake_probes_shade_queries():
    """Awake probes count as active in the query (they shade the moving object)."""
    vol = synth.VolumeDesc(origin=(0, 0, 0), spacing=(1, 1, 1), counts=(2, 2, 2), rays_per_probe=8,
                           self_shadow_bias=0.0, state_machine=1, gamma=5.0)
    st, irr, dist = oracle.new_state(vol)
    irr[:] = 0.5
    dist[..., 0] = 5.0
    dist[..., 1] = 25.0
    x = np.array([[0.5, 0.5, 0.5]])
    n = np.array([[0.0, 0.0, 1.0]])
    for s, want in ((oracle.SLEEPING, 0.0), (oracle.AWAKE, np.pi * 0.5 ** 5)):
        st[:] = s
        E = oracle.query(vol, st, irr, dist, x, n, np.array([0.5, 0.5, 9.0]))
        assert np.allclose(E, want)
