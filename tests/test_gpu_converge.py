"""Optional converge pass for new probes (Sec. 6.3) on the GPU against the
FP64 oracle: the room scene with 3 batches of 64 rays for every Newly
Vigilant probe at frame 0 and for probes woken by a moving box, then regular
frames with hysteresis.  States bit-exact; texels and queries to the FP32
tolerance."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import REL, rel_err, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2009_10796_gb300 as pkg
    pkg.load()
    return pkg


def _box(f):
    c = np.array([[2.0 + 1.5 * f, 5.0, 5.0]])
    h = np.array([[0.5, 0.6, 0.5]])
    return np.concatenate([c - h, c + h], axis=1)


@pytest.mark.parametrize("dynamic", [False, True])
def test_converge_pass_parity(g, dynamic):
    sc = synth.room_scene()
    L = synth.room_lights()
    desc = synth.room_volume(converge_batches=3, hysteresis_irr=0.9, hysteresis_vis=0.9)
    h = oracle.SceneHandle(sc)
    st, irr, dist = oracle.new_state(desc)
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    for f in range(3):
        boxes = _box(f) if dynamic and f >= 1 else np.zeros((0, 6))
        oracle.update(h, L, desc, f, st, irr, dist, dyn_boxes=boxes)
        V.set_dynamic_boxes(boxes)
        V.update(S, L, f)
        gs = V.states().cpu().numpy()
        assert np.array_equal(gs, st), f"states differ at frame {f}"
    torch.cuda.synchronize()
    V.poll_status()
    assert not np.any(st == oracle.NEWLY_VIGILANT) and not np.any(st == oracle.NEWLY_AWAKE)
    if dynamic:
        assert np.any(st == oracle.AWAKE)
    ei = rel_err(V.irr_atlas().cpu().numpy(), irr).max(-1)
    ed = rel_err(V.dist_atlas().cpu().numpy(), dist).max(-1)
    print(f"[converge] irr max {ei.max():.2e}, dist max {ed.max():.2e}")
    assert ei.max() <= REL and ed.max() <= REL
    pos, nrm, cam = synth.room_queries(n=2048)
    want = oracle.query(desc, st, irr, dist, pos, nrm, cam)
    got = V.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy()
    eq = rel_err(got, want).max(-1)
    print(f"[converge] query max {eq.max():.2e}")
    assert eq.max() <= REL


def test_converge_changes_the_first_frame(g):
    """With the pass, a new probe's first texels average 4 x 64 rays instead
    of 64: they differ from the single-pass result and sit closer to a
    many-ray reference."""
    sc = synth.room_scene()
    L = synth.room_lights()
    S = g.Scene.from_arrays(sc)
    base = synth.room_volume(hysteresis_irr=0.0, hysteresis_vis=0.0)
    one = g.Volume(base)
    one.update(S, L, 0)
    conv = g.Volume(synth.room_volume(converge_batches=4, hysteresis_irr=1.0, hysteresis_vis=1.0,
                                      thr_low=10.0, thr_high=20.0))
    conv.update(S, L, 0)
    ref = g.Volume(synth.room_volume(rays_per_probe=1024, hysteresis_irr=0.0, hysteresis_vis=0.0))
    ref.update(S, L, 0)
    torch.cuda.synchronize()
    act = one.states().cpu().numpy() == g.STATE_VIGILANT
    a1 = one.irr_atlas().cpu().numpy()[act]
    ac = conv.irr_atlas().cpu().numpy()[act]
    ar = ref.irr_atlas().cpu().numpy()[act]
    assert not np.allclose(a1, ac)
    assert np.abs(ac - ar).mean() < np.abs(a1 - ar).mean()


def test_converge_descriptor_checks(g):
    with pytest.raises(g.DDGIError):
        g.Volume(synth.room_volume(converge_batches=65))
    with pytest.raises(g.DDGIError):
        g.Cascade([synth.room_volume(converge_batches=2)])
