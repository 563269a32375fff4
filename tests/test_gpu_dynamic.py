"""Dynamic-object wake-up (Sec. 6.3) on the GPU against the FP64 oracle: the
room scene with three boxes moving through it over four frames.  States must
match exactly; texels and queries to the FP32 tolerance."""
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


def _boxes(f):
    c = np.array([[2.0 + 1.5 * f, 5.0, 5.0], [8.0, 2.0 + 1.3 * f, 3.0], [5.0, 8.0, 1.0 + 1.7 * f]])
    h = np.array([[0.4, 0.6, 0.5], [0.7, 0.3, 0.4], [0.5, 0.5, 0.8]])
    return np.concatenate([c - h, c + h], axis=1)


def test_dynamic_wakeup_parity(g):
    sc = synth.room_scene()
    L = synth.room_lights()
    desc = synth.room_volume(hysteresis_irr=0.8, hysteresis_vis=0.8)
    h = oracle.SceneHandle(sc)
    st, irr, dist = oracle.new_state(desc)
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    awake_seen = 0
    for f in range(4):
        boxes = _boxes(f) if f < 3 else np.zeros((0, 6))
        oracle.update(h, L, desc, f, st, irr, dist, dyn_boxes=boxes)
        V.set_dynamic_boxes(boxes)
        V.update(S, L, f)
        gs = V.states().cpu().numpy()
        assert np.array_equal(gs, st), f"states differ at frame {f}"
        awake_seen += int((st == oracle.AWAKE).sum())
    torch.cuda.synchronize()
    V.poll_status()
    assert awake_seen > 0
    assert not np.any(st == oracle.AWAKE)       # the last frame has no objects: all back to sleep
    ei = rel_err(V.irr_atlas().cpu().numpy(), irr).max(-1)
    ed = rel_err(V.dist_atlas().cpu().numpy(), dist).max(-1)
    print(f"[dynamic] awake probe-frames {awake_seen}; irr max {ei.max():.2e}, dist max {ed.max():.2e}")
    assert ei.max() <= REL and ed.max() <= REL


def test_dynamic_boxes_validation(g):
    V = g.Volume(synth.room_volume())
    with pytest.raises(g.DDGIError):
        V.set_dynamic_boxes(np.array([[1, 1, 1, 0, 0, 0]], np.float32))     # lo > hi
    with pytest.raises(g.DDGIError):
        V.set_dynamic_boxes(np.zeros((1025, 6), np.float32))
    W = g.Volume(synth.room_volume(state_machine=0))
    with pytest.raises(g.DDGIError):
        W.set_dynamic_boxes(np.zeros((1, 6), np.float32))
    V.set_dynamic_boxes(np.zeros((0, 6), np.float32))
