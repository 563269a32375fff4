"""Cascades with a camera-tracking window (Sec. 7.2, 7.3) against the oracle."""
import json
import os

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
    torch.cuda.set_device(0)
    return pkg


def _descs(R=32):
    common = dict(rays_per_probe=R, hysteresis_irr=0.5, hysteresis_vis=0.5, seed=4242)
    fine = synth.VolumeDesc(origin=(2.0, 2.0, 2.0), spacing=(0.75, 0.75, 0.75), counts=(6, 6, 6),
                            tracking=1, **common)
    coarse = synth.VolumeDesc(origin=(0.625, 0.625, 0.625), spacing=(1.25, 1.25, 1.25), counts=(8, 8, 8),
                              **common)
    return fine, coarse


def _camera(f):
    # float32-exact, so the window's scroll decisions see the same camera on both sides
    return synth.f32([3.0 + 0.55 * f, 4.0 + 0.3 * np.sin(f), 5.0 - 0.2 * f])


def _track_box(desc, cam):
    h = (0.5 * (np.asarray(desc.counts) - 1) - 1.0) * np.asarray(desc.spacing)
    return cam - h, cam + h


def test_cascade_tracking_update_and_query_parity(g):
    sc = synth.room_scene(n_boxes=12)
    L = synth.room_lights()
    fine, coarse = _descs()
    h = oracle.SceneHandle(sc)
    vf = oracle.make_volume(fine)
    vc = oracle.make_volume(coarse)
    of = oracle.new_state(fine)
    ocs = oracle.new_state(coarse)
    C = g.Cascade([fine, coarse])
    S = g.Scene.from_arrays(sc)
    frames = range(5)
    for f in frames:
        cam = _camera(f)
        oracle.tracking_scroll(vf, cam, *of)
        lo, hi = _track_box(fine, cam)
        vf.blend_lo[:] = list(lo)
        vf.blend_hi[:] = list(hi)
        oracle.update_cascade(h, L, [vf, vc], f, [of[0], ocs[0]], [of[1], ocs[1]], [of[2], ocs[2]])
        C.update(S, L, f, cam)
        torch.cuda.synchronize()
        origin, shift = C.window(0)
        assert np.allclose(origin, list(vf.origin), atol=1e-12) and shift == list(vf.shift)
        for k, (st, irr, dist) in enumerate([of, ocs]):
            assert np.array_equal(C.states(k).cpu().numpy(), st), f"states differ, volume {k}, frame {f}"
            ei = rel_err(C.irr_atlas(k).cpu().numpy(), irr).max(-1)
            ed = rel_err(C.dist_atlas(k).cpu().numpy(), dist).max(-1)
            print(f"[cascade] frame {f} volume {k}: shift {shift if k == 0 else '-'}, irr max rel "
                  f"{ei.max():.2e}, dist max rel {ed.max():.2e}")
            assert np.mean(ei <= REL) >= 0.999 and np.mean(ed <= REL) >= 0.999
    C.poll_status()
    pos, nrm, _ = synth.room_queries(n=4096)
    cam = _camera(frames[-1])
    E_ref = oracle.query_cascade([vf, vc], [of[0], ocs[0]], [of[1], ocs[1]], [of[2], ocs[2]], pos, nrm, cam)
    E = C.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy()
    e = rel_err(E, E_ref).max(-1)
    print(f"[cascade] query max rel {e.max():.2e}, over 1e-4: {int((e > REL).sum())}")
    assert np.mean(e <= REL) >= 0.999


def test_cascade_graph_replay_matches_eager(g):
    sc = synth.room_scene(n_boxes=12)
    L = synth.room_lights()
    fine, coarse = _descs()
    S = g.Scene.from_arrays(sc)
    A = g.Cascade([fine, coarse])
    B = g.Cascade([fine, coarse])
    for f in range(6):
        A.update(S, L, f, _camera(f))
        B.update(S, L, f, _camera(f), use_graph=True)
    torch.cuda.synchronize()
    for k in range(2):
        assert torch.equal(A.states(k), B.states(k))
        assert torch.equal(A.buffer(k, 0), B.buffer(k, 0))
        assert torch.equal(A.buffer(k, 1), B.buffer(k, 1))


def test_cascade_autotune_and_cache(g, tmp_path):
    sc = synth.room_scene(n_boxes=12)
    L = synth.room_lights()
    fine, coarse = _descs()
    S = g.Scene.from_arrays(sc)
    C = g.Cascade([fine, coarse])
    path = str(tmp_path / "tune.json")
    assert C.autotune(S, L, 0, _camera(0), cache_path=path) is False
    t = C.tuning()
    assert t[0] in (2, 4, 8, 16) and t[1] in (4, 8, 16)
    with open(path) as fh:
        entries = json.load(fh)
    assert len(entries) == 1
    D = g.Cascade([fine, coarse])
    assert D.autotune(S, L, 0, _camera(0), cache_path=path) is True
    assert D.tuning() == t
    with pytest.raises(g.DDGIError):
        D.set_tuning(0, 8)
