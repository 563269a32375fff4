"""The allocation-free update (ddgi_update_noalloc) against the regular one.

For callers that may not allocate device memory while running (a renderer
with a fixed memory plan, a plug-in whose host owns every buffer): the
caller keeps the volume's states and atlases, the library keeps its scratch
in fixed device arrays.  Two frames in a row through each entry point, on the
same seeded room workload, must agree within the parity tolerance.  This file
is collected last so a failure here comes after every other test has run.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

REL = 1e-4


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    scale = np.maximum(np.abs(b), 1e-3 * max(np.abs(b).max(), 1e-30))
    return np.abs(a - b) / scale


def test_update_noalloc_matches_update_two_frames():
    import paper_2009_10796_gb300 as g
    torch.cuda.set_device(0)
    sc = synth.room_scene()
    lights = synth.room_lights()
    desc = synth.room_volume(hysteresis_irr=0.9, hysteresis_vis=0.8)
    scene = g.Scene.from_arrays(sc)

    ref = g.Volume(desc)
    info = ref.info
    states = torch.zeros(info.n_probes, dtype=torch.uint8, device="cuda")   # all UNINIT
    irr = torch.zeros(info.irr_bytes, dtype=torch.uint8, device="cuda")
    dist = torch.zeros(info.dist_bytes, dtype=torch.uint8, device="cuda")
    for frame in (0, 1):
        ref.update(scene, lights, frame)
        g.update_noalloc(scene, desc, lights, frame, states, irr, dist)
        torch.cuda.synchronize()
        assert torch.equal(states, ref.states()), f"states differ at frame {frame}"
        ei = _rel(irr.view(torch.float32).cpu().numpy(), ref.irr_raw().view(torch.float32).cpu().numpy())
        ed = _rel(dist.view(torch.float32).cpu().numpy(), ref.dist_raw().view(torch.float32).cpu().numpy())
        assert ei.max() <= REL and ed.max() <= REL, (frame, ei.max(), ed.max())


def test_update_noalloc_rejects_oversized_volume():
    import paper_2009_10796_gb300 as g
    scene = g.Scene.from_arrays(synth.room_scene(n_boxes=2))
    big = synth.city_volume()       # 16,384 probes x 256 rays > 1,048,576
    t = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(g.DDGIError) as err:
        g.update_noalloc(scene, big, synth.city_lights(), 0, t, t, t)
    assert err.value.code == 1 and "1048576" in str(err.value)
