"""The allocation-free update (ddgi_update_noalloc) against the regular one.

For callers that may not allocate device memory while running (a renderer
with a fixed memory plan, a plug-in whose host owns every buffer): the
caller keeps the volume's states and atlases, the library keeps its scratch
in fixed device arrays.  Two frames in a row through each entry point, on the
same seeded room workload, must agree within the parity tolerance, for each
storage format and with the state machine on and off; after a warm-up call,
further calls must leave the device's free memory unchanged; a non-finite
texel must come back through ddgi_update_noalloc_poll_status.  This file is
collected last so a failure here comes after every other test has run.
"""
import gc

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


def _rgb9e5(words):
    w = words.astype(np.int64)
    s = np.exp2((w >> 27) - 24.0)
    return np.stack([(w & 511) * s, ((w >> 9) & 511) * s, ((w >> 18) & 511) * s], -1)


def _decode(raw, which, fmt):
    """Raw atlas bytes (torch uint8 on the device) -> float64 texel values."""
    a = raw.cpu()
    if which == 0:
        if fmt == 0:
            return a.view(torch.float32).numpy().reshape(-1, 4)[:, :3].astype(np.float64)
        if fmt == 1:
            return a.view(torch.float16).float().numpy().reshape(-1, 4)[:, :3].astype(np.float64)
        return _rgb9e5(a.view(torch.int32).numpy())
    if fmt == 0:
        return a.view(torch.float32).numpy().reshape(-1, 2).astype(np.float64)
    return a.view(torch.float16).float().numpy().reshape(-1, 2).astype(np.float64)


# (irradiance format, distance format) -> per-texel tolerance on the decoded
# values: FP32 the parity tolerance; FP16 half an FP16 ulp (2^-11 relative) on
# top, for stored values that round on different sides of a boundary; RGB9E5
# 2^-9 of the texel's largest channel (its mantissa step)
FORMATS = {"fp32": (0, 0), "fp16": (1, 1), "rgb9e5": (2, 0)}


def _close(got, ref, which, fmt):
    if fmt == 0:
        return _rel(got, ref).max() <= REL
    if which == 0 and fmt == 2:
        mx = ref.max(-1, keepdims=True)
        return bool(np.all(np.abs(got - ref) <= 2.0 ** -9 * mx + REL * np.maximum(mx, 1e-3 * ref.max())))
    return _rel(got, ref).max() <= 2.0 ** -11 + REL


@pytest.mark.parametrize("state_machine", [1, 0])
@pytest.mark.parametrize("formats", list(FORMATS))
def test_update_noalloc_matches_update_two_frames(formats, state_machine):
    import paper_2009_10796_gb300 as g
    torch.cuda.set_device(0)
    irr_fmt, dist_fmt = FORMATS[formats]
    sc = synth.room_scene()
    lights = synth.room_lights()
    scene = g.Scene.from_arrays(sc)
    ref = g.Volume(synth.room_volume(hysteresis_irr=0.9, hysteresis_vis=0.8, state_machine=state_machine),
                   irr_format=irr_fmt, dist_format=dist_fmt)
    desc = ref.desc             # the descriptor with the storage formats set
    info = ref.info
    init = 0 if state_machine else g.STATE_VIGILANT
    states = torch.full((info.n_probes,), init, dtype=torch.uint8, device="cuda")
    irr = torch.zeros(info.irr_bytes, dtype=torch.uint8, device="cuda")
    dist = torch.zeros(info.dist_bytes, dtype=torch.uint8, device="cuda")
    for frame in (0, 1):
        ref.update(scene, lights, frame)
        g.update_noalloc(scene, desc, lights, frame, states, irr, dist)
        torch.cuda.synchronize()
        assert torch.equal(states, ref.states()), f"states differ at frame {frame}"
        gi, ri = _decode(irr, 0, irr_fmt), _decode(ref.irr_raw(), 0, irr_fmt)
        gd, rd = _decode(dist, 1, dist_fmt), _decode(ref.dist_raw(), 1, dist_fmt)
        assert _close(gi, ri, 0, irr_fmt), (frame, "irradiance", float(_rel(gi, ri).max()))
        assert _close(gd, rd, 1, dist_fmt), (frame, "distance", float(_rel(gd, rd).max()))
    g.update_noalloc_poll_status()


def test_update_noalloc_allocates_nothing():
    """After a warm-up call (which loads the module and with it the fixed
    arrays on this device), ten more calls, each followed by a synchronise,
    leave the device's free memory exactly as it was."""
    import paper_2009_10796_gb300 as g
    torch.cuda.set_device(0)
    sc = synth.room_scene()
    lights = synth.room_lights()
    desc = synth.room_volume(hysteresis_irr=0.9, hysteresis_vis=0.8)
    scene = g.Scene.from_arrays(sc)
    info = g.Volume(desc).info
    states = torch.zeros(info.n_probes, dtype=torch.uint8, device="cuda")
    irr = torch.zeros(info.irr_bytes, dtype=torch.uint8, device="cuda")
    dist = torch.zeros(info.dist_bytes, dtype=torch.uint8, device="cuda")
    g.update_noalloc(scene, desc, lights, 0, states, irr, dist)
    torch.cuda.synchronize()
    # no garbage collection inside the window: another test's volume freed
    # there would change the free memory as well
    gc.collect()
    gc.disable()
    try:
        free0, _ = torch.cuda.mem_get_info()
        for frame in range(1, 11):
            g.update_noalloc(scene, desc, lights, frame, states, irr, dist)
            torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
    finally:
        gc.enable()
    g.update_noalloc_poll_status()
    assert free1 == free0, f"device free memory changed by {free0 - free1} bytes over 10 calls"


def test_update_noalloc_reports_non_finite_texels():
    """An emitter of infinite radiance makes texels non-finite: the calls
    themselves return OK (the error is found on the device), the poll
    returns NUMERIC once and then OK again."""
    import paper_2009_10796_gb300 as g
    torch.cuda.set_device(0)
    sc = synth.room_scene()
    sc.emitter_radiance = np.full_like(np.asarray(sc.emitter_radiance, dtype=np.float64), np.inf)
    desc = synth.room_volume()
    scene = g.Scene.from_arrays(sc)
    info = g.Volume(desc).info
    states = torch.zeros(info.n_probes, dtype=torch.uint8, device="cuda")
    irr = torch.zeros(info.irr_bytes, dtype=torch.uint8, device="cuda")
    dist = torch.zeros(info.dist_bytes, dtype=torch.uint8, device="cuda")
    g.update_noalloc_poll_status()          # start from a clear word
    for frame in (0, 1):
        g.update_noalloc(scene, desc, synth.room_lights(), frame, states, irr, dist)
    with pytest.raises(g.DDGIError) as err:
        g.update_noalloc_poll_status()
    assert err.value.code == 5
    g.update_noalloc_poll_status()          # the poll cleared it


def test_update_noalloc_rejects_oversized_volume():
    import paper_2009_10796_gb300 as g
    scene = g.Scene.from_arrays(synth.room_scene(n_boxes=2))
    big = synth.city_volume()       # 16,384 probes x 256 rays > 1,048,576
    t = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(g.DDGIError) as err:
        g.update_noalloc(scene, big, synth.city_lights(), 0, t, t, t)
    assert err.value.code == 1 and "1048576" in str(err.value)
