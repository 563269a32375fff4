"""The host-buffer frame call (probe update of Sec. 2.3, then the Sec. 2.2
query of a host G-buffer) against the device-pointer path: the same kernels
on the same data, so atlases, states and irradiance must agree bit for bit.
Also the kept active list: once no probe can change state the update reuses
the previous frame's list, and a restored state buffer must discard it."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2009_10796_gb300 as pkg
    pkg.load()
    return pkg


def _pinned(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).pin_memory()


@pytest.mark.parametrize("n", [4096, 4099, 1, 0])
def test_frame_host_matches_device_path(g, n):
    sc = synth.room_scene()
    L = synth.room_lights()
    desc = synth.room_volume(hysteresis_irr=0.85, hysteresis_vis=0.85)
    pos, nrm, cam = synth.room_queries(n=max(n, 1))
    pos, nrm = pos[:n], nrm[:n]
    S = g.Scene.from_arrays(sc)
    A, B = g.Volume(desc), g.Volume(desc)
    pos_d = torch.from_numpy(np.ascontiguousarray(pos, np.float32)).cuda()
    nrm_d = torch.from_numpy(np.ascontiguousarray(nrm, np.float32)).cuda()
    pos_h, nrm_h = _pinned(pos), _pinned(nrm)
    out_h = torch.full((n, 3), -1.0).pin_memory()
    for f in range(4):
        A.update(S, L, f)
        ref = A.query(pos_d, nrm_d, cam).cpu()
        # pageable host memory on one frame, pinned on the others
        if f == 2:
            got = B.frame_host(S, L, f, torch.from_numpy(np.array(pos, np.float32)),
                               torch.from_numpy(np.array(nrm, np.float32)), cam, torch.empty((n, 3)))
        else:
            got = B.frame_host(S, L, f, pos_h, nrm_h, cam, out_h)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"irradiance differs at frame {f}"
    assert torch.equal(A.states().cpu(), B.states().cpu())
    assert torch.equal(A.irr_atlas().cpu(), B.irr_atlas().cpu())
    assert torch.equal(A.dist_atlas().cpu(), B.dist_atlas().cpu())
    A.poll_status()
    B.poll_status()


def test_frame_host_grows_staging(g):
    sc = synth.room_scene()
    L = synth.room_lights()
    desc = synth.room_volume()
    S = g.Scene.from_arrays(sc)
    A, B = g.Volume(desc), g.Volume(desc)
    for f, n in enumerate([100, 5000, 3000, 9001]):
        pos, nrm, cam = synth.room_queries(seed=4000 + f, n=n)
        A.update(S, L, f)
        ref = A.query(_pinned(pos).cuda(), _pinned(nrm).cuda(), cam).cpu()
        got = B.frame_host(S, L, f, _pinned(pos), _pinned(nrm), cam)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), f"n = {n}"


def test_frame_host_rejects_device_tensors(g):
    V = g.Volume(synth.room_volume())
    S = g.Scene.from_arrays(synth.room_scene())
    x = torch.zeros((8, 3), device="cuda")
    with pytest.raises(ValueError):
        V.frame_host(S, synth.room_lights(), 0, x, x, (5.0, 5.0, 5.0))


def test_restored_states_drop_kept_list(g):
    """Frames 2+ reuse the active list; restoring a state buffer in which a
    third of the probes are OFF must shrink the traced set at once."""
    sc = synth.room_scene()
    L = synth.room_lights()
    desc = synth.room_volume(hysteresis_irr=0.9, hysteresis_vis=0.9)
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    for f in range(3):
        V.update(S, L, f)
    st = V.states().clone()
    n_active = int((st == g.STATE_VIGILANT).sum())
    assert n_active > 0
    assert V.trace_stats(S, L)["rays"] == n_active * desc.rays_per_probe
    cut = st.clone()
    idx = torch.nonzero(cut == g.STATE_VIGILANT).flatten()[::3]
    cut[idx] = g.STATE_OFF
    V.set_buffer(2, cut)
    irr0 = V.irr_atlas().clone()
    V.update(S, L, 3)
    n_now = int((V.states() == g.STATE_VIGILANT).sum())
    assert n_now == n_active - idx.numel()
    assert V.trace_stats(S, L)["rays"] == n_now * desc.rays_per_probe
    # the switched-off probes keep their texels; the others moved on
    irr1 = V.irr_atlas()
    assert torch.equal(irr1[idx], irr0[idx])
    keep = torch.nonzero(V.states() == g.STATE_VIGILANT).flatten()
    assert not torch.equal(irr1[keep], irr0[keep])
    V.poll_status()
