"""Boundary calls: volume save / load, the texel gradient of the query
(ddgi_query_backward) against the oracle's, and the 16-byte rule for caller
device buffers."""
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


def _raw(V):
    return [V.states(), V.irr_raw(), V.dist_raw(), V._get(3, V.n_probes * 16)]


@pytest.mark.parametrize("optimizer", [0, 5])
def test_save_load_round_trip_then_update(g, optimizer):
    """A volume restored from a blob continues exactly as the saved one: the
    same states, atlases and offsets after the load, and after one more update."""
    sc = synth.room_scene()
    L = synth.room_lights()
    desc = synth.room_volume(hysteresis_irr=0.9, hysteresis_vis=0.8, optimizer_iters=optimizer)
    S = g.Scene.from_arrays(sc)
    A = g.Volume(desc)
    for f in range(3):
        A.update(S, L, f)
    blob = A.save()
    B = g.Volume(desc)
    B.load(blob)
    for a, b in zip(_raw(A), _raw(B)):
        assert torch.equal(a, b)
    A.update(S, L, 3)
    B.update(S, L, 3)
    torch.cuda.synchronize()
    for a, b in zip(_raw(A), _raw(B)):
        assert torch.equal(a, b)
    # a blob's size is fixed by the layout; saving twice gives the same bytes
    assert len(A.save()) == len(blob) and A.save() == A.save()


def test_load_rejects_foreign_and_damaged_blobs(g):
    desc = synth.room_volume()
    A = g.Volume(desc)
    blob = A.save()
    other = g.Volume(synth.room_volume(counts=(8, 8, 4)))
    with pytest.raises(g.DDGIError) as e:
        other.load(blob)
    assert e.value.code == 1 and "counts" in str(e.value)
    with pytest.raises(g.DDGIError):
        g.Volume(synth.room_volume(spacing=(1.0, 1.25, 1.25))).load(blob)
    with pytest.raises(g.DDGIError):
        g.Volume(desc, irr_format=g.IRR_FP16).load(blob)
    bad = bytearray(blob)
    bad[-5] ^= 0x40                                    # one bit of the payload
    with pytest.raises(g.DDGIError) as e:
        A.load(bytes(bad))
    assert "checksum" in str(e.value)
    with pytest.raises(g.DDGIError):
        A.load(b"NOTAVOLUME" + blob[10:])
    with pytest.raises(g.DDGIError):
        A.load(blob[:-1])
    A.load(blob)                                       # the volume is still usable


def test_misaligned_device_buffers_are_rejected(g):
    """The check runs on the host before any launch."""
    V = g.Volume(synth.room_volume())
    buf = torch.zeros(3 * 65, dtype=torch.float32, device="cuda")
    pos = buf[1:193].view(64, 3)                       # 4 bytes past a 16-byte boundary
    nrm = torch.zeros(64, 3, dtype=torch.float32, device="cuda")
    with pytest.raises(g.DDGIError) as e:
        V.query(pos, nrm, np.zeros(3))
    assert e.value.code == 1 and "16-byte" in str(e.value)
    with pytest.raises(g.DDGIError):
        V.query(nrm, nrm, np.zeros(3), out=torch.zeros(3 * 65, device="cuda")[1:193].view(64, 3))
    with pytest.raises(g.DDGIError):
        V.set_buffer(2, torch.zeros(V.n_probes + 1, dtype=torch.uint8, device="cuda")[1:])


def _texel_grad_case(g, optimizer=0):
    sc = synth.room_scene()
    L = synth.room_lights()
    desc = synth.room_volume(hysteresis_irr=0.5, hysteresis_vis=0.5, optimizer_iters=optimizer)
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    for f in range(2):
        V.update(S, L, f)
    pos, nrm, cam = synth.room_queries(n=2048)
    dE = synth.f32(synth.Rng(77).uniform(3 * len(pos), 0.5, 1.5).reshape(-1, 3))
    st = V.states().cpu().numpy()
    gi = V.irr_atlas().cpu().numpy().astype(np.float64)
    gd = V.dist_atlas().cpu().numpy().astype(np.float64)
    off = np.ascontiguousarray(V.offsets().cpu().numpy().astype(np.float64)) if optimizer else None
    return desc, V, pos, nrm, cam, dE, st, gi, gd, off


@pytest.mark.parametrize("optimizer", [0, 5])
@pytest.mark.parametrize("fold", [False, True])
def test_query_backward_matches_oracle_texel_gradient(g, fold, optimizer):
    """dLoss/d(irradiance texels) of the query at 2,048 points on the GPU's own
    atlas, against the oracle's (pinned to FP64 central differences).  With
    positive dLoss/dE every contribution to a texel has one sign, so the
    comparison is element by element at the parity tolerance."""
    desc, V, pos, nrm, cam, dE, st, gi, gd, off = _texel_grad_case(g, optimizer)
    G = V.query_backward(to_dev(pos), to_dev(nrm), cam, to_dev(dE), fold_borders=fold).cpu().numpy()
    R = oracle.query_texel_grad(desc, st, gi, gd, pos, nrm, cam, dE, fold=fold, offsets=off)
    e = rel_err(G, R)
    print(f"[texel grad] fold {fold}, optimizer {optimizer}: nonzero {int((R != 0).sum())} of {R.size}, "
          f"max rel {e.max():.2e}")
    assert (R != 0).sum() > 0.1 * R.size
    assert e.max() <= REL


def test_probe_query_autograd(g):
    """ProbeQuery: E as a function of the atlas tensor; its backward is
    ddgi_query_backward's gradient (the unused lane zero), and its forward is
    the volume's query."""
    desc, V, pos, nrm, cam, dE, st, gi, gd, off = _texel_grad_case(g)
    N = desc.irr_n + 2
    atlas = V.irr_raw().view(torch.float32).view(V.n_probes, N, N, 4).clone().requires_grad_(True)
    P, N_ = to_dev(pos), to_dev(nrm)
    E = g.ProbeQuery.apply(atlas, V, P, N_, cam)
    assert torch.equal(E.detach(), V.query(P, N_, cam))
    (E * to_dev(dE)).sum().backward()
    G = V.query_backward(P, N_, cam, to_dev(dE))
    assert torch.all(atlas.grad[..., 3] == 0)
    assert torch.allclose(atlas.grad[..., :3], G, rtol=1e-5, atol=1e-7 * float(G.abs().max()))


def test_measure_l2_read(g):
    """The L2 read-rate helper runs on a resident buffer, reports a rate
    between the HBM copy rate's order and a bound no cache reaches, and
    rejects misaligned or odd-sized buffers before launching."""
    buf = torch.arange(4 << 20, dtype=torch.int32, device="cuda")     # 16 MiB
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    g.measure_l2_read(buf, 2, sink)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    g.measure_l2_read(buf, 8, sink)
    e1.record()
    torch.cuda.synchronize()
    gbs = buf.numel() * 4 * 8 / (e0.elapsed_time(e1) * 1e-3) / 1e9
    print(f"[l2 read] {gbs:.0f} GB/s")
    assert 1000.0 < gbs < 200000.0
    with pytest.raises(g.DDGIError, match="16-byte"):
        g.measure_l2_read(buf[1:5], 1, sink)
    with pytest.raises(g.DDGIError, match="multiple of 16"):
        g.measure_l2_read(buf[:3], 1, sink)


def test_overlapped_launches_match_ordinary_launches(g, monkeypatch):
    """The frame's kernels as programmatic dependent launches (the default)
    give the same bits as ordinary launches (DDGI_NO_PDL=1): a volume's states,
    atlases and query after four updates, and a tracking cascade replayed as a
    CUDA graph."""
    sc = synth.room_scene(n_boxes=12)
    L = synth.room_lights()
    S = g.Scene.from_arrays(sc)
    desc = synth.room_volume(hysteresis_irr=0.9, hysteresis_vis=0.8)
    pos, nrm, _ = synth.room_queries(n=4096)
    P, N_ = to_dev(pos), to_dev(nrm)
    cam = np.array([2.0, 1.5, 2.5])
    common = dict(rays_per_probe=32, hysteresis_irr=0.5, hysteresis_vis=0.5, seed=4242)
    fine = synth.VolumeDesc(origin=(2.0, 2.0, 2.0), spacing=(0.75, 0.75, 0.75), counts=(6, 6, 6), tracking=1,
                            **common)
    coarse = synth.VolumeDesc(origin=(0.625, 0.625, 0.625), spacing=(1.25, 1.25, 1.25), counts=(8, 8, 8),
                              **common)

    def run(ordinary):
        if ordinary:
            monkeypatch.setenv("DDGI_NO_PDL", "1")
        else:
            monkeypatch.delenv("DDGI_NO_PDL", raising=False)
        V = g.Volume(desc)
        C = g.Cascade([fine, coarse])
        for f in range(4):
            V.update(S, L, f)
            C.update(S, L, f, synth.f32([3.0 + 0.55 * f, 4.0, 5.0 - 0.2 * f]), use_graph=True)
        E = V.query(P, N_, cam)
        torch.cuda.synchronize()
        return _raw(V) + [E] + [C.states(k) for k in range(2)] + [C.buffer(k, b) for k in range(2) for b in (0, 1)]

    overlapped = run(False)
    ordinary = run(True)
    monkeypatch.delenv("DDGI_NO_PDL", raising=False)
    for a, b in zip(overlapped, ordinary):
        assert torch.equal(a, b)
