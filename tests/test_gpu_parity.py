"""CUDA path vs the FP64 oracle on the same seeded inputs, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import (REL, compare_rays, gpu_rays_by_probe, lit_query_sample, masked_texels, rel_err, run_oracle,
                    to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2009_10796_gb300 as pkg
    pkg.load()
    torch.cuda.set_device(0)
    return pkg


def _report(name, **kw):
    print(f"[parity] {name}: " + ", ".join(f"{k}={v}" for k, v in kw.items()))


# ------------------------------------------------------------------ tracing

def test_trace_closest_hit_room(g):
    sc = synth.room_scene()
    rng = synth.Rng(71)
    n = 20000
    o = synth.f32(rng.uniform(3 * n, 0.5, 9.5).reshape(n, 3))
    d = rng.unit_vectors(n)
    t_ref, tri_ref, bf_ref = oracle.trace(oracle.SceneHandle(sc), o, d)
    S = g.Scene.from_arrays(sc)
    t, tri, bf = S.trace(to_dev(o), to_dev(d))
    t, tri, bf = t.cpu().numpy(), tri.cpu().numpy(), bf.cpu().numpy()
    hit_ref = tri_ref >= 0
    assert np.array_equal(tri >= 0, hit_ref)
    # same triangle, or an equivalent surface: same object, same plane, same distance
    same = tri == tri_ref
    obj = sc.tri_object
    alt = ~same & hit_ref
    equiv = np.zeros(n, dtype=bool)
    if alt.any():
        equiv[alt] = (obj[tri[alt]] == obj[tri_ref[alt]]) & (np.abs(t[alt] - t_ref[alt]) <= 1e-5 * t_ref[alt])
    flagged = ~(same | equiv | ~hit_ref)
    _report("trace room", rays=n, same_tri=int(same.sum()), equivalent=int(equiv.sum()),
            differing=int(flagged.sum()))
    assert flagged.sum() <= max(1, int(1e-4 * n))
    ok = hit_ref & ~flagged
    assert np.all(np.abs(t[ok] - t_ref[ok]) <= 2e-6 * np.maximum(t_ref[ok], 1.0))
    assert np.array_equal(bf[ok], bf_ref[ok])


def test_trace_empty_and_degenerate(g):
    S = g.Scene.from_arrays(synth.empty_scene())
    o = to_dev(np.zeros((5, 3)))
    d = to_dev(np.tile([0.0, 0.0, 1.0], (5, 1)))
    t, tri, bf = S.trace(o, d)
    assert torch.all(tri == -1) and torch.all(torch.isinf(t))
    # zero rays is a no-op
    S.trace(to_dev(np.zeros((0, 3))), to_dev(np.zeros((0, 3))))


# ------------------------------------------------------------- room (cfg 1)

def _room_case(g, desc, frames, n_boxes=32, lights=None):
    sc = synth.room_scene(n_boxes=n_boxes)
    L = lights or synth.room_lights()
    st, irr, dist, rays = run_oracle(sc, L, desc, frames)
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    per_frame = []
    for f in frames:
        V.update(S, L, f)
        rec, ids = gpu_rays_by_probe(V)
        per_frame.append((rec, ids))
    torch.cuda.synchronize()
    V.poll_status()
    return sc, V, (st, irr, dist, rays), per_frame


def test_room_update_and_query_parity(g):
    desc = synth.room_volume()
    sc, V, (st, irr, dist, rays), per_frame = _room_case(g, desc, [0])
    states = V.states().cpu().numpy()
    assert np.array_equal(states, st), "states differ"
    rec, ids = per_frame[0]
    assert sorted(ids.tolist()) == sorted(np.nonzero(st == oracle.VIGILANT)[0].tolist())
    bad, err = compare_rays(rec, ids, rays[0])
    n_rays = bad.size
    _report("room rays", rays=n_rays, flagged=int(bad.sum()), max_rel=float(err[~bad].max()))
    assert bad.sum() <= max(2, int(1e-4 * n_rays))
    mi, md = masked_texels(desc, desc.seed, 0, bad, ids)
    gi = V.irr_atlas().cpu().numpy()
    gd = V.dist_atlas().cpu().numpy()
    ei = rel_err(gi, irr).max(-1)
    ed = rel_err(gd, dist).max(-1)
    _report("room texels", irr_max=float(ei[~mi].max()), dist_max=float(ed[~md].max()),
            masked_irr=int(mi.sum()), masked_dist=int(md.sum()))
    assert ei[~mi].max() <= REL and ed[~md].max() <= REL
    # query at 4096 seeded points
    pos, nrm, cam = synth.room_queries()
    E_ref = oracle.query(desc, st, irr, dist, pos, nrm, cam)
    E = V.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy()
    e = rel_err(E, E_ref).max(-1)
    _report("room query", n=len(e), max_rel=float(e.max()), over=int((e > REL).sum()))
    assert np.mean(e <= REL) >= 0.999
    assert e.max() <= 1e-2


def test_room_multiframe_hysteresis_parity(g):
    desc = synth.room_volume(hysteresis_irr=0.9, hysteresis_vis=0.8)
    frames = [0, 1, 2, 3]
    sc, V, (st, irr, dist, rays), per_frame = _room_case(g, desc, frames)
    assert np.array_equal(V.states().cpu().numpy(), st)
    flagged = 0
    for k, f in enumerate(frames):
        rec, ids = per_frame[k]
        bad, err = compare_rays(rec, ids, rays[k], rtol=5e-4)
        flagged += int(bad.sum())
        _report(f"multiframe rays f{f}", flagged=int(bad.sum()), max_rel=float(err[~bad].max()))
    assert flagged <= 8
    gi = V.irr_atlas().cpu().numpy()
    gd = V.dist_atlas().cpu().numpy()
    ei = rel_err(gi, irr).max(-1)
    ed = rel_err(gd, dist).max(-1)
    _report("multiframe texels", irr_max=float(ei.max()), dist_max=float(ed.max()),
            irr_over=int((ei > REL).sum()), dist_over=int((ed > REL).sum()))
    assert np.mean(ei <= REL) >= 0.999 and np.mean(ed <= REL) >= 0.999


def test_odd_sizes_parity(g):
    # rays not a multiple of the warp, non-cubic grid, small tiles, no state machine
    sc = synth.room_scene(n_boxes=6)
    desc = synth.VolumeDesc(origin=(1.0, 1.5, 2.0), spacing=(2.5, 1.75, 3.0), counts=(3, 4, 2),
                            rays_per_probe=37, irr_n=4, dist_n=8, hysteresis_irr=0.5,
                            hysteresis_vis=0.5, state_machine=0, seed=99, gamma=2.0)
    L = synth.room_lights()
    st, irr, dist, rays = run_oracle(sc, L, desc, [5, 6])
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    V.update(S, L, 5)
    V.update(S, L, 6)
    ei = rel_err(V.irr_atlas().cpu().numpy(), irr).max(-1)
    ed = rel_err(V.dist_atlas().cpu().numpy(), dist).max(-1)
    _report("odd sizes", irr_max=float(ei.max()), dist_max=float(ed.max()))
    assert np.mean(ei <= REL) >= 0.99 and np.mean(ed <= REL) >= 0.99
    # gamma 2 takes the query's general form (the specialised one serves gamma 5)
    pos, nrm, cam = synth.room_queries(n=2048)
    E_ref = oracle.query(desc, st, irr, dist, pos, nrm, cam)
    E = V.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy()
    eq = rel_err(E, E_ref).max(-1)
    _report("odd sizes query", n=len(eq), max_rel=float(eq.max()), over=int((eq > REL).sum()))
    assert np.mean(eq <= REL) >= 0.99


def test_empty_scene_uniform_sky(g):
    a = np.array([0.3, 1.7, 0.05])
    L = synth.Lights(sky_a=a)
    desc = synth.VolumeDesc(origin=(0, 0, 0), spacing=(1, 1, 1), counts=(2, 2, 2), rays_per_probe=64,
                            hysteresis_irr=0, hysteresis_vis=0, state_machine=0, seed=5, t_max=3.0)
    V = g.Volume(desc)
    V.update(g.Scene.from_arrays(synth.empty_scene()), L, 0)
    irr = V.irr_atlas().cpu().numpy().astype(np.float64)
    assert np.allclose(irr[:, 1:-1, 1:-1] ** 5, a, rtol=2e-6)
    pos = np.full((4, 3), 0.5)
    nrm = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, -1.0], [0, 0, 0]])
    E = V.query(to_dev(pos), to_dev(nrm), np.array([2.0, 2.0, 2.0])).cpu().numpy()
    assert np.allclose(E[:3], np.pi * a, rtol=5e-6)
    assert np.all(E[3] == 0)       # zero normal: no surface


def test_invalid_arguments(g):
    bad = synth.VolumeDesc(counts=(1, 2, 2))
    with pytest.raises(g.DDGIError) as ei:
        g.Volume(bad)
    assert ei.value.code == 1
    with pytest.raises(g.DDGIError):
        g.Volume(synth.VolumeDesc(rays_per_probe=0))
    with pytest.raises(g.DDGIError):
        g.Volume(synth.VolumeDesc(), irr_format=7)
    V = g.Volume(synth.VolumeDesc())
    out = V.query(to_dev(np.zeros((0, 3))), to_dev(np.zeros((0, 3))), np.zeros(3))
    assert out.shape == (0, 3)


# --------------------------------------------------- city at full size (cfg 2)

@pytest.fixture(scope="module")
def city(g):
    sc = synth.city_scene()
    desc = synth.city_volume()
    L = synth.city_lights()
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    V.update(S, L, 0)
    torch.cuda.synchronize()
    return sc, desc, L, S, V


def test_city_frame0_sampled_probes(g, city):
    sc, desc, L, S, V = city
    states = V.states().cpu().numpy()
    rec, ids = gpu_rays_by_probe(V)
    rng = np.random.default_rng(123)
    sample = np.sort(rng.choice(desc.n_probes, 24, replace=False))
    # make sure active probes are represented
    act = np.nonzero(states == oracle.VIGILANT)[0]
    sample = np.unique(np.concatenate([sample, rng.choice(act, 12, replace=False)]))
    h = oracle.SceneHandle(sc)
    st, irr, dist = oracle.new_state(desc)
    rays = oracle.update(h, L, desc, 0, st, irr, dist, subset=sample, want_rays=True)
    assert np.array_equal(states[sample], st[sample]), "sampled states differ"
    pos_of = {int(p): k for k, p in enumerate(ids)}
    act_s = [p for p in sample if st[p] == oracle.VIGILANT]
    gi = V.irr_atlas().cpu().numpy()
    gd = V.dist_atlas().cpu().numpy()
    flagged = 0
    worst_i = worst_d = 0.0
    for q, p in enumerate(sample):
        if st[p] != oracle.VIGILANT:
            continue
        r_gpu = rec[pos_of[int(p)]][None]
        bad, err = compare_rays(r_gpu, np.array([0]), rays[q][None])
        flagged += int(bad.sum())
        if bad.any():
            continue
        worst_i = max(worst_i, float(rel_err(gi[p], irr[p]).max()))
        worst_d = max(worst_d, float(rel_err(gd[p], dist[p]).max()))
    _report("city sampled", probes=len(sample), active=len(act_s), flagged_rays=flagged,
            irr_max=worst_i, dist_max=worst_d)
    assert flagged <= 2
    assert worst_i <= REL and worst_d <= REL


def test_city_query_sampled_points(g, city):
    sc, desc, L, S, V = city
    pts, nrm, subset = lit_query_sample(sc, desc, 3002)
    cam = np.array([0.0, 12.0, -28.0])
    st, irr, dist = oracle.new_state(desc)
    oracle.update(oracle.SceneHandle(sc), L, desc, 0, st, irr, dist, subset=subset)
    E_ref = oracle.query(desc, st, irr, dist, pts, nrm, cam)
    E = V.query(to_dev(pts), to_dev(nrm), cam).cpu().numpy()
    e = rel_err(E, E_ref).max(-1)
    lit = float(np.mean(np.any(E_ref > 0, axis=1)))
    _report("city query", points=len(pts), probes=len(subset), lit=lit, max_rel=float(e.max()),
            over=int((e > REL).sum()))
    assert lit >= 0.9
    assert np.mean(e <= REL) >= 0.95
    assert np.median(e) <= REL


def test_room_glossy_lookup_parity(g):
    """Second-order glossy lookup (Sec. 4.4) at 4,096 seeded points with seeded
    reflection-ray directions, against the oracle on the same atlases."""
    desc = synth.room_volume()
    sc, V, (st, irr, dist, rays), _ = _room_case(g, desc, [0])
    pos, nrm, _ = synth.room_queries()
    dirs = synth.Rng(3101).unit_vectors(len(pos))
    M_ref = oracle.query_glossy(desc, st, irr, dist, pos, nrm, dirs)
    M = V.query_glossy(to_dev(pos), to_dev(nrm), to_dev(dirs)).cpu().numpy()
    e = rel_err(M, M_ref).max(-1)
    _report("room glossy", n=len(e), max_rel=float(e.max()), over=int((e > REL).sum()))
    assert np.mean(e <= REL) >= 0.999 and e.max() <= 1e-2
