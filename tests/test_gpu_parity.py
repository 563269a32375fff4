"""CUDA path vs the FP64 oracle on the same seeded inputs, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import (REL, compare_rays, fp32_neighbourhood_spread, fp32_texel_spread, gpu_rays_by_probe,
                    lit_query_sample, masked_texels, patched, rel_err, run_oracle, to_dev)

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
    # query at 4096 seeded points: end to end against the oracle's atlas
    # (with the listed texels, if any, taken from the GPU's), and the query
    # kernel alone against the oracle's query of the GPU's own atlas
    pos, nrm, cam = synth.room_queries()
    E_ref = oracle.query(desc, st, patched(irr, gi, mi), patched(dist, gd, md), pos, nrm, cam)
    E = V.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy()
    e = rel_err(E, E_ref).max(-1)
    E_own = oracle.query(desc, states, gi.astype(np.float64), gd.astype(np.float64), pos, nrm, cam)
    e_own = rel_err(E, E_own).max(-1)
    _report("room query", n=len(e), max_rel=float(e.max()), own_atlas_max_rel=float(e_own.max()))
    assert e.max() <= REL and e_own.max() <= REL


def test_room_multiframe_hysteresis_parity(g):
    desc = synth.room_volume(hysteresis_irr=0.9, hysteresis_vis=0.8)
    frames = [0, 1, 2, 3]
    sc, V, (st, irr, dist, rays), per_frame = _room_case(g, desc, frames)
    assert np.array_equal(V.states().cpu().numpy(), st)
    flagged = 0
    mi = np.zeros(V.irr_atlas().shape[:3], dtype=bool)
    md = np.zeros(V.dist_atlas().shape[:3], dtype=bool)
    for k, f in enumerate(frames):
        rec, ids = per_frame[k]
        bad, err = compare_rays(rec, ids, rays[k])
        flagged += int(bad.sum())
        a, b = masked_texels(desc, desc.seed, f, bad, ids)
        mi |= a
        md |= b
        _report(f"multiframe rays f{f}", flagged=int(bad.sum()), max_rel=float(err[~bad].max()))
    assert flagged <= 8
    gi = V.irr_atlas().cpu().numpy()
    gd = V.dist_atlas().cpu().numpy()
    ei = rel_err(gi, irr).max(-1)
    ed = rel_err(gd, dist).max(-1)
    _report("multiframe texels", irr_max=float(ei[~mi].max()), dist_max=float(ed[~md].max()),
            masked_irr=int(mi.sum()), masked_dist=int(md.sum()))
    assert ei[~mi].max() <= REL and ed[~md].max() <= REL


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
    assert ei.max() <= REL and ed.max() <= REL
    # gamma 2 takes the query's general form (the specialised one serves gamma 5)
    pos, nrm, cam = synth.room_queries(n=2048)
    E_ref = oracle.query(desc, st, irr, dist, pos, nrm, cam)
    E = V.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy()
    eq = rel_err(E, E_ref).max(-1)
    _report("odd sizes query", n=len(eq), max_rel=float(eq.max()), over=int((eq > REL).sum()))
    assert eq.max() <= REL


@pytest.mark.parametrize("case", ["max_tiles", "max_rays_tf32x3"])
def test_maximum_sizes_parity(g, case):
    """The largest rays per probe (1024) and tiles (32 x 32 irradiance, 64 x
    64 distance interiors) a volume accepts: tiles too large for the
    register-tiled blend take the row kernel, whose probe group shrinks to
    fit its shared memory at this R; the 3xTF32 tensor-core blend at R = 1024
    walks 64 ray chunks per probe group."""
    sc = synth.room_scene(n_boxes=6)
    tiles = dict(irr_n=32, dist_n=64) if case == "max_tiles" else dict(irr_n=6, dist_n=14)
    desc = synth.VolumeDesc(origin=(2.0, 2.5, 1.5), spacing=(5.0, 4.0, 3.0), counts=(2, 2, 3),
                            rays_per_probe=1024, hysteresis_irr=0.5, hysteresis_vis=0.5, state_machine=0,
                            seed=41, **tiles)
    prec = g.BLEND_FP32 if case == "max_tiles" else g.BLEND_TF32X3
    L = synth.room_lights()
    st, irr, dist, rays = run_oracle(sc, L, desc, [2, 3])
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    V.update(S, L, 2, precision=prec)
    V.update(S, L, 3, precision=prec)
    assert np.array_equal(V.states().cpu().numpy(), st)
    ei = rel_err(V.irr_atlas().cpu().numpy(), irr).max(-1)
    ed = rel_err(V.dist_atlas().cpu().numpy(), dist).max(-1)
    pos, nrm, cam = synth.room_queries(n=2048)
    E_ref = oracle.query(desc, st, irr, dist, pos, nrm, cam)
    eq = rel_err(V.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy(), E_ref).max(-1)
    _report(f"maximum sizes {case}", irr_max=float(ei.max()), dist_max=float(ed.max()), query_max=float(eq.max()))
    assert ei.max() <= REL and ed.max() <= REL and eq.max() <= REL


@pytest.mark.parametrize("prec", ["BLEND_FP32", "BLEND_TF32"])
def test_no_active_probe(g, prec):
    """Degenerate volume: every probe inside one solid box sees only back
    faces, so classification turns all of them Off (Sec. 6.1) and the active
    list is empty; every later pass, the blend (SIMT or tensor-core) included,
    runs on zero probes, the atlases stay zero, and a query whose cage holds
    no active probe returns 0 (as the oracle does)."""
    sc = synth.solid_box((-1.0, -1.0, -1.0), (9.0, 9.0, 9.0))
    desc = synth.VolumeDesc(origin=(1.0, 1.0, 1.0), spacing=(2.0, 2.0, 2.0), counts=(4, 4, 4), rays_per_probe=64,
                            hysteresis_irr=0.9, hysteresis_vis=0.9, seed=17)
    L = synth.room_lights()
    st, irr, dist, _ = run_oracle(sc, L, desc, [0, 1])
    assert np.all(st == g.STATE_OFF)
    V = g.Volume(desc)
    S = g.Scene.from_arrays(sc)
    for f in range(3):
        V.update(S, L, f, precision=getattr(g, prec))
    torch.cuda.synchronize()
    V.poll_status()
    assert np.array_equal(V.states().cpu().numpy(), st)
    assert not V.irr_atlas().any() and not V.dist_atlas().any()
    pos, nrm, cam = synth.room_queries(n=256)
    E = V.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy()
    assert np.all(E == 0.0) and np.all(oracle.query(desc, st, irr, dist, pos, nrm, cam) == 0.0)


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
    assert e.max() <= REL


@pytest.fixture(scope="module")
def city_steady(g):
    """The benchmark's city volume run for 60 frames (hysteresis 0.97, per-frame
    rotation, multi-bounce through the previous atlas, per-texel thresholds),
    keeping, at frames 1, 5 and 59, the GPU's state before the update (the
    previous atlas the oracle's one-step update starts from) and after it."""
    sc = synth.city_scene()
    desc = synth.city_volume()
    L = synth.city_lights()
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    snaps = {}
    for f in range(60):
        if f in (1, 5, 59):
            prev = (V.states().cpu().numpy(), np.ascontiguousarray(V.irr_atlas().cpu().numpy(), dtype=np.float64),
                    np.ascontiguousarray(V.dist_atlas().cpu().numpy(), dtype=np.float64))
        V.update(S, L, f)
        if f in (1, 5, 59):
            rec, ids = V.ray_records()
            snaps[f] = dict(prev=prev, rec=rec.cpu().numpy(), ids=ids.cpu().numpy().astype(np.int64),
                            states=V.states().cpu().numpy(), irr=V.irr_atlas().cpu().numpy(),
                            dist=V.dist_atlas().cpu().numpy())
    torch.cuda.synchronize()
    V.poll_status()
    return sc, desc, L, S, V, snaps


@pytest.mark.parametrize("frame", [1, 5, 59])
def test_city_steady_state_one_step(g, city_steady, frame):
    """Steady-state frames of the benchmark workload: the oracle's one-step
    update of 256 seeded active probes, started from the GPU's own previous
    atlas and states, against the GPU's update of the same frame: per-ray
    records (shading reads the lit previous atlas), texels (hysteresis 0.97
    and the per-texel thresholds of Sec. 4.3), states."""
    sc, desc, L, S, V, snaps = city_steady
    sn = snaps[frame]
    st0, irr0, dist0 = sn["prev"]
    act = np.nonzero(st0 == oracle.VIGILANT)[0]
    sample = np.sort(np.random.default_rng(500 + frame).choice(act, 256, replace=False))
    st, irr, dist = st0.copy(), irr0.copy(), dist0.copy()
    rays = oracle.update(oracle.SceneHandle(sc), L, desc, frame, st, irr, dist, subset=sample, want_rays=True)
    assert np.array_equal(sn["states"], np.where(np.isin(np.arange(desc.n_probes), sample), st, sn["states"]))
    pos_of = {int(p): k for k, p in enumerate(sn["ids"])}
    rec = sn["rec"][[pos_of[int(p)] for p in sample]].astype(np.float64)
    bad, err = compare_rays(rec, np.arange(len(sample)), rays)
    # a flagged ray whose distance agrees hit the same surface: its radiance
    # differs through the previous-atlas query at the hit point.  Such a ray
    # is listed when that query is ill-conditioned there: the oracle's query
    # moves by more than half the bound when its inputs move by four FP32
    # ulps, the rounding the GPU's FP32 evaluation adds to them: the hit
    # position (formed as o + t w in FP32) over its 26 neighbours, or the
    # atlas values (the bilinear moments and mu^2) with seeded signs.  Its
    # radiance must then stay within the bound plus twice that spread; rays
    # whose distance differs are the grazing rays of the traversal
    grazing = bad & (err[..., 3] > REL)
    shade = bad & ~grazing
    spread = np.zeros(int(shade.sum()))
    if shade.any():
        pi_, ri = np.nonzero(shade)
        cx, cy, _ = desc.counts
        ijk = np.stack([sample[pi_] % cx, (sample[pi_] // cx) % cy, sample[pi_] // (cx * cy)], 1)
        o = np.asarray(desc.origin) + ijk * np.asarray(desc.spacing)
        w = oracle.frame_dirs(desc.seed, frame, desc.rays_per_probe)[ri]
        t, tri, _ = oracle.trace(oracle.SceneHandle(sc), o, w)
        x = o + t[:, None] * w
        v = sc.verts[sc.tris[tri]]
        n = np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0])
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        for k in range(len(x)):
            spread[k] = fp32_neighbourhood_spread(
                lambda P, N_: oracle.query(desc, st0, irr0, dist0, P, N_, x[k] - w[k]), x[k][None], n[k][None],
                1e-30, ulps=4)[0]
        spread = np.maximum(spread, fp32_texel_spread(desc, st0, irr0, dist0, x, n, x - w, draws=8))
    mi, md = masked_texels(desc, desc.seed, frame, bad, sample)
    ei = rel_err(sn["irr"][sample], irr[sample]).max(-1)
    ed = rel_err(sn["dist"][sample], dist[sample]).max(-1)
    mi, md = mi[sample], md[sample]
    _report(f"city one-step f{frame}", probes=len(sample), rays=bad.size, grazing=int(grazing.sum()),
            shade_listed=int(shade.sum()), shade_err=[float(e) for e in err[shade][:, :3].max(-1)],
            shade_spread=[float(e) for e in spread], ray_max_rel=float(err[~bad].max()),
            irr_max=float(ei[~mi].max()), dist_max=float(ed[~md].max()), masked_irr=int(mi.sum()),
            masked_dist=int(md.sum()))
    assert grazing.sum() <= max(2, int(1e-4 * bad.size))
    assert shade.sum() <= max(2, int(1e-3 * bad.size))
    assert np.all(spread > REL / 2)
    assert np.all(err[shade][:, :3].max(-1) <= REL + 2 * spread)
    assert ei[~mi].max() <= REL and ed[~md].max() <= REL


def test_city_full_1080p_query_own_atlas(g, city_steady):
    """The benchmark's query, every pixel of the 1920x1080 G-buffer, at frame 59,
    against the oracle's query of the GPU's own atlas and states."""
    sc, desc, L, S, V, snaps = city_steady
    cam = synth.city_camera()
    pos, nrm = S.raycast_gbuffer(cam.position, cam.forward, cam.up, cam.vfov_deg, cam.width, cam.height)
    E = V.query(pos, nrm, cam.position).cpu().numpy()
    st = V.states().cpu().numpy()
    gi = np.ascontiguousarray(V.irr_atlas().cpu().numpy(), dtype=np.float64)
    gd = np.ascontiguousarray(V.dist_atlas().cpu().numpy(), dtype=np.float64)
    P = pos.cpu().numpy().astype(np.float64)
    N_ = nrm.cpu().numpy().astype(np.float64)
    E_ref = oracle.query(desc, st, gi, gd, P, N_, cam.position)
    e = rel_err(E, E_ref).max(-1)
    worst = np.argsort(-e)[:5]
    _report("city 1080p query", pixels=len(e), lit=float(np.mean(np.any(E_ref > 0, 1))), max_rel=float(e.max()),
            over=int((e > REL).sum()), worst=[(int(i), float(e[i])) for i in worst])
    assert e.max() <= REL


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
    M_own = oracle.query_glossy(desc, V.states().cpu().numpy(), V.irr_atlas().cpu().numpy().astype(np.float64),
                                V.dist_atlas().cpu().numpy().astype(np.float64), pos, nrm, dirs)
    e_own = rel_err(M, M_own).max(-1)
    _report("room glossy", n=len(e), max_rel=float(e.max()), own_atlas_max_rel=float(e_own.max()))
    assert e.max() <= REL and e_own.max() <= REL
