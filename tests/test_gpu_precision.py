"""Reduced-precision atlas storage against the FP64 oracle.

Tolerances come from the formats: FP16 rounds to nearest with 11 significant
bits (relative error <= 2^-11); RGB9E5 shares one exponent chosen from the
largest channel, so each channel's error is <= 2^-9 of the texel's largest
channel.  Both add the FP32 parity tolerance of the arithmetic itself.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import REL, compare_rays, gpu_rays_by_probe, rel_err, run_oracle, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2009_10796_gb300 as pkg
    pkg.load()
    torch.cuda.set_device(0)
    return pkg


def _decode_rgb9e5(words):
    w = words.astype(np.int64) & 0xFFFFFFFF
    e = (w >> 27) - 15 - 9
    s = np.ldexp(1.0, e)
    return np.stack([(w & 511) * s, ((w >> 9) & 511) * s, ((w >> 18) & 511) * s], axis=-1)


def _room(g, irr_format, dist_format):
    sc = synth.room_scene()
    L = synth.room_lights()
    desc = synth.room_volume()
    st, irr, dist, _ = run_oracle(sc, L, desc, [0])
    V = g.Volume(desc, irr_format=irr_format, dist_format=dist_format)
    V.update(g.Scene.from_arrays(sc), L, 0)
    torch.cuda.synchronize()
    assert np.array_equal(V.states().cpu().numpy(), st)
    return desc, st, irr, dist, V


def test_fp16_irradiance_and_distance_storage(g):
    desc, st, irr, dist, V = _room(g, g.IRR_FP16, g.DIST_FP16)
    gi = V.irr_atlas().cpu().numpy().astype(np.float64)
    gd = V.dist_atlas().cpu().numpy().astype(np.float64)
    tol = 2.0 ** -11 + REL
    ei = rel_err(gi, irr)
    ed = rel_err(gd, dist)
    print(f"[precision] fp16 irr max rel {ei.max():.2e}, dist max rel {ed.max():.2e}")
    assert ei.max() <= tol and ed.max() <= tol
    # the stored value is the FP16 rounding of an FP32 result: never worse than half an ulp + FP32 error
    pos, nrm, cam = synth.room_queries()
    E_ref = oracle.query(desc, st, irr, dist, pos, nrm, cam)
    E = V.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy()
    eq = rel_err(E, E_ref).max(-1)
    # decode raises the encoded value to the 5th power: relative error x5
    print(f"[precision] fp16 query max rel {eq.max():.2e}, median {np.median(eq):.2e}")
    assert np.median(eq) <= 5 * 2.0 ** -11 and np.mean(eq <= 1e-2) >= 0.999


def test_rgb9e5_irradiance_storage(g):
    desc, st, irr, dist, V = _room(g, g.IRR_RGB9E5, g.DIST_FP32)
    words = V.irr_raw().view(torch.int32).cpu().numpy().reshape(irr.shape[:-1])
    gi = _decode_rgb9e5(words)
    mx = np.abs(irr).max(-1, keepdims=True)
    err = np.abs(gi - irr)
    bound = 2.0 ** -9 * mx + REL * np.maximum(mx, 1e-3 * np.abs(irr).max())
    print(f"[precision] rgb9e5 max err / bound {np.max(err / np.maximum(bound, 1e-30)):.3f}")
    assert np.all(err <= bound)
    # the distance atlas stays FP32
    assert rel_err(V.dist_atlas().cpu().numpy(), dist).max() <= REL
    pos, nrm, cam = synth.room_queries()
    E_ref = oracle.query(desc, st, irr, dist, pos, nrm, cam)
    E = V.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy()
    eq = rel_err(E, E_ref).max(-1)
    print(f"[precision] rgb9e5 query max rel {eq.max():.2e}, median {np.median(eq):.2e}")
    assert np.median(eq) <= 5 * 2.0 ** -9 and np.mean(eq <= 5e-2) >= 0.999


# ------------------------------------------------------ tensor-core blend

def _threshold_straddlers(sc, L, desc, tol):
    """Texels whose frame-1 change (encoded domain) lies within `tol` of a
    per-texel threshold: reduced precision may legitimately take the other
    branch there.  The change is the oracle's: frame 1 rerun with hysteresis 0
    gives the new value each texel blends in."""
    h = oracle.SceneHandle(sc)
    st, irr0, dist0 = oracle.new_state(desc)
    oracle.update(h, L, desc, 0, st, irr0, dist0)
    d0 = synth.VolumeDesc(**{**desc.__dict__, "hysteresis_irr": 0.0, "hysteresis_vis": 0.0})
    st1, irr1, dist1 = st.copy(), irr0.copy(), dist0.copy()
    oracle.update(h, L, d0, 1, st1, irr1, dist1)
    delta = np.abs(irr1 - irr0).max(-1)
    near = (np.abs(delta - desc.thr_low) < tol) | (np.abs(delta - desc.thr_high) < tol)
    return np.broadcast_to(near[..., None], irr0.shape)


_TC_MODES = {"tf32": ("BLEND_TF32", 1e-3, 1e-3), "bf16": ("BLEND_BF16", 1e-3, 3e-3),
             "tf32x3": ("BLEND_TF32X3", REL, 1e-5)}


@pytest.mark.parametrize("mode", sorted(_TC_MODES))
@pytest.mark.parametrize("hysteresis", [0.0, 0.9])
def test_tensor_core_blend_against_oracle(g, mode, hysteresis):
    """Irradiance in TF32 / BF16 with FP32-accurate distance moments, or every
    contraction FP32-accurate (TF32X3): texels within 1e-3 (TF32X3: the 1e-4
    parity bound) of the FP64 oracle in the stored domain, over two frames
    (multi-bounce).  With hysteresis, texels whose change sits within the
    format's error of a threshold are excluded and counted."""
    name, tol, band = _TC_MODES[mode]
    prec = getattr(g, name)
    sc = synth.room_scene()
    L = synth.room_lights()
    desc = synth.room_volume(hysteresis_irr=hysteresis, hysteresis_vis=0.8 * hysteresis)
    st, irr, dist, _ = run_oracle(sc, L, desc, [0, 1])
    V = g.Volume(desc)
    S = g.Scene.from_arrays(sc)
    V.update(S, L, 0, precision=prec)
    V.update(S, L, 1, precision=prec)
    torch.cuda.synchronize()
    V.poll_status()
    assert np.array_equal(V.states().cpu().numpy(), st)
    gi = V.irr_atlas().cpu().numpy().astype(np.float64)
    gd = V.dist_atlas().cpu().numpy().astype(np.float64)
    ei = rel_err(gi, irr)
    ed = rel_err(gd, dist)
    skip = np.zeros_like(ei, dtype=bool)
    if hysteresis > 0:
        # band: twice the largest encoded-value error the format showed without thresholds
        skip = _threshold_straddlers(sc, L, desc, tol=band)
    print(f"[precision] {mode} blend (hysteresis {hysteresis}): irr max rel {ei[~skip].max():.2e} "
          f"(median {np.median(ei):.2e}), dist max rel {ed.max():.2e} (median {np.median(ed):.2e}), "
          f"threshold-straddling texels excluded: {int(skip[..., 0].sum())} of {skip[..., 0].size}")
    assert ei[~skip].max() <= tol and ed.max() <= tol
    assert skip[..., 0].mean() < 0.02
    # moments of one weighted distribution: the variance stays non-negative
    mu, mu2 = gd[..., 0], gd[..., 1]
    assert np.all(mu2 >= mu * mu * (1 - 1e-6) - 1e-9)
    pos, nrm, cam = synth.room_queries()
    E_ref = oracle.query(desc, st, irr, dist, pos, nrm, cam)
    E = V.query(to_dev(pos), to_dev(nrm), cam).cpu().numpy()
    eq = rel_err(E, E_ref).max(-1)
    print(f"[precision] {mode} blend query max rel {eq.max():.2e}, median {np.median(eq):.2e}")
    assert np.median(eq) <= 1e-3
    if mode == "tf32x3":
        # the query arithmetic on the GPU's own atlas meets the parity bound
        # at every point.  End to end, against the oracle's atlas with the
        # threshold-straddling texels (excluded above) taken from the GPU:
        # points where that oracle query moves by more than half the bound
        # when every texel moves by its own error in this run with a seeded
        # random sign are listed (a Chebyshev weight where mu2 - mu^2 nearly
        # cancels amplifies texel errors that are themselves within the
        # bound) and held to the bound plus twice that sensitivity
        E_own = oracle.query(desc, st, gi, gd, pos, nrm, cam)
        eo = rel_err(E, E_own).max(-1)
        irr_r = np.where(skip, gi, irr)
        eq = rel_err(E, oracle.query(desc, st, irr_r, dist, pos, nrm, cam)).max(-1)
        rng = np.random.default_rng(7)
        irr_p = irr_r + np.abs(gi - irr_r) * rng.choice([-1.0, 1.0], size=irr.shape)
        dist_p = dist + np.abs(gd - dist) * rng.choice([-1.0, 1.0], size=dist.shape)
        sens = rel_err(oracle.query(desc, st, irr_p, dist_p, pos, nrm, cam),
                       oracle.query(desc, st, irr_r, dist, pos, nrm, cam)).max(-1)
        listed = sens > REL / 2
        print(f"[precision] tf32x3 query on its own atlas max rel {eo.max():.2e}; against the oracle with "
              f"{int(skip[..., 0].sum())} straddling texels patched: listed {int(listed.sum())} of {len(eq)} points "
              f"(texel sensitivity {sens.max():.2e} max), max rel on the rest {eq[~listed].max():.2e}")
        assert eo.max() <= REL
        assert listed.mean() <= 1e-3
        assert eq[~listed].max() <= REL
        assert np.all(eq[listed] <= REL + 2 * sens[listed])


@pytest.mark.parametrize("mode", ["tf32", "bf16", "tf32x3"])
def test_tensor_core_blend_matches_fp32_at_scale(g, mode):
    """City workload, same rays: the tensor-core blend against the FP32 SIMT
    blend, every active probe.  TF32 stays within 1e-3 relative in the stored
    domain; BF16 (8-bit mantissas on weights and radiance) within 2e-3, with
    99.9% of texels within 1e-3; the FP32-accurate TF32X3 split within 1e-5."""
    sc = synth.city_scene()
    L = synth.city_lights()
    desc = synth.city_volume()
    S = g.Scene.from_arrays(sc)
    A = g.Volume(desc)
    B = g.Volume(desc)
    A.update(S, L, 0)
    B.update(S, L, 0, precision=getattr(g, _TC_MODES[mode][0]))
    torch.cuda.synchronize()
    assert torch.equal(A.states(), B.states())
    act = (A.states() == g.STATE_VIGILANT).cpu().numpy()
    ia = A.irr_atlas().cpu().numpy()[act]
    ib = B.irr_atlas().cpu().numpy()[act]
    da = A.dist_atlas().cpu().numpy()[act]
    db = B.dist_atlas().cpu().numpy()[act]
    ei = rel_err(ib, ia)
    ed = rel_err(db, da)
    print(f"[precision] city {mode} vs fp32: irr max {ei.max():.2e} (99.9% {np.quantile(ei, 0.999):.2e}), "
          f"dist max {ed.max():.2e}, probes {act.sum()}")
    assert ed.max() <= 1e-3
    if mode == "tf32":
        assert ei.max() <= 1e-3
    elif mode == "tf32x3":
        assert ei.max() <= 1e-5 and ed.max() <= 1e-5
    else:
        assert ei.max() <= 2e-3 and np.quantile(ei, 0.999) <= 1e-3


# ------------------------------------------- city scale against the oracle

def _window_probes(desc, pos, nrm):
    """Probes within one cell of the cells of the given surface points (4 x 4
    x 4 per cell: the self-shadow bias moves a point by less than a cell, so
    every cage the query reads lies inside)."""
    org, sp, cnt = np.asarray(desc.origin), np.asarray(desc.spacing), np.asarray(desc.counts)
    cells = np.unique(np.clip(np.floor((pos - org) / sp), 0, cnt - 2).astype(np.int64), axis=0)
    off = np.stack(np.meshgrid(*[np.arange(-1, 3)] * 3, indexing="ij"), -1).reshape(-1, 3)
    q = (cells[:, None, :] + off[None]).reshape(-1, 3)
    q = q[np.all((q >= 0) & (q < cnt), axis=1)]
    return np.unique(q[:, 0] + cnt[0] * (q[:, 1] + cnt[1] * q[:, 2]))


@pytest.fixture(scope="module")
def city_ref(g):
    """The 16,384-probe city workload at frame 0 against the oracle's one-step
    update: 256 seeded active probes for texels, and the probes around the
    cages of a 256 x 256 window at the centre of the 1920 x 1080 G-buffer
    (65,536 pixels) for queries.  Probes whose classification flips within
    FP32 rounding are listed (pixels whose cages could read them are left
    out), and probes with a ray that grazes an edge within FP32 rounding are
    left out of the texel comparisons (frame-0 rays do not depend on the
    atlas formats)."""
    sc = synth.city_scene()
    desc = synth.city_volume()
    L = synth.city_lights()
    S = g.Scene.from_arrays(sc)
    A = g.Volume(desc)
    A.update(S, L, 0)
    torch.cuda.synchronize()
    states = A.states().cpu().numpy()
    rec, ids = gpu_rays_by_probe(A)
    act = np.nonzero(states == oracle.VIGILANT)[0]
    sample = np.sort(np.random.default_rng(124).choice(act, 256, replace=False))
    cam = synth.city_camera()
    P, N = S.raycast_gbuffer(cam.position, cam.forward, cam.up, cam.vfov_deg, cam.width, cam.height)
    P = P.cpu().numpy().reshape(cam.height, cam.width, 3)[412:668, 832:1088].reshape(-1, 3)
    N = N.cpu().numpy().reshape(cam.height, cam.width, 3)[412:668, 832:1088].reshape(-1, 3)
    hit = np.any(N != 0, axis=1)
    pts, nrm = P[hit].astype(np.float64), N[hit].astype(np.float64)
    subset = np.union1d(sample, _window_probes(desc, pts, nrm))
    st, irr, dist = oracle.new_state(desc)
    rays = oracle.update(oracle.SceneHandle(sc), L, desc, 0, st, irr, dist, subset=subset, want_rays=True)
    flips = subset[states[subset] != st[subset]]
    assert len(flips) <= max(2, int(1e-3 * len(subset))), f"classification differs at {flips}"
    if len(flips):   # pixels whose cage neighbourhood holds a flipped probe
        near = np.array([np.intersect1d(_window_probes(desc, x[None], None), flips).size > 0 for x in pts])
        pts, nrm = pts[~near], nrm[~near]
    pos_of = {int(p): k for k, p in enumerate(ids)}
    row = {int(p): q for q, p in enumerate(subset)}
    clean = []
    for p in sample:
        if st[p] != oracle.VIGILANT or p in flips:
            continue
        bad, _ = compare_rays(rec[pos_of[int(p)]][None], np.array([0]), rays[row[int(p)]][None])
        if not bad.any():
            clean.append(int(p))
    camp = np.asarray(cam.position, dtype=np.float64)
    E_ref = oracle.query(desc, st, irr, dist, pts, nrm, camp)
    print(f"[precision city] oracle: {len(subset)} probes updated, {len(clean)} of {len(sample)} sampled probes "
          f"clean, {len(flips)} classification flips, {len(pts)} window pixels")
    return sc, desc, L, S, np.array(clean), st, irr, dist, pts, nrm, camp, E_ref


# (atlas formats, blend precision, stored-domain bounds for irradiance and
# distance texels, median bound for queries); the query raises the stored
# value to the power gamma / 2 and squares the normalised sum, so it carries
# 5x the stored relative error: its bound is 5x the irradiance texels' bound
_CITY_VARIANTS = {
    "fp16_storage": ("IRR_FP16", "DIST_FP16", "BLEND_FP32", 2.0 ** -11 + REL, 2.0 ** -11 + REL,
                     5 * (2.0 ** -11 + REL)),
    "rgb9e5_storage": ("IRR_RGB9E5", "DIST_FP32", "BLEND_FP32", None, REL, 5 * 2.0 ** -9),
    "tf32_blend": ("IRR_FP32", "DIST_FP32", "BLEND_TF32", 1e-3, 1e-3, 5e-3),
    "bf16_blend": ("IRR_FP32", "DIST_FP32", "BLEND_BF16", 2e-3, 1e-3, 1e-2),
    "tf32x3_blend": ("IRR_FP32", "DIST_FP32", "BLEND_TF32X3", REL, REL, REL),
}


@pytest.mark.parametrize("variant", sorted(_CITY_VARIANTS))
def test_city_precision_variants_against_oracle(g, city_ref, variant):
    """The precision configuration: the 16,384-probe city volume with reduced
    atlas storage or the tensor-core blend; per-texel error of the sampled
    active probes and per-pixel query error against the FP64 oracle."""
    sc, desc, L, S, clean, st, irr, dist, pts, nrm, cam, E_ref = city_ref
    fi, fd, prec, tol_i, tol_d, tol_q = _CITY_VARIANTS[variant]
    V = g.Volume(desc, irr_format=getattr(g, fi), dist_format=getattr(g, fd))
    V.update(S, L, 0, precision=getattr(g, prec))
    torch.cuda.synchronize()
    assert len(clean) >= 6
    if fi == "IRR_RGB9E5":
        gi = _decode_rgb9e5(V.irr_atlas().cpu().numpy())[clean]
        ref = irr[clean]
        mx = np.abs(ref).max(-1, keepdims=True)
        bound = 2.0 ** -9 * mx + REL * np.maximum(mx, 1e-3 * np.abs(ref).max())
        ei = float(np.max(np.abs(gi - ref) / np.maximum(bound, 1e-30)))
        ok_i = ei <= 1.0
        what_i = f"err / bound {ei:.3f}"
    else:
        gi = V.irr_atlas().cpu().numpy().astype(np.float64)[clean]
        ei = max(float(rel_err(gi[k], irr[p]).max()) for k, p in enumerate(clean))
        ok_i = ei <= tol_i
        what_i = f"max rel {ei:.2e}"
    gd = V.dist_atlas().cpu().numpy().astype(np.float64)[clean]
    ed = max(float(rel_err(gd[k], dist[p]).max()) for k, p in enumerate(clean))
    E = V.query(to_dev(pts), to_dev(nrm), cam).cpu().numpy()
    eq = rel_err(E, E_ref).max(-1)
    # at frame 0 only probes near geometry are active, so most window pixels
    # have no active cage probe: both sides give exactly 0 there, and the
    # median is taken over the lit pixels
    lit = np.any(E_ref > 0, axis=1)
    print(f"[precision city] {variant}: {len(clean)} probes, irr {what_i}, dist max rel {ed:.2e}; "
          f"{len(eq)} queries ({int(lit.sum())} lit), median rel over lit {np.median(eq[lit]):.2e}, "
          f"max {eq.max():.2e}")
    assert ok_i and ed <= tol_d
    assert lit.sum() >= 5000
    assert np.all(E[~lit] == 0.0)
    assert np.median(eq[lit]) <= tol_q
    if prec == "BLEND_TF32X3":
        # FP32-accurate: the parity bound at every pixel but those where the
        # oracle's own query moves by more than half the bound when the
        # updated probes' texels move by their errors in this run (seeded
        # signs); those are listed and held to the bound plus twice that
        gi_all = V.irr_atlas().cpu().numpy().astype(np.float64)
        gd_all = V.dist_atlas().cpu().numpy().astype(np.float64)
        rng = np.random.default_rng(11)
        upd = st != oracle.UNINIT
        irr_p, dist_p = irr.copy(), dist.copy()
        irr_p[upd] += np.abs(gi_all[upd] - irr[upd]) * rng.choice([-1.0, 1.0], size=irr[upd].shape)
        dist_p[upd] += np.abs(gd_all[upd] - dist[upd]) * rng.choice([-1.0, 1.0], size=dist[upd].shape)
        sens = rel_err(oracle.query(desc, st, irr_p, dist_p, pts, nrm, cam), E_ref).max(-1)
        listed = sens > REL / 2
        print(f"[precision city] tf32x3: listed {int(listed.sum())} of {len(eq)} pixels, max rel on the rest "
              f"{eq[~listed].max():.2e}")
        assert listed.mean() <= 1e-3
        assert eq[~listed].max() <= REL
        assert np.all(eq[listed] <= REL + 2 * sens[listed])
