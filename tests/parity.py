"""Helpers shared by the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare them element by element.

Tolerances (FP32 device arithmetic against the FP64 oracle):
  * states and hit/miss: bit-exact, except rays whose FP32 and FP64 results
    legitimately differ (grazing a triangle edge or silhouette within float
    rounding); those are counted, reported and must stay rare.
  * texels and query outputs: |gpu - oracle| <= 1e-4 * max(|oracle|, 1e-3 * max|oracle|)
    at every element; texels in which a flagged ray's share of the normalised
    weight exceeds LISTED_WEIGHT are listed and excluded, and queries that
    read them compare against the oracle's atlas patched with the GPU's
    listed texels (`patched`) and on the GPU's own atlas;
  * query points where the oracle itself moves by more than the bound when
    the point moves by one FP32 ulp (`fp32_neighbourhood_spread`) are listed
    and held to the bound plus twice that spread.
"""
from __future__ import annotations

import numpy as np
import torch

import oracle
import synth

REL = 1e-4


def rel_err(got, ref, floor_frac=1e-3):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.maximum(np.abs(ref), floor_frac * max(np.abs(ref).max(), 1e-30))
    return np.abs(got - ref) / scale


def to_dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def gpu_rays_by_probe(vol):
    rec, ids = vol.ray_records()
    return rec.cpu().numpy().astype(np.float64), ids.cpu().numpy().astype(np.int64)


def compare_rays(gpu_rec, gpu_ids, or_rays, rtol=1e-4):
    """Per-ray comparison.  Returns (bad mask [n_active, R], probe ids)."""
    ref = or_rays[gpu_ids]                                  # [n, R, 4]
    assert not np.isnan(ref).any(), "GPU traced a probe the oracle did not"
    scale = np.maximum(np.abs(ref), 1e-3 * np.maximum(np.abs(ref).max(axis=(0, 1)), 1e-30))
    err = np.abs(gpu_rec - ref) / scale
    bad = (err > rtol).any(axis=-1)
    return bad, err


def texel_weights(desc, seed, frame):
    """Weights used by each texel (for masking texels touched by flagged rays)."""
    dirs = oracle.frame_dirs(seed, frame, desc.rays_per_probe)
    ti = oracle.texel_dirs(desc.irr_n).reshape(-1, 3)
    td = oracle.texel_dirs(desc.dist_n).reshape(-1, 3)
    wi = np.maximum(0.0, ti @ dirs.T)
    wd = np.maximum(0.0, td @ dirs.T) ** desc.dist_cos_power
    wi = wi / np.maximum(wi.sum(1, keepdims=True), 1e-300)
    wd = wd / np.maximum(wd.sum(1, keepdims=True), 1e-300)
    return wi, wd


def border_sources(n):
    """For each bordered-tile texel, the interior texel index (row-major over n x n) it holds."""
    N = n + 2
    tile = np.zeros((N, N, 1))
    tile[1:-1, 1:-1, 0] = np.arange(n * n).reshape(n, n)
    tile = oracle.border_copy(tile, n)
    return tile[..., 0].astype(np.int64)


LISTED_WEIGHT = 1e-7


def masked_texels(desc, seed, frame, bad, ids):
    """Boolean masks [P, N, N] of the texels a flagged ray reaches: its share
    of the texel's normalised weights is above LISTED_WEIGHT.  A listed ray
    can move a texel it reaches by its whole record difference times that
    share (a distance texel's power-cosine weights make shares of 1e-4 .. 1e-3
    common), so the threshold is small enough that whatever is left moves by
    far less than the parity tolerance."""
    P = desc.n_probes
    wi, wd = texel_weights(desc, seed, frame)
    mi = np.zeros((P, desc.irr_n ** 2), dtype=bool)
    md = np.zeros((P, desc.dist_n ** 2), dtype=bool)
    for k in np.nonzero(bad.any(axis=1))[0]:
        rays = np.nonzero(bad[k])[0]
        mi[ids[k]] |= wi[:, rays].sum(1) > LISTED_WEIGHT
        md[ids[k]] |= wd[:, rays].sum(1) > LISTED_WEIGHT
    si, sd = border_sources(desc.irr_n), border_sources(desc.dist_n)
    return mi[:, si], md[:, sd]


def patched(ref, gpu, mask):
    """The oracle's atlas with the listed texels (mask [P, N, N]) taken from
    the GPU's: a query of it differs from the GPU's only by the query's own
    arithmetic and by texels that met the tolerance."""
    out = np.array(ref, dtype=np.float64, copy=True)
    out[mask] = np.asarray(gpu, dtype=np.float64)[mask]
    return out


def run_oracle(sc, lights, desc, frames, subset=None):
    h = oracle.SceneHandle(sc)
    st, irr, dist = oracle.new_state(desc)
    rays = []
    for f in frames:
        rays.append(oracle.update(h, lights, desc, f, st, irr, dist, subset=subset, want_rays=True))
    return st, irr, dist, rays


def lit_query_sample(sc, desc, seed, n_cells=4, per_cell=16, min_active=2, batch=16):
    """Seeded surface points for a volume query that the oracle can check
    with a one-step update of few probes.  Cells are taken in order of how
    many points they hold; in batches, the oracle classifies (frame 0) the
    eight cage probes of each, and the first `n_cells` cells with at least
    `min_active` active cage probes are kept (in the dense city most surface
    points lie inside other boxes, where every cage probe is Off), so the
    query has light to interpolate; `per_cell` points each.  Returns
    (points, normals, the 4x4x4 probes around every kept cell), points and
    normals rounded to FP32."""
    lo = np.asarray(desc.origin) + 1.0
    hi = np.asarray(desc.origin) + (np.asarray(desc.counts) - 1) * np.asarray(desc.spacing) - 1.0
    pts, nrm = synth.surface_points(sc, 20000, seed=seed, region_lo=lo, region_hi=hi)
    cell = np.floor((pts - np.asarray(desc.origin)) / np.asarray(desc.spacing)).astype(int)
    cx, cy, cz = desc.counts
    key = cell[:, 0] + cx * (cell[:, 1] + cy * cell[:, 2])
    uniq, counts = np.unique(key, return_counts=True)
    order = uniq[np.argsort(-counts, kind="stable")]
    corners = np.array([[a & 1, (a >> 1) & 1, (a >> 2) & 1] for a in range(8)])
    h = oracle.SceneHandle(sc)
    st, _, _ = oracle.new_state(desc)
    kept = []
    for b0 in range(0, len(order), batch):
        cand = order[b0:b0 + batch]
        cages = []
        for c in cand:
            base = np.array([c % cx, (c // cx) % cy, c // (cx * cy)])
            q = base + corners
            cages.append(q[:, 0] + cx * (q[:, 1] + cy * q[:, 2]))
        ids = np.unique(np.concatenate(cages))
        ids = ids[st[ids] == oracle.UNINIT]
        if len(ids):
            oracle.classify(h, desc, 0, ids, st)
        active = (st == oracle.NEWLY_VIGILANT) | (st == oracle.VIGILANT)
        kept += [c for c, cage in zip(cand, cages) if active[cage].sum() >= min_active]
        if len(kept) >= n_cells:
            break
    kept = kept[:n_cells]
    assert len(kept) == n_cells, "too few lit cells"
    sel = np.concatenate([np.nonzero(key == c)[0][:per_cell] for c in kept])
    need = set()
    for c in cell[sel]:
        for i in range(max(0, c[0] - 1), min(cx, c[0] + 3)):
            for j in range(max(0, c[1] - 1), min(cy, c[1] + 3)):
                for k in range(max(0, c[2] - 1), min(cz, c[2] + 3)):
                    need.add(i + cx * (j + cy * k))
    return synth.f32(pts[sel]), synth.f32(nrm[sel]), np.array(sorted(need))


def probe_positions(desc, ids):
    """Grid positions [n, 3] of probes (row-major x fastest, no offsets)."""
    ids = np.asarray(ids, dtype=np.int64)
    cx, cy, _ = desc.counts
    ijk = np.stack([ids % cx, (ids // cx) % cy, ids // (cx * cy)], 1)
    return np.asarray(desc.origin, dtype=np.float64) + ijk * np.asarray(desc.spacing, dtype=np.float64)


def near_probes(desc, pos, probe_ids, cells=2.0):
    """Points within `cells` spacings (per axis) of any of the probes: the
    points whose query can read a texel of those probes."""
    pos = np.asarray(pos, dtype=np.float64)
    out = np.zeros(len(pos), dtype=bool)
    sp = np.asarray(desc.spacing, dtype=np.float64)
    for x in probe_positions(desc, probe_ids):
        out |= np.all(np.abs(pos - x) <= cells * sp, axis=1)
    return out


def flagged_probes(bad, ids):
    """Probe ids with at least one flagged ray."""
    return np.asarray(ids)[np.nonzero(np.asarray(bad).any(axis=1))[0]]


def fp32_texel_spread(desc, states, irr, dist, pos, nrm, cams, draws=4, seed=5, ulps=4):
    """For each point (with its own camera, the query's w_o), the largest
    relative change of the oracle's query when every atlas value moves by
    `ulps` FP32 ulps with a seeded random sign, over `draws` draws: the size
    of the rounding an FP32 evaluation adds to its inputs (the bilinear
    moments, mu^2).  Where this exceeds the parity tolerance the FP32
    evaluation cannot fix the query to that tolerance (a Chebyshev weight
    where mu2 - mu^2 nearly cancels)."""
    pos = np.asarray(pos, dtype=np.float64).reshape(-1, 3)
    nrm = np.asarray(nrm, dtype=np.float64).reshape(-1, 3)
    cams = np.asarray(cams, dtype=np.float64).reshape(-1, 3)
    E0 = np.stack([oracle.query(desc, states, irr, dist, pos[k][None], nrm[k][None], cams[k])[0]
                   for k in range(len(pos))])
    rng = np.random.default_rng(seed)
    ui = ulps * np.abs(np.spacing(np.asarray(irr, dtype=np.float32))).astype(np.float64)
    ud = ulps * np.abs(np.spacing(np.asarray(dist, dtype=np.float32))).astype(np.float64)
    out = np.zeros(len(pos))
    for _ in range(draws):
        ip = irr + ui * rng.choice([-1.0, 1.0], size=irr.shape)
        dp = dist + ud * rng.choice([-1.0, 1.0], size=dist.shape)
        for k in range(len(pos)):
            E = oracle.query(desc, states, ip, dp, pos[k][None], nrm[k][None], cams[k])[0]
            out[k] = max(out[k], float((np.abs(E - E0[k]) / np.maximum(np.abs(E0[k]), 1e-30)).max()))
    return out


def fp32_neighbourhood_spread(fn, pos, nrm, floor_scale, ulps=1):
    """For each point, the largest change of the oracle's result fn(pos, nrm)
    over the 26 neighbouring FP32 positions (`ulps` ulps per axis), relative
    to the scale rel_err uses (max(|ref|, floor_scale)).  Where this exceeds
    the parity tolerance the FP32 input does not fix the result to that
    tolerance: rounding at the input's scale alone moves it further."""
    pos = np.asarray(pos, dtype=np.float64)
    nrm = np.asarray(nrm, dtype=np.float64)
    nb = np.array([[a, b, c] for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1) if (a, b, c) != (0, 0, 0)],
                  dtype=np.float64)
    p32 = pos.astype(np.float32)
    ulp = np.abs(np.nextafter(p32, np.float32(np.inf)) - p32).astype(np.float64)
    P = (pos[:, None, :] + ulps * nb[None] * ulp[:, None, :]).reshape(-1, 3)
    N_ = np.repeat(nrm, len(nb), axis=0)
    E0 = fn(pos, nrm)
    En = fn(P, N_).reshape(len(pos), len(nb), -1)
    scale = np.maximum(np.abs(E0), floor_scale)
    return (np.abs(En - E0[:, None, :]) / scale[:, None, :]).max(axis=(1, 2))
