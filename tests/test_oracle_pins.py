"""Pins that tie the FP64 oracle to what the paper and mathematics fix.

Each test checks the oracle against something other than itself: published
test vectors, closed forms, exact rational arithmetic, invariants or values
worked by hand.  Every piece of oracle arithmetic is reached by at least one
of them.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth

PI = np.pi


# ---------------------------------------------------------------- frame rays

def test_splitmix64_published_stream():
    # Reference output of SplitMix64 seeded with 0 (Vigna's splitmix64.c).
    assert oracle.splitmix64(0, 3) == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_rotation_is_uniform_proper_rotation():
    traces, z_axes = [], []
    for f in range(2000):
        R = oracle.rotation(12345, f)
        assert np.allclose(R @ R.T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1.0) < 1e-13
        traces.append(np.trace(R))
        z_axes.append(R[:, 2])
    t = np.array(traces)
    z = np.array(z_axes)
    # Haar measure on SO(3): E[tr R] = 0, E[tr^2 R] = 1; rotated axis uniform on S^2
    assert abs(t.mean()) < 0.08
    assert abs((t ** 2).mean() - 1.0) < 0.1
    assert np.all(np.abs(z.mean(0)) < 0.06)
    assert np.all(np.abs((z ** 2).mean(0) - 1.0 / 3.0) < 0.04)
    # different frames give different rotations; same (seed, frame) is reproducible
    assert not np.allclose(oracle.rotation(1, 0), oracle.rotation(1, 1))
    assert np.array_equal(oracle.rotation(7, 3), oracle.rotation(7, 3))


@pytest.mark.parametrize("n", [1, 7, 64, 256, 288])
def test_spherical_fibonacci_structure(n):
    d = oracle.sf_dirs(n)
    assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-15)
    # z equispaced: z_i = 1 - (2i+1)/n
    assert np.allclose(d[:, 2], 1.0 - (2 * np.arange(n) + 1) / n, atol=1e-15)
    # successive azimuths advance by 2 pi / phi (mod 2 pi), i.e. minus the golden angle
    if n > 2:
        az = np.arctan2(d[:, 1], d[:, 0])
        step = np.mod(np.diff(az), 2 * PI)
        golden = 2 * PI * 0.6180339887498949
        assert np.allclose(np.minimum(np.abs(step - golden), 2 * PI - np.abs(step - golden)),
                           0.0, atol=1e-12)
    if n >= 64:
        assert np.linalg.norm(d.sum(0)) / n < 2.0 / n


def test_frame_dirs_are_rotated_sf():
    R = oracle.rotation(99, 5)
    d = oracle.frame_dirs(99, 5, 64)
    assert np.allclose(d, oracle.sf_dirs(64) @ R.T, atol=1e-15)


# ------------------------------------------------------------ octahedral map

def test_oct_axes_closed_form():
    cases = {(0, 0, 1): (0, 0), (1, 0, 0): (1, 0), (-1, 0, 0): (-1, 0), (0, 1, 0): (0, 1),
             (0, -1, 0): (0, -1)}
    for v, u in cases.items():
        assert np.allclose(oracle.oct_encode(v)[0], u, atol=1e-15)
    assert np.allclose(np.abs(oracle.oct_encode((0, 0, -1))[0]), (1, 1), atol=1e-15)
    # hand-worked decodes
    s = 2 ** -0.5
    assert np.allclose(oracle.oct_decode((0.5, 0.0))[0], (s, 0, s), atol=1e-15)
    assert np.allclose(oracle.oct_decode((0.5, 0.5))[0], (s, s, 0), atol=1e-15)
    v = np.array([0.5, 0.25, -0.25])
    assert np.allclose(oracle.oct_decode((0.75, 0.5))[0], v / np.linalg.norm(v), atol=1e-15)
    v = np.array([-0.5, -0.25, -0.25])
    assert np.allclose(oracle.oct_decode((-0.75, -0.5))[0], v / np.linalg.norm(v), atol=1e-15)


def test_oct_round_trips():
    rng = synth.Rng(5)
    v = rng.normal(3 * 20000).reshape(-1, 3)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    u = oracle.oct_encode(v)
    assert np.all(np.abs(u) <= 1.0)
    assert np.allclose(oracle.oct_decode(u), v, atol=1e-15)
    uu = rng.uniform(2 * 20000, -1, 1).reshape(-1, 2)
    assert np.allclose(oracle.oct_encode(oracle.oct_decode(uu)), uu, atol=1e-14)
    # upper hemisphere is the diamond |u|+|v| <= 1 with u = (x, y)/(|x|+|y|+|z|)
    up = v[v[:, 2] > 0]
    assert np.allclose(oracle.oct_encode(up), up[:, :2] / np.abs(up).sum(1, keepdims=True),
                       atol=1e-15)


def test_texel_directions_symmetry():
    for n in (6, 14):
        t = oracle.texel_dirs(n)
        assert np.allclose(np.linalg.norm(t, axis=-1), 1.0)
        # mirror of column i is column n-1-i with x negated (and same for rows / y)
        assert np.allclose(t[:, ::-1, 0], -t[:, :, 0], atol=1e-15)
        assert np.allclose(t[:, ::-1, 1:], t[:, :, 1:], atol=1e-15)
        assert np.allclose(t[::-1, :, 1], -t[:, :, 1], atol=1e-15)
        # the map is injective: no two texels share a direction
        flat = t.reshape(-1, 3)
        dots = flat @ flat.T - 2 * np.eye(len(flat))
        assert dots.max() < 1 - 1e-6


# ------------------------------------------------------ tiles and filtering

@pytest.mark.parametrize("n", [6, 14])
def test_bilinear_reproduces_affine_tile(n):
    # bilinear filtering reproduces an affine function of the texel position
    # exactly, which pins the octahedral-to-texel coordinate mapping.
    N = n + 2
    ys, xs = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    tile = np.stack([xs + 0.5 + 10 * (ys + 0.5), 3.0 - 2 * xs], axis=-1).astype(np.float64)
    rng = synth.Rng(11)
    v = rng.normal(3 * 500).reshape(-1, 3)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    got = oracle.sample_bilinear(tile, n, v)
    u = oracle.oct_encode(v)
    sx = 1 + (u[:, 0] + 1) / 2 * n       # sample position in texel units from the tile corner
    sy = 1 + (u[:, 1] + 1) / 2 * n
    assert np.allclose(got[:, 0], sx + 10 * sy, atol=1e-11)
    assert np.allclose(got[:, 1], 3.0 - 2 * (sx - 0.5), atol=1e-11)


def _seam_pairs(eps, m=400, seed=12):
    """Pairs of directions that approach one seam point from the two folded
    sides of the octahedral square: across each edge the map is mirrored,
    and the four corners meet at -z."""
    rng = synth.Rng(seed)
    y = rng.uniform(m, -0.98, 0.98)
    pairs = []
    e = 1.0 - eps
    for a, b in (((-e, 1), (-e, -1)), ((e, 1), (e, -1))):   # left / right edges
        pairs.append((np.stack([np.full(m, a[0]), y], 1), np.stack([np.full(m, b[0]), -y], 1)))
    for a in (-e, e):                                        # bottom / top edges
        pairs.append((np.stack([y, np.full(m, a)], 1), np.stack([-y, np.full(m, a)], 1)))
    corners = np.array([[-e, -e], [e, -e], [-e, e], [e, e]])
    for k in range(1, 4):
        pairs.append((corners[:1], corners[k:k + 1]))
    return pairs


@pytest.mark.parametrize("n", [6, 14])
def test_border_copy_makes_sampling_continuous_across_seams(n):
    N = n + 2
    rng = synth.Rng(13)
    interior = rng.uniform(n * n * 2, 0.0, 1.0).reshape(n, n, 2)
    tile = np.zeros((N, N, 2))
    tile[1:-1, 1:-1] = interior
    tile = oracle.border_copy(tile, n)
    assert np.array_equal(tile[1:-1, 1:-1], interior)
    bare = np.zeros((N, N, 2))
    bare[1:-1, 1:-1] = interior
    for ua, ub in _seam_pairs(1e-9):
        va, vb = oracle.oct_decode(ua), oracle.oct_decode(ub)
        assert np.max(np.linalg.norm(va - vb, axis=1)) < 1e-8     # same seam point
        sa, sb = oracle.sample_bilinear(tile, n, va), oracle.sample_bilinear(tile, n, vb)
        assert np.max(np.abs(sa - sb)) < 1e-7
        # without a border (or with an unmirrored one) the two sides disagree
        ba, bb = oracle.sample_bilinear(bare, n, va), oracle.sample_bilinear(bare, n, vb)
        assert np.max(np.abs(ba - bb)) > 1e-2


@pytest.mark.parametrize("n", [6, 14])
def test_bilinear_tracks_smooth_function(n):
    def f(v):
        return 1.0 + 0.6 * v[..., 0] - 0.3 * v[..., 1] + 0.45 * v[..., 2] + 0.5 * v[..., 0] * v[..., 2]
    N = n + 2
    tile = np.zeros((N, N, 1))
    tile[1:-1, 1:-1, 0] = f(oracle.texel_dirs(n))
    tile = oracle.border_copy(tile, n)
    v = synth.Rng(12).normal(3 * 6000).reshape(-1, 3)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    err = np.abs(oracle.sample_bilinear(tile, n, v)[:, 0] - f(v))
    assert err.max() < 1.3 / n            # first order at the kinks of the map
    assert err.mean() < 2.5 / n ** 2      # second order elsewhere


# --------------------------------------------------------------- tracing

def _exact_hits(scene, o, d):
    """Closest hit in exact rational arithmetic (inputs are exact binary fractions)."""
    V = [[Fraction(float(x)) for x in row] for row in scene.verts]
    out = []
    for k in range(len(o)):
        O = [Fraction(float(x)) for x in o[k]]
        D = [Fraction(float(x)) for x in d[k]]
        best, bi = None, -1
        for ti, (a, b, c) in enumerate(scene.tris):
            v0, v1, v2 = V[a], V[b], V[c]
            e1 = [v1[i] - v0[i] for i in range(3)]
            e2 = [v2[i] - v0[i] for i in range(3)]
            nrm = [e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                   e1[0] * e2[1] - e1[1] * e2[0]]
            den = sum(nrm[i] * D[i] for i in range(3))
            if den == 0:
                continue
            t = sum(nrm[i] * (v0[i] - O[i]) for i in range(3)) / den
            if t <= 0:
                continue
            p = [O[i] + t * D[i] for i in range(3)]
            # inside test with signed areas relative to the face normal (edges included)
            ok = True
            for (A, B) in ((v0, v1), (v1, v2), (v2, v0)):
                ab = [B[i] - A[i] for i in range(3)]
                ap = [p[i] - A[i] for i in range(3)]
                cr = [ab[1] * ap[2] - ab[2] * ap[1], ab[2] * ap[0] - ab[0] * ap[2],
                      ab[0] * ap[1] - ab[1] * ap[0]]
                if sum(cr[i] * nrm[i] for i in range(3)) < 0:
                    ok = False
                    break
            if ok and (best is None or t < best):
                best, bi = t, ti
        out.append((bi, None if best is None else float(best)))
    return out


def test_trace_matches_exact_rational_brute_force():
    b = synth._Builder()
    b.box((0, 0, 0), (4, 4, 4), obj=0, inward=True)
    b.box((1, 1, 1), (2, 2.5, 1.75), obj=1)
    b.box((2.5, 0.5, 2.0), (3.25, 1.5, 3.5), obj=1)
    sc = b.finish(np.full((2, 3), 0.5), [1, 1], np.zeros((0, 3)), "tiny")
    rng = synth.Rng(21)
    o = synth.f32(rng.uniform(3 * 150, 0.2, 3.8).reshape(-1, 3))
    d = rng.unit_vectors(150)
    t, tri, bf = oracle.trace(oracle.SceneHandle(sc), o, d)
    exact = _exact_hits(sc, o, d)
    for k, (ei, et) in enumerate(exact):
        if ei < 0:
            assert tri[k] < 0
            continue
        assert tri[k] >= 0
        assert abs(t[k] - et) <= 1e-12 * max(1.0, et)
        if tri[k] != ei:   # only allowed for an exact tie on a shared edge
            assert abs(t[k] - et) <= 1e-12 * et
        # backface flag: direction along the CCW normal
        v = sc.verts[sc.tris[tri[k]]]
        ng = np.cross(v[1] - v[0], v[2] - v[0])
        assert bool(bf[k]) == bool(np.dot(d[k], ng) > 0)


def test_enclosing_box_distances_closed_form():
    h = np.array([1.5, 2.25, 0.75])
    sc = synth.box_room(-h, h)
    d = synth.Rng(3).unit_vectors(3000)
    o = np.zeros_like(d)
    t, tri, bf = oracle.trace(oracle.SceneHandle(sc), o, d)
    with np.errstate(divide="ignore"):
        closed = np.min(h[None, :] / np.abs(d), axis=1)
    assert np.all(tri >= 0) and not bf.any()
    assert np.allclose(t, closed, rtol=1e-13)


def test_enclosing_sphere_distances_and_moments():
    rad = 2.5
    sc = synth.icosphere(rad, 3, inward=True)
    vol = synth.VolumeDesc(origin=(0, 0, 0), spacing=(1, 1, 1), counts=(2, 2, 2), rays_per_probe=256,
                           hysteresis_irr=0, hysteresis_vis=0, t_max=1e9, state_machine=0, seed=4)
    # the probe at the origin (logical 0,0,0) sits at the sphere centre
    st, irr, dist = oracle.new_state(vol)
    oracle.update(oracle.SceneHandle(sc), synth.Lights(), vol, 0, st, irr, dist, subset=[0])
    mu = dist[0, 1:-1, 1:-1, 0]
    mu2 = dist[0, 1:-1, 1:-1, 1]
    # every hit lies between the faces' inscribed distance and the radius
    V = sc.verts[sc.tris]
    ctr = V.mean(1)
    nrm = np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    inner = np.min(np.abs(np.einsum("ij,ij->i", ctr, nrm)))
    assert np.all(mu >= inner - 1e-12) and np.all(mu <= rad + 1e-12)
    assert np.all(mu2 >= inner ** 2 - 1e-12) and np.all(mu2 <= rad ** 2 + 1e-12)
    # Jensen: mean of squares >= square of mean
    assert np.all(mu2 >= mu ** 2 - 1e-12)
    # a finer sphere converges to mu = r, mu2 = r^2 (sigma^2 -> 0)
    assert np.all(np.abs(mu - rad) < 0.02 * rad)


# ------------------------------------------------------ update closed forms

def _empty_vol(**kw):
    d = dict(origin=(0, 0, 0), spacing=(1, 1, 1), counts=(2, 2, 2), rays_per_probe=64,
             hysteresis_irr=0, hysteresis_vis=0, state_machine=0, seed=77, t_max=3.0)
    d.update(kw)
    return synth.VolumeDesc(**d)


def _decode(e, gamma):
    return np.power(e, gamma)


@pytest.mark.parametrize("R", [1, 5, 64, 256])
def test_uniform_sky_gives_exact_mean(R):
    a = np.array([0.3, 1.7, 0.05])
    L = synth.Lights(sky_a=a, sky_b=np.zeros(3))
    vol = _empty_vol(rays_per_probe=R)
    st, irr, dist = oracle.new_state(vol)
    oracle.update(oracle.SceneHandle(synth.empty_scene()), L, vol, 3, st, irr, dist)
    inner = irr[:, 1:-1, 1:-1, :]
    # texels seen by at least one ray hold exactly a (encoded a^(1/gamma))
    seen = inner.max(-1) > 0
    if R >= 5:
        assert seen.all()
    assert np.allclose(_decode(inner[seen], vol.gamma), np.broadcast_to(a, inner[seen].shape),
                       rtol=1e-13)
    dseen = dist[:, 1:-1, 1:-1, 0] > 0
    if R >= 64:
        assert dseen.all()
    assert np.allclose(dist[:, 1:-1, 1:-1, 0][dseen], vol.t_max, rtol=1e-14)
    assert np.allclose(dist[:, 1:-1, 1:-1, 1][dseen], vol.t_max ** 2, rtol=1e-14)
    if R >= 5:
        pos, nrm, cam = synth.room_queries(n=200)
        pos = pos / 10.0   # inside the 1 m cell
        E = oracle.query(vol, st, irr, dist, pos, nrm, cam)
        assert np.allclose(E, PI * a[None, :], rtol=1e-12)


def test_linear_sky_converges_to_cosine_mean():
    a = np.full(3, 1.0)
    b = np.array([0.8, -0.5, 0.3])
    up = synth.f32([0.2, 0.9, -0.3])
    up = up / np.linalg.norm(up)
    L = synth.Lights(sky_a=a, sky_b=b, sky_up=up)
    errs = []
    for R in (64, 256, 1024, 4096):
        vol = _empty_vol(rays_per_probe=R, counts=(2, 2, 2), gamma=1.0)
        st, irr, dist = oracle.new_state(vol)
        oracle.update(oracle.SceneHandle(synth.empty_scene()), L, vol, 1, st, irr, dist,
                      subset=[0])
        tex = oracle.texel_dirs(vol.irr_n)
        # closed form: hemisphere cosine mean of a + b (w.up) is a + (2/3) b (n.up)
        want = a[None, None, :] + (2.0 / 3.0) * (tex @ up)[..., None] * b[None, None, :]
        errs.append(np.abs(irr[0, 1:-1, 1:-1, :] - want).max())
    assert errs[-1] < 2e-3
    assert errs[0] > errs[-1] * 4
    assert all(e < 0.06 for e in errs)


def test_hysteresis_gamma_closed_forms():
    sc = oracle.SceneHandle(synth.empty_scene())
    alpha = 0.9

    def run(a_val, frames):
        vol = _empty_vol(hysteresis_irr=alpha, rays_per_probe=32)
        st, irr, dist = oracle.new_state(vol)
        L = synth.Lights(sky_a=np.full(3, a_val))
        seq = []
        for f in range(frames):
            oracle.update(sc, L, vol, f, st, irr, dist, subset=[0])
            seq.append(irr[0, 3, 3, 0])
        return np.array(seq)

    # below both thresholds: e_k = (1 - alpha^k) c with c = a^(1/5)
    c = 1e-4 ** 0.2
    assert c < 0.25
    k = np.arange(1, 9)
    assert np.allclose(run(1e-4, 8), (1 - alpha ** k) * c, rtol=1e-13)
    # first change above 0.8: hysteresis drops to 0, value jumps to c and stays
    c = 0.5 ** 0.2
    assert c > 0.8
    assert np.allclose(run(0.5, 5), c, rtol=1e-13)
    # between thresholds: hysteresis lowered by 0.15 while the change exceeds 0.25
    c = 0.01 ** 0.2                                # 0.398
    seq = run(0.01, 4)
    assert np.isclose(seq[0], 0.25 * c)            # delta = c > 0.25: alpha 0.75
    assert np.isclose(seq[1], c * (1 - 0.75 ** 2))  # delta = 0.75 c = 0.299 > 0.25
    assert np.isclose(seq[2], c * (1 - 0.75 ** 2 * 0.9))  # delta = 0.224 < 0.25: alpha 0.9
    # visibility hysteresis has no thresholds
    vol = _empty_vol(hysteresis_vis=0.5, rays_per_probe=32)
    st, irr, dist = oracle.new_state(vol)
    for f in range(3):
        oracle.update(sc, synth.Lights(), vol, f, st, irr, dist, subset=[0])
    assert np.isclose(dist[0, 5, 5, 0], vol.t_max * (1 - 0.5 ** 3))


def test_furnace_multibounce_exact():
    # closed room, every triangle emits Le with albedo rho, sun off, hysteresis 0:
    # all probes agree, so M_t = Le (1 - rho^(t+1)) / (1 - rho) exactly.
    Le, rho = 0.8, 0.6
    sc = synth.box_room((0, 0, 0), (4, 4, 4), albedo=rho, emit=[Le, Le, Le])
    vol = synth.VolumeDesc(origin=(0.5, 0.5, 0.5), spacing=(1.5, 1.5, 1.5), counts=(3, 3, 3),
                           rays_per_probe=48, hysteresis_irr=0, hysteresis_vis=0,
                           state_machine=0, seed=8, gamma=5.0)
    h = oracle.SceneHandle(sc)
    st, irr, dist = oracle.new_state(vol)
    for t in range(6):
        oracle.update(h, synth.Lights(), vol, t, st, irr, dist)
        want = Le * (1 - rho ** (t + 1)) / (1 - rho)
        assert np.allclose(irr[:, 1:-1, 1:-1, :] ** vol.gamma, want, rtol=1e-12)


def test_direct_light_and_sky_per_ray():
    # probe above a large ground quad: down rays see rho E cos/pi (unshadowed, zero
    # previous atlas), up rays see the sky, depths h/|w_y| clamped to t_max.
    b = synth._Builder()
    b.quad([(-1e3, 0, -1e3), (1e3, 0, -1e3), (1e3, 0, 1e3), (-1e3, 0, 1e3)],
           np.array([0.0, 1, 0]), obj=0)
    rho = np.array([0.3, 0.5, 0.7])
    sc = b.finish(rho[None, :], [1], np.zeros((0, 3)), "ground")
    sun = synth.f32(np.array([0.3, -0.8, 0.2]) / np.linalg.norm([0.3, -0.8, 0.2]))
    E = np.array([2.0, 3.0, 4.0])
    L = synth.Lights(sun_dir=sun, sun_irradiance=E, sky_a=np.full(3, 0.4), sky_b=np.full(3, 0.2))
    hgt = 1.25
    vol = _empty_vol(origin=(0, hgt, 0), rays_per_probe=128, t_max=2.0)
    st, irr, dist = oracle.new_state(vol)
    rays = oracle.update(oracle.SceneHandle(sc), L, vol, 2, st, irr, dist, subset=[0],
                         want_rays=True)[0]
    w = oracle.frame_dirs(vol.seed, 2, 128)
    down = w[:, 1] < 0
    cos = -sun[1]
    assert np.allclose(rays[down, :3], rho[None, :] * E[None, :] * cos / PI, rtol=1e-13)
    assert np.allclose(rays[down, 3], np.minimum(hgt / -w[down, 1], 2.0), rtol=1e-13)
    assert np.allclose(rays[~down, :3], 0.4 + 0.2 * w[~down, 1][:, None], rtol=1e-13)
    assert np.allclose(rays[~down, 3], 2.0)
    # from below the ground every down... up ray hits the back face: radiance 0, depth 0.2 t
    vol2 = _empty_vol(origin=(0, -0.5, 0), rays_per_probe=128, t_max=50.0)
    st, irr, dist = oracle.new_state(vol2)
    rays = oracle.update(oracle.SceneHandle(sc), L, vol2, 2, st, irr, dist, subset=[0],
                         want_rays=True)[0]
    up = w[:, 1] > 0
    assert np.all(rays[up, :3] == 0)
    assert np.allclose(rays[up, 3], np.minimum(0.2 * 0.5 / w[up, 1], 50.0), rtol=1e-13)


def test_shadow_ray_blocks_sun():
    # an occluder box between the ground and the sun: rays hitting the ground
    # under it get no direct light
    b = synth._Builder()
    b.quad([(-50, 0, -50), (50, 0, -50), (50, 0, 50), (-50, 0, 50)], np.array([0.0, 1, 0]), obj=0)
    b.box((-20, 3, -20), (20, 3.5, 20), obj=1)
    sc = b.finish(np.full((2, 3), 0.5), [1, 1], np.zeros((0, 3)), "roof")
    L = synth.Lights(sun_dir=np.array([0.0, -1.0, 0.0]), sun_irradiance=np.full(3, 2.0))
    vol = _empty_vol(origin=(0, 1.0, 0), rays_per_probe=64, t_max=10.0)
    st, irr, dist = oracle.new_state(vol)
    rays = oracle.update(oracle.SceneHandle(sc), L, vol, 0, st, irr, dist, subset=[0],
                         want_rays=True)[0]
    w = oracle.frame_dirs(vol.seed, 0, 64)
    down = w[:, 1] < 0
    hit = np.abs(1.0 / w[:, 1])[:, None] * w[:, [0, 2]]       # ground hit, horizontal offset
    far = (np.max(np.abs(hit), axis=1) > 20) & (np.max(np.abs(hit), axis=1) < 50)  # lit ground
    assert np.all(rays[down & ~far, :3] == 0.0)
    assert np.allclose(rays[down & far, :3], 0.5 * 2.0 / PI)


# ------------------------------------------------------------- the query

def _two_cube(B=0.0, **kw):
    d = dict(origin=(0, 0, 0), spacing=(1, 1, 1), counts=(2, 2, 2), rays_per_probe=8,
             self_shadow_bias=B, state_machine=0, gamma=5.0)
    d.update(kw)
    return synth.VolumeDesc(**d)


def test_query_agreeing_probes_return_common_value():
    vol = synth.VolumeDesc(origin=(0, 0, 0), spacing=(1.0, 0.75, 1.25), counts=(3, 4, 3),
                           state_machine=0, gamma=5.0, self_shadow_bias=0.3)
    st, irr, dist = oracle.new_state(vol)
    rng = synth.Rng(31)
    tile_i = rng.uniform(irr[0].size, 0.1, 1.0).reshape(irr[0].shape)
    tile_d = np.stack([rng.uniform(dist[0, ..., 0].size, 0.2, 2.0).reshape(dist.shape[1:3]),
                       rng.uniform(dist[0, ..., 0].size, 0.0, 5.0).reshape(dist.shape[1:3])], -1)
    irr[:] = tile_i
    dist[:] = tile_d
    st[:] = rng.uniform(len(st)).round().astype(np.uint8) + 3   # mix of newly/vigilant
    n = 300
    pos = synth.f32(rng.uniform(3 * n, 0.0, 2.0).reshape(n, 3) * np.array([1, 1.5, 1.25]) * 1.2)
    nrm = rng.unit_vectors(n)
    cam = np.array([0.3, 5.0, -2.0])
    E = oracle.query(vol, st, irr, dist, pos, nrm, cam)
    s = oracle.sample_bilinear(tile_i, vol.irr_n, nrm)
    assert np.allclose(E, PI * s ** vol.gamma, rtol=1e-12)


def test_glossy_lookup_reads_the_mirror_direction():
    """Second-order glossy (Sec. 4.4): with every probe holding the same tiles
    and no occlusion, the lookup is the tile's bilinear sample in the mirror
    direction r = d - 2 (d.n) n, decoded, as radiance M (no factor pi)."""
    vol = synth.VolumeDesc(origin=(0, 0, 0), spacing=(1.0, 1.0, 1.0), counts=(3, 3, 3),
                           state_machine=0, gamma=5.0, self_shadow_bias=0.3)
    st, irr, dist = oracle.new_state(vol)
    rng = synth.Rng(33)
    tile = rng.uniform(irr[0].size, 0.1, 1.0).reshape(irr[0].shape)
    irr[:] = tile
    dist[..., 0] = 10.0
    dist[..., 1] = 100.0
    st[:] = oracle.VIGILANT
    n = 200
    pos = synth.f32(rng.uniform(3 * n, 0.3, 1.7).reshape(n, 3))
    nrm = rng.unit_vectors(n)
    d = rng.unit_vectors(n)
    M = oracle.query_glossy(vol, st, irr, dist, pos, nrm, d)
    dn = np.sum(d * nrm, -1, keepdims=True)
    r = d - 2 * dn * nrm
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    assert np.allclose(M, oracle.sample_bilinear(tile, vol.irr_n, r) ** vol.gamma, rtol=1e-12)
    # the mirror direction differs from the normal: a normal lookup would not match
    assert not np.allclose(M, oracle.sample_bilinear(tile, vol.irr_n, nrm) ** vol.gamma, rtol=1e-3)
    # head-on arrival (d = -n) mirrors back along n: E / pi of the irradiance
    # query with the camera straight above
    x = pos[:1]
    nn = nrm[:1]
    Mg = oracle.query_glossy(vol, st, irr, dist, x, nn, -nn)
    E = oracle.query(vol, st, irr, dist, x, nn, x[0] + 4.0 * nn[0])
    assert np.allclose(Mg, E / PI, rtol=1e-12)
    # no surface: zero
    assert np.all(oracle.query_glossy(vol, st, irr, dist, x, np.zeros((1, 3)), -nn) == 0)


def test_query_chebyshev_and_backface_weights_by_hand():
    vol = _two_cube(B=0.0)
    st, irr, dist = oracle.new_state(vol)
    irr[:] = 0.5
    x = np.array([[0.5, 0.5, 0.5]])
    n = np.array([[0.0, 0.0, 1.0]])
    cam = np.array([0.5, 0.5, 9.0])
    r = np.sqrt(0.75)
    c = 1.0 / np.sqrt(3.0)
    wb_low = ((1 - c) / 2) ** 2 + 0.2     # probes below the point (z = 0)
    wb_high = ((1 + c) / 2) ** 2 + 0.2
    wb = np.array([wb_low] * 4 + [wb_high] * 4)
    # unoccluded: r <= mu everywhere -> Chebyshev weight exactly 1
    dist[..., 0] = 2.0
    dist[..., 1] = 4.0
    _, w = oracle.query(vol, st, irr, dist, x, n, cam, want_weights=True)
    assert np.allclose(w[0], wb / 8.0, rtol=1e-14)
    # occluded at mu = 0.5 with mu2 = 0.26: sigma^2 = 0.01, weight 0.01 / (0.01 + (r - 0.5)^2)
    dist[..., 0] = 0.5
    dist[..., 1] = 0.26
    _, w = oracle.query(vol, st, irr, dist, x, n, cam, want_weights=True)
    wc = 0.01 / (0.01 + (r - 0.5) ** 2)
    assert np.allclose(w[0], wb / 8.0 * wc, rtol=1e-12)
    # zero variance behind the surface: the weight floor keeps the sum positive
    dist[..., 1] = 0.25
    E, w = oracle.query(vol, st, irr, dist, x, n, cam, want_weights=True)
    assert np.allclose(w[0], wb / 8.0 * 1e-6, rtol=1e-12)
    assert np.allclose(E, PI * 0.5 ** 5)
    # inactive probes carry no weight
    st[:4] = oracle.SLEEPING
    _, w = oracle.query(vol, st, irr, dist, x, n, cam, want_weights=True)
    assert np.all(w[0, :4] == 0) and np.all(w[0, 4:] > 0)
    st[:] = oracle.OFF
    E = oracle.query(vol, st, irr, dist, x, n, cam)
    assert np.all(E == 0)


def test_query_at_a_probe_uses_only_that_probe():
    vol = _two_cube(B=0.0, counts=(3, 3, 3))
    st, irr, dist = oracle.new_state(vol)
    vals = synth.Rng(41).uniform(27, 0.2, 0.9)
    for p in range(27):
        irr[p] = vals[p]
    dist[..., 0] = 5.0
    dist[..., 1] = 25.0
    pts, want = [], []
    for p in range(27):
        i, j, k = p % 3, (p // 3) % 3, p // 9
        pts.append((i, j, k))
        want.append(PI * vals[p] ** 5)
    nrm = synth.Rng(42).unit_vectors(27)
    E = oracle.query(vol, st, irr, dist, np.array(pts, float), nrm, np.array([9.0, 9, 9]))
    assert np.allclose(E[:, 0], want, rtol=1e-12)


def test_self_shadow_bias_moves_the_sample_point():
    # the bias (n 0.2 + w_o 0.8) (0.75 D) B moves a point at x=0.5 onto the
    # x = 1 probe plane when B = 0.5 / (0.75 * 0.8)
    vol = _two_cube(B=0.5 / 0.6)
    st, irr, dist = oracle.new_state(vol)
    vals = [0.3, 0.6] * 4          # probes at x = 0 hold 0.3, at x = 1 hold 0.6
    for p in range(8):
        irr[p] = vals[p]
    dist[..., 0] = 5.0
    dist[..., 1] = 25.0
    x = np.array([[0.5, 0.5, 0.5]])
    n = np.array([[0.0, 1.0, 0.0]])     # normal perpendicular: moves y by 0.2*0.75*B... keep it
    n_perp_bias = 0.2 * 0.75 * (0.5 / 0.6)
    cam = np.array([100.0, 0.5, 0.5])   # w_o = +x
    E = oracle.query(vol, st, irr, dist, x, n, cam)
    # all weight on the x = 1 face (trilinear x-fraction = 1)
    assert np.allclose(E, PI * 0.6 ** 5, rtol=1e-10)
    assert n_perp_bias < 0.5


# ------------------------------------------------------------- states

def test_states_hand_built():
    # solid box around probe 0, wall near probe 1, empty space around probe 2
    b = synth._Builder()
    b.box((-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), obj=0)         # probe at origin is inside
    b.box((9.5, -5, -5), (12, 5, 5), obj=0)                    # wall 0.5 from probe at x=9
    sc = b.finish(np.full((1, 3), 0.5), [1], np.zeros((0, 3)), "states")
    vol = synth.VolumeDesc(origin=(0, 0, 0), spacing=(1.0, 1.0, 1.0), counts=(30, 1, 1),
                           rays_per_probe=64, seed=3)
    st = np.zeros(30, dtype=np.uint8)
    # counts (30,1,1): counts-2 < 0 is fine for classification (no query)
    bf, dmin = oracle.classify(oracle.SceneHandle(sc), vol, 0, [0, 9, 4], st)
    assert st[0] == oracle.OFF and bf[0] == 64
    assert st[9] == oracle.NEWLY_VIGILANT and 0.5 <= dmin[1] < 1.0
    assert st[4] == oracle.SLEEPING and dmin[2] >= 3.5


def test_states_backface_fraction_threshold():
    # a downward-facing square below the probe: the rays that reach it hit its back
    # face.  The fraction is counted geometrically from the frame's rays; more than
    # 25% backfaces means Off; below it, with no front face in reach, Sleeping.
    R = 128
    seed, frame = 9, 0
    w = oracle.frame_dirs(seed, frame, R)
    down = w[:, 1] < 0
    reach = np.zeros(R)
    reach[down] = np.max(np.abs(w[down][:, [0, 2]] / w[down][:, 1:2]), axis=1)  # half-size needed
    for target, want in ((0.35, oracle.OFF), (0.20, oracle.SLEEPING)):
        k = int(round(target * R))
        s_half = 0.5 * (np.sort(reach[down])[k - 1] + np.sort(reach[down])[k])
        s_half = float(synth.f32(s_half))
        b = synth._Builder()
        b.quad([(-s_half, -1, -s_half), (s_half, -1, -s_half), (s_half, -1, s_half),
                (-s_half, -1, s_half)], np.array([0.0, -1, 0]), obj=0)
        sc = b.finish(np.full((1, 3), 0.5), [1], np.zeros((0, 3)), "plate")
        vol = synth.VolumeDesc(origin=(0, 0, 0), spacing=(4.0, 4.0, 4.0), counts=(2, 2, 2),
                               rays_per_probe=R, seed=seed)
        st = np.zeros(8, dtype=np.uint8)
        bf, dmin = oracle.classify(oracle.SceneHandle(sc), vol, frame, [0], st)
        assert bf[0] == k
        assert st[0] == want


def test_update_state_machine_transitions():
    sc = synth.room_scene()
    vol = synth.room_volume(counts=(4, 4, 4), spacing=(2.5, 2.5, 2.5), origin=(1.25, 1.25, 1.25))
    st, irr, dist = oracle.new_state(vol)
    h = oracle.SceneHandle(sc)
    oracle.update(h, synth.room_lights(), vol, 0, st, irr, dist)
    assert set(np.unique(st)) <= {oracle.OFF, oracle.SLEEPING, oracle.VIGILANT}
    # inactive probes keep zero atlases; active ones got values
    act = st == oracle.VIGILANT
    assert np.all(irr[~act] == 0) and np.all(dist[~act] == 0)
    assert np.all(dist[act][..., 0] > 0)
    before = st.copy()
    oracle.update(h, synth.room_lights(), vol, 1, st, irr, dist)
    assert np.array_equal(before, st)


# ------------------------------------------------------------- cascades

def test_cascade_weights_nested():
    fine = synth.VolumeDesc(origin=(-4, -4, -4), spacing=(1, 1, 1), counts=(9, 9, 9), state_machine=0)
    coarse = synth.VolumeDesc(origin=(-16, -16, -16), spacing=(4, 4, 4), counts=(9, 9, 9),
                              state_machine=0)
    vf, vc = oracle.make_volume(fine), oracle.make_volume(coarse)
    sf, irf, df = oracle.new_state(fine)
    sc_, irc, dc = oracle.new_state(coarse)
    irf[:] = 0.5
    irc[:] = 0.8
    df[..., 0] = 50
    df[..., 1] = 2500
    dc[..., 0] = 50
    dc[..., 1] = 2500
    xs = np.linspace(-6, 6, 121)
    pos = np.stack([xs, np.zeros_like(xs), np.zeros_like(xs)], 1)
    nrm = np.tile([0.0, 1.0, 0.0], (len(xs), 1))
    E, w = oracle.query_cascade([vf, vc], [sf, sc_], [irf, irc], [df, dc], pos, nrm,
                                np.array([0.0, 3.0, 0.0]), want_weights=True)
    # weights sum to 1 everywhere the coarse volume covers
    assert np.allclose(w.sum(1), 1.0)
    inner = np.abs(xs) <= 3.0
    assert np.allclose(w[inner, 0], 1.0) and np.all(w[inner, 1] == 0)
    outer = np.abs(xs) >= 4.0
    assert np.allclose(w[outer, 1], 1.0)
    # linear fall-off over the last cell
    ramp = (np.abs(xs) > 3.0) & (np.abs(xs) < 4.0)
    assert np.allclose(w[ramp, 0], 4.0 - np.abs(xs[ramp]))
    want = PI * (w[:, 0] * 0.5 ** 5 + w[:, 1] * 0.8 ** 5)
    assert np.allclose(E[:, 0], want, rtol=1e-12)
