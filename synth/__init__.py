"""Seeded synthetic inputs for the probe-based irradiance field.

This module builds the inputs that both the CUDA path and the FP64 oracle
consume: triangle scenes, lights, probe-volume descriptors, query points and
camera descriptions.  It holds none of the method's arithmetic (no ray
directions, no intersection, no blending, no query); it only draws seeded
numbers and lays out geometry.

Every coordinate it emits is exactly representable in float32, so the FP32
device path and the FP64 oracle see the same geometry bit for bit.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) evaluated in counter form, so a
stream is fully determined by its seed on every machine and numpy version.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


class Rng:
    """Counter-based SplitMix64 stream: draw k returns mix64(seed + (k+1)*golden)."""

    def __init__(self, seed: int):
        self.seed = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def bits(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix64(self.seed + k * _GOLDEN)

    def uniform(self, n: int, lo=0.0, hi=1.0) -> np.ndarray:
        u = (self.bits(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int) -> np.ndarray:
        u1 = self.uniform(n)
        u2 = self.uniform(n)
        return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)

    def unit_vectors(self, n: int) -> np.ndarray:
        # uniform on S^2: z uniform in [-1,1], azimuth uniform (Archimedes)
        z = self.uniform(n, -1.0, 1.0)
        phi = self.uniform(n, 0.0, 2.0 * np.pi)
        r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
        v = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
        return f32(v)


def f32(a) -> np.ndarray:
    """Round to float32 and return as float64 (exactly float32-representable)."""
    return np.asarray(a, dtype=np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# Scene container
# --------------------------------------------------------------------------

CASTS_SHADOW = 1


@dataclass
class Scene:
    """Triangle scene. Triangles are counter-clockwise seen from their front side."""

    verts: np.ndarray            # [V,3] float64, float32-exact
    tris: np.ndarray             # [T,3] int32
    tri_object: np.ndarray       # [T] int32
    object_albedo: np.ndarray    # [O,3] float64
    object_flags: np.ndarray     # [O] int32, bit0 = casts shadow
    tri_emitter: np.ndarray      # [T] int32, -1 = not emissive
    emitter_radiance: np.ndarray  # [E,3] float64
    name: str = ""

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


@dataclass
class Lights:
    """One directional light plus a linear sky L(w) = a + b (w . up)."""

    sun_dir: np.ndarray = field(default_factory=lambda: np.zeros(3))   # direction the light travels
    sun_irradiance: np.ndarray = field(default_factory=lambda: np.zeros(3))
    sky_a: np.ndarray = field(default_factory=lambda: np.zeros(3))
    sky_b: np.ndarray = field(default_factory=lambda: np.zeros(3))
    sky_up: np.ndarray = field(default_factory=lambda: np.array([0.0, 1.0, 0.0]))


@dataclass
class VolumeDesc:
    """Probe grid and update parameters (one volume)."""

    origin: tuple = (0.0, 0.0, 0.0)
    spacing: tuple = (1.0, 1.0, 1.0)
    counts: tuple = (2, 2, 2)
    rays_per_probe: int = 64
    irr_n: int = 6            # interior irradiance texels per side
    dist_n: int = 14          # interior distance texels per side
    hysteresis_irr: float = 0.97
    hysteresis_vis: float = 0.97
    gamma: float = 5.0
    self_shadow_bias: float = 0.3
    dist_cos_power: float = 50.0
    t_max: float = -1.0       # <0: 2 * |cell diagonal|
    state_machine: int = 1
    seed: int = 0
    thr_low: float = 0.25
    thr_high: float = 0.8
    thr_step: float = 0.15
    tracking: int = 0
    optimizer_iters: int = 0  # position-optimizer iterations for new probes (Sec. 5; the paper uses 5)
    offset_limit: float = 0.45  # largest probe offset per axis, fraction of the spacing
    converge_batches: int = 0  # optional converge pass for new probes (Sec. 6.3), batches of R rays

    def resolved_t_max(self) -> float:
        if self.t_max >= 0:
            return float(self.t_max)
        return float(2.0 * np.linalg.norm(np.asarray(self.spacing, dtype=np.float64)))

    @property
    def n_probes(self) -> int:
        return int(self.counts[0] * self.counts[1] * self.counts[2])


class _Builder:
    def __init__(self):
        self.verts: list = []
        self.tris: list = []
        self.tri_object: list = []
        self.tri_emitter: list = []

    def quad(self, corners, normal, obj, emitter=-1):
        """Two triangles over 4 corners in cyclic order; winding faces `normal`."""
        c = [np.asarray(p, dtype=np.float64) for p in corners]
        base = len(self.verts)
        self.verts.extend(c)
        for (a, b, d) in ((0, 1, 2), (0, 2, 3)):
            cr = np.cross(c[b] - c[a], c[d] - c[a])
            if np.dot(cr, normal) < 0:
                b, d = d, b
            self.tris.append((base + a, base + b, base + d))
            self.tri_object.append(obj)
            self.tri_emitter.append(emitter)

    def box(self, lo, hi, obj, inward=False):
        """Axis-aligned box as 12 triangles, fronts facing out (or in)."""
        lo = np.asarray(lo, dtype=np.float64)
        hi = np.asarray(hi, dtype=np.float64)
        s = -1.0 if inward else 1.0
        for ax in range(3):
            u, v = (ax + 1) % 3, (ax + 2) % 3
            for side, val in ((-1.0, lo[ax]), (1.0, hi[ax])):
                pts = []
                for (a, b) in ((0, 0), (1, 0), (1, 1), (0, 1)):
                    p = np.zeros(3)
                    p[ax] = val
                    p[u] = lo[u] if a == 0 else hi[u]
                    p[v] = lo[v] if b == 0 else hi[v]
                    pts.append(p)
                n = np.zeros(3)
                n[ax] = side * s
                self.quad(pts, n, obj)

    def boxes(self, lo, hi, obj):
        """Many outward axis-aligned boxes at once (same triangle layout as box())."""
        lo = np.asarray(lo, dtype=np.float64).reshape(-1, 3)
        hi = np.asarray(hi, dtype=np.float64).reshape(-1, 3)
        nb = len(lo)
        obj = np.broadcast_to(np.asarray(obj, dtype=np.int32), (nb,))
        verts, tris = [], []
        base0 = len(self.verts)
        for ax in range(3):
            u, v = (ax + 1) % 3, (ax + 2) % 3
            for side, val in ((-1.0, lo[:, ax]), (1.0, hi[:, ax])):
                pts = np.zeros((nb, 4, 3))
                for c, (a, b) in enumerate(((0, 0), (1, 0), (1, 1), (0, 1))):
                    pts[:, c, ax] = val
                    pts[:, c, u] = lo[:, u] if a == 0 else hi[:, u]
                    pts[:, c, v] = lo[:, v] if b == 0 else hi[:, v]
                n = np.zeros(3)
                n[ax] = side
                verts.append(pts)
                for (a, b, d) in ((0, 1, 2), (0, 2, 3)):
                    cr = np.cross(pts[:, b] - pts[:, a], pts[:, d] - pts[:, a])
                    ok = cr @ n >= 0
                    tb = np.where(ok, b, d)
                    td = np.where(ok, d, b)
                    tris.append(np.stack([np.full(nb, a), tb, td], axis=1))
        # verts: 6 faces x [nb,4,3] -> per box contiguous 24 verts
        V = np.stack(verts, axis=1).reshape(nb, 24, 3)
        T = np.stack(tris, axis=1).reshape(nb, 6, 2, 3)
        T = T + (np.arange(6) * 4)[None, :, None, None]
        T = T.reshape(nb, 12, 3) + (base0 + 24 * np.arange(nb))[:, None, None]
        self.verts.extend(list(V.reshape(-1, 3)))
        self.tris.extend([tuple(t) for t in T.reshape(-1, 3)])
        self.tri_object.extend(list(np.repeat(obj, 12)))
        self.tri_emitter.extend([-1] * (12 * nb))

    def finish(self, object_albedo, object_flags, emitter_radiance, name) -> Scene:
        return Scene(
            verts=f32(np.array(self.verts, dtype=np.float64).reshape(-1, 3)),
            tris=np.array(self.tris, dtype=np.int32).reshape(-1, 3),
            tri_object=np.array(self.tri_object, dtype=np.int32),
            object_albedo=np.asarray(object_albedo, dtype=np.float64).reshape(-1, 3),
            object_flags=np.asarray(object_flags, dtype=np.int32),
            tri_emitter=np.array(self.tri_emitter, dtype=np.int32),
            emitter_radiance=np.asarray(emitter_radiance, dtype=np.float64).reshape(-1, 3),
            name=name,
        )


def _normalize(v):
    v = np.asarray(v, dtype=np.float64)
    return f32(v / np.linalg.norm(v))


# --------------------------------------------------------------------------
# Workload 1: closed 10 m room, 32 box occluders, one emissive quad (~398 tris)
# --------------------------------------------------------------------------

def room_scene(seed: int = 1001, n_boxes: int = 32, albedo: float = 0.7,
               emit: float = 5.0) -> Scene:
    """10 m room shell (inward, casts no shadow so sunlight enters), seeded box
    occluders and a 2x2 m emissive quad on the x=0 wall facing +x."""
    rng = Rng(seed)
    b = _Builder()
    b.box((0, 0, 0), (10, 10, 10), obj=0, inward=True)
    centres = rng.uniform(3 * n_boxes, 1.0, 9.0).reshape(n_boxes, 3)
    halves = rng.uniform(3 * n_boxes, 0.25, 1.0).reshape(n_boxes, 3)
    for k in range(n_boxes):
        lo = f32(centres[k] - halves[k])
        hi = f32(centres[k] + halves[k])
        b.box(lo, hi, obj=1 + k)
    q = n_boxes + 1
    x = f32(0.01)
    b.quad([(x, 4, 4), (x, 6, 4), (x, 6, 6), (x, 4, 6)], np.array([1.0, 0, 0]), obj=q, emitter=0)
    n_obj = n_boxes + 2
    alb = np.full((n_obj, 3), albedo)
    flags = np.full(n_obj, CASTS_SHADOW, dtype=np.int32)
    flags[0] = 0
    return b.finish(alb, flags, [[emit, emit, emit]], "room")


def room_lights() -> Lights:
    return Lights(sun_dir=_normalize([0.3, -1.0, 0.2]), sun_irradiance=np.full(3, 3.0),
                  sky_a=np.zeros(3), sky_b=np.zeros(3), sky_up=np.array([0.0, 1.0, 0.0]))


def room_volume(**kw) -> VolumeDesc:
    d = dict(origin=(0.625, 0.625, 0.625), spacing=(1.25, 1.25, 1.25), counts=(8, 8, 8),
             rays_per_probe=64, hysteresis_irr=0.0, hysteresis_vis=0.0, seed=2001)
    d.update(kw)
    return VolumeDesc(**d)


def room_queries(seed: int = 3001, n: int = 4096):
    """Query points uniform in [0.625, 9.375]^3 with normals uniform on the sphere."""
    rng = Rng(seed)
    pos = f32(rng.uniform(3 * n, 0.625, 9.375).reshape(n, 3))
    nrm = rng.unit_vectors(n)
    camera = np.array([5.0, 5.0, 5.0])
    return pos, nrm, camera


# --------------------------------------------------------------------------
# Workload 2: procedural city, 128x128 lots of 4 m, one box per lot (196,610 tris)
# --------------------------------------------------------------------------

def city_scene(seed: int = 1002, lots: int = 128, lot: float = 4.0, albedo: float = 0.7) -> Scene:
    rng = Rng(seed)
    b = _Builder()
    half = lots * lot / 2.0
    b.quad([(-half, 0, -half), (half, 0, -half), (half, 0, half), (-half, 0, half)],
           np.array([0.0, 1.0, 0.0]), obj=0)
    n = lots * lots
    fx = rng.uniform(n, 2.0, 3.5)
    fz = rng.uniform(n, 2.0, 3.5)
    h = rng.uniform(n, 4.0, 40.0)
    iz, ix = np.meshgrid(np.arange(lots), np.arange(lots), indexing="ij")
    cx = (-half + (ix.ravel() + 0.5) * lot)
    cz = (-half + (iz.ravel() + 0.5) * lot)
    lo = f32(np.stack([cx - fx / 2, np.zeros(n), cz - fz / 2], axis=1))
    hi = f32(np.stack([cx + fx / 2, h, cz + fz / 2], axis=1))
    b.boxes(lo, hi, obj=1)
    alb = np.full((2, 3), albedo)
    flags = np.full(2, CASTS_SHADOW, dtype=np.int32)
    return b.finish(alb, flags, np.zeros((0, 3)), "city")


def city_lights() -> Lights:
    return Lights(sun_dir=_normalize([0.3, -1.0, 0.5]), sun_irradiance=np.full(3, 3.0),
                  sky_a=np.full(3, 0.2), sky_b=np.full(3, 0.1), sky_up=np.array([0.0, 1.0, 0.0]))


def city_volume(**kw) -> VolumeDesc:
    d = dict(origin=(-31.0, 1.0, -31.0), spacing=(2.0, 2.0, 2.0), counts=(32, 16, 32),
             rays_per_probe=256, hysteresis_irr=0.97, hysteresis_vis=0.97, seed=2002)
    d.update(kw)
    return VolumeDesc(**d)


@dataclass
class PinholeCamera:
    """Pinhole camera: position, yaw-free forward tilted by `pitch_deg`, vertical FOV."""

    position: np.ndarray
    forward: np.ndarray
    up: np.ndarray
    vfov_deg: float
    width: int
    height: int


def city_camera(width: int = 1920, height: int = 1080) -> PinholeCamera:
    pitch = np.deg2rad(-10.0)
    fwd = _normalize([0.0, np.sin(pitch), np.cos(pitch)])
    return PinholeCamera(position=f32([0.0, 12.0, -28.0]), forward=fwd,
                         up=np.array([0.0, 1.0, 0.0]), vfov_deg=60.0, width=width, height=height)


def camera_ray_dirs(cam: PinholeCamera) -> np.ndarray:
    """Unit directions through pixel centres, row-major [H*W,3] float32-exact."""
    f = np.asarray(cam.forward, dtype=np.float64)
    r = np.cross(f, cam.up)
    r /= np.linalg.norm(r)
    u = np.cross(r, f)
    th = np.tan(np.deg2rad(cam.vfov_deg) / 2.0)
    aspect = cam.width / cam.height
    ys, xs = np.meshgrid(np.arange(cam.height), np.arange(cam.width), indexing="ij")
    sx = ((xs + 0.5) / cam.width * 2.0 - 1.0) * th * aspect
    sy = (1.0 - (ys + 0.5) / cam.height * 2.0) * th
    d = f[None, None, :] + sx[..., None] * r[None, None, :] + sy[..., None] * u[None, None, :]
    d /= np.linalg.norm(d, axis=-1, keepdims=True)
    return f32(d.reshape(-1, 3))


def surface_points(scene: Scene, n: int, seed: int, offset: float = 1e-3,
                   region_lo=None, region_hi=None):
    """Area-weighted random points on front faces, lifted `offset` along the
    geometric normal; optional axis-aligned region filter (rejection)."""
    rng = Rng(seed)
    v = scene.verts
    t = scene.tris
    e1 = v[t[:, 1]] - v[t[:, 0]]
    e2 = v[t[:, 2]] - v[t[:, 0]]
    cr = np.cross(e1, e2)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    cdf = np.cumsum(area)
    cdf /= cdf[-1]
    out_p, out_n = [], []
    got = 0
    while got < n:
        m = 4 * (n - got) + 64
        tri = np.searchsorted(cdf, rng.uniform(m), side="right").clip(0, len(t) - 1)
        a = rng.uniform(m)
        bb = rng.uniform(m)
        flip = a + bb > 1.0
        a = np.where(flip, 1.0 - a, a)
        bb = np.where(flip, 1.0 - bb, bb)
        nn = cr[tri] / np.linalg.norm(cr[tri], axis=1, keepdims=True)
        p = v[t[tri, 0]] + a[:, None] * e1[tri] + bb[:, None] * e2[tri] + offset * nn
        keep = np.ones(m, dtype=bool)
        if region_lo is not None:
            keep &= np.all(p >= np.asarray(region_lo), axis=1)
        if region_hi is not None:
            keep &= np.all(p <= np.asarray(region_hi), axis=1)
        out_p.append(p[keep])
        out_n.append(nn[keep])
        got += int(keep.sum())
    return f32(np.concatenate(out_p)[:n]), f32(np.concatenate(out_n)[:n])


# --------------------------------------------------------------------------
# Small analytic scenes used to pin the oracle
# --------------------------------------------------------------------------

def empty_scene() -> Scene:
    return Scene(verts=np.zeros((0, 3)), tris=np.zeros((0, 3), dtype=np.int32),
                 tri_object=np.zeros(0, dtype=np.int32), object_albedo=np.full((1, 3), 0.5),
                 object_flags=np.ones(1, dtype=np.int32), tri_emitter=np.zeros(0, dtype=np.int32),
                 emitter_radiance=np.zeros((0, 3)), name="empty")


def box_room(lo, hi, albedo=0.5, emit=None, casts_shadow=1) -> Scene:
    """Closed box seen from inside; with `emit`, every triangle is an emitter."""
    b = _Builder()
    b.box(lo, hi, obj=0, inward=True)
    sc = b.finish(np.full((1, 3), albedo), [casts_shadow], np.zeros((0, 3)), "box_room")
    if emit is not None:
        sc.tri_emitter = np.zeros(sc.n_tris, dtype=np.int32)
        sc.emitter_radiance = np.asarray(emit, dtype=np.float64).reshape(1, 3)
    return sc


def solid_box(lo, hi, albedo=0.5) -> Scene:
    b = _Builder()
    b.box(lo, hi, obj=0)
    return b.finish(np.full((1, 3), albedo), [CASTS_SHADOW], np.zeros((0, 3)), "solid_box")


def icosphere(radius: float, subdiv: int, inward: bool = True) -> Scene:
    """Icosphere with vertices on the sphere; faces toward the centre if inward."""
    phi = (1.0 + 5 ** 0.5) / 2.0
    vs = [(-1, phi, 0), (1, phi, 0), (-1, -phi, 0), (1, -phi, 0), (0, -1, phi), (0, 1, phi),
          (0, -1, -phi), (0, 1, -phi), (phi, 0, -1), (phi, 0, 1), (-phi, 0, -1), (-phi, 0, 1)]
    vs = [np.asarray(v, dtype=np.float64) / np.linalg.norm(v) for v in vs]
    fs = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
          (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
          (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}
        nf = []

        def mid(a, b):
            k = (min(a, b), max(a, b))
            if k not in cache:
                m = vs[a] + vs[b]
                vs.append(m / np.linalg.norm(m))
                cache[k] = len(vs) - 1
            return cache[k]
        for (a, b, c) in fs:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        fs = nf
    V = np.array(vs) * radius
    F = np.array(fs, dtype=np.int32)
    # orient: outward means (v1-v0)x(v2-v0) . centroid > 0
    cr = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    outward = np.einsum("ij,ij->i", cr, V[F].mean(axis=1)) > 0
    want_out = not inward
    flip = outward != want_out
    F[flip] = F[flip][:, [0, 2, 1]]
    T = len(F)
    return Scene(verts=f32(V), tris=F, tri_object=np.zeros(T, dtype=np.int32),
                 object_albedo=np.full((1, 3), 0.5), object_flags=np.ones(1, dtype=np.int32),
                 tri_emitter=np.full(T, -1, dtype=np.int32), emitter_radiance=np.zeros((0, 3)),
                 name="icosphere")


# --------------------------------------------------------------------------
# Workload 3: terrain + buildings (~1M tris), four camera-tracking cascades
# --------------------------------------------------------------------------

def _terrain_params(seed):
    rng = Rng(seed)
    k = 8
    fx = rng.uniform(k, 0.002, 0.02)
    fz = rng.uniform(k, 0.002, 0.02)
    px = rng.uniform(k, 0.0, 2 * np.pi)
    pz = rng.uniform(k, 0.0, 2 * np.pi)
    amp = rng.uniform(k, 0.5, 1.0)
    return fx, fz, px, pz, amp


def terrain_height(x, z, seed: int = 1003, amplitude: float = 20.0):
    """Seeded sum of 8 sinusoid products, peak amplitude `amplitude` metres."""
    fx, fz, px, pz, amp = _terrain_params(seed)
    x = np.asarray(x, dtype=np.float64)[..., None]
    z = np.asarray(z, dtype=np.float64)[..., None]
    h = (amp * np.sin(fx * x + px) * np.cos(fz * z + pz)).sum(-1)
    return amplitude * h / amp.sum()


def terrain_scene(seed: int = 1003, quads: int = 512, size: float = 1024.0, n_boxes: int = 43690,
                  albedo: float = 0.7) -> Scene:
    """Heightfield of quads x quads cells over size x size metres (faces up),
    plus seeded boxes standing on it (footprint U[4,16] m, height U[4,40] m)."""
    rng = Rng(seed + 7)
    n = quads + 1
    xs = np.linspace(-size / 2, size / 2, n)
    X, Z = np.meshgrid(xs, xs, indexing="ij")
    Y = terrain_height(X, Z, seed)
    V = f32(np.stack([X, Y, Z], axis=-1).reshape(-1, 3))
    i, j = np.meshgrid(np.arange(quads), np.arange(quads), indexing="ij")
    a = (i * n + j).ravel()
    b = a + n          # +x
    c = a + n + 1      # +x +z
    d = a + 1          # +z
    # (a, d, c) and (a, c, b): counter-clockwise seen from +y
    T = np.concatenate([np.stack([a, d, c], 1), np.stack([a, c, b], 1)]).astype(np.int32)
    bld = _Builder()
    bld.verts = list(V)
    bld.tris = [tuple(t) for t in T]
    bld.tri_object = [0] * len(T)
    bld.tri_emitter = [-1] * len(T)
    cx = rng.uniform(n_boxes, -size / 2 + 10, size / 2 - 10)
    cz = rng.uniform(n_boxes, -size / 2 + 10, size / 2 - 10)
    fx = rng.uniform(n_boxes, 4.0, 16.0)
    fz = rng.uniform(n_boxes, 4.0, 16.0)
    hh = rng.uniform(n_boxes, 4.0, 40.0)
    base = terrain_height(cx, cz, seed) - 3.0
    lo = f32(np.stack([cx - fx / 2, base, cz - fz / 2], axis=1))
    hi = f32(np.stack([cx + fx / 2, base + 3.0 + hh, cz + fz / 2], axis=1))
    bld.boxes(lo, hi, obj=1)
    return bld.finish(np.full((2, 3), albedo), np.full(2, CASTS_SHADOW, dtype=np.int32), np.zeros((0, 3)),
                      "terrain")


def terrain_camera_path(frame: int, seed: int = 1003):
    """0.6 m per frame along +x with a sinusoidal z wobble, 10 m above the terrain."""
    x = -100.0 + 0.6 * frame
    z = 15.0 * np.sin(0.05 * frame)
    return f32([x, float(terrain_height(x, z, seed)) + 10.0, z])


def terrain_cascades(rays: int = 288, seed: int = 2003):
    """Four 32^3 tracking cascades at 1 / 2 / 4 / 8 m, densest first."""
    out = []
    for s in (1.0, 2.0, 4.0, 8.0):
        out.append(VolumeDesc(origin=(-15.5 * s, -15.5 * s, -15.5 * s), spacing=(s, s, s),
                              counts=(32, 32, 32), rays_per_probe=rays, hysteresis_irr=0.97,
                              hysteresis_vis=0.97, seed=seed, tracking=1))
    return out


# --------------------------------------------------------------------------
# Workload 5: interior for differentiation (~200k tris, 256 objects, 64 emitters)
# --------------------------------------------------------------------------

def interior_scene(seed: int = 1005, n_boxes: int = 16000, n_objects: int = 256, n_emitters: int = 64):
    """40 x 20 x 40 m shell (object 0) with seeded boxes grouped into objects
    1..n_objects-1 and emissive quads on the ceiling and walls.  Returns the
    scene and its hidden ground-truth materials (albedo [O,3], radiance [E,3])."""
    rng = Rng(seed)
    b = _Builder()
    b.box((-20, 0, -20), (20, 20, 20), obj=0, inward=True)
    c = np.stack([rng.uniform(n_boxes, -19, 19), rng.uniform(n_boxes, 0.5, 18), rng.uniform(n_boxes, -19, 19)], 1)
    h = np.stack([rng.uniform(n_boxes, 0.1, 0.6), rng.uniform(n_boxes, 0.1, 0.6), rng.uniform(n_boxes, 0.1, 0.6)], 1)
    obj = 1 + (np.arange(n_boxes) % (n_objects - 1))
    b.boxes(f32(c - h), f32(c + h), obj=obj.astype(np.int32))
    for k in range(n_emitters):
        u = rng.uniform(2, -17, 17)
        if k % 2 == 0:      # ceiling, facing down
            y = f32(19.99)
            b.quad([(u[0], y, u[1]), (u[0] + 1.5, y, u[1]), (u[0] + 1.5, y, u[1] + 1.5), (u[0], y, u[1] + 1.5)],
                   np.array([0.0, -1, 0]), obj=n_objects, emitter=k)
        else:               # x = -20 wall, facing +x
            x = f32(-19.99)
            yy = 2.0 + abs(u[0]) / 17 * 15
            b.quad([(x, yy, u[1]), (x, yy + 1.5, u[1]), (x, yy + 1.5, u[1] + 1.5), (x, yy, u[1] + 1.5)],
                   np.array([1.0, 0, 0]), obj=n_objects, emitter=k)
    truth_alb = rng.uniform(3 * (n_objects + 1), 0.2, 0.9).reshape(-1, 3)
    truth_em = np.repeat(rng.uniform(n_emitters, 0.1, 2.0)[:, None], 3, axis=1)
    sc = b.finish(truth_alb, np.ones(n_objects + 1, dtype=np.int32), truth_em, "interior")
    return sc, truth_alb, truth_em


def interior_volume(**kw) -> VolumeDesc:
    d = dict(origin=(-18.75, 1.25, -18.75), spacing=(2.5, 2.5, 2.5), counts=(16, 8, 16), rays_per_probe=128,
             hysteresis_irr=0.0, hysteresis_vis=0.0, gamma=1.0, state_machine=0, seed=2005)
    d.update(kw)
    return VolumeDesc(**d)
