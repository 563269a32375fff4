"""Python binding of the FP64 CPU oracle (``ddgi_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product package never imports
it.  The oracle is written from the paper (Majercik et al., JCGT 2021): see
the header of ``ddgi_oracle.c`` for the section each function follows and the
readings taken where the paper is silent.

Array conventions (all float64, C-contiguous):
  states   uint8  [P]                     probe states (0 uninit, 1 off, 2 sleeping,
                                          3 newly vigilant, 4 vigilant)
  irr      [P, irr_n+2, irr_n+2, 3]       encoded irradiance, bordered tiles
  dist     [P, dist_n+2, dist_n+2, 2]     mean distance and mean squared distance
Probe index p = i + cx*(j + cy*k) over the stored (physical) grid.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ddgi_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libddgi_oracle.so")
_lock = threading.Lock()
_lib = None

UNINIT, OFF, SLEEPING, NEWLY_VIGILANT, VIGILANT, NEWLY_AWAKE, AWAKE = 0, 1, 2, 3, 4, 5, 6

_dp = C.POINTER(C.c_double)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_u8p = C.POINTER(C.c_uint8)


class OrScene(C.Structure):
    _fields_ = [("verts", _dp), ("n_verts", C.c_int64), ("tris", _i32p), ("n_tris", C.c_int64),
                ("tri_object", _i32p), ("object_albedo", _dp), ("object_flags", _i32p),
                ("tri_emitter", _i32p), ("emitter_radiance", _dp)]


class OrLights(C.Structure):
    _fields_ = [("sun_dir", C.c_double * 3), ("sun_irradiance", C.c_double * 3),
                ("sky_a", C.c_double * 3), ("sky_b", C.c_double * 3), ("sky_up", C.c_double * 3)]


class OrVolume(C.Structure):
    _fields_ = [("origin", C.c_double * 3), ("spacing", C.c_double * 3), ("counts", C.c_int64 * 3),
                ("rays", C.c_int64), ("irr_n", C.c_int64), ("dist_n", C.c_int64),
                ("hyst_irr", C.c_double), ("hyst_vis", C.c_double), ("gamma", C.c_double),
                ("bias_B", C.c_double), ("cos_power", C.c_double), ("t_max", C.c_double),
                ("thr_low", C.c_double), ("thr_high", C.c_double), ("thr_step", C.c_double),
                ("state_machine", C.c_int64), ("seed", C.c_uint64), ("shift", C.c_int64 * 3),
                ("blend_lo", C.c_double * 3), ("blend_hi", C.c_double * 3),
                ("offsets", C.POINTER(C.c_double)), ("opt_iters", C.c_int64), ("offset_limit", C.c_double),
                ("dyn_boxes", C.POINTER(C.c_double)), ("n_dyn", C.c_int64),
                ("converge_batches", C.c_int64)]


def build(force: bool = False, extra_flags=()) -> str:
    """Compile the oracle with gcc (no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ddgi_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", *extra_flags, _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def build_variant(src: str, path: str) -> C.CDLL:
    """Compile another source file with the oracle's flags and load it (the
    mutation tests use this to plant mistakes in a temporary copy)."""
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
           "-I", _HERE, src, "-o", path, "-lm"]
    subprocess.run(cmd, check=True)
    return _declare(C.CDLL(path))


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


class use_library:
    """Context manager: route this module's wrappers through another build."""

    def __init__(self, handle):
        self.handle = handle

    def __enter__(self):
        global _lib
        lib()
        self.saved = _lib
        _lib = self.handle
        return self.handle

    def __exit__(self, *exc):
        global _lib
        _lib = self.saved
        return False


def _declare(lib):
    lib.or_rotation.argtypes = [C.c_uint64, C.c_int64, _dp]
    lib.or_sf_dir.argtypes = [C.c_int64, C.c_int64, _dp]
    lib.or_frame_dirs.argtypes = [C.c_uint64, C.c_int64, C.c_int64, _dp]
    lib.or_splitmix64_next.argtypes = [C.POINTER(C.c_uint64)]
    lib.or_splitmix64_next.restype = C.c_uint64
    lib.or_oct_encode.argtypes = [_dp, _dp]
    lib.or_oct_decode.argtypes = [_dp, _dp]
    lib.or_texel_dir.argtypes = [C.c_int64, C.c_int64, C.c_int64, _dp]
    lib.or_border_copy.argtypes = [_dp, C.c_int64, C.c_int64]
    lib.or_sample_bilinear.argtypes = [_dp, C.c_int64, C.c_int64, _dp, _dp]
    lib.or_trace_batch.argtypes = [C.POINTER(OrScene), C.c_int64, _dp, _dp, _dp, _i64p, _i32p]
    lib.or_any_hit_shadow.argtypes = [C.POINTER(OrScene), _dp, _dp]
    lib.or_any_hit_shadow.restype = C.c_int
    lib.or_probe_phys.argtypes = [C.POINTER(OrVolume), C.c_int64, C.c_int64, C.c_int64]
    lib.or_probe_phys.restype = C.c_int64
    lib.or_classify.argtypes = [C.POINTER(OrScene), C.POINTER(OrVolume), C.c_int64, C.c_int64,
                                _i64p, _u8p, _i32p, _dp]
    lib.or_update.argtypes = [C.POINTER(OrScene), C.POINTER(OrLights), C.POINTER(OrVolume),
                              C.c_int64, C.c_double, C.c_double, _u8p, _dp, _dp, C.c_int64,
                              _i64p, _dp]
    lib.or_query.argtypes = [C.POINTER(OrVolume), _u8p, _dp, _dp, C.c_int64, _dp, _dp, _dp, _dp, _dp]
    lib.or_optimize.argtypes = [C.c_void_p, C.POINTER(OrVolume), C.c_int64, C.c_int64, _i64p]
    lib.or_query_glossy.argtypes = [C.POINTER(OrVolume), _u8p, _dp, _dp, C.c_int64, _dp, _dp, _dp, _dp]
    lib.or_query_cascade.argtypes = [C.c_int64, C.POINTER(OrVolume), C.POINTER(_u8p),
                                     C.POINTER(_dp), C.POINTER(_dp), C.c_int64, _dp, _dp, _dp,
                                     _dp, _dp]
    lib.or_diff.argtypes = [C.POINTER(OrScene), C.POINTER(OrLights), C.POINTER(OrVolume), C.c_int64,
                            C.c_int64, C.c_int64, _dp, _dp, _dp, _dp, _dp, _dp, _dp, C.c_int64, C.c_int64]
    lib.or_query_texel_grad.argtypes = [C.POINTER(OrVolume), _u8p, _dp, _dp, C.c_int64, _dp, _dp, _dp, _dp,
                                        C.c_int, _dp]
    lib.or_tracking_scroll.argtypes = [C.POINTER(OrVolume), _dp, _u8p, _dp, _dp]
    lib.or_tracking_scroll.restype = C.c_int64
    lib.or_update_cascade.argtypes = [C.POINTER(OrScene), C.POINTER(OrLights), C.c_int64,
                                      C.POINTER(OrVolume), C.c_int64, C.c_double, C.c_double,
                                      C.POINTER(_u8p), C.POINTER(_dp), C.POINTER(_dp), _i64p,
                                      C.POINTER(_i64p), C.POINTER(_dp)]
    return lib


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _declare(C.CDLL(_LIB_PATH))
    return _lib


def _ptr(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a.reshape(shape) if shape is not None else a


# --------------------------------------------------------------------------
# Structure builders
# --------------------------------------------------------------------------

class SceneHandle:
    """Keeps the numpy buffers alive behind an OrScene."""

    def __init__(self, scene):
        self.verts = _f64(scene.verts, (-1, 3))
        self.tris = np.ascontiguousarray(scene.tris, dtype=np.int32).reshape(-1, 3)
        self.tri_object = np.ascontiguousarray(scene.tri_object, dtype=np.int32)
        self.object_albedo = _f64(scene.object_albedo, (-1, 3))
        self.object_flags = np.ascontiguousarray(scene.object_flags, dtype=np.int32)
        self.tri_emitter = np.ascontiguousarray(scene.tri_emitter, dtype=np.int32)
        em = _f64(scene.emitter_radiance).reshape(-1, 3)
        self.emitter_radiance = em if em.size else np.zeros((1, 3))
        self.s = OrScene(_ptr(self.verts, _dp), len(self.verts), _ptr(self.tris, _i32p),
                         len(self.tris), _ptr(self.tri_object, _i32p),
                         _ptr(self.object_albedo, _dp), _ptr(self.object_flags, _i32p),
                         _ptr(self.tri_emitter, _i32p), _ptr(self.emitter_radiance, _dp))


def make_lights(lights) -> OrLights:
    L = OrLights()
    for name in ("sun_dir", "sun_irradiance", "sky_a", "sky_b", "sky_up"):
        getattr(L, name)[:] = [float(x) for x in np.asarray(getattr(lights, name), dtype=np.float64)]
    return L


def make_volume(desc, shift=(0, 0, 0), origin=None, blend_lo=None, blend_hi=None, offsets=None,
                dyn_boxes=None) -> OrVolume:
    """`offsets`: float64 [P, 3] probe offsets (Sec. 5), written in place by the
    position optimizer; `dyn_boxes`: float64 [n, 6] dynamic-object boxes (lo,
    hi) that wake sleeping probes (Sec. 6.3).  The caller keeps both alive
    while the struct is used."""
    v = OrVolume()
    if dyn_boxes is not None and len(dyn_boxes):
        assert dyn_boxes.dtype == np.float64 and dyn_boxes.flags.c_contiguous and dyn_boxes.shape[1] == 6
        v.dyn_boxes = dyn_boxes.ctypes.data_as(C.POINTER(C.c_double))
        v.n_dyn = len(dyn_boxes)
    if offsets is not None:
        assert offsets.dtype == np.float64 and offsets.flags.c_contiguous and offsets.shape == (desc.n_probes, 3)
        v.offsets = offsets.ctypes.data_as(C.POINTER(C.c_double))
    v.opt_iters = int(getattr(desc, "optimizer_iters", 0))
    v.offset_limit = float(getattr(desc, "offset_limit", 0.45))
    v.converge_batches = int(getattr(desc, "converge_batches", 0))
    org = desc.origin if origin is None else origin
    v.origin[:] = [float(x) for x in org]
    v.spacing[:] = [float(x) for x in desc.spacing]
    v.counts[:] = [int(x) for x in desc.counts]
    v.rays = int(desc.rays_per_probe)
    v.irr_n = int(desc.irr_n)
    v.dist_n = int(desc.dist_n)
    v.hyst_irr = float(desc.hysteresis_irr)
    v.hyst_vis = float(desc.hysteresis_vis)
    v.gamma = float(desc.gamma)
    v.bias_B = float(desc.self_shadow_bias)
    v.cos_power = float(desc.dist_cos_power)
    v.t_max = float(desc.resolved_t_max())
    v.thr_low = float(desc.thr_low)
    v.thr_high = float(desc.thr_high)
    v.thr_step = float(desc.thr_step)
    v.state_machine = int(desc.state_machine)
    v.seed = int(desc.seed)
    v.shift[:] = [int(x) for x in shift]
    org = np.asarray(org, dtype=np.float64)
    lo = org if blend_lo is None else np.asarray(blend_lo, dtype=np.float64)
    hi = (org + (np.asarray(desc.counts) - 1) * np.asarray(desc.spacing)) if blend_hi is None \
        else np.asarray(blend_hi, dtype=np.float64)
    v.blend_lo[:] = [float(x) for x in lo]
    v.blend_hi[:] = [float(x) for x in hi]
    return v


def new_offsets(desc):
    """Zero probe offsets [P, 3] (every probe on its grid point)."""
    return np.zeros((desc.n_probes, 3), dtype=np.float64)


def new_state(desc, initial=None):
    """Zero atlases; states UNINIT (or VIGILANT when the state machine is off)."""
    P = desc.n_probes
    if initial is None:
        initial = UNINIT if desc.state_machine else VIGILANT
    states = np.full(P, initial, dtype=np.uint8)
    irr = np.zeros((P, desc.irr_n + 2, desc.irr_n + 2, 3))
    dist = np.zeros((P, desc.dist_n + 2, desc.dist_n + 2, 2))
    return states, irr, dist


# --------------------------------------------------------------------------
# Function wrappers
# --------------------------------------------------------------------------

def rotation(seed: int, frame: int) -> np.ndarray:
    R = np.zeros(9)
    lib().or_rotation(C.c_uint64(seed), frame, _ptr(R, _dp))
    return R.reshape(3, 3)


def splitmix64(seed: int, n: int):
    st = C.c_uint64(seed)
    return [lib().or_splitmix64_next(C.byref(st)) for _ in range(n)]


def sf_dirs(n: int) -> np.ndarray:
    out = np.zeros((n, 3))
    for i in range(n):
        lib().or_sf_dir(i, n, _ptr(out[i], _dp))
    return out


def frame_dirs(seed: int, frame: int, n: int) -> np.ndarray:
    out = np.zeros((n, 3))
    lib().or_frame_dirs(C.c_uint64(seed), frame, n, _ptr(out, _dp))
    return out


def oct_encode(v) -> np.ndarray:
    v = _f64(v, (-1, 3))
    out = np.zeros((len(v), 2))
    L = lib()
    for k in range(len(v)):
        L.or_oct_encode(_ptr(v[k], _dp), _ptr(out[k], _dp))
    return out


def oct_decode(u) -> np.ndarray:
    u = _f64(u, (-1, 2))
    out = np.zeros((len(u), 3))
    L = lib()
    for k in range(len(u)):
        L.or_oct_decode(_ptr(u[k], _dp), _ptr(out[k], _dp))
    return out


def texel_dirs(n: int) -> np.ndarray:
    """[n, n, 3] directions of interior texels, indexed [row j, column i]."""
    out = np.zeros((n, n, 3))
    for j in range(n):
        for i in range(n):
            lib().or_texel_dir(i, j, n, _ptr(out[j, i], _dp))
    return out


def border_copy(tile: np.ndarray, n: int) -> np.ndarray:
    t = _f64(tile).copy()
    lib().or_border_copy(_ptr(t, _dp), n, t.shape[-1])
    return t


def sample_bilinear(tile: np.ndarray, n: int, dirs) -> np.ndarray:
    t = _f64(tile)
    Cn = t.shape[-1]
    d = _f64(dirs, (-1, 3))
    out = np.zeros((len(d), Cn))
    for k in range(len(d)):
        lib().or_sample_bilinear(_ptr(t, _dp), n, Cn, _ptr(d[k], _dp), _ptr(out[k], _dp))
    return out


def trace(scene_h: SceneHandle, o, d):
    o = _f64(o, (-1, 3))
    d = _f64(d, (-1, 3))
    n = len(o)
    t = np.zeros(n)
    tri = np.zeros(n, dtype=np.int64)
    bf = np.zeros(n, dtype=np.int32)
    lib().or_trace_batch(C.byref(scene_h.s), n, _ptr(o, _dp), _ptr(d, _dp), _ptr(t, _dp),
                         _ptr(tri, _i64p), _ptr(bf, _i32p))
    return t, tri, bf


def optimize(scene_h, desc, frame, probe_ids, offsets):
    """desc.optimizer_iters iterations of the probe position optimizer (Sec. 5)
    on the probes `probe_ids`, in place on `offsets` [P, 3]."""
    ids = np.ascontiguousarray(probe_ids, dtype=np.int64)
    v = make_volume(desc, offsets=offsets)
    lib().or_optimize(C.byref(scene_h.s), C.byref(v), frame, len(ids), _ptr(ids, _i64p))
    return offsets


def classify(scene_h, desc, frame, probe_ids, states, shift=(0, 0, 0), origin=None, offsets=None):
    ids = np.ascontiguousarray(probe_ids, dtype=np.int64)
    bf = np.zeros(len(ids), dtype=np.int32)
    dmin = np.zeros(len(ids))
    v = make_volume(desc, shift, origin, offsets=offsets)
    lib().or_classify(C.byref(scene_h.s), C.byref(v), frame, len(ids), _ptr(ids, _i64p),
                      _ptr(states, _u8p), _ptr(bf, _i32p), _ptr(dmin, _dp))
    return bf, dmin


def update(scene_h, lights, desc, frame, states, irr, dist, subset=None, irr_scale=1.0,
           vis_scale=1.0, want_rays=False, shift=(0, 0, 0), origin=None, offsets=None, dyn_boxes=None):
    """One update frame, in place on (states, irr, dist) and, with the position
    optimizer on, on `offsets` [P, 3].  Returns per-ray records [n_list, R, 4]
    (r, g, b, d) when want_rays (NaN for inactive probes)."""
    assert states.dtype == np.uint8 and states.flags.c_contiguous
    assert irr.dtype == np.float64 and irr.flags.c_contiguous
    assert dist.dtype == np.float64 and dist.flags.c_contiguous
    boxes = None if dyn_boxes is None else np.ascontiguousarray(dyn_boxes, dtype=np.float64).reshape(-1, 6)
    v = make_volume(desc, shift, origin, offsets=offsets, dyn_boxes=boxes)
    L = make_lights(lights)
    sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int64)
    n_list = desc.n_probes if sub is None else len(sub)
    rays = np.full((n_list, desc.rays_per_probe, 4), np.nan) if want_rays else None
    lib().or_update(C.byref(scene_h.s), C.byref(L), C.byref(v), frame, irr_scale, vis_scale,
                    _ptr(states, _u8p), _ptr(irr, _dp), _ptr(dist, _dp),
                    0 if sub is None else len(sub), _ptr(sub, _i64p), _ptr(rays, _dp))
    return rays


def query(desc, states, irr, dist, pos, nrm, camera, want_weights=False, shift=(0, 0, 0),
          origin=None, offsets=None):
    pos = _f64(pos, (-1, 3))
    nrm = _f64(nrm, (-1, 3))
    cam = _f64(camera, (3,))
    n = len(pos)
    out = np.zeros((n, 3))
    w = np.zeros((n, 8)) if want_weights else None
    v = make_volume(desc, shift, origin, offsets=offsets)
    lib().or_query(C.byref(v), _ptr(states, _u8p), _ptr(_f64(irr), _dp), _ptr(_f64(dist), _dp),
                   n, _ptr(pos, _dp), _ptr(nrm, _dp), _ptr(cam, _dp), _ptr(out, _dp), _ptr(w, _dp))
    return (out, w) if want_weights else out


def query_texel_grad(desc, states, irr, dist, pos, nrm, camera, dE, fold=False, offsets=None):
    """Gradient of sum(dE * E), E = query(...), with respect to every stored
    irradiance texel [P, n+2, n+2, 3] (exact: the query's weights do not
    involve irradiance texels); fold adds border gradients to the interior
    texels they copy and zeroes the borders."""
    pos = _f64(pos, (-1, 3))
    nrm = _f64(nrm, (-1, 3))
    dE = _f64(dE, (-1, 3))
    cam = _f64(camera, (3,))
    g = np.zeros((desc.n_probes, desc.irr_n + 2, desc.irr_n + 2, 3))
    v = make_volume(desc, offsets=offsets)
    lib().or_query_texel_grad(C.byref(v), _ptr(states, _u8p), _ptr(_f64(irr), _dp), _ptr(_f64(dist), _dp), len(pos),
                              _ptr(pos, _dp), _ptr(nrm, _dp), _ptr(cam, _dp), _ptr(dE, _dp), int(bool(fold)),
                              _ptr(g, _dp))
    return g


def query_glossy(desc, states, irr, dist, pos, nrm, dirs, shift=(0, 0, 0), origin=None, offsets=None):
    """Second-order glossy lookup (Sec. 4.4): prefiltered radiance M [n, 3] at
    reflection-ray hits `pos` (normals `nrm`) reached along unit `dirs`,
    read in the mirror direction."""
    pos = _f64(pos, (-1, 3))
    nrm = _f64(nrm, (-1, 3))
    dirs = _f64(dirs, (-1, 3))
    n = len(pos)
    out = np.zeros((n, 3))
    v = make_volume(desc, shift, origin, offsets=offsets)
    lib().or_query_glossy(C.byref(v), _ptr(states, _u8p), _ptr(_f64(irr), _dp), _ptr(_f64(dist), _dp),
                          n, _ptr(pos, _dp), _ptr(nrm, _dp), _ptr(dirs, _dp), _ptr(out, _dp))
    return out


def query_cascade(vol_structs, states_list, irr_list, dist_list, pos, nrm, camera,
                  want_weights=False):
    pos = _f64(pos, (-1, 3))
    nrm = _f64(nrm, (-1, 3))
    cam = _f64(camera, (3,))
    n = len(pos)
    k = len(vol_structs)
    vols = (OrVolume * k)(*vol_structs)
    irr_c = [_f64(a) for a in irr_list]
    dist_c = [_f64(a) for a in dist_list]
    sp = (_u8p * k)(*[_ptr(s, _u8p) for s in states_list])
    ip = (_dp * k)(*[_ptr(a, _dp) for a in irr_c])
    dp = (_dp * k)(*[_ptr(a, _dp) for a in dist_c])
    out = np.zeros((n, 3))
    w = np.zeros((n, k)) if want_weights else None
    lib().or_query_cascade(k, vols, sp, ip, dp, n, _ptr(pos, _dp), _ptr(nrm, _dp), _ptr(cam, _dp),
                           _ptr(out, _dp), _ptr(w, _dp))
    return (out, w) if want_weights else out


def tracking_scroll(vol: OrVolume, camera, states, irr, dist) -> int:
    """Scroll a tracking window to the camera (Sec. 7.2); updates vol's origin
    and shift in place and resets the planes that leapfrog."""
    cam = _f64(camera, (3,))
    return int(lib().or_tracking_scroll(C.byref(vol), _ptr(cam, _dp), _ptr(states, _u8p),
                                        _ptr(irr, _dp), _ptr(dist, _dp)))


def update_cascade(scene_h, lights, vol_structs, frame, states_list, irr_list, dist_list,
                   subsets=None, irr_scale=1.0, vis_scale=1.0, want_rays=False):
    """One cascade update frame in place; hit shading samples the whole cascade."""
    k = len(vol_structs)
    vols = (OrVolume * k)(*vol_structs)
    sp = (_u8p * k)(*[_ptr(a, _u8p) for a in states_list])
    ip = (_dp * k)(*[_ptr(a, _dp) for a in irr_list])
    dp = (_dp * k)(*[_ptr(a, _dp) for a in dist_list])
    nsub = None
    subp = None
    keep = []
    if subsets is not None:
        arrs = [np.ascontiguousarray(x, dtype=np.int64) for x in subsets]
        keep += arrs
        nsub = np.array([len(a) for a in arrs], dtype=np.int64)
        subp = (_i64p * k)(*[_ptr(a, _i64p) for a in arrs])
    rays = None
    rp = None
    if want_rays:
        R = vol_structs[0].rays
        rays = []
        for j in range(k):
            n = len(subsets[j]) if subsets is not None else int(np.prod(list(vol_structs[j].counts)))
            rays.append(np.full((n, R, 4), np.nan))
        rp = (_dp * k)(*[_ptr(a, _dp) for a in rays])
    lib().or_update_cascade(C.byref(scene_h.s), C.byref(make_lights(lights)), k, vols, frame,
                            irr_scale, vis_scale, sp, ip, dp, _ptr(nsub, _i64p), subp, rp)
    return rays


def diff(scene_h, lights, desc, pos, nrm, camera, dE, first_frame=0, n_frames=2):
    """Forward E and the reverse-mode gradient of sum(dE * E) with respect to
    emitter radiance [E,3] and object albedo [O,3] (hysteresis 0, every probe
    tracing, n_frames updates from a zero atlas)."""
    pos = _f64(pos, (-1, 3))
    nrm = _f64(nrm, (-1, 3))
    dE = _f64(dE, (-1, 3))
    cam = _f64(camera, (3,))
    n = len(pos)
    E = np.zeros((n, 3))
    ne = len(scene_h.emitter_radiance) if scene_h.tri_emitter.max(initial=-1) >= 0 else 0
    no = len(scene_h.object_albedo)
    g_em = np.zeros((max(ne, 1), 3))
    g_al = np.zeros((no, 3))
    v = make_volume(desc)
    lib().or_diff(C.byref(scene_h.s), C.byref(make_lights(lights)), C.byref(v), first_frame, n_frames, n,
                  _ptr(pos, _dp), _ptr(nrm, _dp), _ptr(cam, _dp), _ptr(dE, _dp), _ptr(E, _dp),
                  _ptr(g_em, _dp), _ptr(g_al, _dp), ne, no)
    return E, g_em[:ne], g_al
