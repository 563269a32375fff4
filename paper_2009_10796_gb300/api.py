"""Python front end of the C ABI (``include/ddgi.h``).

Argument marshalling only: tensors are passed by device pointer, every step
of the update and query runs in the CUDA library.  PyTorch provides device
memory and streams.  Calls enqueue on the current torch stream unless a
stream is given.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import check, load

__all__ = ["Scene", "Volume", "Cascade", "IrradianceField", "trace", "lights_struct", "update_noalloc",
           "bvh_check"]


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def _ptr(t: torch.Tensor):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return C.c_void_p(t.data_ptr())


def _np(a, dtype):
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _f3(v):
    return _lib.F3(*[float(x) for x in np.asarray(v, dtype=np.float64).reshape(3)])


def lights_struct(lights) -> _lib.Lights:
    """Any object with sun_dir, sun_irradiance, sky_a, sky_b, sky_up."""
    return _lib.Lights(_f3(lights.sun_dir), _f3(lights.sun_irradiance), _f3(lights.sky_a),
                       _f3(lights.sky_b), _f3(lights.sky_up))


def bvh_check(verts, tris) -> dict:
    """Host-only check of the hierarchy a scene of these triangles gets
    (``ddgi_bvh_check``): sizes, depths, stack bound and violations."""
    v = _np(verts, np.float32).reshape(-1, 3)
    t = _np(tris, np.int32).reshape(-1, 3)
    st = (C.c_int64 * 9)()
    check(load().ddgi_bvh_check(v.ctypes.data if len(v) else None, len(v), t.ctypes.data if len(t) else None,
                                len(t), st))
    keys = ["nodes", "nodes4", "leaves", "depth", "depth4", "max_stack", "empty_slots", "violations", "tris"]
    return {k: int(st[i]) for i, k in enumerate(keys)}


class Scene:
    """A registered triangle scene (BVH built on the host, then uploaded)."""

    def __init__(self, verts, tris, tri_object, object_albedo, object_flags, tri_emitter,
                 emitter_radiance):
        lib = load()
        self._arrays = [
            _np(verts, np.float32).reshape(-1, 3), _np(tris, np.int32).reshape(-1, 3),
            _np(tri_object, np.int32), _np(object_albedo, np.float32).reshape(-1, 3),
            _np(object_flags, np.int32), _np(tri_emitter, np.int32),
            _np(emitter_radiance, np.float32).reshape(-1, 3)]
        v, t, to, alb, fl, te, er = self._arrays
        h = C.c_void_p()
        check(lib.ddgi_scene_create(v.ctypes.data, len(v), t.ctypes.data, len(t), to.ctypes.data,
                                    len(alb), alb.ctypes.data, fl.ctypes.data, te.ctypes.data,
                                    len(er), er.ctypes.data if len(er) else None, C.byref(h)))
        self.handle = h
        self.n_tris = len(t)

    @classmethod
    def from_arrays(cls, sc):
        """From any object with the scene fields (verts, tris, tri_object, ...)."""
        return cls(sc.verts, sc.tris, sc.tri_object, sc.object_albedo, sc.object_flags,
                   sc.tri_emitter, sc.emitter_radiance)

    def info(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        check(load().ddgi_scene_info(self.handle, C.byref(a), C.byref(b), C.byref(c)))
        return {"nodes": a.value, "leaves": b.value, "tris": c.value}

    def trace(self, orig: torch.Tensor, dirs: torch.Tensor, stream=None):
        n = orig.shape[0]
        t = torch.empty(n, dtype=torch.float32, device=orig.device)
        tri = torch.empty(n, dtype=torch.int32, device=orig.device)
        bf = torch.empty(n, dtype=torch.int32, device=orig.device)
        check(load().ddgi_trace(self.handle, _ptr(orig), _ptr(dirs), n, _ptr(t), _ptr(tri), _ptr(bf),
                                _stream(stream)))
        return t, tri, bf

    def set_materials(self, albedo: torch.Tensor = None, emit: torch.Tensor = None, stream=None):
        """Object albedo [O,3] and emitter radiance [E,3] from device tensors."""
        a = albedo.detach().float().contiguous() if albedo is not None else None
        e = emit.detach().float().contiguous() if emit is not None else None
        check(load().ddgi_scene_set_materials(self.handle, _ptr(a), _ptr(e), _stream(stream)))

    def raycast_gbuffer(self, position, forward, up, vfov_deg, width, height, stream=None,
                        device="cuda"):
        pos = torch.empty((height * width, 3), dtype=torch.float32, device=device)
        nrm = torch.empty((height * width, 3), dtype=torch.float32, device=device)
        check(load().ddgi_raycast_gbuffer(self.handle, _f3(position), _f3(forward), _f3(up),
                                          float(vfov_deg), int(width), int(height), _ptr(pos),
                                          _ptr(nrm), _stream(stream)))
        return pos, nrm

    def close(self):
        if getattr(self, "handle", None):
            load().ddgi_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def desc_struct(d) -> _lib.VolumeDesc:
    """From any object with the volume fields (origin, spacing, counts, ...)."""
    s = _lib.VolumeDesc()
    s.origin = _f3(d.origin)
    s.spacing = _f3(d.spacing)
    s.counts = (C.c_int32 * 3)(*[int(x) for x in d.counts])
    s.rays_per_probe = int(d.rays_per_probe)
    s.irr_n = int(getattr(d, "irr_n", 6))
    s.dist_n = int(getattr(d, "dist_n", 14))
    s.hysteresis_irr = float(d.hysteresis_irr)
    s.hysteresis_vis = float(d.hysteresis_vis)
    s.gamma = float(getattr(d, "gamma", 5.0))
    s.self_shadow_bias = float(getattr(d, "self_shadow_bias", 0.3))
    s.dist_cos_power = float(getattr(d, "dist_cos_power", 50.0))
    s.t_max = float(getattr(d, "t_max", -1.0))
    s.thr_low = float(getattr(d, "thr_low", 0.25))
    s.thr_high = float(getattr(d, "thr_high", 0.8))
    s.thr_step = float(getattr(d, "thr_step", 0.15))
    s.state_machine = int(getattr(d, "state_machine", 1))
    s.irr_format = int(getattr(d, "irr_format", _lib.IRR_FP32))
    s.dist_format = int(getattr(d, "dist_format", _lib.DIST_FP32))
    s.tracking = int(getattr(d, "tracking", 0))
    s.seed = int(getattr(d, "seed", 0))
    s.optimizer_iters = int(getattr(d, "optimizer_iters", 0))
    s.offset_limit = float(getattr(d, "offset_limit", 0.45))
    s.converge_batches = int(getattr(d, "converge_batches", 0))
    return s


class Volume:
    """A probe volume: atlases, states and the per-frame ray buffer on the device."""

    def __init__(self, desc, irr_format=None, dist_format=None):
        s = desc_struct(desc)
        if irr_format is not None:
            s.irr_format = irr_format
        if dist_format is not None:
            s.dist_format = dist_format
        self.desc = s
        h = C.c_void_p()
        check(load().ddgi_volume_create(C.byref(s), C.byref(h)))
        self.handle = h
        info = _lib.VolumeInfo()
        check(load().ddgi_volume_get_info(h, C.byref(info)))
        self.info = info
        self.n_probes = info.n_probes
        self.R = s.rays_per_probe

    def update(self, scene: Scene, lights, frame: int, irr_scale=1.0, vis_scale=1.0,
               precision=_lib.BLEND_FP32, stream=None):
        p = _lib.UpdateParams(int(frame), float(irr_scale), float(vis_scale), int(precision), 0)
        L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
        check(load().ddgi_update(self.handle, scene.handle, C.byref(L), C.byref(p), _stream(stream)))

    def set_dynamic_boxes(self, boxes):
        """Dynamic-object boxes [n, 6] (lo xyz, hi xyz) that wake sleeping probes
        from the next update on (Sec. 6.3); an empty array clears them."""
        b = _np(boxes, np.float32).reshape(-1, 6)
        check(load().ddgi_set_dynamic_boxes(self.handle, b.ctypes.data if len(b) else None, len(b)))

    def update_range(self, scene: Scene, lights, frame: int, probe_begin: int, probe_end: int, irr_scale=1.0,
                     vis_scale=1.0, precision=_lib.BLEND_FP32, stream=None):
        """Update only probes [probe_begin, probe_end) (one shard of the grid)."""
        p = _lib.UpdateParams(int(frame), float(irr_scale), float(vis_scale), int(precision), 0)
        L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
        check(load().ddgi_update_range(self.handle, scene.handle, C.byref(L), C.byref(p), int(probe_begin),
                                       int(probe_end), _stream(stream)))

    def query(self, pos: torch.Tensor, nrm: torch.Tensor, camera, out: torch.Tensor = None,
              stream=None) -> torch.Tensor:
        n = pos.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        check(load().ddgi_query(self.handle, _ptr(pos), _ptr(nrm), n, _f3(camera), _ptr(out),
                                _stream(stream)))
        return out

    def frame_host(self, scene: Scene, lights, frame: int, pos: torch.Tensor, nrm: torch.Tensor, camera,
                   out: torch.Tensor = None, irr_scale=1.0, vis_scale=1.0, precision=_lib.BLEND_FP32,
                   stream=None) -> torch.Tensor:
        """One frame from host memory: the probe update, then the query of the
        host G-buffer `pos`, `nrm` ([n, 3] float32 CPU tensors, best pinned)
        into the host tensor `out`.  Asynchronous: `out` is complete once
        `stream` has run the enqueued work (synchronise it before reading)."""
        for t in (pos, nrm) + ((out,) if out is not None else ()):
            if t.device.type != "cpu" or t.dtype != torch.float32 or not t.is_contiguous():
                raise ValueError("frame_host takes contiguous float32 CPU tensors")
        n = pos.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32).pin_memory()
        if any(t.dim() != 2 or t.shape != (n, 3) for t in (pos, nrm, out)):
            raise ValueError("pos, nrm and out must be [n, 3]")
        p = _lib.UpdateParams(int(frame), float(irr_scale), float(vis_scale), int(precision), 0)
        L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
        check(load().ddgi_frame_host(self.handle, scene.handle, C.byref(L), C.byref(p), pos.data_ptr(),
                                     nrm.data_ptr(), n, _f3(camera), out.data_ptr(), _stream(stream)))
        return out

    def query_glossy(self, pos: torch.Tensor, nrm: torch.Tensor, dirs: torch.Tensor, out: torch.Tensor = None,
                     stream=None) -> torch.Tensor:
        """Prefiltered radiance M read in the mirror direction at reflection-ray
        hits reached along `dirs` (second-order glossy, Sec. 4.4)."""
        n = pos.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        check(load().ddgi_query_glossy(self.handle, _ptr(pos), _ptr(nrm), _ptr(dirs), n, _ptr(out),
                                       _stream(stream)))
        return out

    def _get(self, which, nbytes, stream=None, device="cuda"):
        buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        check(load().ddgi_get_buffer(self.handle, which, _ptr(buf), nbytes, _stream(stream)))
        return buf

    def states(self, stream=None) -> torch.Tensor:
        return self._get(2, self.n_probes, stream)

    def offsets(self, stream=None) -> torch.Tensor:
        """Probe offsets from the grid [P, 3] (position optimizer, Sec. 5)."""
        return self._get(3, self.n_probes * 16, stream).view(torch.float32).view(self.n_probes, 4)[:, :3]

    def irr_raw(self, stream=None) -> torch.Tensor:
        return self._get(0, self.info.irr_bytes, stream)

    def dist_raw(self, stream=None) -> torch.Tensor:
        return self._get(1, self.info.dist_bytes, stream)

    def irr_atlas(self, stream=None) -> torch.Tensor:
        """Encoded irradiance as float32 [P, n+2, n+2, 3] (FP32 storage only)."""
        n = self.desc.irr_n + 2
        raw = self.irr_raw(stream)
        if self.desc.irr_format == _lib.IRR_FP32:
            return raw.view(torch.float32).view(self.n_probes, n, n, 4)[..., :3]
        if self.desc.irr_format == _lib.IRR_FP16:
            return raw.view(torch.float16).view(self.n_probes, n, n, 4)[..., :3].float()
        return raw.view(torch.int32).view(self.n_probes, n, n)

    def dist_atlas(self, stream=None) -> torch.Tensor:
        n = self.desc.dist_n + 2
        raw = self.dist_raw(stream)
        if self.desc.dist_format == _lib.DIST_FP32:
            return raw.view(torch.float32).view(self.n_probes, n, n, 2)
        return raw.view(torch.float16).view(self.n_probes, n, n, 2).float()

    def copy_buffer(self, which: int, dst: torch.Tensor, stream=None):
        """Copy buffer `which` (ddgi_get_buffer) into the caller's device tensor."""
        check(load().ddgi_get_buffer(self.handle, which, _ptr(dst), dst.numel() * dst.element_size(),
                                     _stream(stream)))

    def set_buffer(self, which: int, src: torch.Tensor, stream=None):
        check(load().ddgi_set_buffer(self.handle, which, _ptr(src), src.numel() * src.element_size(),
                                     _stream(stream)))

    def ray_records(self, stream=None):
        """(records [n_active, R, 4], probe ids [n_active]) of the last update."""
        rec = torch.empty((self.n_probes * self.R, 4), dtype=torch.float32, device="cuda")
        ids = torch.empty(self.n_probes, dtype=torch.int32, device="cuda")
        n = C.c_int64()
        check(load().ddgi_get_ray_records(self.handle, _ptr(rec), _ptr(ids), C.byref(n),
                                          _stream(stream)))
        k = n.value
        return rec[: k * self.R].view(k, self.R, 4), ids[:k]

    def trace_stats(self, scene: Scene, lights, stream=None):
        """Work counters of the last update's trace (instrumented re-trace)."""
        st = (C.c_uint64 * 7)()
        L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
        check(load().ddgi_trace_stats(self.handle, scene.handle, C.byref(L), st, _stream(stream)))
        keys = ["rays", "nodes", "tris", "shadow_rays", "shadow_nodes", "shadow_tris", "queries"]
        return {k: int(st[i]) for i, k in enumerate(keys)}

    def diff_forward(self, scene: Scene, lights, pos, nrm, camera, first_frame=0, n_frames=2, stream=None):
        out = torch.empty((pos.shape[0], 3), dtype=torch.float32, device=pos.device)
        L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
        check(load().ddgi_diff_forward(self.handle, scene.handle, C.byref(L), int(first_frame), int(n_frames),
                                       _ptr(pos), _ptr(nrm), pos.shape[0], _f3(camera), _ptr(out),
                                       _stream(stream)))
        return out

    def diff_backward(self, scene: Scene, lights, pos, nrm, camera, dE, n_objects, n_emitters, first_frame=0,
                      n_frames=2, stream=None):
        d_alb = torch.empty((n_objects, 3), dtype=torch.float32, device=pos.device)
        d_em = torch.empty((max(n_emitters, 1), 3), dtype=torch.float32, device=pos.device)
        L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
        dE = dE.float().contiguous()
        check(load().ddgi_diff_backward(self.handle, scene.handle, C.byref(L), int(first_frame), int(n_frames),
                                        _ptr(pos), _ptr(nrm), pos.shape[0], _f3(camera), _ptr(dE), _ptr(d_alb),
                                        _ptr(d_em), _stream(stream)))
        return d_alb, d_em[:n_emitters]

    def diff_forward_f64(self, scene: Scene, lights, albedo, emit, pos, nrm, camera, first_frame=0, n_frames=2,
                         stream=None):
        """E [n, 3] float64 of the FP64 differentiable forward (ddgi_diff_forward_f64)
        for albedo [O, 3] and emitter radiance [E, 3] float64 device tensors."""
        out = torch.empty((pos.shape[0], 3), dtype=torch.float64, device=pos.device)
        L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
        check(load().ddgi_diff_forward_f64(self.handle, scene.handle, C.byref(L), int(first_frame), int(n_frames),
                                           _ptr(albedo.contiguous()), _ptr(emit.contiguous()) if emit.numel() else None,
                                           _ptr(pos), _ptr(nrm), pos.shape[0], _f3(camera), _ptr(out),
                                           _stream(stream)))
        return out

    def diff_backward_f64(self, scene: Scene, lights, albedo, pos, nrm, camera, dE, n_emitters, first_frame=0,
                          n_frames=2, stream=None):
        """(dLoss/d albedo, dLoss/d emitter radiance) float64 of the FP64 reverse
        pass (ddgi_diff_backward_f64) for dE = dLoss/dE [n, 3] float64."""
        d_alb = torch.empty((albedo.shape[0], 3), dtype=torch.float64, device=pos.device)
        d_em = torch.empty((max(n_emitters, 1), 3), dtype=torch.float64, device=pos.device)
        L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
        check(load().ddgi_diff_backward_f64(self.handle, scene.handle, C.byref(L), int(first_frame), int(n_frames),
                                            _ptr(albedo.contiguous()), _ptr(pos), _ptr(nrm), pos.shape[0],
                                            _f3(camera), _ptr(dE.double().contiguous()), _ptr(d_alb), _ptr(d_em),
                                            _stream(stream)))
        return d_alb, d_em[:n_emitters]

    def query_backward(self, pos, nrm, camera, dE, fold_borders=False, stream=None):
        """dLoss/d(stored irradiance texels) [P, n+2, n+2, 3] float32 of a query
        at (pos, nrm, camera) on the current atlases, given dE = dLoss/dE [n, 3]
        (ddgi_query_backward); fold_borders adds border gradients to the
        interior texels they copy."""
        N = self.desc.irr_n + 2
        g = torch.empty((self.n_probes, N, N, 3), dtype=torch.float32, device=pos.device)
        dE = dE.float().contiguous()
        check(load().ddgi_query_backward(self.handle, _ptr(pos), _ptr(nrm), pos.shape[0], _f3(camera), _ptr(dE),
                                         int(bool(fold_borders)), _ptr(g), _stream(stream)))
        return g

    def save(self, stream=None) -> bytes:
        """The volume's states, atlases and offsets as a versioned blob (ddgi_volume_save)."""
        n = C.c_size_t(0)
        check(load().ddgi_volume_save(self.handle, None, C.byref(n), _stream(stream)))
        buf = C.create_string_buffer(n.value)
        check(load().ddgi_volume_save(self.handle, buf, C.byref(n), _stream(stream)))
        return buf.raw[: n.value]

    def load(self, blob: bytes, stream=None):
        """Restore a blob from `save` of a volume with the same layout (ddgi_volume_load)."""
        buf = C.create_string_buffer(bytes(blob), len(blob))
        check(load().ddgi_volume_load(self.handle, buf, len(blob), _stream(stream)))

    def enable_timing(self, on=True):
        check(load().ddgi_enable_timing(self.handle, int(bool(on))))

    def read_timings(self):
        ms = (C.c_float * 8)()
        cnt = (C.c_int32 * 8)()
        check(load().ddgi_read_timings(self.handle, ms, cnt))
        names = ["classify", "lists", "trace_shade", "blend", "frame_setup", "trace_primary", "trace_shadow",
                 "shade"]
        return {n: (ms[i], cnt[i]) for i, n in enumerate(names)}

    def poll_status(self, stream=None):
        check(load().ddgi_poll_status(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            load().ddgi_volume_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def trace(scene: Scene, orig, dirs, stream=None):
    return scene.trace(orig, dirs, stream)


def update_noalloc(scene: Scene, desc, lights, frame: int, states: torch.Tensor,
                   irr: torch.Tensor, dist: torch.Tensor, irr_scale=1.0, vis_scale=1.0,
                   stream=None):
    """One update frame on caller-owned state, allocating no device memory
    (ddgi_update_noalloc): `states`, `irr` and `dist` are the volume's state
    buffers, owned and kept by the caller between frames."""
    d = desc if isinstance(desc, _lib.VolumeDesc) else desc_struct(desc)
    p = _lib.UpdateParams(int(frame), float(irr_scale), float(vis_scale), _lib.BLEND_FP32, 0)
    L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
    check(load().ddgi_update_noalloc(scene.handle, C.byref(d), C.byref(L), C.byref(p), _ptr(states),
                                     _ptr(irr), _ptr(dist), _stream(stream)))


def update_noalloc_poll_status(stream=None):
    """Raise DDGIError if an update_noalloc call on the current device flagged
    a device-side error since the last poll (reads and clears the shared
    status word; synchronises the stream)."""
    check(load().ddgi_update_noalloc_poll_status(_stream(stream)))


def measure_l2_read(buf, passes, sink, stream=None):
    """Enqueue one read of the device tensor `buf` (16-byte aligned, a
    multiple of 16 bytes) `passes` times through L2 (ddgi_measure_l2_read);
    `sink` is a one-element int32 device tensor.  Time it with events on
    `stream` after an untimed call."""
    check(load().ddgi_measure_l2_read(_ptr(buf), C.c_size_t(buf.numel() * buf.element_size()), int(passes),
                                      _ptr(sink), _stream(stream)))


class Cascade:
    """Nested probe volumes updated together (densest first), optionally
    camera-tracking windows; see ddgi_cascade_* in include/ddgi.h."""

    def __init__(self, descs):
        arr = (_lib.VolumeDesc * len(descs))(*[d if isinstance(d, _lib.VolumeDesc) else desc_struct(d)
                                               for d in descs])
        self.descs = list(arr)
        h = C.c_void_p()
        check(load().ddgi_cascade_create(arr, len(descs), C.byref(h)))
        self.handle = h
        self.n = len(descs)

    def _params(self, frame, camera, irr_scale, vis_scale, precision, use_graph):
        return _lib.CascadeParams(int(frame), _f3(camera), float(irr_scale), float(vis_scale),
                                  int(precision), int(bool(use_graph)))

    def update(self, scene: Scene, lights, frame: int, camera, irr_scale=1.0, vis_scale=1.0,
               precision=_lib.BLEND_FP32, use_graph=False, stream=None):
        p = self._params(frame, camera, irr_scale, vis_scale, precision, use_graph)
        L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
        check(load().ddgi_cascade_update(self.handle, scene.handle, C.byref(L), C.byref(p), _stream(stream)))

    def query(self, pos: torch.Tensor, nrm: torch.Tensor, camera, out: torch.Tensor = None, stream=None):
        n = pos.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, device=pos.device)
        check(load().ddgi_cascade_query(self.handle, _ptr(pos), _ptr(nrm), n, _f3(camera), _ptr(out),
                                        _stream(stream)))
        return out

    def _sizes(self, k):
        d = self.descs[k]
        P = d.counts[0] * d.counts[1] * d.counts[2]
        tb = load().ddgi_texel_bytes(0, int(d.irr_format))
        db = load().ddgi_texel_bytes(1, int(d.dist_format))
        return P, P * (d.irr_n + 2) ** 2 * tb, P * (d.dist_n + 2) ** 2 * db

    def buffer(self, k, which, stream=None):
        P, bi, bd = self._sizes(k)
        nb = {0: bi, 1: bd, 2: P}[which]
        buf = torch.empty(nb, dtype=torch.uint8, device="cuda")
        check(load().ddgi_cascade_get_buffer(self.handle, k, which, _ptr(buf), nb, _stream(stream)))
        return buf

    def states(self, k):
        return self.buffer(k, 2)

    def irr_atlas(self, k):
        d = self.descs[k]
        n = d.irr_n + 2
        return self.buffer(k, 0).view(torch.float32).view(-1, n, n, 4)[..., :3]

    def dist_atlas(self, k):
        d = self.descs[k]
        n = d.dist_n + 2
        return self.buffer(k, 1).view(torch.float32).view(-1, n, n, 2)

    def window(self, k):
        o = (C.c_double * 3)()
        sh = (C.c_int32 * 3)()
        check(load().ddgi_cascade_get_window(self.handle, k, o, sh))
        return list(o), list(sh)

    def ray_records(self, stream=None):
        """(records [n_active, R, 4], volume index [n_active], stored probe
        index [n_active]) of the last update, in active-list order."""
        total = sum(d.counts[0] * d.counts[1] * d.counts[2] for d in self.descs)
        R = self.descs[0].rays_per_probe
        rec = torch.empty((total * R, 4), dtype=torch.float32, device="cuda")
        ent = torch.empty(total, dtype=torch.int32, device="cuda")
        n = C.c_int64()
        check(load().ddgi_cascade_get_ray_records(self.handle, _ptr(rec), _ptr(ent), C.byref(n), _stream(stream)))
        k = n.value
        ent = ent[:k]
        return rec[: k * R].view(k, R, 4), ent >> 24, ent & ((1 << 24) - 1)

    def set_tuning(self, trace_blocks_per_sm, blend_probes_per_cta):
        check(load().ddgi_cascade_set_tuning(self.handle, int(trace_blocks_per_sm), int(blend_probes_per_cta)))

    def tuning(self):
        a, b = C.c_int32(), C.c_int32()
        check(load().ddgi_cascade_get_tuning(self.handle, C.byref(a), C.byref(b)))
        return a.value, b.value

    def autotune(self, scene: Scene, lights, frame, camera, cache_path=None, precision=_lib.BLEND_FP32,
                 stream=None):
        p = self._params(frame, camera, 1.0, 1.0, precision, False)
        L = lights if isinstance(lights, _lib.Lights) else lights_struct(lights)
        fc = C.c_int32(0)
        check(load().ddgi_cascade_autotune(self.handle, scene.handle, C.byref(L), C.byref(p),
                                           cache_path.encode() if cache_path else None, C.byref(fc),
                                           _stream(stream)))
        return bool(fc.value)

    def poll_status(self, stream=None):
        check(load().ddgi_cascade_poll_status(self.handle, _stream(stream)))

    def close(self):
        if getattr(self, "handle", None):
            load().ddgi_cascade_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ProbeQuery(torch.autograd.Function):
    """E = query(irradiance atlas) at fixed points: the volume's query with the
    FP32 irradiance atlas given as a tensor [P, n+2, n+2, 4] (rgb + the unused
    lane, the stored layout), differentiable with respect to it through
    ddgi_query_backward (the unused lane gets zero gradient).  The forward
    copies the atlas into the volume.

    Usage: ProbeQuery.apply(irr_atlas, volume, pos, nrm, camera)."""

    @staticmethod
    def forward(ctx, irr_atlas, volume, pos, nrm, camera):
        if volume.desc.irr_format != _lib.IRR_FP32:
            raise ValueError("ProbeQuery needs an FP32 irradiance atlas")
        volume.set_buffer(0, irr_atlas.detach().contiguous())
        ctx.args = (volume, pos, nrm, camera)
        return volume.query(pos, nrm, camera)

    @staticmethod
    def backward(ctx, dE):
        volume, pos, nrm, camera = ctx.args
        g = volume.query_backward(pos, nrm, camera, dE)
        return torch.nn.functional.pad(g, (0, 1)), None, None, None, None


class IrradianceField(torch.autograd.Function):
    """E = field(albedo, emit): the probe update (n_frames from a zero atlas,
    hysteresis 0) and the query at fixed points, differentiable with respect
    to per-object albedo [O,3] and per-emitter radiance [E,3].  The backward
    pass is the library's adjoint (ddgi_diff_backward); rays are re-traced.

    Usage: IrradianceField.apply(albedo, emit, volume, scene, lights, pos, nrm,
    camera, first_frame, n_frames)."""

    @staticmethod
    def forward(ctx, albedo, emit, volume, scene, lights, pos, nrm, camera, first_frame=0, n_frames=2):
        scene.set_materials(albedo, emit)
        E = volume.diff_forward(scene, lights, pos, nrm, camera, first_frame, n_frames)
        ctx.save_for_backward(albedo, emit)
        ctx.args = (volume, scene, lights, pos, nrm, camera, first_frame, n_frames)
        return E

    @staticmethod
    def backward(ctx, dE):
        albedo, emit = ctx.saved_tensors
        volume, scene, lights, pos, nrm, camera, first_frame, n_frames = ctx.args
        d_alb, d_em = volume.diff_backward(scene, lights, pos, nrm, camera, dE, albedo.shape[0], emit.shape[0],
                                           first_frame, n_frames)
        return d_alb, d_em, None, None, None, None, None, None, None, None
