"""The oracle's reverse-mode gradient against FP64 central finite differences.

Forward: two update frames from a zero atlas with hysteresis 0 (direct light
and one bounce through the previous frame's probes), then the query.  The
gradient of sum(G * E) with respect to every emitter radiance and object
albedo component must match central differences to 1e-5 relative."""
import numpy as np
import pytest

import oracle
import synth


def _scene():
    b = synth._Builder()
    b.box((0, 0, 0), (6, 6, 6), obj=0, inward=True)
    x = synth.f32(0.01)
    b.quad([(x, 2, 2), (x, 4, 2), (x, 4, 4), (x, 2, 4)], np.array([1.0, 0, 0]), obj=1, emitter=0)
    y = synth.f32(5.99)
    b.quad([(2, y, 2), (4, y, 2), (4, y, 4), (2, y, 4)], np.array([0.0, -1, 0]), obj=2, emitter=1)
    z = synth.f32(0.01)
    b.quad([(1, 1, z), (3, 1, z), (3, 3, z), (1, 3, z)], np.array([0.0, 0, 1]), obj=3, emitter=2)
    b.box((3.5, 0.0, 3.5), (4.5, 2.5, 4.5), obj=4)
    b.box((1.0, 3.0, 1.0), (2.0, 4.0, 2.0), obj=5)
    alb = np.array([[0.6, 0.5, 0.4], [0.3, 0.3, 0.3], [0.2, 0.4, 0.3], [0.5, 0.5, 0.2], [0.7, 0.6, 0.5],
                    [0.4, 0.7, 0.6]])
    flags = np.array([0, 1, 1, 1, 1, 1], dtype=np.int32)
    em = np.array([[2.0, 1.5, 1.0], [1.0, 2.0, 1.2], [0.8, 0.9, 2.5]])
    return b.finish(alb, flags, em, "diff")


@pytest.mark.parametrize("gamma", [1.0, 5.0])
def test_adjoint_matches_central_differences(gamma):
    sc = _scene()
    L = synth.Lights(sun_dir=synth.f32(np.array([0.2, -1.0, 0.3]) / np.linalg.norm([0.2, -1.0, 0.3])),
                     sun_irradiance=np.array([1.5, 1.2, 1.0]))
    desc = synth.VolumeDesc(origin=(0.75, 0.75, 0.75), spacing=(1.5, 1.5, 1.5), counts=(4, 4, 4),
                            rays_per_probe=32, gamma=gamma, state_machine=0, seed=17, hysteresis_irr=0,
                            hysteresis_vis=0)
    rng = synth.Rng(9)
    n = 64
    pos = synth.f32(rng.uniform(3 * n, 0.8, 5.2).reshape(n, 3))
    nrm = rng.unit_vectors(n)
    G = rng.uniform(3 * n, -1.0, 1.0).reshape(n, 3)
    cam = np.array([3.0, 3.0, 3.0])
    E, g_em, g_al = oracle.diff(oracle.SceneHandle(sc), L, desc, pos, nrm, cam, G)
    assert g_em.shape == (3, 3) and g_al.shape == (6, 3)

    def loss(emit, alb):
        s2 = synth.Scene(**{**sc.__dict__, "emitter_radiance": emit, "object_albedo": alb})
        E2, _, _ = oracle.diff(oracle.SceneHandle(s2), L, desc, pos, nrm, cam, G)
        return float((G * E2).sum())

    fd_em = np.zeros_like(g_em)
    fd_al = np.zeros_like(g_al)
    for arr, fd in ((sc.emitter_radiance, fd_em), (sc.object_albedo, fd_al)):
        for idx in np.ndindex(arr.shape):
            h = 1e-6 * max(1.0, abs(arr[idx]))
            a_p = arr.copy()
            a_m = arr.copy()
            a_p[idx] += h
            a_m[idx] -= h
            if arr is sc.emitter_radiance:
                fd[idx] = (loss(a_p, sc.object_albedo) - loss(a_m, sc.object_albedo)) / (2 * h)
            else:
                fd[idx] = (loss(sc.emitter_radiance, a_p) - loss(sc.emitter_radiance, a_m)) / (2 * h)
    for g, fd in ((g_em, fd_em), (g_al, fd_al)):
        scale = np.maximum(np.abs(fd), 1e-3 * np.abs(fd).max())
        err = np.abs(g - fd) / scale
        print(f"[adjoint] gamma {gamma}: max rel err {err.max():.2e}")
        assert err.max() < 1e-5
    # every parameter matters here: the emitters are seen, the albedos reflect
    assert np.all(np.abs(fd_em) > 0) and np.count_nonzero(fd_al) >= 12
