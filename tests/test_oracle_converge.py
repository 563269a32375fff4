"""Pins of the oracle's optional converge pass for new probes (Sec. 6.3): a
Newly Vigilant / Newly Awake probe traces converge_batches batches of R rays,
takes per texel the weighted average over all of them (encoded, hysteresis
0) and becomes Vigilant / Awake before the frame's regular update.

The pins are closed forms of the sky integral and of an enclosing sphere, and
the state transitions; the regular pass after the converge pass is made
neutral (hysteresis 1, thresholds out of reach) so the texels it leaves are
the converge pass's own."""
import numpy as np
import pytest

import oracle
import synth


def _vol(**kw):
    d = dict(origin=(0, 0, 0), spacing=(1, 1, 1), counts=(2, 2, 2), rays_per_probe=64,
             hysteresis_irr=1.0, hysteresis_vis=1.0, thr_low=10.0, thr_high=20.0,
             state_machine=1, seed=91, t_max=3.0)
    d.update(kw)
    return synth.VolumeDesc(**d)


def _newly_state(desc):
    return oracle.new_state(desc, initial=oracle.NEWLY_VIGILANT)


def test_converge_uniform_sky_exact_and_states():
    a = np.array([0.4, 1.3, 0.07])
    L = synth.Lights(sky_a=a, sky_b=np.zeros(3))
    desc = _vol(converge_batches=3)
    st, irr, dist = _newly_state(desc)
    oracle.update(oracle.SceneHandle(synth.empty_scene()), L, desc, 5, st, irr, dist)
    assert np.all(st == oracle.VIGILANT)
    inner = irr[:, 1:-1, 1:-1, :]
    # whatever the weights, a constant sky averages to itself (encoded a^(1/gamma))
    assert np.allclose(np.power(inner, desc.gamma), np.broadcast_to(a, inner.shape), rtol=1e-13)
    assert np.allclose(dist[:, 1:-1, 1:-1, 0], desc.t_max, rtol=1e-14)
    assert np.allclose(dist[:, 1:-1, 1:-1, 1], desc.t_max ** 2, rtol=1e-14)


def test_converge_newly_awake_becomes_awake():
    L = synth.Lights(sky_a=np.ones(3), sky_b=np.zeros(3))
    desc = _vol(converge_batches=1)
    st, irr, dist = oracle.new_state(desc, initial=oracle.NEWLY_AWAKE)
    oracle.update(oracle.SceneHandle(synth.empty_scene()), L, desc, 0, st, irr, dist)
    assert np.all(st == oracle.AWAKE)
    assert np.all(irr[:, 1:-1, 1:-1, :] > 0)


def test_converge_linear_sky_tends_to_cosine_mean():
    """More batches, more rays: the texels tend to the hemisphere cosine mean
    a + (2/3) b (n.up) of a linear sky, as a single pass with B R rays does."""
    a = np.full(3, 1.0)
    b = np.array([0.8, -0.5, 0.3])
    up = synth.f32([0.2, 0.9, -0.3])
    up = up / np.linalg.norm(up)
    L = synth.Lights(sky_a=a, sky_b=b, sky_up=up)
    tex = oracle.texel_dirs(6)
    want = a[None, None, :] + (2.0 / 3.0) * (tex @ up)[..., None] * b[None, None, :]
    errs = []
    for B in (1, 4, 16, 64):
        desc = _vol(converge_batches=B, gamma=1.0)
        st, irr, dist = _newly_state(desc)
        oracle.update(oracle.SceneHandle(synth.empty_scene()), L, desc, 1, st, irr, dist, subset=[0])
        errs.append(np.abs(irr[0, 1:-1, 1:-1, :] - want).max())
    assert errs[-1] < 2e-3
    assert errs[0] > errs[-1] * 4
    assert all(e < 0.06 for e in errs)


def test_converge_batches_are_distinct_rotations():
    """Batch b is rotated by (seed + 0xD1B54A32D192ED03 (b + 1), frame): the
    converge pass equals one pass over the union of the batches' rays, and
    that union differs from repeating one batch (checked on a linear sky)."""
    a = np.full(3, 1.0)
    b = np.array([0.8, -0.5, 0.3])
    up = np.array([0.0, 1.0, 0.0])
    L = synth.Lights(sky_a=a, sky_b=b, sky_up=up)
    B, R, seed, frame = 4, 16, 91, 2
    desc = _vol(converge_batches=B, rays_per_probe=R, gamma=1.0, seed=seed)
    st, irr, dist = _newly_state(desc)
    oracle.update(oracle.SceneHandle(synth.empty_scene()), L, desc, frame, st, irr, dist, subset=[0])
    mask = (1 << 64) - 1
    dirs = np.concatenate([oracle.frame_dirs((seed + 0xD1B54A32D192ED03 * (k + 1)) & mask, frame, R)
                           for k in range(B)])
    tex = oracle.texel_dirs(6).reshape(-1, 3)
    w = np.maximum(0.0, tex @ dirs.T)
    rad = a[None, :] + (dirs @ up)[:, None] * b[None, :]
    ok = w.sum(1) > 0
    union = (w @ rad)[ok] / w.sum(1)[ok][:, None]
    got = irr[0, 1:-1, 1:-1, :].reshape(-1, 3)[ok]
    assert np.allclose(got, union, rtol=1e-12, atol=1e-14)
    one = oracle.frame_dirs((seed + 0xD1B54A32D192ED03) & mask, frame, R)
    assert not np.allclose(dirs[:R], dirs[R:2 * R])
    assert np.abs(one - dirs[:R]).max() == 0


def test_converge_enclosing_sphere_moments():
    rad = 2.5
    sc = synth.icosphere(rad, 3, inward=True)
    desc = _vol(converge_batches=4, rays_per_probe=64, t_max=1e9)
    st, irr, dist = _newly_state(desc)
    oracle.update(oracle.SceneHandle(sc), synth.Lights(), desc, 0, st, irr, dist, subset=[0])
    mu = dist[0, 1:-1, 1:-1, 0]
    mu2 = dist[0, 1:-1, 1:-1, 1]
    V = sc.verts[sc.tris]
    ctr = V.mean(1)
    nrm = np.cross(V[:, 1] - V[:, 0], V[:, 2] - V[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    inner = np.min(np.abs(np.einsum("ij,ij->i", ctr, nrm)))
    assert np.all(mu >= inner - 1e-12) and np.all(mu <= rad + 1e-12)
    assert np.all(mu2 >= mu ** 2 - 1e-12) and np.all(mu2 <= rad ** 2 + 1e-12)
    assert st[0] == oracle.VIGILANT


def test_converge_off_keeps_single_pass():
    """converge_batches = 0: new probes blend their R rays with hysteresis 0
    in the regular pass, as before."""
    a = np.array([0.5, 0.5, 0.5])
    L = synth.Lights(sky_a=a, sky_b=np.zeros(3))
    desc = _vol(converge_batches=0, hysteresis_irr=0.9, hysteresis_vis=0.9)
    st, irr, dist = _newly_state(desc)
    oracle.update(oracle.SceneHandle(synth.empty_scene()), L, desc, 0, st, irr, dist)
    assert np.all(st == oracle.VIGILANT)
    assert np.allclose(np.power(irr[:, 1:-1, 1:-1, :], desc.gamma), 0.5, rtol=1e-13)
