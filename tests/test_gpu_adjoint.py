"""GPU adjoint (ddgi_diff_forward / ddgi_diff_backward behind
torch.autograd.Function) against the oracle's FP64 reverse-mode gradient,
which test_oracle_adjoint pins to FP64 central differences."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import REL, compare_rays, gpu_rays_by_probe, masked_texels, patched, rel_err, run_oracle, to_dev
from test_oracle_adjoint import _scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    import paper_2009_10796_gb300 as pkg
    pkg.load()
    torch.cuda.set_device(0)
    return pkg


def _setup(gamma):
    sc = _scene()
    L = synth.Lights(sun_dir=synth.f32(np.array([0.2, -1.0, 0.3]) / np.linalg.norm([0.2, -1.0, 0.3])),
                     sun_irradiance=np.array([1.5, 1.2, 1.0]))
    desc = synth.VolumeDesc(origin=(0.75, 0.75, 0.75), spacing=(1.5, 1.5, 1.5), counts=(4, 4, 4),
                            rays_per_probe=32, gamma=gamma, state_machine=0, seed=17, hysteresis_irr=0,
                            hysteresis_vis=0)
    rng = synth.Rng(9)
    n = 256
    pos = synth.f32(rng.uniform(3 * n, 0.8, 5.2).reshape(n, 3))
    nrm = rng.unit_vectors(n)
    G = synth.f32(rng.uniform(3 * n, -1.0, 1.0).reshape(n, 3))
    return sc, L, desc, pos, nrm, G, np.array([3.0, 3.0, 3.0])


@pytest.mark.parametrize("gamma", [1.0, 5.0])
def test_adjoint_matches_oracle_gradient(g, gamma):
    """The differentiable forward (two updates from a zero atlas, hysteresis 0,
    then the query) and its adjoint against the oracle.  The forward's
    updates are replayed through the plain update and compared ray by ray;
    rays whose FP32 and FP64 hits differ (an edge grazed within rounding) are
    listed with the texels they reach (weight > 1e-3 of the texel's row) and
    the query points near those probes; everything else meets 1e-4."""
    sc, L, desc, pos, nrm, G, cam = _setup(gamma)
    E_ref, g_em_ref, g_al_ref = oracle.diff(oracle.SceneHandle(sc), L, desc, pos, nrm, cam, G)
    st_o, irr_o, dist_o, rays_o = run_oracle(sc, L, desc, [0, 1])
    S = g.Scene.from_arrays(sc)
    W = g.Volume(desc)
    mi = np.zeros(irr_o.shape[:3], dtype=bool)
    md = np.zeros(dist_o.shape[:3], dtype=bool)
    flagged = 0
    for k, f in enumerate([0, 1]):
        W.update(S, L, f)
        rec, ids = gpu_rays_by_probe(W)
        bad, err = compare_rays(rec, ids, rays_o[k])
        a, b = masked_texels(desc, desc.seed, f, bad, ids)
        mi |= a
        md |= b
        flagged += int(bad.sum())
        if bad.any():
            print(f"[adjoint] gamma {gamma} frame {f}: listed rays (probe, ray): "
                  f"{[(int(ids[i]), int(r)) for i, r in zip(*np.nonzero(bad))][:12]}")
    V = g.Volume(desc)
    albedo = torch.tensor(sc.object_albedo, dtype=torch.float32, device="cuda", requires_grad=True)
    emit = torch.tensor(sc.emitter_radiance, dtype=torch.float32, device="cuda", requires_grad=True)
    P, N_ = to_dev(pos), to_dev(nrm)
    E = g.IrradianceField.apply(albedo, emit, V, S, L, P, N_, cam, 0, 2)
    # the differentiable forward runs the same updates: its atlas is the plain update's, bit for bit
    assert torch.equal(V.irr_raw(), W.irr_raw()) and torch.equal(V.dist_raw(), W.dist_raw())
    (E * to_dev(G)).sum().backward()
    gi = V.irr_atlas().cpu().numpy().astype(np.float64)
    gd = V.dist_atlas().cpu().numpy().astype(np.float64)
    ei = rel_err(gi, irr_o).max(-1)
    ed = rel_err(gd, dist_o).max(-1)
    # end to end: the oracle's query of its own atlas with the listed texels
    # taken from the GPU's (the rest of the forward must then meet 1e-4)
    E_gpu = E.detach().cpu().numpy()
    E_patch = oracle.query(desc, st_o, patched(irr_o, gi, mi), patched(dist_o, gd, md), pos, nrm, cam)
    e = rel_err(E_gpu, E_patch).max(-1)
    e_all = rel_err(E_gpu, E_ref).max(-1)
    E_own = oracle.query(desc, V.states().cpu().numpy(), gi, gd, pos, nrm, cam)
    e_own = rel_err(E_gpu, E_own).max(-1)
    ea = rel_err(albedo.grad.cpu().numpy(), g_al_ref).max()
    ee = rel_err(emit.grad.cpu().numpy(), g_em_ref).max()
    print(f"[adjoint] gamma {gamma}: listed rays {flagged} of {2 * desc.n_probes * desc.rays_per_probe}, masked "
          f"texels {int(mi.sum())} + {int(md.sum())}; texels irr {ei[~mi].max():.2e}, dist {ed[~md].max():.2e}; "
          f"forward: against the listed-texel-patched oracle atlas {e.max():.2e} (unpatched {e_all.max():.2e}), "
          f"on the GPU's own atlas {e_own.max():.2e}; albedo grad {ea:.2e}, emitter grad {ee:.2e}")
    assert flagged <= max(2, int(1e-3 * 2 * desc.n_probes * desc.rays_per_probe))
    assert ei[~mi].max() <= REL and ed[~md].max() <= REL
    assert e.max() <= REL and e_own.max() <= REL
    assert ea <= 1e-3 and ee <= 1e-3


def test_adam_recovers_materials(g):
    """Targets from hidden materials; starting from perturbed ones, Adam on
    the adjoint's gradients drives the query loss down."""
    sc, L, desc, pos, nrm, _, cam = _setup(1.0)
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    P, N_ = to_dev(pos), to_dev(nrm)
    true_alb = torch.tensor(sc.object_albedo, dtype=torch.float32, device="cuda")
    true_em = torch.tensor(sc.emitter_radiance, dtype=torch.float32, device="cuda")
    with torch.no_grad():
        target = g.IrradianceField.apply(true_alb, true_em, V, S, L, P, N_, cam, 0, 2).clone()
    albedo = torch.full_like(true_alb, 0.5).requires_grad_(True)
    emit = torch.full_like(true_em, 1.0).requires_grad_(True)
    opt = torch.optim.Adam([albedo, emit], lr=0.05)
    losses = []
    for step in range(120):
        opt.zero_grad()
        E = g.IrradianceField.apply(albedo, emit, V, S, L, P, N_, cam, 0, 2)
        loss = ((E - target) ** 2).mean()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    print(f"[adjoint] adam: loss {losses[0]:.3e} -> {losses[-1]:.3e}, emitter error "
          f"{float((emit - true_em).abs().max()):.3f}")
    assert losses[-1] < 0.01 * losses[0]


def test_interior_full_size_gradient_properties(g):
    """The differentiation workload at full size and as the bench runs it
    (2,048 probes x 128 rays, 192,140 triangles, 257 objects, 64 emitters, 1M
    query points, two frames from a zero atlas, gamma 1, no sun or sky), with
    checks that hold at any size, for the loss sum(G * E), G > 0:
    (1) lit by its emitters alone, E is positively homogeneous of degree 1 in
    the emitter radiances (frame-0 texels, the frame-1 bounce through them,
    the frame-1 texels and the query all scale with them; no weight depends
    on radiance), so Euler's theorem gives, per channel c,
    sum_k L_e[k, c] dloss/dL_e[k, c] = sum_i G[i, c] E[i, c];
    (2) E is smooth in the albedos (they enter affinely before the query), so
    the albedo gradient along a positive seeded direction matches the central
    difference of the forward, summed in FP64."""
    sc, truth_alb, truth_em = synth.interior_scene()
    L = synth.Lights()
    S = g.Scene.from_arrays(sc)
    V = g.Volume(synth.interior_volume())
    pts, nrm = synth.surface_points(sc, 1_000_000, seed=3005)
    P = to_dev(pts)
    N_ = to_dev(nrm)
    cam = np.array([0.0, 10.0, 0.0])
    rng = synth.Rng(4006)
    G = rng.uniform(3 * len(pts), 0.5, 1.5).reshape(-1, 3)
    Gd = to_dev(G)
    albedo = torch.tensor(truth_alb, dtype=torch.float32, device="cuda", requires_grad=True)
    emit = torch.tensor(truth_em, dtype=torch.float32, device="cuda", requires_grad=True)
    E = g.IrradianceField.apply(albedo, emit, V, S, L, P, N_, cam, 0, 2)
    (E * Gd).sum().backward()
    E = E.detach().cpu().numpy().astype(np.float64)
    g_em = emit.grad.cpu().numpy().astype(np.float64)
    g_al = albedo.grad.cpu().numpy().astype(np.float64)
    Gf = Gd.cpu().numpy().astype(np.float64)
    lhs = (truth_em.astype(np.float32).astype(np.float64) * g_em).sum(0)
    rhs = (Gf * E).sum(0)
    e_euler = np.abs(lhs - rhs) / np.abs(rhs)
    print(f"[adjoint full size] Euler: lhs {lhs}, rhs {rhs}, rel {e_euler.max():.2e}")
    assert np.all(rhs > 0) and e_euler.max() <= 1e-3

    delta = rng.uniform(truth_alb.size, 0.0, 1.0).reshape(truth_alb.shape)
    h = 0.01

    def loss(a):
        with torch.no_grad():
            Ea = g.IrradianceField.apply(torch.tensor(a, dtype=torch.float32, device="cuda"), emit.detach(), V, S,
                                         L, P, N_, cam, 0, 2)
        return float((Gf * Ea.cpu().numpy().astype(np.float64)).sum())

    a0 = truth_alb.astype(np.float32).astype(np.float64)
    fd = (loss(a0 + h * delta) - loss(a0 - h * delta)) / (2 * h)
    ad = float((g_al * delta.astype(np.float32).astype(np.float64)).sum())
    e_fd = abs(ad - fd) / abs(fd)
    print(f"[adjoint full size] albedo direction: adjoint {ad:.6e}, central difference {fd:.6e}, rel {e_fd:.2e}")
    assert fd > 0 and e_fd <= 1e-3


@pytest.mark.parametrize("gamma", [1.0, 5.0])
def test_fp64_adjoint_matches_central_differences(g, gamma):
    """The FP64 instantiation of the GPU adjoint (ddgi_diff_backward_f64)
    against FP64 central differences of the GPU's own FP64 forward
    (ddgi_diff_forward_f64), every albedo and emitter component, h = 1e-6
    max(1, |theta|): within 1e-5 relative.  Hits are the same in both
    evaluations (FP32 geometry, a constant of the parameters), so this checks
    the adjoint's arithmetic.  The FP64 forward and gradient are also
    compared with the oracle's, which differ from them only through the
    FP32 ray directions and hit distances."""
    sc, L, desc, pos, nrm, G, cam = _setup(gamma)
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    alb = torch.tensor(sc.object_albedo, dtype=torch.float64, device="cuda")
    em = torch.tensor(sc.emitter_radiance, dtype=torch.float64, device="cuda")
    P, N_ = to_dev(pos), to_dev(nrm)
    Gd = torch.tensor(G, dtype=torch.float64, device="cuda")
    E = V.diff_forward_f64(S, L, alb, em, P, N_, cam)
    ga, ge = V.diff_backward_f64(S, L, alb, P, N_, cam, Gd, em.shape[0])
    ga, ge = ga.cpu().numpy(), ge.cpu().numpy()

    def loss(a, e):
        return float((V.diff_forward_f64(S, L, a, e, P, N_, cam) * Gd).sum())

    scale = max(np.abs(ga).max(), np.abs(ge).max())
    worst = 0.0
    for which, base, grad in (("albedo", alb, ga), ("emit", em, ge)):
        for k in range(base.shape[0]):
            for c in range(3):
                th = float(base[k, c])
                h = 1e-6 * max(1.0, abs(th))
                up, dn = base.clone(), base.clone()
                up[k, c] += h
                dn[k, c] -= h
                fd = ((loss(up, em) - loss(dn, em)) if which == "albedo" else (loss(alb, up) - loss(alb, dn))) / (2 * h)
                worst = max(worst, abs(grad[k, c] - fd) / max(abs(fd), 1e-3 * scale))
    E_ref, g_em_ref, g_al_ref = oracle.diff(oracle.SceneHandle(sc), L, desc, pos, nrm, cam, G)
    eE = rel_err(E.cpu().numpy(), E_ref)
    print(f"[adjoint fp64] gamma {gamma}: adjoint vs central differences max rel {worst:.2e}; against the oracle: "
          f"forward median {np.median(eE):.2e} (max {eE.max():.2e}), albedo grad {rel_err(ga, g_al_ref).max():.2e}, "
          f"emitter grad {rel_err(ge, g_em_ref).max():.2e}")
    assert worst <= 1e-5
    assert np.median(eE) <= 1e-5
