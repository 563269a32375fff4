"""GPU adjoint (ddgi_diff_forward / ddgi_diff_backward behind
torch.autograd.Function) against the oracle's FP64 reverse-mode gradient,
which test_oracle_adjoint pins to FP64 central differences."""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity import rel_err, to_dev
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
    sc, L, desc, pos, nrm, G, cam = _setup(gamma)
    E_ref, g_em_ref, g_al_ref = oracle.diff(oracle.SceneHandle(sc), L, desc, pos, nrm, cam, G)
    S = g.Scene.from_arrays(sc)
    V = g.Volume(desc)
    albedo = torch.tensor(sc.object_albedo, dtype=torch.float32, device="cuda", requires_grad=True)
    emit = torch.tensor(sc.emitter_radiance, dtype=torch.float32, device="cuda", requires_grad=True)
    P, N_ = to_dev(pos), to_dev(nrm)
    E = g.IrradianceField.apply(albedo, emit, V, S, L, P, N_, cam, 0, 2)
    (E * to_dev(G)).sum().backward()
    e = rel_err(E.detach().cpu().numpy(), E_ref).max()
    ea = rel_err(albedo.grad.cpu().numpy(), g_al_ref).max()
    ee = rel_err(emit.grad.cpu().numpy(), g_em_ref).max()
    print(f"[adjoint] gamma {gamma}: forward max rel {e:.2e}, albedo grad {ea:.2e}, emitter grad {ee:.2e}")
    # the forward is the FP32 update + query; with 32 rays per probe the query's
    # Chebyshev variance (mu2 - mu^2 of a few rays) cancels most in FP32
    assert e <= 1e-3
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
