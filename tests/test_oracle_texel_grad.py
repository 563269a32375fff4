"""The oracle's texel gradient of the query (the texel half of the adjoint),
pinned to FP64 central differences of the oracle's forward query (Sec. 2.2
query, Sec. 4.2 gamma decode), which the other oracle pins fix
independently.  CPU only."""
import numpy as np
import pytest

import oracle
import synth


def _case(gamma, seed=5):
    desc = synth.VolumeDesc(origin=(0.5, 0.5, 0.5), spacing=(1.0, 1.25, 1.5), counts=(3, 3, 3), rays_per_probe=16,
                            irr_n=4, dist_n=6, gamma=gamma, state_machine=1, seed=1)
    rng = np.random.default_rng(seed)
    P = desc.n_probes
    st = np.full(P, oracle.VIGILANT, dtype=np.uint8)
    st[rng.choice(P, 3, replace=False)] = oracle.SLEEPING          # some cage probes unused
    N, M = desc.irr_n + 2, desc.dist_n + 2
    irr = np.zeros((P, N, N, 3))
    dist = np.zeros((P, M, M, 2))
    for p in range(P):
        t = np.zeros((N, N, 3))
        t[1:-1, 1:-1] = rng.uniform(0.2, 1.0, (desc.irr_n, desc.irr_n, 3))
        irr[p] = oracle.border_copy(t, desc.irr_n)
        mu = rng.uniform(0.3, 2.0, (desc.dist_n, desc.dist_n))
        d = np.zeros((M, M, 2))
        d[1:-1, 1:-1, 0] = mu
        d[1:-1, 1:-1, 1] = mu * mu + rng.uniform(0.0, 0.3, mu.shape)
        dist[p] = oracle.border_copy(d, desc.dist_n)
    n = 48
    lo = np.asarray(desc.origin) + 0.1
    hi = np.asarray(desc.origin) + (np.asarray(desc.counts) - 1) * np.asarray(desc.spacing) - 0.1
    pos = rng.uniform(lo, hi, (n, 3))
    nrm = rng.normal(size=(n, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    nrm[0] = 0.0                                                     # a background pixel: no gradient
    dE = rng.uniform(-1.0, 1.0, (n, 3))
    return desc, st, irr, dist, pos, nrm, dE, np.array([3.0, 4.0, -2.0])


def _loss(desc, st, irr, dist, pos, nrm, cam, dE):
    return float((oracle.query(desc, st, irr, dist, pos, nrm, cam) * dE).sum())


@pytest.mark.parametrize("gamma", [1.0, 5.0])
def test_texel_gradient_matches_central_differences(gamma):
    desc, st, irr, dist, pos, nrm, dE, cam = _case(gamma)
    g = oracle.query_texel_grad(desc, st, irr, dist, pos, nrm, cam, dE)
    assert g.shape == irr.shape
    rng = np.random.default_rng(7)
    nz = np.argwhere(g != 0.0)
    zs = np.argwhere(g == 0.0)
    assert len(nz) > 50 and len(zs) > 0
    pick = np.concatenate([nz[rng.choice(len(nz), 60, replace=False)], zs[rng.choice(len(zs), 12, replace=False)]])
    worst = 0.0
    for idx in map(tuple, pick):
        h = 1e-6 * max(1.0, abs(irr[idx]))
        a, b = irr.copy(), irr.copy()
        a[idx] += h
        b[idx] -= h
        fd = (_loss(desc, st, a, dist, pos, nrm, cam, dE) - _loss(desc, st, b, dist, pos, nrm, cam, dE)) / (2 * h)
        err = abs(g[idx] - fd) / max(abs(fd), 1e-3 * np.abs(g).max())
        worst = max(worst, err)
    print(f"texel gradient vs central differences (gamma {gamma}): max rel {worst:.2e}")
    assert worst <= 1e-5


def test_texel_gradient_fold_is_the_interior_gradient():
    """Folded gradients are those of the interior texels as free parameters,
    the borders following them by the Sec. 7.1 copy: perturbing an interior
    texel together with its border copies moves the loss by the folded value;
    the folded border entries are zero."""
    desc, st, irr, dist, pos, nrm, dE, cam = _case(5.0, seed=11)
    gf = oracle.query_texel_grad(desc, st, irr, dist, pos, nrm, cam, dE, fold=True)
    g = oracle.query_texel_grad(desc, st, irr, dist, pos, nrm, cam, dE)
    n = desc.irr_n
    assert np.all(gf[:, 0, :] == 0) and np.all(gf[:, -1, :] == 0)
    assert np.all(gf[:, :, 0] == 0) and np.all(gf[:, :, -1] == 0)
    assert np.isclose(gf.sum(), g.sum(), rtol=1e-12, atol=1e-12)   # the fold moves gradient, it adds none
    rng = np.random.default_rng(3)
    worst = 0.0
    active = np.nonzero(np.abs(gf).reshape(len(gf), -1).sum(1) > 0)[0]
    for _ in range(40):
        p = int(rng.choice(active))
        i, j, c = int(rng.integers(1, n + 1)), int(rng.integers(1, n + 1)), int(rng.integers(0, 3))
        h = 1e-6

        def moved(sign):
            t = irr[p].copy()
            t[j, i, c] += sign * h
            out = irr.copy()
            out[p] = oracle.border_copy(t, n)
            return out
        fd = (_loss(desc, st, moved(1), dist, pos, nrm, cam, dE) - _loss(desc, st, moved(-1), dist, pos, nrm, cam,
                                                                         dE)) / (2 * h)
        worst = max(worst, abs(gf[p, j, i, c] - fd) / max(abs(fd), 1e-3 * np.abs(gf).max()))
    print(f"folded texel gradient vs central differences: max rel {worst:.2e}")
    assert worst <= 1e-5
