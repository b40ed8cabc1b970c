"""Pins of the oracle's predictor network (CPU only).

The forward pass is checked against torch.nn layers (a library routine), the
backward pass against central finite differences of the loss, and the Adam
step against torch.optim.Adam; the descriptors against closed forms on a clean
lattice (moments of the SC density of states count closed walks).
"""
import numpy as np
import pytest

from oracle import descriptors, mlp, systems
from workloads import C1_SYSTEM, C3_SYSTEM, scaled

torch = pytest.importorskip("torch")


def _data(n=64, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((n, mlp.D_IN)), rng.standard_normal(n)


def test_forward_matches_torch_layers():
    p = mlp.init_params(3)
    X, _ = _data()
    net = torch.nn.Sequential(torch.nn.Linear(32, 64), torch.nn.Tanh(), torch.nn.Linear(64, 64), torch.nn.Tanh(),
                              torch.nn.Linear(64, 1)).double()
    with torch.no_grad():
        net[0].weight.copy_(torch.from_numpy(p["W1"]))
        net[0].bias.copy_(torch.from_numpy(p["b1"] + 0.1))
        net[2].weight.copy_(torch.from_numpy(p["W2"]))
        net[2].bias.copy_(torch.from_numpy(p["b2"] - 0.2))
        net[4].weight.copy_(torch.from_numpy(p["w3"][None, :]))
        net[4].bias.copy_(torch.from_numpy(p["b3"] + 0.3))
    p["b1"] = p["b1"] + 0.1
    p["b2"] = p["b2"] - 0.2
    p["b3"] = p["b3"] + 0.3
    y, _ = mlp.forward(p, X)
    ref = net(torch.from_numpy(X)).detach().numpy()[:, 0]
    assert np.abs(y - ref).max() < 1e-12


def test_backward_matches_finite_differences():
    p = mlp.init_params(5)
    X, t = _data(40, 1)
    g = mlp.backward(p, X, t)
    rng = np.random.default_rng(2)
    for name in mlp.PARAM_NAMES:
        for _ in range(6):
            idx = tuple(rng.integers(0, s) for s in p[name].shape)
            h = 1e-6
            pp = {k: v.copy() for k, v in p.items()}
            pm = {k: v.copy() for k, v in p.items()}
            pp[name][idx] += h
            pm[name][idx] -= h
            fd = (mlp.loss(pp, X, t) - mlp.loss(pm, X, t)) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * max(1.0, abs(fd))


def test_adam_matches_torch():
    p = mlp.init_params(7)
    X, t = _data(32, 3)
    tp = {k: torch.tensor(v.copy(), requires_grad=True) for k, v in p.items()}
    opt = torch.optim.Adam(list(tp.values()), lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    ours = mlp.Adam(lr=1e-2)
    for _ in range(3):
        g = mlp.backward(p, X, t)
        ours.step(p, g)
        opt.zero_grad()
        for k in mlp.PARAM_NAMES:
            tp[k].grad = torch.from_numpy(mlp.backward({kk: vv.detach().numpy() for kk, vv in tp.items()}, X, t)[k])
        opt.step()
    for k in mlp.PARAM_NAMES:
        assert np.abs(p[k] - tp[k].detach().numpy()).max() < 1e-12


def test_training_reduces_loss_on_a_learnable_target():
    rng = np.random.default_rng(4)
    X = rng.standard_normal((512, 32))
    t = np.tanh(X[:, 0] - 0.5 * X[:, 3]) + 0.1 * X[:, 7]
    p = mlp.init_params(0)
    hist = mlp.train(p, X, t, epochs=30, batch=64, lr=3e-3, seed=1)
    assert hist[-1] < 0.1 * hist[0]


def test_descriptor_moments_on_clean_sc_lattice():
    """Clean SC lattice, t = -1, onsite 0: e_j^T H^k e_j counts closed walks of
    length k (0, 6, 0, 90, 0, 1860 for k = 1..6), exact while the subspace
    radius covers the walk's reach (R >= k/2)."""
    s = systems.build_system(scaled(C1_SYSTEM, L=9, onsite_lo=0.0, onsite_hi=0.0), 1)
    d = descriptors.descriptor(s, 0, 4)
    walks = {2: 6.0, 3: 0.0, 4: 90.0, 5: 0.0, 6: 1860.0, 7: 0.0, 8: 44730.0}
    for k, w in walks.items():
        got = np.sign(d[9 + k - 2]) * abs(d[9 + k - 2]) ** k
        assert abs(got - w) < 1e-8 * max(1.0, w)
    assert d[2] * 100 == 6 and d[3] * 100 == 18 and d[4] * 100 == 38 and d[5] * 100 == 66
    assert d[7] == 0.5 and d[8] == 0.0
    # FCC bulk atom: 12 neighbours, shells 12, 42, 92
    f = systems.build_system(scaled(C3_SYSTEM, n_sites=3000, bdim=1), 1)
    origin = int(np.nonzero((f.coords == 0).all(axis=1))[0][0])
    d = descriptors.descriptor(f, origin, 3)
    assert d[7] == 1.0 and np.allclose(d[2:5] * 100, [12, 42, 92])
