"""Pins for the fp64 reference of the branching-order network (oracle/mlp.py):
central finite differences for the gradient, closed forms for the forward
pass and the loss, and hand-computed vertex features."""
import numpy as np

import synth
from oracle import mlp


def _edges(n, e, directed=False):
    a = np.zeros((n, n), np.uint8)
    for i, j in e:
        a[i, j] = 1
        if not directed:
            a[j, i] = 1
    return a


def test_features_hand_cases():
    # path 0-1-2: degrees 1, 2, 1
    f = mlp.vertex_features(_edges(3, [(0, 1), (1, 2)]))
    assert np.allclose(f[:, 0], [1 / 16, 2 / 16, 1 / 16])
    assert f[0, 2 + 2] == 0.25 and f[0, 2:].sum() == 0.25        # neighbour 1 has degree 2
    assert f[1, 2 + 1] == 0.5 and f[1, 2:].sum() == 0.5          # neighbours 0, 2 have degree 1
    assert (f[:, 1] == 0).all()
    # labels
    f = mlp.vertex_features(_edges(3, [(0, 1)]), labels=np.array([0, 5, 100]))
    assert np.allclose(f[:, 1], [0, 5 / 8, 63 / 8])
    # directed: arcs both ways count twice in the degree, the neighbour once
    a = _edges(3, [(0, 1), (1, 0), (1, 2)], directed=True)
    f = mlp.vertex_features(a, directed=True)
    assert np.allclose(f[:, 0], [2 / 16, 3 / 16, 1 / 16])
    assert f[1, 2 + 2] == 0.25 and f[1, 2 + 1] == 0.25           # nbrs 0 (deg 2) and 2 (deg 1)
    # degrees above 15 share the last bin; self-loops are ignored
    k = np.ones((20, 20), np.uint8)
    f = mlp.vertex_features(k)
    assert np.allclose(f[:, 0], 19 / 16) and np.allclose(f[:, 2 + 15], 19 * 0.25)


def test_features_permutation_equivariant():
    rng = synth.rng_for(5, 0, 0)
    a = synth.er_undirected(15, 0.3, rng)
    perm = rng.permutation(15)
    f = mlp.vertex_features(a)
    fp = mlp.vertex_features(a[np.ix_(perm, perm)])
    assert np.allclose(fp, f[perm])


def test_forward_closed_form():
    th = np.zeros(mlp.N_PARAMS)
    W1, b1, W2, b2, w3, b3 = mlp.unpack(th)   # views are copies; build by layout instead
    i = mlp.D_PAD * mlp.H
    th[i:i + mlp.H] = 1.0                          # b1 = 1  -> h1 = 1
    i += mlp.H + mlp.H * mlp.H
    th[i:i + mlp.H] = 2.0                          # b2 = 2, W2 = 0 -> h2 = 2
    i += mlp.H
    th[i:i + mlp.H] = 0.5                          # w3 = 0.5
    th[-1] = -3.0                                  # b3
    x = np.random.default_rng(0).normal(size=(4, mlp.D_PAD))
    s, _ = mlp.forward(th, x)
    assert np.allclose(s, 128 * 2 * 0.5 - 3.0)
    # negative pre-activations are cut by the ReLU
    th2 = th.copy()
    th2[mlp.D_PAD * mlp.H:mlp.D_PAD * mlp.H + mlp.H] = -1.0
    s2, _ = mlp.forward(th2, x)
    assert np.allclose(s2, 128 * 2 * 0.5 - 3.0)   # h1 = 0 but b2 still gives h2 = 2
    # loss at s = 0 is log 2 whatever the label
    th3 = np.zeros(mlp.N_PARAMS)
    loss, g = mlp.loss_and_grad(th3, x, np.array([0, 1, 0, 1.0]))
    assert np.isclose(loss, np.log(2.0))
    # the bias gradient at s = 0 is mean(0.5 - y)
    assert np.isclose(g[-1], np.mean(0.5 - np.array([0, 1, 0, 1.0])))


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(7)
    th = mlp.init_params(3) + rng.normal(0, 0.05, mlp.N_PARAMS)
    x = np.zeros((12, mlp.D_PAD))
    x[:, :36] = rng.uniform(0, 1, (12, 36))
    y = (rng.random(12) < 0.4).astype(float)
    w = rng.uniform(0.5, 2.0, 12)
    loss, g = mlp.loss_and_grad(th, x, y, w)
    idx = rng.choice(mlp.N_PARAMS, 300, replace=False)
    idx = np.concatenate([idx, [mlp.N_PARAMS - 1]])
    eps = 1e-6
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += eps
        tm[i] -= eps
        fd = (mlp.loss_and_grad(tp, x, y, w)[0] - mlp.loss_and_grad(tm, x, y, w)[0]) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-4 * abs(fd), (i, fd, g[i])


def test_init_keeps_padding_zero():
    th = mlp.init_params(0)
    W1 = th[:mlp.D_PAD * mlp.H].reshape(mlp.D_PAD, mlp.H)
    assert (W1[mlp.D_IN:] == 0).all()
    assert th.size == mlp.N_PARAMS == 22913
