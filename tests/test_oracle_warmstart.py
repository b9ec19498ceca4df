"""Pins of the warm-start network oracle (oracle/warmstart.py) against facts that do not come from
the oracle itself: BF16 values of known numbers, closed forms of the network, central finite
differences of the loss, the closed form of Adam's first step, and the 1-ring of a lattice node.
"""
import numpy as np
import pytest

from oracle import warmstart as ws
from paper_0809_4802_gb300 import inputs


def test_bf16_rounding_of_known_values():
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties go to the even mantissa (1.0)
    vals = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -9, np.pi, -2.5, 65504.0, 1e-3], np.float32)
    expect = np.array([1.0, 1.0, 1.0078125, 3.140625, -2.5, 65536.0, 0.00099945068359375])
    np.testing.assert_array_equal(ws.bf16_round(vals), expect)


def random_params(seed, scale=0.3):
    rng = np.random.default_rng(seed)
    return ws.unpack(rng.uniform(-scale, scale, ws.N_PARAMS))


def test_forward_closed_forms():
    p = random_params(1)
    x = np.random.default_rng(2).normal(size=(5, ws.N_IN))
    # with the second layer switched off the output is the last bias
    q = dict(p, W2=np.zeros_like(p["W2"]), b2=np.zeros_like(p["b2"]))
    y, _ = ws.forward(q, x)
    np.testing.assert_array_equal(y, np.broadcast_to(q["b3"], y.shape))
    # one path through the network: y_0 = w3 tanh(w2 tanh(w1 x_0 + c1) + c2) + c3
    q = {k: np.zeros_like(v) for k, v in p.items()}
    q["W1"][0, 0], q["b1"][0] = 0.7, -0.2
    q["W2"][0, 0], q["b2"][0] = -1.3, 0.4
    q["W3"][0, 0], q["b3"][0] = 2.0, 0.1
    y, _ = ws.forward(q, x)
    ref = 2.0 * np.tanh(-1.3 * np.tanh(0.7 * x[:, 0] - 0.2) + 0.4) + 0.1
    np.testing.assert_allclose(y[:, 0], ref, rtol=1e-15, atol=0)
    np.testing.assert_array_equal(y[:, 1:], 0.0)


def test_gradient_matches_central_differences():
    p = random_params(3)
    rng = np.random.default_rng(4)
    x = rng.normal(size=(6, ws.N_IN))
    t = rng.normal(size=(6, ws.N_OUT))
    _, g = ws.loss_and_grad(p, x, t)
    flat, gflat = ws.pack(p), ws.pack(g)
    idx = np.concatenate([rng.choice(ws.N_PARAMS, 300, replace=False),
                          np.arange(ws.N_PARAMS - 4, ws.N_PARAMS)])   # and every b3
    h = 1e-6
    for i in idx:
        fp, fm = flat.copy(), flat.copy()
        fp[i] += h
        fm[i] -= h
        lp, _ = ws.loss_and_grad(ws.unpack(fp), x, t)
        lm, _ = ws.loss_and_grad(ws.unpack(fm), x, t)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gflat[i]) <= 1e-7 + 1e-6 * abs(gflat[i]), (i, fd, gflat[i])


def test_adam_first_step_is_a_signed_step():
    rng = np.random.default_rng(5)
    w, g = rng.normal(size=50), rng.normal(size=50)
    w1, m1, v1 = ws.adam_step(w, g, np.zeros(50), np.zeros(50), t=1, lr=1e-2)
    # mhat = g, vhat = g^2 after the first step: the update is lr * g / (|g| + eps)
    np.testing.assert_allclose(w1, w - 1e-2 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g)
    np.testing.assert_allclose(v1, 0.001 * g * g)


def test_ring_mean_on_a_lattice():
    mesh = inputs.cavity_mesh(4)
    n = mesh.n_nodes
    const = np.full((n, 4), 2.5)
    np.testing.assert_allclose(ws.ring_mean(mesh.conn, n, const), const)
    # an interior node has 26 neighbours placed symmetrically: the ring mean of a linear field
    # is its own value there
    lin = np.stack([mesh.xyz @ c for c in ([1.0, 2.0, -1.0], [0.3, 0, 0], [0, 0, 1], [1, 1, 1])], 1)
    inner = np.all((mesh.node_ijk > 0) & (mesh.node_ijk < 4), axis=1)
    np.testing.assert_allclose(ws.ring_mean(mesh.conn, n, lin)[inner], lin[inner], atol=1e-13)
    # a corner node of the cube has 7 neighbours
    corner = np.nonzero(np.all(mesh.node_ijk == 0, axis=1))[0][0]
    x = np.zeros((n, 1))
    x[:, 0] = np.arange(n)
    nb = sorted(set(mesh.conn[np.any(mesh.conn == corner, axis=1)].ravel()) - {corner})
    assert len(nb) == 7
    assert ws.ring_mean(mesh.conn, n, x)[corner, 0] == pytest.approx(np.mean(nb))


def test_features_layout_and_scaling():
    mesh = inputs.cavity_mesh(2)
    rng = np.random.default_rng(6)
    un, um = rng.normal(size=(mesh.n_nodes, 4)), rng.normal(size=(mesh.n_nodes, 4))
    s = np.arange(1, 13, dtype=np.float64)
    x = ws.features(mesh.conn, un, um, s)
    np.testing.assert_allclose(x[:, :4] * s[:4], un)
    np.testing.assert_allclose(x[:, 4:8] * s[4:8], un - um)
    np.testing.assert_allclose(x[:, 8:] * s[8:], ws.ring_mean(mesh.conn, mesh.n_nodes, un - um))
