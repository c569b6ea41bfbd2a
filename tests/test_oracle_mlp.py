"""Pins of the FP64 reference network (oracle/mlp.py): its analytic gradient
against central finite differences of its own loss, its forward pass and loss
on a hand-built network (fixing each layer's [out][in] layout), and bf16
rounding against known values."""
import numpy as np

from oracle import mlp as M


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    p = rng.normal(size=M.NPARAM) * 0.3
    X = rng.normal(size=(40, M.NIN))
    t = rng.normal(size=40)
    L, g = M.loss_and_grad(p, X, t)
    idx = rng.choice(M.NPARAM, size=60, replace=False)
    idx = np.concatenate([idx, [M.NPARAM - 1, 0, 320, 384, 4544]])   # b3, W1, b1, W2, w3 entries
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (M.loss_and_grad(pp, X, t)[0] - M.loss_and_grad(pm, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-6 * abs(fd), (i, fd, g[i])


def test_bf16_rounding():
    assert M.bf16_round(1.0) == 1.0
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert M.bf16_round(1.0 + 2.0 ** -8) == 1.0
    assert M.bf16_round(1.0 + 3 * 2.0 ** -9) == 1.0 + 2.0 ** -7
    assert M.bf16_round(-2.0) == -2.0


def test_forward_hand_network():
    """A network of single weights routes feature 0 through hidden units 7 and
    3: W1[7][0] = 1 (W1 is [out][in]), W2[3][7] = 1, w3[3] = 1, so
    y = tanh(tanh(x_0)) + b3 with the biases b1 = b2 = 0.  A transposed W2
    (shape-valid at 64 x 64) would give y = b3; a bias b1[7] = s shifts the
    inner argument.  The loss is the mean of (y - t)^2."""
    p = np.zeros(M.NPARAM)
    o_b1 = M.NH * M.NIN
    o_W2 = o_b1 + M.NH
    o_w3 = o_W2 + M.NH * M.NH + M.NH
    p[7 * M.NIN + 0] = 1.0
    p[o_W2 + 3 * M.NH + 7] = 1.0
    p[o_w3 + 3] = 1.0
    p[-1] = 0.25
    X = np.array([[0.3, 9.0, -9.0, 9.0, -9.0], [-1.2, 0.0, 0.0, 0.0, 0.0]])
    y, _ = M.forward(p, X)
    assert np.allclose(y, np.tanh(np.tanh(X[:, 0])) + 0.25, rtol=0, atol=1e-15)
    p[o_b1 + 7] = 0.5
    y, _ = M.forward(p, X)
    assert np.allclose(y, np.tanh(np.tanh(X[:, 0] + 0.5)) + 0.25, rtol=0, atol=1e-15)
    t = np.array([1.0, -1.0])
    L, _ = M.loss_and_grad(p, X, t)
    assert abs(L - np.mean((y - t) ** 2)) <= 1e-15
