"""Pins of the FP64 reference network (oracle/mlp.py): its analytic gradient
against central finite differences of its own loss, and bf16 rounding against
known values."""
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
