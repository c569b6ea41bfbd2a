"""Learned con2prim guess on the GPU: the tensor-core network against the FP64
reference (forward and gradients), and the learned con2prim against the plain
one and the oracle (same root, fewer FP64 iterations)."""
import numpy as np
import pytest

import oracle as O
from oracle import mlp as M
from paper_2409_10384_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10384_gb300 import build, grmhd
    build.build()
    return grmhd


def _state(p, fmean=None, finv=None, ym=0.0, ys=1.0, delta=0.1):
    st = np.zeros(M.NPARAM + 13, np.float32)
    st[:M.NPARAM] = p
    st[M.NPARAM:M.NPARAM + 5] = 0.0 if fmean is None else fmean
    st[M.NPARAM + 5:M.NPARAM + 10] = 1.0 if finv is None else finv
    st[M.NPARAM + 10] = ym
    st[M.NPARAM + 11] = ys
    st[M.NPARAM + 12] = delta
    return st


def _bf16_forward(p, X):
    """The reference forward with the tensor-core operand roundings: weights,
    inputs and hidden activations rounded to bf16, FP64 elsewhere."""
    W1, b1, W2, b2, w3, b3 = M.unpack(p)
    r = M.bf16_round
    H1 = np.tanh(r(X) @ r(W1).T + b1)
    H2 = np.tanh(r(H1) @ r(W2).T + b2)
    return r(H2) @ r(w3) + b3


def test_forward_matches_reference(G):
    import torch
    rng = np.random.default_rng(1)
    p = (rng.normal(size=M.NPARAM) * 0.2).astype(np.float32)
    ctx = G.Context(G.params())
    ctx.mlp_set(_state(p))
    n = 1000
    X = rng.normal(size=(n, M.NIN)).astype(np.float32)
    feat = np.zeros((n, 8), np.float32)
    feat[:, :5] = X
    y = ctx.mlp_infer(torch.from_numpy(feat).cuda()).cpu().numpy()
    ref = _bf16_forward(p.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(y - ref)) < 2e-3 * (1 + np.abs(ref).max())
    ref64, _ = M.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(y - ref64)) < 5e-2 * (1 + np.abs(ref64).max())


def test_gradients_match_reference(G):
    """Gradients of the mean squared error from the hand-written backward
    kernels against the FP64 reference within 1e-2 (bf16 operands)."""
    import torch
    rng = np.random.default_rng(2)
    p = (rng.normal(size=M.NPARAM) * 0.2).astype(np.float32)
    ctx = G.Context(G.params())
    ctx.mlp_set(_state(p))
    n = 512
    X = rng.normal(size=(n, M.NIN)).astype(np.float32)
    t = rng.normal(size=n).astype(np.float32)
    feat = np.zeros((n, 8), np.float32)
    feat[:, :5] = X
    g, L = ctx.mlp_grad(torch.from_numpy(feat).cuda(), torch.from_numpy(t).cuda())
    Lr, gr = M.loss_and_grad(p.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(L - Lr) <= 2e-2 * Lr
    assert np.linalg.norm(g - gr) <= 1e-2 * np.linalg.norm(gr)
    # every block of parameters on its own
    o = 0
    for size in (320, 64, 4096, 64, 64, 1):
        a, b = g[o:o + size], gr[o:o + size]
        assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-6, (o, size)
        o += size


def _cells(G, n, seed):
    import torch
    prim, Bd, g = synth.c2p_stress(n, seed=seed)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return prim, Bd, g, t(Bd), t(g), t(prim)


def test_learned_con2prim_same_root_fewer_iterations(G):
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-20, T_atm=1e-14, f_thr=0.0)
    kw = {k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"}
    ctx = G.Context(G.params(**kw, c2p_guess=0))
    # training data (disjoint seeds), made by the plain solver
    _, _, _, dB, dg, dprim = _cells(G, 300000, 104)
    cons = torch.zeros_like(dprim)
    ctx.prim2cons(dprim, dB, dg, cons)
    feat, logmu = ctx.mlp_dataset(cons, dB, dg)
    assert torch.isfinite(logmu).all()
    ctx.mlp_init(3)
    loss = ctx.mlp_train(feat, logmu, epochs=30, batch=4096, lr=3e-3)
    assert loss < 0.02
    _, _, _, vB, vg, vprim = _cells(G, 100000, 105)
    vcons = torch.zeros_like(vprim)
    ctx.prim2cons(vprim, vB, vg, vcons)
    vf, vl = ctx.mlp_dataset(vcons, vB, vg)
    delta = ctx.mlp_calibrate(vf, vl, 0.95)
    assert 0 < delta < 0.3
    # test set: plain vs learned vs oracle
    n = 50000
    prim, Bd, g, tB, tg, tprim = _cells(G, n, 106)
    c0 = torch.zeros_like(tprim)
    ctx.prim2cons(tprim, tB, tg, c0)
    out = {}
    for guess in (0, 1, 2):
        ctx.set_params(G.params(**kw, c2p_guess=guess))
        cc = c0.clone()
        pr = torch.zeros_like(tprim)
        fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
        it = torch.zeros(n, dtype=torch.int32, device="cuda")
        ctx.reset_stats()
        ctx.c2p_cells(cc, tB, tg, pr, fl, it)
        st = ctx.read_stats()
        out[guess] = (pr.cpu().numpy(), fl.cpu().numpy(), it.cpu().numpy())
        # cells whose FP32 root missed the 4e-6 bracket: none without a guess,
        # a small fraction with one
        assert st["cells"] == n
        assert st["guess_fallbacks"] == 0 if guess == 0 else st["guess_fallbacks"] <= 0.1 * n, (guess, st)
    p0, f0, i0 = out[0]
    cons = c0.cpu().numpy()
    det = g[0] * (g[3] * g[5] - g[4] ** 2) - g[1] * (g[1] * g[5] - g[4] * g[2]) + g[2] * (g[1] * g[4] - g[3] * g[2])
    scale = (p.gamma - 1) * (cons[0] + cons[4]) / np.sqrt(det)
    W = np.sqrt(1 + (p0[1:4] ** 2).sum(0))
    ref = O.c2p_cells(p, cons, Bd, g)
    for guess in (1, 2):
        p1, f1, i1 = out[guess]
        # the same root: identical flags, primitives within the parity bars
        assert np.array_equal(f0, f1)
        assert np.max(np.abs(p1[0] - p0[0]) / p0[0]) < 1e-10
        assert np.max(np.abs(p1[1:4] - p0[1:4]) / W) < 1e-10
        assert np.all(np.abs(p1[4] - p0[4]) <= 1e-10 * np.abs(p0[4]) + 1e-12 * scale)
        assert np.max(np.abs(p1[0] - ref["prim"][0]) / ref["prim"][0]) < 1e-10
    # FP64 evaluations of the master function per cell (plain: + the mu+ steps)
    print("FP64 evaluations per cell: plain %.2f  learned %.2f  fp32-search %.2f"
          % (i0.mean(), out[1][2].mean(), out[2][2].mean()))
    assert out[1][2].mean() < i0.mean()
