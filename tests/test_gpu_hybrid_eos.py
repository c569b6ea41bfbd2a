"""The hybrid piecewise-polytrope EOS (Sec. 3.4) on the CUDA path against the
oracle: prim -> cons, con2prim on stress cells and on hostile and cold inputs,
and whole RK3 stages of star sub-blocks (surface and core, FOFC) with fluxes."""
import numpy as np
import pytest

import oracle as O
from paper_2409_10384_gb300 import synth
from tests import gpu_util as U
from tests.helpers import rel_err
import tests.test_gpu_parity as T

pytestmark = pytest.mark.gpu

G = T.G   # the module fixture: the built library

# three pieces on the stress distribution's density range
HYB = dict(eos=1, eos_pieces=3, eos_K0=1e-4, eos_gamma_th=1.8, eos_rho=(1e-8, 1e-4, 0.0),
           eos_gamma=(1.7, 2.4, 2.1, 0.0))
# three pieces under the star's pressure P = 100 rho^2: the cold part is at
# most half of it, at every density of the star and its atmosphere
HYB_STAR = dict(eos=1, eos_pieces=3, eos_K0=50.0 * (1e-5) ** -0.5, eos_gamma_th=2.0, eos_rho=(1e-5, 5e-4, 0.0),
                eos_gamma=(2.5, 2.0, 1.8, 0.0))


def _stress(n, seed, p):
    prim, Bd, g = synth.c2p_stress(n, seed=seed)
    T_ = prim[4] / prim[0]
    Pc = np.array([O.eos(p, r, 1.0)["Pc"] for r in prim[0]])
    prim[4] = Pc + prim[0] * np.maximum(T_, 10 * p.T_atm)
    return prim, Bd, g


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_hybrid_prim2cons_cells(G):
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-20, T_atm=1e-14, f_thr=0.0, **HYB)
    prim, Bd, g = _stress(20000, 21, p)
    ref = O.prim2cons(p, prim, Bd, g)
    ctx = T._ctx(G, p)
    out = torch.zeros((5, prim.shape[1]), dtype=torch.float64, device="cuda")
    ctx.prim2cons(_t(prim), _t(Bd), _t(g), out)
    got = out.cpu().numpy()
    assert rel_err(got[0], ref[0]) < U.CONS_TOL
    smag = np.abs(ref[1:4]).max(axis=0)
    assert np.max(np.abs(got[1:4] - ref[1:4]) / smag) < U.CONS_TOL
    assert np.max(np.abs(got[4] - ref[4]) / (np.abs(ref[4]) + np.abs(ref[0]))) < U.CONS_TOL


@pytest.mark.parametrize("n", [1, 40000])
def test_hybrid_c2p_cells_stress(G, n):
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-20, T_atm=1e-14, f_thr=0.0, **HYB)
    prim, Bd, g = _stress(n, 22, p)
    cons = O.prim2cons(p, prim, Bd, g)
    ref = O.c2p_cells(p, cons, Bd, g)
    ctx = T._ctx(G, p)
    dp = torch.zeros((5, n), dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    it = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.c2p_cells(_t(cons), _t(Bd), _t(g), dp, fl, it)
    got = dp.cpu().numpy()
    assert np.array_equal(fl.cpu().numpy(), ref["flags"])
    assert np.all(ref["flags"] == 0)
    assert rel_err(got[0], ref["prim"][0], 0.0) < U.PRIM_TOL
    W = np.sqrt(1 + (ref["prim"][1:4] ** 2).sum(0))
    assert np.max(np.abs(got[1:4] - ref["prim"][1:4]) / W) < U.PRIM_TOL
    det = g[0] * (g[3] * g[5] - g[4] ** 2) - g[1] * (g[1] * g[5] - g[4] * g[2]) + g[2] * (g[1] * g[4] - g[3] * g[2])
    scale = (p.eos_gamma_th - 1) * (cons[0] + cons[4]) / np.sqrt(det)
    assert np.all(np.abs(got[4] - ref["prim"][4]) <= 1e-10 * np.abs(ref["prim"][4]) + 1e-12 * scale)
    assert ctx.read_stats()["fails"] == 0


def test_hybrid_c2p_floors_and_cold_matter(G):
    """Atmosphere reset, tau floor, NaN, and matter on the cold curve (T = 0):
    the same flags as the oracle and the floored pressure P_c + rho T_atm."""
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-10, T_atm=1e-8, f_thr=1.0, **HYB)
    g1 = np.array([[1.0], [0], [0], [1.0], [0], [1.0]])
    B1 = np.array([[0.0], [1e-6], [0.0]])
    cols = [np.array([1e-12, 1e-13, 0.0, 0.0, 1e-20]), np.array([1e-3, 0.0, 0.0, 0.0, 1e-30]),
            np.array([np.nan, 0.0, 0.0, 0.0, 1.0])]
    for rho in (1e-9, 1e-5, 1e-2):
        Pc = O.eos(p, rho, 1.0)["Pc"]
        cols.append(O.prim2cons(p, np.array([[rho], [0.2], [0.0], [0.0], [Pc]]), B1, g1)[:, 0])
    cons = np.stack(cols, axis=1)
    n = cons.shape[1]
    g, Bd = np.tile(g1, (1, n)), np.tile(B1, (1, n))
    ref = O.c2p_cells(p, cons, Bd, g)
    ctx = T._ctx(G, p)
    dc = _t(cons)
    dp = torch.zeros((5, n), dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ctx.c2p_cells(dc, _t(Bd), _t(g), dp, fl)
    got = dp.cpu().numpy()
    assert np.array_equal(fl.cpu().numpy(), ref["flags"]), (fl.cpu().numpy(), ref["flags"])
    assert np.all(ref["flags"][3:] & O.F_TEMP)
    for c in range(n):
        assert np.allclose(got[:, c], ref["prim"][:, c], rtol=1e-10, atol=1e-300), (c, got[:, c], ref["prim"][:, c])


def test_hybrid_rejects_fp32_guesses_and_bad_pieces(G):
    for kw in (dict(c2p_guess=1), dict(c2p_guess=2), dict(eos_pieces=0), dict(eos_pieces=5),
               dict(eos_rho=(1e-4, 1e-8, 0.0)), dict(eos_gamma_th=1.0), dict(eos_K0=0.0)):
        d = dict(HYB)
        d.update(kw)
        with pytest.raises(RuntimeError):
            G.Context(G.params(gamma=2.0, **d))


def _star_hyb(p, corner):
    inp = synth.star_subblock(sub=24, corner=corner)
    # the star's atmosphere sits at P = rho T_atm; lift it to the hybrid floor
    prim = inp.prim.copy()
    rho = prim[0].ravel()
    pf = np.array([O.eos(p, r, 1.0)["Pc"] for r in rho]) + rho * p.T_atm
    prim[4] = np.maximum(prim[4].ravel(), pf).reshape(prim[4].shape)
    return inp, prim


@pytest.mark.parametrize("where,recon,rs,guess", [("surface", 2, 1, 0), ("core", 2, 0, 0), ("surface", 3, 1, 0),
                                                 ("surface", 2, 1, 3)])
def test_hybrid_stage_star(G, where, recon, rs, guess):
    """All three RK3 substeps of a star sub-block with the hybrid EOS and FOFC,
    fluxes and states against the oracle; guess 3: the warm-started bracket."""
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=recon, rsolver=rs, rk_order=3,
                 fofc=1, **HYB_STAR)
    corner = (104, 52, 52) if where == "surface" else (52, 52, 52)
    inp, prim = _star_hyb(p, corner)
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, prim, inp.A)
    ctx = G.Context(G.params(**{k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"}, c2p_guess=guess))
    dt = 0.25 * inp.dx[0]
    for s in range(3):
        ref, got, flips = T._run_stage_pair(G, ctx, p, ob, dt, s)
        U.compare_prims(ref, got, p, f"stage {s}")
        U.compare_state(ref, got, f"stage {s}", scales=ref.scales)
        ob.cons[...] = got["cons"]
        ob.cons0[...] = got["cons0"]
        for d in range(3):
            ob.bf[d][...] = got["bf"][d]
            ob.bf0[d][...] = got["bf0"][d]
