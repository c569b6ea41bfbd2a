"""GPU (libgrmhd through its C-ABI) against the FP64 oracle, element by element.

Bars: conserved variables and face fields 1e-12 per cell per substep, primitives
1e-10 (relative, per cell, floored at 1e-10 of the field maximum); the pressure
against its recovery scale (see tests/gpu_util.compare_prims).  FOFC flags are a
threshold decision: the oracle is re-run with the GPU's flags injected for the
value comparison, and every flag that differs must sit within rounding of its
threshold.
"""
import numpy as np
import pytest

import oracle as O
from paper_2409_10384_gb300 import synth
from tests import gpu_util as U
from tests.helpers import fill_ghosts, interior, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10384_gb300 import build, grmhd
    build.build()
    return grmhd


def _ctx(G, p):
    gp = G.params(**{k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"})
    return G.Context(gp)


def test_prim2cons_cells(G):
    import torch
    p = O.params(gamma=2.0)
    prim, Bd, g = synth.c2p_stress(50000, seed=4)
    ref = O.prim2cons(p, prim, Bd, g)
    ctx = _ctx(G, p)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    out = torch.zeros((5, prim.shape[1]), dtype=torch.float64, device="cuda")
    ctx.prim2cons(t(prim), t(Bd), t(g), out)
    got = out.cpu().numpy()
    # D~ per cell; S~_i against the momentum magnitude of the cell; tau~ = E~ - D~
    # against E~ (its absolute precision is that of D~)
    assert rel_err(got[0], ref[0]) < U.CONS_TOL
    smag = np.abs(ref[1:4]).max(axis=0)
    assert np.max(np.abs(got[1:4] - ref[1:4]) / smag) < U.CONS_TOL
    assert np.max(np.abs(got[4] - ref[4]) / (np.abs(ref[4]) + np.abs(ref[0]))) < U.CONS_TOL


@pytest.mark.parametrize("n", [1, 33, 200000])
def test_c2p_cells_stress(G, n):
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-20, T_atm=1e-14, f_thr=0.0)
    prim, Bd, g = synth.c2p_stress(n, seed=4)
    cons = O.prim2cons(p, prim, Bd, g)
    ref = O.c2p_cells(p, cons, Bd, g)
    ctx = _ctx(G, p)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dc = t(cons)
    dp = torch.zeros((5, n), dtype=torch.float64, device="cuda")
    fl = torch.zeros(n, dtype=torch.uint8, device="cuda")
    it = torch.zeros(n, dtype=torch.int32, device="cuda")
    ctx.c2p_cells(dc, t(Bd), t(g), dp, fl, it)
    got = dp.cpu().numpy()
    assert np.array_equal(fl.cpu().numpy(), ref["flags"])
    assert rel_err(got[0], ref["prim"][0], 0.0) < U.PRIM_TOL
    W = np.sqrt(1 + (ref["prim"][1:4] ** 2).sum(0))
    assert np.max(np.abs(got[1:4] - ref["prim"][1:4]) / W) < U.PRIM_TOL
    det = g[0] * (g[3] * g[5] - g[4] ** 2) - g[1] * (g[1] * g[5] - g[4] * g[2]) + g[2] * (g[1] * g[4] - g[3] * g[2])
    scale = (p.gamma - 1) * (cons[0] + cons[4]) / np.sqrt(det)
    assert np.all(np.abs(got[4] - ref["prim"][4]) <= 1e-10 * np.abs(ref["prim"][4]) + 1e-12 * scale)
    assert it.cpu().numpy().max() <= p.c2p_maxit + 2
    st = ctx.read_stats()
    assert st["cells"] == n and st["fails"] == 0


def test_c2p_cells_floors_and_bad_input(G):
    """Atmosphere floors and the error policy on hostile inputs: NaN, negative
    D, tau below the floor, momentum beyond causality, a cold state."""
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-10, T_atm=1e-8, f_thr=1.0)
    g = np.tile(np.array([[1.0], [0], [0], [1.0], [0], [1.0]]), (1, 6))
    Bd = np.tile(np.array([[0.0], [1e-6], [0.0]]), (1, 6))
    prim_cold = np.array([[1e-3], [0.3], [0.0], [0.0], [1e-12]])
    cold = O.prim2cons(p, prim_cold, Bd[:, :1], g[:, :1])[:, 0]
    cons = np.array([
        [np.nan, 0.0, 0.0, 0.0, 1.0],
        [-1e-3, 0.0, 0.0, 0.0, 1e-3],
        [1e-3, 0.0, 0.0, 0.0, 1e-30],
        [1.0, 50.0, 0.0, 0.0, 1.0],
        [1e-12, 1e-13, 0.0, 0.0, 1e-20],
        list(cold),
    ]).T.copy()
    ref = O.c2p_cells(p, cons, Bd, g)
    ctx = _ctx(G, p)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dc = t(cons)
    dp = torch.zeros((5, 6), dtype=torch.float64, device="cuda")
    fl = torch.zeros(6, dtype=torch.uint8, device="cuda")
    ctx.c2p_cells(dc, t(Bd), t(g), dp, fl)
    got = dp.cpu().numpy()
    assert np.array_equal(fl.cpu().numpy(), ref["flags"]), (fl.cpu().numpy(), ref["flags"])
    assert np.all(np.isfinite(got))
    for c in range(6):
        assert np.allclose(got[:, c], ref["prim"][:, c], rtol=1e-10, atol=1e-300), c
    gc = dc.cpu().numpy()
    rc = ref["cons"][:, 1:]
    assert np.allclose(gc[:4, 1:], rc[:4], rtol=1e-12, atol=0)
    assert np.all(np.abs(gc[4, 1:] - rc[4]) <= 1e-12 * (np.abs(rc[4]) + np.abs(rc[0])))


def test_init_block_matches_oracle(G):
    import torch
    p = O.params(gamma=5.0 / 3.0)
    inp = synth.periodic_flat(1)
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    ctx = _ctx(G, p)
    db = G.DeviceBlock(inp.n, inp.ng, inp.dx, inp.adm)
    db.prim.copy_(torch.from_numpy(inp.prim))
    ctx.init_block(db, [torch.from_numpy(a).cuda() for a in inp.A])
    got = U.from_device(db)
    for d in range(3):
        assert rel_err(got["bf"][d], ob.bf[d]) < 1e-14
    for v in range(5):
        assert rel_err(got["cons"][v], ob.cons[v]) < 1e-13


def _run_stage_pair(G, ctx, p, ob, dt, s, check_fluxes=True, inject=True):
    """One stage on both sides from the same input; returns (oracle out, gpu
    dict, FOFC flips).  FOFC flags that differ must sit within rounding of
    their threshold, and the oracle is re-run with the GPU's flags.  Faces at
    a reconstruction tie (a limiter decision within rounding) are taken down
    the GPU's branch by the oracle itself (tie_branch_flux) and the stage is
    re-run with those oracle fluxes, so every cell is compared."""
    db = U.to_device(G, ob)
    ctx.stage([db], dt, s)
    got = U.from_device(db)
    mask = None
    flips = []
    if p.fofc and inject:
        I = interior(ob)
        gm = (got["flags"] & O.F_FOFC) != 0
        mask = np.zeros(ob.cons.shape[1:], np.uint8)
        mask[I] = gm[I]
        own = ob.copy()
        O.stage(p, own, dt, s)
        om = (own.flags & O.F_FOFC) != 0
        diff = np.argwhere(gm[I] != om[I])
        if len(diff):
            Us, Upost, bpost = U.ho_ustar(p, ob, dt, s)
            cells = [tuple(int(x) + ob.ng for x in c) for c in diff]
            okk = U.flip_is_rounding(p, Us, Upost, bpost, cells)
            assert all(okk), f"FOFC flag flips away from a threshold at {[c for c, o in zip(cells, okk) if not o]}"
            flips = cells
    ref = ob.copy()
    out = O.stage(p, ref, dt, s, mask=mask, keep=True)
    ref.scales = U.term_scales(p, ob, out, dt, s)
    ref.ties = 0
    ref.flips = len(flips)
    if check_fluxes:
        ties = []
        for d in range(3):
            Fg = ctx.scratch(0, d, out["flux"][d].shape)
            # compare the faces the stage computes (nonzero in the oracle's array)
            m = np.any(out["flux"][d] != 0, axis=0)
            # a flux is a difference of O(U) terms: compare against the field
            # maximum; the tau~ flux carries the precision of the D~ flux
            off = np.zeros(m.shape, bool)
            scd = []
            for c in range(7):
                sc = np.abs(out["flux"][d][c][m]).max() + (np.abs(out["flux"][d][0][m]).max() if c == 4 else 0.0)
                scd.append(sc)
                off |= m & (np.abs(Fg[c] - out["flux"][d][c]) > 1e-13 * sc)
            for face in np.argwhere(off):
                face = tuple(int(x) for x in face)
                assert U.recon_is_tie(p, ref, d, face), ("flux", d, face)
                ties.append((d, face, Fg[(slice(None),) + face].copy(), np.array(scd)))
        assert len(ties) <= 1e-3 * sum(np.prod(ob.face_shape(d)) for d in range(3)), len(ties)
        if ties:
            # the oracle down the GPU's branch at every tie face, then the whole
            # stage again with those (oracle) fluxes: no cell is left out
            ov = [((d,) + face, U.tie_branch_flux(p, ob, d, face, Fgf, scale=scd)) for d, face, Fgf, scd in ties]
            ref = ob.copy()
            out = O.stage(p, ref, dt, s, mask=mask, keep=True, override=ov)
            ref.scales = U.term_scales(p, ob, out, dt, s)
            ref.ties = len(ties)
            ref.flips = len(flips)
    return ref, got, flips


def test_stage_periodic_flat_plm_hlle(G):
    """Configuration 1: 32^3 + 4 ghosts, flat, Gamma 5/3, PLM + HLLE + CT, RK2."""
    p = O.params(gamma=5.0 / 3.0, recon=1, rsolver=1, rk_order=2, fofc=0)
    inp = synth.periodic_flat(1)
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    ctx = _ctx(G, p)
    dt = 0.25 / 32
    for s in range(2):
        fill_ghosts(ob)
        ref, got, _ = _run_stage_pair(G, ctx, p, ob, dt, s)
        U.compare_prims(ref, got, p, f"stage {s}")
        U.compare_state(ref, got, f"stage {s}", scales=ref.scales)
        # next substep starts from the GPU result (per-substep parity)
        ob.cons[...] = got["cons"]
        ob.cons0[...] = got["cons0"]
        for d in range(3):
            ob.bf[d][...] = got["bf"][d]
            ob.bf0[d][...] = got["bf0"][d]


@pytest.mark.parametrize("where,recon,rs,dmp", [("surface", 2, 1, 0.0), ("surface", 2, 0, 1.1),
                                                ("surface", 0, 1, 0.0), ("core", 2, 1, 0.0), ("core", 1, 0, 1.2),
                                                ("surface", 3, 1, 0.0), ("surface", 4, 1, 0.0),
                                                ("core", 3, 0, 0.0), ("core", 4, 1, 1.2), ("surface", 4, 0, 1.1)])
def test_stage_star_fofc(G, where, recon, rs, dmp):
    """Sub-blocks of the 128^3 star workload (dynamical metric with K_ij): over the
    stellar surface (atmosphere, FOFC fires) and over the magnetised core;
    WENO-Z/PLM/PPM4/PPMX/donor + HLLE/LLF + FOFC (+DMP) + CT, all three RK3
    substeps."""
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=recon, rsolver=rs, rk_order=3,
                 fofc=1, dmp_M=dmp)
    corner = (104, 52, 52) if where == "surface" else (52, 52, 52)
    inp = synth.star_subblock(sub=24, corner=corner)
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    ctx = _ctx(G, p)
    dt = 0.25 * inp.dx[0]
    total_flips = 0
    for s in range(3):
        ref, got, flips = _run_stage_pair(G, ctx, p, ob, dt, s)
        total_flips += len(flips)
        U.compare_prims(ref, got, p, f"stage {s}")
        U.compare_state(ref, got, f"stage {s}", scales=ref.scales)
        ob.cons[...] = got["cons"]
        ob.cons0[...] = got["cons0"]
        for d in range(3):
            ob.bf[d][...] = got["bf"][d]
            ob.bf0[d][...] = got["bf0"][d]
    st = ctx.read_stats()
    if where == "surface":
        assert st["fofc_cells"] > 0  # the surface and the atmosphere trigger FOFC
    # every flip was verified above to sit within rounding of its threshold
    assert total_flips <= 0.02 * 24 ** 3


def test_stage_with_excision_matches_oracle(G):
    """The excision floor (Sec. 4.7) over the star's centre, where the lapse
    dips to 0.29 on the grid (alpha_exc = 0.4): all three RK3 substeps against
    the oracle."""
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=2, rsolver=1, rk_order=3, fofc=1,
                 alpha_exc=0.4)
    inp = synth.star_subblock(sub=16, corner=(56, 56, 56))
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    ctx = _ctx(G, p)
    dt = 0.25 * inp.dx[0]
    for s in range(3):
        ref, got, flips = _run_stage_pair(G, ctx, p, ob, dt, s)
        U.compare_prims(ref, got, p, f"stage {s}")
        U.compare_state(ref, got, f"stage {s}", scales=ref.scales)
        ex = inp.adm[0] < 0.4
        assert np.all(got["prim"][0][ex & (ref.flags > 0)] == 1e-12)
        ob.cons[...] = got["cons"]
        ob.cons0[...] = got["cons0"]
        for d in range(3):
            ob.bf[d][...] = got["bf"][d]
            ob.bf0[d][...] = got["bf0"][d]
    assert ctx.read_stats()["floors"] > 0


def test_graph_step_equals_stage_calls(G):
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, recon=2, rsolver=1, rk_order=3, fofc=1)
    inp = synth.star_subblock(sub=16, corner=(56, 56, 56))
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    ctx = _ctx(G, p)
    dt = 0.25 * inp.dx[0]
    a = U.to_device(G, ob)
    b = U.to_device(G, ob)
    for s in range(3):
        ctx.stage([a], dt, s)
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        ctx.step([b], dt, graph=True, stream=stream)
        ctx.step([b], dt, graph=True, stream=stream)   # replay
    stream.synchronize()
    torch.cuda.synchronize()
    for s in range(3):
        ctx.stage([a], dt, s)
    torch.cuda.synchronize()
    assert torch.equal(a.cons, b.cons)
    for d in range(3):
        assert torch.equal(a.bf[d], b.bf[d])


def test_batched_uneven_blocks(G):
    """Several blocks of different sizes and levels in one launch per kernel,
    each against the oracle on its own."""
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, recon=2, rsolver=1, rk_order=3, fofc=1)
    st = synth.spacetime(3)
    specs = [((8, 8, 8), 0.75, (-3.0, -3.0, -3.0)), ((12, 12, 12), 0.375, (-2.0, 0.5, -1.0)),
             ((16, 16, 16), 0.1875, (0.3, -1.2, 0.4)), ((8, 8, 8), 0.75, (-40.0, -3.0, 5.0))]
    obs = []
    for n, dx, x0 in specs:
        inp = synth.star_block(st, n, 4, (dx,) * 3, x0)
        obs.append(O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A))
    ctx = _ctx(G, p)
    dt = 0.25 * 0.1875
    dbs = [U.to_device(G, ob) for ob in obs]
    ctx.stage(dbs, dt, 0)
    for ob, db in zip(obs, dbs):
        got = U.from_device(db)
        I = interior(ob)
        gm = (got["flags"] & O.F_FOFC) != 0
        mask = np.zeros(ob.cons.shape[1:], np.uint8)
        mask[I] = gm[I]
        ref = ob.copy()
        out = O.stage(p, ref, dt, 0, mask=mask, keep=True)
        U.compare_prims(ref, got, p)
        U.compare_state(ref, got, scales=U.term_scales(p, ob, out, dt, 0))


def _uneven(G, p):
    st = synth.spacetime(3)
    specs = [((8, 8, 8), 0.75, (-3.0, -3.0, -3.0)), ((16, 16, 16), 0.375, (-2.0, 0.5, -1.0)),
             ((12, 12, 12), 0.1875, (0.3, -1.2, 0.4)), ((8, 8, 8), 0.75, (-40.0, -3.0, 5.0))]
    obs = []
    for n, dx, x0 in specs:
        inp = synth.star_block(st, n, 4, (dx,) * 3, x0)
        obs.append(O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A))
    return obs


def test_per_block_launches_and_autotune_reproduce_batched(G):
    """One launch sequence per block, and the autotuner's launch shapes, give
    bit-identical results to the batched launches (launch shape never changes
    the arithmetic of a cell or face)."""
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, recon=2, rsolver=1, rk_order=3, fofc=1)
    obs = _uneven(G, p)
    kw = {k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"}
    dt = 0.25 * 0.1875
    A = [U.to_device(G, ob) for ob in obs]
    B = [U.to_device(G, ob) for ob in obs]
    Cb = [U.to_device(G, ob) for ob in obs]
    T = [U.to_device(G, ob) for ob in obs]
    c1 = G.Context(G.params(**kw))
    c1.step(A, dt)
    c1.step(B, dt, per_block=True)
    c2 = G.Context(G.params(**kw))
    cfg = c2.autotune(T, dt)
    assert all(th in (64, 128, 256) and wv in (1, 2, 4) for th, wv in cfg.values())
    c2.step(Cb, dt)
    torch.cuda.synchronize()
    for a, b, c in zip(A, B, Cb):
        assert torch.equal(a.cons, b.cons) and torch.equal(a.cons, c.cons)
        for d in range(3):
            assert torch.equal(a.bf[d], b.bf[d]) and torch.equal(a.bf[d], c.bf[d])


def test_segment_length_leaves_every_face_unchanged(G):
    """A face's flux does not depend on how its line is cut into sweep
    segments.  Two ragged blocks stepped on their own get one-face segments
    (too few sweeps for longer ones).  In one list with a 104^3 block they get
    the 128^3 bench block's length, at most 16 faces: along x as equal
    segments plus a remainder per line (11 + 11 and 16 + 15 faces here), along
    y and z near-equal.  Every cell and face must agree bit for bit."""
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, recon=2, rsolver=1, rk_order=3, fofc=1)
    st = synth.spacetime(2)
    specs = [((21, 13, 10), 0.75, (-6.0, -4.0, -3.0)), ((30, 9, 17), 0.375, (1.0, -2.0, 0.5))]
    obs = []
    for n, dx, x0 in specs:
        inp = synth.star_block(st, n, 4, (dx,) * 3, x0)
        obs.append(O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A))
    dt = 0.25 * 0.375
    alone = [U.to_device(G, ob) for ob in obs]
    listed = [U.to_device(G, ob) for ob in obs]
    ctx = _ctx(G, p)
    big_in = synth.star_uniform(seed=2, n=104, ng=4)
    big = G.DeviceBlock(big_in.n, big_in.ng, big_in.dx, big_in.adm)
    big.prim.copy_(torch.from_numpy(big_in.prim))
    ctx.init_block(big, [torch.from_numpy(a).cuda() for a in big_in.A])
    ctx.step(alone, dt)
    ctx.step([big] + listed, dt)
    torch.cuda.synchronize()
    for a, b in zip(alone, listed):
        assert torch.equal(a.cons, b.cons) and torch.equal(a.prim, b.prim)
        assert torch.equal(a.flags, b.flags)
        for d in range(3):
            assert torch.equal(a.bf[d], b.bf[d]), d


def test_degenerate_and_ragged_block_shapes(G):
    """Blocks one cell thick along one or more directions, and non-cubic
    blocks, in one batched stage (RK3 substeps 0 and 1), each against the
    oracle; flux sweeps of one face and segment lengths that do not divide n."""
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, recon=2, rsolver=1, rk_order=3, fofc=1)
    st = synth.spacetime(3)
    specs = [((1, 1, 1), 0.75, (-3.0, -3.0, -3.0)), ((1, 6, 2), 0.375, (-2.0, 0.5, -1.0)),
             ((5, 1, 3), 0.375, (0.3, -1.2, 0.4)), ((17, 2, 9), 0.75, (-4.0, -3.0, 1.0)),
             ((33, 3, 1), 0.1875, (-2.5, 0.2, 0.1))]
    obs = []
    for n, dx, x0 in specs:
        inp = synth.star_block(st, n, 4, (dx,) * 3, x0)
        obs.append(O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A))
    ctx = _ctx(G, p)
    dt = 0.25 * 0.1875
    for s in range(2):
        dbs = [U.to_device(G, ob) for ob in obs]
        ctx.stage(dbs, dt, s)
        for ob, db in zip(obs, dbs):
            got = U.from_device(db)
            I = interior(ob)
            gm = (got["flags"] & O.F_FOFC) != 0
            mask = np.zeros(ob.cons.shape[1:], np.uint8)
            mask[I] = gm[I]
            ref = ob.copy()
            out = O.stage(p, ref, dt, s, mask=mask, keep=True)
            U.compare_prims(ref, got, p, f"{ob.n} stage {s}")
            U.compare_state(ref, got, f"{ob.n} stage {s}", scales=U.term_scales(p, ob, out, dt, s))
            ob.cons[...] = got["cons"]
            ob.cons0[...] = got["cons0"]
            for d in range(3):
                ob.bf[d][...] = got["bf"][d]
                ob.bf0[d][...] = got["bf0"][d]


def test_empty_inputs(G):
    """Zero cells is a no-op; an empty block list is an argument error."""
    import torch
    p = O.params(gamma=2.0)
    ctx = _ctx(G, p)
    z = lambda *s: torch.zeros(s, dtype=torch.float64, device="cuda")
    ctx.c2p_cells(z(5, 0), z(3, 0), z(6, 0), z(5, 0), torch.zeros(0, dtype=torch.uint8, device="cuda"))
    ctx.prim2cons(z(5, 0), z(3, 0), z(6, 0), z(5, 0))
    assert ctx.read_stats()["cells"] == 0
    with pytest.raises(RuntimeError):
        ctx.stage([], 0.1, 0)
