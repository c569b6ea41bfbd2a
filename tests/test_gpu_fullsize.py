"""Full-size parity: the 128^3 star workload of bench.py (WENO-Z + HLLE + FOFC
+ CT, RK3), in bench.py's launch configuration (launch shapes picked by the
autotuner, and the con2prim root search bench.py times), every substep of one
RK3 step against the FP64 oracle on every cell and face.  Same bars and flag handling as tests/test_gpu_parity.py."""
import numpy as np
import pytest

import bench
import oracle as O
from paper_2409_10384_gb300 import synth
from tests import gpu_util as U
from tests.helpers import interior

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10384_gb300 import build, grmhd
    build.build()
    return grmhd


def test_star128_rk3_step_matches_oracle(G):
    p = O.params(**bench.PARAMS)
    inp = synth.star_uniform(seed=2, n=bench.N_INT, ng=bench.NG)
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    ctx = G.Context(G.params(**bench.PARAMS, c2p_guess=bench.C2P_GUESS))
    dt = bench.CFL * inp.dx[0]
    ctx.autotune([U.to_device(G, ob)], dt)   # on a copy: the launch shapes bench.py times
    total_flips = 0
    for s in range(3):
        db = U.to_device(G, ob)
        ctx.stage([db], dt, s)
        got = U.from_device(db)
        I = interior(ob)
        gm = (got["flags"] & O.F_FOFC) != 0
        mask = np.zeros(ob.cons.shape[1:], np.uint8)
        mask[I] = gm[I]
        own = ob.copy()
        O.stage(p, own, dt, s)
        diff = np.argwhere(gm[I] != ((own.flags & O.F_FOFC) != 0)[I])
        if len(diff):
            Us, Upost, bpost = U.ho_ustar(p, ob, dt, s)
            cells = [tuple(int(x) + ob.ng for x in c) for c in diff]
            ok = U.flip_is_rounding(p, Us, Upost, bpost, cells)
            bad = [c for c, o in zip(cells, ok) if not o]
            assert not bad, (f"stage {s}: {len(bad)} of {len(cells)} FOFC flips away from a threshold", bad[:10],
                             [(bool(gm[c]), Us[:, c[0], c[1], c[2]].tolist()) for c in bad[:3]])
            total_flips += len(cells)
        ref = ob.copy()
        out = O.stage(p, ref, dt, s, mask=mask, keep=True)
        U.compare_prims(ref, got, p, f"stage {s}")
        U.compare_state(ref, got, f"stage {s}", scales=U.term_scales(p, ob, out, dt, s))
        ob.cons[...] = got["cons"]
        ob.cons0[...] = got["cons0"]
        for d in range(3):
            ob.bf[d][...] = got["bf"][d]
            ob.bf0[d][...] = got["bf0"][d]
    assert total_flips <= 1e-3 * bench.N_INT ** 3


def _stage_block_vs_oracle(p, ob, got, dt, s):
    """One block's GPU stage result against the oracle run from the same
    input, FOFC flags injected after the flip check (as above)."""
    I = interior(ob)
    gm = (got["flags"] & O.F_FOFC) != 0
    own = ob.copy()
    O.stage(p, own, dt, s)
    diff = np.argwhere(gm[I] != ((own.flags & O.F_FOFC) != 0)[I])
    if len(diff):
        Us, Upost, bpost = U.ho_ustar(p, ob, dt, s)
        cells = [tuple(int(x) + ob.ng for x in c) for c in diff]
        assert all(U.flip_is_rounding(p, Us, Upost, bpost, cells))
    mask = np.zeros(ob.cons.shape[1:], np.uint8)
    mask[I] = gm[I]
    ref = ob.copy()
    out = O.stage(p, ref, dt, s, mask=mask, keep=True)
    U.compare_prims(ref, got, p)
    U.compare_state(ref, got, scales=U.term_scales(p, ob, out, dt, s))


def _sampled_list_parity(G, specs, st, guess, pick):
    """Every block of a list through one batched stage; the picked blocks
    against the oracle one by one."""
    import torch
    p = O.params(**bench.PARAMS)
    ctx = G.Context(G.params(**bench.PARAMS, c2p_guess=0))
    if guess == 1:
        bench.train_guess(ctx, samples=1 << 18, epochs=10)
        ctx.set_params(G.params(**bench.PARAMS, c2p_guess=1))
    dbs, obs = [], {}
    for bi, sp in enumerate(specs):
        inp = synth.star_block(st, (sp.n,) * 3, bench.NG, (sp.dx,) * 3, sp.x0)
        if bi in pick:
            ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
            obs[bi] = ob
            dbs.append(U.to_device(G, ob))
        else:
            db = G.DeviceBlock(inp.n, inp.ng, inp.dx, inp.adm)
            db.prim.copy_(torch.from_numpy(inp.prim))
            ctx.init_block(db, [torch.from_numpy(a).cuda() for a in inp.A])
            dbs.append(db)
    dt = bench.CFL * min(sp.dx for sp in specs)
    ctx.autotune(dbs, dt)
    ctx.stage(dbs, dt, 0)
    torch.cuda.synchronize()
    assert ctx.read_stats()["fails"] == 0
    for bi, ob in obs.items():
        _stage_block_vs_oracle(p, ob, U.from_device(dbs[bi]), dt, 0)


def _picks(specs, centres):
    """A finest-level block nearest a star centre, a block at the stellar
    surface and a coarse atmosphere block."""
    d = [min(np.linalg.norm(np.array(sp.x0) + 0.5 * sp.n * sp.dx - np.array(c)) for c in centres) for sp in specs]
    fine = min(range(len(specs)), key=lambda b: (-specs[b].level, d[b]))
    surf = min(range(len(specs)), key=lambda b: abs(d[b] - 36.0))
    atm = max(range(len(specs)), key=lambda b: d[b])
    return {fine, surf, atm}


def test_binary_block_list_sampled(G):
    """The 1968-block binary list of bench.py (32^3 blocks on 6 levels, two
    stars moving in y) with the learned-guess con2prim: one batched stage,
    three sampled blocks against the oracle."""
    specs, centres = synth.bns_blocks(seed=5)
    st = synth.spacetime(5, centres=centres, vy=(-0.15, 0.15))
    _sampled_list_parity(G, specs, st, 1, _picks(specs, centres))


def test_amr512_block_list_sampled(G):
    """The 512-block AMR list of bench.py (16^3/32^3/64^3): one batched
    stage, three sampled blocks (of each size where possible) against the
    oracle."""
    specs = synth.amr_blocks(seed=3)
    st = synth.spacetime(3)
    pick = set()
    for n in (16, 32, 64):
        pick.add(next(b for b, sp in enumerate(specs) if sp.n == n))
    _sampled_list_parity(G, specs, st, 0, pick)
