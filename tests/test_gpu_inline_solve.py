"""The finish kernels' own root solve (c2p_guess 2): with the FP64 polish in
the prep a status-0 cell is a rare fallback, so the finish kernels solve such
cells themselves (the iteration of the refill solve kernel, from the same
bracket) and the solve launch is left out.  The star never falls back; a
block of hostile stress states does (about a fifth of its cells), and its
con2prim must match the oracle's cell by cell (Sec. 3.4 recovery, Sec. 3.3
floors), and its FOFC flags those of the plain con2prim, whose status-0 cells
go through the refill solve kernel."""
import numpy as np
import pytest

import oracle as O
from paper_2409_10384_gb300 import synth
from tests import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10384_gb300 import build, grmhd
    build.build()
    return grmhd


def _kw(p):
    return {k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"}


def _hostile_block(p, n=16, ng=4, seed=41):
    """A 16^3 block (4 ghosts) whose every cell holds a con2prim stress state
    (rho 1e-12..1e-2, T 1e-8..10, W 1..10, gamma_ij = delta + h with |h| <=
    0.2, per cell), with face B~ the curl of a random edge potential (B ~
    1e-4)."""
    N = n + 2 * ng
    prim, _, g = synth.c2p_stress(N ** 3, seed=seed)
    adm = np.zeros((16, N, N, N))
    adm[0] = 1.0
    adm[4:10] = g.reshape(6, N, N, N)
    shape = O.new_block((n,) * 3, ng, (1.0,) * 3, adm)
    rng = np.random.default_rng(seed + 1)
    A = [rng.normal(scale=1e-4, size=shape.edge_shape(c)) for c in range(3)]
    return O.init_block(p, (n,) * 3, ng, (1.0,) * 3, adm, prim.reshape(5, N, N, N), A)


def test_block_con2prim_with_fallbacks_matches_oracle(G):
    p = O.params(gamma=2.0, rho_atm=1e-20, T_atm=1e-14, f_thr=0.0)
    ob = _hostile_block(p)
    ctx = G.Context(G.params(**_kw(p), c2p_guess=2))
    db = U.to_device(G, ob)
    st = ctx.c2p([db], stats=True)
    got = U.from_device(db)
    O.c2p_block(p, ob)
    R = U.region(ob)
    assert np.array_equal(got["flags"][R], ob.flags[R])
    U.compare_prims(ob, got, p, "hostile block, c2p_guess 2")
    n = got["flags"][R].size
    print(f"fallbacks {st['guess_fallbacks']} of {n} cells, FP64 evaluations {st['iters'] / n:.2f} per cell")
    assert st["guess_fallbacks"] > 0.05 * n   # the finish's own solve ran


def test_fofc_flags_with_inline_solve_equal_refill_solve(G):
    p = O.params(gamma=2.0, rho_atm=1e-20, T_atm=1e-14, f_thr=0.0, recon=2, rsolver=1, rk_order=3, fofc=1)
    ob = _hostile_block(p)
    out = {}
    for guess in (0, 2):
        ctx = G.Context(G.params(**_kw(p), c2p_guess=guess))
        db = U.to_device(G, ob)
        ctx.c2p([db])
        ctx.reset_stats()
        ctx.rhs([db], 0.1, 0)
        st = ctx.read_stats()
        out[guess] = (U.from_device(db)["flags"] & O.F_FOFC, st)
    nflag = int((out[0][0] != 0).sum())
    print(f"FOFC cells: plain {out[0][1]['fofc_cells']}, guess 2 {out[2][1]['fofc_cells']}; "
          f"decided in FP32 {out[2][1]['fofc_fp32']}; fallbacks {out[2][1]['guess_fallbacks']}")
    assert np.array_equal(out[0][0], out[2][0]), (nflag, int((out[2][0] != 0).sum()))
    assert out[2][1]["guess_fallbacks"] > 0   # FOFC cells reached the finish's own solve
