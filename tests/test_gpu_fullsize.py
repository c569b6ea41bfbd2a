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
