"""The allocation-free stage entry point against the regular one.

mhd_stage_noalloc serves callers that cannot let a library allocate device
memory (their GPU memory belongs to their own pool allocator, or they cannot
take the device-wide synchronisation of a cudaFree inside a step): its scratch
is a static device array.  Here it must give the same results as the regular
entry points (mhd_c2p + mhd_rhs + mhd_rk_update through a context) on two
consecutive calls, and reject a block too large for its scratch.  This file is
collected last so that a failure here leaves every other test already run.
"""
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


@pytest.mark.parametrize("eos,recon,dmp", [(0, 2, 0.0), (1, 2, 0.0), (0, 1, 1.1), (0, 4, 1.2)])
def test_noalloc_stage_matches_context_stage_twice(G, eos, recon, dmp):
    """Every RK3 stage in a row (the calls share the static array, which keeps
    the previous call's contents), with WENO-Z, PLM or PPMX and with the DMP
    test of the FOFC estimate on or off."""
    import torch
    from tests.test_gpu_hybrid_eos import HYB_STAR, _star_hyb
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=recon, rsolver=1, rk_order=3, fofc=1,
                 dmp_M=dmp, **(HYB_STAR if eos else {}))
    if eos:
        inp, prim = _star_hyb(p, (104, 52, 52))
    else:
        inp = synth.star_subblock(sub=24, corner=(104, 52, 52))   # over the stellar surface: FOFC fires
        prim = inp.prim
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, prim, inp.A)
    gp = G.params(**{k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"})
    ctx = G.Context(gp)
    a = U.to_device(G, ob)
    b = U.to_device(G, ob)
    dt = 0.25 * inp.dx[0]
    for s in range(3):   # three calls in a row
        ctx.stage([a], dt, s)
        assert G.stage_noalloc(gp, b, dt, s) == 0
        torch.cuda.synchronize()
        ga, gb = U.from_device(a), U.from_device(b)
        for v in range(5):
            ref = ga["cons"][v]
            assert np.max(np.abs(gb["cons"][v] - ref)) <= U.CONS_TOL * np.abs(ref).max(), (s, v)
            ref = ga["prim"][v]
            assert np.max(np.abs(gb["prim"][v] - ref)) <= U.PRIM_TOL * np.abs(ref).max(), (s, v)
        for d in range(3):
            ref = ga["bf"][d]
            assert np.max(np.abs(gb["bf"][d] - ref)) <= U.CONS_TOL * np.abs(ref).max(), (s, d)
        assert np.array_equal(ga["flags"], gb["flags"])


def test_noalloc_rejects_blocks_beyond_its_scratch(G):
    gp = G.params()
    N = 48 + 8
    big = G.DeviceBlock((48, 48, 48), 4, (0.1, 0.1, 0.1), np.zeros((16, N, N, N)))
    assert G.stage_noalloc(gp, big, 0.01, 0) == -6
