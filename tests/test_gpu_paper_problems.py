"""The flat-space problems of Sec. 4.1-4.3 run through the library's C-ABI
with its own ghost fill between stages: Balsara shock tubes (Table 1, LLF +
PPM4), magnetic loop advection (WENO-Z + HLLE + FOFC, one period) and the
magnetised cylindrical blast (WENO-Z + HLLE + FOFC, FOFC + DMP).  Exact
solutions are not available here; the checks are what the physics and the
scheme fix (conservation to round-off, div B at round-off after a full period
of CT, first-order convergence of shock-tube density, no con2prim failure in
the blast) and agreement with the CPU oracle run through the same problem.
The limiters and FOFC take threshold decisions, so runs that start a rounding
apart (a mirror image, the oracle) drift apart where a decision flips: the
oracle keeps the blast's mirror symmetry only to ~2% at t = 4 on 100^2, which
is why agreement with the oracle, not symmetry, is checked."""
import numpy as np
import pytest

import oracle as O
from paper_2409_10384_gb300 import synth
from tests import gpu_util as U
from tests.helpers import fill_ghosts, interior

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10384_gb300 import build, grmhd
    build.build()
    return grmhd


def _nbr(modes):
    """Neighbour table of one block over the sides -x, +x, -y, +y, -z, +z: the
    block itself (periodic) or outflow (-1), per axis."""
    return np.array([[-1 if modes[a // 2] == "outflow" else 0 for a in range(6)]], np.int32)


def _device(G, inp, ctx):
    import torch
    db = G.DeviceBlock(inp.n, inp.ng, inp.dx, inp.adm)
    db.prim.copy_(torch.from_numpy(inp.prim))
    ctx.init_block(db, [torch.from_numpy(a).cuda() for a in inp.A])
    return db


def _run(ctx, db, nbr, dt, steps, rk):
    for _ in range(steps):
        for s in range(rk):
            ctx.fill_ghosts([db], nbr)
            ctx.stage([db], dt, s)


def _interior(db, a):
    g = db.ng
    n1, n2, n3 = db.n
    return a[..., g:g + n3, g:g + n2, g:g + n1]


def _divb(db):
    bx, by, bz = (x.cpu().numpy() for x in db.bf)
    g = db.ng
    n1, n2, n3 = db.n
    K, J, I = slice(g, g + n3), slice(g, g + n2), slice(g, g + n1)
    dx, dy, dz = db.dx
    return ((bx[K, J, g + 1:g + n1 + 1] - bx[K, J, g:g + n1]) / dx +
            (by[K, g + 1:g + n2 + 1, I] - by[K, g:g + n2, I]) / dy +
            (bz[g + 1:g + n3 + 1, J, I] - bz[g:g + n3, J, I]) / dz)


TUBE = dict(rho_atm=1e-12, T_atm=1e-12, recon=3, rsolver=0, rk_order=3, fofc=0)   # LLF + PPM4, no FOFC


def _tube(G, test, n, t_end=0.5, cfl=0.25):
    import torch
    gam = synth.BALSARA[test][0]
    ctx = G.Context(G.params(gamma=gam, **TUBE))
    ctx.ledger(True)
    db = _device(G, synth.balsara_tube(test, n, ny=1), ctx)
    dt = cfl / n
    steps = int(round(t_end / dt))
    m0 = ctx.block_mass([db])[0]
    _run(ctx, db, _nbr(("outflow", "periodic", "periodic")), dt, steps, 3)
    torch.cuda.synchronize()
    return ctx, db, m0


@pytest.mark.parametrize("test", [1, 2, 3, 4, 5])
def test_balsara_tubes(G, test):
    """Table 1, 400 cells, LLF + PPM4, RK3, to t = 0.5: no con2prim failure and
    the baryon mass balanced by the boundary fluxes to round-off (fast waves
    reach the outflow sides by t = 0.5, so mass and energy do change)."""
    ctx, db, m0 = _tube(G, test, 400)
    c = _interior(db, db.cons).cpu().numpy()
    assert np.all(np.isfinite(c))
    assert ctx.read_stats()["fails"] == 0
    m1 = ctx.block_mass([db])[0]
    bal = ctx.ledger_read(1)[0]
    assert abs(m1 - m0 - bal) <= 1e-13 * m0


def test_balsara1_first_order_convergence(G):
    """L2 error of rho at t = 0.5 against a 1600-cell run: the error falls
    with resolution at about first order (the solution is shock-dominated;
    Sec. 4.1 reports approximately first order)."""
    _, dref, _ = _tube(G, 1, 1600)
    g = dref.ng
    rr = dref.prim[0].cpu().numpy()[g, g, g:g + 1600]
    errs = []
    for n in (100, 200, 400, 800):
        _, d, _ = _tube(G, 1, n)
        r = d.prim[0].cpu().numpy()[g, g, g:g + n]
        coarse = rr.reshape(n, 1600 // n).mean(axis=1)
        errs.append(float(np.sqrt(np.mean((r - coarse) ** 2))))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    print("balsara 1 L2(rho)", errs, "rates", rates)
    assert np.all(np.diff(errs) < 0), errs
    assert 0.5 < rates.mean() < 1.6, rates


def test_balsara1_matches_oracle(G):
    """Tube 1 on 100 cells to t = 0.5 through the library and through the
    oracle (the harness's ghost fill): the densities agree."""
    n = 100
    _, d, _ = _tube(G, 1, n)
    g = d.ng
    rg = d.prim[0].cpu().numpy()[g, g, g:g + n]
    p = O.params(gamma=synth.BALSARA[1][0], **TUBE)
    inp = synth.balsara_tube(1, n, ny=1)
    b = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    dt = 0.25 / n
    for _ in range(int(round(0.5 / dt))):
        for s in range(3):
            fill_ghosts(b, ("outflow", "periodic", "periodic"))
            O.stage(p, b, dt, s)
    ro = b.prim[0][g, g, g:g + n]
    diff = float(np.max(np.abs(rg - ro)) / np.abs(ro).max())
    print("balsara 1, 100 cells: max |rho_gpu - rho_oracle| / max rho =", diff)
    assert diff < 1e-6


def test_loop_advection_one_period(G):
    """128^2 periodic loop, WENO-Z + HLLE + FOFC, RK3, CFL 0.25, t = 2.4: div B
    stays at round-off relative to max |B| (Sec. 4.3 reports 7e-14 -> 3e-12),
    mass is conserved to round-off, and the loop returns to its place."""
    import torch
    n = 128
    ctx = G.Context(G.params(gamma=5.0 / 3.0, rho_atm=1e-12, T_atm=1e-12, recon=2, rsolver=1, rk_order=3, fofc=1))
    db = _device(G, synth.field_loop(n), ctx)
    steps = int(round(2.4 / (0.25 / n)))
    dt = 2.4 / steps
    b0 = db.bf[0].cpu().numpy().copy()
    bmax = np.abs(b0).max()
    d0 = np.abs(_divb(db)).max() / bmax
    m0 = float(_interior(db, db.cons[0]).sum().item())
    _run(ctx, db, _nbr(("periodic",) * 3), dt, steps, 3)
    torch.cuda.synchronize()
    d1 = np.abs(_divb(db)).max() / bmax
    assert d0 < 1e-13 and d1 < 1e-11, (d0, d1)
    m1 = float(_interior(db, db.cons[0]).sum().item())
    assert abs(m1 - m0) <= 1e-13 * m0
    b1 = db.bf[0].cpu().numpy()
    g = db.ng
    a0, a1 = b0[g, g:g + n, g:g + n + 1].ravel(), b1[g, g:g + n, g:g + n + 1].ravel()
    corr = float(np.dot(a0, a1) / np.sqrt(np.dot(a0, a0) * np.dot(a1, a1)))
    assert corr > 0.9, corr
    assert ctx.read_stats()["fails"] == 0


def test_loop_advection_matches_oracle_over_steps(G):
    """32^2 loop, two RK3 steps with ghost fills between stages on both sides
    (the library's fill and the harness's numpy fill): the states agree to
    1e-11 of their magnitude."""
    n = 32
    p = O.params(gamma=5.0 / 3.0, rho_atm=1e-12, T_atm=1e-12, recon=2, rsolver=1, rk_order=3, fofc=1)
    inp = synth.field_loop(n)
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    kw = {k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"}
    ctx = G.Context(G.params(**kw))
    db = U.to_device(G, ob)
    dt = 0.25 / n
    nbr = _nbr(("periodic",) * 3)
    for _ in range(2):
        for s in range(3):
            fill_ghosts(ob)
            O.stage(p, ob, dt, s)
            ctx.fill_ghosts([db], nbr)
            ctx.stage([db], dt, s)
    got = U.from_device(db)
    I = interior(ob)
    for v in range(5):
        sc = np.abs(ob.cons[v][I]).max() + np.abs(ob.cons[0][I]).max()
        assert np.max(np.abs(got["cons"][v][I] - ob.cons[v][I])) <= 1e-11 * sc, v
    # every face-field component against the field's magnitude: the z
    # component of this planar loop is zero in exact arithmetic, and the
    # rounding of its constrained-transport update (EMFs with v^z B terms
    # that cancel) leaves ~1e-18 of |B~|
    sc = max(np.abs(ob.bf[d]).max() for d in range(3))
    for d in range(3):
        assert np.max(np.abs(got["bf"][d][U.face_interior(ob, d)] - ob.bf[d][U.face_interior(ob, d)])) <= 1e-11 * sc


@pytest.mark.parametrize("dmp", [0.0, 1.1])
def test_cylindrical_blast(G, dmp):
    """B_x = 0.1, 100^2 cells on [-6, 6]^2, Gamma = 4/3, WENO-Z + HLLE + FOFC
    (+ DMP, M = 1.1), RK3, CFL 0.1, rho_atm = 1e-10, T_atm = 1e-8, f_thr = 1, to
    t = 4: no con2prim failure, FOFC engaged, baryon mass balanced (floors
    included) to round-off; without DMP, the density against the oracle run
    through the same problem."""
    import torch
    n = 100
    kw = dict(gamma=4.0 / 3.0, rho_atm=1e-10, T_atm=1e-8, f_thr=1.0, recon=2, rsolver=1, rk_order=3, fofc=1,
              dmp_M=dmp)
    ctx = G.Context(G.params(**kw))
    ctx.ledger(True)
    db = _device(G, synth.cylindrical_blast(0.1, n), ctx)
    dt = 0.1 * 12.0 / n
    steps = int(round(4.0 / dt))
    m0 = ctx.block_mass([db])[0]
    ctx.reset_stats()
    _run(ctx, db, _nbr(("outflow", "outflow", "periodic")), dt, steps, 3)
    torch.cuda.synchronize()
    st = ctx.read_stats()
    c = _interior(db, db.cons).cpu().numpy()
    assert np.all(np.isfinite(c))
    assert st["fails"] == 0 and st["fofc_cells"] > 0, st
    m1 = ctx.block_mass([db])[0]
    bal = ctx.ledger_read(1)[0]
    assert abs(m1 - m0 - bal) <= 1e-12 * m0
    if dmp == 0.0:
        p = O.params(**kw)
        inp = synth.cylindrical_blast(0.1, n)
        b = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
        for _ in range(steps):
            for s in range(3):
                fill_ghosts(b, ("outflow", "outflow", "periodic"))
                O.stage(p, b, dt, s)
        g = b.ng
        rg = _interior(db, db.prim[0]).cpu().numpy()[0]
        ro = b.prim[0][g, g:g + n, g:g + n]
        l1 = float(np.abs(rg - ro).sum() / np.abs(ro).sum())
        print("blast B_x = 0.1, t = 4: L1 |rho_gpu - rho_oracle| / L1 rho =", l1,
              "max rel", float(np.max(np.abs(rg - ro) / ro)))
        assert l1 < 1e-3
