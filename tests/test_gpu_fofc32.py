"""The FOFC estimate's flags from FP32 values (Sec. 3.3: the estimate only asks
whether con2prim of U* fails or a floor fires).  With the ideal gas the library
decides most cells from FP32 interval enclosures of the KRP variables, of the
master function around the FP32 root and of v^2, rho and eps_raw, and leaves
the rest to the FP64 recovery.
Every decision must equal the FP64 recovery's: mhd_c2p_cells with prim = NULL
(flags only, the same decision) is compared cell by cell with the full
con2prim of the same cells, on stress states where floors fire and on states
placed at relative distances 1e-1 .. 1e-9 from each threshold."""
import numpy as np
import pytest

import oracle as O
from paper_2409_10384_gb300 import synth

pytestmark = pytest.mark.gpu

FLAG_BITS = 1 | 2 | 4 | 8 | 16 | 32 | 64   # F_FAIL and every floor bit


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10384_gb300 import build, grmhd
    build.build()
    return grmhd


def _both(G, p, prim, Bd, g, guess):
    """flags-only and full con2prim of the same cells: (flag_only, flag_full,
    stats of the flags-only call, cons after the flags-only call, cons)."""
    import torch
    kw = {k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"}
    kw["c2p_guess"] = guess
    ctx = G.Context(G.params(**kw))
    cons = O.prim2cons(p, prim, Bd, g)
    n = cons.shape[1]
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dB, dg = t(Bd), t(g)
    dc = t(cons)
    fo = torch.zeros(n, dtype=torch.uint8, device="cuda")
    it = torch.zeros(n, dtype=torch.int32, device="cuda")
    st = ctx.c2p_cells(dc, dB, dg, None, fo, it, stats=True)
    c_after = dc.cpu().numpy()
    dc2 = t(cons)
    dp = torch.zeros((5, n), dtype=torch.float64, device="cuda")
    ff = torch.zeros(n, dtype=torch.uint8, device="cuda")
    ctx.c2p_cells(dc2, dB, dg, dp, ff)
    full = (ff.cpu().numpy() & FLAG_BITS) != 0
    return fo.cpu().numpy(), full, st, c_after, cons, it.cpu().numpy()


@pytest.mark.parametrize("guess", [0, 2])
def test_flags_only_equal_full_recovery_on_stress_cells(G, guess):
    """1M stress cells (rho 1e-12..1e-2, T 1e-8..10, W 1..10, sigma 1e-4..1e2)
    with the floors inside those ranges: rho_thr = 1e-8, T_atm = 1e-4 and W_max
    = 5, so every floor fires on a share of the cells."""
    p = O.params(gamma=2.0, rho_atm=1e-8, T_atm=1e-4, f_thr=1.0, W_max=5.0)
    n = 1 << 20
    prim, Bd, g = synth.c2p_stress(n, seed=11)
    fo, full, st, c_after, cons, it = _both(G, p, prim, Bd, g, guess)
    assert set(np.unique(fo)) <= {0, 1}
    bad = np.nonzero((fo != 0) != full)[0]
    assert bad.size == 0, (bad.size, bad[:10])
    assert np.array_equal(c_after, cons)   # flags only: cons untouched
    assert st["fofc_cells"] == int(full.sum())
    assert 0.1 * n < full.sum() < 0.9 * n   # the floors fire on part of the cells
    print(f"guess {guess}: flagged {full.mean():.3f}, decided in FP32 {st['fofc_fp32'] / n:.4f}, "
          f"FP64 evaluations {st['iters'] / n:.3f} per cell")
    # the cells a floor on the conserved state flags (rho W < rho_thr for about
    # 40% of them) take no root at all and are not counted in fofc_fp32; of
    # the rest, the hot and fast ones (W up to 10) are beyond the FP32 bounds
    assert st["fofc_fp32"] >= 0.05 * n
    assert st["iters"] == int(it.sum())


def test_flags_only_on_star_states(G):
    """Cells of the 128^3 star's blocks with the bench's floors: the core and
    inner layers (no floor: every cell decided in FP32, none flagged) and the
    surface and atmosphere (a mixture), against the full recovery."""
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, W_max=1e3)
    kw = {k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"}
    ctx = G.Context(G.params(**kw, c2p_guess=2))
    st = synth.spacetime(2)

    def cells(x0, n=32, dx=0.75):
        inp = synth.star_block(st, (n,) * 3, 4, (dx,) * 3, x0)
        db = G.DeviceBlock(inp.n, inp.ng, inp.dx, inp.adm)
        db.prim.copy_(torch.from_numpy(inp.prim))
        ctx.init_block(db, [torch.from_numpy(a).cuda() for a in inp.A])
        return (db.cons.reshape(5, -1).contiguous(), db.bcc.reshape(3, -1).contiguous(),
                db.adm.reshape(16, -1)[4:10].contiguous())

    for x0, inner in (((-12.0, -12.0, -12.0), True), ((0.0, -12.0, -12.0), False), ((8.0, 8.0, 8.0), False)):
        c, b, g = cells(x0)
        n = c.shape[1]
        fo = torch.zeros(n, dtype=torch.uint8, device="cuda")
        s1 = ctx.c2p_cells(c.clone(), b, g, None, fo, stats=True)
        ff = torch.zeros(n, dtype=torch.uint8, device="cuda")
        ctx.c2p_cells(c.clone(), b, g, torch.zeros_like(c), ff)
        full = (ff.cpu().numpy() & FLAG_BITS) != 0
        assert np.array_equal(fo.cpu().numpy() != 0, full), x0
        print(f"star block at {x0}: {n} cells, flagged {full.mean():.3f}, decided in FP32 "
              f"{s1['fofc_fp32'] / n:.4f}, FP64 evaluations {s1['iters'] / n:.3f} per cell")
        if inner:
            assert not full.any() and s1["fofc_fp32"] == n and s1["iters"] == 0


def _near(n, seed, which, rel):
    """Stress states moved to a relative distance rel (signs mixed) from one
    threshold: 'rho' rho = rho_thr (1 + d), 'T' p = rho T_atm (1 + d), 'W' W =
    W_max (1 + d), with p from O.params(gamma=2, rho_atm=1e-8, T_atm=1e-4,
    f_thr=1, W_max=5)."""
    prim, Bd, g = synth.c2p_stress(n, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 100))
    d = rel * np.where(rng.uniform(size=n) < 0.5, -1.0, 1.0)
    if which == "rho":
        rho = 1e-8 * (1.0 + d)
        prim[4] = prim[4] / prim[0] * rho
        prim[1:4] *= 0.5    # below the velocity cap
        prim[0] = rho
    elif which == "T":
        prim[0] = np.maximum(prim[0], 1e-6)
        prim[4] = prim[0] * 1e-4 * (1.0 + d)
        prim[1:4] *= 0.5
    else:
        u = prim[1:4]
        # scale u^i so that W = W_max (1 + d) in the cell's own metric
        ul = np.stack([g[0] * u[0] + g[1] * u[1] + g[2] * u[2], g[1] * u[0] + g[3] * u[1] + g[4] * u[2],
                       g[2] * u[0] + g[4] * u[1] + g[5] * u[2]])
        uu = (u * ul).sum(0)
        Wt = 5.0 * (1.0 + d)
        prim[1:4] = u * np.sqrt((Wt * Wt - 1.0) / uu)
        prim[0] = np.maximum(prim[0], 1e-6)
        prim[4] = np.maximum(prim[4], prim[0] * 1e-2)
    return prim, Bd, g


@pytest.mark.parametrize("which", ["rho", "T", "W"])
def test_flags_only_equal_full_recovery_near_thresholds(G, which):
    p = O.params(gamma=2.0, rho_atm=1e-8, T_atm=1e-4, f_thr=1.0, W_max=5.0)
    n = 1 << 16
    decided = []
    for k in range(1, 10):
        prim, Bd, g = _near(n, 20 + k, which, 10.0 ** -k)
        fo, full, st, _, _, _ = _both(G, p, prim, Bd, g, 2)
        bad = np.nonzero((fo != 0) != full)[0]
        assert bad.size == 0, (which, k, bad.size, bad[:10])
        decided.append(st["fofc_fp32"] / n)
    print(which, "decided in FP32 at 1e-1 .. 1e-9:", " ".join(f"{x:.3f}" for x in decided))
    assert decided[0] > 0.2            # far from the threshold a share is decided
    assert decided[-1] < decided[0]    # near it they go to the FP64 recovery


def test_enclosures_contain_their_values(G):
    """The FP32 interval operations of the decision (ival.cuh): the interval
    of a double, the widened hardware reciprocal and reciprocal square root,
    products, squares, sums and differences contain the FP64 value they
    enclose, over log-uniform values of both signs across the FP32 range,
    powers of two and their neighbours, and values outside the FP32 range
    (whose enclosure is empty and decides nothing)."""
    import torch
    rng = np.random.default_rng(31)
    n = 1 << 20
    x = np.concatenate([10.0 ** rng.uniform(-37.5, 37.5, n) * rng.choice([-1.0, 1.0], n),
                        2.0 ** np.arange(-125, 127, dtype=np.float64),
                        np.nextafter(2.0 ** np.arange(-125, 127, dtype=np.float64), 0.0),
                        np.nextafter(2.0 ** np.arange(-125, 127, dtype=np.float64), np.inf),
                        np.array([0.0, -0.0, 1e-300, -1e-300, 1e300, 1.0 + 2.0 ** -30, 1.0 - 2.0 ** -30])])
    miss = G.check_enclosures(torch.from_numpy(np.ascontiguousarray(x)).cuda()).cpu().numpy()
    bad = np.nonzero(miss)[0]
    assert bad.size == 0, (bad.size, x[bad[:5]], miss[bad[:5]])
