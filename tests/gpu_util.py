"""Test-side glue between oracle blocks (numpy) and library blocks (torch, cuda)."""
import numpy as np

import oracle as O
from tests.helpers import interior, rel_err

CONS_TOL = 1e-12   # conserved variables per substep, per cell (floor 1e-10 max)
PRIM_TOL = 1e-10   # primitives


def to_device(G, ob: O.Block, with_cons0=True):
    import torch
    db = G.DeviceBlock(ob.n, ob.ng, ob.dx, ob.adm)
    db.cons.copy_(torch.from_numpy(ob.cons))
    if with_cons0:
        db.cons0.copy_(torch.from_numpy(ob.cons0))
    for d in range(3):
        db.bf[d].copy_(torch.from_numpy(ob.bf[d]))
        db.bf0[d].copy_(torch.from_numpy(ob.bf0[d]))
    return db


def from_device(db) -> dict:
    return dict(cons=db.cons.cpu().numpy(), cons0=db.cons0.cpu().numpy(), prim=db.prim.cpu().numpy(),
                bcc=db.bcc.cpu().numpy(), flags=db.flags.cpu().numpy(),
                bf=[x.cpu().numpy() for x in db.bf], bf0=[x.cpu().numpy() for x in db.bf0])


def region(b, h=3):
    ng = b.ng
    n1, n2, n3 = b.n
    return (slice(ng - h, ng + n3 + h), slice(ng - h, ng + n2 + h), slice(ng - h, ng + n1 + h))


def face_interior(b, d):
    """Faces bounding interior cells (the ones the update writes)."""
    ng = b.ng
    n = b.n
    sl = []
    for ax in (2, 1, 0):
        hi = ng + n[ax] + (1 if ax == d else 0)
        sl.append(slice(ng, hi))
    return tuple(sl)


def rk_w(p, stage):
    if p.rk_order == 2:
        return [(0.0, 1.0, 1.0), (0.5, 0.5, 0.5)][stage]
    return [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25), (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)][stage]


def pgm1(p):
    """The factor that turns an absolute error of eps into one of P: Gamma - 1
    for the ideal gas; for the hybrid EOS the largest index minus 1."""
    if not getattr(p, "eos", 0):
        return p.gamma - 1.0
    return max([p.eos_gamma_th] + [p.eos_gamma[i] for i in range(p.eos_pieces)]) - 1.0


def term_scales(p, ob_in: O.Block, out: dict, dt: float, stage: int):
    """Magnitude of the terms that form each updated value (the scale of its
    rounding error): for U_v, g1|U_v| + g0|U^n_v| + b dt sum_d (|F_d(+)| +
    |F_d(-)|)/dx_d; tau~ = E~ - D~ also carries the scale of D~, the three
    momentum components share the largest scale of the cell, and they also
    carry the pressure's rounding (Gamma-1)(D~ + |tau~|) through the faces.  For a face B~,
    g1|B| + g0|B^n| + b dt sum over its four edges of the term magnitude of the
    edge EMF (the four face EMFs it is built from) / dx, and the field
    magnitude of the two adjacent cells.  Inputs are taken after the con2prim
    floors."""
    g0, g1, be = rk_w(p, stage)
    post = ob_in.copy()
    O.c2p_block(p, post)
    U, Un = np.abs(post.cons), np.abs(ob_in.cons0)
    F = [np.abs(f) for f in out["flux"]]
    T = g1 * U + (g0 * Un if g0 else 0.0)
    T[:, :, :, :] += be * dt * (F[0][:5, :, :, 1:] + F[0][:5, :, :, :-1]) / ob_in.dx[0]
    T[:, :, :, :] += be * dt * (F[1][:5, :, 1:, :] + F[1][:5, :, :-1, :]) / ob_in.dx[1]
    T[:, :, :, :] += be * dt * (F[2][:5, 1:, :, :] + F[2][:5, :-1, :, :]) / ob_in.dx[2]
    T[4] += g1 * U[0] + (g0 * Un[0] if g0 else 0.0)
    T[1:4] = T[1:4].max(axis=0)
    # the pressure recovered from tau~ = E~ - D~ has the absolute precision of
    # (Gamma-1)(D~ + |tau~|), and the momentum update takes its differences
    # over the faces: that rounding enters the momentum scale too
    Pscale = pgm1(p) * (U[0] + U[4])
    T[1:4] += be * dt * 2.0 * Pscale * sum(1.0 / dx for dx in ob_in.dx)
    # term magnitude of every edge EMF: the four face EMFs it averages and
    # corrects (|F_a[5]| on a-faces, |F_b[6]| on b-faces)
    F0, F1, F2 = F
    N3, N2, N1 = post.cons.shape[1:]
    E = [np.zeros((N3 + 1, N2 + 1, N1)), np.zeros((N3 + 1, N2, N1 + 1)), np.zeros((N3, N2 + 1, N1 + 1))]
    E[2][:, :N2, :] += F0[5]
    E[2][:, 1:, :] += F0[5]
    E[2][:, :, :N1] += F1[6]
    E[2][:, :, 1:] += F1[6]
    E[0][:N3, :, :] += F1[5]
    E[0][1:, :, :] += F1[5]
    E[0][:, :N2, :] += F2[6]
    E[0][:, 1:, :] += F2[6]
    E[1][:, :, :N1] += F2[5]
    E[1][:, :, 1:] += F2[5]
    E[1][:N3, :, :] += F0[6]
    E[1][1:, :, :] += F0[6]
    bmag = np.sqrt((post.bcc ** 2).sum(0))
    TB = []
    for d in range(3):
        tb = g1 * np.abs(post.bf[d]) + (g0 * np.abs(ob_in.bf0[d]) if g0 else 0.0)
        if d == 0:
            tb[:, :, :] += be * dt * ((E[2][:, 1:, :] + E[2][:, :-1, :]) / ob_in.dx[1] +
                                      (E[1][1:, :, :] + E[1][:-1, :, :]) / ob_in.dx[2])
            nb = np.zeros_like(tb)
            nb[:, :, :-1] = bmag
            nb[:, :, 1:] = np.maximum(nb[:, :, 1:], bmag)
        elif d == 1:
            tb[:, :, :] += be * dt * ((E[0][1:, :, :] + E[0][:-1, :, :]) / ob_in.dx[2] +
                                      (E[2][:, :, 1:] + E[2][:, :, :-1]) / ob_in.dx[0])
            nb = np.zeros_like(tb)
            nb[:, :-1, :] = bmag
            nb[:, 1:, :] = np.maximum(nb[:, 1:, :], bmag)
        else:
            tb[:, :, :] += be * dt * ((E[1][:, :, 1:] + E[1][:, :, :-1]) / ob_in.dx[0] +
                                      (E[0][:, 1:, :] + E[0][:, :-1, :]) / ob_in.dx[1])
            nb = np.zeros_like(tb)
            nb[:-1, :, :] = bmag
            nb[1:, :, :] = np.maximum(nb[1:, :, :], bmag)
        TB.append(np.maximum(tb, nb))
    return T, TB


def _err(a, b, T, floor_frac=1e-10):
    s = max(np.abs(b).max(), 1e-300) * floor_frac
    return float(np.max(np.abs(a - b) / np.maximum(np.maximum(np.abs(b), T), s)))


def plain_rel_err(a, b, floor_frac=1e-10):
    """The plain error measure max|a - b| / max(|b|, s_f), s_f = 1e-10 max|b|,
    per cell, without the term scales (reported beside the bar, not a bar)."""
    if a.size == 0:
        return 0.0
    s = max(np.abs(b).max(), 1e-300) * floor_frac
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), s)))


# Per-test parity records (printed by tests/conftest.py at the end of the run):
# {nodeid: {"calls", "bar": {field: max}, "plain": {field: max}, "ties", "flips"}}
REPORT = {}


def _record(kind, errs, plain, ties=0, flips=0):
    import os
    node = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    r = REPORT.setdefault(node, {"calls": 0, "bar": {}, "plain": {}, "ties": 0, "flips": 0})
    r["calls"] += 1
    for k, v in errs.items():
        r["bar"][k] = max(r["bar"].get(k, 0.0), v)
    for k, v in plain.items():
        r["plain"][k] = max(r["plain"].get(k, 0.0), v)
    r["ties"] += ties
    r["flips"] += flips


def tie_branch_flux(p, ob_in: O.Block, d: int, face, Fg, rel=1e-13, tol=1e-13, scale=None):
    """The oracle's flux of a tie face taken down the branch the GPU took.
    At a limiter decision (recon_is_tie) both branches are valid for data
    within rounding; the oracle computes the face's flux from its own stage
    primitives with one stencil value moved by `rel` (relative), for every
    value, variable and sign, and the candidate nearest the GPU's flux Fg is
    returned: every value comes from the oracle, the GPU only picks among its
    branches.  The candidate must match Fg within `tol` of the flux scale
    (per component: `scale`), else AssertionError."""
    b = ob_in.copy()
    O.c2p_block(p, b)
    k, j, i = face
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    off = [0, 0, 0]
    off[2 - d] = 1        # (k, j, i) offset of one cell along d
    sc = np.abs(Fg) + 1e-300 if scale is None else np.asarray(scale)
    best, best_e = None, np.inf
    for v in range(7):
        arr = b.prim[v] if v < 5 else b.bcc[t1 if v == 5 else t2]
        for m in range(-3, 3):
            c = (k + m * off[0], j + m * off[1], i + m * off[2])
            x0 = arr[c]
            q = np.array([arr[(k + mm * off[0], j + mm * off[1], i + mm * off[2])] for mm in range(-3, 3)])
            step = rel * max(abs(x0), 1e-3 * (np.abs(q).max() + 1e-300))
            for sgn in (1.0, -1.0):
                arr[c] = x0 + sgn * step
                F = O.face_flux_at(p, b, d, face)
                arr[c] = x0
                e = float(np.max(np.abs(F - Fg) / sc))
                if e < best_e:
                    best, best_e = F, e
    assert best_e <= tol, ("no branch of the oracle reproduces the GPU's tie flux", d, face, best_e)
    return best



def recon_is_tie(p, ob: O.Block, d: int, face, rel=1e-13, jump=1e-11):
    """True when the face's reconstruction by the oracle (from the oracle's
    stage primitives in ob) is at a limiter decision: moving one of the six
    stencil values of one of the seven reconstructed variables by `rel`
    (relative) changes a face state by more than `jump` (relative), where a
    method continuous in its data would move it by ~`rel`.  PPM's branches
    (CW84 flattening, the CS08 extremum test) switch discontinuously, and at
    such a tie both branches are valid outputs for data within rounding."""
    k, j, i = face
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    arrays = [ob.prim[v] for v in range(5)] + [ob.bcc[t1], ob.bcc[t2]]
    for a in arrays:
        if d == 0:
            q = a[k, j, i - 3:i + 3]
        elif d == 1:
            q = a[k, j - 3:j + 3, i]
        else:
            q = a[k - 3:k + 3, j, i]
        q = np.array(q, dtype=np.float64)
        L0, R0 = O.recon_line(p.recon, q)
        sc = np.abs(q).max() + 1e-300
        for m in range(6):
            for sgn in (1.0, -1.0):
                qq = q.copy()
                qq[m] += sgn * rel * max(abs(q[m]), 1e-3 * sc)
                L1, R1 = O.recon_line(p.recon, qq)
                if abs(L1[3] - L0[3]) > jump * sc or abs(R1[3] - R0[3]) > jump * sc:
                    return True
    return False


def compare_state(ob: O.Block, got: dict, what="", cons_tol=CONS_TOL, scales=None):
    """Per-cell relative errors of the conserved variables and face fields,
    each against the magnitude of the terms that formed it (term_scales): the
    bar.  Every interior cell and face is compared.  The plain measure
    max|a - b| / max(|b|, 1e-10 max|b|) of each field is recorded beside it
    (REPORT), not asserted."""
    I = interior(ob)
    errs = {}
    T, TB = scales if scales is not None else (np.zeros_like(ob.cons), [np.zeros_like(x) for x in ob.bf])
    for v in range(5):
        errs[f"cons{v}"] = _err(got["cons"][v][I], ob.cons[v][I], T[v][I])
    for d in range(3):
        F = face_interior(ob, d)
        errs[f"bf{d}"] = _err(got["bf"][d][F], ob.bf[d][F], TB[d][F])
    plain = {}
    for v in range(5):
        plain[f"cons{v}"] = plain_rel_err(got["cons"][v][I], ob.cons[v][I])
    for d in range(3):
        F = face_interior(ob, d)
        plain[f"bf{d}"] = plain_rel_err(got["bf"][d][F], ob.bf[d][F])
    _record("state", errs, plain, ties=getattr(ob, "ties", 0), flips=getattr(ob, "flips", 0))
    bad = {k: e for k, e in errs.items() if not e <= cons_tol}
    assert not bad, f"{what}: {bad}"
    return errs


def compare_prims(ob: O.Block, got: dict, p, what=""):
    R = region(ob)
    errs = {}
    errs["rho"] = rel_err(got["prim"][0][R], ob.prim[0][R])
    W = np.sqrt(1.0 + (ob.prim[1:4][(slice(None),) + R] ** 2).sum(0))
    for v in (1, 2, 3):
        errs[f"w{v}"] = float(np.max(np.abs(got["prim"][v][R] - ob.prim[v][R]) / W))
    # P: absolute error scale (Gamma-1)(D~+tau~)/sqrt(gamma) of the recovery
    g = ob.adm[4:10][(slice(None),) + R]
    det = g[0] * (g[3] * g[5] - g[4] ** 2) - g[1] * (g[1] * g[5] - g[4] * g[2]) + g[2] * (g[1] * g[4] - g[3] * g[2])
    scale = pgm1(p) * np.abs(ob.cons[0][R] + ob.cons[4][R]) / np.sqrt(det)
    dP = np.abs(got["prim"][4][R] - ob.prim[4][R])
    errs["P"] = float(np.max(dP / (1e-10 * np.abs(ob.prim[4][R]) + 1e-12 * scale)))
    plain = {f"prim{v}": plain_rel_err(got["prim"][v][R], ob.prim[v][R]) for v in range(5)}
    _record("prims", {("P/bar" if k == "P" else k): v for k, v in errs.items()}, plain)
    bad = {k: e for k, e in errs.items() if not (e <= PRIM_TOL if k != "P" else e <= 1.0)}
    assert not bad, f"{what}: {bad}"
    return errs


def ho_ustar(p, ob_in: O.Block, dt, stage):
    """U* of every interior cell from the high-order fluxes (no FOFC) of the
    stage input, and the post-floor stage input U (for the DMP bounds)."""
    b = ob_in.copy()
    O.c2p_block(p, b)
    U = b.cons.copy()
    ph = O.params(**{k: getattr(p, k) for k, _ in p._fields_})
    ph.fofc = 0
    bb = ob_in.copy()
    out = O.stage(ph, bb, dt, stage, keep=True)
    F = out["flux"]
    g0, g1, be = [(0.0, 1.0, 1.0), (0.5, 0.5, 0.5)][stage] if p.rk_order == 2 else \
        [(0.0, 1.0, 1.0), (0.75, 0.25, 0.25), (1.0 / 3.0, 2.0 / 3.0, 2.0 / 3.0)][stage]
    div = np.zeros_like(U)
    div -= (F[0][:5, :, :, 1:] - F[0][:5, :, :, :-1]) / b.dx[0]
    div -= (F[1][:5, :, 1:, :] - F[1][:5, :, :-1, :]) / b.dx[1]
    div -= (F[2][:5, 1:, :, :] - F[2][:5, :-1, :, :]) / b.dx[2]
    Us = g1 * U + be * dt * div
    if g0 != 0.0:
        Us += g0 * ob_in.cons0
    return Us, U, b


def flip_is_rounding(p, Us, U, b, cells, rel=1e-12):
    """True for each flipped cell whose FOFC decision changes when U* moves by
    its rounding scale: `rel` relative for D~ and S~_i, 1e-13 (D~ + |tau~|)
    absolute for tau~ (tau = E - D is a difference of O(D) terms), or whose
    DMP test sits within that scale of a bound: a decision taken within
    rounding of its threshold."""
    ok = []
    for (k, j, i) in cells:
        u = Us[:, k, j, i].reshape(5, 1)
        Bd = b.bcc[:, k, j, i].reshape(3, 1)
        g = b.adm[4:10, k, j, i].reshape(6, 1)
        dtau = 1e-13 * (abs(u[0, 0]) + abs(u[4, 0]))
        base = O.c2p_cells(p, u, Bd, g)["flags"][0] & (O.FLOOR_BITS | O.F_FAIL) != 0
        sens = False
        for sgn in (1.0, -1.0):
            for v in range(5):
                uu = u.copy()
                if v == 4:
                    uu[4] += sgn * dtau
                else:
                    uu[v] *= 1.0 + sgn * rel
                f = O.c2p_cells(p, uu, Bd, g)["flags"][0] & (O.FLOOR_BITS | O.F_FAIL) != 0
                sens |= f != base
        if p.dmp_M > 0:
            for v in (0, 4):
                nb = U[v, k - 1:k + 2, j - 1:j + 2, i - 1:i + 2]
                mn, mx = nb.min(), nb.max()
                M = p.dmp_M
                lo = mn / M if mn > 0 else mn * M
                hi = mx * M if mx > 0 else mx / M
                tol = rel * abs(Us[v, k, j, i]) if v == 0 else dtau
                for bound in (lo, hi):
                    sens |= abs(Us[v, k, j, i] - bound) <= tol + rel * abs(bound)
        ok.append(sens)
    return ok
