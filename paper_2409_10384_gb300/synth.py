"""Seeded synthetic inputs shaped like the paper's workloads.

This module evaluates analytic fields (density, pressure, velocity primitive,
ADM metric, edge vector potential) at cell centres and cell edges.  It holds
none of the method's arithmetic: no conserved variables, no fluxes, no
con2prim.  Both the CUDA path and the CPU oracle consume what it returns, each
turning it into conserved variables and face fields with its own code.

Layout: SoA float64, ``[var][k][j][i]`` with i fastest, ghost-inclusive,
``N_d = n_d + 2 ng``.  Cell (i) centre: ``x0 + (i - ng + 1/2) dx``.  Edge
arrays follow the library's EMF layout: A_x at (i, j-1/2, k-1/2) shape
``[N3+1][N2+1][N1]``, A_y at (i-1/2, j, k-1/2) ``[N3+1][N2][N1+1]``, A_z at
(i-1/2, j-1/2, k) ``[N3][N2+1][N1+1]``.  ADM: alpha, beta^1..3,
gamma_11,12,13,22,23,33, K_11,12,13,22,23,33 (16 fields).

Workloads (the paper's test sections set the shapes and values):
  * periodic flat block (Sec. 4.1-4.3 flat-space limit): 32^3, Gamma 5/3;
  * Gaussian "star" in a conformally flat metric (polytrope K=100, Gamma=2,
    rho_c = 1.28e-3, Sec. 4.4), poloidal field from A_phi (Eq. 21 shape);
  * con2prim stress cells with log-uniform rho, T, W, sigma (Sec. 3.3-3.4 ranges);
  * AMR-shaped block lists (Sec. 5: 6 levels, 16^3/32^3/64^3 blocks).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class BlockInputs:
    n: tuple      # interior (n1, n2, n3)
    ng: int
    dx: tuple     # (dx, dy, dz)
    x0: tuple     # lower corner of the interior
    prim: np.ndarray   # [5][N3][N2][N1]: rho, w^1..3 (= W v^i), P
    A: tuple      # edge vector potential (A_x, A_y, A_z)
    adm: np.ndarray    # [16][N3][N2][N1]

    @property
    def N(self):
        return tuple(x + 2 * self.ng for x in self.n)


def _axes(n, ng, dx, x0, stag, wrap=None):
    """Coordinates along one axis: stag=0 cell centres (N), 1 faces (N+1).
    With ``wrap`` (period in cells) indices are folded into the interior so
    that periodic images are bitwise identical."""
    N = n + 2 * ng
    idx = np.arange(N + stag) - ng
    if wrap is not None:
        idx = np.mod(idx, wrap)
    return x0 + (idx + (0.0 if stag else 0.5)) * dx


def _grid(n, ng, dx, x0, stag=(0, 0, 0), wrap=False):
    xs = [_axes(n[d], ng, dx[d], x0[d], stag[d], n[d] if wrap else None) for d in range(3)]
    z, y, x = np.meshgrid(xs[2], xs[1], xs[0], indexing="ij")
    return x, y, z


# ---------------------------------------------------------------------------
# Periodic flat-space block (the 32^3 + 4-ghost parity case).

def periodic_flat(seed: int = 1, n: int = 32, ng: int = 4) -> BlockInputs:
    """rho = 1 + 0.1 sum_3 sin(k.x + phi), P = 0.1, |v| <= 0.3 from 3 smooth
    modes, B = curl A with A from 3 modes scaled to |B| ~ 0.1; flat metric;
    unit periodic box.  All fields periodic with integer wavenumbers."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nn = (n, n, n)
    dx = (1.0 / n,) * 3
    x0 = (0.0, 0.0, 0.0)
    N = n + 2 * ng

    def modes(m):
        ks = rng.integers(1, 4, size=(m, 3)) * rng.choice([-1, 1], size=(m, 3))
        ph = rng.uniform(0, 2 * np.pi, size=m)
        return ks.astype(np.float64) * 2 * np.pi, ph

    x, y, z = _grid(nn, ng, dx, x0, wrap=True)
    kr, pr = modes(3)
    rho = 1.0 + 0.1 * sum(np.sin(kr[m, 0] * x + kr[m, 1] * y + kr[m, 2] * z + pr[m]) for m in range(3))
    P = np.full_like(rho, 0.1)
    kv, pv = modes(3)
    cv = rng.normal(size=(3, 3))
    cv /= np.linalg.norm(cv, axis=1, keepdims=True)
    vel = np.zeros((3,) + rho.shape)
    for m in range(3):
        s = np.sin(kv[m, 0] * x + kv[m, 1] * y + kv[m, 2] * z + pv[m])
        for c in range(3):
            vel[c] += cv[m, c] * s
    vmag = np.sqrt((vel ** 2).sum(0)).max()
    vel *= 0.3 / vmag
    # the velocity primitive w^i = W v^i of a field with |v| <= 0.3 (flat metric)
    W = 1.0 / np.sqrt(1.0 - (vel ** 2).sum(0))
    prim = np.stack([rho, W * vel[0], W * vel[1], W * vel[2], P])
    # vector potential: 3 modes, amplitude so that |curl A| ~ 0.1
    ka, pa = modes(3)
    ca = rng.normal(size=(3, 3))
    A = []
    stags = [(0, 1, 1), (1, 0, 1), (1, 1, 0)]
    for c in range(3):
        ex, ey, ez = _grid(nn, ng, dx, x0, stag=stags[c], wrap=True)
        a = np.zeros_like(ex)
        for m in range(3):
            amp = 0.1 / (np.linalg.norm(ka[m]) * np.sqrt(3.0))
            a += amp * ca[m, c] * np.cos(ka[m, 0] * ex + ka[m, 1] * ey + ka[m, 2] * ez + pa[m])
        A.append(np.ascontiguousarray(a))
    adm = np.zeros((16, N, N, N))
    adm[0] = 1.0
    adm[4] = adm[7] = adm[9] = 1.0
    return BlockInputs(nn, ng, dx, x0, np.ascontiguousarray(prim), tuple(A), adm)


# ---------------------------------------------------------------------------
# Star in a conformally flat metric (the 128^3 dynamical-metric workload and
# the AMR block lists).

STAR = dict(M=1.4, rs=0.5, rho_c=1.28e-3, width=8.0, rho_floor=1e-12, K=100.0, Ab=1e-3, cut=0.04)


@dataclass
class Spacetime:
    """Seeded smooth shift and extrinsic curvature shared by every block of a
    workload, plus the star centres and their coordinate velocities."""
    kb: np.ndarray   # shift modes
    pb: np.ndarray
    cb: np.ndarray
    kk: np.ndarray   # K_ij modes
    pk: np.ndarray
    ck: np.ndarray
    centres: tuple
    vy: tuple
    with_K: bool


def spacetime(seed: int, centres=((0.0, 0.0, 0.0),), vy=(0.0,), with_K=True, L=96.0) -> Spacetime:
    rng = np.random.Generator(np.random.PCG64(seed))
    kb = rng.integers(1, 4, size=(3, 3)) * rng.choice([-1, 1], size=(3, 3)) * (2 * np.pi / L)
    pb = rng.uniform(0, 2 * np.pi, size=3)
    cb = rng.uniform(-1, 1, size=(3, 3))
    kk = rng.integers(1, 4, size=(3, 3)) * rng.choice([-1, 1], size=(3, 3)) * (2 * np.pi / L)
    pk = rng.uniform(0, 2 * np.pi, size=3)
    ck = rng.uniform(-1, 1, size=(3, 6))
    return Spacetime(kb, pb, cb, kk, pk, ck, tuple(centres), tuple(vy), with_K)


def _star_fields(st: Spacetime, x, y, z):
    """Conformal factor psi = 1 + sum M/(2 sqrt(r^2 + rs^2)); rho Gaussian of
    width 8 over a 1e-12 floor (max over stars); P = K rho^2; per-star v^y."""
    S = STAR
    psi = np.ones_like(x)
    rho = np.full_like(x, S["rho_floor"])
    vy = np.zeros_like(x)
    for (cx, cy, cz), v in zip(st.centres, st.vy):
        r2 = (x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2
        psi += S["M"] / (2.0 * np.sqrt(r2 + S["rs"] ** 2))
        r_ = S["rho_c"] * np.exp(-r2 / S["width"] ** 2)
        vy = np.where(r_ > rho, v, vy)
        rho = np.maximum(rho, r_)
    vy = np.where(rho > 1e3 * S["rho_floor"], vy, 0.0)
    P = S["K"] * rho * rho
    return psi, rho, P, vy


def _pressure_only(st: Spacetime, x, y, z):
    _, _, P, _ = _star_fields(st, x, y, z)
    return P


def star_block(st: Spacetime, n, ng: int, dx, x0) -> BlockInputs:
    """Evaluate the star workload on one block (interior n, lower corner x0)."""
    n = tuple(int(v) for v in n)
    dx = tuple(float(v) for v in dx)
    x0 = tuple(float(v) for v in x0)
    x, y, z = _grid(n, ng, dx, x0)
    psi, rho, P, vy = _star_fields(st, x, y, z)
    adm = np.zeros((16,) + x.shape)
    psi4 = psi ** 4
    adm[0] = 1.0 / psi ** 2
    for m in range(3):
        s = np.sin(st.kb[m, 0] * x + st.kb[m, 1] * y + st.kb[m, 2] * z + st.pb[m])
        for c in range(3):
            adm[1 + c] += (0.05 / (3.0 * np.sqrt(3.0))) * st.cb[m, c] * s
    adm[4] = adm[7] = adm[9] = psi4
    if st.with_K:
        for m in range(3):
            s = np.cos(st.kk[m, 0] * x + st.kk[m, 1] * y + st.kk[m, 2] * z + st.pk[m])
            for c in range(6):
                adm[10 + c] += (1e-3 / 3.0) * st.ck[m, c] * s
    # velocity primitive w^y = W v^y with |v|^2 = psi^4 (v^y)^2
    W = 1.0 / np.sqrt(1.0 - psi4 * vy * vy)
    prim = np.zeros((5,) + x.shape)
    prim[0] = rho
    prim[2] = W * vy
    prim[4] = P
    # poloidal field: A = A_b (-y', x', 0) about each star, A_b = Ab max(P - cut P_max, 0)
    S = STAR
    Pmax = S["K"] * S["rho_c"] ** 2
    A = []
    stags = [(0, 1, 1), (1, 0, 1), (1, 1, 0)]
    for c in range(3):
        ex, ey, ez = _grid(n, ng, dx, x0, stag=stags[c])
        a = np.zeros_like(ex)
        if c < 2:
            for (cx, cy, cz) in st.centres:
                r2 = (ex - cx) ** 2 + (ey - cy) ** 2 + (ez - cz) ** 2
                Pl = S["K"] * (S["rho_c"] * np.exp(-r2 / S["width"] ** 2)) ** 2
                Ab = S["Ab"] * np.maximum(Pl - S["cut"] * Pmax, 0.0)
                a += (-(ey - cy) * Ab) if c == 0 else ((ex - cx) * Ab)
        A.append(np.ascontiguousarray(a))
    return BlockInputs(n, ng, dx, x0, np.ascontiguousarray(prim), tuple(A), np.ascontiguousarray(adm))


def star_uniform(seed: int = 2, n: int = 128, ng: int = 4, L: float = 96.0, with_K: bool = True) -> BlockInputs:
    """The uniform 128^3 dynamical-metric workload: one star at the origin on
    [-L/2, L/2]^3 (dx = 0.75 at n = 128)."""
    st = spacetime(seed, with_K=with_K, L=L)
    dx = L / n
    return star_block(st, (n, n, n), ng, (dx, dx, dx), (-L / 2,) * 3)


def star_subblock(seed: int = 2, n_full: int = 128, sub: int = 32, corner=(48, 48, 48), ng: int = 4,
                  L: float = 96.0, with_K: bool = True) -> BlockInputs:
    """A sub-cube of the uniform star workload (same fields and dx), used where
    the CPU oracle needs a bounded sample of the 128^3 case."""
    st = spacetime(seed, with_K=with_K, L=L)
    dx = L / n_full
    x0 = tuple(-L / 2 + c * dx for c in corner)
    return star_block(st, (sub, sub, sub), ng, (dx, dx, dx), x0)


# ---------------------------------------------------------------------------
# Con2prim stress cells.

def c2p_stress(n: int, seed: int = 4, gamma: float = 2.0):
    """Independent cells: rho log-U[1e-12,1e-2], T log-U[1e-8,10], W log-U[1,10]
    with isotropic direction, magnetisation sigma = b^2/rho log-U[1e-4,1e2] with
    isotropic B direction, gamma_ij = delta_ij + h_ij with |h_ij| <= 0.2
    (positive definite).  Returns prim [5,n], densitised B~ [3,n], gamma [6,n]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lu = lambda lo, hi: np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))
    rho = lu(1e-12, 1e-2)
    T = lu(1e-8, 1e1)
    W = lu(1.0, 10.0)
    sig = lu(1e-4, 1e2)
    h = rng.uniform(-0.2, 0.2, size=(6, n))
    g = h.copy()
    g[0] += 1.0
    g[3] += 1.0
    g[5] += 1.0
    # |h_ij| <= 0.2 keeps every eigenvalue of delta + h above 1 - 3*0.2 = 0.4

    def unit():
        u = rng.normal(size=(3, n))
        return u / np.linalg.norm(u, axis=0)

    def lower(vec):
        return np.stack([g[0] * vec[0] + g[1] * vec[1] + g[2] * vec[2],
                         g[1] * vec[0] + g[3] * vec[1] + g[4] * vec[2],
                         g[2] * vec[0] + g[4] * vec[1] + g[5] * vec[2]])

    nv = unit()
    nn = np.sqrt((nv * lower(nv)).sum(0))
    vmag = np.sqrt(1.0 - 1.0 / (W * W))
    v = nv * (vmag / nn)
    w = W * v
    nb = unit()
    # B^i = s nb^i with b^2 = B^2/W^2 + (B.v)^2 = sigma rho
    Bl = lower(nb)
    B2u = (nb * Bl).sum(0)
    Bvu = (Bl * v).sum(0)
    s = np.sqrt(sig * rho / (B2u / (W * W) + Bvu * Bvu))
    B = nb * s
    det = (g[0] * (g[3] * g[5] - g[4] * g[4]) - g[1] * (g[1] * g[5] - g[4] * g[2])
           + g[2] * (g[1] * g[4] - g[3] * g[2]))
    Bd = B * np.sqrt(det)
    prim = np.stack([rho, w[0], w[1], w[2], rho * T])
    return np.ascontiguousarray(prim), np.ascontiguousarray(Bd), np.ascontiguousarray(g)


# ---------------------------------------------------------------------------
# AMR-shaped block lists.

@dataclass
class BlockSpec:
    n: int
    level: int
    x0: tuple
    dx: float


def amr_blocks(seed: int = 3, counts=((16, 293), (32, 146), (64, 73)), levels: int = 6,
               dx0: float = 0.75, L: float = 96.0):
    """Blocks of uneven sizes at seeded positions on levels 0..levels-1 with
    dx_l = dx0 2^-l, each inside the [-L/2, L/2]^3 domain of the star."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for n, count in counts:
        for _ in range(count):
            lev = int(rng.integers(0, levels))
            dx = dx0 / 2 ** lev
            ext = n * dx
            lo = -L / 2
            hi = L / 2 - ext
            # centre finer levels on the star, as refinement would
            span = (hi - lo) / 2 ** lev
            c = rng.uniform(-span / 2, span / 2, size=3) - ext / 2
            c = np.clip(c, lo, hi)
            specs.append(BlockSpec(n, lev, tuple(float(v) for v in c), dx))
    return specs


def bns_blocks(seed: int = 5, n: int = 32, levels: int = 6, dx0: float = 0.75, L: float = 96.0,
               target: int = 2000, sep: float = 15.0):
    """Block layout shaped like the paper's binary runs (Sec. 4.5, 5): 32^3
    blocks on 6 levels over [-L/2, L/2]^3, two stars at x = -+sep.  A block of
    level l is refined when its box comes within R_l = s 2^(5-l) 8 of a star
    centre (nested refinement shells around each star); the scale s is the
    largest (by bisection) whose leaf count does not exceed ``target``.
    Returns (leaf BlockSpecs, star centres); ``seed`` is unused (the layout
    is deterministic) and kept for the config-index convention."""
    centres = ((-sep, 0.0, 0.0), (sep, 0.0, 0.0))
    nb0 = int(round(L / (n * dx0)))

    def layout(scale):
        leaves = []
        stack = [(0, (i, j, k)) for k in range(nb0) for j in range(nb0) for i in range(nb0)]
        while stack:
            lev, (i, j, k) = stack.pop()
            dx = dx0 / 2 ** lev
            ext = n * dx
            x0 = (-L / 2 + i * ext, -L / 2 + j * ext, -L / 2 + k * ext)
            R = scale * 2 ** (levels - 1 - lev) * 8.0
            near = any(sum(max(c[a] - (x0[a] + ext), 0.0, x0[a] - c[a]) ** 2 for a in range(3)) < R * R
                       for c in centres)
            if lev < levels - 1 and near:
                for ck in range(2):
                    for cj in range(2):
                        for ci in range(2):
                            stack.append((lev + 1, (2 * i + ci, 2 * j + cj, 2 * k + ck)))
            else:
                leaves.append(BlockSpec(n, lev, x0, dx))
        return leaves

    lo, hi = 0.0, 1.0
    best = layout(lo)
    for _ in range(40):
        mid = 0.5 * (lo + hi)
        cand = layout(mid)
        if len(cand) <= target:
            lo, best = mid, cand
        else:
            hi = mid
    return best, centres


# ---------------------------------------------------------------------------
# Flat-space test problems of Sec. 4.1-4.3 (initial data only).

# Balsara shock tubes (Table 1): Gamma, then left and right states
# (rho, P, v^x, v^y, v^z, B^x, B^y, B^z); discontinuity at x = 0.5.
BALSARA = {
    1: (2.0, (1.0, 1.0, 0.0, 0.0, 0.0, 0.5, 1.0, 0.0), (0.125, 0.1, 0.0, 0.0, 0.0, 0.5, -1.0, 0.0)),
    2: (5.0 / 3.0, (1.0, 30.0, 0.0, 0.0, 0.0, 5.0, 6.0, 6.0), (1.0, 1.0, 0.0, 0.0, 0.0, 5.0, 0.7, 0.7)),
    3: (5.0 / 3.0, (1.0, 1e3, 0.0, 0.0, 0.0, 10.0, 7.0, 7.0), (1.0, 0.1, 0.0, 0.0, 0.0, 10.0, 0.7, 0.7)),
    4: (5.0 / 3.0, (1.0, 0.1, 0.999, 0.0, 0.0, 10.0, 7.0, 7.0), (1.0, 0.1, -0.999, 0.0, 0.0, 10.0, -7.0, -7.0)),
    5: (5.0 / 3.0, (1.08, 0.95, 0.4, 0.3, 0.2, 2.0, 0.3, 0.3), (1.0, 1.0, -0.45, -0.2, 0.2, 2.0, -0.7, 0.5)),
}


def _flat_adm(shape):
    adm = np.zeros((16,) + shape)
    adm[0] = 1.0
    adm[4] = adm[7] = adm[9] = 1.0
    return adm


def _w(vx, vy, vz):
    W = 1.0 / np.sqrt(1.0 - (vx * vx + vy * vy + vz * vz))
    return W * vx, W * vy, W * vz


def balsara_tube(test: int, n: int, ny: int = 2, ng: int = 4) -> BlockInputs:
    """Table 1 Riemann problem on x in [0, 1] (n cells), ny x ny cells of the
    same width across.  Face B~ from an edge potential whose discrete curl is
    exactly the piecewise-constant field: A_y = int_0^x B^z, A_z = B^x y -
    int_0^x B^y (the jump sits on a face for even n)."""
    _, Ls, Rs = BALSARA[test]
    nn = (n, ny, ny)
    dx = (1.0 / n,) * 3
    x0 = (0.0, 0.0, 0.0)
    x, y, z = _grid(nn, ng, dx, x0)
    left = x < 0.5
    pick = lambda a, b: np.where(left, a, b)
    rho, P = pick(Ls[0], Rs[0]), pick(Ls[1], Rs[1])
    wx, wy, wz = (pick(a, b) for a, b in zip(_w(*Ls[2:5]), _w(*Rs[2:5])))
    prim = np.stack([rho, wx, wy, wz, P])
    prim = np.ascontiguousarray(prim * np.ones_like(x))

    def integral(xe, cL, cR):   # int_0^x of the piecewise-constant field
        return np.where(xe < 0.5, cL * xe, cL * 0.5 + cR * (xe - 0.5))

    A = []
    stags = [(0, 1, 1), (1, 0, 1), (1, 1, 0)]
    for c in range(3):
        ex, ey, ez = _grid(nn, ng, dx, x0, stag=stags[c])
        if c == 0:
            a = np.zeros_like(ex)
        elif c == 1:
            a = integral(ex, Ls[7], Rs[7])
        else:
            a = Ls[5] * ey - integral(ex, Ls[6], Rs[6])
        A.append(np.ascontiguousarray(a))
    return BlockInputs(nn, ng, dx, x0, prim, tuple(A), _flat_adm(x.shape))


def field_loop(n: int, ng: int = 4, A0: float = 1e-3, R: float = 0.3) -> BlockInputs:
    """Magnetic loop advection (Sec. 4.3): A_z = A0 (R - r) inside r = R on the
    periodic square [-0.5, 0.5]^2 (n x n cells, one cell across z), rho = 1,
    P = 3, v = (1/1.2, 1/2.4, 0)."""
    nn = (n, n, 1)
    dx = (1.0 / n,) * 3
    x0 = (-0.5, -0.5, 0.0)
    x, y, z = _grid(nn, ng, dx, x0, wrap=True)
    wx, wy, wz = _w(1.0 / 1.2, 1.0 / 2.4, 0.0)
    prim = np.stack([np.ones_like(x), wx * np.ones_like(x), wy * np.ones_like(x), np.zeros_like(x),
                     3.0 * np.ones_like(x)])
    A = []
    stags = [(0, 1, 1), (1, 0, 1), (1, 1, 0)]
    for c in range(3):
        ex, ey, ez = _grid(nn, ng, dx, x0, stag=stags[c], wrap=True)
        if c < 2:
            a = np.zeros_like(ex)
        else:
            r = np.sqrt(ex * ex + ey * ey)
            a = np.where(r <= R, A0 * (R - r), 0.0)
        A.append(np.ascontiguousarray(a))
    return BlockInputs(nn, ng, dx, x0, np.ascontiguousarray(prim), tuple(A), _flat_adm(x.shape))


def cylindrical_blast(bx: float, n: int, ng: int = 4, L: float = 12.0) -> BlockInputs:
    """Magnetised cylindrical blast (Sec. 4.2, after Komissarov 1999) on
    [-6, 6]^2 (n x n cells, one across z): rho = 1e-2, P = 1 inside r = 0.8,
    rho = 1e-4, P = 3e-5 outside r = 1, log-linear in between (our reading of
    "decay exponentially"); v = 0; B = (bx, 0, 0) from A_z = bx y."""
    nn = (n, n, 1)
    dx = (L / n,) * 3
    x0 = (-L / 2, -L / 2, 0.0)
    x, y, z = _grid(nn, ng, dx, x0)
    r = np.sqrt(x * x + y * y)
    t = np.clip((r - 0.8) / 0.2, 0.0, 1.0)
    rho = np.exp((1 - t) * np.log(1e-2) + t * np.log(1e-4))
    P = np.exp((1 - t) * np.log(1.0) + t * np.log(3e-5))
    prim = np.stack([rho, np.zeros_like(x), np.zeros_like(x), np.zeros_like(x), P])
    A = []
    stags = [(0, 1, 1), (1, 0, 1), (1, 1, 0)]
    for c in range(3):
        ex, ey, ez = _grid(nn, ng, dx, x0, stag=stags[c])
        A.append(np.ascontiguousarray(bx * ey if c == 2 else np.zeros_like(ex)))
    return BlockInputs(nn, ng, dx, x0, np.ascontiguousarray(prim), tuple(A), _flat_adm(x.shape))
