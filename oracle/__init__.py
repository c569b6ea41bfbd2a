"""FP64 CPU oracle of the Valencia GRMHD meshblock stage (arXiv:2409.10384).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the library under
``paper_2409_10384_gb300`` never does.  The arithmetic lives in
``grmhd_oracle.cpp`` (plain scalar C++17, built with ``-ffp-contract=off``);
this module only builds it and marshals numpy arrays through ctypes.

Which paper passage each function follows is stated in the C++ source:
prim->cons Eq. 6, fluxes Eq. 8, sources Eq. 9, floors Sec. 3.3, FOFC and the
relaxed DMP Sec. 3.3 / Eq. 19, con2prim Sec. 3.4, reconstruction, Riemann
solvers, CT and SSP-RK Sec. 3.2.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ORACLE_SRC / ORACLE_BUILD point the loader at another copy of the source and
# its build folder (tests/mutation_sweep.py builds mutated copies there).
_SRC = os.environ.get("ORACLE_SRC") or os.path.join(_HERE, "grmhd_oracle.cpp")
_BUILD = os.environ.get("ORACLE_BUILD") or os.path.join(_HERE, "_build")
_LOCK = threading.Lock()
_LIBS: dict = {}

F_FAIL, F_DFLOOR, F_SIGMA, F_TAU, F_RHO, F_TEMP, F_VMAX, F_FOFC = 1, 2, 4, 8, 16, 32, 64, 128
FLOOR_BITS = F_DFLOOR | F_SIGMA | F_TAU | F_RHO | F_TEMP | F_VMAX


def _so(counting: bool) -> str:
    return os.path.join(_BUILD, "liboracle_count.so" if counting else "liboracle.so")


def build(force: bool = False) -> None:
    """Compile both oracle variants (plain and op-counting) in-tree."""
    os.makedirs(_BUILD, exist_ok=True)
    base = ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-shared", "-fPIC", _SRC]
    for counting in (False, True):
        out = _so(counting)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
            continue
        cmd = list(base) + (["-DORACLE_COUNT_FLOPS"] if counting else ["-fopenmp"]) + ["-o", out + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(out + ".tmp", out)


class Params(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("rho_atm", C.c_double), ("T_atm", C.c_double), ("f_thr", C.c_double),
        ("sigma_max", C.c_double), ("dmp_M", C.c_double), ("c2p_tol", C.c_double), ("W_max", C.c_double),
        ("alpha_exc", C.c_double),
        ("recon", C.c_int), ("rsolver", C.c_int), ("fofc", C.c_int), ("rk_order", C.c_int),
        ("c2p_maxit", C.c_int), ("pad_", C.c_int),
        ("eos", C.c_int), ("eos_pieces", C.c_int), ("eos_K0", C.c_double), ("eos_gamma_th", C.c_double),
        ("eos_rho", C.c_double * 3), ("eos_gamma", C.c_double * 4),
    ]


class _Block(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3), ("ng", C.c_int), ("dx", C.c_double * 3),
        ("cons", C.c_void_p), ("cons0", C.c_void_p), ("prim", C.c_void_p),
        ("bf", C.c_void_p * 3), ("bf0", C.c_void_p * 3), ("bcc", C.c_void_p), ("adm", C.c_void_p),
        ("flags", C.c_void_p), ("flux", C.c_void_p * 3), ("emf", C.c_void_p * 3), ("fofc_mask", C.c_void_p),
        ("n_override", C.c_int), ("ov_face", C.c_void_p), ("ov_flux", C.c_void_p),
    ]


class Stats(C.Structure):
    _fields_ = [("cells", C.c_longlong), ("iters", C.c_longlong), ("fails", C.c_longlong),
                ("floors", C.c_longlong), ("fofc_cells", C.c_longlong), ("dmp_cells", C.c_longlong),
                ("fofc_faces", C.c_longlong)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


def lib(counting: bool = False):
    with _LOCK:
        if counting not in _LIBS:
            path = _so(counting)
            if not os.path.exists(path) or os.path.getmtime(path) < os.path.getmtime(_SRC):
                build()
            L = C.CDLL(path)
            dp = C.POINTER(C.c_double)
            L.or_prim2cons.argtypes = [C.POINTER(Params), C.c_long, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_c2p_cells.argtypes = [C.POINTER(Params), C.c_long, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_c2p_master.argtypes = [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]
            L.or_c2p_master.restype = C.c_double
            L.or_bface_from_A.argtypes = [C.POINTER(_Block), C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_bcc.argtypes = [C.POINTER(_Block), C.POINTER(Params)]
            L.or_divb.argtypes = [C.POINTER(_Block), C.c_void_p]
            L.or_c2p_block.argtypes = [C.POINTER(_Block), C.POINTER(Params), C.POINTER(Stats)]
            L.or_stage.argtypes = [C.POINTER(_Block), C.POINTER(Params), C.c_double, C.c_int, C.POINTER(Stats)]
            L.or_stage.restype = C.c_int
            L.or_recon_line.argtypes = [C.c_int, C.c_long, C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_face_flux_at.argtypes = [C.POINTER(_Block), C.POINTER(Params), C.c_int, C.c_int, C.c_int, C.c_int,
                                          C.c_void_p]
            L.or_face_flux_at.restype = C.c_int
            L.or_face_side.argtypes = [C.POINTER(Params), C.c_int, C.c_void_p, C.c_double, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p]
            L.or_face_flux.argtypes = [C.POINTER(Params), C.c_int, C.c_void_p, C.c_void_p, C.c_double,
                                       C.c_void_p, C.c_void_p]
            L.or_eos.argtypes = [C.POINTER(Params), C.c_double, C.c_double, C.c_void_p]
            L.or_eos_press.argtypes = [C.POINTER(Params), C.c_double, C.c_double]
            L.or_eos_press.restype = C.c_double
            L.or_emf_edge.argtypes = [C.c_void_p, C.c_void_p]
            L.or_emf_edge.restype = C.c_double
            L.or_flop_counts.argtypes = [C.POINTER(C.c_longlong)]
            L.or_flop_counts.restype = C.c_int
            L.or_flop_reset.argtypes = []
            L.or_flop_phases.argtypes = [C.POINTER(C.c_longlong)]
            L.or_flop_phases.restype = C.c_int
            _LIBS[counting] = L
            del dp
        return _LIBS[counting]


def params(**kw) -> Params:
    """Defaults: ideal gas Gamma=5/3, flat-space parity setup (configuration 1)."""
    d = dict(gamma=5.0 / 3.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, sigma_max=0.0, dmp_M=0.0,
             c2p_tol=1e-10, W_max=1e3, alpha_exc=0.0, recon=1, rsolver=1, fofc=0, rk_order=2, c2p_maxit=64,
             eos=0, eos_pieces=1, eos_K0=100.0, eos_gamma_th=2.0, eos_rho=(0.0, 0.0, 0.0),
             eos_gamma=(2.0, 2.0, 2.0, 2.0))
    d.update(kw)
    p = Params()
    for k, v in d.items():
        if k in ("eos_rho", "eos_gamma"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def eos(p: Params, rho: float, P: float) -> dict:
    """The oracle's EOS at (rho, P): cold pressure and eps, local index, eps,
    h and rho h c_s^2."""
    out = np.zeros(6)
    lib().or_eos(C.byref(p), float(rho), float(P), _ptr(out))
    return dict(zip(("Pc", "epsc", "Gi", "eps", "h", "chi"), out.tolist()))


def eos_press(p: Params, rho: float, eps: float) -> float:
    return float(lib().or_eos_press(C.byref(p), float(rho), float(eps)))


def _ptr(a: np.ndarray | None):
    if a is None:
        return None
    assert a.flags["C_CONTIGUOUS"] and a.dtype in (np.float64, np.uint8, np.int32)
    return a.ctypes.data


def prim2cons(p: Params, prim: np.ndarray, Bd: np.ndarray, g: np.ndarray, counting: bool = False) -> np.ndarray:
    """Eq. 6 on flat SoA arrays prim [5,n], Bd [3,n], g [6,n] -> cons [5,n]."""
    n = prim.shape[1]
    prim, Bd, g = (np.ascontiguousarray(x, dtype=np.float64) for x in (prim, Bd, g))
    out = np.empty((5, n))
    lib(counting).or_prim2cons(C.byref(p), n, _ptr(prim), _ptr(Bd), _ptr(g), _ptr(out))
    return out


def c2p_cells(p: Params, cons: np.ndarray, Bd: np.ndarray, g: np.ndarray, counting: bool = False):
    """con2prim on independent cells.  Returns dict(prim, cons (floored), flags, iters, mu, eps_margin)."""
    n = cons.shape[1]
    cons = np.array(cons, dtype=np.float64, order="C", copy=True)
    Bd, g = (np.ascontiguousarray(x, dtype=np.float64) for x in (Bd, g))
    prim = np.empty((5, n))
    flags = np.empty(n, np.uint8)
    iters = np.empty(n, np.int32)
    mu = np.empty(n)
    em = np.empty(n)
    lib(counting).or_c2p_cells(C.byref(p), n, _ptr(cons), _ptr(Bd), _ptr(g), _ptr(prim), _ptr(flags),
                               _ptr(iters), _ptr(mu), _ptr(em))
    return dict(prim=prim, cons=cons, flags=flags, iters=iters, mu=mu, eps_margin=em)


def c2p_master(p: Params, cons5, Bd3, g6, mu: float):
    """KRP master function f(mu) of one cell; also (mu_plus, f(0), f(mu_plus))."""
    c = np.ascontiguousarray(cons5, dtype=np.float64)
    b = np.ascontiguousarray(Bd3, dtype=np.float64)
    g = np.ascontiguousarray(g6, dtype=np.float64)
    out = np.zeros(3)
    f = lib().or_c2p_master(C.byref(p), _ptr(c), _ptr(b), _ptr(g), float(mu), _ptr(out))
    return f, out


@dataclass
class Block:
    """Numpy-held meshblock in the library's layout (SoA, ghost-inclusive)."""
    n: tuple
    ng: int
    dx: tuple
    adm: np.ndarray
    cons: np.ndarray = None
    cons0: np.ndarray = None
    prim: np.ndarray = None
    bf: list = field(default_factory=list)
    bf0: list = field(default_factory=list)
    bcc: np.ndarray = None
    flags: np.ndarray = None

    @property
    def N(self):
        return tuple(x + 2 * self.ng for x in self.n)  # (N1, N2, N3)

    def face_shape(self, d):
        N1, N2, N3 = self.N
        return [(N3, N2, N1 + 1), (N3, N2 + 1, N1), (N3 + 1, N2, N1)][d]

    def edge_shape(self, c):
        N1, N2, N3 = self.N
        return [(N3 + 1, N2 + 1, N1), (N3 + 1, N2, N1 + 1), (N3, N2 + 1, N1 + 1)][c]

    def copy(self) -> "Block":
        b = Block(self.n, self.ng, self.dx, self.adm)
        for k in ("cons", "cons0", "prim", "bcc", "flags"):
            setattr(b, k, None if getattr(self, k) is None else getattr(self, k).copy())
        b.bf = [x.copy() for x in self.bf]
        b.bf0 = [x.copy() for x in self.bf0]
        return b

    def _struct(self, flux=None, emf=None, mask=None, override=None) -> _Block:
        s = _Block()
        s.n = (C.c_int * 3)(*self.n)
        s.ng = self.ng
        s.dx = (C.c_double * 3)(*self.dx)
        s.cons, s.cons0, s.prim, s.bcc = _ptr(self.cons), _ptr(self.cons0), _ptr(self.prim), _ptr(self.bcc)
        s.adm, s.flags = _ptr(self.adm), _ptr(self.flags)
        for d in range(3):
            s.bf[d] = _ptr(self.bf[d])
            s.bf0[d] = _ptr(self.bf0[d])
            s.flux[d] = _ptr(flux[d]) if flux is not None else None
            s.emf[d] = _ptr(emf[d]) if emf is not None else None
        s.fofc_mask = _ptr(mask)
        s.n_override = 0
        if override is not None:
            faces, fl = override
            s.n_override = len(faces)
            s.ov_face = _ptr(faces)
            s.ov_flux = _ptr(fl)
        return s


def new_block(n, ng, dx, adm: np.ndarray) -> Block:
    b = Block(tuple(int(x) for x in n), int(ng), tuple(float(x) for x in dx), np.ascontiguousarray(adm, np.float64))
    N1, N2, N3 = b.N
    b.cons = np.zeros((5, N3, N2, N1))
    b.cons0 = np.zeros((5, N3, N2, N1))
    b.prim = np.zeros((5, N3, N2, N1))
    b.bcc = np.zeros((3, N3, N2, N1))
    b.flags = np.zeros((N3, N2, N1), np.uint8)
    b.bf = [np.zeros(b.face_shape(d)) for d in range(3)]
    b.bf0 = [np.zeros(b.face_shape(d)) for d in range(3)]
    return b


def init_block(p: Params, n, ng, dx, adm, prim, A) -> Block:
    """Face B~ = discrete curl of the edge potential A, bcc = face average,
    cons = prim->cons (Eq. 6) on every cell."""
    b = new_block(n, ng, dx, adm)
    A = [np.ascontiguousarray(a, np.float64) for a in A]
    for c in range(3):
        assert A[c].shape == b.edge_shape(c), (A[c].shape, b.edge_shape(c))
    s = b._struct()
    lib().or_bface_from_A(C.byref(s), _ptr(A[0]), _ptr(A[1]), _ptr(A[2]))
    lib().or_bcc(C.byref(s), C.byref(p))
    b.prim[...] = prim
    ncell = b.prim[0].size
    g = np.ascontiguousarray(b.adm[4:10].reshape(6, ncell))
    b.cons[...] = prim2cons(p, b.prim.reshape(5, ncell), b.bcc.reshape(3, ncell), g).reshape(b.cons.shape)
    return b


def bcc(p: Params, b: Block) -> None:
    lib().or_bcc(C.byref(b._struct()), C.byref(p))


def divb(b: Block) -> np.ndarray:
    out = np.zeros(b.cons.shape[1:])
    lib().or_divb(C.byref(b._struct()), _ptr(out))
    return out


def c2p_block(p: Params, b: Block) -> dict:
    st = Stats()
    lib().or_c2p_block(C.byref(b._struct()), C.byref(p), C.byref(st))
    return st.as_dict()


def stage(p: Params, b: Block, dt: float, stage_idx: int, mask: np.ndarray | None = None,
          keep: bool = False, counting: bool = False, override=None):
    """One RK stage in place.  Returns stats, plus fluxes/EMFs when keep=True.
    ``mask`` (uint8 per cell) replaces the FOFC flags computed by the oracle.
    ``override``: [((d, k, j, i), F7), ...], faces whose high-order flux is
    replaced by F7 before FOFC (a limiter decision taken down its other
    branch; F7 from ``face_flux_at`` on data within rounding)."""
    flux = [np.zeros((7,) + b.face_shape(d)) for d in range(3)] if keep else None
    emf = [np.zeros(b.edge_shape(c)) for c in range(3)] if keep else None
    if mask is not None:
        mask = np.ascontiguousarray(mask, np.uint8)
    ov = None
    if override:
        ov = (np.ascontiguousarray([[int(x) for x in f] for f, _ in override], np.int32),
              np.ascontiguousarray([np.asarray(F, np.float64) for _, F in override], np.float64))
    st = Stats()
    rc = lib(counting).or_stage(C.byref(b._struct(flux, emf, mask, ov)), C.byref(p), float(dt), int(stage_idx),
                                C.byref(st))
    if rc != 0:
        raise RuntimeError(f"or_stage failed with code {rc}")
    out = st.as_dict()
    if keep:
        out["flux"] = flux
        out["emf"] = emf
    return out


def step(p: Params, b: Block, dt: float, fill=None) -> list:
    """A full SSP-RK step; ``fill(b)`` refreshes ghost zones between stages."""
    stats = []
    for s in range(p.rk_order):
        if fill is not None:
            fill(b)
        stats.append(stage(p, b, dt, s))
    return stats


PHASES = ("c2p", "flux", "fofc_flag", "fofc_fix", "emf", "update")


def flop_phases(p: Params, b: Block, dt: float, stage_idx: int) -> dict:
    """Algorithmic FP64 operations of each phase of one stage (counting build):
    {phase: {add, mul, div, sqrt, cmp}} plus the stage stats."""
    L = lib(True)
    L.or_flop_reset()
    st = stage(p, b.copy(), dt, stage_idx, counting=True)
    out = (C.c_longlong * 30)()
    L.or_flop_phases(out)
    cum = [[int(out[5 * k + m]) for m in range(5)] for k in range(6)]
    res = {}
    prev = [0] * 5
    for k, name in enumerate(PHASES):
        res[name] = dict(zip(("add", "mul", "div", "sqrt", "cmp"), (cum[k][m] - prev[m] for m in range(5))))
        prev = cum[k]
    res["stats"] = st
    return res


def flop_counts(p: Params, b: Block, dt: float, stage_idx: int) -> dict:
    """Algorithmic FP64 operations of one stage on block ``b`` (counting build)."""
    L = lib(True)
    L.or_flop_reset()
    stage(p, b.copy(), dt, stage_idx, counting=True)
    out = (C.c_longlong * 5)()
    L.or_flop_counts(out)
    return dict(zip(("add", "mul", "div", "sqrt", "cmp"), (int(x) for x in out)))


def face_flux_at(p: Params, b: Block, d: int, face) -> np.ndarray:
    """The high-order flux (Eq. 8, 7 components) of face (k, j, i) of
    direction d from the block's primitives, cell-centred and face B~ and
    metric as they stand (the caller fills prim and bcc, e.g. by c2p_block)."""
    k, j, i = (int(x) for x in face)
    F = np.zeros(7)
    rc = lib().or_face_flux_at(C.byref(b._struct()), C.byref(p), int(d), k, j, i, _ptr(F))
    if rc != 0:
        raise ValueError(f"face ({d}, {k}, {j}, {i}) outside the block's stencil range")
    return F


def recon_line(recon: int, q: np.ndarray):
    """Left/right states at the faces between q[f-1] and q[f], f = 3..n-3 (NaN elsewhere)."""
    q = np.ascontiguousarray(q, np.float64)
    L = np.full(q.shape, np.nan)
    R = np.full(q.shape, np.nan)
    lib().or_recon_line(int(recon), q.size, _ptr(q), _ptr(L), _ptr(R))
    return L, R


def face_side(p: Params, d: int, st7, Bn: float, m10):
    """One side of a face: (U7, F7, (lambda-, lambda+))."""
    st = np.ascontiguousarray(st7, np.float64)
    m = np.ascontiguousarray(m10, np.float64)
    U = np.zeros(7)
    F = np.zeros(7)
    sp = np.zeros(2)
    lib().or_face_side(C.byref(p), int(d), _ptr(st), float(Bn), _ptr(m), _ptr(U), _ptr(F), _ptr(sp))
    return U, F, sp


def face_flux(p: Params, d: int, L7, R7, Bn: float, m10):
    Lq = np.ascontiguousarray(L7, np.float64)
    Rq = np.ascontiguousarray(R7, np.float64)
    m = np.ascontiguousarray(m10, np.float64)
    F = np.zeros(7)
    lib().or_face_flux(C.byref(p), int(d), _ptr(Lq), _ptr(Rq), float(Bn), _ptr(m), _ptr(F))
    return F


def emf_edge(e8, f4) -> float:
    e = np.ascontiguousarray(e8, np.float64)
    f = np.ascontiguousarray(f4, np.float64)
    return float(lib().or_emf_edge(_ptr(e), _ptr(f)))
