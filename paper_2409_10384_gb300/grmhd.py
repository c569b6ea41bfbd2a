"""Thin ctypes binding of libgrmhd (include/grmhd.h): argument marshalling only.

Every step of the path runs in the library's CUDA kernels; this module turns
torch tensors into the C structs and raw pointers the C-ABI takes.  There is no
CPU fallback: if the compiled library is missing the import of ``lib()``
raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

import numpy as np

from . import build as _build

MHD_F_FAIL, MHD_F_DFLOOR, MHD_F_SIGMA, MHD_F_TAU, MHD_F_RHO, MHD_F_TEMP, MHD_F_VMAX, MHD_F_FOFC = (
    1, 2, 4, 8, 16, 32, 64, 128)
_ERR = {0: "ok", -1: "invalid argument", -2: "CUDA runtime error", -3: "device allocation failed",
        -4: "call out of order", -5: "learned guess requested but no network loaded",
        -6: "block exceeds the 16 MiB static scratch of mhd_stage_noalloc"}


class mhd_params(C.Structure):
    _fields_ = [
        ("gamma", C.c_double), ("rho_atm", C.c_double), ("T_atm", C.c_double), ("f_thr", C.c_double),
        ("sigma_max", C.c_double), ("dmp_M", C.c_double), ("c2p_tol", C.c_double), ("W_max", C.c_double),
        ("alpha_exc", C.c_double),
        ("recon", C.c_int), ("rsolver", C.c_int), ("fofc", C.c_int), ("rk_order", C.c_int),
        ("c2p_maxit", C.c_int), ("c2p_guess", C.c_int),
        ("eos", C.c_int), ("eos_pieces", C.c_int), ("eos_K0", C.c_double), ("eos_gamma_th", C.c_double),
        ("eos_rho", C.c_double * 3), ("eos_gamma", C.c_double * 4), ("fixed_metric", C.c_int),
    ]


class mhd_block(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3), ("ng", C.c_int), ("dx", C.c_double * 3),
        ("cons", C.c_void_p), ("cons0", C.c_void_p), ("prim", C.c_void_p),
        ("bf", C.c_void_p * 3), ("bf0", C.c_void_p * 3), ("bcc", C.c_void_p), ("adm", C.c_void_p),
        ("flags", C.c_void_p),
    ]


class mhd_stats(C.Structure):
    _fields_ = [("cells", C.c_longlong), ("iters", C.c_longlong), ("fails", C.c_longlong),
                ("floors", C.c_longlong), ("fofc_cells", C.c_longlong), ("dmp_cells", C.c_longlong),
                ("fofc_faces", C.c_longlong), ("guess_fallbacks", C.c_longlong), ("fp32_evals", C.c_longlong),
                ("fofc_fp32", C.c_longlong)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_LOCK = threading.Lock()
_LIB = None

# name -> (restype, argtypes)
_VP, _I, _L, _D = C.c_void_p, C.c_int, C.c_long, C.c_double
_SIGS = {
    "mhd_init": (_I, [C.POINTER(mhd_params), C.POINTER(_VP)]),
    "mhd_set_params": (_I, [_VP, C.POINTER(mhd_params)]),
    "mhd_finalize": (None, [_VP]),
    "mhd_strerror": (C.c_char_p, [_I]),
    "mhd_init_block": (_I, [_VP, C.POINTER(mhd_block), C.POINTER(_VP), _VP]),
    "mhd_prim2cons": (_I, [_VP, _L, _VP, _VP, _VP, _VP, _VP]),
    "mhd_c2p_cells": (_I, [_VP, _L, _VP, _VP, _VP, _VP, _VP, _VP, _VP, C.POINTER(mhd_stats)]),
    "mhd_c2p": (_I, [_VP, C.POINTER(mhd_block), _I, _VP, C.POINTER(mhd_stats)]),
    "mhd_rhs": (_I, [_VP, C.POINTER(mhd_block), _I, _D, _I, _VP]),
    "mhd_rk_update": (_I, [_VP, C.POINTER(mhd_block), _I, _D, _I, _VP]),
    "mhd_step": (_I, [_VP, C.POINTER(mhd_block), _I, _D, _I, _VP]),
    "mhd_graph_step": (_I, [_VP, C.POINTER(mhd_block), _I, _D, _VP]),
    "mhd_step_overlap": (_I, [_VP, C.POINTER(mhd_block), _I, _D, _VP, _VP]),
    "mhd_read_stats": (_I, [_VP, C.POINTER(mhd_stats), _VP]),
    "mhd_reset_stats": (_I, [_VP, _VP]),
    "mhd_scratch_copy": (_I, [_VP, _I, _I, _VP, _L, C.POINTER(_L), _VP]),
    "mhd_kernel_launches": (C.c_longlong, [_VP]),
    "mhd_profile": (_I, [_VP, _I]),
    "mhd_profile_read": (_I, [_VP, _VP, _VP]),
    "mhd_kernel_name": (C.c_char_p, [_I]),
    "mhd_stage_noalloc": (_I, [C.POINTER(mhd_params), C.POINTER(mhd_block), _D, _I, _VP]),
    "mhd_autotune": (_I, [_VP, C.POINTER(mhd_block), _I, _D, _VP, _VP]),
    "mhd_set_launch": (_I, [_VP, _I, _I, _I]),
    "mhd_ledger": (_I, [_VP, _I]),
    "mhd_fill_ghosts": (_I, [_VP, C.POINTER(mhd_block), _I, C.POINTER(C.c_int), _VP]),
    "mhd_ledger_read": (_I, [_VP, C.POINTER(C.c_double), _I, _VP]),
    "mhd_block_mass": (_I, [_VP, C.POINTER(mhd_block), _I, C.POINTER(C.c_double), _VP]),
    "mhd_get_launch": (_I, [_VP, _I, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "mhd_mlp_init": (_I, [_VP, C.c_ulonglong]),
    "mhd_mlp_dataset": (_I, [_VP, _L, _VP, _VP, _VP, _VP, _VP, _VP]),
    "mhd_mlp_train": (_I, [_VP, _VP, _VP, _L, _I, _I, C.c_float, C.c_ulonglong, C.POINTER(C.c_float), _VP]),
    "mhd_mlp_calibrate": (_I, [_VP, _VP, _VP, _L, _D, C.POINTER(_D), _VP]),
    "mhd_mlp_infer": (_I, [_VP, _VP, _L, _VP, _VP]),
    "mhd_mlp_grad": (_I, [_VP, _VP, _VP, _L, _VP, C.POINTER(C.c_float), _VP]),
    "mhd_mlp_get": (_I, [_VP, _VP]),
    "mhd_mlp_set": (_I, [_VP, _VP]),
    "mhd_mlp_save": (_I, [_VP, _VP, _L, C.POINTER(_L)]),
    "mhd_mlp_load": (_I, [_VP, _VP, _L]),
    "mhd_check_rcp": (_I, [_VP, _L, _VP, _VP]),
    "mhd_check_enclosures": (_I, [_VP, _L, _VP, _VP]),
}
MHD_NKERNEL = 13
MLP_NPARAM = 4609
MLP_NSTATE = 4609 + 13
MLP_FSTRIDE = 8
MLP_BLOB_BYTES = 2 * 4609 + 4 * 13


def header_symbols() -> list:
    """Every function name declared in include/grmhd.h."""
    h = open(os.path.join(_build.ROOT, "include", "grmhd.h")).read()
    h = re.sub(r"/\*.*?\*/", "", h, flags=re.S)
    return sorted(set(re.findall(r"\b(mhd_[a-z0-9_]+)\s*\(", h)))


def lib(path: str | None = None):
    """Load libgrmhd.so (built in-tree by ``build.build()``); raises if absent."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            p = path or _build.LIB
            if not os.path.exists(p):
                raise RuntimeError(f"libgrmhd.so not built ({p}); run paper_2409_10384_gb300.build.build()")
            L = C.CDLL(p)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _LIB = L
        return _LIB


class MHDError(RuntimeError):
    pass


def check(rc: int, what: str = ""):
    if rc != 0:
        raise MHDError(f"{what}: {_ERR.get(rc, rc)} ({rc})")


def params(**kw) -> mhd_params:
    d = dict(gamma=5.0 / 3.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, sigma_max=0.0, dmp_M=0.0, c2p_tol=1e-10,
             W_max=1e3, alpha_exc=0.0, recon=1, rsolver=1, fofc=0, rk_order=2, c2p_maxit=64, c2p_guess=0,
             eos=0, eos_pieces=1, eos_K0=100.0, eos_gamma_th=2.0, eos_rho=(0.0, 0.0, 0.0),
             eos_gamma=(2.0, 2.0, 2.0, 2.0), fixed_metric=0)
    d.update(kw)
    p = mhd_params()
    for k, v in d.items():
        if k in ("eos_rho", "eos_gamma"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(p, k, v)
    return p


def _ptr(t):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device, contiguous tensors only"
    return C.c_void_p(t.data_ptr())


def _sptr(stream):
    if stream is None:
        return None
    return C.c_void_p(int(stream.cuda_stream))


class DeviceBlock:
    """Caller-owned device arrays of one meshblock (torch tensors, FP64)."""

    def __init__(self, n, ng, dx, adm, device="cuda"):
        import torch
        self.n = tuple(int(x) for x in n)
        self.ng = int(ng)
        self.dx = tuple(float(x) for x in dx)
        N1, N2, N3 = (x + 2 * self.ng for x in self.n)
        self.N = (N1, N2, N3)
        f64 = dict(dtype=torch.float64, device=device)
        self.adm = torch.as_tensor(adm, **f64).contiguous()
        assert tuple(self.adm.shape) == (16, N3, N2, N1)
        self.cons = torch.zeros((5, N3, N2, N1), **f64)
        self.cons0 = torch.zeros((5, N3, N2, N1), **f64)
        self.prim = torch.zeros((5, N3, N2, N1), **f64)
        self.bcc = torch.zeros((3, N3, N2, N1), **f64)
        self.flags = torch.zeros((N3, N2, N1), dtype=torch.uint8, device=device)
        shp = [(N3, N2, N1 + 1), (N3, N2 + 1, N1), (N3 + 1, N2, N1)]
        self.bf = [torch.zeros(s, **f64) for s in shp]
        self.bf0 = [torch.zeros(s, **f64) for s in shp]

    def edge_shape(self, c):
        N1, N2, N3 = self.N
        return [(N3 + 1, N2 + 1, N1), (N3 + 1, N2, N1 + 1), (N3, N2 + 1, N1 + 1)][c]

    def desc(self) -> mhd_block:
        b = mhd_block()
        b.n = (C.c_int * 3)(*self.n)
        b.ng = self.ng
        b.dx = (C.c_double * 3)(*self.dx)
        b.cons, b.cons0, b.prim = self.cons.data_ptr(), self.cons0.data_ptr(), self.prim.data_ptr()
        b.bcc, b.adm, b.flags = self.bcc.data_ptr(), self.adm.data_ptr(), self.flags.data_ptr()
        for d in range(3):
            b.bf[d] = self.bf[d].data_ptr()
            b.bf0[d] = self.bf0[d].data_ptr()
        return b


def _block_ptrs(b: DeviceBlock) -> tuple:
    return (b.n, b.ng, b.dx, b.cons.data_ptr(), b.cons0.data_ptr(), b.prim.data_ptr(), b.bcc.data_ptr(),
            b.adm.data_ptr(), b.flags.data_ptr()) + tuple(x.data_ptr() for x in b.bf) + \
        tuple(x.data_ptr() for x in b.bf0)


def stage_noalloc(p: mhd_params, blk: DeviceBlock, dt: float, stage: int, stream=None) -> int:
    """mhd_stage_noalloc on one block (no context, no device allocation);
    returns the status code."""
    d = blk.desc()
    return int(lib().mhd_stage_noalloc(C.byref(p), C.byref(d), float(dt), int(stage), _sptr(stream)))


def check_rcp(x, stream=None):
    """mhd_check_rcp: relative differences of the library's fast reciprocal
    from the correctly rounded division, [n][2] (1/x, (x + 1)/x)."""
    import torch
    out = torch.empty((x.shape[0], 2), dtype=torch.float64, device="cuda")
    check(lib().mhd_check_rcp(_ptr(x), x.shape[0], _ptr(out), _sptr(stream)), "mhd_check_rcp")
    return out


def check_enclosures(x, stream=None):
    """mhd_check_enclosures: per value, the bits of the FP32 enclosures that
    miss their FP64 value (0: all enclose), [n] uint8."""
    import torch
    out = torch.empty((x.shape[0],), dtype=torch.uint8, device="cuda")
    check(lib().mhd_check_enclosures(_ptr(x), x.shape[0], _ptr(out), _sptr(stream)), "mhd_check_enclosures")
    return out


def block_array(blocks) -> C.Array:
    arr = (mhd_block * len(blocks))()
    for i, b in enumerate(blocks):
        arr[i] = b.desc()
    return arr


class Context:
    """Owns one mhd_ctx.  Method names follow the C-ABI entry points."""

    def __init__(self, p: mhd_params):
        self.L = lib()
        self.p = p
        h = C.c_void_p()
        check(self.L.mhd_init(C.byref(p), C.byref(h)), "mhd_init")
        self.h = h
        self._arr = None
        self._key = None
        self._held = []

    def close(self):
        self._arr, self._key, self._held = None, None, []
        if self.h:
            self.L.mhd_finalize(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p: mhd_params):
        check(self.L.mhd_set_params(self.h, C.byref(p)), "mhd_set_params")
        self.p = p

    def _blocks(self, blocks):
        """Descriptor array of a block list, rebuilt whenever any device
        pointer differs from the cached list's.  Object ids alone are not a
        key: a freed block's id can be reused by a new block whose arrays live
        elsewhere."""
        blocks = list(blocks)
        key = tuple(_block_ptrs(b) for b in blocks)
        if key != self._key:
            self._arr = block_array(blocks)
            self._key = key
            self._held = blocks   # the cached descriptors point into these blocks
        return self._arr, len(blocks)

    def init_block(self, blk: DeviceBlock, A, stream=None):
        d = blk.desc()
        At = [a.contiguous() for a in A]
        for c in range(3):
            assert tuple(At[c].shape) == blk.edge_shape(c)
        arr = (C.c_void_p * 3)(*[a.data_ptr() for a in At])
        check(self.L.mhd_init_block(self.h, C.byref(d), arr, _sptr(stream)), "mhd_init_block")
        self._keep = At

    def prim2cons(self, prim, Bd, g, cons, stream=None):
        n = prim.shape[1]
        check(self.L.mhd_prim2cons(self.h, n, _ptr(prim), _ptr(Bd), _ptr(g), _ptr(cons), _sptr(stream)),
              "mhd_prim2cons")

    def c2p_cells(self, cons, Bd, g, prim, flags, iters=None, stream=None, stats=False):
        """con2prim of independent cells; with stats=True returns the counters
        this call added (the call then synchronises the stream).  prim=None:
        flags only (1 where con2prim fails or a floor fires; cons untouched)."""
        n = cons.shape[1]
        st = mhd_stats() if stats else None
        check(self.L.mhd_c2p_cells(self.h, n, _ptr(cons), _ptr(Bd), _ptr(g), _ptr(prim), _ptr(flags),
                                   _ptr(iters), _sptr(stream), C.byref(st) if stats else None), "mhd_c2p_cells")
        return st.as_dict() if stats else None

    def c2p(self, blocks, stream=None, stats=False):
        arr, nb = self._blocks(blocks)
        st = mhd_stats() if stats else None
        check(self.L.mhd_c2p(self.h, arr, nb, _sptr(stream), C.byref(st) if stats else None), "mhd_c2p")
        return st.as_dict() if stats else None

    def rhs(self, blocks, dt, stage, stream=None):
        arr, nb = self._blocks(blocks)
        check(self.L.mhd_rhs(self.h, arr, nb, float(dt), int(stage), _sptr(stream)), "mhd_rhs")

    def rk_update(self, blocks, dt, stage, stream=None):
        arr, nb = self._blocks(blocks)
        check(self.L.mhd_rk_update(self.h, arr, nb, float(dt), int(stage), _sptr(stream)), "mhd_rk_update")

    def stage(self, blocks, dt, stage, stream=None):
        self.c2p(blocks, stream)
        self.rhs(blocks, dt, stage, stream)
        self.rk_update(blocks, dt, stage, stream)

    def step(self, blocks, dt, graph=False, stream=None, per_block=False):
        arr, nb = self._blocks(blocks)
        mode = 2 if per_block else int(bool(graph))
        check(self.L.mhd_step(self.h, arr, nb, float(dt), mode, _sptr(stream)), "mhd_step")

    def graph_step(self, blocks, dt, stream):
        """mhd_graph_step: the captured full RK step (stream must not be the
        legacy default stream)."""
        arr, nb = self._blocks(blocks)
        check(self.L.mhd_graph_step(self.h, arr, nb, float(dt), _sptr(stream)), "mhd_graph_step")

    def step_overlap(self, blocks, dt, stream=None, state_ready=None):
        """mhd_step_overlap: an ungraphed step whose stages wait for the torch
        CUDA event state_ready (recorded after the state's copies) while its
        metric kernel runs."""
        arr, nb = self._blocks(blocks)
        ev = None if state_ready is None else C.c_void_p(int(state_ready.cuda_event))
        check(self.L.mhd_step_overlap(self.h, arr, nb, float(dt), _sptr(stream), ev), "mhd_step_overlap")

    def step_host(self, blk: DeviceBlock, host: dict, dt, stream=None, graph=False):
        """One RK step of a block whose state lives in (pinned) host memory:
        host["cons"], host["bf"][0..2] and host["adm"] are copied in, the step
        runs, and the conserved state and face B~ are copied back, all on
        `stream`."""
        import torch
        s = stream or torch.cuda.current_stream()
        with torch.cuda.stream(s):
            blk.cons.copy_(host["cons"], non_blocking=True)
            blk.adm.copy_(host["adm"], non_blocking=True)
            for d in range(3):
                blk.bf[d].copy_(host["bf"][d], non_blocking=True)
            self.step([blk], dt, graph=graph, stream=s)
            host["cons"].copy_(blk.cons, non_blocking=True)
            for d in range(3):
                host["bf"][d].copy_(blk.bf[d], non_blocking=True)

    def host_stepper(self, blk: "DeviceBlock", host: dict, stream=None) -> "HostStepper":
        """A stepper for a block whose state and metric live in pinned host
        memory, with its host copies pipelined (see HostStepper)."""
        return HostStepper(self, blk, host, stream)

    def autotune(self, blocks, dt, stream=None) -> dict:
        """Tune the launch configuration of this block list; {kernel: (CTA size, waves)}."""
        arr, nb = self._blocks(blocks)
        out = (C.c_int * 18)()
        check(self.L.mhd_autotune(self.h, arr, nb, float(dt), _sptr(stream), out), "mhd_autotune")
        names = ("c2p_prep", "c2p_finish", "flux_x", "flux_y", "flux_z", "fofc_prep", "fofc_finish", "emf", "update")
        return {nm: (out[2 * k], out[2 * k + 1]) for k, nm in enumerate(names)}

    TUNABLE = ("c2p_prep", "c2p_finish", "flux_x", "flux_y", "flux_z", "fofc_prep", "fofc_finish", "emf", "update")

    def set_launch(self, kernel: str, threads: int, waves: int):
        """Pin the launch shape (CTA size, waves) of one tunable kernel."""
        check(self.L.mhd_set_launch(self.h, self.TUNABLE.index(kernel), int(threads), int(waves)), "mhd_set_launch")

    def get_launch(self, kernel: str):
        t, w = C.c_int(), C.c_int()
        check(self.L.mhd_get_launch(self.h, self.TUNABLE.index(kernel), C.byref(t), C.byref(w)), "mhd_get_launch")
        return t.value, w.value

    def fill_ghosts(self, blocks, nbr, stream=None):
        """Ghost zones from same-level neighbours: nbr int [nblocks][6] over
        the sides -x, +x, -y, +y, -z, +z (neighbour block index, -1 outflow,
        -2 untouched)."""
        arr, nb = self._blocks(blocks)
        t = np.ascontiguousarray(np.asarray(nbr, dtype=np.int32).reshape(nb, 6))
        check(self.L.mhd_fill_ghosts(self.h, arr, nb, t.ctypes.data_as(C.POINTER(C.c_int)), _sptr(stream)),
              "mhd_fill_ghosts")

    # --------------------------------------------------- baryon-mass ledger
    def ledger(self, enable: bool = True):
        """Switch the per-block baryon-mass ledger on or off."""
        check(self.L.mhd_ledger(self.h, 1 if enable else 0), "mhd_ledger")
        self._key = None   # the library re-plans its scratch on the next call

    def ledger_read(self, nblocks: int, reset=False, stream=None) -> np.ndarray:
        """Balance of each block since the last reset: floor mass plus
        -dt b_s x boundary D~ flux, summed over stages with RK weights."""
        out = np.zeros(nblocks)
        check(self.L.mhd_ledger_read(self.h, out.ctypes.data_as(C.POINTER(C.c_double)), 1 if reset else 0,
                                     _sptr(stream)), "mhd_ledger_read")
        return out

    def block_mass(self, blocks, stream=None) -> np.ndarray:
        """Interior sum of D~ dx dy dz of every block."""
        arr, nb = self._blocks(blocks)
        out = np.zeros(nb)
        check(self.L.mhd_block_mass(self.h, arr, nb, out.ctypes.data_as(C.POINTER(C.c_double)), _sptr(stream)),
              "mhd_block_mass")
        return out

    def read_stats(self, stream=None) -> dict:
        s = mhd_stats()
        check(self.L.mhd_read_stats(self.h, C.byref(s), _sptr(stream)), "mhd_read_stats")
        return s.as_dict()

    def reset_stats(self, stream=None):
        check(self.L.mhd_reset_stats(self.h, _sptr(stream)), "mhd_reset_stats")

    def scratch(self, b: int, which: int, shape=None, stream=None):
        """Host copy of a scratch array (fluxes 0..2, EMFs 3..5) of block b."""
        n = C.c_long()
        check(self.L.mhd_scratch_copy(self.h, int(b), int(which), None, 0, C.byref(n), _sptr(stream)),
              "mhd_scratch_copy")
        host = np.empty(n.value, np.float64)
        check(self.L.mhd_scratch_copy(self.h, int(b), int(which), host.ctypes.data_as(C.c_void_p), n.value, None,
                                      _sptr(stream)), "mhd_scratch_copy")
        return host if shape is None else host.reshape(shape)

    # ----------------------------------------------------- learned guess
    def mlp_init(self, seed=1):
        check(self.L.mhd_mlp_init(self.h, int(seed)), "mhd_mlp_init")

    def mlp_dataset(self, cons, Bd, g, stream=None):
        """(features [n][8] float32, log(mu) [n] float32) device tensors."""
        import torch
        n = cons.shape[1]
        feat = torch.zeros((n, MLP_FSTRIDE), dtype=torch.float32, device="cuda")
        logmu = torch.zeros(n, dtype=torch.float32, device="cuda")
        check(self.L.mhd_mlp_dataset(self.h, n, _ptr(cons), _ptr(Bd), _ptr(g), _ptr(feat), _ptr(logmu),
                                     _sptr(stream)), "mhd_mlp_dataset")
        return feat, logmu

    def mlp_train(self, feat, logmu, epochs=20, batch=4096, lr=3e-3, seed=7, stream=None) -> float:
        loss = C.c_float()
        check(self.L.mhd_mlp_train(self.h, _ptr(feat), _ptr(logmu), feat.shape[0], int(epochs), int(batch),
                                   float(lr), int(seed), C.byref(loss), _sptr(stream)), "mhd_mlp_train")
        return float(loss.value)

    def mlp_calibrate(self, feat, logmu, quantile=0.999, stream=None) -> float:
        d = C.c_double()
        check(self.L.mhd_mlp_calibrate(self.h, _ptr(feat), _ptr(logmu), feat.shape[0], float(quantile),
                                       C.byref(d), _sptr(stream)), "mhd_mlp_calibrate")
        return float(d.value)

    def mlp_infer(self, feat, stream=None):
        import torch
        out = torch.zeros(feat.shape[0], dtype=torch.float32, device="cuda")
        check(self.L.mhd_mlp_infer(self.h, _ptr(feat), feat.shape[0], _ptr(out), _sptr(stream)), "mhd_mlp_infer")
        return out

    def mlp_grad(self, feat, logmu, stream=None):
        g = np.zeros(MLP_NPARAM, np.float32)
        loss = C.c_float()
        check(self.L.mhd_mlp_grad(self.h, _ptr(feat), _ptr(logmu), feat.shape[0], g.ctypes.data_as(C.c_void_p),
                                  C.byref(loss), _sptr(stream)), "mhd_mlp_grad")
        return g, float(loss.value)

    def mlp_get(self) -> np.ndarray:
        st = np.zeros(MLP_NSTATE, np.float32)
        check(self.L.mhd_mlp_get(self.h, st.ctypes.data_as(C.c_void_p)), "mhd_mlp_get")
        return st

    def mlp_set(self, state):
        st = np.ascontiguousarray(state, np.float32)
        assert st.size == MLP_NSTATE
        check(self.L.mhd_mlp_set(self.h, st.ctypes.data_as(C.c_void_p)), "mhd_mlp_set")

    def mlp_save(self) -> bytes:
        """The network as the BF16 weight blob of mhd_mlp_save."""
        buf = (C.c_ubyte * MLP_BLOB_BYTES)()
        n = C.c_long()
        check(self.L.mhd_mlp_save(self.h, buf, MLP_BLOB_BYTES, C.byref(n)), "mhd_mlp_save")
        return bytes(buf)[:n.value]

    def mlp_load(self, blob: bytes):
        """mhd_mlp_load of a BF16 weight blob."""
        buf = (C.c_ubyte * len(blob)).from_buffer_copy(blob)
        check(self.L.mhd_mlp_load(self.h, buf, len(blob)), "mhd_mlp_load")

    def launches(self) -> int:
        return int(self.L.mhd_kernel_launches(self.h))

    def profile(self, enable: bool):
        check(self.L.mhd_profile(self.h, int(bool(enable))), "mhd_profile")

    def profile_read(self) -> dict:
        """{kernel name: (milliseconds, launches)} since the previous read."""
        ms = (C.c_double * MHD_NKERNEL)()
        n = (C.c_longlong * MHD_NKERNEL)()
        check(self.L.mhd_profile_read(self.h, ms, n), "mhd_profile_read")
        return {self.L.mhd_kernel_name(k).decode(): (ms[k], n[k]) for k in range(MHD_NKERNEL)}


class HostStepper:
    """RK steps of a block whose state (host["cons"], host["bf"][0..2]) and
    metric (host["adm"]) live in pinned host memory.  Every step copies its
    metric and its state in from the host and its state out to the host, as
    Context.step_host does, with the copies pipelined:

    - the metric of step k+1 travels into a device staging array on a side
      stream while step k runs; step k+1 moves it into the block with one
      device-to-device copy;
    - after step k the state goes out array by array (five conserved
      variables, three face fields) on a second stream, and each array comes
      back in for step k+1 on a third as soon as it has reached the host, so
      the two directions of the link overlap; step k+1 starts its metric
      kernel meanwhile and its stages wait for the state (mhd_step_overlap).

    The host state is read back as soon as it is written, so changes a caller
    makes to it between steps are not seen (use Context.step_host for that).

    step(dt, adm_next=None): one RK step; adm_next (pinned host, the shape of
    host["adm"]) is the metric of the following step, host["adm"] when None.
    join(): makes the stepper's stream wait until the last step's state has
    reached the host (for timing on that stream, or before reading the host
    state).  finish(): waits for every copy in flight."""

    def __init__(self, ctx: Context, blk: DeviceBlock, host: dict, stream=None):
        import torch
        self.ctx, self.blk, self.host = ctx, blk, host
        dev = blk.cons.device
        self.s = stream or torch.cuda.current_stream()
        self.sp = torch.cuda.Stream(device=dev)   # the metric coming in
        self.so = torch.cuda.Stream(device=dev)   # the state going out
        self.si = torch.cuda.Stream(device=dev)   # the state coming back in
        self.stage = torch.empty_like(blk.adm)
        self.ready = None      # event: the staging array holds the next step's metric
        self.free = None       # event: the step has copied the staging array out
        self.state_in = None   # event: the state of the next step is on the device
        self.out = None        # event: the last step's state is on the host
        self.pairs = [(blk.cons[v], host["cons"][v]) for v in range(5)] + \
                     [(blk.bf[d], host["bf"][d]) for d in range(3)]

    def _prefetch(self, adm_host):
        # after the staging array is free and after the current step's state
        # is in (the state's copies are on the critical path; the metric has
        # the whole step to arrive)
        import torch
        with torch.cuda.stream(self.sp):
            if self.free is not None:
                self.sp.wait_event(self.free)
            if self.state_in is not None:
                self.sp.wait_event(self.state_in)
            self.stage.copy_(adm_host, non_blocking=True)
            self.ready = torch.cuda.Event()
            self.ready.record(self.sp)

    def step(self, dt, adm_next=None):
        import torch
        if self.ready is None:
            self._prefetch(self.host["adm"])
        s, blk = self.s, self.blk
        with torch.cuda.stream(s):
            if self.state_in is None:   # the first step copies its state in here
                for dev, hst in self.pairs:
                    dev.copy_(hst, non_blocking=True)
            s.wait_event(self.ready)
            blk.adm.copy_(self.stage, non_blocking=True)
            self.free = torch.cuda.Event()
            self.free.record(s)
        self._prefetch(self.host["adm"] if adm_next is None else adm_next)
        self.ctx.step_overlap([blk], dt, stream=s, state_ready=self.state_in)
        done = torch.cuda.Event()
        done.record(s)
        evs = []
        with torch.cuda.stream(self.so):
            self.so.wait_event(done)
            for dev, hst in self.pairs:
                hst.copy_(dev, non_blocking=True)
                e = torch.cuda.Event()
                e.record(self.so)
                evs.append(e)
        self.out = evs[-1]
        with torch.cuda.stream(self.si):
            for (dev, hst), e in zip(self.pairs, evs):
                self.si.wait_event(e)
                dev.copy_(hst, non_blocking=True)
            self.state_in = torch.cuda.Event()
            self.state_in.record(self.si)

    def join(self):
        if self.out is not None:
            self.s.wait_event(self.out)

    def finish(self):
        self.sp.synchronize()
        self.so.synchronize()
        self.si.synchronize()
