"""Host-side checks of the C-ABI library (no GPU compute): it builds, loads and
exports every entry point that include/grmhd.h declares; host-side argument
validation rejects bad input before any device work."""
import ctypes as C

import numpy as np

import pytest

from paper_2409_10384_gb300 import build, grmhd


@pytest.fixture(scope="module")
def L():
    build.build()
    return grmhd.lib()


def test_exports_every_declared_symbol(L):
    names = grmhd.header_symbols()
    assert len(names) >= 14
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(grmhd._SIGS)


def test_strerror_names_every_code(L):
    for code in (0, -1, -2, -3, -4, -5):
        assert L.mhd_strerror(code).decode() == grmhd._ERR[code]
    assert L.mhd_strerror(-99).decode() == "unknown error"


def test_null_and_bad_arguments_rejected_without_device(L):
    h = C.c_void_p()
    assert L.mhd_init(None, C.byref(h)) == -1
    p = grmhd.params(gamma=0.5)
    assert L.mhd_init(C.byref(p), C.byref(h)) == -1
    p = grmhd.params(rk_order=4)
    assert L.mhd_init(C.byref(p), C.byref(h)) == -1
    p = grmhd.params(dmp_M=0.5)
    assert L.mhd_init(C.byref(p), C.byref(h)) == -1
    p = grmhd.params(fixed_metric=2)
    assert L.mhd_init(C.byref(p), C.byref(h)) == -1
    # hybrid EOS: pieces out of range, non-increasing dividing densities, a
    # thermal index <= 1, and the FP32 root searches (ideal gas only)
    for kw in (dict(eos_pieces=0), dict(eos_pieces=5), dict(eos_rho=(1e-4, 1e-8, 0.0)),
               dict(eos_gamma_th=1.0), dict(eos_K0=-1.0), dict(c2p_guess=1), dict(c2p_guess=2), dict(eos=2)):
        d = dict(eos=1, eos_pieces=3, eos_K0=1e-4, eos_gamma_th=1.8, eos_rho=(1e-8, 1e-4, 0.0),
                 eos_gamma=(1.7, 2.4, 2.1, 0.0))
        d.update(kw)
        p = grmhd.params(gamma=2.0, **d)
        assert L.mhd_init(C.byref(p), C.byref(h)) == -1, kw
    assert L.mhd_c2p(None, None, 0, None, None) == -1
    assert L.mhd_c2p_cells(None, 1, None, None, None, None, None, None, None, None) == -1
    assert L.mhd_step(None, None, 1, 0.1, 0, None) == -1
    assert L.mhd_graph_step(None, None, 1, 0.1, None) == -1
    assert L.mhd_mlp_load(None, None, grmhd.MLP_BLOB_BYTES) == -1
    assert L.mhd_mlp_save(None, None, 0, None) == -1
    assert L.mhd_kernel_launches(None) == 0


def test_blob_size_matches_header():
    import re
    h = open(grmhd._build.ROOT + "/include/grmhd.h").read()
    m = re.search(r"#define MHD_MLP_BLOB_BYTES \((\d+) \* (\d+) \+ (\d+) \* (\d+)\)", h)
    assert m, "MHD_MLP_BLOB_BYTES"
    a, b, c, d = (int(x) for x in m.groups())
    assert a * b + c * d == grmhd.MLP_BLOB_BYTES == 2 * grmhd.MLP_NPARAM + 4 * (grmhd.MLP_NSTATE - grmhd.MLP_NPARAM)


def test_struct_layouts_match_header():
    # mhd_params: 9 doubles + 8 ints + 9 doubles (EOS) + one int (fixed_metric) padded to 8;
    # mhd_block: 3+1 ints, 3 doubles, 12 pointers; mhd_stats: MHD_NSTATS int64
    import re
    h = open(grmhd._build.ROOT + "/include/grmhd.h").read()
    nst = int(re.search(r"#define MHD_NSTATS (\d+)", h).group(1))
    assert C.sizeof(grmhd.mhd_params) == 9 * 8 + 8 * 4 + 9 * 8 + 8
    assert C.sizeof(grmhd.mhd_block) == 16 + 24 + 12 * 8
    assert C.sizeof(grmhd.mhd_stats) == nst * 8 == 10 * 8


def test_block_list_cache_follows_device_pointers():
    """The binding's descriptor cache must follow the arrays, not Python object
    ids: a block freed and replaced by a new one (which CPython may give the
    same id) has to be described by the new block's pointers."""
    import torch
    from paper_2409_10384_gb300 import grmhd as G
    ctx = G.Context.__new__(G.Context)   # the cache logic alone; no library context
    ctx._arr, ctx._key, ctx._held = None, None, []
    adm = np.zeros((16, 10, 10, 10))
    for _ in range(20):
        b = G.DeviceBlock((2, 2, 2), 4, (1.0, 1.0, 1.0), adm, device="cpu")
        arr, nb = ctx._blocks([b])
        assert nb == 1
        assert arr[0].cons == b.cons.data_ptr() and arr[0].prim == b.prim.data_ptr()
        assert arr[0].bf[2] == b.bf[2].data_ptr() and arr[0].flags == b.flags.data_ptr()
        b.cons = torch.zeros_like(b.cons)   # replaced array inside a live block
        arr, _ = ctx._blocks([b])
        assert arr[0].cons == b.cons.data_ptr()
        del b
