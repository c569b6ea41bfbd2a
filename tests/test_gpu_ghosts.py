"""Ghost fill of the library (same-level copies and outflow) against the test
harness's numpy fills: bitwise, for the conserved variables and the three face
fields, on one periodic block, one outflow block and two blocks that tile a
periodic domain."""
import numpy as np
import pytest

import oracle as O
from paper_2409_10384_gb300 import synth
from tests import gpu_util as U
from tests.helpers import fill_ghosts

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2409_10384_gb300 import build, grmhd
    build.build()
    return grmhd


def _garbled(ob, seed):
    """A copy of ob whose ghost zones hold noise (the interior is kept)."""
    rng = np.random.default_rng(seed)
    b = ob.copy()
    g = b.ng
    n1, n2, n3 = b.n
    keep = b.cons[:, g:g + n3, g:g + n2, g:g + n1].copy()
    b.cons[...] = rng.normal(size=b.cons.shape)
    b.cons[:, g:g + n3, g:g + n2, g:g + n1] = keep
    for d in range(3):
        sl = [slice(g, g + n3), slice(g, g + n2), slice(g, g + n1)]
        sl[2 - d] = slice(g, g + b.n[d] + 1)
        keep = b.bf[d][tuple(sl)].copy()
        b.bf[d][...] = rng.normal(size=b.bf[d].shape)
        b.bf[d][tuple(sl)] = keep
    return b


def _check(G, blocks_np, expect, nbr):
    ctx = G.Context(G.params())
    dbs = [U.to_device(G, b) for b in blocks_np]
    ctx.fill_ghosts(dbs, nbr)
    for db, ex in zip(dbs, expect):
        got = U.from_device(db)
        assert np.array_equal(got["cons"], ex.cons)
        for d in range(3):
            assert np.array_equal(got["bf"][d], ex.bf[d]), d


@pytest.mark.parametrize("mode", ["periodic", "outflow"])
def test_single_block(G, mode):
    p = O.params()
    inp = synth.periodic_flat(seed=1, n=16)
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    b = _garbled(ob, 5)
    ex = b.copy()
    fill_ghosts(ex, (mode,) * 3)
    _check(G, [b], [ex], np.full((1, 6), 0 if mode == "periodic" else -1))


def test_two_blocks_tile_a_periodic_domain(G):
    """Blocks A (x in [0, n)) and B (x in [n, 2n)) of a periodic 2n x n x n
    domain: A's x neighbours on both sides are B and vice versa; y and z wrap
    onto the block itself."""
    p = O.params()
    n, g = 8, 4
    rng = np.random.default_rng(7)
    big = O.new_block((2 * n, n, n), g, (1.0, 1.0, 1.0), np.zeros((16, n + 2 * g, n + 2 * g, 2 * n + 2 * g)))
    big.cons = rng.normal(size=(5, n + 2 * g, n + 2 * g, 2 * n + 2 * g))
    big.bf = [rng.normal(size=big.face_shape(d)) for d in range(3)]
    ref = big.copy()
    fill_ghosts(ref)
    blocks, expect = [], []
    for ix in range(2):
        x0 = ix * n
        adm = np.zeros((16, n + 2 * g, n + 2 * g, n + 2 * g))
        b = O.new_block((n, n, n), g, (1.0, 1.0, 1.0), adm)
        e = O.new_block((n, n, n), g, (1.0, 1.0, 1.0), adm)
        b.cons = np.ascontiguousarray(big.cons[..., x0:x0 + n + 2 * g])
        e.cons = np.ascontiguousarray(ref.cons[..., x0:x0 + n + 2 * g])
        b.bf = [np.ascontiguousarray(big.bf[0][..., x0:x0 + n + 2 * g + 1])] + \
               [np.ascontiguousarray(big.bf[d][..., x0:x0 + n + 2 * g]) for d in (1, 2)]
        e.bf = [np.ascontiguousarray(ref.bf[0][..., x0:x0 + n + 2 * g + 1])] + \
               [np.ascontiguousarray(ref.bf[d][..., x0:x0 + n + 2 * g]) for d in (1, 2)]
        b.cons0 = b.cons.copy()
        b.bf0 = [x.copy() for x in b.bf]
        blocks.append(b)
        expect.append(e)
    nbr = np.array([[1, 1, 0, 0, 0, 0], [0, 0, 1, 1, 1, 1]], np.int32)
    _check(G, blocks, expect, nbr)


def test_mixed_outflow_and_periodic_sides(G):
    """Outflow along x, periodic along y and z, on a block thinner than its
    ghost depth across (4 ghosts, 2 and 1 cells): the edges and corners
    combine the rules of their sides, as the harness's axis-by-axis fill."""
    p = O.params()
    inp = synth.balsara_tube(1, 16, ny=2)
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    b = _garbled(ob, 11)
    ex = b.copy()
    fill_ghosts(ex, ("outflow", "periodic", "periodic"))
    _check(G, [b], [ex], np.array([[-1, -1, 0, 0, 0, 0]], np.int32))


def test_untouched_sides(G):
    """-2 leaves the ghosts of a side as they were: with both z sides at -2,
    the x and y passes still fill their ghosts in every z layer."""
    p = O.params()
    inp = synth.periodic_flat(seed=2, n=8)
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    b = _garbled(ob, 9)
    ex = b.copy()
    fill_ghosts(ex, ("periodic", "periodic", "none"))
    _check(G, [b], [ex], np.array([[0, 0, 0, 0, -2, -2]], np.int32))
