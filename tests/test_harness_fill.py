"""The test harness's numpy ghost fill (tests/helpers.fill_ghosts), which the
GPU ghost-fill tests compare against bit for bit, pinned to its definition on
integer labels: a cell (face) takes the label of the interior index its axis
rule maps it to, periodic (the congruent index modulo n, any n) or outflow
(the nearest interior index; faces along their own axis up to n), combined
axis by axis, so edges and corners take the label of the mapped triple."""
import itertools
import types

import numpy as np
import pytest

from tests.helpers import fill_ghosts


def _map(idx, n, ng, mode, stag):
    top = n + ng if stag else n + ng - 1      # last interior index
    if mode == "periodic":
        if ng <= idx <= top:
            return idx
        return ng + (idx - ng) % n
    if mode == "outflow":
        return min(max(idx, ng), top)
    return idx                                # "none": untouched


def _label(i, j, k):
    return i + 100 * j + 10000 * k


@pytest.mark.parametrize("modes", list(itertools.product(("periodic", "outflow"), repeat=3)) +
                         [("periodic", "periodic", "none")])
def test_fill_matches_its_definition(modes):
    n, ng = (5, 3, 2), 4
    N = [x + 2 * ng for x in n]
    rng = np.random.default_rng(3)
    b = types.SimpleNamespace(n=n, ng=ng)
    shapes = [(N[2], N[1], N[0] + 1), (N[2], N[1] + 1, N[0]), (N[2] + 1, N[1], N[0])]

    def labels(shape, stag_axis):
        out = np.empty(shape)
        for k, j, i in itertools.product(*(range(s) for s in shape)):
            out[k, j, i] = _label(i, j, k)
        return out

    def expected(shape, stag_axis):
        out = np.empty(shape)
        for k, j, i in itertools.product(*(range(s) for s in shape)):
            m = [_map(x, n[a], ng, modes[a], a == stag_axis) for a, x in enumerate((i, j, k))]
            out[k, j, i] = _label(*m)
        return out

    def interior_mask(shape, stag_axis):
        keep = np.ones(shape, bool)
        for a in range(3):
            top = n[a] + ng + (1 if a == stag_axis else 0)
            idx = np.arange(shape[2 - a])
            inside = (idx >= ng) & (idx < top)
            keep &= inside.reshape([-1 if ax == 2 - a else 1 for ax in range(3)])
        return keep

    cell = labels((N[2], N[1], N[0]), -1)
    b.cons = np.stack([cell + 0.5 * v for v in range(5)])
    b.bf = [labels(shapes[d], d) for d in range(3)]
    # noise in every ghost (the interior keeps its labels)
    m = interior_mask(cell.shape, -1)
    for v in range(5):
        b.cons[v][~m] = rng.normal(size=(~m).sum())
    for d in range(3):
        md = interior_mask(shapes[d], d)
        b.bf[d][~md] = rng.normal(size=(~md).sum())
    if "none" in modes:   # untouched sides keep their labels
        b.cons = np.stack([cell + 0.5 * v for v in range(5)])
        b.bf = [labels(shapes[d], d) for d in range(3)]
    fill_ghosts(b, modes)
    ex = expected(cell.shape, -1)
    for v in range(5):
        assert np.array_equal(b.cons[v], ex + 0.5 * v), (modes, v)
    for d in range(3):
        assert np.array_equal(b.bf[d], expected(shapes[d], d)), (modes, d)
