"""tests/mutation_sweep.py stays runnable: every planted mistake names text
that occurs exactly once in the oracle source, and changes it."""
import os

from tests import mutation_sweep as M


def test_every_mutation_anchor_occurs_once():
    src = open(M.SRC).read()
    names = [m[0] for m in M.MUTATIONS]
    assert len(set(names)) == len(names)
    for name, a, b in M.MUTATIONS:
        assert a != b, name
        assert src.count(a) == 1, name
    assert M.EQUIVALENT <= set(names)
    assert os.path.basename(M.SRC) == "grmhd_oracle.cpp"
