"""The algorithmic FP64 operation counts per unit that bench.py uses for the
roofline are re-derived here with the op-counting build of the oracle on
sub-blocks of the 128^3 star workload (core, surface, atmosphere)."""
import numpy as np

import bench
import oracle as O
from paper_2409_10384_gb300 import synth


def test_flops_per_unit_match_counting_oracle():
    p = O.params(**bench.PARAMS)
    n = 16
    acc = {k: [] for k in O.PHASES}
    for corner in [(52, 52, 52), (104, 52, 52), (90, 90, 90)]:
        inp = synth.star_subblock(sub=n, corner=corner)
        b = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
        ph = O.flop_phases(p, b, bench.CFL * inp.dx[0], 0)
        units = dict(c2p=(n + 6) ** 3, flux=3 * (n + 1) * (n + 2) ** 2, fofc_flag=n ** 3,
                     fofc_fix=ph["stats"]["fofc_faces"], emf=3 * (n + 1) ** 2 * n, update=n ** 3)
        for k in O.PHASES:
            if units[k] == 0:
                continue
            c = ph[k]
            acc[k].append((c["add"] + c["mul"] + c["div"] + c["sqrt"]) / units[k])
    for k, v in bench.FLOPS_PER_UNIT.items():
        got = float(np.mean(acc[k]))
        assert abs(got - v) <= 0.15 * v, (k, got, v)
    # flux count is data independent to within the face floors
    assert np.ptp(acc["flux"]) < 0.01 * np.mean(acc["flux"])
