"""The oracle's single-face flux and its flux override (test infrastructure
for taking a reconstruction tie down its other branch): the face flux from
the stage's primitives is the flux the stage itself computes, bit for bit; an
override with the stage's own fluxes changes nothing; an override of one face
changes exactly the two cells that share it, and face fields only next to it."""
import numpy as np
import pytest

import oracle as O
from paper_2409_10384_gb300 import synth


@pytest.fixture(scope="module")
def setup():
    O.build()
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=2, rsolver=1, rk_order=3, fofc=1)
    inp = synth.star_subblock(sub=8, corner=(56, 56, 56))
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    return p, ob, 0.25 * inp.dx[0]


def test_face_flux_at_is_the_stage_flux(setup):
    p, ob, dt = setup
    ref = ob.copy()
    out = O.stage(p, ref, dt, 0, keep=True)
    b = ob.copy()
    O.c2p_block(p, b)
    ng = ob.ng
    for d, face in ((0, (ng + 2, ng + 3, ng)), (1, (ng + 1, ng + 8, ng + 4)), (2, (ng + 5, ng + 2, ng + 7)),
                    (0, (ng - 1, ng + 8, ng + 8))):
        F = O.face_flux_at(p, b, d, face)
        assert np.array_equal(F, out["flux"][d][(slice(None),) + face]), (d, face)
    with pytest.raises(ValueError):
        O.face_flux_at(p, b, 0, (ng, ng, 2))


def test_override_with_own_flux_is_identity_and_one_face_moves_its_cells(setup):
    p, ob, dt = setup
    ref = ob.copy()
    out = O.stage(p, ref, dt, 0, keep=True)
    ng = ob.ng
    face = (ng + 3, ng + 4, ng + 5)   # x face between cells i = ng+4 and ng+5
    F = out["flux"][0][(slice(None),) + face].copy()
    same = ob.copy()
    O.stage(p, same, dt, 0, override=[((0,) + face, F)])
    assert np.array_equal(same.cons, ref.cons)
    for d in range(3):
        assert np.array_equal(same.bf[d], ref.bf[d])
    moved = ob.copy()
    F2 = F * (1.0 + 1e-6)
    O.stage(p, moved, dt, 0, override=[((0,) + face, F2)])
    k, j, i = face
    diff = np.argwhere(np.any(moved.cons != ref.cons, axis=0))
    assert {tuple(x) for x in diff} == {(k, j, i - 1), (k, j, i)}
    # face B~ moves only through the EMFs of the four edges of that face: on
    # faces whose low corner lies within one cell of it
    for d in range(3):
        ch = np.argwhere(moved.bf[d] != ref.bf[d])
        assert len(ch) > 0, d
        assert np.all(np.abs(ch - np.array(face)) <= 1), (d, ch)
