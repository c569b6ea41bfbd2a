"""Test-side harness: ghost fills, block set-up from face fields, error measures.

These are index copies and comparisons only (no method arithmetic)."""
import numpy as np


def interior(b):
    ng = b.ng
    n1, n2, n3 = b.n
    return (slice(ng, ng + n3), slice(ng, ng + n2), slice(ng, ng + n1))


def _fill_axis(a, axis, n, ng, mode, stag):
    if mode == "none":
        return
    a_ = np.moveaxis(a, axis, -1)
    if mode == "periodic":
        # every ghost index takes the interior index congruent modulo n (any n)
        L = a_.shape[-1]
        idx = np.arange(L)
        if stag:
            ghost = (idx < ng) | (idx > n + ng)
        else:
            ghost = (idx < ng) | (idx >= n + ng)
        src = ng + np.mod(idx - ng, n)
        a_[..., ghost] = a_[..., src[ghost]]
    else:  # outflow: copy the edge value outward
        if stag:
            a_[..., :ng] = a_[..., ng:ng + 1]
            a_[..., n + ng + 1:] = a_[..., n + ng:n + ng + 1]
        else:
            a_[..., :ng] = a_[..., ng:ng + 1]
            a_[..., n + ng:] = a_[..., n + ng - 1:n + ng]


def fill_ghosts(b, modes=("periodic", "periodic", "periodic")):
    """Refresh ghost cons and face B~ (numpy blocks, layout [..][k][j][i])."""
    for ax in range(3):
        axis = 2 - ax  # array axis of direction ax in a [k][j][i] array
        _fill_axis(b.cons, axis + 1, b.n[ax], b.ng, modes[ax], False)
        for d in range(3):
            _fill_axis(b.bf[d], axis, b.n[ax], b.ng, modes[ax], d == ax)


def rel_err(a, b, floor_frac=1e-10):
    """max over cells of |a-b| / max(|b|, floor_frac * max|b|) for one field."""
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    s = max(np.abs(b).max(), 1e-300) * floor_frac
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), s)))


def uniform_metric(N, alpha=1.0, beta=(0.0, 0.0, 0.0), g6=(1, 0, 0, 1, 0, 1), K6=(0, 0, 0, 0, 0, 0)):
    adm = np.zeros((16,) + tuple(N[::-1]))
    adm[0] = alpha
    for c in range(3):
        adm[1 + c] = beta[c]
    for c in range(6):
        adm[4 + c] = g6[c]
        adm[10 + c] = K6[c]
    return adm


def init_from_faces(O, p, n, ng, dx, adm, prim, bf):
    """Block from primitives and given face fields (cons via the oracle's Eq. 6)."""
    b = O.new_block(n, ng, dx, adm)
    for d in range(3):
        b.bf[d][...] = bf[d]
    O.bcc(p, b)
    b.prim[...] = prim
    nc = b.prim[0].size
    b.cons[...] = O.prim2cons(p, b.prim.reshape(5, nc), b.bcc.reshape(3, nc),
                              np.ascontiguousarray(b.adm[4:10].reshape(6, nc))).reshape(b.cons.shape)
    return b
