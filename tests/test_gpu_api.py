"""Entry points of the C-ABI not covered by the parity files: pinned launch
shapes, the per-kernel profile, the network state round trip, the captured
step entry point, the con2prim counters out-argument and the BF16 weight
blob."""
import numpy as np
import pytest

import oracle as O
from paper_2409_10384_gb300 import synth
from tests import gpu_util as U
import tests.test_gpu_parity as T

pytestmark = pytest.mark.gpu

G = T.G


def _star(G, p, sub=16, corner=(56, 56, 56)):
    inp = synth.star_subblock(sub=sub, corner=corner)
    ob = O.init_block(p, inp.n, inp.ng, inp.dx, inp.adm, inp.prim, inp.A)
    return inp, ob


def test_pinned_launch_shapes_are_bit_identical(G):
    """Every tunable kernel pinned to other CTA sizes and waves gives the same
    bits as the default shapes; get_launch reads back what set_launch pinned;
    out-of-range shapes are rejected."""
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=2, rsolver=1, rk_order=3, fofc=1)
    inp, ob = _star(G, p)
    dt = 0.25 * inp.dx[0]
    ctx = T._ctx(G, p)
    a = U.to_device(G, ob)
    ctx.step([a], dt)
    ref = U.from_device(a)
    ctx2 = T._ctx(G, p)
    for k, (th, wv) in zip(G.Context.TUNABLE, [(64, 1), (256, 2), (64, 3), (256, 1), (128, 4), (64, 2),
                                                (256, 3), (128, 1), (256, 4)]):
        ctx2.set_launch(k, th, wv)
        assert ctx2.get_launch(k) == (th, wv)
    b = U.to_device(G, ob)
    ctx2.step([b], dt)
    got = U.from_device(b)
    for key in ("cons", "prim", "flags"):
        assert np.array_equal(got[key], ref[key]), key
    for d in range(3):
        assert np.array_equal(got["bf"][d], ref["bf"][d])
    for bad in ((96, 1), (128, 0), (128, 65)):
        with pytest.raises(RuntimeError):
            ctx2.set_launch("flux_x", *bad)


def test_profile_counts_every_launch(G):
    """Per-kernel CUDA-event profile: one entry per launch of the stage, the
    launch total matching the context's counter, positive times."""
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=2, rsolver=1, rk_order=3, fofc=1)
    inp, ob = _star(G, p)
    ctx = T._ctx(G, p)
    a = U.to_device(G, ob)
    ctx.step([a], 0.25 * inp.dx[0])    # first call: list set-up outside the profile
    ctx.profile(True)
    ctx.profile_read()
    l0 = ctx.launches()
    ctx.step([a], 0.25 * inp.dx[0])
    prof = ctx.profile_read()
    ctx.profile(False)
    n = sum(v[1] for v in prof.values())
    assert n == ctx.launches() - l0
    # per RK3 step: one launch per stage, the con2prim's prep and finish two
    for name, k in (("flux_x", 3), ("flux_y", 3), ("flux_z", 3), ("c2p", 6), ("update", 3), ("emf", 3)):
        assert prof[name][1] == k and prof[name][0] > 0.0, (name, prof[name])


def test_network_state_round_trip(G):
    """mlp_get / mlp_set carry the trained network (weights, normalisation,
    bracket width) to another context: the same inference bits."""
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-20, T_atm=1e-14, f_thr=0.0)
    kw = {k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"}
    a = G.Context(G.params(**kw))
    prim, Bd, g = synth.c2p_stress(20000, seed=31)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    cons = torch.zeros((5, prim.shape[1]), dtype=torch.float64, device="cuda")
    a.prim2cons(t(prim), t(Bd), t(g), cons)
    feat, logmu = a.mlp_dataset(cons, t(Bd), t(g))
    a.mlp_init(5)
    a.mlp_train(feat, logmu, epochs=2, batch=2048, lr=3e-3)
    st = a.mlp_get()
    b = G.Context(G.params(**kw))
    b.mlp_set(st)
    assert np.array_equal(b.mlp_get(), st)
    assert torch.equal(a.mlp_infer(feat), b.mlp_infer(feat))


def test_graph_step_entry_point_equals_ungraphed_step(G):
    """mhd_graph_step (the captured full RK step) gives the bits of mhd_step
    without a graph, on two calls (capture, then replay)."""
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=2, rsolver=1, rk_order=3, fofc=1)
    inp, ob = _star(G, p)
    dt = 0.25 * inp.dx[0]
    ctx = T._ctx(G, p)
    a = U.to_device(G, ob)
    b = U.to_device(G, ob)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for _ in range(2):
            ctx.step([a], dt, stream=s)
            ctx.graph_step([b], dt, s)
    s.synchronize()
    ga, gb = U.from_device(a), U.from_device(b)
    for key in ("cons", "prim", "flags"):
        assert np.array_equal(ga[key], gb[key]), key
    for d in range(3):
        assert np.array_equal(ga["bf"][d], gb["bf"][d])


def test_c2p_stats_out_argument(G):
    """The mhd_stats out-argument of mhd_c2p and mhd_c2p_cells holds the
    counters the call added, as read_stats differences show them."""
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=2, rsolver=1, rk_order=3, fofc=1)
    inp, ob = _star(G, p, corner=(100, 56, 56))   # over the surface: floors fire
    ctx = T._ctx(G, p)
    a = U.to_device(G, ob)
    before = ctx.read_stats()
    st = ctx.c2p([a], stats=True)
    after = ctx.read_stats()
    assert st == {k: after[k] - before[k] for k in st}
    assert st["cells"] == 22 ** 3 and st["floors"] > 0
    prim, Bd, g = synth.c2p_stress(3000, seed=9)
    q = O.params(gamma=2.0, rho_atm=1e-20, T_atm=1e-14, f_thr=0.0)
    c2 = T._ctx(G, q)
    t = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    cons = torch.zeros((5, 3000), dtype=torch.float64, device="cuda")
    c2.prim2cons(t(prim), t(Bd), t(g), cons)
    pr = torch.zeros_like(cons)
    fl = torch.zeros(3000, dtype=torch.uint8, device="cuda")
    it = torch.zeros(3000, dtype=torch.int32, device="cuda")
    st = c2.c2p_cells(cons, t(Bd), t(g), pr, fl, it, stats=True)
    assert st["cells"] == 3000 and st["iters"] == int(it.sum().item())
    st0 = c2.c2p_cells(cons[:, :0], t(Bd)[:, :0], t(g)[:, :0], pr[:, :0], fl[:0], None, stats=True)
    assert all(v == 0 for v in st0.values())


def test_network_bf16_blob_round_trip(G):
    """mhd_mlp_save / mhd_mlp_load: the BF16 weight blob carries the network
    to another context, which infers what a context holding the same
    bf16-rounded parameters infers, and saves the same bytes again."""
    import torch
    from oracle import mlp as M
    rng = np.random.default_rng(11)
    a = G.Context(G.params())
    st = np.zeros(G.MLP_NSTATE, np.float32)
    st[:M.NPARAM] = rng.normal(size=M.NPARAM) * 0.2
    st[M.NPARAM:M.NPARAM + 5] = rng.normal(size=5)
    st[M.NPARAM + 5:M.NPARAM + 10] = 0.5 + rng.random(5)
    st[M.NPARAM + 10:M.NPARAM + 13] = (-1.5, 2.0, 0.05)
    a.mlp_set(st)
    blob = a.mlp_save()
    assert len(blob) == G.MLP_BLOB_BYTES
    b = G.Context(G.params())
    b.mlp_load(blob)
    assert b.mlp_save() == blob
    rounded = st.copy()
    rounded[:M.NPARAM] = M.bf16_round(st[:M.NPARAM]).astype(np.float32)
    c = G.Context(G.params())
    c.mlp_set(rounded)
    feat = torch.from_numpy(rng.normal(size=(777, 8)).astype(np.float32)).cuda()
    assert torch.equal(b.mlp_infer(feat), c.mlp_infer(feat))
    assert np.array_equal(b.mlp_get(), rounded)
    with pytest.raises(RuntimeError):
        b.mlp_load(blob[:-1])


def test_fast_reciprocal_within_two_ulp_of_the_division(G):
    """The reciprocal the hot divisions use (approximation refined by two
    Newton-Raphson steps) against CUDA's correctly rounded division, on
    log-uniform values over the normal range of both signs, powers of two and
    their neighbours: within 2^-51 relative (two units in the last place)."""
    import torch
    rng = np.random.default_rng(21)
    x = np.concatenate([10.0 ** rng.uniform(-280, 280, 400000) * rng.choice([-1.0, 1.0], 400000),
                        2.0 ** np.arange(-900, 901, dtype=np.float64),
                        np.nextafter(2.0 ** np.arange(-300, 301, dtype=np.float64), 0.0),
                        np.nextafter(2.0 ** np.arange(-300, 301, dtype=np.float64), np.inf),
                        np.array([1.0, 3.0, 6.0, 7.0, 1.0 / 3.0, 127.9999, 1e-280, 1e280])])
    d = G.check_rcp(torch.from_numpy(np.ascontiguousarray(x)).cuda()).cpu().numpy()
    assert np.all(np.isfinite(d))
    assert d.max() <= 2.0 ** -51, float(d.max())


def test_host_stepper_equals_step_host(G):
    """The pipelined host stepper (next metric copied in on a side stream while
    the step runs, the state out and back in array by array while the next
    step's metric kernel runs) gives the same bits as step_host over three RK3
    steps, with the metric changing between steps (each step's own metric
    arrives)."""
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=2, rsolver=1, rk_order=3, fofc=1)
    inp, ob = _star(G, p)
    dt = 0.25 * inp.dx[0]

    def host_of(db):
        h = {"cons": db.cons.cpu().pin_memory(), "adm": db.adm.cpu().pin_memory(),
             "bf": [x.cpu().pin_memory() for x in db.bf]}
        return h

    # three metrics: the block's, and two perturbed lapses (the step reads all 16 slots)
    base = torch.from_numpy(np.ascontiguousarray(inp.adm))
    adms = [base.clone().pin_memory()]
    for k in (1, 2):
        a = base.clone()
        a[0] *= 1.0 + 1e-3 * k
        adms.append(a.pin_memory())
    s = torch.cuda.Stream()
    ctx = T._ctx(G, p)
    a = U.to_device(G, ob)
    ha = host_of(a)
    for k in range(3):
        s.synchronize()   # the previous step's copy out of ha["adm"] has run
        ha["adm"].copy_(adms[k])
        ctx.step_host(a, ha, dt, s)
    s.synchronize()
    ctx2 = T._ctx(G, p)
    b = U.to_device(G, ob)
    hb = host_of(b)
    hb["adm"] = adms[0]
    st = ctx2.host_stepper(b, hb, stream=s)
    for k in range(3):
        st.step(dt, adm_next=adms[k + 1] if k + 1 < 3 else adms[0])
    s.synchronize()
    st.finish()
    assert torch.equal(ha["cons"], hb["cons"])
    for d in range(3):
        assert torch.equal(ha["bf"][d], hb["bf"][d])
    assert torch.equal(b.adm.cpu(), adms[2])


def test_fixed_metric_reuses_the_cache(G):
    """mhd_params.fixed_metric (a fixed spacetime, the Cowling runs of Sec.
    4.4): three RK3 steps, direct and graphed, give the bits of ordinary steps
    with the ADM arrays unchanged; after the first step each step launches one
    kernel fewer (no metric kernel), and a new block list computes the metric
    again."""
    import torch
    p = O.params(gamma=2.0, rho_atm=1e-12, T_atm=1e-10, f_thr=0.1, recon=2, rsolver=1, rk_order=3, fofc=1)
    kw = {k: getattr(p, k) for k, _ in p._fields_ if k != "pad_"}
    inp, ob = _star(G, p)
    dt = 0.25 * inp.dx[0]
    s = torch.cuda.Stream()
    ref = G.Context(G.params(**kw))
    a = U.to_device(G, ob)
    for _ in range(3):
        ref.step([a], dt, stream=s)
    s.synchronize()
    for graph in (False, True):
        ctx = G.Context(G.params(**kw, fixed_metric=1))
        b = U.to_device(G, ob)
        n = []
        for _ in range(3):
            l0 = ctx.launches()
            ctx.step([b], dt, graph=graph, stream=s)
            n.append(ctx.launches() - l0)
        s.synchronize()
        assert torch.equal(a.cons, b.cons), graph
        for d in range(3):
            assert torch.equal(a.bf[d], b.bf[d]), graph
        assert n[1] == n[2] == n[0] - 1, (graph, n)
        # another block list, then the first again: each computes its metric
        c = U.to_device(G, ob)
        l0 = ctx.launches()
        ctx.step([c], dt, graph=graph, stream=s)
        assert ctx.launches() - l0 == n[0], graph
        l0 = ctx.launches()
        ctx.step([b], dt, graph=graph, stream=s)
        assert ctx.launches() - l0 == n[0], graph
        s.synchronize()
