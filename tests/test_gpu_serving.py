"""Serving (bc_submit / bc_poll / bc_cancel): continuous batching of concurrent
queries. Every query's result must be bit-identical to the same query run alone
through the synchronous entry points, and to the CPU oracle."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1608_04472_gb300 as p
    return p


@pytest.fixture(scope="module")
def ctx(pkg):
    c = pkg.Context(0, batch_width=64)
    yield c
    c.close()


@pytest.fixture(scope="module")
def graphs(ctx):
    er = gg.erdos_renyi(2000, 8, 1)
    ba = gg.barabasi_albert(3000, 3, 4)
    hs = {"er": ctx.load_graph(er.row_ptr, er.col), "ba": ctx.load_graph(ba.row_ptr, ba.col)}
    yield {"er": er, "ba": ba}, hs


def _same(a, b, what):
    assert np.array_equal(np.asarray(a), np.asarray(b)), what


def _mixed_queries(pkg, g):
    er, ba = g
    return [
        ("er", pkg.BC_QUERY_SOURCES, dict(targets=gg.uniform_targets(er.n, 16, 1), c=5.0, cap=20000, seed=1, qid=1)),
        ("er", pkg.BC_QUERY_SOURCES, dict(targets=gg.uniform_targets(er.n, 3, 9), c=2.0, cap=700, seed=4, qid=2)),
        ("er", pkg.BC_QUERY_SOURCES, dict(targets=[0, 1, 2, 3], c=1e9, cap=130, seed=5, qid=3)),
        ("ba", pkg.BC_QUERY_SOURCES, dict(targets=gg.degree_targets(ba, 8, 2), c=3.0, cap=5000, seed=6, qid=4)),
        ("ba", pkg.BC_QUERY_PAIRS, dict(targets=gg.degree_targets(ba, 4, 3), c=1.0, cap=500, seed=7, qid=5)),
        ("ba", pkg.BC_QUERY_PAIRS, dict(targets=[0, 1], c=1.0, cap=300, seed=8, qid=6, threshold_scale=float(ba.n - 1))),
        ("er", pkg.BC_QUERY_UNIFORM, dict(k=150, seed=9, qid=7)),
    ]


def _sync(ctx, h, kind, kw, pkg):
    if kind == pkg.BC_QUERY_SOURCES:
        return ctx.adaptive_sources(h, kw["targets"], kw["c"], kw["cap"], kw["seed"], kw["qid"])
    if kind == pkg.BC_QUERY_PAIRS:
        return ctx.adaptive_pairs(h, kw["targets"], kw["c"], kw["cap"], kw["seed"], kw["qid"],
                                  kw.get("threshold_scale", 1.0))
    return dict(est=ctx.uniform_sources(h, kw["k"], kw["seed"], kw["qid"]))


def test_concurrent_queries_match_synchronous(ctx, graphs, pkg):
    g, hs = graphs
    qs = _mixed_queries(pkg, (g["er"], g["ba"]))
    tickets = [ctx.submit(hs[name], kind, **kw) for name, kind, kw in qs]
    for tk in tickets:
        assert ctx.poll(tk, -1) == pkg.BC_OK
    for (name, kind, kw), tk in zip(qs, tickets):
        ref = _sync(ctx, hs[name], kind, kw, pkg)
        out = tk.outputs()
        for key in out:
            _same(out[key], ref[key], f"{name} kind={kind} {key}")
        st = tk.stats_dict()
        assert st["samples"] >= 1 and st["batches"] >= 1


def test_alone_vs_mix_bit_identical(ctx, graphs, pkg):
    g, hs = graphs
    kw = dict(targets=gg.uniform_targets(g["er"].n, 12, 33), c=4.0, cap=9000, seed=3, qid=99)
    alone = ctx.submit(hs["er"], pkg.BC_QUERY_SOURCES, **kw)
    ctx.poll(alone, -1)
    others = [ctx.submit(hs["er"], pkg.BC_QUERY_SOURCES, targets=gg.uniform_targets(g["er"].n, 5, 100 + i),
                         c=2.0 + i, cap=3000, seed=50 + i, qid=i) for i in range(5)]
    mixed = ctx.submit(hs["er"], pkg.BC_QUERY_SOURCES, **kw)
    for tk in others + [mixed]:
        ctx.poll(tk, -1)
    for key in ["est", "k", "S", "status"]:
        _same(alone.outputs()[key], mixed.outputs()[key], key)
    assert mixed.stats_dict()["batches"] >= 1


def test_serving_matches_oracle(ctx, graphs, pkg):
    g, hs = graphs
    targets = gg.uniform_targets(g["er"].n, 6, 77)
    tk = ctx.submit(hs["er"], pkg.BC_QUERY_SOURCES, targets=targets, c=3.0, cap=4000, seed=2, qid=8)
    ctx.poll(tk, -1)
    ref = oracle.adaptive_sources(g["er"], targets, 3.0, 4000, 2, 8)
    for key in ["est", "k", "S", "status"]:
        _same(tk.outputs()[key], ref[key], key)


def test_cancel(ctx, graphs, pkg):
    g, hs = graphs
    tk = ctx.submit(hs["er"], pkg.BC_QUERY_SOURCES, targets=[5], c=1e15, cap=1 << 30, seed=1, qid=1)
    time.sleep(0.05)
    assert ctx.poll(tk, 0) == pkg.BC_PENDING
    ctx.cancel(tk)
    with pytest.raises(pkg.BCError) as e:
        ctx.poll(tk, -1)
    assert e.value.code == -7


def test_admission_limits(ctx, graphs, pkg):
    g, hs = graphs
    ctx.server_limits(max_active=2)
    try:
        qs = [dict(targets=gg.uniform_targets(g["er"].n, 4, 200 + i), c=2.0, cap=2000, seed=10 + i, qid=i)
              for i in range(6)]
        tks = [ctx.submit(hs["er"], pkg.BC_QUERY_SOURCES, **kw) for kw in qs]
        for tk in tks:
            ctx.poll(tk, -1)
        for kw, tk in zip(qs, tks):
            ref = ctx.adaptive_sources(hs["er"], kw["targets"], kw["c"], kw["cap"], kw["seed"], kw["qid"])
            for key in ["est", "k", "S", "status"]:
                _same(tk.outputs()[key], ref[key], key)
    finally:
        ctx.server_limits(max_active=64)


def test_graph_in_use_and_bad_submissions(ctx, graphs, pkg):
    g, hs = graphs
    er = g["er"]
    h = ctx.load_graph(er.row_ptr, er.col)
    tk = ctx.submit(h, pkg.BC_QUERY_SOURCES, targets=[1, 2], c=1e15, cap=1 << 30, seed=1, qid=1)
    with pytest.raises(pkg.BCError):
        ctx.free_graph(h)
    ctx.cancel(tk)
    with pytest.raises(pkg.BCError):
        ctx.poll(tk, -1)
    ctx.free_graph(h)
    with pytest.raises(pkg.BCError):
        ctx.submit(hs["er"], pkg.BC_QUERY_SOURCES, targets=[1, 1], c=2.0, cap=10)
    with pytest.raises(pkg.BCError):
        ctx.submit(hs["er"], pkg.BC_QUERY_SOURCES, targets=[1], c=0.5, cap=10)
    with pytest.raises(pkg.BCError):
        ctx.submit(hs["er"], 99, targets=[1], c=2.0, cap=10)


def _served_intervals(ctx, pkg, h, specs):
    """Submits all queries at once; returns (tickets, [(admit, done)] in seconds
    on the host clock), from each ticket's queue and run times."""
    t_sub, tks = [], []
    for kw in specs:
        # stamped after the call returns: the call itself may wait for the
        # context while the server runs a batch, and the library stamps the
        # submission inside it (the host stamp is then at most microseconds late)
        tks.append(ctx.submit(h, pkg.BC_QUERY_PAIRS, **kw))
        t_sub.append(time.perf_counter())
    for tk in tks:
        ctx.poll(tk, -1)
    iv = []
    for t0, tk in zip(t_sub, tks):
        admit = t0 + tk.stats.queue_ms / 1e3
        iv.append((admit, admit + tk.stats.run_ms / 1e3))
    return tks, iv


def test_admission_by_device_memory(ctx, graphs, pkg):
    """A pair query holds d(v,.) and sigma_v. for its T targets (T*n*12 bytes +
    T*64). With a budget that fits one such query, three submitted together run
    one after another (each admitted only once the previous one has finished and
    freed its memory); with the default budget they overlap. Results are
    bit-identical to the queries run alone either way; a query larger than the
    budget is refused at submit."""
    g, hs = graphs
    ba = g["ba"]
    T = 4
    need = T * ba.n * 12 + T * 64
    # long enough (40k pair draws each) to be running still when the next one is submitted
    specs = [dict(targets=gg.degree_targets(ba, T, 30 + i), c=1.0, cap=40000, seed=40 + i, qid=i) for i in range(3)]
    refs = [ctx.adaptive_pairs(hs["ba"], kw["targets"], kw["c"], kw["cap"], kw["seed"], kw["qid"]) for kw in specs]
    try:
        ctx.server_limits(max_active=64, mem_budget_bytes=need + need // 2)
        tks, iv = _served_intervals(ctx, pkg, hs["ba"], specs)
        for tk, ref in zip(tks, refs):
            for key in ["est", "k", "S", "status"]:
                _same(tk.outputs()[key], ref[key], key)
        for (a0, d0), (a1, d1) in zip(iv, iv[1:]):
            assert a1 >= d0 - 2e-3, f"admitted at {a1 - d0:+.4f} s relative to the previous query's end"
        assert all(tk.stats.queue_ms > 0 for tk in tks[1:])
        with pytest.raises(pkg.BCError) as e:
            ctx.submit(hs["ba"], pkg.BC_QUERY_PAIRS, targets=gg.degree_targets(ba, 2 * T, 9), c=1.0, cap=10)
        assert e.value.code == -2  # BC_E_NOMEM: more than the whole budget
    finally:
        # back to the default budget, a quarter of the device's memory
        torch = pytest.importorskip("torch")
        ctx.server_limits(max_active=64, mem_budget_bytes=torch.cuda.get_device_properties(0).total_memory // 4)
    tks, iv = _served_intervals(ctx, pkg, hs["ba"], specs)
    for tk, ref in zip(tks, refs):
        for key in ["est", "k", "S", "status"]:
            _same(tk.outputs()[key], ref[key], key)
    assert any(a1 < d0 for (a0, d0), (a1, d1) in zip(iv, iv[1:])), "with room for all, the queries should overlap"
