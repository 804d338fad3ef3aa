"""GPU parity of the uneven multi-graph persistent TabuCol launch: every individual equals the
single-graph launch with the same Philox stream, and sampled individuals equal the oracle."""
import numpy as np
import pytest

import oracle
from paper_2109_05948_gb300 import dlmcol, inputs

from gpu_util import device_graph, oracle_tabu_many

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2109_05948_gb300 import build

    build.build()
    c = dlmcol.Context(0)
    yield c
    c.close()


def _batch(num_graphs, seed, n_hi, pop):
    specs = inputs.uneven_batch(num_graphs, seed=seed, n_lo=100, n_hi=n_hi)
    return specs, [pop] * num_graphs


@pytest.mark.parametrize("num,n_hi,pop", [(12, 500, 6), (64, 1000, 2)])
def test_multi_matches_single_graph_launches_and_oracle(ctx, num, n_hi, pop):
    """The second case is the uneven workload's graph set (64 graphs, n up to 1000, k = n/10):
    the largest states exceed shared memory and spill rows to the CTAs' slabs."""
    specs, pops = _batch(num, seed=3, n_hi=n_hi, pop=pop)
    graphs = [device_graph(ctx, s["n"], s["edges"]) for s in specs]
    ks = [s["k"] for s in specs]
    iters = [(16 if num <= 12 else 2) * s["n"] for s in specs]  # shortened depths (the paper uses 128 |V|)
    starts = [oracle.init_colors(s["n"], k, p, 5, ind_base=sum(pops[:g])) for g, (s, k, p) in enumerate(zip(specs, ks, pops))]
    cols = [torch.from_numpy(st.copy()).cuda() for st in starts]
    bfs = [torch.zeros(p, dtype=torch.int64, device="cuda") for p in pops]
    mvs = [torch.zeros(p, dtype=torch.int64, device="cuda") for p in pops]
    dlmcol.dlm_tabucol_multi(ctx, graphs, ks, pops, cols, bfs, mvs, iters, dlmcol.COL_TENURE, 5, 1, 0)
    ctx.sync()
    base = 0
    jobs = []
    for g, (s, k, p) in enumerate(zip(specs, ks, pops)):
        col1 = torch.from_numpy(starts[g].copy()).cuda()
        bf1 = torch.zeros(p, dtype=torch.int64, device="cuda")
        mv1 = torch.zeros(p, dtype=torch.int64, device="cuda")
        dlmcol.dlm_tabucol_batch(ctx, graphs[g], k, p, col1, bf1, mv1, iters[g], dlmcol.COL_TENURE, 5, 1, base)
        ctx.sync()
        assert torch.equal(col1, cols[g]) and torch.equal(bf1, bfs[g]) and torch.equal(mv1, mvs[g]), g
        if num <= 12 or s["n"] >= 900:
            adj = inputs.edges_to_adj(s["n"], s["edges"])
            jobs.append((g, (adj, k, starts[g][0], iters[g], 5, base, 1, False)))
        base += p
    refs = oracle_tabu_many([j for _, j in jobs])
    for (g, _), r in zip(jobs, refs):
        assert bfs[g][0].item() == r["best_f"] and mvs[g][0].item() == r["moves"]
        assert np.array_equal(cols[g][0].cpu().numpy(), r["best_col"])


def test_multi_rejects_bad_arguments(ctx):
    specs, pops = _batch(2, seed=1, n_hi=200, pop=2)
    graphs = [device_graph(ctx, s["n"], s["edges"]) for s in specs]
    cols = [torch.zeros((2, s["n"]), dtype=torch.int16, device="cuda") for s in specs]
    bfs = [torch.zeros(2, dtype=torch.int64, device="cuda") for _ in specs]
    with pytest.raises(dlmcol.DlmError):
        dlmcol.dlm_tabucol_multi(ctx, graphs, [300, 10], pops, cols, bfs, None, [10, 10])


def test_multi_plan_graph_replay_matches_direct_launch(ctx):
    """The captured plan replays the same launch: identical results to dlm_tabucol_multi, twice."""
    specs, pops = _batch(10, seed=9, n_hi=1000, pop=3)
    graphs = [device_graph(ctx, s["n"], s["edges"]) for s in specs]
    ks = [s["k"] for s in specs]
    iters = [3 * s["n"] for s in specs]
    starts = [oracle.init_colors(s["n"], k, p, 2) for s, k, p in zip(specs, ks, pops)]
    ref_c = [torch.from_numpy(st.copy()).cuda() for st in starts]
    ref_b = [torch.zeros(p, dtype=torch.int64, device="cuda") for p in pops]
    dlmcol.dlm_tabucol_multi(ctx, graphs, ks, pops, ref_c, ref_b, None, iters, dlmcol.COL_TENURE, 4, 2, 7)
    cols = [torch.from_numpy(st.copy()).cuda() for st in starts]
    bfs = [torch.zeros(p, dtype=torch.int64, device="cuda") for p in pops]
    plan = dlmcol.MultiPlan(ctx, graphs, ks, pops, cols, bfs, None, iters, dlmcol.COL_TENURE, 4, 2, 7)
    for _ in range(2):
        for c, st in zip(cols, starts):
            c.copy_(torch.from_numpy(st))
        dlmcol.dlm_tabucol_multi_plan_launch(ctx, plan)
        ctx.sync()
        for a, b in zip(cols, ref_c):
            assert torch.equal(a, b)
        for a, b in zip(bfs, ref_b):
            assert torch.equal(a, b)
    plan.close()


@pytest.mark.parametrize("n,p,k", [(120, 0.5, 14), (1000, 0.5, 100)])
def test_autotune_then_launches_stay_exact(ctx, n, p, k):
    """The autotuner times every warp count that fits (the second shape spills rows to the CTA
    slabs, which share the context workspace); afterwards a batch and a multi-graph launch with
    the tuned warp count still replay the oracle exactly."""
    e = inputs.gnp(n, p, 11)
    g = device_graph(ctx, n, e)
    w = dlmcol.dlm_tabucol_autotune(ctx, g, k, 40, 300)
    assert w in (1, 2, 4, 8, 16)
    pop, iters = 2, 2 * n
    start = oracle.init_colors(n, k, pop, 6)
    col = torch.from_numpy(start.copy()).cuda()
    bf = torch.zeros(pop, dtype=torch.int64, device="cuda")
    mv = torch.zeros(pop, dtype=torch.int64, device="cuda")
    dlmcol.dlm_tabucol_multi(ctx, [g], [k], [pop], [col], [bf], [mv], [iters], dlmcol.COL_TENURE, 6, 0, 0)
    ctx.sync()
    adj = inputs.edges_to_adj(n, e)
    ref = oracle_tabu_many([(adj, k, start[0], iters, 6, 0, 0, False)])[0]
    assert bf[0].item() == ref["best_f"] and mv[0].item() == ref["moves"]
    assert np.array_equal(col[0].cpu().numpy(), ref["best_col"])


def test_multi_full_workload_sampled(ctx):
    """The uneven workload as the bench runs it: 64 graphs (n in [100, 1000], k = n/10), 256
    individuals each, 128 n iterations, one persistent launch replayed from a captured plan.
    Every returned conflict count recounts from its colouring, and two individuals of each of
    the four smallest graphs equal the oracle over the whole budget."""
    specs = inputs.uneven_batch(64, seed=0)
    graphs = [device_graph(ctx, s["n"], s["edges"]) for s in specs]
    ks = [s["k"] for s in specs]
    pops = [256] * len(specs)
    iters = [128 * s["n"] for s in specs]
    starts, cols, bfs, mvs = [], [], [], []
    base = 0
    for g, (s, k, p) in enumerate(zip(specs, ks, pops)):
        c = torch.empty((p, s["n"]), dtype=torch.int16, device="cuda")
        dlmcol.dlm_init_colors(ctx, s["n"], k, p, 0, base, c)
        starts.append(c.cpu().numpy())
        cols.append(c)
        bfs.append(torch.zeros(p, dtype=torch.int64, device="cuda"))
        mvs.append(torch.zeros(p, dtype=torch.int64, device="cuda"))
        base += p
    plan = dlmcol.MultiPlan(ctx, graphs, ks, pops, cols, bfs, mvs, iters, dlmcol.COL_TENURE, 0, 0, 0)
    dlmcol.dlm_tabucol_multi_plan_launch(ctx, plan)
    ctx.sync()
    for g, (s, k, p) in enumerate(zip(specs, ks, pops)):
        f = torch.zeros(p, dtype=torch.int64, device="cuda")
        dlmcol.dlm_gamma(ctx, graphs[g], k, p, cols[g], None, f)
        ctx.sync()
        assert torch.equal(f, bfs[g]), g
    small = sorted(range(len(specs)), key=lambda g: specs[g]["n"])[:4]
    jobs = []
    for g in small:
        adj = inputs.edges_to_adj(specs[g]["n"], specs[g]["edges"])
        gbase = 256 * g
        for i in (0, 255):
            jobs.append((g, i, (adj, ks[g], starts[g][i], iters[g], 0, gbase + i, 0, False)))
    refs = oracle_tabu_many([j for _, _, j in jobs])
    for (g, i, _), r in zip(jobs, refs):
        assert bfs[g][i].item() == r["best_f"] and mvs[g][i].item() == r["moves"], (g, i)
        assert np.array_equal(cols[g][i].cpu().numpy(), r["best_col"]), (g, i)
    plan.close()
