"""The allocation-free uneven-batch entry point (dlm_tabucol_multi_noalloc) against the regular
one (dlm_tabucol_multi), through the C-ABI.

dlm_tabucol_multi_noalloc serves callers that must not allocate device memory (latency-critical
code that cannot afford cudaMalloc's implicit synchronisation, or processes whose device memory
belongs to another allocator); it keeps its job list and work queue in a static device array of
the library. TabuCol is integer work, so the tolerance is exact equality. This file is collected
last so that a failure here does not hide the other tests."""
import numpy as np
import pytest

from paper_2109_05948_gb300 import dlmcol, inputs

from gpu_util import device_graph

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


def _run(fn, ctx, graphs, ks, pops, starts, iters):
    cols = [torch.from_numpy(st.copy()).cuda() for st in starts]
    bfs = [torch.zeros(p, dtype=torch.int64, device="cuda") for p in pops]
    mvs = [torch.zeros(p, dtype=torch.int64, device="cuda") for p in pops]
    fn(ctx, graphs, ks, pops, cols, bfs, mvs, iters, dlmcol.COL_TENURE, 11, 2, 100)
    ctx.sync()
    return [c.cpu().numpy() for c in cols], [b.cpu().numpy() for b in bfs], [m.cpu().numpy() for m in mvs]


def test_noalloc_matches_regular_entry_point_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2109_05948_gb300 import build

    build.build()
    ctx = dlmcol.Context(0)
    specs = inputs.uneven_batch(6, seed=7, n_lo=60, n_hi=300)
    graphs = [device_graph(ctx, s["n"], s["edges"]) for s in specs]
    ks = [s["k"] for s in specs]
    pops = [5, 3, 7, 2, 4, 6]
    iters = [8 * s["n"] for s in specs]
    rng = np.random.default_rng(0)
    for call in range(2):  # two calls in a row share (and must reset) the static scratch array
        starts = [rng.integers(0, k, size=(p, s["n"])).astype(np.int16) for s, k, p in zip(specs, ks, pops)]
        ref = _run(dlmcol.dlm_tabucol_multi, ctx, graphs, ks, pops, starts, iters)
        got = _run(dlmcol.dlm_tabucol_multi_noalloc, ctx, graphs, ks, pops, starts, iters)
        for a, b in zip(ref, got):
            for x, y in zip(a, b):
                assert np.array_equal(x, y), f"call {call}"
    ctx.close()


def test_noalloc_rejects_more_jobs_than_the_static_array_holds(ctx):
    n = 12
    g = device_graph(ctx, n, inputs.cycle(n))
    pop = 16385
    col = torch.zeros((pop, n), dtype=torch.int16, device="cuda")
    bf = torch.zeros(pop, dtype=torch.int64, device="cuda")
    with pytest.raises(dlmcol.DlmError) as e:
        dlmcol.dlm_tabucol_multi_noalloc(ctx, [g], [3], [pop], [col], [bf], None, [10])
    assert e.value.status == dlmcol.DLM_EUNSUPPORTED
