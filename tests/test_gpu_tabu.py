"""GPU parity of graph build, initialisation, conflict table and batched TabuCol against the
oracle, through the C-ABI. TabuCol must match bit for bit: the move of every iteration (trace),
the best colouring, its conflicts and the number of moves."""
import numpy as np
import pytest

import oracle
from paper_2109_05948_gb300 import dlmcol, inputs

from gpu_util import _oracle_tabu_alpha_job, _oracle_tabu_job, oracle_pool, device_graph, gnp_case, oracle_tabu_many

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


def _run_gpu(ctx, g, k, col_np, iters, seed=0, gen=0, ind_base=0, warps=0, trace=False):
    pop, n = col_np.shape
    col = torch.from_numpy(col_np.copy()).cuda()
    bf = torch.zeros(pop, dtype=torch.int64, device="cuda")
    mv = torch.zeros(pop, dtype=torch.int64, device="cuda")
    tr = torch.full((pop, iters, 4), -7, dtype=torch.int32, device="cuda") if trace else None
    dlmcol.dlm_tabucol_batch_ex(ctx, g, k, pop, col, bf, mv, iters, dlmcol.COL_TENURE, seed, gen, ind_base, warps, tr)
    ctx.sync()
    out = dict(col=col.cpu().numpy(), best_f=bf.cpu().numpy(), moves=mv.cpu().numpy())
    if trace:
        out["trace"] = tr.cpu().numpy()
    return out


def test_graph_build_matches_oracle(ctx):
    for n, p, s in [(125, 0.5, 0), (500, 0.5, 0), (97, 0.1, 3), (1000, 0.9, 1), (33, 1.0, 0)]:
        e, adj = gnp_case(n, p, s)
        g = device_graph(ctx, n, e)
        off, idx, bits = oracle.graph_csr(adj)
        assert g.m == len(e)
        doff = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
        didx = torch.zeros(max(1, 2 * g.m), dtype=torch.int32, device="cuda")
        dbits = torch.zeros((n, (n + 31) // 32), dtype=torch.int32, device="cuda")
        dlmcol.dlm_graph_export(ctx, g, doff, didx, dbits)
        ctx.sync()
        assert np.array_equal(doff.cpu().numpy(), off)
        assert np.array_equal(didx.cpu().numpy()[: 2 * g.m], idx)
        assert np.array_equal(dbits.cpu().numpy().view(np.uint32), bits)


def test_graph_rejects_bad_edges(ctx):
    with pytest.raises(dlmcol.DlmError):
        device_graph(ctx, 5, np.array([[0, 1], [2, 5]], np.int32))
    with pytest.raises(dlmcol.DlmError):
        device_graph(ctx, 5, np.array([[3, 3]], np.int32))


def test_init_colors_matches_oracle(ctx):
    for n, k, pop, seed, base in [(125, 17, 8, 0, 0), (500, 48, 64, 5, 3), (1000, 100, 3, 2**40 + 7, 11)]:
        col = torch.zeros((pop, n), dtype=torch.int16, device="cuda")
        dlmcol.dlm_init_colors(ctx, n, k, pop, seed, base, col)
        ctx.sync()
        assert np.array_equal(col.cpu().numpy(), oracle.init_colors(n, k, pop, seed, base))


def test_gamma_matches_oracle(ctx):
    n, k, pop = 300, 23, 5
    e, adj = gnp_case(n, 0.3, 2)
    g = device_graph(ctx, n, e)
    cols = inputs.random_colorings(pop, n, k, seed=4)
    gam = torch.zeros((pop, n, k), dtype=torch.int32, device="cuda")
    f = torch.zeros(pop, dtype=torch.int64, device="cuda")
    dlmcol.dlm_gamma(ctx, g, k, pop, torch.from_numpy(cols).cuda(), gam, f)
    ctx.sync()
    for i in range(pop):
        g_ref, f_ref = oracle.gamma(adj, k, cols[i])
        assert np.array_equal(gam[i].cpu().numpy(), g_ref) and f[i].item() == f_ref


@pytest.mark.parametrize("warps", [1, 2, 4, 8, 16, 32])
def test_tabucol_small_random_graph_trace_bitexact(ctx, warps):
    """8 individuals on G(125, 0.5), k = 17, 10^4 iterations, seed 0 (gamma is exact in u16 for n < 65536): every
    iteration's move, the best colouring, best f and moves equal the oracle's."""
    n, k, pop, iters = 125, 17, 8, 10_000
    e, adj = gnp_case(n, 0.5, 0)
    g = device_graph(ctx, n, e)
    start = oracle.init_colors(n, k, pop, 0)
    gpu = _run_gpu(ctx, g, k, start, iters, seed=0, warps=warps, trace=True)
    refs = oracle_tabu_many([(adj, k, start[i], iters, 0, i, 0, True) for i in range(pop)])
    for i, r in enumerate(refs):
        T = r["iters"]
        assert np.array_equal(gpu["trace"][i, :T], r["trace"]), f"individual {i}: first divergence at " \
            f"{int(np.argmax(np.any(gpu['trace'][i, :T] != r['trace'], axis=1)))}"
        assert gpu["best_f"][i] == r["best_f"] and gpu["moves"][i] == r["moves"]
        assert np.array_equal(gpu["col"][i], r["best_col"])


@pytest.mark.parametrize("n,k,p,iters,pop,seed", [
    (64, 5, 0.3, 3000, 7, 1),      # n a multiple of 32, odd k
    (101, 9, 0.2, 2000, 5, 2),     # ragged n
    (260, 100, 0.9, 1500, 3, 3),   # k > 64: several words per lane
    (700, 30, 0.5, 1000, 2, 4),    # n > 512: two bitmap words per lane
    (2, 2, 1.0, 50, 3, 5),         # a single edge
    (1000, 100, 0.5, 800, 3, 6),   # state above shared memory: the last rows live in a slab
    (1500, 128, 0.9, 400, 2, 7),   # larger spill, maximum k
])
def test_tabucol_shapes_bitexact(ctx, n, k, p, iters, pop, seed):
    e, adj = gnp_case(n, p, seed)
    g = device_graph(ctx, n, e)
    start = oracle.init_colors(n, k, pop, seed)
    gpu = _run_gpu(ctx, g, k, start, iters, seed=seed, gen=3, ind_base=10, trace=True)
    refs = oracle_tabu_many([(adj, k, start[i], iters, seed, 10 + i, 3, True) for i in range(pop)])
    for i, r in enumerate(refs):
        assert np.array_equal(gpu["trace"][i, :r["iters"]], r["trace"])
        assert gpu["best_f"][i] == r["best_f"] and gpu["moves"][i] == r["moves"]
        assert np.array_equal(gpu["col"][i], r["best_col"])


@pytest.mark.parametrize("warps", [16, 32])
def test_tabucol_planted_1000_k48_trace_bitexact(ctx, warps):
    """The memetic workload's graph (planted 48-colourable, n = 1000, p = 0.5 across parts): one
    vertex (32 warps) or two vertices (16 warps) per thread, every move equal to the oracle's."""
    n, k, pop, iters = 1000, 48, 3, 2000
    e, _ = inputs.planted(n, k, 0.5, seed=0)
    adj = inputs.edges_to_adj(n, e)
    g = device_graph(ctx, n, e)
    start = oracle.init_colors(n, k, pop, 5, 40)
    gpu = _run_gpu(ctx, g, k, start, iters, seed=5, gen=1, ind_base=40, warps=warps, trace=True)
    refs = oracle_tabu_many([(adj, k, start[i], iters, 5, 40 + i, 1, True) for i in range(pop)])
    for i, r in enumerate(refs):
        assert np.array_equal(gpu["trace"][i, :r["iters"]], r["trace"])
        assert gpu["best_f"][i] == r["best_f"] and gpu["moves"][i] == r["moves"]
        assert np.array_equal(gpu["col"][i], r["best_col"])


def test_tabucol_planted_early_stop_and_legal_start(ctx):
    n, k = 200, 8
    e, part = inputs.planted(n, k, 0.5, seed=2)
    adj = inputs.edges_to_adj(n, e)
    g = device_graph(ctx, n, e)
    start = oracle.init_colors(n, k, 4, 1)
    start[3] = part  # already legal: no iteration runs
    gpu = _run_gpu(ctx, g, k, start, 50_000, seed=1, trace=False)
    refs = oracle_tabu_many([(adj, k, start[i], 50_000, 1, i, 0, False) for i in range(4)])
    for i, r in enumerate(refs):
        assert gpu["best_f"][i] == r["best_f"] == 0 and gpu["moves"][i] == r["moves"]
        assert np.array_equal(gpu["col"][i], r["best_col"])
    assert gpu["moves"][3] == 0


@pytest.mark.parametrize("case", ["no_budget", "edgeless", "max_n", "k_above_n"])
def test_tabucol_degenerate_cases_match_oracle(ctx, case):
    """Degenerate inputs: a zero budget (the start colouring and its conflicts come back, no
    move), an edgeless graph (f = 0 at the start: nothing runs), the largest n the kernel takes
    (2048, sparse) and more colours than vertices (K_10 with k = 20 reaches 0)."""
    n, k, p, iters, pop = {"no_budget": (300, 20, 0.5, 0, 3), "edgeless": (64, 3, 0.0, 100, 2),
                           "max_n": (2048, 8, 0.004, 300, 2), "k_above_n": (10, 20, 1.0, 200, 3)}[case]
    e, adj = gnp_case(n, p, 9)
    g = device_graph(ctx, n, e)
    start = oracle.init_colors(n, k, pop, 9)
    gpu = _run_gpu(ctx, g, k, start, iters, seed=9, trace=iters > 0)
    refs = oracle_tabu_many([(adj, k, start[i], iters, 9, i, 0, iters > 0) for i in range(pop)])
    for i, r in enumerate(refs):
        if iters > 0:
            assert np.array_equal(gpu["trace"][i, :r["iters"]], r["trace"])
        assert gpu["best_f"][i] == r["best_f"] and gpu["moves"][i] == r["moves"]
        assert np.array_equal(gpu["col"][i], r["best_col"])
    if case in ("no_budget", "edgeless"):
        assert np.array_equal(gpu["col"], start) and not gpu["moves"].any()
    if case == "k_above_n":
        assert not gpu["best_f"].any()


def test_tabucol_long_run_crosses_tabu_sweeps(ctx):
    """70 000 iterations cross the 2^14 sweep of the 16-bit tabu expiries four times and wrap 2^16."""
    n, k, pop, iters = 150, 15, 2, 70_000
    e, adj = gnp_case(n, 0.5, 7)
    g = device_graph(ctx, n, e)
    start = oracle.init_colors(n, k, pop, 7)
    gpu = _run_gpu(ctx, g, k, start, iters, seed=7)
    refs = oracle_tabu_many([(adj, k, start[i], iters, 7, i, 0, False) for i in range(pop)])
    for i, r in enumerate(refs):
        assert gpu["best_f"][i] == r["best_f"] and gpu["moves"][i] == r["moves"]
        assert np.array_equal(gpu["col"][i], r["best_col"])


def test_tabucol_rejects_bad_input(ctx):
    n, k = 50, 4
    e, adj = gnp_case(n, 0.3, 1)
    g = device_graph(ctx, n, e)
    col = torch.zeros((2, n), dtype=torch.int16, device="cuda")
    col[1, 7] = 4  # colour outside 0..k-1
    bf = torch.zeros(2, dtype=torch.int64, device="cuda")
    dlmcol.dlm_tabucol_batch(ctx, g, k, 2, col, bf, None, 10)
    with pytest.raises(dlmcol.DlmError):
        ctx.sync()
    with pytest.raises(dlmcol.DlmError):
        dlmcol.dlm_tabucol_batch(ctx, g, 200, 2, col, bf, None, 10)  # k above 128
    with pytest.raises(dlmcol.DlmError):
        dlmcol.dlm_tabucol_batch_ex(ctx, g, k, 2, col, bf, None, 10, warps=3)
    dlmcol.dlm_tabucol_batch(ctx, g, k, 0, col, bf, None, 10)  # empty population is a no-op
    ctx.sync()
    for bad_n in (1, 2049):  # graphs take 2..2048 vertices
        with pytest.raises(dlmcol.DlmError):
            device_graph(ctx, bad_n, np.zeros((0, 2), np.int32))


def test_tabucol_full_size_all_individuals(ctx):
    """The benchmarked launch: G(500, 0.5), k = 48, population 4096, 10^5 iterations, random
    starts from seed 0. All 4096 individuals are replayed by the oracle (best conflicts, moves and
    best colouring equal), the best conflicts equal the recount of the returned colouring, and 32
    individuals (ids 0..15 and 4080..4095, launched again with a trace) match the oracle move by
    move over the whole budget."""
    n, k, pop, iters = 500, 48, 4096, 100_000
    e, adj = gnp_case(n, 0.5, 0)
    g = device_graph(ctx, n, e)
    col = torch.zeros((pop, n), dtype=torch.int16, device="cuda")
    dlmcol.dlm_init_colors(ctx, n, k, pop, 0, 0, col)
    start = col.cpu().numpy()
    bf = torch.zeros(pop, dtype=torch.int64, device="cuda")
    mv = torch.zeros(pop, dtype=torch.int64, device="cuda")
    dlmcol.dlm_tabucol_batch(ctx, g, k, pop, col, bf, mv, iters, dlmcol.COL_TENURE, 0, 0, 0)
    f2 = torch.zeros(pop, dtype=torch.int64, device="cuda")
    dlmcol.dlm_gamma(ctx, g, k, pop, col, None, f2)
    ctx.sync()
    assert torch.equal(bf, f2)
    traced = list(range(16)) + list(range(pop - 16, pop))
    gtr = {}
    for base in (0, pop - 16):
        out = _run_gpu(ctx, g, k, start[base:base + 16], iters, seed=0, ind_base=base, trace=True)
        for j in range(16):
            gtr[base + j] = out["trace"][j]
    jobs = [(adj, k, start[i], iters, 0, i, 0, i in gtr) for i in range(pop)]
    refs = oracle_pool().map(_oracle_tabu_job, jobs, chunksize=8)
    colh, bfh, mvh = col.cpu().numpy(), bf.cpu().numpy(), mv.cpu().numpy()
    bad = [i for i, r in enumerate(refs)
           if bfh[i] != r["best_f"] or mvh[i] != r["moves"] or not np.array_equal(colh[i], r["best_col"])]
    assert not bad, f"{len(bad)} individuals differ from the oracle, first {bad[:8]}"
    for i in traced:
        T = refs[i]["iters"]
        assert np.array_equal(gtr[i][:T], refs[i]["trace"]), i


def test_tabucol_cancel_flag(ctx):
    """A set flag stops every search at its first poll (iteration 0: no move, the start colouring
    is returned); a pinned host flag raised while the launch runs stops it early. In both cases
    dlm_sync reports DLM_ECANCELLED and the returned best conflicts recount from the returned
    colouring."""
    n, k, pop = 200, 10, 4
    e, adj = gnp_case(n, 0.5, 3)
    g = device_graph(ctx, n, e)
    start = oracle.init_colors(n, k, pop, 3)
    col = torch.from_numpy(start.copy()).cuda()
    bf = torch.zeros(pop, dtype=torch.int64, device="cuda")
    mv = torch.zeros(pop, dtype=torch.int64, device="cuda")
    flag = torch.ones(1, dtype=torch.int32, device="cuda")
    try:
        dlmcol.dlm_set_cancel_flag(ctx, flag)
        dlmcol.dlm_tabucol_batch(ctx, g, k, pop, col, bf, mv, 10_000)
        with pytest.raises(dlmcol.DlmError, match="ECANCELLED"):
            ctx.sync()
        assert torch.equal(col.cpu(), torch.from_numpy(start)) and int(mv.sum()) == 0
        f0 = torch.zeros(pop, dtype=torch.int64, device="cuda")
        dlmcol.dlm_gamma(ctx, g, k, pop, col, None, f0)
        ctx.sync()
        assert torch.equal(bf, f0)
        # a pinned host flag raised by the host while the kernels run
        hflag = torch.zeros(1, dtype=torch.int32).pin_memory()
        dlmcol.dlm_set_cancel_flag(ctx, hflag)
        iters = 2_000_000
        col.copy_(torch.from_numpy(start))
        dlmcol.dlm_tabucol_batch(ctx, g, k, pop, col, bf, mv, iters)
        import time
        time.sleep(0.2)
        hflag[0] = 1
        with pytest.raises(dlmcol.DlmError, match="ECANCELLED"):
            ctx.sync()
        assert 0 < int(mv.max()) < iters
        dlmcol.dlm_gamma(ctx, g, k, pop, col, None, f0)
        ctx.sync()
        assert torch.equal(bf, f0)
    finally:
        dlmcol.dlm_set_cancel_flag(ctx, None)
    # without the flag the context runs normally again
    dlmcol.dlm_tabucol_batch(ctx, g, k, pop, col, bf, mv, 100)
    ctx.sync()


def _run_opts(ctx, g, k, col_np, iters, seed=0, gen=0, ind_base=0, warps=0, ring=0, legacy=0, trace=False,
              tenure=None, work=False, entry_bits=0):
    pop, n = col_np.shape
    col = torch.from_numpy(col_np.copy()).cuda()
    bf = torch.zeros(pop, dtype=torch.int64, device="cuda")
    mv = torch.zeros(pop, dtype=torch.int64, device="cuda")
    tr = torch.full((pop, iters, 4), -7, dtype=torch.int32, device="cuda") if trace else None
    wk = torch.zeros((pop, 3), dtype=torch.int64, device="cuda") if work else None
    dlmcol.dlm_tabucol_batch_opts(ctx, g, k, pop, col, bf, mv, iters, tenure or dlmcol.COL_TENURE, seed, gen,
                                  ind_base, warps=warps, ring=ring, legacy=legacy, trace=tr, work=wk,
                                  entry_bits=entry_bits)
    ctx.sync()
    out = dict(col=col.cpu().numpy(), best_f=bf.cpu().numpy(), moves=mv.cpu().numpy())
    if trace:
        out["trace"] = tr.cpu().numpy()
    if work:
        out["work"] = wk.cpu().numpy()
    return out


@pytest.mark.parametrize("entry_bits", [16, 8])
@pytest.mark.parametrize("warps,ring,alpha", [(2, 64, (6, 10)), (4, 64, (30, 10)), (8, 128, (6, 10)),
                                              (1, 64, (60, 10)), (4, 0, (6, 10))])
def test_tabucol_grouped_rings_and_far_list_bitexact(ctx, warps, ring, alpha, entry_bits):
    """The grouped kernel with small tabu rings: tenures of 64 iterations and more go to the
    global far list (alpha = 3 and 6 make them common), and several individuals share a CTA
    (population 400). Every move, best colouring, best f and move count equal the oracle's."""
    n, k, pop, iters = 90, 7, 400, 1500
    e, adj = gnp_case(n, 0.5, 17)
    g = device_graph(ctx, n, e)
    start = oracle.init_colors(n, k, pop, 17)
    ten = dlmcol.Tenure(9, alpha[0], alpha[1])
    if entry_bits == 8 and 32 * warps * 4 < n:  # u8 entries: kernels for up to 4 vertices a thread
        return
    gpu = _run_opts(ctx, g, k, start, iters, seed=17, gen=2, warps=warps, ring=ring, trace=True, tenure=ten,
                    entry_bits=entry_bits)
    sample = list(range(0, pop, 37)) + [pop - 1]
    jobs = [(adj, k, start[i], iters, 17, i, 2, True) for i in sample]
    refs = oracle_pool().map(_oracle_tabu_alpha_job, [(j, alpha) for j in jobs])
    for i, r in zip(sample, refs):
        T = r["iters"]
        assert np.array_equal(gpu["trace"][i, :T], r["trace"]), f"individual {i}: first divergence at " \
            f"{int(np.argmax(np.any(gpu['trace'][i, :T] != r['trace'], axis=1)))}"
        assert gpu["best_f"][i] == r["best_f"] and gpu["moves"][i] == r["moves"]
        assert np.array_equal(gpu["col"][i], r["best_col"])


@pytest.mark.parametrize("case", ["start_class_too_large", "first_move_overflows", "mixed"])
def test_tabucol_u8_entries_fall_back_to_u16(ctx, case):
    """8-bit conflict-table entries hold counts up to 126, guaranteed by keeping every colour class
    at most 126 vertices; an individual whose start colouring has a larger class, or whose search
    would grow one, is searched again with 16-bit entries. Traces, results and move counts equal the
    oracle's in every case, and individuals that never reach the bound keep their u8 results."""
    if case == "start_class_too_large":
        n, k, pop, iters = 300, 2, 24, 400
        e, adj = gnp_case(n, 0.1, 5)
        start = oracle.init_colors(n, k, pop, 5)
    elif case == "first_move_overflows":
        # two classes of exactly 126: the first move makes one of them 127
        n, k, pop, iters = 252, 2, 16, 300
        e, adj = gnp_case(n, 0.05, 6)
        rng = np.random.default_rng(6)
        start = np.stack([rng.permutation(np.repeat(np.arange(k), n // k)) for _ in range(pop)]).astype(np.int16)
    else:
        # half the population starts with a class of 127 (searched again), half balanced far below
        n, k, pop, iters = 254, 4, 20, 500
        e, adj = gnp_case(n, 0.2, 7)
        start = oracle.init_colors(n, k, pop, 7)
        for i in range(0, pop, 2):
            start[i] = 0
            start[i][127:] = np.random.default_rng(i).integers(1, k, size=n - 127)
    g = device_graph(ctx, n, e)
    gpu = _run_opts(ctx, g, k, start, iters, seed=8, gen=1, warps=4, trace=True, entry_bits=8)
    ref16 = _run_opts(ctx, g, k, start, iters, seed=8, gen=1, warps=4, trace=True, entry_bits=16)
    for key in ("col", "best_f", "moves", "trace"):
        assert np.array_equal(gpu[key], ref16[key]), key
    refs = oracle_tabu_many([(adj, k, start[i], iters, 8, i, 1, True) for i in range(0, pop, 5)])
    for i, r in zip(range(0, pop, 5), refs):
        T = r["iters"]
        assert np.array_equal(gpu["trace"][i, :T], r["trace"])
        assert gpu["best_f"][i] == r["best_f"] and np.array_equal(gpu["col"][i], r["best_col"])


@pytest.mark.parametrize("n,k,pop,iters,dens", [(1000, 128, 64, 1500, 0.5), (2048, 100, 24, 600, 0.1)])
def test_tabucol_u8_on_chip_beyond_the_u16_state(ctx, n, k, pop, iters, dens):
    """States whose u16 conflict table exceeds one SM (n = 1000, k = 128: 266 KB; n = 2048,
    k = 100: 418 KB) run on chip with u8 entries; the individuals a u8 launch gives up (here every
    other one starts with a class of 127 vertices) are searched by the one-individual-per-CTA
    kernel with its L2 slab. Results, moves and traces equal that kernel's on every individual and
    the oracle's on a sample."""
    e, adj = gnp_case(n, dens, 9)
    g = device_graph(ctx, n, e)
    info = dlmcol.dlm_tabucol_launch_info(ctx, g, k, pop)
    assert info["grouped"] == 2
    start = oracle.init_colors(n, k, pop, 9)
    for i in range(0, pop, 2):
        start[i][:127] = 0
        start[i][127:] = np.random.default_rng(i).integers(1, k, size=n - 127)
    a = _run_opts(ctx, g, k, start, iters, seed=9, gen=1, trace=True)
    b = _run_opts(ctx, g, k, start, iters, seed=9, gen=1, trace=True, legacy=1)
    for key in ("col", "best_f", "moves", "trace"):
        assert np.array_equal(a[key], b[key]), key
    sample = [0, 1, pop - 1]
    refs = oracle_tabu_many([(adj, k, start[i], iters, 9, i, 1, True) for i in sample])
    for i, r in zip(sample, refs):
        T = r["iters"]
        assert np.array_equal(a["trace"][i, :T], r["trace"])
        assert a["best_f"][i] == r["best_f"] and np.array_equal(a["col"][i], r["best_col"])


def test_tabucol_u8_entries_on_the_benchmark_graph(ctx):
    """The library's choice on G(500, 0.5), k = 48 is u8 entries (more individuals per SM); its
    results equal the u16 kernel's and the oracle's."""
    n, k, pop, iters = 500, 48, 1000, 3000
    e, adj = gnp_case(n, 0.5, 0)
    g = device_graph(ctx, n, e)
    info = dlmcol.dlm_tabucol_launch_info(ctx, g, k, 4096)
    assert info["grouped"] == 2 and info["groups"] > 4
    start = oracle.init_colors(n, k, pop, 4)
    a = _run_opts(ctx, g, k, start, iters, seed=4, work=True)
    b = _run_opts(ctx, g, k, start, iters, seed=4, work=True, entry_bits=16)
    for key in ("col", "best_f", "moves", "work"):
        assert np.array_equal(a[key], b[key]), key
    refs = oracle_tabu_many([(adj, k, start[i], iters, 4, i, 0, False) for i in (0, 499, 999)])
    for i, r in zip((0, 499, 999), refs):
        assert a["best_f"][i] == r["best_f"] and np.array_equal(a["col"][i], r["best_col"])


def test_tabucol_grouped_equals_legacy_path(ctx):
    """The grouped kernel (tabu flags inside gamma, several individuals per CTA, bit rows in shared
    memory) and the one-individual-per-CTA kernel (expiry table) return the same results on the
    benchmark's graph, G(500, 0.5), k = 48."""
    n, k, pop, iters = 500, 48, 912, 4000
    e, adj = gnp_case(n, 0.5, 0)
    g = device_graph(ctx, n, e)
    start = oracle.init_colors(n, k, pop, 3)
    a = _run_opts(ctx, g, k, start, iters, seed=3, work=True)
    b = _run_opts(ctx, g, k, start, iters, seed=3, legacy=1, warps=16, work=True)
    assert np.array_equal(a["best_f"], b["best_f"]) and np.array_equal(a["moves"], b["moves"])
    assert np.array_equal(a["col"], b["col"])
    # the selection and the update visit the same rows on both paths
    assert np.array_equal(a["work"][:, :2], b["work"][:, :2])
    refs = oracle_tabu_many([(adj, k, start[i], iters, 3, i, 0, False) for i in (0, 455, 911)])
    for i, r in zip((0, 455, 911), refs):
        assert a["best_f"][i] == r["best_f"] and np.array_equal(a["col"][i], r["best_col"])
