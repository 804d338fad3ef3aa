"""GPU parity of the paper-size invariant network with invariant batch normalisation
(dlm_deepnet_*) against the FP64 oracle (oracle/deepnet.py), through the C-ABI: scores per
candidate in evaluation and training mode, the running estimates, gradients per parameter block,
Adam steps and the online training, at widths that span several 64-column tiles with ragged
tails, k above 64, and the paper's layer widths on a 200-vertex graph."""
import numpy as np
import pytest

from oracle import deepnet as dn
from paper_2109_05948_gb300 import dlmcol, inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

TOL = 1e-2


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2109_05948_gb300 import build

    build.build()
    c = dlmcol.Context(0)
    yield c
    c.close()


def _params(dims, seed):
    rng = np.random.default_rng(seed)
    th = dn.init_params(dims, rng)
    v = dims.view(th)
    for name, (off, shape) in dims.offsets().items():
        if name.startswith("mu"):
            v[name][:] = rng.normal(0, 0.3, size=shape)
        elif name.startswith("g") and not name.startswith("gam"):
            v[name][:] = rng.uniform(0.6, 1.4, size=shape)
    return th


def _stats(dims, seed):
    rng = np.random.default_rng(seed)
    st = dims.initial_stats()
    for m, var in dims.stats_view(st):
        m[:] = rng.normal(0, 0.5, size=m.shape)
        var[:] = rng.uniform(0.3, 3.0, size=var.shape)
    return st


def _net(ctx, dims, k, th, st):
    net = dlmcol.DeepNet(ctx, dims.n, k, dims.widths, seed=1)
    assert net.nparams == dims.nparams() and net.nstats == dims.nstats()
    net.set(0, torch.from_numpy(th.astype(np.float32)).cuda())
    net.set(1, torch.from_numpy(st.astype(np.float32)).cuda())
    return net


def _f32(th):
    return th.astype(np.float32).astype(np.float64)


def _per_element(got, ref, bias):
    cg = np.asarray(got, np.float64) - bias
    cr = np.asarray(ref, np.float64) - bias
    floor = max(float(np.sqrt(np.mean(cr * cr))), 1e-30)
    return float(np.max(np.abs(cg - cr) / np.maximum(np.abs(cr), floor)))


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


CASES = [(60, (96, 80, 40), 7, 20), (200, (512, 256, 130), 20, 33), (150, (200, 100), 100, 6),
         (33, (17,), 5, 9)]


@pytest.mark.parametrize("n,widths,k,c", CASES)
def test_deepnet_forward_matches_oracle(ctx, n, widths, k, c):
    dims = dn.DeepDims(n, widths)
    th = _f32(_params(dims, seed=n))
    st = _f32(_stats(dims, seed=n + 1))
    cols = inputs.random_colorings(c, n, k, seed=c)
    net = _net(ctx, dims, k, th, st)
    out = torch.zeros(c, dtype=torch.float32, device="cuda")
    dc = torch.from_numpy(cols).cuda()
    bh = dims.view(th)["bh"][0]
    # evaluation (running statistics)
    net.forward(dc, c, 0, out)
    ctx.sync()
    ref = dn.forward(dims, k, th, cols, False, st.copy())
    assert _per_element(out.cpu().numpy(), ref, bh) <= TOL
    # training mode: the batch's own statistics, running estimates updated
    st_ref = st.copy()
    ref_t = dn.forward(dims, k, th, cols, True, st_ref)
    net.forward(dc, c, 1, out)
    got_st = torch.zeros(dims.nstats(), dtype=torch.float32, device="cuda")
    net.get(1, got_st)
    ctx.sync()
    assert _per_element(out.cpu().numpy(), ref_t, bh) <= TOL
    assert _rel(got_st.cpu().numpy(), st_ref) <= 1e-4
    net.close()


@pytest.mark.parametrize("n,widths,k,B", [(60, (96, 80, 40), 7, 20), (120, (256, 130, 70), 30, 12),
                                          (90, (150,), 70, 5)])
def test_deepnet_gradients_match_oracle(ctx, n, widths, k, B):
    dims = dn.DeepDims(n, widths)
    th = _f32(_params(dims, seed=k))
    st = _f32(_stats(dims, seed=k + 2))
    cols = inputs.random_colorings(B, n, k, seed=B + 3)
    y = np.random.default_rng(1).normal(size=B)
    loss_ref, g_ref, out_ref = dn.loss_grad(dims, k, th, cols, y)
    net = _net(ctx, dims, k, th, st)
    grad = torch.zeros(dims.nparams(), dtype=torch.float32, device="cuda")
    out = torch.zeros(B, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    net.loss_grad(torch.from_numpy(cols).cuda(), torch.from_numpy(y.astype(np.float32)).cuda(), B, grad, out, loss)
    ctx.sync()
    assert _per_element(out.cpu().numpy(), out_ref, dims.view(th)["bh"][0]) <= TOL
    assert abs(loss.item() - loss_ref) <= TOL * loss_ref
    g = grad.cpu().numpy()
    errs = {}
    for name, (off, shape) in dims.offsets().items():
        sz = int(np.prod(shape))
        ref_b = g_ref[off:off + sz]
        if name.startswith("b") and name != "bh":
            # beta before a normalisation has a zero gradient in exact arithmetic: compare on the
            # scale of the layer's other gradients
            assert np.abs(g[off:off + sz]).max() <= 1e-3 * max(1e-30, np.abs(g_ref).max())
            continue
        errs[name] = _rel(g[off:off + sz], ref_b)
    assert max(errs.values()) <= TOL, errs
    net.close()


def test_deepnet_training_matches_oracle(ctx):
    """Two epochs of Adam (lr 1e-3, b = 40) on p = 100 samples: parameters per block and running
    estimates against the FP64 oracle run in the same epoch order."""
    n, widths, k, p = 50, (80, 64, 30), 6, 100
    dims = dn.DeepDims(n, widths)
    th0 = _f32(_params(dims, seed=5))
    st0 = dims.initial_stats()
    cols = inputs.random_colorings(p, n, k, seed=3)
    fvals = np.random.default_rng(2).integers(0, 40, size=p).astype(np.int64)
    th = th0.copy()
    st = st0.copy()
    am, av = np.zeros_like(th), np.zeros_like(th)
    dn.train(dims, k, th, am, av, 0, st, cols, fvals, epochs=2, b=40, lr=1e-3, seed=9, gen=4)
    net = _net(ctx, dims, k, th0, st0)
    net.train(torch.from_numpy(cols).cuda(), torch.from_numpy(fvals).cuda(), p, 2, 40, 1e-3, 9, 4)
    got = torch.zeros(dims.nparams(), dtype=torch.float32, device="cuda")
    got_st = torch.zeros(dims.nstats(), dtype=torch.float32, device="cuda")
    net.get(0, got)
    net.get(1, got_st)
    ctx.sync()
    gp = got.cpu().numpy().astype(np.float64)
    steps = 2 * 3
    for name, (off, shape) in dims.offsets().items():
        sz = int(np.prod(shape))
        if name.startswith("b") and name != "bh":
            # beta_l sits right before a normalisation: its gradient is zero in exact arithmetic,
            # so Adam turns rounding noise into steps of up to about 3.2 lr on either side; both
            # runs stay within that of the start
            for side in (gp, th):
                assert np.abs(side[off:off + sz] - th0[off:off + sz]).max() <= steps * 3.2e-3 + 1e-6, name
            continue
        assert _rel(gp[off:off + sz], th[off:off + sz]) <= TOL, name
    # the trained networks agree where beta has no effect: training-mode scores of fresh colourings
    test_cols = inputs.random_colorings(16, n, k, seed=77)
    out = torch.zeros(16, dtype=torch.float32, device="cuda")
    net.forward(torch.from_numpy(test_cols).cuda(), 16, 1, out)
    ctx.sync()
    ref = dn.forward(dims, k, th, test_cols, True)
    assert _per_element(out.cpu().numpy(), ref, dims.view(th)["bh"][0]) <= TOL
    assert _rel(got_st.cpu().numpy(), st) <= 1e-3
    net.close()


def test_deepnet_paper_widths_on_200_vertices(ctx):
    """The paper's k-COL network shape (9 hidden layers of 10|V| ... |V|//2) at |V| = 200, k = 20:
    evaluation and training-mode scores per candidate against the oracle."""
    n, k, c = 200, 20, 6
    dims = dn.DeepDims(n, dn.paper_widths(n, "col"))
    th = _f32(_params(dims, seed=11))
    st = _f32(_stats(dims, seed=12))
    cols = inputs.random_colorings(c, n, k, seed=7)
    net = _net(ctx, dims, k, th, st)
    out = torch.zeros(c, dtype=torch.float32, device="cuda")
    dc = torch.from_numpy(cols).cuda()
    net.forward(dc, c, 0, out)
    ctx.sync()
    bh = dims.view(th)["bh"][0]
    assert _per_element(out.cpu().numpy(), dn.forward(dims, k, th, cols, False, st.copy()), bh) <= TOL
    net.forward(dc, c, 1, out)
    ctx.sync()
    assert _per_element(out.cpu().numpy(), dn.forward(dims, k, th, cols, True, st.copy()), bh) <= TOL
    net.close()


def test_deepnet_bf16_operands_and_invariance(ctx):
    """bf16 operands alone (two fewer MMA passes) stay within 3e-2 per candidate; relabelling the
    colours leaves the scores unchanged up to the FP32 summation order."""
    n, widths, k, c = 120, (256, 128, 64), 12, 24
    dims = dn.DeepDims(n, widths)
    th = _f32(_params(dims, seed=21))
    st = _f32(_stats(dims, seed=22))
    cols = inputs.random_colorings(c, n, k, seed=4)
    net = _net(ctx, dims, k, th, st)
    out = torch.zeros(c, dtype=torch.float32, device="cuda")
    out2 = torch.zeros(c, dtype=torch.float32, device="cuda")
    ref = dn.forward(dims, k, th, cols, False, st.copy())
    bh = dims.view(th)["bh"][0]
    net.set_precision(0)
    net.forward(torch.from_numpy(cols).cuda(), c, 0, out)
    ctx.sync()
    assert _per_element(out.cpu().numpy(), ref, bh) <= 3 * TOL
    net.set_precision(1)
    sigma = np.random.default_rng(0).permutation(k)
    net.forward(torch.from_numpy(cols).cuda(), c, 0, out)
    net.forward(torch.from_numpy(sigma[cols].astype(np.int16)).cuda(), c, 0, out2)
    ctx.sync()
    cen = np.abs(out.cpu().numpy() - bh).max()
    assert np.abs(out.cpu().numpy() - out2.cpu().numpy()).max() <= 1e-4 * max(cen, 1e-6)
    net.close()


def test_deepnet_rejects_bad_arguments(ctx):
    with pytest.raises(dlmcol.DlmError):
        dlmcol.DeepNet(ctx, 10, 3, [])
    with pytest.raises(dlmcol.DlmError):
        dlmcol.DeepNet(ctx, 10, 300, [8])
    with pytest.raises(dlmcol.DlmError):
        dlmcol.DeepNet(ctx, 10, 3, [20000])
