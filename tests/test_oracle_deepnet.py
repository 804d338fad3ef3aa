"""Pins of the FP64 oracle of the paper-size invariant network with invariant batch
normalisation (oracle/deepnet.py): finite differences of the hand-derived backward pass, colour
permutation invariance, the invariances batch normalisation implies, the reduction to the plain
network of the C++ oracle when the normalisation is the identity, and the running estimates."""
import numpy as np
import pytest

import oracle
from oracle import deepnet as dn
from paper_2109_05948_gb300 import inputs


def _case(n=11, widths=(9, 7, 5), k=3, B=6, seed=0):
    dims = dn.DeepDims(n, widths)
    rng = np.random.default_rng(seed)
    th = dn.init_params(dims, rng)
    v = dims.view(th)
    for name, (off, shape) in dims.offsets().items():  # BN affine parameters away from 1 / 0
        if name.startswith("mu"):
            v[name][:] = rng.normal(0, 0.3, size=shape)
        elif name.startswith("g") and not name.startswith("gam"):
            v[name][:] = rng.uniform(0.5, 1.5, size=shape)
    cols = inputs.random_colorings(B, n, k, seed=seed + 1)
    y = rng.normal(size=B)
    return dims, th, cols, y, k


def test_paper_widths():
    assert dn.paper_widths(1000, "col") == [10000, 5000, 2000, 2000, 2000, 2000, 2000, 1000, 500]
    assert dn.paper_widths(1000, "wvcp") == [5000, 2000, 1000, 500]


@pytest.mark.parametrize("seed", [0, 1])
def test_deepnet_gradient_matches_finite_differences(seed):
    dims, th, cols, y, k = _case(seed=seed)
    loss, g, _ = dn.loss_grad(dims, k, th, cols, y)
    h = 1e-6
    rng = np.random.default_rng(seed + 10)
    for name, (off, shape) in dims.offsets().items():
        size = int(np.prod(shape))
        for idx in rng.choice(size, min(size, 6), replace=False):
            tp, tm = th.copy(), th.copy()
            tp[off + idx] += h
            tm[off + idx] -= h
            fd = (dn.loss_grad(dims, k, tp, cols, y)[0] - dn.loss_grad(dims, k, tm, cols, y)[0]) / (2 * h)
            assert abs(fd - g[off + idx]) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, g[off + idx])


def test_deepnet_colour_permutation_invariance():
    dims, th, cols, y, k = _case(n=14, widths=(10, 8), k=4, B=5, seed=3)
    sigma = np.random.default_rng(0).permutation(k)
    st = dims.initial_stats()
    a = dn.forward(dims, k, th, cols, True)
    b = dn.forward(dims, k, th, sigma[cols], True)
    assert np.allclose(a, b, rtol=0, atol=1e-12)
    st2 = st.copy()
    rng = np.random.default_rng(5)
    st2[:] = rng.uniform(0.5, 2.0, size=st2.shape)
    a = dn.forward(dims, k, th, cols, False, st2)
    b = dn.forward(dims, k, th, sigma[cols], False, st2)
    assert np.allclose(a, b, rtol=0, atol=1e-12)


def test_batch_normalisation_removes_scale_and_shift():
    """In training mode the normalisation makes the output independent of a positive rescaling of
    a layer's pre-activation (Lambda, Gamma, beta scaled together) and of a constant shift of it
    (beta shifted), up to the eps term."""
    dims, th, cols, y, k = _case(n=12, widths=(8, 6, 5), k=3, B=7, seed=4)
    base = dn.forward(dims, k, th, cols, True)
    t2 = th.copy()
    v = dims.view(t2)
    v["lam1"][:] *= 3.0
    v["gam1"][:] *= 3.0
    v["b1"][:] *= 3.0
    v["b0"][:] += 5.0
    v["b2"][:] -= 2.0
    got = dn.forward(dims, k, t2, cols, True)
    assert np.allclose(got, base, rtol=0, atol=1e-4 * max(1.0, np.abs(base).max()))
    # a scale the eps term cannot hide: the output changes when the normalisation is dropped
    # (evaluation mode with the initial running estimates)
    st = dims.initial_stats()
    assert not np.allclose(dn.forward(dims, k, t2, cols, False, st), dn.forward(dims, k, th, cols, False, st))


def test_identity_normalisation_reduces_to_the_plain_network():
    """Evaluation mode with running mean 0, running variance 1 - eps, gamma = 1 and mu = 0 makes
    every normalisation the identity; the network is then the plain invariant network of the C++
    oracle (64-d embedding, three 256-wide layers, linear head), parameter for parameter."""
    n, k, B = 30, 5, 4
    sd = oracle.ScorerDims(n)
    th0 = oracle.scorer_init(sd, seed=7)
    dims = dn.DeepDims(n, [sd.d0] + [sd.d] * sd.nl)
    th = np.zeros(dims.nparams())
    v = dims.view(th)
    for name, (off, shape) in sd.offsets().items():
        v[name][:] = th0[off:off + int(np.prod(shape))].reshape(shape)
    for l in range(len(dims.widths)):
        v[f"g{l}"][:] = 1.0
    st = dims.initial_stats()
    for _, var in dims.stats_view(st):
        var[:] = 1.0 - dn.EPS
    cols = inputs.random_colorings(B, n, k, seed=2)
    got = dn.forward(dims, k, th, cols, False, st)
    ref = oracle.scorer_forward(sd, k, th0, cols)
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_running_estimates_reproduce_the_batch_statistics():
    """After one training-mode pass from mean 0 / variance 1, the running estimates hold
    0.1 x the batch mean and 0.9 + 0.1 x the unbiased batch variance of every layer; evaluation
    with the batch statistics recovered from them (biased variance) equals the training pass."""
    dims, th, cols, y, k = _case(n=13, widths=(9, 7, 6), k=4, B=5, seed=6)
    st = dims.initial_stats()
    train_out = dn.forward(dims, k, th, cols, True, st)
    R = cols.shape[0] * k
    rec = st.copy()
    for m, var in dims.stats_view(rec):
        m[:] = m / dn.MOMENTUM
        var[:] = (var - (1 - dn.MOMENTUM)) / dn.MOMENTUM * (R - 1) / R
    eval_out = dn.forward(dims, k, th, cols, False, rec)
    assert np.allclose(eval_out, train_out, rtol=1e-9, atol=1e-9)


def test_training_reduces_the_loss():
    dims, th, cols, y, k = _case(n=12, widths=(10, 8, 6), k=3, B=40, seed=8)
    fvals = np.random.default_rng(3).integers(0, 30, size=cols.shape[0]).astype(np.int64)
    f = fvals.astype(np.float64)
    yy = (f - f.mean()) / f.std()
    st = dims.initial_stats()
    before = dn.loss_grad(dims, k, th, cols, yy)[0]
    am, av = np.zeros_like(th), np.zeros_like(th)
    dn.train(dims, k, th, am, av, 0, st, cols, fvals, epochs=30, b=10, lr=1e-2, seed=1, gen=0)
    after = dn.loss_grad(dims, k, th, cols, yy)[0]
    assert after < 0.5 * before
