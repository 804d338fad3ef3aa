"""FP64 oracle of the paper-size colour-permutation invariant network with invariant batch
normalisation.

TEST INFRASTRUCTURE ONLY: the tests and ``bench.py``'s CPU legs are the only callers; the CUDA
library never imports it.

Network (section "Deep neural network training"): for a colouring S with k classes,
f(S) = (1/k) sum_i (phi_P o ... o phi_0 (S))_i, where layer j maps the k class rows H_i
(k x l) to LeakyReLU_0.2(BN(beta + H_i Lambda + rho(H) Gamma)), rho(H) the mean of the k rows.
The input rows are the classes' indicator vectors over V, so layer 0 is the sum of the rows
E[v] = Lambda_0[v] over each class (plus beta_0; rho Gamma_0 is the same for every partition and
is folded into beta_0). BN is the invariant batch normalisation (same section): per feature,
mean and variance over the mini-batch and all k classes, y = (x - E[x]) / sqrt(Var[x] + eps) *
gamma + mu, eps = 1e-5; in training the batch statistics are used and running estimates are kept
with momentum 0.1 (the running variance unbiased, as in the batch normalisation paper's
implementation); in evaluation the running estimates are used. The output layer is linear
(L = 1, no BN), averaged over the classes. Hidden widths (section "Implementation and parameter
setting"): 10|V|, 5|V|, 2|V| x 5, |V|, |V|//2 for k-COL and 5|V|, 2|V|, |V|, |V|//2 for the WVCP.
Reading: gamma and mu are per-feature vectors (the text's "in R" read as one value per feature).

Flat parameter order: E [n][h1], b0 [h1], g0 [h1], mu0 [h1]; for l = 1 .. H-1: lam_l [h_l][h_l+1],
gam_l [h_l][h_l+1], b_l [h_l+1], g_l [h_l+1], mu_l [h_l+1]; then wh [h_H], bh [1]. Running
statistics (not parameters): for each of the H normalisations, mean [h] and variance [h].
"""
from __future__ import annotations

import numpy as np

EPS = 1e-5
MOMENTUM = 0.1
SLOPE = 0.2


def paper_widths(n: int, problem: str) -> list[int]:
    if problem == "col":
        return [10 * n, 5 * n, 2 * n, 2 * n, 2 * n, 2 * n, 2 * n, n, n // 2]
    if problem == "wvcp":
        return [5 * n, 2 * n, n, n // 2]
    raise ValueError(problem)


class DeepDims:
    def __init__(self, n: int, widths):
        self.n = int(n)
        self.widths = [int(w) for w in widths]
        if not self.widths or min(self.widths) < 1:
            raise ValueError("at least one hidden layer of positive width")

    def blocks(self):
        h = self.widths
        out = [("E", (self.n, h[0])), ("b0", (h[0],)), ("g0", (h[0],)), ("mu0", (h[0],))]
        for l in range(1, len(h)):
            out += [(f"lam{l}", (h[l - 1], h[l])), (f"gam{l}", (h[l - 1], h[l])), (f"b{l}", (h[l],)),
                    (f"g{l}", (h[l],)), (f"mu{l}", (h[l],))]
        out += [("wh", (h[-1],)), ("bh", (1,))]
        return out

    def offsets(self) -> dict:
        o, pos = {}, 0
        for name, shape in self.blocks():
            o[name] = (pos, shape)
            pos += int(np.prod(shape))
        return o

    def nparams(self) -> int:
        return sum(int(np.prod(s)) for _, s in self.blocks())

    def nstats(self) -> int:
        return 2 * sum(self.widths)

    def view(self, th):
        return {name: th[off:off + int(np.prod(shape))].reshape(shape) for name, (off, shape) in self.offsets().items()}

    def stats_view(self, st):
        out, pos = [], 0
        for h in self.widths:
            out.append((st[pos:pos + h], st[pos + h:pos + 2 * h]))
            pos += 2 * h
        return out

    def initial_stats(self) -> np.ndarray:
        st = np.zeros(self.nstats(), np.float64)
        for _, var in self.stats_view(st):
            var[:] = 1.0
        return st


def _class_sums(E, cols, k):
    B, n = cols.shape
    Z = np.zeros((B, k, E.shape[1]), np.float64)
    for b in range(B):
        np.add.at(Z[b], cols[b].astype(np.int64), E)
    return Z


def forward(dims: DeepDims, k, th, cols, train: bool, stats=None, cache=None):
    """Scores of the colourings cols [B][n]. train = True: batch statistics (and, when stats is
    given, the running estimates updated in place); train = False: the running estimates in
    stats. cache (a list) receives what the backward pass needs."""
    p = dims.view(np.asarray(th, np.float64))
    cols = np.atleast_2d(np.asarray(cols))
    B = cols.shape[0]
    sv = dims.stats_view(stats) if stats is not None else None
    H = None
    Z = _class_sums(p["E"], cols, k) + p["b0"]
    nl = len(dims.widths)
    for l in range(nl):
        if l > 0:
            rho = H.mean(axis=1)
            Z = H @ p[f"lam{l}"] + (rho @ p[f"gam{l}"])[:, None, :] + p[f"b{l}"]
        if train:
            m = Z.mean(axis=(0, 1))
            var = Z.var(axis=(0, 1))
            if sv is not None:
                R = B * k
                sv[l][0][:] = (1 - MOMENTUM) * sv[l][0] + MOMENTUM * m
                sv[l][1][:] = (1 - MOMENTUM) * sv[l][1] + MOMENTUM * var * (R / max(R - 1, 1))
        else:
            m, var = sv[l]
        inv = 1.0 / np.sqrt(var + EPS)
        xhat = (Z - m) * inv
        y = xhat * p[f"g{l}"] + p[f"mu{l}"]
        Hn = np.where(y > 0, y, SLOPE * y)
        if cache is not None:
            cache.append({"H": H, "xhat": xhat, "inv": inv, "y": y})
        H = Hn
    out = (H @ p["wh"]).mean(axis=1) + p["bh"][0]
    if cache is not None:
        cache.append({"H": H})
    return out


def loss_grad(dims: DeepDims, k, th, cols, y, stats=None):
    """Mean squared error of a training-mode batch and its gradient (flat, the parameter order)."""
    cols = np.atleast_2d(np.asarray(cols))
    y = np.asarray(y, np.float64)
    B = cols.shape[0]
    cache = []
    out = forward(dims, k, th, cols, True, stats, cache)
    loss = float(np.mean((out - y) ** 2))
    p = dims.view(np.asarray(th, np.float64))
    g = np.zeros(dims.nparams(), np.float64)
    gv = dims.view(g)
    dout = 2.0 * (out - y) / B
    HH = cache[-1]["H"]
    gv["bh"][0] = dout.sum()
    gv["wh"][:] = (dout[:, None] * HH.mean(axis=1)).sum(axis=0)
    dH = np.broadcast_to((dout[:, None, None] * p["wh"][None, None, :]) / k, HH.shape).copy()
    nl = len(dims.widths)
    for l in range(nl - 1, -1, -1):
        c = cache[l]
        dy = dH * np.where(c["y"] > 0, 1.0, SLOPE)
        xhat, inv = c["xhat"], c["inv"]
        gv[f"g{l}"][:] = (dy * xhat).sum(axis=(0, 1))
        gv[f"mu{l}"][:] = dy.sum(axis=(0, 1))
        dxh = dy * p[f"g{l}"]
        dZ = inv * (dxh - dxh.mean(axis=(0, 1)) - xhat * (dxh * xhat).mean(axis=(0, 1)))
        gv[f"b{l}"][:] = dZ.sum(axis=(0, 1))
        if l > 0:
            Hin = c["H"]
            rho = Hin.mean(axis=1)
            drho = dZ.sum(axis=1)
            gv[f"lam{l}"][:] = np.einsum("bki,bko->io", Hin, dZ)
            gv[f"gam{l}"][:] = rho.T @ drho
            dH = dZ @ p[f"lam{l}"].T + ((drho @ p[f"gam{l}"].T) / k)[:, None, :]
        else:
            dE = np.zeros_like(p["E"])
            for b in range(B):
                dE += dZ[b][cols[b].astype(np.int64)]
            gv["E"][:] = dE
    return loss, g, out


def init_params(dims: DeepDims, rng) -> np.ndarray:
    """Uniform +-1/sqrt(fan_in) weights and biases, BN gamma = 1 and mu = 0 (for tests; the CUDA
    library draws its own initial parameters)."""
    th = np.zeros(dims.nparams(), np.float64)
    v = dims.view(th)
    h = dims.widths
    for name, (off, shape) in dims.offsets().items():
        if name.startswith("g") and not name.startswith("gam"):
            v[name][:] = 1.0
            continue
        if name.startswith("mu"):
            continue
        if name in ("E", "b0"):
            fan = dims.n
        elif name in ("wh", "bh"):
            fan = h[-1]
        else:
            lidx = int(name.lstrip("lamgb"))
            fan = h[lidx - 1]
        v[name][:] = rng.uniform(-1.0, 1.0, size=shape) / np.sqrt(fan)
    return th


def epoch_order(p: int, seed, epoch: int, gen: int) -> np.ndarray:
    """The visiting order of the p samples in one epoch: sorted by the keys
    Philox(a = i, b = epoch, c = generation, tag = BATCH).r0, ties by i."""
    from . import TAG_BATCH, draw

    keys = [(int(draw(seed, i, epoch, gen, TAG_BATCH)[0]), i) for i in range(p)]
    return np.array([i for _, i in sorted(keys)], np.int64)


def train(dims: DeepDims, k, th, am, av, adam_t, stats, cols, fvals, epochs, b, lr, seed, gen):
    """Online training as in section "Deep neural network training": targets standardised by
    their mean and (population) standard deviation, N epochs of Adam (lr, betas 0.9 / 0.999,
    eps 1e-8) over batches of b samples in the epoch order; th, am, av and stats are updated in
    place. Returns (last loss, new adam_t)."""
    from . import adam_step

    cols = np.asarray(cols)
    f = np.asarray(fvals, np.float64)
    sd = f.std()
    y = (f - f.mean()) / (sd if sd > 0 else 1.0)
    p = cols.shape[0]
    loss = 0.0
    t = int(adam_t)
    for e in range(epochs):
        order = epoch_order(p, seed, e, gen)
        for s0 in range(0, p, b):
            idx = order[s0:s0 + b]
            loss, g, _ = loss_grad(dims, k, th, cols[idx], y[idx], stats)
            t += 1
            adam_step(th, am, av, g, t, lr)
    return loss, t
