"""Python access to the DLMCOL oracle (``dlmcol_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers. The CUDA library and its binding never import this package.

The oracle is plain single-threaded C++ compiled with g++ (``build()``); these wrappers only
marshal numpy arrays into it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dlmcol_oracle.cpp")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Philox stream tags (counter word 3); the CUDA library defines the same numbers independently.
TAG_INIT, TAG_TABU, TAG_GPX, TAG_SELECT, TAG_NNINIT, TAG_BATCH, TAG_WINIT = 1, 2, 3, 4, 7, 8, 9


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (g++ -O2, no CUDA)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            _declare(_lib)
    return _lib


_P = ctypes.c_void_p
_i32, _i64, _u32, _u64, _f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double


def _declare(L):
    sig = {
        "oracle_philox4x32_10": (None, [_P, _P, _P]),
        "oracle_draw": (None, [_u64, _u32, _u32, _u32, _u32, _P]),
        "oracle_graph_csr": (None, [_i32, _P, _P, _P, _P]),
        "oracle_init_colors": (None, [_i32, _i32, _i32, _u64, _u32, _P]),
        "oracle_gamma": (_i64, [_i32, _P, _i32, _P, _P]),
        "oracle_tabucol": (_i32, [_i32, _P, _i32, _P, _i64, _i32, _i32, _i32, _u64, _u32, _u32,
                                  _P, _P, _P, _P, _P, _i32]),
        "oracle_gpx": (None, [_i32, _i32, _P, _P, _u64, _u32, _u32, _P]),
        "oracle_distance": (_i32, [_i32, _i32, _P, _P]),
        "oracle_distance_matrix": (None, [_i32, _i32, _P, _i32, _P, _i32, _P]),
        "oracle_pool_update": (None, [_i32, _i32, _P, _P, _P]),
        "oracle_knn": (None, [_i32, _P, _i32, _P]),
        "oracle_scorer_nparams": (ctypes.c_size_t, [_i32, _i32, _i32, _i32]),
        "oracle_scorer_init": (None, [_i32, _i32, _i32, _i32, _u64, _P]),
        "oracle_scorer_forward": (None, [_i32, _i32, _i32, _i32, _i32, _P, _P, _i32, _P]),
        "oracle_scorer_loss_grad": (_f64, [_i32, _i32, _i32, _i32, _i32, _P, _P, _P, _i32, _P, _P]),
        "oracle_adam_step": (None, [_i64, _P, _P, _P, _P, _i64, _f64]),
        "oracle_scorer_train": (_f64, [_i32, _i32, _i32, _i32, _i32, _P, _P, _P, _P, _i32, _P, _P,
                                       _i32, _i32, _f64, _u64, _u32]),
        "oracle_memetic_generation": (_i32, [_i32, _P, _i32, _i32, _i32, _P, _P, _P, _P, _i64, _i32,
                                             _i32, _i32, _i32, _i32, _i32, _i32, _P, _P, _P, _P, _i32,
                                             _i32, _f64, _P, _u64, _u32, _P, _P, _P, _P]),
        "oracle_wvcp_score": (_i64, [_i32, _P, _P, _i32, _P, _P]),
        "oracle_wvcp_memetic_generation": (_i32, [_i32, _P, _P, _i32, _i32, _i32, _P, _P, _P, _P, _i64, _i32, _i32,
                                                  _i32, _i32, _i64, _i64, _i64, _i32, _i32, _i32, _i32, _P, _P, _P,
                                                  _P, _i32, _i32, _f64, _P, _u64, _u32, _P, _P, _P, _P]),
        "oracle_wvcp_greedy": (_i32, [_i32, _P, _P, _u64, _u32, _P]),
        "oracle_wvcp_tabu": (_i32, [_i32, _P, _P, _i32, _P, _i64, _i32, _i32, _i32, _i64, _u64, _u32,
                                    _u32, _P, _P, _P, _P, _P, _i32]),
        "oracle_wvcp_tabu_scaled": (_i32, [_i32, _P, _P, _i32, _P, _i64, _i32, _i32, _i32, _i64, _i64, _u64,
                                           _u32, _u32, _P, _P, _P, _P, _P, _i32]),
        "oracle_wvcp_iterated": (_i32, [_i32, _P, _P, _i32, _P, _i64, _i32, _i32, _i32, _i32, _i64, _i64, _i64,
                                        _u64, _u32, _u32, _P, _P, _P, _P]),
    }
    for name, (res, args) in sig.items():
        if not hasattr(L, name):
            continue
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------------------------
# numpy wrappers
# ---------------------------------------------------------------------------------------------
def philox(ctr, key) -> np.ndarray:
    c = _c(ctr, np.uint32)
    k = _c(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def draw(seed, a, b, c, tag) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().oracle_draw(seed, a, b, c, tag, _ptr(out))
    return out


def graph_csr(adj: np.ndarray):
    adj = _c(adj, np.uint8)
    n = adj.shape[0]
    m2 = int(adj.sum() - np.trace(adj))
    off = np.zeros(n + 1, np.int32)
    idx = np.zeros(max(m2, 1), np.int32)
    words = (n + 31) // 32
    bits = np.zeros((n, words), np.uint32)
    lib().oracle_graph_csr(n, _ptr(adj), _ptr(off), _ptr(idx), _ptr(bits))
    return off, idx[:m2], bits


def init_colors(n, k, pop, seed, ind_base=0) -> np.ndarray:
    col = np.zeros((pop, n), np.int16)
    lib().oracle_init_colors(n, k, pop, seed, ind_base, _ptr(col))
    return col


def gamma(adj, k, col):
    adj = _c(adj, np.uint8)
    col = _c(col, np.int16)
    n = adj.shape[0]
    g = np.zeros((n, k), np.int32)
    f = lib().oracle_gamma(n, _ptr(adj), k, _ptr(col), _ptr(g))
    return g, int(f)


def tabucol(adj, k, col, iters, seed, ind, gen=0, L_max=9, alpha=(6, 10), trace=False, check=False):
    """Returns dict(best_col, best_f, moves, iters, trace)."""
    adj = _c(adj, np.uint8)
    col = _c(col, np.int16)
    n = adj.shape[0]
    best = np.zeros(n, np.int16)
    bf, mv, it = np.zeros(1, np.int64), np.zeros(1, np.int64), np.zeros(1, np.int64)
    tr = np.full((iters, 4), -7, np.int32) if trace else None
    rc = lib().oracle_tabucol(n, _ptr(adj), k, _ptr(col), iters, L_max, alpha[0], alpha[1], seed, ind, gen,
                              _ptr(best), _ptr(bf), _ptr(mv), _ptr(it),
                              _ptr(tr) if trace else None, 1 if check else 0)
    if rc != 0:
        raise RuntimeError(f"oracle_tabucol failed with {rc}")
    res = dict(best_col=best, best_f=int(bf[0]), moves=int(mv[0]), iters=int(it[0]))
    if trace:
        res["trace"] = tr[: int(it[0])]
    return res


def gpx(k, A, B, seed, child_id, gen=0) -> np.ndarray:
    A = _c(A, np.int16)
    B = _c(B, np.int16)
    n = A.shape[0]
    child = np.zeros(n, np.int16)
    lib().oracle_gpx(n, k, _ptr(A), _ptr(B), seed, child_id, gen, _ptr(child))
    return child


def distance(k, A, B) -> int:
    A = _c(A, np.int16)
    B = _c(B, np.int16)
    return int(lib().oracle_distance(A.shape[0], k, _ptr(A), _ptr(B)))


def distance_matrix(k, X, Y) -> np.ndarray:
    X = _c(X, np.int16)
    Y = _c(Y, np.int16)
    out = np.zeros((X.shape[0], Y.shape[0]), np.int16)
    lib().oracle_distance_matrix(X.shape[1], k, _ptr(X), X.shape[0], _ptr(Y), Y.shape[0], _ptr(out))
    return out


def distance_exact(k, A, B) -> int:
    """Exact partition distance (section "Distance computation"): n minus the largest total
    class overlap over one-to-one matchings of the k classes of A with those of B. The overlap
    matrix is counted directly; the matching is a library assignment solver (scipy)."""
    from scipy.optimize import linear_sum_assignment

    A = np.asarray(A, np.int64)
    B = np.asarray(B, np.int64)
    M = np.zeros((k, k), np.int64)
    np.add.at(M, (A, B), 1)
    r, c = linear_sum_assignment(-M)
    return int(len(A) - M[r, c].sum())


def distance_exact_matrix(k, X, Y) -> np.ndarray:
    return np.array([[distance_exact(k, x, y) for y in Y] for x in X], np.int16).reshape(len(X), len(Y))


def pool_update(p, n, fit, D) -> np.ndarray:
    fit = _c(fit, np.int64)
    D = _c(D, np.int16)
    sel = np.zeros(p, np.int32)
    lib().oracle_pool_update(p, n, _ptr(fit), _ptr(D), _ptr(sel))
    return sel


def knn(D, K) -> np.ndarray:
    D = _c(D, np.int16)
    p = D.shape[0]
    nbr = np.zeros((p, K), np.int32)
    lib().oracle_knn(p, _ptr(D), K, _ptr(nbr))
    return nbr


class ScorerDims:
    def __init__(self, n, d0=64, d=256, nl=3):
        self.n, self.d0, self.d, self.nl = n, d0, d, nl

    @property
    def args(self):
        return (self.n, self.d0, self.d, self.nl)

    def nparams(self) -> int:
        return int(lib().oracle_scorer_nparams(*self.args))

    def offsets(self) -> dict:
        """Offsets of each parameter block in the flat parameter vector."""
        n, d0, d, nl = self.args
        o = {"E": (0, (n, d0))}
        pos = n * d0
        o["b0"] = (pos, (d0,))
        pos += d0
        for l in range(1, nl + 1):
            din = d0 if l == 1 else d
            o[f"lam{l}"] = (pos, (din, d))
            pos += din * d
            o[f"gam{l}"] = (pos, (din, d))
            pos += din * d
            o[f"b{l}"] = (pos, (d,))
            pos += d
        o["wh"] = (pos, (d,))
        pos += d
        o["bh"] = (pos, (1,))
        return o


def scorer_init(dims: ScorerDims, seed) -> np.ndarray:
    th = np.zeros(dims.nparams(), np.float64)
    lib().oracle_scorer_init(*dims.args, seed, _ptr(th))
    return th


def scorer_forward(dims: ScorerDims, k, th, cols) -> np.ndarray:
    th = _c(th, np.float64)
    cols = _c(np.atleast_2d(cols), np.int16)
    out = np.zeros(cols.shape[0], np.float64)
    lib().oracle_scorer_forward(*dims.args, k, _ptr(th), _ptr(cols), cols.shape[0], _ptr(out))
    return out


def scorer_loss_grad(dims: ScorerDims, k, th, cols, y):
    th = _c(th, np.float64)
    cols = _c(np.atleast_2d(cols), np.int16)
    y = _c(y, np.float64)
    grad = np.zeros_like(th)
    out = np.zeros(cols.shape[0], np.float64)
    loss = lib().oracle_scorer_loss_grad(*dims.args, k, _ptr(th), _ptr(cols), _ptr(y), cols.shape[0],
                                         _ptr(grad), _ptr(out))
    return float(loss), grad, out


def adam_step(th, m, v, g, t, lr):
    """In-place Adam step on float64 arrays."""
    g = _c(g, np.float64)
    lib().oracle_adam_step(th.size, _ptr(th), _ptr(m), _ptr(v), _ptr(g), t, lr)


def scorer_train(dims: ScorerDims, k, th, am, av, adam_t, cols, fvals, epochs, b, lr, seed, gen):
    """In-place training; returns (last loss, new adam_t)."""
    cols = _c(cols, np.int16)
    fvals = _c(fvals, np.int64)
    t = np.array([adam_t], np.int64)
    loss = lib().oracle_scorer_train(*dims.args, k, _ptr(th), _ptr(am), _ptr(av), _ptr(t), cols.shape[0],
                                     _ptr(cols), _ptr(fvals), epochs, b, lr, seed, gen)
    return float(loss), int(t[0])


class MemeticState:
    """State of the memetic loop (Algorithm 1) held as numpy arrays for the oracle."""

    def __init__(self, adj, k, p, K, seed, iters, use_scorer, d0=64, d=256, nl=3, epochs=5, batch=100,
                 lr=1e-3, L_max=9, alpha=(6, 10)):
        self.adj = _c(adj, np.uint8)
        self.n = self.adj.shape[0]
        self.k, self.p, self.K, self.seed, self.iters = k, p, K, seed, iters
        self.use_scorer = 1 if use_scorer else 0
        self.dims = ScorerDims(self.n, d0, d, nl)
        self.epochs, self.batch, self.lr, self.L_max, self.alpha = epochs, batch, lr, L_max, alpha
        self.P = init_colors(self.n, k, p, seed)
        self.fP = np.array([gamma(self.adj, k, c)[1] for c in self.P], np.int64)
        self.DP = distance_matrix(k, self.P, self.P)
        self.SO = self.P.copy()
        self.th = scorer_init(self.dims, seed)
        self.am = np.zeros_like(self.th)
        self.av = np.zeros_like(self.th)
        self.adam_t = np.zeros(1, np.int64)
        self.best_col = np.zeros(self.n, np.int16)
        self.best_f = np.array([np.iinfo(np.int64).max], np.int64)
        self.gen = 0

    def generation(self, ext_scores=None):
        fprime = np.zeros(self.p, np.int64)
        pick = np.zeros(self.p, np.int32)
        ext = None if ext_scores is None else _c(ext_scores, np.float32)
        rc = lib().oracle_memetic_generation(
            self.n, _ptr(self.adj), self.k, self.p, self.K, _ptr(self.P), _ptr(self.fP), _ptr(self.DP),
            _ptr(self.SO), self.iters, self.L_max, self.alpha[0], self.alpha[1], self.use_scorer,
            self.dims.d0, self.dims.d, self.dims.nl, _ptr(self.th), _ptr(self.am), _ptr(self.av),
            _ptr(self.adam_t), self.epochs, self.batch, self.lr, _ptr(ext) if ext is not None else None,
            self.seed, self.gen, _ptr(self.best_col), _ptr(self.best_f), _ptr(fprime), _ptr(pick))
        if rc != 0:
            raise RuntimeError(f"oracle_memetic_generation failed with {rc}")
        self.gen += 1
        return fprime, pick


def wvcp_tabu(adj, w, k, col, iters, phi, seed, ind, gen=0, fscale=1, L_max=9, alpha=(2, 10), trace=False,
              check=False):
    """Feasible/infeasible tabu search on g = fscale f + phi c; dict(best_col, best_g, f, c, moves, trace)."""
    adj = _c(adj, np.uint8)
    w = _c(w, np.int32)
    col = _c(col, np.int16)
    n = adj.shape[0]
    best = np.zeros(n, np.int16)
    bg, fc, mv = np.zeros(1, np.int64), np.zeros(2, np.int64), np.zeros(1, np.int64)
    tr = np.full((iters, 4), -7, np.int32) if trace else None
    rc = lib().oracle_wvcp_tabu_scaled(n, _ptr(adj), _ptr(w), k, _ptr(col), iters, L_max, alpha[0], alpha[1], fscale,
                                       phi, seed, ind, gen, _ptr(best), _ptr(bg), _ptr(fc), _ptr(mv),
                                       _ptr(tr) if trace else None, 1 if check else 0)
    if rc != 0:
        raise RuntimeError(f"oracle_wvcp_tabu_scaled failed ({rc})")
    return dict(best_col=best, best_g=int(bg[0]), f=int(fc[0]), c=int(fc[1]), moves=int(mv[0]), trace=tr)


def wvcp_iterated(adj, w, k, col, iters, max_ls, fscale, phi0, phi_last, seed, ind, gen=0, L_max=9, alpha=(2, 10)):
    """Iterated feasible/infeasible tabu search (Algorithm 2) of one individual:
    dict(best_col, best_f (-1: never legal), phi (per search), fc (per search))."""
    adj = _c(adj, np.uint8)
    w = _c(w, np.int32)
    col = _c(col, np.int16)
    n = adj.shape[0]
    best = np.zeros(n, np.int16)
    bf = np.zeros(1, np.int64)
    phis = np.zeros(max_ls, np.int64)
    fcs = np.zeros((max_ls, 2), np.int64)
    rc = lib().oracle_wvcp_iterated(n, _ptr(adj), _ptr(w), k, _ptr(col), iters, max_ls, L_max, alpha[0], alpha[1],
                                    fscale, phi0, phi_last, seed, ind, gen, _ptr(best), _ptr(bf), _ptr(phis), _ptr(fcs))
    if rc != 0:
        raise RuntimeError(f"oracle_wvcp_iterated failed ({rc})")
    return dict(best_col=best, best_f=int(bf[0]), phi=phis, fc=fcs)


def wvcp_greedy(adj, w, seed, ind=0):
    """Randomised greedy WVCP initialisation of one individual: (colouring, colours opened)."""
    adj = _c(adj, np.uint8)
    w = _c(w, np.int32)
    n = adj.shape[0]
    col = np.zeros(n, np.int16)
    used = lib().oracle_wvcp_greedy(n, _ptr(adj), _ptr(w), seed, ind, _ptr(col))
    return col, int(used)


def wvcp_score(adj, w, k, col):
    """(f, conflicts) of a colouring (Eq. score_WVCP)."""
    adj = _c(adj, np.uint8)
    w = _c(w, np.int32)
    col = _c(col, np.int16)
    conf = np.zeros(1, np.int64)
    f = lib().oracle_wvcp_score(adj.shape[0], _ptr(adj), _ptr(w), k, _ptr(col), _ptr(conf))
    return int(f), int(conf[0])


class WvcpMemeticState(MemeticState):
    """State of Algorithm 1 for the WVCP: the initial population from the randomised greedy
    initialisation (individual i with stream i), fitness = WVCP score, the iterated feasible and
    infeasible tabu search (Algorithm 2) as the local search."""

    def __init__(self, adj, w, k, p, K, seed, iters, max_ls, fscale, phi0, phi_last, use_scorer, d0=64, d=256,
                 nl=3, epochs=5, batch=100, lr=1e-3, L_max=9, alpha=(2, 10)):
        self.adj = _c(adj, np.uint8)
        self.w = _c(w, np.int32)
        self.n = self.adj.shape[0]
        self.k, self.p, self.K, self.seed, self.iters = k, p, K, seed, iters
        self.max_ls, self.fscale, self.phi0, self.phi_last = max_ls, fscale, phi0, phi_last
        self.use_scorer = 1 if use_scorer else 0
        self.dims = ScorerDims(self.n, d0, d, nl)
        self.epochs, self.batch, self.lr, self.L_max, self.alpha = epochs, batch, lr, L_max, alpha
        cols = [wvcp_greedy(self.adj, self.w, seed, i) for i in range(p)]
        if max(u for _, u in cols) > k:
            raise ValueError("the greedy initialisation opens more than k colours")
        self.P = np.stack([c for c, _ in cols]).astype(np.int16)
        self.fP = np.array([wvcp_score(self.adj, self.w, k, c)[0] for c in self.P], np.int64)
        self.DP = distance_matrix(k, self.P, self.P)
        self.SO = self.P.copy()
        self.th = scorer_init(self.dims, seed)
        self.am = np.zeros_like(self.th)
        self.av = np.zeros_like(self.th)
        self.adam_t = np.zeros(1, np.int64)
        self.best_col = np.zeros(self.n, np.int16)
        self.best_f = np.array([np.iinfo(np.int64).max], np.int64)
        self.gen = 0

    def generation(self, ext_scores=None):
        fprime = np.zeros(self.p, np.int64)
        pick = np.zeros(self.p, np.int32)
        ext = None if ext_scores is None else _c(ext_scores, np.float32)
        rc = lib().oracle_wvcp_memetic_generation(
            self.n, _ptr(self.adj), _ptr(self.w), self.k, self.p, self.K, _ptr(self.P), _ptr(self.fP), _ptr(self.DP),
            _ptr(self.SO), self.iters, self.max_ls, self.L_max, self.alpha[0], self.alpha[1], self.fscale, self.phi0,
            self.phi_last, self.use_scorer, self.dims.d0, self.dims.d, self.dims.nl, _ptr(self.th), _ptr(self.am),
            _ptr(self.av), _ptr(self.adam_t), self.epochs, self.batch, self.lr, _ptr(ext) if ext is not None else None,
            self.seed, self.gen, _ptr(self.best_col), _ptr(self.best_f), _ptr(fprime), _ptr(pick))
        if rc != 0:
            raise RuntimeError(f"oracle_wvcp_memetic_generation failed with {rc}")
        self.gen += 1
        return fprime, pick
