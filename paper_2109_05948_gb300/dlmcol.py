"""Thin ctypes binding of ``libdlmcol.so`` (C-ABI in ``include/dlmcol.h``).

The functions keep the C names. They only marshal arguments: torch tensors are passed by their
device pointers, streams by their CUDA handles. Every step of the computation runs in the CUDA
library; importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdlmcol.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "dlmcol.h")

DLM_OK, DLM_EINVAL, DLM_ENOMEM, DLM_ECUDA, DLM_ETIMEOUT, DLM_ECANCELLED, DLM_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "DLM_OK", -1: "DLM_EINVAL", -2: "DLM_ENOMEM", -3: "DLM_ECUDA", -4: "DLM_ETIMEOUT",
                -5: "DLM_ECANCELLED", -6: "DLM_EUNSUPPORTED"}


class DlmError(RuntimeError):
    def __init__(self, status, msg=""):
        self.status = status
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")


class Tenure(ctypes.Structure):
    _fields_ = [("L_max", ctypes.c_int32), ("alpha_num", ctypes.c_int32), ("alpha_den", ctypes.c_int32)]


class MemeticParams(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("p", ctypes.c_int32), ("K", ctypes.c_int32), ("iters", ctypes.c_int64),
                ("tenure", Tenure), ("use_scorer", ctypes.c_int32), ("epochs", ctypes.c_int32),
                ("batch", ctypes.c_int32), ("lr", ctypes.c_float), ("seed", ctypes.c_uint64),
                ("problem", ctypes.c_int32), ("max_ls", ctypes.c_int32)]


class TabuOpts(ctypes.Structure):
    _fields_ = [("warps_per_individual", ctypes.c_int32), ("ring", ctypes.c_int32), ("legacy", ctypes.c_int32),
                ("entry_bits", ctypes.c_int32)]


COL_TENURE = Tenure(9, 6, 10)    # Table params-COL: alpha = 0.6, L in 0..9
WVCP_TENURE = Tenure(9, 2, 10)   # Table params-WVCP: alpha = 0.2 (times |V|), L in 0..9

_P = ctypes.c_void_p
_i32, _i64, _u32, _u64, _f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_float
_PP = ctypes.POINTER(ctypes.c_void_p)

_SIGS = {
    "dlm_create": (_i32, [_PP, _i32, _P]),
    "dlm_destroy": (None, [_P]),
    "dlm_set_stream": (_i32, [_P, _P]),
    "dlm_set_cancel_flag": (_i32, [_P, _P]),
    "dlm_last_error": (ctypes.c_char_p, [_P]),
    "dlm_sync": (_i32, [_P]),
    "dlm_graph_create": (_i32, [_P, _i32, _i64, _P, _P, _PP]),
    "dlm_graph_destroy": (None, [_P]),
    "dlm_graph_n": (_i32, [_P]),
    "dlm_graph_m": (_i64, [_P]),
    "dlm_graph_export": (_i32, [_P, _P, _P, _P, _P]),
    "dlm_init_colors": (_i32, [_P, _i32, _i32, _i32, _u64, _u32, _P]),
    "dlm_gamma": (_i32, [_P, _P, _i32, _i32, _P, _P, _P]),
    "dlm_tabucol_batch": (_i32, [_P, _P, _i32, _i32, _P, _P, _P, _i64, Tenure, _u64, _u32, _u32]),
    "dlm_tabucol_batch_ex": (_i32, [_P, _P, _i32, _i32, _P, _P, _P, _i64, Tenure, _u64, _u32, _u32, _i32, _P, _P]),
    "dlm_tabucol_batch_opts": (_i32, [_P, _P, _i32, _i32, _P, _P, _P, _i64, Tenure, _u64, _u32, _u32, _P, _P, _P]),
    "dlm_tabucol_multi": (_i32, [_P, _i32, _P, _P, _P, _P, _P, _P, _P, Tenure, _u64, _u32, _u32]),
    "dlm_tabucol_multi_noalloc": (_i32, [_P, _i32, _P, _P, _P, _P, _P, _P, _P, Tenure, _u64, _u32, _u32]),
    "dlm_tabucol_autotune": (_i32, [_P, _P, _i32, _i32, _i64, _P]),
    "dlm_tabucol_multi_plan_create": (_i32, [_P, _i32, _P, _P, _P, _P, _P, _P, _P, Tenure, _u64, _u32, _u32, _PP]),
    "dlm_tabucol_multi_plan_launch": (_i32, [_P, _P]),
    "dlm_tabucol_multi_plan_destroy": (None, [_P]),
    "dlm_gpx_batch": (_i32, [_P, _i32, _i32, _P, _i32, _P, _P, _i32, _P, _u64, _u32]),
    "dlm_distance_batch": (_i32, [_P, _i32, _i32, _P, _i32, _P, _i32, _P, _i64, _i32]),
    "dlm_distance_batch_ex": (_i32, [_P, _i32, _i32, _P, _i32, _P, _i32, _P, _i64, _i32, _i32]),
    "dlm_distance_exact_batch": (_i32, [_P, _i32, _i32, _P, _i32, _P, _i32, _P, _i64, _i32]),
    "dlm_deepnet_create": (_i32, [_P, _i32, _i32, _i32, _P, _u64, _P]),
    "dlm_deepnet_destroy": (None, [_P]),
    "dlm_deepnet_nparams": (_i64, [_P]),
    "dlm_deepnet_nstats": (_i64, [_P]),
    "dlm_deepnet_get": (_i32, [_P, _P, _i32, _P]),
    "dlm_deepnet_set": (_i32, [_P, _P, _i32, _P]),
    "dlm_deepnet_set_precision": (_i32, [_P, _P, _i32]),
    "dlm_deepnet_forward": (_i32, [_P, _P, _P, _i32, _i32, _P]),
    "dlm_deepnet_loss_grad": (_i32, [_P, _P, _P, _P, _i32, _P, _P, _P]),
    "dlm_deepnet_adam_step": (_i32, [_P, _P, _P, ctypes.c_float]),
    "dlm_deepnet_train": (_i32, [_P, _P, _P, _P, _i32, _i32, _i32, ctypes.c_float, _u64, _u32]),
    "dlm_deepnet_state_bytes": (_i64, [_P]),
    "dlm_deepnet_save": (_i32, [_P, _P, _P]),
    "dlm_deepnet_load": (_i32, [_P, _P, _P]),
    "dlm_pool_update": (_i32, [_P, _i32, _i32, _P, _P, _P]),
    "dlm_knn": (_i32, [_P, _i32, _P, _i32, _P]),
    "dlm_scorer_create": (_i32, [_P, _i32, _i32, _u64, _PP]),
    "dlm_scorer_destroy": (None, [_P]),
    "dlm_scorer_nparams": (_i64, [_P]),
    "dlm_scorer_get_params": (_i32, [_P, _P, _P]),
    "dlm_scorer_set_params": (_i32, [_P, _P, _P]),
    "dlm_score_offspring": (_i32, [_P, _P, _P, _i32, _P]),
    "dlm_scorer_set_scoring_precision": (_i32, [_P, _P, _i32]),
    "dlm_scorer_loss_grad": (_i32, [_P, _P, _P, _P, _i32, _P, _P, _P]),
    "dlm_scorer_train": (_i32, [_P, _P, _P, _P, _i32, _i32, _i32, _f32, _u64, _u32]),
    "dlm_memetic_create": (_i32, [_P, _P, _P, _PP]),
    "dlm_memetic_stats": (_i32, [_P, _P, _P]),
    "dlm_memetic_destroy": (None, [_P]),
    "dlm_memetic_step": (_i32, [_P, _P, _P]),
    "dlm_memetic_get": (_i32, [_P, _P, _i32, _P]),
    "dlm_memetic_set": (_i32, [_P, _P, _i32, _P]),
    "dlm_col_descend": (_i32, [_P, _P, _P, _i32, _P, _P, _P]),
    "dlm_memetic_profile": (_i32, [_P, _P, _i32, _P]),
    "dlm_memetic_found_ms": (_i32, [_P, _P, _P]),
    "dlm_memetic_state_bytes": (_i64, [_P]),
    "dlm_memetic_save": (_i32, [_P, _P, _P]),
    "dlm_memetic_load": (_i32, [_P, _P, _P]),
    "dlm_scorer_state_bytes": (_i64, [_P]),
    "dlm_scorer_save": (_i32, [_P, _P, _P]),
    "dlm_scorer_load": (_i32, [_P, _P, _P]),
    "dlm_probe_smem_bandwidth": (_i32, [_P, _P]),
    "dlm_probe_l2_bandwidth": (_i32, [_P, _P]),
    "dlm_tabucol_launch_info": (_i32, [_P, _P, _i32, _i32, _i32, _P]),
    "dlm_gemm_bf16": (_i32, [_P, _P, _P, _P, _i32, _i32, _i32]),
    "dlm_gemm_profile": (_i32, [_P, _i32]),
    "dlm_gemm_profile_read": (_i32, [_P, _P, _P, _P]),
    "dlm_wvcp_tabu_batch": (_i32, [_P, _P, _i32, _i32, _P, _P, _P, _P, _i64, Tenure, _i64, _u64, _u32, _u32]),
    "dlm_wvcp_tabu_batch_ex": (_i32, [_P, _P, _i32, _i32, _P, _P, _P, _P, _i64, Tenure, _i64, _u64, _u32, _u32, _P,
                                      _i32]),
    "dlm_wvcp_entry_bits": (_i32, [_P, _P, _i32, _P]),
    "dlm_wvcp_greedy": (_i32, [_P, _P, _i32, _u64, _u32, _P, _P]),
    "dlm_wvcp_iterated": (_i32, [_P, _P, _i32, _i32, _P, _P, _P, _i64, _i32, Tenure, _i32, _i64, _i64, _u64, _u32,
                                 _u32]),
}

_lib = None


def lib():
    """The loaded library; raises when it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_2109_05948_gb300.build.build() first")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            if hasattr(L, name):
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
        _lib = L
    return _lib


def header_symbols():
    """Names of the entry points declared in include/dlmcol.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(dlm_[a-z0-9_]+)\s*\(", txt)))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if hasattr(t, "__array_interface__"):  # numpy array in host memory
        return ctypes.c_void_p(t.__array_interface__["data"][0])
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        return None
    return ctypes.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


class Context:
    """dlm_ctx on one device and stream (default: torch's current stream)."""

    def __init__(self, device: int = 0, stream=None):
        import torch

        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        h = ctypes.c_void_p()
        st = lib().dlm_create(ctypes.byref(h), device, _stream_handle(stream))
        if st != DLM_OK:
            raise DlmError(st, "dlm_create")
        self.h = h

    def check(self, st, what=""):
        if st != DLM_OK:
            raise DlmError(st, f"{what}: {lib().dlm_last_error(self.h).decode()}")

    def set_stream(self, stream):
        self.check(lib().dlm_set_stream(self.h, _stream_handle(stream)), "dlm_set_stream")

    def sync(self):
        self.check(lib().dlm_sync(self.h), "dlm_sync")

    def close(self):
        if getattr(self, "h", None):
            lib().dlm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Graph:
    """dlm_graph built on the GPU from a device edge list [m][2] int32 (and weights [n] int32)."""

    def __init__(self, ctx: Context, n: int, edges, weights=None):
        h = ctypes.c_void_p()
        m = 0 if edges is None else int(edges.shape[0])
        ctx.check(lib().dlm_graph_create(ctx.h, n, m, _ptr(edges), _ptr(weights), ctypes.byref(h)), "dlm_graph_create")
        self.h, self.n = h, n
        self.m = int(lib().dlm_graph_m(h))

    def close(self):
        if getattr(self, "h", None):
            lib().dlm_graph_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------------------
# entry points (same names as the C ABI); tensors are device tensors of the documented dtype
# ------------------------------------------------------------------------------------------------
def dlm_graph_export(ctx, g, off, idx, bits):
    ctx.check(lib().dlm_graph_export(ctx.h, g.h, _ptr(off), _ptr(idx), _ptr(bits)), "dlm_graph_export")


def dlm_init_colors(ctx, n, k, pop, seed, ind_base, col):
    ctx.check(lib().dlm_init_colors(ctx.h, n, k, pop, seed, ind_base, _ptr(col)), "dlm_init_colors")


def dlm_gamma(ctx, g, k, pop, col, gamma, f):
    ctx.check(lib().dlm_gamma(ctx.h, g.h, k, pop, _ptr(col), _ptr(gamma), _ptr(f)), "dlm_gamma")


def dlm_tabucol_batch(ctx, g, k, pop, col, best_f, moves, iters, tenure=COL_TENURE, seed=0, generation=0,
                      ind_base=0):
    ctx.check(lib().dlm_tabucol_batch(ctx.h, g.h, k, pop, _ptr(col), _ptr(best_f), _ptr(moves), iters, tenure,
                                      seed, generation, ind_base), "dlm_tabucol_batch")


def dlm_tabucol_batch_ex(ctx, g, k, pop, col, best_f, moves, iters, tenure=COL_TENURE, seed=0, generation=0,
                         ind_base=0, warps=0, trace=None, work=None):
    ctx.check(lib().dlm_tabucol_batch_ex(ctx.h, g.h, k, pop, _ptr(col), _ptr(best_f), _ptr(moves), iters, tenure,
                                         seed, generation, ind_base, warps, _ptr(trace), _ptr(work)),
              "dlm_tabucol_batch_ex")


def dlm_tabucol_batch_opts(ctx, g, k, pop, col, best_f, moves, iters, tenure=COL_TENURE, seed=0, generation=0,
                           ind_base=0, warps=0, ring=0, legacy=0, trace=None, work=None, entry_bits=0):
    o = TabuOpts(warps, ring, legacy, entry_bits)
    ctx.check(lib().dlm_tabucol_batch_opts(ctx.h, g.h, k, pop, _ptr(col), _ptr(best_f), _ptr(moves), iters, tenure,
                                           seed, generation, ind_base, ctypes.byref(o), _ptr(trace), _ptr(work)),
              "dlm_tabucol_batch_opts")


def _multi_args(graphs, ks, pops, cols, best_fs, moves, iters):
    G = len(graphs)
    arr_g = (ctypes.c_void_p * G)(*[g.h.value for g in graphs])
    arr_k = (ctypes.c_int32 * G)(*ks)
    arr_p = (ctypes.c_int32 * G)(*pops)
    arr_c = (ctypes.c_void_p * G)(*[c.data_ptr() for c in cols])
    arr_b = (ctypes.c_void_p * G)(*[b.data_ptr() for b in best_fs])
    arr_m = (ctypes.c_void_p * G)(*[(m.data_ptr() if m is not None else 0) for m in moves]) if moves else None
    arr_i = (ctypes.c_int64 * G)(*iters)
    return G, arr_g, arr_k, arr_p, arr_c, arr_b, arr_m, arr_i


def dlm_tabucol_multi_noalloc(ctx, graphs, ks, pops, cols, best_fs, moves, iters, tenure=COL_TENURE, seed=0,
                              generation=0, ind_base=0):
    """dlm_tabucol_multi for callers that must not allocate device memory (see include/dlmcol.h)."""
    a = _multi_args(graphs, ks, pops, cols, best_fs, moves, iters)
    ctx.check(lib().dlm_tabucol_multi_noalloc(ctx.h, *a, tenure, seed, generation, ind_base),
              "dlm_tabucol_multi_noalloc")


def dlm_tabucol_multi(ctx, graphs, ks, pops, cols, best_fs, moves, iters, tenure=COL_TENURE, seed=0, generation=0,
                      ind_base=0):
    G = len(graphs)
    arr_g = (ctypes.c_void_p * G)(*[g.h.value for g in graphs])
    arr_k = (ctypes.c_int32 * G)(*ks)
    arr_p = (ctypes.c_int32 * G)(*pops)
    arr_c = (ctypes.c_void_p * G)(*[c.data_ptr() for c in cols])
    arr_b = (ctypes.c_void_p * G)(*[b.data_ptr() for b in best_fs])
    arr_m = (ctypes.c_void_p * G)(*[(m.data_ptr() if m is not None else 0) for m in moves]) if moves else None
    arr_i = (ctypes.c_int64 * G)(*iters)
    ctx.check(lib().dlm_tabucol_multi(ctx.h, G, arr_g, arr_k, arr_p, arr_c, arr_b, arr_m, arr_i, tenure, seed,
                                      generation, ind_base), "dlm_tabucol_multi")


def dlm_tabucol_autotune(ctx, g, k, pop, iters):
    best = ctypes.c_int32(0)
    ctx.check(lib().dlm_tabucol_autotune(ctx.h, g.h, k, pop, iters, ctypes.byref(best)), "dlm_tabucol_autotune")
    return best.value


def dlm_gpx_batch(ctx, n, k, parents, pop, pairs, child_id, m, children, seed, generation):
    ctx.check(lib().dlm_gpx_batch(ctx.h, n, k, _ptr(parents), pop, _ptr(pairs), _ptr(child_id), m, _ptr(children),
                                  seed, generation), "dlm_gpx_batch")


def dlm_distance_exact_batch(ctx, n, k, X, a, Y, b, D, ldD, upper=0):
    ctx.check(lib().dlm_distance_exact_batch(ctx.h, n, k, _ptr(X), a, _ptr(Y), b, _ptr(D), ldD, upper),
              "dlm_distance_exact_batch")


def dlm_distance_batch(ctx, n, k, X, a, Y, b, D, ldD, upper=0, method=None):
    if method is None:
        ctx.check(lib().dlm_distance_batch(ctx.h, n, k, _ptr(X), a, _ptr(Y), b, _ptr(D), ldD, upper),
                  "dlm_distance_batch")
    else:
        ctx.check(lib().dlm_distance_batch_ex(ctx.h, n, k, _ptr(X), a, _ptr(Y), b, _ptr(D), ldD, upper, method),
                  "dlm_distance_batch_ex")


def dlm_pool_update(ctx, p, n, fit, D, sel):
    ctx.check(lib().dlm_pool_update(ctx.h, p, n, _ptr(fit), _ptr(D), _ptr(sel)), "dlm_pool_update")


def dlm_knn(ctx, p, D, K, nbr):
    ctx.check(lib().dlm_knn(ctx.h, p, _ptr(D), K, _ptr(nbr)), "dlm_knn")


class Scorer:
    def __init__(self, ctx: Context, n: int, k: int, seed: int):
        h = ctypes.c_void_p()
        ctx.check(lib().dlm_scorer_create(ctx.h, n, k, seed, ctypes.byref(h)), "dlm_scorer_create")
        self.h, self.n, self.k = h, n, k
        self.nparams = int(lib().dlm_scorer_nparams(h))

    def close(self):
        if getattr(self, "h", None):
            lib().dlm_scorer_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dlm_scorer_get_params(ctx, s, params):
    ctx.check(lib().dlm_scorer_get_params(ctx.h, s.h, _ptr(params)), "dlm_scorer_get_params")


def dlm_scorer_set_params(ctx, s, params):
    ctx.check(lib().dlm_scorer_set_params(ctx.h, s.h, _ptr(params)), "dlm_scorer_set_params")


def dlm_scorer_set_scoring_precision(ctx, scorer, split):
    ctx.check(lib().dlm_scorer_set_scoring_precision(ctx.h, scorer.h, int(split)), "dlm_scorer_set_scoring_precision")


def dlm_score_offspring(ctx, s, col, c, out):
    ctx.check(lib().dlm_score_offspring(ctx.h, s.h, _ptr(col), c, _ptr(out)), "dlm_score_offspring")


def dlm_scorer_loss_grad(ctx, s, col, y, B, grad, out, loss):
    ctx.check(lib().dlm_scorer_loss_grad(ctx.h, s.h, _ptr(col), _ptr(y), B, _ptr(grad), _ptr(out), _ptr(loss)),
              "dlm_scorer_loss_grad")


def dlm_scorer_train(ctx, s, cols, fvals, p, epochs, b, lr, seed, generation):
    ctx.check(lib().dlm_scorer_train(ctx.h, s.h, _ptr(cols), _ptr(fvals), p, epochs, b, lr, seed, generation),
              "dlm_scorer_train")


class DeepNet:
    """The paper-size invariant network with invariant batch normalisation (dlm_deepnet_*)."""

    def __init__(self, ctx: Context, n, k, widths, seed=0):
        arr = (ctypes.c_int32 * len(widths))(*[int(w) for w in widths])
        h = ctypes.c_void_p()
        ctx.check(lib().dlm_deepnet_create(ctx.h, n, k, len(widths), arr, seed, ctypes.byref(h)), "dlm_deepnet_create")
        self.h, self.ctx = h, ctx
        self.nparams = int(lib().dlm_deepnet_nparams(h))
        self.nstats = int(lib().dlm_deepnet_nstats(h))

    def get(self, which, dst):
        self.ctx.check(lib().dlm_deepnet_get(self.ctx.h, self.h, which, _ptr(dst)), "dlm_deepnet_get")

    def set(self, which, src):
        self.ctx.check(lib().dlm_deepnet_set(self.ctx.h, self.h, which, _ptr(src)), "dlm_deepnet_set")

    def set_precision(self, split):
        self.ctx.check(lib().dlm_deepnet_set_precision(self.ctx.h, self.h, split), "dlm_deepnet_set_precision")

    def forward(self, col, c, train, out):
        self.ctx.check(lib().dlm_deepnet_forward(self.ctx.h, self.h, _ptr(col), c, train, _ptr(out)),
                       "dlm_deepnet_forward")

    def loss_grad(self, col, y, B, grad=None, out=None, loss=None):
        self.ctx.check(lib().dlm_deepnet_loss_grad(self.ctx.h, self.h, _ptr(col), _ptr(y), B, _ptr(grad), _ptr(out),
                                                   _ptr(loss)), "dlm_deepnet_loss_grad")

    def adam_step(self, grad, lr):
        self.ctx.check(lib().dlm_deepnet_adam_step(self.ctx.h, self.h, _ptr(grad), lr), "dlm_deepnet_adam_step")

    def train(self, cols, fvals, p, epochs, b, lr, seed, generation):
        self.ctx.check(lib().dlm_deepnet_train(self.ctx.h, self.h, _ptr(cols), _ptr(fvals), p, epochs, b, lr, seed,
                                               generation), "dlm_deepnet_train")

    def close(self):
        if getattr(self, "h", None):
            lib().dlm_deepnet_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Memetic:
    def __init__(self, ctx: Context, g: Graph, params: MemeticParams):
        h = ctypes.c_void_p()
        ctx.check(lib().dlm_memetic_create(ctx.h, g.h, ctypes.byref(params), ctypes.byref(h)), "dlm_memetic_create")
        self.h, self.params = h, params

    def close(self):
        if getattr(self, "h", None):
            lib().dlm_memetic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dlm_memetic_stats(ctx, mm):
    """dict of the last generation's diagnostics (include/dlmcol.h, dlm_memetic_stats)."""
    out = (ctypes.c_double * 8)()
    ctx.check(lib().dlm_memetic_stats(ctx.h, mm.h, out), "dlm_memetic_stats")
    keys = ("generation", "pred_pearson", "pred_rel_err", "f_mean", "f_min", "dist_mean", "dist_min", "dist_max")
    return dict(zip(keys, [float(x) for x in out]))


def dlm_memetic_step(ctx, mm):
    best = ctypes.c_int64(0)
    ctx.check(lib().dlm_memetic_step(ctx.h, mm.h, ctypes.byref(best)), "dlm_memetic_step")
    return best.value


def dlm_memetic_found_ms(ctx, mm):
    """ms from the start of the last generation to the end of its best-so-far update."""
    out = ctypes.c_double(0.0)
    ctx.check(lib().dlm_memetic_found_ms(ctx.h, mm.h, ctypes.byref(out)), "dlm_memetic_found_ms")
    return out.value


def dlm_memetic_get(ctx, mm, which, dst):
    ctx.check(lib().dlm_memetic_get(ctx.h, mm.h, which, _ptr(dst)), "dlm_memetic_get")


def dlm_memetic_set(ctx, mm, which, src):
    ctx.check(lib().dlm_memetic_set(ctx.h, mm.h, which, _ptr(src)), "dlm_memetic_set")


def dlm_set_cancel_flag(ctx, flag):
    """flag: an int32 tensor the device can read (CUDA or pinned host memory), or None."""
    ctx.check(lib().dlm_set_cancel_flag(ctx.h, _ptr(flag)), "dlm_set_cancel_flag")


def dlm_memetic_save(ctx, mm):
    """The checkpoint blob of the memetic state as a host numpy uint8 array."""
    import numpy as np

    buf = np.empty(int(lib().dlm_memetic_state_bytes(mm.h)), np.uint8)
    ctx.check(lib().dlm_memetic_save(ctx.h, mm.h, _ptr(buf)), "dlm_memetic_save")
    return buf


def dlm_memetic_load(ctx, mm, buf):
    import numpy as np

    buf = np.ascontiguousarray(buf, np.uint8)
    ctx.check(lib().dlm_memetic_load(ctx.h, mm.h, _ptr(buf)), "dlm_memetic_load")


def dlm_scorer_save(ctx, s):
    import numpy as np

    buf = np.empty(int(lib().dlm_scorer_state_bytes(s.h)), np.uint8)
    ctx.check(lib().dlm_scorer_save(ctx.h, s.h, _ptr(buf)), "dlm_scorer_save")
    return buf


def dlm_scorer_load(ctx, s, buf):
    import numpy as np

    buf = np.ascontiguousarray(buf, np.uint8)
    ctx.check(lib().dlm_scorer_load(ctx.h, s.h, _ptr(buf)), "dlm_scorer_load")


def dlm_gemm_bf16(ctx, A, B, C, M, N, K):
    ctx.check(lib().dlm_gemm_bf16(ctx.h, _ptr(A), _ptr(B), _ptr(C), M, N, K), "dlm_gemm_bf16")


def dlm_gemm_profile(ctx, enable):
    ctx.check(lib().dlm_gemm_profile(ctx.h, 1 if enable else 0), "dlm_gemm_profile")


def dlm_gemm_profile_read(ctx):
    """(summed GEMM launch ms, executed tensor-core FLOPs, launches) since the last read."""
    ms, fl, n = ctypes.c_double(0.0), ctypes.c_double(0.0), ctypes.c_int64(0)
    ctx.check(lib().dlm_gemm_profile_read(ctx.h, ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(n)),
              "dlm_gemm_profile_read")
    return ms.value, fl.value, n.value


def dlm_probe_smem_bandwidth(ctx):
    g = ctypes.c_double(0.0)
    ctx.check(lib().dlm_probe_smem_bandwidth(ctx.h, ctypes.byref(g)), "dlm_probe_smem_bandwidth")
    return g.value


def dlm_probe_l2_bandwidth(ctx):
    g = ctypes.c_double(0)
    ctx.check(lib().dlm_probe_l2_bandwidth(ctx.h, ctypes.byref(g)), "dlm_probe_l2_bandwidth")
    return g.value


def dlm_tabucol_launch_info(ctx, g, k, pop, warps=0):
    """dict(grouped, warps, groups, ring, per, bits_in_smem, grid, slots) of the launch the library
    would make for this problem."""
    info = (ctypes.c_int32 * 8)()
    ctx.check(lib().dlm_tabucol_launch_info(ctx.h, g.h, k, pop, warps, info), "dlm_tabucol_launch_info")
    keys = ("grouped", "warps", "groups", "ring", "per", "bits_in_smem", "grid", "slots")  # grouped 2: u8 entries
    return dict(zip(keys, [int(x) for x in info]))


def dlm_wvcp_tabu_batch(ctx, g, k, pop, col, best_g, best_fc, moves, iters, tenure=WVCP_TENURE, phi=0, seed=0,
                        generation=0, ind_base=0):
    ctx.check(lib().dlm_wvcp_tabu_batch(ctx.h, g.h, k, pop, _ptr(col), _ptr(best_g), _ptr(best_fc), _ptr(moves),
                                        iters, tenure, phi, seed, generation, ind_base), "dlm_wvcp_tabu_batch")


def dlm_wvcp_tabu_batch_ex(ctx, g, k, pop, col, best_g, best_fc, moves, iters, tenure=WVCP_TENURE, phi=0, seed=0,
                           generation=0, ind_base=0, trace=None, entry_bits=0):
    ctx.check(lib().dlm_wvcp_tabu_batch_ex(ctx.h, g.h, k, pop, _ptr(col), _ptr(best_g), _ptr(best_fc), _ptr(moves),
                                           iters, tenure, phi, seed, generation, ind_base, _ptr(trace), entry_bits),
              "dlm_wvcp_tabu_batch_ex")


def dlm_wvcp_entry_bits(ctx, g, k):
    """The conflict-table entry size (8 or 16, 0 if the state does not fit) of the weighted tabu
    search on graph g with k colours."""
    out = ctypes.c_int32(0)
    ctx.check(lib().dlm_wvcp_entry_bits(ctx.h, g.h, k, ctypes.byref(out)), "dlm_wvcp_entry_bits")
    return out.value


def dlm_wvcp_greedy(ctx, g, pop, seed, ind_base, col, used):
    ctx.check(lib().dlm_wvcp_greedy(ctx.h, g.h, pop, seed, ind_base, _ptr(col), _ptr(used)), "dlm_wvcp_greedy")


class MultiPlan:
    """dlm_multi_plan: an uneven batch captured once into a CUDA graph (see include/dlmcol.h)."""

    def __init__(self, ctx, graphs, ks, pops, cols, best_fs, moves, iters, tenure=COL_TENURE, seed=0, generation=0,
                 ind_base=0):
        a = _multi_args(graphs, ks, pops, cols, best_fs, moves, iters)
        h = ctypes.c_void_p()
        ctx.check(lib().dlm_tabucol_multi_plan_create(ctx.h, *a, tenure, seed, generation, ind_base, ctypes.byref(h)),
                  "dlm_tabucol_multi_plan_create")
        self.h = h
        self._keep = a

    def close(self):
        if getattr(self, "h", None):
            lib().dlm_tabucol_multi_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dlm_tabucol_multi_plan_launch(ctx, plan):
    ctx.check(lib().dlm_tabucol_multi_plan_launch(ctx.h, plan.h), "dlm_tabucol_multi_plan_launch")


def dlm_wvcp_iterated(ctx, g, k, pop, col, best_col, best_f, iters, max_ls=10, tenure=WVCP_TENURE, fscale=256,
                      phi0=1, phi_last=1, seed=0, generation=0, ind_base=0):
    ctx.check(lib().dlm_wvcp_iterated(ctx.h, g.h, k, pop, _ptr(col), _ptr(best_col), _ptr(best_f), iters, max_ls,
                                      tenure, fscale, phi0, phi_last, seed, generation, ind_base), "dlm_wvcp_iterated")


def dlm_col_descend(ctx, g, params, max_gens, best_col):
    """k-COL with decreasing k from params.k: returns (k_best, generations run per k)."""
    import numpy as np

    kb = ctypes.c_int32(0)
    gens = np.zeros(params.k + 1, np.int32)
    ctx.check(lib().dlm_col_descend(ctx.h, g.h, ctypes.byref(params), max_gens, ctypes.byref(kb), _ptr(best_col),
                                    _ptr(gens)), "dlm_col_descend")
    return kb.value, gens


MEMETIC_STAGES = ("tabu", "best_of", "distances", "pool_update", "matching", "offspring", "training")
MEMETIC_OFFSPRING_PARTS = ("offspring_gpx", "offspring_wait_training", "offspring_scoring")


def dlm_memetic_profile(ctx, mm, enable):
    """Mean ms per generation of each stage since the last call (dict), then (re)sets recording."""
    import numpy as np

    out = np.zeros(11, np.float64)
    ctx.check(lib().dlm_memetic_profile(ctx.h, mm.h, 1 if enable else 0, _ptr(out)), "dlm_memetic_profile")
    d = dict(zip(MEMETIC_STAGES, out[:7].tolist()), generations=int(out[7]))
    d.update(zip(MEMETIC_OFFSPRING_PARTS, out[8:11].tolist()))
    return d
