"""Helpers shared by the GPU tests: contexts, graphs on the device, a spawn pool for the oracle."""
import multiprocessing as mp
import os

import numpy as np

from paper_2109_05948_gb300 import inputs


def torch_cuda():
    import torch

    return torch


_POOL = None


def oracle_pool():
    """A process pool for oracle runs, started with spawn (safe after CUDA is initialised)."""
    global _POOL
    if _POOL is None:
        _POOL = mp.get_context("spawn").Pool(min(16, os.cpu_count() or 4))
    return _POOL


def _oracle_tabu_job(args):
    import oracle

    adj, k, col, iters, seed, ind, gen, trace = args
    return oracle.tabucol(adj, k, col, iters, seed=seed, ind=ind, gen=gen, trace=trace)


def _oracle_tabu_alpha_job(args):
    import oracle

    (adj, k, col, iters, seed, ind, gen, trace), alpha = args
    return oracle.tabucol(adj, k, col, iters, seed=seed, ind=ind, gen=gen, alpha=alpha, trace=trace)


def oracle_tabu_many(jobs):
    """jobs: list of (adj, k, col, iters, seed, ind, gen, trace) -> list of oracle results."""
    if len(jobs) <= 2:
        return [_oracle_tabu_job(j) for j in jobs]
    return oracle_pool().map(_oracle_tabu_job, jobs)


def device_graph(ctx, n, edges, weights=None):
    import torch

    from paper_2109_05948_gb300 import dlmcol

    e = torch.from_numpy(np.ascontiguousarray(edges, np.int32)).cuda()
    w = torch.from_numpy(np.ascontiguousarray(weights, np.int32)).cuda() if weights is not None else None
    g = dlmcol.Graph(ctx, n, e, w)
    return g


def gnp_case(n, p, seed):
    e = inputs.gnp(n, p, seed)
    return e, inputs.edges_to_adj(n, e)
