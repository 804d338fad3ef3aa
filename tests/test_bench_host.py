"""Host-side accounting of bench.py, checked on the CPU against the oracle: the work of the pool
update's greedy visit (candidates examined, kept-member checks) that the population bench
reconstructs from the kernel's output equals a direct count of the visit."""
import numpy as np
import pytest

import bench
import oracle


def _direct(p, n, fit, D):
    m = 2 * p
    order = np.lexsort((np.arange(m), fit))
    kept, entries, examined = [], 0, 0
    for x in order:
        if len(kept) >= p:
            break
        examined += 1
        entries += len(kept)
        if all(10 * int(D[x][a]) > n for a in kept):
            kept.append(x)
    return examined, entries


@pytest.mark.parametrize("seed", range(12))
def test_pool_work_matches_a_direct_count(seed):
    rng = np.random.default_rng(seed)
    p = int(rng.integers(2, 60))
    n = int(rng.choice([10, 50, 100, 400]))
    spread = int(rng.choice([5, 15, 40, 200, 30000]))
    m = 2 * p
    D = np.triu(rng.integers(0, spread, (m, m)), 1)
    D = (D + D.T).astype(np.int16)
    fit = rng.integers(0, 5, m).astype(np.int64)
    sel = oracle.pool_update(p, n, fit, D)
    DP = D[sel][:, sel].astype(np.int64)
    close = ((10 * DP <= n) & np.tril(np.ones((p, p), bool), -1)).any(axis=1)
    assert bench.pool_work(p, fit, sel, close) == _direct(p, n, fit, D)
