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


def test_traffic_record_sums_the_launches_of_one_call(tmp_path, monkeypatch):
    """--traffic-from sums the DRAM counters of every tabu launch of one call (the u8 launch and
    the u16 pass) and keys the record by the kernel source hash; other kernels are ignored."""
    csv = tmp_path / "dram.csv"
    rows = ['"ID","Kernel Name","Metric Name","Metric Unit","Metric Value"']
    for i, (kern, rd, wr, t) in enumerate([("void tabucol_group_kernel<4, 1, 8>(GroupArgs)", 4661760, 35840, 1770046464),
                                           ("void tabucol_group_kernel<4, 0, 16>(GroupArgs)", 84992, 0, 7264),
                                           ("k_smem_probe(int, uint4 *)", 999, 999, 999)]):
        rows += [f'"{i}","{kern}","dram__bytes_read.sum","byte","{rd}"',
                 f'"{i}","{kern}","dram__bytes_write.sum","byte","{wr}"',
                 f'"{i}","{kern}","gpu__time_duration.sum","ns","{t}"']
    csv.write_text("==PROF== header line\n" + "\n".join(rows) + "\n")
    out = tmp_path / "rec.json"
    monkeypatch.setattr(bench, "TRAFFIC_JSON", str(out))
    bench.write_traffic(str(csv), "ncu ...")
    import json

    rec = json.loads(out.read_text())
    assert rec["dram_read_bytes"] == 4661760 + 84992 and rec["dram_write_bytes"] == 35840
    assert rec["dram_bytes_per_launch"] == 4661760 + 84992 + 35840
    assert rec["duration_ns"] == 1770046464 + 7264
    assert rec["kernel_source_sha256_16"] == bench.tabu_source_hash()
    assert bench.recorded_traffic() == rec


def test_generation_log_lines(tmp_path):
    path = tmp_path / "gens.jsonl"
    bench.log_generation(str(path), "memetic", "learned", 1000, 0, 0.51234, 17, {"pred_pearson": None, "f_mean": 3.5})
    bench.log_generation(str(path), "memetic", "learned", 1000, 1, 1.0, 0, {"pred_pearson": 0.7, "f_mean": 1.0})
    bench.log_generation(None, "memetic", "learned", 1000, 2, 1.5, 0, {})
    import json

    lines = [json.loads(x) for x in path.read_text().splitlines()]
    assert [x["generation"] for x in lines] == [0, 1]
    assert lines[0]["elapsed_s"] == 0.5123 and lines[1]["pred_pearson"] == 0.7 and lines[0]["best"] == 17


def test_memetic_summary_reports_both_times():
    """The summary gives the time at the end of the generation that reached the target and the
    earlier time at which its best-so-far update recorded the target (per mode, with medians)."""
    def run(seed, hit, found, gens):
        traj = [[round(hit * (g + 1) / gens, 3), 0 if g == gens - 1 else 5] for g in range(gens)]
        return {"seed": seed, "time_to_target_s": hit, "time_to_best_found_s": found, "generations": gens,
                "best": 0, "trajectory": traj,
                "diagnostics": [{"f_mean": 1.0, "pred_pearson": None} for _ in range(gens)]}

    runs = {"learned": [run(0, 1.4, 1.1, 3), run(1, 1.4, 1.2, 3), run(2, 1.8, 1.5, 4)],
            "random": [run(0, 1.3, 1.2, 4), run(1, 1.0, 0.9, 3), run(2, 1.3, 1.25, 4)]}
    out = bench.memetic_summary(runs)
    assert out["value"] == 1.4 and out["random_gpx"] == 1.3
    assert out["summary"]["learned"]["median_time_to_best_found_s"] == 1.2
    assert out["summary"]["random"]["median_time_to_best_found_s"] == 1.2
    assert out["found_learned_over_random"] == 1.0
    assert out["summary"]["learned"]["mean_time_to_best_found_s"] == pytest.approx((1.1 + 1.2 + 1.5) / 3)
    runs["random"][0]["time_to_best_found_s"] = None  # a run that never reached the target
    assert bench.memetic_summary(runs)["summary"]["random"]["median_time_to_best_found_s"] is None
