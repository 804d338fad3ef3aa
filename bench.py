#!/usr/bin/env python
"""Benchmark of the DLMCOL hot path on GB300: batched TabuCol moves per second.

Workload (one step): TabuCol on G(n=500, p=0.5), k = 48, population 4096 per GPU, 10^5
iterations per individual, random start colourings (Philox seed 0), through the C-ABI call
dlm_tabucol_batch. value = tabu moves (iterations that moved) of all GPUs / device time.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank runs its own 4096 individuals (weak scaling, no data-path collective).
--impl reference times the CPU oracle (the plain C++ statement of the method) on the host cores.
The default run also compares learned and random GPX selection (the metric's second half) in two
child processes: time to a legal colouring on the planted k-COL workload (memetic_time_to_target)
and the best WVCP score at a fixed wall time on the weighted one (wvcp_memetic_score_at_wall);
--no-memetic leaves both out.

Other workloads (one JSON line each, single GPU):
  --workload memetic  learned vs random GPX time to a legal colouring, planted n = 1000, k = 48
  --workload multi    the uneven 64-graph batch (one grouped launch per graph) replayed from a CUDA graph
  --workload wvcp     the weighted feasible/infeasible tabu search, G(1000, 0.5), weights 1..100
  --workload scorer   one learned generation's scoring and training with the tensor-core roofline
  --workload wvcp_iterated  Algorithm 2 (iterated weighted search with the adaptive penalty)
  --workload popsweep best conflicts against population size at a fixed tabu budget
  --workload wvcp_memetic  learned vs random GPX on the weighted problem, WVCP score at fixed wall time
  --workload deepnet  the paper-size invariant network (batch normalisation): scoring and training
  --workload population  distances, pool update, K nearest neighbours and GPX of one generation,
                         each kernel against its roofline
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N, P_EDGE, K, POP, ITERS, SEED = 500, 0.5, 48, 4096, 100_000, 0
METRIC = "tabu moves/s at n=500,k=48"
UNIT = "moves/s"


def shard(rank: int, pop: int) -> tuple[int, int]:
    """Weak scaling: rank r owns the individuals [r * pop, (r + 1) * pop) of the global population.
    Individual ids key the Philox streams, so the union over ranks computes exactly what one GPU
    would compute on world * pop individuals; no data crosses ranks."""
    return rank * pop, pop


def reduce_over_ranks(dist, ms: float, units: int, device) -> tuple[float, int]:
    """The job's time is the slowest rank's, its work the sum over ranks."""
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    m = torch.tensor([units], dtype=torch.int64, device=device)
    dist.all_reduce(m)
    return float(t.item()), int(m.item())


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--iters", type=int, default=ITERS)
    ap.add_argument("--pop", type=int, default=POP)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-memetic", action="store_true",
                    help="leave out the learned-vs-random GPX comparison of the default run")
    ap.add_argument("--workload", default="tabu", choices=["tabu", "memetic", "multi", "wvcp", "wvcp_iterated", "scorer", "popsweep",
                                                   "population", "wvcp_memetic", "deepnet"],
                    help="tabu: the headline moves/s step; memetic: learned vs random GPX time-to-target; "
                         "multi: the uneven 64-graph batch in one captured persistent launch; wvcp: the "
                         "weighted tabu search; wvcp_iterated: its iterated form with the adaptive penalty "
                         "(Algorithm 2); scorer: one generation's scoring and training on the tensor cores; "
                         "popsweep: best conflicts against population size at a fixed tabu budget; population: "
                         "distances, pool update, K nearest neighbours and GPX of one generation")
    ap.add_argument("--multi-pop", type=int, default=256)
    ap.add_argument("--multi-depth", type=int, default=128, help="tabu iterations per individual = depth * n")
    ap.add_argument("--mem-n", type=int, default=1000)
    ap.add_argument("--mem-k", type=int, default=48)
    ap.add_argument("--mem-pop", type=int, default=8192)
    ap.add_argument("--mem-iters", type=int, default=2000,
                    help="tabu iterations per generation; 2 |V|: at 10 |V| tabu alone solves the graph in the "
                         "first generation and the crossover never matters")
    ap.add_argument("--mem-target", type=int, default=0, help="conflict level to reach")
    ap.add_argument("--mem-graph", default="planted", choices=["planted", "gnp"],
                    help="planted k-colourable (p = 0.5 across parts) or uniform random G(n, 0.5)")
    ap.add_argument("--mem-seeds", type=int, default=10)
    ap.add_argument("--wvcp-entry-bits", type=int, default=0, choices=(0, 8, 16),
                    help="--workload wvcp: conflict-table entry size (0: the library's choice)")
    ap.add_argument("--scorer-k", type=int, default=48,
                    help="--workload scorer: colours (48: the planted learned workload; 145: the weighted one)")
    ap.add_argument("--scorer-epochs", type=int, default=5, help="--workload scorer: training epochs")
    ap.add_argument("--scorer-split", type=int, default=1, choices=(0, 1),
                    help="--workload scorer: scoring activations bf16 hi + lo (1) or bf16 alone (0, the memetic "
                         "selection's setting)")
    ap.add_argument("--wvcp-pop", type=int, default=8192, help="--workload wvcp: population (small cases for ncu)")
    ap.add_argument("--wvcp-iters", type=int, default=10000, help="--workload wvcp: iterations per individual")
    ap.add_argument("--mem-log", default=None,
                    help="append one JSON line per generation (mode, seed, generation, elapsed s, best, the "
                         "dlm_memetic_stats diagnostics) to this file (memetic and wvcp_memetic workloads)")
    ap.add_argument("--mem-max-gens", type=int, default=40)
    ap.add_argument("--mem-time-limit", type=float, default=120.0, help="seconds per run")
    ap.add_argument("--wm-pop", type=int, default=8192)
    ap.add_argument("--wm-iters", type=int, default=500, help="iterations of each search of the weighted local search")
    ap.add_argument("--wm-ls", type=int, default=2,
                    help="searches per generation (the paper's 10 x 10 |V| takes minutes per generation at "
                         "population 8192)")
    ap.add_argument("--wm-epochs", type=int, default=20)
    ap.add_argument("--wm-seeds", type=int, default=3)
    ap.add_argument("--wm-time", type=float, default=60.0, help="wall budget per run, seconds")
    ap.add_argument("--wm-max-gens", type=int, default=400)
    ap.add_argument("--wm-short-seeds", type=int, default=2, help="seeds of the default run's weighted comparison")
    ap.add_argument("--wm-short-time", type=float, default=15.0, help="wall budget per run of that comparison, s")
    ap.add_argument("--dn-problem", default="col", choices=["col", "wvcp"])
    ap.add_argument("--dn-cands", type=int, default=1024)
    ap.add_argument("--dn-samples", type=int, default=500)
    ap.add_argument("--dn-bf16", action="store_true", help="bf16 operands alone (no hi + lo split)")
    ap.add_argument("--warps", type=int, default=0, help="warps per individual (0: the library's default)")
    ap.add_argument("--traffic-from", default=None,
                    help="write profiles/tabucol_C2_dram.json from this ncu CSV of one tabu launch and exit")
    ap.add_argument("--traffic-command", default="", help="the ncu command that wrote --traffic-from")
    ap.add_argument("--warm-start", type=int, default=0,
                    help="run this many iterations first (untimed) and start every step from their best "
                         "colourings (profiling the late phase of the search)")
    return ap.parse_args()


def config(args, extra=None):
    c = {"workload": f"batched TabuCol G(n={N}, p={P_EDGE}), k={K}, population {args.pop} per GPU, "
                     f"{args.iters} iterations per individual, random starts (Philox seed {SEED})",
         "n": N, "k": K, "edge_p": P_EDGE, "population_per_gpu": args.pop, "iters": args.iters,
         "tenure": "U{0..9} + floor(0.6 f)", "parallelism": f"population sharded over {args.gpus} GPU(s)",
         "l2": "flushed between timed steps (256 MiB write)"}
    if extra:
        c.update(extra)
    return c


# ------------------------------------------------------------------------------------------------
# CPU oracle (baseline / reference arm)
# ------------------------------------------------------------------------------------------------
def _oracle_job(args):
    import oracle
    from paper_2109_05948_gb300 import inputs

    ind, iters = args
    adj = inputs.edges_to_adj(N, inputs.gnp(N, P_EDGE, SEED))
    col = oracle.init_colors(N, K, 1, SEED, ind_base=ind)[0]
    t = time.perf_counter()
    r = oracle.tabucol(adj, K, col, iters, seed=SEED, ind=ind)
    return r["moves"], time.perf_counter() - t


def oracle_sample(n_ind: int, iters: int):
    """Runs n_ind individuals of the workload through the oracle, one process per host core
    (spawned); returns (moves, wall seconds, processes, cpu seconds)."""
    import multiprocessing as mp

    import oracle

    oracle.build()
    procs = min(n_ind, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(procs) as pool:
        pool.map(_oracle_job, [(0, 10)] * procs)  # start-up outside the timing
        t = time.perf_counter()
        res = pool.map(_oracle_job, [(i, iters) for i in range(n_ind)])
        wall = time.perf_counter() - t
    return sum(r[0] for r in res), wall, procs, sum(r[1] for r in res)


def cpu_baseline(args):
    # two individuals per host core (at most 32): about 10-15 s of CPU work at the full budget
    n_ind = 2 * min(16, os.cpu_count() or 1)
    moves, wall, procs, cpu_s = oracle_sample(n_ind, args.iters)
    return {"value": moves / wall, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{n_ind} individuals x {args.iters} iterations of the same workload on {procs} spawned "
                      f"worker processes, one per host core ({cpu_s:.1f} s of CPU work)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # one individual per host core over the workload's full budget: the same per-individual work as
    # the GPU arm, on a sample of the population
    n_ind = min(16, os.cpu_count() or 1)
    iters = args.iters
    for _ in range(args.warmup):
        oracle_sample(n_ind, iters)
    moves = 0
    wall = 0.0
    cpu = 0.0
    for _ in range(args.steps):
        mv, w, procs, c = oracle_sample(n_ind, iters)
        moves += mv
        wall += w
        cpu += c
    v = moves / wall
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int16/int32",
           "data": "synthetic", "config": config(args, {"reference_sample": f"{n_ind} individuals x {iters} iterations per step"}),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                            "sample": f"{n_ind} individuals x {iters} iterations per step, {cpu:.1f} s CPU"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


TRAFFIC_JSON = os.path.join(ROOT, "profiles", "tabucol_C2_dram.json")
TABU_SOURCES = [os.path.join(ROOT, "paper_2109_05948_gb300", "csrc", f) for f in ("tabu_group.cu", "tabu_group.cuh")]


def tabu_source_hash():
    import hashlib

    h = hashlib.sha256()
    for f in TABU_SOURCES:
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM (and L2) bytes per launch of the tabu kernel, written by --traffic-from from an ncu
    capture, or None when the kernel's source has changed since the counters were taken."""
    try:
        rec = json.load(open(TRAFFIC_JSON))
    except Exception:
        return None
    return rec if rec.get("kernel_source_sha256_16") == tabu_source_hash() else None


def write_traffic(csv_path, command):
    """Reads the ncu CSV of the tabu launches of one dlm_tabucol_batch call (dram__bytes_read.sum,
    dram__bytes_write.sum, lts__t_bytes.sum, gpu__time_duration.sum; --print-units base; with u8
    conflict-table entries the call is the u8 launch and the u16 pass over the individuals it gave
    up) and writes their summed counters with the hash of the kernel's source to
    profiles/tabucol_C2_dram.json."""
    import csv

    vals = {}
    with open(csv_path) as fh:
        lines = [ln for ln in fh if ln.startswith('"')]
    for row in csv.DictReader(lines):
        if "tabucol_group" not in row.get("Kernel Name", ""):
            continue
        name = row.get("Metric Name")
        try:
            vals[name] = vals.get(name, 0.0) + float(row.get("Metric Value", "").replace(",", ""))
        except ValueError:
            pass
    need = ("dram__bytes_read.sum", "dram__bytes_write.sum", "gpu__time_duration.sum")
    if not all(k in vals for k in need):
        raise SystemExit(f"{csv_path}: no tabucol_group launch with {need}")
    rec = {"dram_bytes_per_launch": vals["dram__bytes_read.sum"] + vals["dram__bytes_write.sum"],
           "dram_read_bytes": vals["dram__bytes_read.sum"], "dram_write_bytes": vals["dram__bytes_write.sum"],
           "l2_bytes_per_launch": vals.get("lts__t_bytes.sum"), "duration_ns": vals["gpu__time_duration.sum"],
           "kernel_source_sha256_16": tabu_source_hash(), "command": command}
    with open(TRAFFIC_JSON, "w") as fh:
        json.dump(rec, fh, indent=1)
        fh.write("\n")
    print(json.dumps(rec))


# ------------------------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------------------------
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.device)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------------------------
def log_generation(path, workload, mode, seed, gen, elapsed, best, diag):
    """One JSON line per memetic generation (the per-generation prediction and population
    diagnostics of section "Analysis of the contributions of deep learning")."""
    if not path:
        return
    with open(path, "a") as fh:
        fh.write(json.dumps({"workload": workload, "mode": mode, "seed": seed, "generation": gen,
                             "elapsed_s": round(elapsed, 4), "best": int(best), **diag}) + "\n")


def run_memetic(args):
    """Learned-guided vs random-GPX memetic search (Algorithm 1 and the ablation of section
    "Benefits of the neural network based crossover selection") on a planted 48-colourable graph:
    wall time until the population's best colouring has at most `mem_target` conflicts, at equal
    population size, per seed; one JSON line with both modes' medians and per-seed values."""
    import torch

    from paper_2109_05948_gb300 import build as libbuild
    from paper_2109_05948_gb300 import dlmcol, inputs

    libbuild.build()
    torch.cuda.set_device(0)
    ctx = dlmcol.Context(0)
    n, k = args.mem_n, args.mem_k
    e = inputs.planted(n, k, 0.5, seed=0)[0] if args.mem_graph == "planted" else inputs.gnp(n, 0.5, seed=0)
    g = dlmcol.Graph(ctx, n, torch.from_numpy(e).cuda())
    runs = {"learned": [], "random": []}
    clocks = Clocks(0)
    clocks.start()
    for seed in range(args.mem_seeds):
        for mode in ("learned", "random"):
            prm = dlmcol.MemeticParams(k=k, p=args.mem_pop, K=32, iters=args.mem_iters, tenure=dlmcol.COL_TENURE,
                                       use_scorer=1 if mode == "learned" else 0, epochs=5, batch=100, lr=1e-3,
                                       seed=1000 + seed)
            mm = dlmcol.Memetic(ctx, g, prm)
            dlmcol.dlm_memetic_profile(ctx, mm, True)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            traj, diag, hit, found = [], [], None, None
            el_prev = 0.0
            for gen in range(args.mem_max_gens):
                best = dlmcol.dlm_memetic_step(ctx, mm)
                el = time.perf_counter() - t0
                traj.append([round(el, 3), int(best)])
                # diagnostics read after the timing of the generation (they wait for the stream)
                st = dlmcol.dlm_memetic_stats(ctx, mm)
                diag.append({key: (None if v != v else round(v, 4)) for key, v in st.items()})
                log_generation(args.mem_log, "memetic", mode, 1000 + seed, gen, el, best, diag[-1])
                if best <= args.mem_target:
                    hit = el
                    # the moment S* reached the target: the generation's start plus the device
                    # time to the end of its best-so-far update (Algorithm 1 records S* after
                    # the local search)
                    found = el_prev + dlmcol.dlm_memetic_found_ms(ctx, mm) / 1e3
                    break
                t0 += time.perf_counter() - t0 - el  # the diagnostics' read is not search time
                el_prev = el
                if el > args.mem_time_limit:
                    break
            stages = dlmcol.dlm_memetic_profile(ctx, mm, False)
            runs[mode].append({"seed": 1000 + seed, "time_to_target_s": hit, "time_to_best_found_s": found,
                               "generations": len(traj),
                               "best": traj[-1][1], "trajectory": traj, "diagnostics": diag,
                               "stage_ms_per_generation": {key: round(v, 2) for key, v in stages.items()
                                                           if key != "generations"}})
            print(json.dumps({"progress": mode, "seed": 1000 + seed, "time_to_target_s": hit,
                              "time_to_best_found_s": found,
                              "generations": len(traj), "best": traj[-1][1]}), file=sys.stderr, flush=True)
            mm.close()

    ck = clocks.stop()
    out = {"metric": "time-to-target conflicts learned vs plain GPX", "workload": "memetic",
           "unit": "s", "higher_is_better": False,
           "config": {"workload": (f"planted {k}-colourable n={n}, p=0.5 across parts" if args.mem_graph == "planted"
                                   else f"G(n={n}, p=0.5), k={k}") + f", population {args.mem_pop}, "
                                  f"K=32 GPX candidates, {args.mem_iters} tabu iterations per generation, "
                                  f"scorer 64-d embedding + 3 x 256 invariant layers, N=5 epochs, b=100, lr=1e-3",
                      "target_conflicts": args.mem_target, "seeds": args.mem_seeds,
                      "time_limit_s": args.mem_time_limit, "max_generations": args.mem_max_gens},
           "clocks": ck, "data": "synthetic"}
    out.update(memetic_summary(runs))
    out["runs"] = runs
    print(json.dumps(out), flush=True)
    return out


def memetic_compare(args):
    """run_memetic at the learned workload's defaults, as a child process (its JSON line, per-seed
    runs left out)."""
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "memetic", "--mem-seeds", str(args.mem_seeds),
           "--mem-iters", str(args.mem_iters), "--mem-pop", str(args.mem_pop)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as exc:  # reported, never fatal to the headline
        return {"error": f"{type(exc).__name__}: {exc}"}
    sm = d["summary"]
    return {"metric": d["metric"], "unit": d["unit"], "higher_is_better": False, "learned_median_s": d["value"],
            "random_gpx_median_s": d["random_gpx"], "learned_over_random": d["learned_over_random"],
            "best_found": {"learned_median_s": sm["learned"]["median_time_to_best_found_s"],
                           "random_gpx_median_s": sm["random"]["median_time_to_best_found_s"],
                           "learned_over_random": d.get("found_learned_over_random"),
                           "per_seed_s": {m: [x.get("time_to_best_found_s") for x in d["runs"][m]]
                                          for m in d["runs"]}},
            "config": d["config"], "summary": sm,
            "per_seed_s": {m: [x["time_to_target_s"] for x in d["runs"][m]] for m in d["runs"]}}


def wvcp_memetic_compare(args):
    """run_wvcp_memetic on the weighted workload (G(1000, 0.5), weights 1..100, population
    8192) with a short wall budget, as a child process: the learned and random modes' best WVCP
    scores at fixed wall time (per-seed trajectories left out)."""
    cmd = [sys.executable, os.path.abspath(__file__), "--workload", "wvcp_memetic", "--wm-seeds", str(args.wm_short_seeds),
           "--wm-time", str(args.wm_short_time)]
    try:
        r = subprocess.run(cmd, capture_output=True, text=True, timeout=900)
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception as exc:  # reported, never fatal to the headline
        return {"error": f"{type(exc).__name__}: {exc}"}
    sm = d["summary"]
    return {"metric": d["metric"], "unit": d["unit"], "higher_is_better": False,
            "learned_median_best": d["value"], "random_gpx_median_best": d["random_gpx"],
            "level": d["level"], "config": d["config"],
            "per_seed_best": {m: sm[m]["per_seed_best"] for m in sm},
            "time_to_level_s": {m: sm[m]["time_to_level_s"] for m in sm},
            "median_generations": {m: sm[m]["median_generations"] for m in sm}}


def memetic_summary(runs, wall_points=(0.5, 1.0, 1.5, 2.0)):
    """Medians, means with bootstrap 95 % intervals of the time to target, best conflicts at fixed
    wall times and the mean post-tabu conflicts of each generation's offspring, per mode."""
    import random as _r

    def boot(xs, reps=2000):
        if not xs:
            return None
        g = _r.Random(0)
        ms = sorted(statistics.mean(g.choice(xs) for _ in xs) for _ in range(reps))
        return [ms[int(0.025 * reps)], ms[int(0.975 * reps) - 1]]

    res = {}
    for mode, rs in runs.items():
        ts = [r["time_to_target_s"] for r in rs if r["time_to_target_s"] is not None]
        at = {}
        for w in wall_points:
            vals = []
            for r in rs:
                done = [b for (t, b) in r["trajectory"] if t <= w]
                if done:
                    vals.append(done[-1])
                elif r["time_to_target_s"] is not None and r["time_to_target_s"] <= w:
                    vals.append(0)
            at[str(w)] = statistics.median(vals) if len(vals) == len(rs) else None
        gmax = max(len(r["diagnostics"]) for r in rs)
        fmean = [statistics.median([r["diagnostics"][i]["f_mean"] for r in rs if len(r["diagnostics"]) > i])
                 for i in range(gmax)]
        pear = [statistics.median([r["diagnostics"][i]["pred_pearson"] for r in rs
                                   if len(r["diagnostics"]) > i and r["diagnostics"][i]["pred_pearson"] is not None]
                                  or [float("nan")]) for i in range(gmax)]
        fs = [r["time_to_best_found_s"] for r in rs if r.get("time_to_best_found_s") is not None]
        res[mode] = {"reached": len(ts), "runs": len(rs),
                     "median_time_to_target_s": statistics.median(ts) if len(ts) == len(rs) else None,
                     "mean_time_to_target_s": statistics.mean(ts) if len(ts) == len(rs) else None,
                     "mean_ci95_s": boot(ts) if len(ts) == len(rs) else None,
                     "median_time_to_best_found_s": statistics.median(fs) if fs and len(fs) == len(rs) else None,
                     "mean_time_to_best_found_s": statistics.mean(fs) if fs and len(fs) == len(rs) else None,
                     "found_mean_ci95_s": boot(fs) if fs and len(fs) == len(rs) else None,
                     "median_generations": statistics.median(r["generations"] for r in rs),
                     "median_best_at_wall_s": at,
                     "median_offspring_f_mean_by_generation": [round(x, 1) for x in fmean],
                     "median_prediction_pearson_by_generation": [None if x != x else round(x, 3) for x in pear]}
    lm, rm = res["learned"]["median_time_to_target_s"], res["random"]["median_time_to_target_s"]
    lf, rf = res["learned"]["median_time_to_best_found_s"], res["random"]["median_time_to_best_found_s"]
    return {"value": lm, "random_gpx": rm, "summary": res,
            "learned_over_random": (lm / rm) if lm and rm else None,
            "found_learned_over_random": (lf / rf) if lf and rf else None}


def run_wvcp_memetic(args):
    """Learned-guided vs random-GPX memetic search on the weighted problem (Algorithm 1 with the
    iterated feasible / infeasible tabu search of Algorithm 2 as the local search): G(1000, 0.5),
    weights uniform in 1..100, population 8192, K = 32, N = 20 epochs (the WVCP parameter table),
    k = the largest colour count of the seed's greedy initial population. Each run has a wall
    budget; value = the learned mode's median best WVCP score at that budget, beside the random
    mode's, their medians at intermediate wall times and the time each run needs to reach the
    worst final best over all runs (a level every run reaches)."""
    import torch

    from paper_2109_05948_gb300 import build as libbuild
    from paper_2109_05948_gb300 import dlmcol, inputs

    libbuild.build()
    torch.cuda.set_device(0)
    ctx = dlmcol.Context(0)
    n, pop = 1000, args.wm_pop
    e = inputs.gnp(n, 0.5, 0)
    w = inputs.weights(n, 0)
    g = dlmcol.Graph(ctx, n, torch.from_numpy(e).cuda(), torch.from_numpy(w).cuda())
    used = torch.empty(pop, dtype=torch.int32, device="cuda")
    scratch = torch.empty((pop, n), dtype=torch.int16, device="cuda")
    runs = {"learned": [], "random": []}
    clocks = Clocks(0)
    clocks.start()
    for si in range(args.wm_seeds):
        seed = 2000 + si
        dlmcol.dlm_wvcp_greedy(ctx, g, pop, seed, 0, scratch, used)
        ctx.sync()
        k = int(used.max())
        for mode in ("learned", "random"):
            prm = dlmcol.MemeticParams(k=k, p=pop, K=32, iters=args.wm_iters, tenure=dlmcol.WVCP_TENURE,
                                       use_scorer=1 if mode == "learned" else 0, epochs=args.wm_epochs, batch=100,
                                       lr=1e-3, seed=seed, problem=1, max_ls=args.wm_ls)
            mm = dlmcol.Memetic(ctx, g, prm)
            dlmcol.dlm_memetic_profile(ctx, mm, True)
            f0 = torch.empty(pop, dtype=torch.int64, device="cuda")
            dlmcol.dlm_memetic_get(ctx, mm, 1, f0)
            ctx.sync()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            traj, diag = [[0.0, int(f0.min())]], []
            for gen in range(args.wm_max_gens):
                best = dlmcol.dlm_memetic_step(ctx, mm)
                el = time.perf_counter() - t0
                traj.append([round(el, 3), int(best)])
                st = dlmcol.dlm_memetic_stats(ctx, mm)
                diag.append({key: (None if v != v else round(v, 4)) for key, v in st.items()})
                log_generation(args.mem_log, "wvcp_memetic", mode, seed, gen, el, best, diag[-1])
                t0 += time.perf_counter() - t0 - el  # the diagnostics' read is not search time
                if el > args.wm_time:
                    break
            stages = dlmcol.dlm_memetic_profile(ctx, mm, False)
            runs[mode].append({"seed": seed, "k": k, "generations": len(traj) - 1, "best": traj[-1][1],
                               "trajectory": traj, "diagnostics": diag,
                               "stage_ms_per_generation": {key: round(v, 2) for key, v in stages.items()
                                                           if key != "generations"}})
            print(json.dumps({"progress": mode, "seed": seed, "k": k, "generations": len(traj) - 1,
                              "best": traj[-1][1], "stage_ms": runs[mode][-1]["stage_ms_per_generation"]}),
                  file=sys.stderr, flush=True)
            mm.close()
    ck = clocks.stop()

    def best_at(r, t):
        return [b for (x, b) in r["trajectory"] if x <= t][-1]

    level = max(r["best"] for rs in runs.values() for r in rs)
    res = {}
    for mode, rs in runs.items():
        hit = [next(x for (x, b) in r["trajectory"] if b <= level) for r in rs]
        res[mode] = {"median_best_at_budget": statistics.median(best_at(r, args.wm_time) for r in rs),
                     "per_seed_best": [r["best"] for r in rs],
                     "median_best_at_wall_s": {str(t): statistics.median(best_at(r, t) for r in rs)
                                               for t in (args.wm_time / 4, args.wm_time / 2, 3 * args.wm_time / 4)},
                     "time_to_level_s": hit, "median_time_to_level_s": statistics.median(hit),
                     "median_generations": statistics.median(r["generations"] for r in rs),
                     "median_offspring_f_mean_by_generation": [
                         round(statistics.median(r["diagnostics"][i]["f_mean"] for r in rs
                                                 if len(r["diagnostics"]) > i), 1)
                         for i in range(max(len(r["diagnostics"]) for r in rs))],
                     "median_prediction_pearson_by_generation": [
                         (lambda xs: round(statistics.median(xs), 3) if xs else None)(
                             [r["diagnostics"][i]["pred_pearson"] for r in rs if len(r["diagnostics"]) > i
                              and r["diagnostics"][i]["pred_pearson"] is not None])
                         for i in range(max(len(r["diagnostics"]) for r in rs))]}
    out = {"metric": "WVCP score at fixed wall time, learned vs plain GPX", "workload": "wvcp_memetic",
           "value": res["learned"]["median_best_at_budget"], "unit": "WVCP score", "higher_is_better": False,
           "random_gpx": res["random"]["median_best_at_budget"], "level": level, "summary": res,
           "config": {"workload": f"G(n={n}, p=0.5), weights 1..100, population {pop}, K=32 GPX candidates, "
                                  f"k = greedy colours per seed, local search {args.wm_ls} x {args.wm_iters} "
                                  f"iterations per generation (fscale 256, adaptive penalty), scorer 64-d "
                                  f"embedding + 3 x 256 invariant layers, N={args.wm_epochs} epochs, b=100, "
                                  f"lr=1e-3", "seeds": args.wm_seeds, "wall_budget_s": args.wm_time},
           "clocks": ck, "data": "synthetic", "runs": runs}
    print(json.dumps(out), flush=True)
    return out


def run_deepnet(args):
    """The paper-size invariant network with invariant batch normalisation (section
    "Implementation and parameter setting"): hidden widths 10|V|, 5|V|, 2|V| x 5, |V|, |V|//2 for
    k-COL (n = 1000, k = 48) or 5|V|, 2|V|, |V|, |V|//2 for the WVCP (n = 1000, k = 145). Times
    the scoring of a batch of candidates (evaluation mode) and online training (Adam, b = 100)
    with CUDA events; value = candidates scored per second."""
    import numpy as np
    import torch

    from paper_2109_05948_gb300 import build as libbuild
    from paper_2109_05948_gb300 import dlmcol, inputs

    libbuild.build()
    torch.cuda.set_device(0)
    ctx = dlmcol.Context(0)
    n = 1000
    k = 48 if args.dn_problem == "col" else 145
    widths = ([10 * n, 5 * n, 2 * n, 2 * n, 2 * n, 2 * n, 2 * n, n, n // 2] if args.dn_problem == "col"
              else [5 * n, 2 * n, n, n // 2])
    net = dlmcol.DeepNet(ctx, n, k, widths, seed=SEED)
    net.set_precision(0 if args.dn_bf16 else 1)
    C, P, B = args.dn_cands, args.dn_samples, 100
    cols = torch.from_numpy(inputs.random_colorings(C, n, k, seed=1)).cuda()
    fvals = torch.from_numpy(np.random.default_rng(0).integers(0, 1000, size=P).astype(np.int64)).cuda()
    out = torch.empty(C, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        return a, b

    for _ in range(args.warmup):
        net.forward(cols, C, 0, out)
        net.train(cols[:P], fvals, P, 1, B, 1e-3, SEED, 0)
    ctx.sync()
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    ev_s, ev_t = [], []
    for st in range(args.steps):
        ev_s.append(timed(lambda: net.forward(cols, C, 0, out)))
        ev_t.append(timed(lambda: net.train(cols[:P], fvals, P, 1, B, 1e-3, SEED, st + 1)))
    torch.cuda.synchronize()
    ctx.sync()
    ck = clocks.stop()
    ms_s = sum(a.elapsed_time(b) for a, b in ev_s) / args.steps
    ms_t = sum(a.elapsed_time(b) for a, b in ev_t) / args.steps
    h = widths
    pad = [64 * ((x + 63) // 64) for x in h]
    # algorithmic tensor work per scored candidate: every layer l >= 1 multiplies the k class rows
    # and the colour average by Lambda_l and Gamma_l (2 h_l-1 h_l flops each per row); a training
    # sample adds the input-gradient and weight-gradient products (three times the forward)
    fwd = sum(2.0 * (k + 1) * h[l - 1] * h[l] for l in range(1, len(h)))
    fwd_exec = sum(2.0 * (k + 1) * pad[l - 1] * pad[l] for l in range(1, len(h))) * (1 if args.dn_bf16 else 3)
    peaks = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained") or 1700.0
    src = "of measured (MEASURED_PEAKS.json bf16_tflops_sustained)" if peaks.get("bf16_tflops_sustained") else "of fallback"
    ach_s = fwd * C / (ms_s / 1e3) / 1e12
    ach_t = 3 * fwd * P / (ms_t / 1e3) / 1e12
    roof = {"bound": "tensor", "achieved": ach_s, "peak": peak, "unit": "TFLOP/s", "frac": ach_s / peak,
            "peak_source": src, "traffic": None, "kernel": "gemm_kernel (all layer products of the scoring pass)",
            "executed_tflops": fwd_exec * C / (ms_s / 1e3) / 1e12,
            "training_achieved_tflops": ach_t, "training_frac": ach_t / peak}
    res = {"metric": f"paper-size invariant network: candidates scored per second ({args.dn_problem})",
           "workload": "deepnet", "value": C / (ms_s / 1e3), "unit": "candidates/s", "higher_is_better": True,
           "training_samples_per_s": P / (ms_t / 1e3), "ms_scoring": ms_s, "ms_training_epoch": ms_t,
           "steps": args.steps, "warmup": args.warmup, "dtype": "bf16 (hi + lo split)" if not args.dn_bf16 else "bf16",
           "data": "synthetic", "clocks": ck, "roofline": roof, "nparams": net.nparams,
           "config": {"workload": f"n={n}, k={k}, hidden widths {widths}, invariant batch normalisation, "
                                  f"{C} random colourings scored, one epoch of Adam over {P} samples (b={B})"}}
    print(json.dumps(res), flush=True)
    net.close()


def run_multi(args):
    """Uneven batch: 64 graphs (n uniform in [100, 1000], p in {0.1, 0.5, 0.9}, odd graphs planted,
    k = n/10), `multi_pop` individuals each, depth * n iterations, one persistent launch replayed
    from a CUDA graph; warps per individual autotuned per graph. value = moves/s."""
    import torch

    from paper_2109_05948_gb300 import build as libbuild
    from paper_2109_05948_gb300 import dlmcol, inputs

    libbuild.build()
    torch.cuda.set_device(0)
    ctx = dlmcol.Context(0)
    specs = inputs.uneven_batch(64, seed=0)
    graphs = [dlmcol.Graph(ctx, s["n"], torch.from_numpy(s["edges"]).cuda()) for s in specs]
    ks = [s["k"] for s in specs]
    pops = [args.multi_pop] * len(specs)
    iters = [args.multi_depth * s["n"] for s in specs]
    tuned = {}
    for g, s in zip(graphs, specs):
        key = (s["n"], s["k"])
        if key not in tuned:
            tuned[key] = dlmcol.dlm_tabucol_autotune(ctx, g, s["k"], 2 * 152, 2000)
    starts, cols, bfs, mvs = [], [], [], []
    base = 0
    for g, s, k, p in zip(graphs, specs, ks, pops):
        c = torch.empty((p, s["n"]), dtype=torch.int16, device="cuda")
        dlmcol.dlm_init_colors(ctx, s["n"], k, p, SEED, base, c)
        starts.append(c.clone())
        cols.append(c)
        bfs.append(torch.zeros(p, dtype=torch.int64, device="cuda"))
        mvs.append(torch.zeros(p, dtype=torch.int64, device="cuda"))
        base += p
    plan = dlmcol.MultiPlan(ctx, graphs, ks, pops, cols, bfs, mvs, iters, dlmcol.COL_TENURE, SEED, 0, 0)
    stream = torch.cuda.current_stream()

    def step():
        for c, st in zip(cols, starts):
            c.copy_(st)
        dlmcol.dlm_tabucol_multi_plan_launch(ctx, plan)

    for _ in range(args.warmup):
        step()
    ctx.sync()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    e0.record(stream)
    moves = 0
    for _ in range(args.steps):
        step()
        moves += sum(int(m.sum()) for m in mvs)  # reads after the step (stream-ordered)
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.sync()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    solved = sum(int((b == 0).sum()) for b in bfs)
    out = {"metric": "tabu moves/s, uneven 64-graph batch", "workload": "multi", "value": moves / (ms / 1e3),
           "unit": "moves/s", "higher_is_better": True, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "gpu_launches": args.steps, "clocks": ck, "data": "synthetic",
           "config": {"workload": f"64 graphs, n uniform in [100, 1000], p in {{0.1, 0.5, 0.9}}, odd graphs planted, "
                                  f"k = n/10, population {args.multi_pop} per graph, {args.multi_depth} n iterations, "
                                  "one persistent launch replayed from a CUDA graph",
                      "individuals": sum(pops), "warps_per_individual": sorted(set(tuned.values())),
                      "solved_individuals": solved}}
    print(json.dumps(out), flush=True)
    plan.close()


def run_wvcp(args):
    """Weighted colouring: G(1000, 0.5), weights uniform in 1..100, population 8192, k = colours of
    the GPU randomised greedy initialisation, 10 |V| iterations of the feasible/infeasible tabu
    search with phi = 2 max w. value = moves/s."""
    import torch

    from paper_2109_05948_gb300 import build as libbuild
    from paper_2109_05948_gb300 import dlmcol, inputs

    libbuild.build()
    torch.cuda.set_device(0)
    ctx = dlmcol.Context(0)
    n, pop, iters = 1000, args.wvcp_pop, args.wvcp_iters
    e = inputs.gnp(n, 0.5, 0)
    w = inputs.weights(n, 0)
    g = dlmcol.Graph(ctx, n, torch.from_numpy(e).cuda(), torch.from_numpy(w).cuda())
    col0 = torch.empty((pop, n), dtype=torch.int16, device="cuda")
    used = torch.empty(pop, dtype=torch.int32, device="cuda")
    dlmcol.dlm_wvcp_greedy(ctx, g, pop, SEED, 0, col0, used)
    ctx.sync()
    k = int(used.max())
    phi = 2 * int(w.max())
    col = torch.empty_like(col0)
    bg = torch.empty(pop, dtype=torch.int64, device="cuda")
    fc = torch.empty((pop, 2), dtype=torch.int64, device="cuda")
    mv = torch.empty(pop, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    eb = args.wvcp_entry_bits or dlmcol.dlm_wvcp_entry_bits(ctx, g, k)

    def search():
        dlmcol.dlm_wvcp_tabu_batch_ex(ctx, g, k, pop, col, bg, fc, mv, iters, dlmcol.WVCP_TENURE, phi, SEED, 0, 0,
                                      None, eb)

    for _ in range(args.warmup):
        col.copy_(col0)
        search()
    ctx.sync()
    f0 = None
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    e0.record(stream)
    moves = 0
    for _ in range(args.steps):
        col.copy_(col0)
        search()
        moves += int(mv.sum())
    e1.record(stream)
    torch.cuda.synchronize()
    ctx.sync()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    legal = fc[:, 1] == 0
    best_legal = int(fc[legal, 0].min()) if bool(legal.any()) else None
    # algorithmic work per iteration: every (v, c) pair reads one gamma entry (1 B with u8
    # entries, 2 B with u16); iterations are counted by their moves (an iteration without an
    # admissible move is not counted)
    pairs = n * (k - 1)
    eb_bytes = eb // 8
    smem_gbps = dlmcol.dlm_probe_smem_bandwidth(ctx)
    ach = eb_bytes * pairs * moves / (ms / 1e3) / 1e9
    where = ("the whole conflict table in shared memory (u8 entries)" if eb == 8 else
             "u16 entries: the conflict table's last colours live in an L2-resident slab")
    roof = {"bound": "smem", "achieved": ach, "peak": smem_gbps, "unit": "GB/s", "frac": ach / smem_gbps,
            "traffic": None, "kernel": "k_wvcp_tabu", "kernel_ms": ms / args.steps,
            "algorithmic_bytes_per_launch": eb_bytes * pairs * moves / args.steps, "entry_bits": eb,
            "peak_source": "measured by dlm_probe_smem_bandwidth on this GPU (conflict-free 16 B loads); " + where}
    out = {"metric": "weighted tabu moves/s, G(1000, 0.5), weights 1..100", "workload": "wvcp",
           "value": moves / (ms / 1e3), "unit": "moves/s", "higher_is_better": True, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "gpu_launches": args.steps, "clocks": ck,
           "pair_evaluations_per_s": moves / (ms / 1e3) * pairs, "data": "synthetic", "roofline": roof,
           "config": {"workload": f"G(1000, 0.5), weights 1..100, population {pop}, k = {k} (greedy), "
                                  f"{iters} iterations, phi = {phi}", "k": k, "phi": phi,
                      "best_legal_f": best_legal, "legal_individuals": int(legal.sum())}}
    print(json.dumps(out), flush=True)


def run_wvcp_iterated(args):
    """Algorithm 2 on the weighted workload: G(1000, 0.5), weights 1..100, population 1024 (the
    iterated search is 10 times the single search's work per individual), maxLSIters = 10
    searches of 10 |V| iterations each, phi in fixed point (resolution 1/256) from k max w / (2|V|),
    the last search at 2 max w. value = tabu moves/s over the ten searches; the line also reports
    the best legal score found."""
    import torch

    from paper_2109_05948_gb300 import build as libbuild
    from paper_2109_05948_gb300 import dlmcol, inputs

    libbuild.build()
    torch.cuda.set_device(0)
    ctx = dlmcol.Context(0)
    n, pop, depth, max_ls, fscale = 1000, 1024, 10 * 1000, 10, 256
    e = inputs.gnp(n, 0.5, 0)
    w = inputs.weights(n, 0)
    g = dlmcol.Graph(ctx, n, torch.from_numpy(e).cuda(), torch.from_numpy(w).cuda())
    col0 = torch.empty((pop, n), dtype=torch.int16, device="cuda")
    used = torch.empty(pop, dtype=torch.int32, device="cuda")
    dlmcol.dlm_wvcp_greedy(ctx, g, pop, SEED, 0, col0, used)
    ctx.sync()
    k = int(used.max())
    wmax = int(w.max())
    phi0 = (fscale * k * wmax + n) // (2 * n)
    phi_last = fscale * 2 * wmax
    col = torch.empty_like(col0)
    best_col = torch.empty_like(col0)
    best_f = torch.empty(pop, dtype=torch.int64, device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(args.warmup):
        col.copy_(col0)
        dlmcol.dlm_wvcp_iterated(ctx, g, k, pop, col, best_col, best_f, depth, max_ls, dlmcol.WVCP_TENURE, fscale,
                                 phi0, phi_last, SEED, 0, 0)
    ctx.sync()
    clocks = Clocks(0)
    clocks.start()
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(args.steps):
        col.copy_(col0)
        dlmcol.dlm_wvcp_iterated(ctx, g, k, pop, col, best_col, best_f, depth, max_ls, dlmcol.WVCP_TENURE, fscale,
                                 phi0, phi_last, SEED, 0, 0)
    e1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = e0.elapsed_time(e1)
    legal = best_f >= 0
    its = args.steps * pop * depth * max_ls  # every search runs its full depth (no early stop in WVCP)
    out = {"metric": "iterated weighted tabu moves/s, G(1000, 0.5), weights 1..100", "workload": "wvcp_iterated",
           "value": its / (ms / 1e3), "unit": "iterations/s", "higher_is_better": True, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "gpu_launches": args.steps * (2 * max_ls + 2),
           "clocks": ck, "data": "synthetic",
           "config": {"workload": f"G(1000, 0.5), weights 1..100, population {pop}, k = {k} (greedy), maxLSIters = "
                                  f"{max_ls} searches of {depth} iterations, phi0 = {phi0}/{fscale}, "
                                  f"phi_last = {phi_last}/{fscale}", "k": k,
                      "best_legal_f": int(best_f[legal].min()) if bool(legal.any()) else None,
                      "legal_individuals": int(legal.sum())}}
    print(json.dumps(out), flush=True)


def run_popsweep(args):
    """Sensitivity to the population size (section "Sensitivity to the population size", on k-COL
    here): G(500, 0.5), k = 47, random-GPX memetic search, the same total tabu budget (8192 x 4
    generations x 5000 iterations) for every population size; the line reports the best conflicts
    reached and the wall time per size."""
    import torch

    from paper_2109_05948_gb300 import build as libbuild
    from paper_2109_05948_gb300 import dlmcol, inputs

    libbuild.build()
    torch.cuda.set_device(0)
    ctx = dlmcol.Context(0)
    n, k, iters = 500, 47, 5000
    budget = 8192 * 4 * iters
    e = inputs.gnp(n, 0.5, SEED)
    g = dlmcol.Graph(ctx, n, torch.from_numpy(e).cuda())
    res = []
    for p in (128, 512, 2048, 8192):
        gens = max(1, budget // (p * iters))
        prm = dlmcol.MemeticParams(k=k, p=p, K=min(16, p - 1), iters=iters, tenure=dlmcol.COL_TENURE, use_scorer=0,
                                   epochs=0, batch=100, lr=1e-3, seed=2000 + p)
        mm = dlmcol.Memetic(ctx, g, prm)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        best = None
        for _ in range(gens):
            best = dlmcol.dlm_memetic_step(ctx, mm)
            if best == 0:
                break
        res.append({"population": p, "generations": gens, "best_conflicts": int(best),
                    "seconds": round(time.perf_counter() - t0, 3)})
        print(json.dumps({"progress": res[-1]}), file=sys.stderr, flush=True)
        mm.close()
    out = {"metric": "best conflicts at a fixed tabu budget vs population size, G(500, 0.5), k = 47",
           "workload": "popsweep", "value": min(r["best_conflicts"] for r in res), "unit": "conflicts",
           "higher_is_better": False, "data": "synthetic", "runs": res,
           "config": {"workload": f"G(500, 0.5), k = {k}, random GPX, K = 16, {iters} tabu iterations per generation, "
                                  f"total tabu budget {budget} iterations per population size"}}
    print(json.dumps(out), flush=True)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def pool_work(p: int, fit, sel, close_to_earlier):
    """Work of the pool update's greedy visit, reconstructed from its inputs and output: the number
    of candidates it examined and the number of (examined candidate, member kept before it) checks,
    each one entry of D. sel lists the greedily kept members in increasing (f, index) rank, then
    any fill; close_to_earlier[j] says whether sel[j] is within n/10 of some sel[i], i < j. A fill
    member is within n/10 of an earlier kept one, so the greedy prefix of sel ends at the first
    member that breaks the rank order or is close to an earlier member. The visit examines
    candidates until p are kept (all 2p when it falls short)."""
    import numpy as np

    m = 2 * p
    order = np.lexsort((np.arange(m), fit))
    rank = np.empty(m, np.int64)
    rank[order] = np.arange(m)
    r = rank[np.asarray(sel)]
    brk = np.array(close_to_earlier, dtype=bool, copy=True)
    brk[1:] |= np.diff(r) <= 0
    g_len = int(np.argmax(brk)) if brk.any() else p
    kept = np.zeros(m, bool)
    kept[np.asarray(sel)[:g_len]] = True
    before = np.concatenate([[0], np.cumsum(kept[order])[:-1]])
    stop = int(np.searchsorted(before, p)) if g_len >= p else m
    return stop, int(before[:stop].sum())


def run_population(args):
    """Population management and crossover of one generation at the planted n = 1000, k = 48,
    p = 8192, K = 32 size (sections "Distance computation", "Population update", "Parent matching
    and selection of crossovers"): distances P x P' and P' x P' (upper triangle), the pool update
    over the 2p candidates, the K nearest neighbours of the new population and GPX for its p K
    pairs. The colourings are TabuCol results (2 |V| iterations from random starts), so the
    overlap tables look like those of a running search. Each kernel is timed with CUDA events on
    the context's stream; value = distance pairs per second (the dominant kernel)."""
    import torch

    from paper_2109_05948_gb300 import build as libbuild
    from paper_2109_05948_gb300 import dlmcol, inputs

    libbuild.build()
    torch.cuda.set_device(0)
    ctx = dlmcol.Context(0)
    n, k, p, Kn, iters = 1000, 48, 8192, 32, 2000
    m = 2 * p
    dev = torch.device("cuda", 0)
    e, _ = inputs.planted(n, k, 0.5, seed=0)
    g = dlmcol.Graph(ctx, n, torch.from_numpy(e).to(dev))
    allc = torch.empty((m, n), dtype=torch.int16, device=dev)  # P (rows < p) then P'
    fit = torch.empty(m, dtype=torch.int64, device=dev)
    dlmcol.dlm_init_colors(ctx, n, k, m, SEED, 0, allc)
    dlmcol.dlm_tabucol_batch(ctx, g, k, m, allc, fit, None, iters, dlmcol.COL_TENURE, SEED, 0, 0)
    P, Sp = allc[:p], allc[p:]
    D = torch.zeros((m, m), dtype=torch.int16, device=dev)  # 512 MiB: larger than L2
    dlmcol.dlm_distance_batch(ctx, n, k, P, p, P, p, D, m, 0)
    sel = torch.empty(p, dtype=torch.int32, device=dev)
    nbr = torch.empty((p, Kn), dtype=torch.int32, device=dev)
    kids = torch.empty((p * Kn, n), dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream(dev)
    names = ("distance_PxPp", "distance_PpxPp", "pool_update", "knn", "gpx")
    tms = {nm: [] for nm in names}

    def timed(name, fn, rec):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        if rec:
            tms[name].append((a, b))

    def step(rec):
        timed("distance_PxPp", lambda: dlmcol.dlm_distance_batch(ctx, n, k, P, p, Sp, p, D[:, p:], m, 0), rec)
        timed("distance_PpxPp", lambda: dlmcol.dlm_distance_batch(ctx, n, k, Sp, p, Sp, p, D[p:, p:], m, 1), rec)
        # symmetric completion of the matrix (plumbing between the timed kernels)
        D[p:, :p] = D[:p, p:].t()
        lower = torch.tril(torch.ones((p, p), dtype=torch.bool, device=dev), -1)
        blk = D[p:, p:]
        blk[lower] = blk.t()[lower]
        del lower
        timed("pool_update", lambda: dlmcol.dlm_pool_update(ctx, p, n, fit, D, sel), rec)
        idx = sel.long()
        DP = D[idx][:, idx].contiguous()
        Pn = allc[idx].contiguous()
        timed("knn", lambda: dlmcol.dlm_knn(ctx, p, DP, Kn, nbr), rec)
        pairs = torch.stack([torch.arange(p, device=dev, dtype=torch.int32).repeat_interleave(Kn),
                             nbr.reshape(-1)], dim=1).contiguous()
        timed("gpx", lambda: dlmcol.dlm_gpx_batch(ctx, n, k, Pn, p, pairs, None, p * Kn, kids, SEED, 1), rec)
        return DP

    for _ in range(args.warmup):
        step(False)
    ctx.sync()
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    for _ in range(args.steps):
        DP = step(True)
    torch.cuda.synchronize()
    ctx.sync()
    ck = clocks.stop()
    ms = {nm: sum(a.elapsed_time(b) for a, b in tms[nm]) / len(tms[nm]) for nm in names}
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    hbm_src = "of measured (MEASURED_PEAKS.json hbm_gbs)"
    if hbm is None:
        hbm, hbm_src = 6800.0, "of fallback"
    smem = dlmcol.dlm_probe_smem_bandwidth(ctx)
    smem_src = "measured by dlm_probe_smem_bandwidth on this GPU (conflict-free 16 B loads)"
    f_np, s_np = fit.cpu().numpy(), sel.cpu().numpy()
    close = (10 * DP.int() <= n) & torch.tril(torch.ones((p, p), dtype=torch.bool, device=dev), -1)
    stop, pool_entries = pool_work(p, f_np, s_np, close.any(dim=1).cpu().numpy())
    del close

    def roof(bound, alg_bytes, t_ms, peak, src):
        a = alg_bytes / (t_ms / 1e3) / 1e9
        return {"bound": bound, "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak, "peak_source": src,
                "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": t_ms}

    pairs1, pairs2 = p * p, p * (p - 1) // 2
    # distance: per pair, n overlap-counter increments (u16 read-modify-write, 4 B each) and two
    # passes over the k x k u16 table (row maxima and column maxima, 4 k^2 B)
    dist_b = 4 * n + 4 * k * k
    kern = {
        "distance_PxPp": {"units": pairs1, "work_unit": "pairs", **roof("smem", dist_b * pairs1, ms["distance_PxPp"], smem, smem_src)},
        "distance_PpxPp": {"units": pairs2, "work_unit": "pairs", **roof("smem", dist_b * pairs2, ms["distance_PpxPp"], smem, smem_src)},
        # pool update: 2 B of D per (examined candidate, admitted member) check, from HBM
        "pool_update": {"units": stop, "work_unit": "candidates examined",
                        **roof("hbm", 2 * pool_entries, ms["pool_update"], hbm, hbm_src)},
        # KNN: every row of D (2 p B) read once, K int32 written
        "knn": {"units": p, "work_unit": "rows", **roof("hbm", p * (2 * p + 4 * Kn), ms["knn"], hbm, hbm_src)},
        # GPX: two parents (2 n B each) read and one child (2 n B) written
        "gpx": {"units": p * Kn, "work_unit": "children", **roof("hbm", p * Kn * 6 * n, ms["gpx"], hbm, hbm_src)},
    }
    dist_ms = ms["distance_PxPp"] + ms["distance_PpxPp"]
    top = dict(kern["distance_PxPp"])
    top.update({"kernel": "k_distance (P x P' launch)", "traffic": None})
    for v in kern.values():
        v["units_per_s"] = v["units"] / (v["kernel_ms"] / 1e3)
    out = {"metric": "population stage: distance pairs/s, n=1000, k=48, p=8192", "workload": "population",
           "value": (pairs1 + pairs2) / (dist_ms / 1e3), "unit": "pairs/s", "higher_is_better": True,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": sum(ms.values()),
           "dtype": "int16/int32", "data": "synthetic", "gpu_launches": 5 * args.steps, "clocks": ck,
           "roofline": top, "kernels": kern,
           "config": {"workload": f"planted 48-colourable n={n}, p={p} TabuCol results ({iters} iterations) as P and "
                                  f"P', K={Kn}: distances P x P' and P' x P' (upper), pool update over {m} "
                                  f"candidates, K nearest neighbours, GPX for {p * Kn} pairs",
                      "l2": "the 512 MiB distance matrix exceeds L2", "smem_probe_gbps": smem}}
    print(json.dumps(out), flush=True)
    g.close()
    ctx.close()


def run_scorer(args):
    """The scorer's share of one learned generation at the planted n = 1000, k = 48 size: score
    p K = 8192 x 32 GPX-sized candidates, then train on p = 8192 samples (N = 5 epochs, b = 100,
    Adam lr 1e-3). value = candidates scored per second; the roofline is the tensor-core GEMM
    kernel's, every launch timed with CUDA events on the context's stream."""
    import torch

    from paper_2109_05948_gb300 import build as libbuild
    from paper_2109_05948_gb300 import dlmcol, inputs

    libbuild.build()
    torch.cuda.set_device(0)
    ctx = dlmcol.Context(0)
    n, k, p, Kc, epochs, b = 1000, args.scorer_k, 8192, 32, args.scorer_epochs, 100
    C = p * Kc
    e = inputs.planted(n, k, 0.5, seed=0)[0] if k == 48 else inputs.gnp(n, 0.5, 0)
    g = dlmcol.Graph(ctx, n, torch.from_numpy(e).cuda())
    cand = torch.empty((C, n), dtype=torch.int16, device="cuda")
    dlmcol.dlm_init_colors(ctx, n, k, C, SEED, 0, cand)
    samples = cand[:p]
    fvals = torch.empty(p, dtype=torch.int64, device="cuda")
    dlmcol.dlm_gamma(ctx, g, k, p, samples, None, fvals)
    out = torch.empty(C, dtype=torch.float32, device="cuda")
    sc = dlmcol.Scorer(ctx, n, k, SEED)
    if args.scorer_split == 0:
        dlmcol.dlm_scorer_set_scoring_precision(ctx, sc, 0)
    stream = torch.cuda.current_stream()

    prof = {"fwd": [0.0, 0.0, 0], "train": [0.0, 0.0, 0]}

    def step(s, timed=False):
        dlmcol.dlm_score_offspring(ctx, sc, cand, C, out)
        evs[s][1].record(stream)
        if timed:  # the GEMM launches of the scoring pass, then of the training
            for key in ("fwd",):
                ms_, fl_, n_ = dlmcol.dlm_gemm_profile_read(ctx)
                prof[key] = [prof[key][0] + ms_, prof[key][1] + fl_, prof[key][2] + n_]
        dlmcol.dlm_scorer_train(ctx, sc, samples, fvals, p, epochs, b, 1e-3, SEED, s)
        if timed:
            ms_, fl_, n_ = dlmcol.dlm_gemm_profile_read(ctx)
            prof["train"] = [prof["train"][0] + ms_, prof["train"][1] + fl_, prof["train"][2] + n_]

    evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(3)) for _ in range(max(args.steps, args.warmup))]
    for w in range(args.warmup):
        step(w)
    ctx.sync()
    dlmcol.dlm_gemm_profile_read(ctx)  # clear
    dlmcol.dlm_gemm_profile(ctx, True)
    clocks = Clocks(0)
    clocks.start()
    torch.cuda.synchronize()
    for s in range(args.steps):
        evs[s][0].record(stream)
        step(s, timed=True)
        evs[s][2].record(stream)
    torch.cuda.synchronize()
    ctx.sync()
    ck = clocks.stop()
    dlmcol.dlm_gemm_profile(ctx, False)
    fwd_ms = sum(a.elapsed_time(m) for a, m, _ in evs[: args.steps])
    trn_ms = sum(m.elapsed_time(z) for _, m, z in evs[: args.steps])
    # algorithmic tensor work (the head and the class pooling run on CUDA cores): a forward pass is
    # 2 k (64 x 256 + 2 x 256 x 256) FLOP for the k class rows of a colouring plus 2 (64 x 256 +
    # 2 x 256 x 256) for its per-candidate Gamma terms; a training sample costs a forward pass and
    # a backward pass of twice that (input and weight gradients)
    fwd_flop = 2.0 * (k + 1) * (64 * 256 + 2 * 256 * 256)
    alg_fwd = args.steps * C * fwd_flop
    alg_trn = args.steps * p * epochs * 3 * fwd_flop
    alg = alg_fwd + alg_trn
    peaks = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained")
    src = "of measured (MEASURED_PEAKS.json bf16_tflops_sustained: the GEMMs run inside a long step)"
    if peak is None:
        peak, src = 1700.0, "of fallback (sustained bf16)"
    # the roofline is the scoring pass's GEMMs (large, one kernel per layer per 8192 candidates);
    # the training steps (batches of 100 candidates, latency bound) replay a CUDA graph, so their
    # GEMM launches carry no events and only the training time is reported
    fms, ffl, fn_ = prof["fwd"]
    achieved = alg_fwd / (fms / 1e3) / 1e12
    roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": "gemm_kernel (tcgen05, TMA, TMEM), scoring pass", "peak_source": src,
            "kernel_ms_per_launch": fms / max(1, fn_), "launches": fn_,
            "executed_tflops": ffl / (fms / 1e3) / 1e12, "executed_over_algorithmic": ffl / alg_fwd,
            "gemm_share_of_scoring": fms / fwd_ms}
    res = {"metric": f"scorer candidates/s, n=1000, k={k}", "workload": "scorer", "value": C * args.steps / (fwd_ms / 1e3),
           "unit": "candidates/s", "higher_is_better": True, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": (fwd_ms + trn_ms) / args.steps, "forward_ms_per_step": fwd_ms / args.steps,
           "train_ms_per_step": trn_ms / args.steps,
           "train_samples_per_s": p * epochs * args.steps / (trn_ms / 1e3), "dtype": "bf16 (fp32 accumulate)",
           "gpu_launches": None, "clocks": ck, "roofline": roof, "data": "synthetic",
           "config": {"workload": (f"planted 48-colourable n={n}" if k == 48 else f"G(n={n}, 0.5), k={k}") +
                                  f", {C} candidates ({p} x {Kc}) scored, training on "
                                  f"{p} samples, {epochs} epochs, batch {b}, scorer 64-d embedding + 3 x 256 "
                                  f"invariant layers (weights split hi/lo; training activations split; scoring "
                                  f"activations {'split' if args.scorer_split else 'bf16 alone'})"}}
    print(json.dumps(res), flush=True)
    sc.close()
    g.close()
    ctx.close()


def main():
    args = parse()
    if args.traffic_from:
        write_traffic(args.traffic_from, args.traffic_command)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "memetic":
        run_memetic(args)
        return
    if args.workload == "multi":
        run_multi(args)
        return
    if args.workload == "wvcp":
        run_wvcp(args)
        return
    if args.workload == "scorer":
        run_scorer(args)
        return
    if args.workload == "wvcp_iterated":
        run_wvcp_iterated(args)
        return
    if args.workload == "popsweep":
        run_popsweep(args)
        return
    if args.workload == "population":
        run_population(args)
        return
    if args.workload == "wvcp_memetic":
        run_wvcp_memetic(args)
        return
    if args.workload == "deepnet":
        run_deepnet(args)
        return
    import torch
    import torch.distributed as dist

    from paper_2109_05948_gb300 import build as libbuild
    from paper_2109_05948_gb300 import dlmcol, inputs

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        libbuild.build()
    if world > 1:
        dist.barrier()
    ctx = dlmcol.Context(local)
    dev = torch.device("cuda", local)
    e = inputs.gnp(N, P_EDGE, SEED)
    g = dlmcol.Graph(ctx, N, torch.from_numpy(e).to(dev))
    base, pop = shard(rank, args.pop)
    iters = args.iters
    col0 = torch.empty((pop, N), dtype=torch.int16, device=dev)
    dlmcol.dlm_init_colors(ctx, N, K, pop, SEED, base, col0)
    if args.warm_start > 0:
        wf = torch.empty(pop, dtype=torch.int64, device=dev)
        dlmcol.dlm_tabucol_batch(ctx, g, K, pop, col0, wf, None, args.warm_start, dlmcol.COL_TENURE, SEED, 1, base)
        ctx.sync()
    col = torch.empty_like(col0)
    best_f = torch.empty(pop, dtype=torch.int64, device=dev)
    moves = torch.zeros((max(1, args.steps), pop), dtype=torch.int64, device=dev)
    work = torch.zeros((max(1, args.steps), pop, 3), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    smem_gbps = dlmcol.dlm_probe_smem_bandwidth(ctx)
    l2_gbps = dlmcol.dlm_probe_l2_bandwidth(ctx)
    launch = dlmcol.dlm_tabucol_launch_info(ctx, g, K, pop, args.warps)
    stream = torch.cuda.current_stream(dev)

    def step(s, timed):
        col.copy_(col0)
        flush.fill_(s & 0xFF)
        if timed:
            kev[s][0].record(stream)
        dlmcol.dlm_tabucol_batch_ex(ctx, g, K, pop, col, best_f, moves[s if timed else 0], iters, dlmcol.COL_TENURE,
                                    SEED, 0, base, args.warps, None, work[s if timed else 0])
        if timed:
            kev[s][1].record(stream)

    kev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for w in range(args.warmup):
        step(w, False)
    ctx.sync()
    clocks = Clocks(local)
    if rank == 0:
        clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for s in range(args.steps):
        step(s, True)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    ctx.sync()
    if world > 1:
        dist.barrier()
    ck = clocks.stop() if rank == 0 else None
    ms = t0.elapsed_time(t1)
    kms = [a.elapsed_time(b) for a, b in kev]
    tot_moves = int(moves[: args.steps].sum().item())
    local_moves = tot_moves
    wk = work[: args.steps].sum(dim=(0, 1)).tolist()
    if world > 1:
        ms, tot_moves = reduce_over_ranks(dist, ms, tot_moves, dev)
    value = tot_moves / (ms / 1e3)

    # algorithmic bytes of one TabuCol iteration (the method's neighbourhood evaluation, whatever
    # the kernel does to avoid it): each conflicting vertex's k - 1 moves read a gamma and a tabu
    # entry (2 B + 2 B), each neighbour of the moved vertex has two u16 gamma read-modify-writes
    # (8 B), and each move reads the moved vertex's adjacency bit row (ceil(n / 8) B). The
    # conflicting rows and the degrees are counted by the kernel itself over the timed launches.
    alg_bytes = (4 * (K - 1) * wk[0] + 8 * wk[1] + ((N + 7) // 8) * local_moves) / args.steps
    # bytes the kernel itself moves in shared memory: the grouped kernel keeps every row's colour,
    # gamma[v][col v] and class summaries in its owner thread's registers, so it evaluates a
    # conflicting row without touching shared memory; each neighbour of a moved vertex costs two
    # gamma read-modify-writes (4 e B, e the entry size: 2 B, or 1 B with u8 entries), and each
    # move (the colour search of the moved vertex) and each row summarised again reads the row's
    # gamma entries with their tabu flags (e ks B, ks the row stride in entries)
    if launch["grouped"] == 2:
        esz, epw = 1, 4
    else:
        esz, epw = 2, 2
    kw = (K + epw - 1) // epw
    ks = epw * (kw if kw % 2 else kw + 1)
    kern_bytes = (4 * esz * wk[1] + esz * ks * (local_moves + wk[2])) / args.steps
    # L2: the moved vertex's adjacency bit row (ceil(n / 8) B per move) when the bit rows are not
    # held in shared memory
    l2_bytes = 0 if launch["bits_in_smem"] else ((N + 7) // 8) * local_moves / args.steps
    kmean = sum(kms) / len(kms)
    achieved = alg_bytes / (kmean / 1e3) / 1e9
    kern_gbps = kern_bytes / (kmean / 1e3) / 1e9
    l2_achieved = l2_bytes / (kmean / 1e3) / 1e9
    # cycles of one iteration of one individual: the launch's time at the sampled SM clock over the
    # iterations each individual slot runs
    sm_mhz = (ck or {}).get("sm_mhz") or 0.0
    slot_iters = pop * iters / max(1, launch["slots"])
    cyc_it = kmean * 1e-3 * sm_mhz * 1e6 / slot_iters if sm_mhz else None
    per_sm = launch["slots"] / max(1, min(launch["grid"], torch.cuda.get_device_properties(dev).multi_processor_count))
    roofline = {"bound": "smem", "achieved": achieved, "peak": smem_gbps, "unit": "GB/s",
                "frac": achieved / smem_gbps, "traffic": None,
                "kernel": "tabucol_group_kernel" if launch["grouped"] else "tabucol_batch_kernel", "kernel_ms": kmean,
                "algorithmic_bytes_per_launch": alg_bytes,
                "peak_source": "measured by dlm_probe_smem_bandwidth on this GPU (conflict-free 16 B loads)",
                "kernel_smem_bytes_per_launch": kern_bytes, "kernel_smem_gbps": kern_gbps,
                "kernel_smem_frac": kern_gbps / smem_gbps,
                "l2": {"achieved": l2_achieved, "peak": l2_gbps, "unit": "GB/s", "frac": l2_achieved / l2_gbps,
                       "bytes_per_launch": l2_bytes,
                       "peak_source": "measured by dlm_probe_l2_bandwidth on this GPU (L1-bypassing 16 B loads)"},
                "launch": launch,
                "cycles_per_iteration_per_individual": cyc_it,
                "cycles_per_iteration_per_sm": cyc_it / per_sm if cyc_it else None,
                "work": {"rows_evaluated_per_launch": wk[0] / args.steps,
                         "neighbour_updates_per_launch": wk[1] / args.steps,
                         "rows_resummarised_per_launch": wk[2] / args.steps}}
    rec = recorded_traffic()  # counters of one launch of this default workload, same kernel source
    if rec and pop == POP and iters == ITERS:
        roofline["traffic"] = rec["dram_bytes_per_launch"]
        roofline["traffic_source"] = os.path.relpath(TRAFFIC_JSON, ROOT)

    e2e = None
    if not args.no_e2e:
        # the same metric through the C-ABI with host buffers: start colourings copied in from
        # pinned host memory and best colourings, conflicts and moves copied back every step
        h_col0 = col0.cpu().pin_memory()
        h_col = torch.empty_like(h_col0).pin_memory()
        h_bf = torch.empty(pop, dtype=torch.int64).pin_memory()
        h_mv = torch.empty(pop, dtype=torch.int64).pin_memory()
        mvd = torch.zeros(pop, dtype=torch.int64, device=dev)
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0 = time.perf_counter()
        emoves = 0
        for s in range(args.steps):
            col.copy_(h_col0, non_blocking=True)
            dlmcol.dlm_tabucol_batch(ctx, g, K, pop, col, best_f, mvd, iters, dlmcol.COL_TENURE, SEED, 0, base)
            h_col.copy_(col, non_blocking=True)
            h_bf.copy_(best_f, non_blocking=True)
            h_mv.copy_(mvd, non_blocking=True)
            torch.cuda.synchronize(dev)
            emoves += int(h_mv.sum())
        el = time.perf_counter() - e0
        ctx.sync()
        if world > 1:
            el, emoves = reduce_over_ranks(dist, el, emoves, dev)
        e2e = {"value": emoves / el, "unit": UNIT, "h2d_bytes_per_step": pop * N * 2,
               "d2h_bytes_per_step": pop * N * 2 + 2 * pop * 8}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args)
    memetic = wmem = None
    if rank == 0 and world == 1 and not args.no_memetic and pop == POP and iters == ITERS:
        # the second half of the metric: learned selection against random GPX on the learned
        # workload (planted 48-colourable n = 1000, population 8192), 10 seeds per mode
        memetic = memetic_compare(args)
        # and on the weighted workload, where the memetic search has more to do
        wmem = wvcp_memetic_compare(args)
    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "int16/int32", "data": "synthetic",
               "config": config(args, {"smem_probe_gbps": smem_gbps}), "roofline": roofline,
               "cpu_baseline": cpu, "e2e": e2e, "clocks": ck, "gpu_launches": args.steps,
               "moves": tot_moves, "memetic_time_to_target": memetic, "wvcp_memetic_score_at_wall": wmem}
        print(json.dumps(out), flush=True)
    g.close()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
