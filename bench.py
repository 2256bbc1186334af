"""Benchmark: Monte Carlo samples/s and 1/(sigma^2 s) on a generated graph set,
learned+batched against the plain density.

Workload (default): all 28 three-loop vertex graphs without lepton loops.
Set-up (untimed, reported): compile the graphs; train one learned proposal
per graph on 2^20 plain samples (the network's own GPU kernels).
Timed step: every graph integrated over 2^24 fresh Philox samples in ONE
persistent batched launch with the learned mixture density (seed = step
number; under torchrun each rank adds rank * 1000003, so ranks draw disjoint
streams: weak scaling, no data-path collective; per-graph sums are merged
once at the end).  The plain density (one launch per graph, the same sample
budget) is timed after the timed region for the comparison.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle on a
bounded sample of the same workload instead.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MC samples/s and 1/(σ²·s) per graph set, learned+batched vs plain pdf, 1 B300"

# DRAM bytes (read + write) per batched_kernel launch in the default
# workload's timed region: ncu dram__bytes_read.sum + dram__bytes_write.sum,
# mean of the three launches of one step (53.4 MB read + 1206.8 MB write in
# all; profiles/batched_kernel_3loop_learned_set.md).  Set to None whenever
# the kernel changes until it is captured again.
TRAFFIC_DEFAULT_BYTES = 420.09e6


# FP64 operations of the table-driven elementary functions (one division
# counted as one operation): exp2 = range reduction (10) + degree-7 Horner
# (14) + table product; log2 = reduction (9) + 3-step Horner (6) + 5.
EXP2_OPS = 25
LOG2_OPS = 20
# the learned sampler's fused-multiply-add forms (FMA = 2): exp2 = reduction
# (2 + 1 + 2) + degree-6 Horner (12) + table product and scaling (2);
# log2 = reduction (5) + degree-7 Horner (14) + final FMA and sum (3)
FEXP2_OPS = 19
FLOG2_OPS = 22
# per sample, both forms: the weight y = I/g = I 2^(kf - log2 g) 2^-kf
# (floor, difference, exp2, product) and the double-double accumulation of
# sum y, sum y^2, sum |y| (three two-sum updates of 10 operations, one square)
ESTIMATOR_OPS = (3 + EXP2_OPS) + (3 * 10 + 1)


def sampler_flops(M, learned=False):
    """FP64 operations of one draw of the sampler and density (FMA = 2),
    counted from the steps of the code.

    Plain density: uniforms (4 ops each, 2M of them); M-1 walk steps
    (product, |T| additions, one log2, a product with 1/Deg and a sum);
    normalisation (M exp2 and sums, one log2, one reciprocal, M products and
    differences); three sector
    densities (3 ops per level) and the four-component mixture (4 exp2,
    one log2).

    Learned mixture: the same uniforms; M-1 walk steps of |T| additions, one
    log2, a product and a sum; normalisation (M exp2, M sums, one log2, one
    reciprocal, 2M products/differences); three sector densities; the
    learned density (5 ops per level); one five-term log-sum-exp (5 exp2, one
    log2), with the fused-multiply-add exp2/log2; its uniforms cost two
    additions each.

    Both forms add the estimator's own per-sample work (ESTIMATOR_OPS)."""
    if learned:
        walk = sum((M - l) + 2 + FLOG2_OPS for l in range(M - 1))
        norm = M * FEXP2_OPS + M + FLOG2_OPS + 1 + 2 * M
        pdf = 9 * (M - 1) + 14 + 5 * (M - 1) + 2 + 5 * (FEXP2_OPS + 2) + FLOG2_OPS + 1
        return 4 * M + walk + norm + pdf + ESTIMATOR_OPS
    walk = sum(1 + (M - l) + LOG2_OPS + 2 for l in range(M - 1))
    norm = M * EXP2_OPS + M + LOG2_OPS + 1 + 2 * M
    pdf = M + 3 * (M - 1) * 3 + 9 + 4 * (2 + EXP2_OPS) + LOG2_OPS + 2
    return 8 * M + 2 + walk + norm + pdf + ESTIMATOR_OPS


def oracle_rate(n_loops, graph_ids, per_graph, seed=0):
    """Time the CPU oracle (as it stands) on a bounded sample: the listed
    graphs, per_graph samples each, evaluation time after per-graph setup.
    Runs one process per host core (spawned)."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    jobs = []
    chunk = max(1, per_graph // max(1, cores // max(1, len(graph_ids))))
    for gi in graph_ids:
        for lo in range(0, per_graph, chunk):
            jobs.append((n_loops, gi, lo, min(chunk, per_graph - lo), seed))
    with mp.get_context("spawn").Pool(min(cores, len(jobs))) as pool:
        res = pool.map(_oracle_job, jobs)
    evals = sum(r[0] for r in res)
    eval_cpu_s = sum(r[1] for r in res)
    used = min(cores, len(jobs))
    wall = eval_cpu_s / used
    return evals / wall, used, evals, wall


def _oracle_job(args):
    n_loops, gi, lo, cnt, seed = args
    sys.path.insert(0, ROOT)
    from oracle.estimate import GraphOracle
    from oracle.graphs import enumerate_graphs
    o = GraphOracle(enumerate_graphs(n_loops)[gi], gi)
    t = time.perf_counter()
    o.samples(lo, cnt, seed)
    return cnt, time.perf_counter() - t


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons while timing."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, path):
        self.path = path
        self.p = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self, gpu_index):
        if self.p is None:
            return None
        self.p.terminate()
        self.p.wait()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9 or f[0] != str(gpu_index):
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    ids = [0, 13, 27]
    rate, cores, evals, wall = oracle_rate(3, ids, args.oracle_samples)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "3-loop vertex graphs without lepton loops, plain pdf",
                       "graphs": len(ids), "samples_per_graph": args.oracle_samples},
            "cpu_baseline": {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": "graphs %s of the 3-loop set, %d samples each, evaluation after "
                                       "per-graph setup, %.1f s" % (ids, args.oracle_samples, wall)},
            "e2e": {"value": rate, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line))


def merge(per_steps, ids, info):
    """Per-graph (sum y, sum y^2, N) over steps -> (value, sigma_down)."""
    import numpy as np
    sums = np.zeros((len(ids), 3))
    for per in per_steps:
        for i, p in enumerate(per):
            sums[i] += (p["sum_y"], p["sum_y2"], p["n"])
    return sums


def estimate(sums, info):
    val = var = 0.0
    for i in range(len(sums)):
        sy, sy2, N = sums[i]
        v1 = sy2 / N ** 2 - sy ** 2 / N ** 3
        val += info[i]["mult"] * sy / N
        var += info[i]["mult"] ** 2 * max(v1, 0.0)
    return val, math.sqrt(var)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--loops", type=int, default=3)
    ap.add_argument("--graphs", type=int, default=0,
                    help="seeded subset of this many graphs of the loop order (0: all of them)")
    ap.add_argument("--samples", type=int, default=1 << 24, help="samples per graph per step")
    ap.add_argument("--train", type=int, default=1 << 20, help="training samples per graph")
    ap.add_argument("--train-steps", type=int, default=150)
    ap.add_argument("--cost-ratio", type=float, default=0.0,
                    help="cost-aware proposal training: weight |y|/sqrt(1+R) for samples that need double-double")
    ap.add_argument("--plain", action="store_true", help="time the plain density only, one launch per graph")
    ap.add_argument("--plain-batched", action="store_true",
                    help="time the plain density in the batched persistent launch with pilot allocation")
    ap.add_argument("--no-alloc", action="store_true", help="equal samples per graph in the learned+batched form")
    ap.add_argument("--oracle-samples", type=int, default=96)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import paper_1909_08015_b300 as ae

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    stream = torch.cuda.current_stream()
    opts = ae.default_opts()
    opts.stream = stream.cuda_stream
    ctx = ae.Context(local, opts)
    t0 = time.perf_counter()
    canon = None
    if args.graphs > 0:
        total_graphs = {1: 1, 2: 4, 3: 28, 4: 269, 5: 3213}[args.loops]
        canon = ae.seeded_subset(total_graphs, min(args.graphs, total_graphs), 0)
        ngr = ctx.load_graph_subset(args.loops, canon)
    else:
        ngr = ctx.load_graphs(args.loops)
    compile_s = time.perf_counter() - t0
    ids = list(range(ngr))
    info = [ctx.graph_info(i) for i in ids]
    M = info[0]["M"]
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")   # 256 MB > L2
    learned = not args.plain and not args.plain_batched
    batched = not args.plain
    # initialisation pass (Sec. IV.A), plain density: 2^16 samples per graph; their mean |y|
    # becomes the graph's floor in the acceptance test of FP64 values (a
    # value is kept when its certified rounding bound, carried to y, is at
    # most 1e-10 max(|y|, floor); the rest are re-evaluated in double-double)
    t0 = time.perf_counter()
    _, _, per0 = ctx.integrate_batched(ids, [1 << 16] * ngr, seed=77 + rank)
    for i in ids:
        ctx.set_accept_floor(i, per0[i]["mean_abs"])
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0

    train_s = 0.0
    if learned:
        ctx.set_train_cost_ratio(args.cost_ratio)
        t0 = time.perf_counter()
        for i in ids:
            ctx.train_proposal(i, args.train, seed=7 + rank, steps=args.train_steps, lr=3e-3, beta=0.1)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0

    # inter-graph allocation (Sec. IV.C) from a pilot, for the learned+batched
    # form: the same total budget per step, split n_j ~ sigma_j / sqrt(t_j)
    alloc = [args.samples] * ngr
    pilot_s = 0.0
    if batched and not args.no_alloc:
        t0 = time.perf_counter()
        n_j, _ = ctx.allocate(ids, 1 << 18, args.samples * ngr, seed=99 + rank, mode=0)
        alloc = [int(x) for x in n_j]
        torch.cuda.synchronize()
        pilot_s = time.perf_counter() - t0

    def step(seed):
        if batched:
            return ctx.integrate_batched(ids, alloc, seed=seed + rank * 1000003)
        return ctx.integrate(ids, args.samples, seed=seed + rank * 1000003)

    for w in range(args.warmup):
        step(10 ** 6 + w)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(os.path.join(ROOT, "gpurun_out", "bench_clocks.csv") if os.path.isdir(
        os.path.join(ROOT, "gpurun_out")) else "/tmp/bench_clocks.csv")
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    dev_ms = 0.0
    e2e_s = 0.0
    per_all = []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(stream)
        v, s, per = step(k)
        ev1.record(stream)
        torch.cuda.synchronize()
        e2e_s += time.perf_counter() - t0
        dev_ms += ev0.elapsed_time(ev1)
        per_all.append(per)
    torch.cuda.nvtx.range_pop()
    ck = clocks.stop(local)
    t_dev = dev_ms / 1e3
    if dist:
        tt = torch.tensor([t_dev, e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_dev, e2e_s = tt.tolist()
    sums = merge(per_all, ids, info)
    if dist:
        ts = torch.tensor(sums, dtype=torch.float64, device="cuda")
        dist.all_reduce(ts)
        sums = ts.cpu().numpy()
    val, sigma = estimate(sums, info)
    total = args.samples * len(ids) * args.steps * world
    rate = total / t_dev
    # roofline of the dominant kernel: FP64 integrand kernel (sampler + tape)
    kern_s = sum(p["kernel_seconds"] for per in per_all for p in per)
    # device time of the whole step (FP64 kernels, queue sort, double-double
    # pass, reduction): the part after the FP64 kernels is reported apart
    step_s = sum(p["seconds"] for per in per_all for p in per)
    flops_per = [info[i]["flops"] + sampler_flops(M, learned) for i in ids]
    fl_total = sum(flops_per[i] * alloc[i] for i in ids) * args.steps
    achieved = fl_total / kern_s / 1e12
    launches = sum(p["launches"] for per in per_all for p in per)
    d2h = sum(p["d2h_bytes"] for per in per_all for p in per) / args.steps
    h2d = sum(p["h2d_bytes"] for per in per_all for p in per) / args.steps
    n_dd = sum(p["n_dd"] for per in per_all for p in per)
    zeroed = sum(p["n_nonfinite"] for per in per_all for p in per)
    # the plain density on the same budget, after the timed region
    plain = None
    if learned and rank == 0:
        for i in ids:
            ctx.set_proposal(i, 0)
        pp = []
        pt = 0.0
        for k in range(args.steps):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            _, _, per = ctx.integrate(ids, args.samples, seed=k)
            ev1.record(stream)
            torch.cuda.synchronize()
            pt += ev0.elapsed_time(ev1) / 1e3
            pp.append(per)
        pv, ps = estimate(merge(pp, ids, info), info)
        ptot = args.samples * len(ids) * args.steps
        plain = {"samples_per_s": ptot / pt, "inv_sigma2_per_s": 1.0 / (ps * ps * pt),
                 "value": pv, "sigma_down": ps, "seconds": pt,
                 "dd_reevaluated": int(sum(p["n_dd"] for per in pp for p in per))}
    peak = ctx.fp64_peak() if rank == 0 else 0.0
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cids = [0, ngr // 2, ngr - 1] if canon is None else [canon[0], canon[len(canon) // 2], canon[-1]]
        crate, cores, evals, wall = oracle_rate(args.loops, cids, args.oracle_samples)
        cpu = {"value": crate, "unit": "samples/s", "cores": cores, "kind": "oracle",
               "sample": "canonical graphs %s of the %d-loop list, %d samples each, plain density (evaluation "
                         "after per-graph setup, %.1f s on %d processes)" % (cids, args.loops, args.oracle_samples,
                                                                             wall, cores)}
    isps = 1.0 / (sigma ** 2 * t_dev) if sigma > 0 else None
    default_workload = (args.loops == 3 and args.graphs == 0 and args.samples == 1 << 24 and learned
                        and not args.no_alloc)
    traffic = TRAFFIC_DEFAULT_BYTES if default_workload else None
    line = {
        "metric": METRIC, "value": rate, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "%s %d %d-loop vertex graphs without lepton loops, %s" % (
                       "all" if canon is None else "seeded subset of", len(ids), args.loops,
                       "learned mixture density, one batched persistent launch per step" if learned
                       else "plain density, one batched persistent launch per step" if batched
                       else "plain density, one launch per graph"),
                   "samples_per_graph_per_step": args.samples, "seed": "step index (+ rank offset)",
                   "train_samples_per_graph": args.train if learned else 0,
                   "train_cost_ratio": args.cost_ratio if learned else None,
                   "l2": "256 MB buffer written between timed steps", "parallelism": "dp%d" % world},
        "inv_sigma2_per_s": isps,
        "inv_sigma2_per_s_incl_training": (1.0 / (sigma ** 2 * (t_dev + train_s + pilot_s + init_s)) if sigma > 0 else None),
        "estimate": {"value": val, "sigma_down": sigma, "samples": total, "dd_reevaluated": int(n_dd),
                     "zeroed": int(zeroed)},
        "dd_pass": {"reevaluated": int(n_dd), "zeroed": int(zeroed),
                    "seconds": max(step_s - kern_s, 0.0),
                    "share_of_step": (max(step_s - kern_s, 0.0) / step_s) if step_s > 0 else None,
                    "note": "double-double re-evaluation, queue sort and reduction; not credited to the FP64 fraction"},
        "plain_pdf": plain,
        "setup_seconds": {"compile": compile_s, "train": train_s, "pilot_allocation": pilot_s,
                          "initialisation": init_s},
        "allocation": {"min": min(alloc), "max": max(alloc), "mode": "pilot, n_j ~ sigma_j/sqrt(t_j)"}
        if batched and not args.no_alloc else None,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None, "traffic": traffic,
                     "kernel": ("batched_kernel" if batched else "integrate_kernel") + " (sampler + FP64 tape)",
                     "peak_source": "measured: own DFMA probe (ae_fp64_peak)"},
        "e2e": {"value": total / e2e_s, "unit": "samples/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "paper_v100": {"note": "context, not a target: the paper's own figures (five-loop set, Calc 2)",
                       "hardware": "NVIDIA Tesla V100, supercomputer Govorun (JINR)",
                       "integrand_gflops_eia": 2227.99, "samples_per_s_all_phases_derived": 2.32e6,
                       "eia_fraction_of_v100_fp64_peak_derived": 0.297},
        "clocks": ck,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
