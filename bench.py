"""Benchmark: Monte Carlo samples/s and 1/(sigma^2 s) on a generated graph set,
learned+batched against the plain density at equal wall time.

Workload (default): 20 four-loop vertex graphs without lepton loops, chosen
from the 269 by the library's Philox-seeded shuffle (ae_seeded_subset, seed
0).  Set-up (untimed, reported): compile the graphs; an initialisation pass
(plain density, 2^16 samples per graph) whose sigma_down sets the widths of
the paper's acceptance test (Sec. IV.A, Eq. eq_interval_accept); train one
learned proposal per graph on the GPU (its own kernels; 2^24 plain samples,
300 full-batch Adam steps); a pilot that splits
each step's budget over the graphs (n_j ~ sigma_j / sqrt(t_j), Sec. IV.C).

Timed step: one block of a run (ae_run_step): every graph continues its own
Philox stream by its allocated count, all in ONE persistent batched launch
with the learned mixture density, captured in a CUDA graph.  Under torchrun
each rank runs its own stream (seed offset by rank): weak scaling, no
data-path collective; the per-graph sums are merged once at the end.

After the timed region (rank 0): the plain density in the same batched,
allocated form, with the step budget scaled so that the same number of
steps takes the same device time (equal wall time); and a few learned steps
under the other acceptance test (the library's relative one), so that both
modes are reported.

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
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MC samples/s and 1/(σ²·s) per graph set, learned+batched vs plain pdf, 1 B300"
N_GRAPHS = {1: 1, 2: 4, 3: 28, 4: 269, 5: 3213}

# DRAM bytes (read + write) per launch of the dominant kernel (batched_kernel)
# in the default workload's timed step: ncu dram__bytes_read.sum +
# dram__bytes_write.sum of the step's three launches (13.9, 17.6 and 9.3 MB;
# one-pass capture, profiles/bench_4loop_20graphs_launches.md), their mean.
# Tapes, tables, chunk partials and the re-evaluation queue: about one byte
# per sample against some 4e4 FP64 flops.  Set to None whenever the kernel
# changes until it is captured again.
TRAFFIC_DEFAULT_BYTES = 13.6e6

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
    differences); three sector densities (3 ops per level) and the
    four-component mixture (4 exp2, one log2).

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


def workload_graphs(loops, graphs):
    """Canonical ids of the workload's graphs (all, or the seeded subset)."""
    import paper_1909_08015_b300 as ae
    total = N_GRAPHS[loops]
    if graphs <= 0 or graphs >= total:
        return list(range(total))
    return ae.seeded_subset(total, graphs, 0)


GOLDEN = os.path.join(ROOT, "tests", "golden")


def stored_tables(n_loops, gi):
    """Path of the oracle's stored coefficient tables of a graph, or None
    (written by tests/golden/make_oracle_tables.py: at four loops the
    oracle's own set-up of one graph takes 8 to 30+ minutes)."""
    p = os.path.join(GOLDEN, "oracle_tables_%dloop_%d.json.gz" % (n_loops, gi))
    return p if os.path.exists(p) else None


def baseline_graphs(n_loops, canon):
    """Graphs of the workload the CPU baseline times: at four loops and more
    those whose oracle tables are stored (none: no bounded sample exists),
    else the first, middle and last."""
    if n_loops >= 4:
        return [g for g in canon if stored_tables(n_loops, g)]
    return [canon[0], canon[len(canon) // 2], canon[-1]]


NO_ORACLE_SAMPLE = ("not measured: the oracle's own set-up of one graph of this workload takes from minutes "
               "(four loops) to hours (five loops), and no stored coefficient tables cover it")


def oracle_rate(n_loops, canon_ids, per_graph, seed=0):
    """Time the CPU oracle (as it stands) on a bounded sample: the listed
    graphs, per_graph samples each (plain density), evaluation time after
    each worker's per-graph set-up (stored coefficient tables where they
    exist); one spawned process per host core."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    per_core = max(1, cores // max(1, len(canon_ids)))
    chunk = max(1, (per_graph + per_core - 1) // per_core)
    jobs = []
    for gi in canon_ids:
        for lo in range(0, per_graph, chunk):
            jobs.append((n_loops, gi, lo, min(chunk, per_graph - lo), seed))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(min(cores, len(jobs))) as pool:
        res = pool.map(_oracle_job, jobs)
    wall_all = time.perf_counter() - t0
    evals = sum(r[0] for r in res)
    used = min(cores, len(jobs))
    eval_wall = sum(r[1] for r in res) / used
    setup = max(r[2] for r in res)
    stored = [gi for gi in canon_ids if stored_tables(n_loops, gi)]
    return evals / eval_wall, used, evals, eval_wall, setup, wall_all, stored


def _oracle_job(args):
    n_loops, gi, lo, cnt, seed = args
    sys.path.insert(0, ROOT)
    import gzip
    from oracle.estimate import GraphOracle
    from oracle.graphs import enumerate_graphs
    from oracle.integrand import Integrand
    t = time.perf_counter()
    tables = None
    path = stored_tables(n_loops, gi)
    if path:
        with gzip.open(path, "rt") as f:
            tables = Integrand.tables_from_records(json.load(f)["tables"])
    o = GraphOracle(enumerate_graphs(n_loops)[gi], gi, tables=tables)
    setup = time.perf_counter() - t
    t = time.perf_counter()
    o.samples(lo, cnt, seed)
    return cnt, time.perf_counter() - t, setup


def oracle_samples_default(n_loops, n_graphs=1):
    """Samples per graph for about 10-30 s of oracle evaluation on the host."""
    cores = os.cpu_count() or 1
    return {1: 4096, 2: 2048, 3: 96}.get(n_loops, max(1, 16 * cores // max(1, n_graphs)))


def cpu_sample_text(cids, n_loops, per_graph, wall, cores, setup, stored):
    txt = ("canonical graphs %s of the %d-loop list, %d samples each, plain density, exact evaluation; "
           "%.1f s on %d processes after a per-graph set-up of up to %.1f s" % (cids, n_loops, per_graph, wall,
                                                                               cores, setup))
    if stored:
        txt += ("; the coefficient tables of %s are read from tests/golden (written by "
                "tests/golden/make_oracle_tables.py: their own set-up takes 8 to 30+ minutes per graph)" % stored)
    return txt


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


def workload_name(loops, n, total, learned_vs_plain=True):
    what = ("%d seeded %d-loop vertex graphs without lepton loops (Philox-seeded subset of the %d)"
            % (n, loops, total)) if n < total else ("all %d %d-loop vertex graphs without lepton loops" % (n, loops))
    return what + (", learned mixture density vs plain density at equal wall time, one batched persistent "
                   "launch per step" if learned_vs_plain else ", plain density, one batched persistent launch per step")


def run_reference(args, rank, world):
    """The oracle (plain, unoptimised CPU restatement) on a bounded sample of
    the same workload; rank 0 only."""
    if rank != 0:
        return
    canon = workload_graphs(args.loops, args.graphs)
    cids = baseline_graphs(args.loops, canon)
    if not cids:
        print(json.dumps({"impl": "reference", "unavailable": NO_ORACLE_SAMPLE}))
        return
    per = args.oracle_samples or oracle_samples_default(args.loops, len(cids))
    rate, cores, evals, wall, setup, wall_all, stored = oracle_rate(args.loops, cids, per)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "samples/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.loops, len(canon), N_GRAPHS[args.loops]),
                       "oracle_graphs": cids, "samples_per_graph": per},
            "cpu_baseline": {"value": rate, "unit": "samples/s", "cores": cores, "kind": "oracle",
                             "sample": cpu_sample_text(cids, args.loops, per, wall, cores, setup, stored)},
            "e2e": {"value": rate, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--loops", type=int, default=4)
    ap.add_argument("--graphs", type=int, default=20,
                    help="seeded subset of this many graphs of the loop order (0: all of them)")
    ap.add_argument("--samples", type=int, default=1 << 21, help="mean samples per graph per step")
    ap.add_argument("--train", type=int, default=1 << 24, help="training samples per graph")
    ap.add_argument("--train-steps", type=int, default=300)
    ap.add_argument("--beta", type=float, default=0.1, help="weight of the plain density in the learned mixture")
    ap.add_argument("--refine", type=int, default=0,
                    help="rounds of proposal refinement on samples of the current mixture (--train samples each)")
    ap.add_argument("--refine-steps", type=int, default=150)
    ap.add_argument("--seed", type=int, default=0, help="run seed of the timed steps (rank offsets added)")
    ap.add_argument("--cost-ratio", type=float, default=0.0,
                    help="cost-aware proposal training: weight |y|/sqrt(1+R) for samples that need double-double")
    ap.add_argument("--accept", default="paper", choices=["paper", "relative"],
                    help="acceptance test of FP64 values: the paper's interval width (Eq. eq_interval_accept) "
                         "or the library's relative 1e-10 test")
    ap.add_argument("--plain", action="store_true", help="time the plain density only (no training)")
    ap.add_argument("--no-compare", action="store_true", help="skip the plain and other-acceptance arms")
    ap.add_argument("--init-samples", type=int, default=1 << 16)
    ap.add_argument("--pilot", type=int, default=1 << 18)
    ap.add_argument("--oracle-samples", type=int, default=0, help="CPU baseline samples per graph (0: auto)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-file", default=None, help="where nvidia-smi samples go (default: a temp file)")
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
    from paper_1909_08015_b300.runstate import rank_seed

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
    canon = workload_graphs(args.loops, args.graphs)
    ngr = ctx.load_graph_subset(args.loops, canon)
    compile_s = time.perf_counter() - t0
    ids = list(range(ngr))
    info = [ctx.graph_info(i) for i in ids]
    M = info[0]["M"]
    flush = torch.empty(64 << 20, dtype=torch.float32, device="cuda")   # 256 MB > L2
    learned = not args.plain

    # initialisation pass (Sec. IV.A), plain density: sigma_down per graph
    # sets the widths of the paper's acceptance test; mean |y| the floor of
    # the library's relative test
    t0 = time.perf_counter()
    _, _, per0 = ctx.integrate_batched(ids, [args.init_samples] * ngr, seed=77 + rank)
    widths = ae.accept_widths([p["sigma"] for p in per0])

    def set_accept(mode):
        for i in ids:
            if mode == "paper":
                ctx.set_accept_width(i, widths[i])
            else:
                ctx.set_accept_width(i, 0.0)
                ctx.set_accept_floor(i, per0[i]["mean_abs"])
    set_accept(args.accept)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0

    train_s = 0.0
    if learned:
        ctx.set_train_cost_ratio(args.cost_ratio)
        t0 = time.perf_counter()
        for i in ids:
            ctx.train_proposal(i, args.train, seed=7 + rank, steps=args.train_steps, lr=3e-3, beta=args.beta)
            for r in range(args.refine):
                ctx.refine_proposal(i, args.train, seed=17 + r + rank, steps=args.refine_steps, lr=1e-3)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0

    def allocate():
        n_j, _ = ctx.allocate(ids, args.pilot, args.samples * ngr, seed=99 + rank, mode=0)
        return [int(x) for x in n_j]

    t0 = time.perf_counter()
    alloc = allocate()
    torch.cuda.synchronize()
    pilot_s = time.perf_counter() - t0

    def timed_steps(alloc_, steps, seed, flush_l2=True):
        """steps run blocks timed with CUDA events on the launching stream;
        returns (device seconds, host seconds, per-step results)."""
        ctx.run_reset(seed)
        dev_ms = 0.0
        host_s = 0.0
        per_steps = []
        for _ in range(steps):
            if flush_l2:
                flush.zero_()
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            t = time.perf_counter()
            ev0.record(stream)
            per = ctx.run_step(ids, alloc_)
            ev1.record(stream)
            torch.cuda.synchronize()
            host_s += time.perf_counter() - t
            dev_ms += ev0.elapsed_time(ev1)
            per_steps.append(per)
        return dev_ms / 1e3, host_s, per_steps

    # warm-up (tunes, captures the step's CUDA graph), then the timed region
    timed_steps(alloc, args.warmup, 10 ** 6 + rank)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks_path = args.clocks_file or os.path.join(tempfile.gettempdir(), "bench_clocks_%d.csv" % os.getpid())
    clocks = Clocks(clocks_path)
    clocks.start()
    torch.cuda.nvtx.range_push("timed")
    t_dev, e2e_s, per_all = timed_steps(alloc, args.steps, rank_seed(args.seed, rank))
    torch.cuda.nvtx.range_pop()
    ck = clocks.stop(local)
    if dist:
        tt = torch.tensor([t_dev, e2e_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_dev, e2e_s = tt.tolist()
        from paper_1909_08015_b300.runstate import RunState
        RunState.attach(ctx).merge_ranks()
    val, sigma, sigma_up, per_run = ctx.run_estimate()
    total = sum(alloc) * args.steps * world
    rate = total / t_dev
    isps = 1.0 / (sigma ** 2 * t_dev) if sigma > 0 else None

    # roofline of the dominant kernel: the FP64 integrand kernel (sampler + tape)
    kern_s = sum(p["kernel_seconds"] for per in per_all for p in per)
    step_s = sum(p["seconds"] for per in per_all for p in per)
    flops_per = [info[i]["flops"] + sampler_flops(M, learned) for i in ids]
    twin_per = [info[i]["flops_bound"] for i in ids]
    fl_total = sum(flops_per[i] * alloc[i] for i in ids) * args.steps
    fl_method = sum((flops_per[i] - twin_per[i]) * alloc[i] for i in ids) * args.steps
    achieved = fl_total / kern_s / 1e12
    launches = sum(p["launches"] for per in per_all for p in per)
    d2h = sum(p["d2h_bytes"] for per in per_all for p in per) / args.steps
    h2d = sum(p["h2d_bytes"] for per in per_all for p in per) / args.steps
    n_dd = sum(p["n_dd"] for per in per_all for p in per)
    zeroed = sum(p["n_nonfinite"] for per in per_all for p in per)
    # the double-double pass's own work: re-evaluated samples x (double-double
    # tape flops + sampler), over the device time after the FP64 kernels
    dd_s = max(step_s - kern_s, 0.0)
    dd_fl = sum((info[i]["flops_dd"] + sampler_flops(M, learned)) * per[i]["n_dd"] for per in per_all for i in ids)

    plain = other = None
    if rank == 0 and learned and not args.no_compare:
        # the other acceptance test, same learned proposal, a few steps
        other_mode = "relative" if args.accept == "paper" else "paper"
        set_accept(other_mode)
        k2 = min(args.steps, 3)
        timed_steps(alloc, 1, 2 * 10 ** 6)
        o_dev, _, o_per = timed_steps(alloc, k2, 3 * 10 ** 6)
        o_val, o_sig, _, _ = ctx.run_estimate()
        o_steps = sum(p["seconds"] for per in o_per for p in per)
        o_kern = sum(p["kernel_seconds"] for per in o_per for p in per)
        other = {"accept": other_mode, "steps": k2, "samples_per_s": sum(alloc) * k2 / o_dev,
                 "inv_sigma2_per_s": 1.0 / (o_sig ** 2 * o_dev) if o_sig > 0 else None,
                 "value": o_val, "sigma_down": o_sig,
                 "dd_reevaluated": int(sum(p["n_dd"] for per in o_per for p in per)),
                 "dd_share_of_step": max(o_steps - o_kern, 0.0) / o_steps if o_steps > 0 else None}
        set_accept(args.accept)
        # the plain density in the same batched, allocated form, at equal
        # device time: its own pilot allocation, the step budget scaled by
        # the measured time per sample of one plain step
        for i in ids:
            ctx.set_proposal(i, 0)
        alloc_p = allocate()
        p_dev1, _, _ = timed_steps(alloc_p, 1, 4 * 10 ** 6)
        scale = (t_dev / args.steps) / max(p_dev1, 1e-9)
        alloc_p = [max(1, int(round(n * scale))) for n in alloc_p]
        p_dev, _, p_per = timed_steps(alloc_p, args.steps, 5 * 10 ** 6)
        p_val, p_sig, p_up, _ = ctx.run_estimate()
        p_steps = sum(p["seconds"] for per in p_per for p in per)
        p_kern = sum(p["kernel_seconds"] for per in p_per for p in per)
        plain = {"samples_per_s": sum(alloc_p) * args.steps / p_dev,
                 "inv_sigma2_per_s": 1.0 / (p_sig ** 2 * p_dev) if p_sig > 0 else None,
                 "value": p_val, "sigma_down": p_sig, "sigma_up": p_up, "seconds": p_dev,
                 "seconds_learned": t_dev, "samples": sum(alloc_p) * args.steps,
                 "dd_reevaluated": int(sum(p["n_dd"] for per in p_per for p in per)),
                 "dd_share_of_step": max(p_steps - p_kern, 0.0) / p_steps if p_steps > 0 else None,
                 "form": "same batched launch, own pilot allocation, step budget scaled to equal device time"}
        for i in ids:
            ctx.set_proposal(i, 1, args.beta)
    peak = ctx.fp64_peak() if rank == 0 else 0.0
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cids = baseline_graphs(args.loops, canon)
        if cids:
            per = args.oracle_samples or oracle_samples_default(args.loops, len(cids))
            crate, cores, evals, wall, setup, _, stored = oracle_rate(args.loops, cids, per)
            cpu = {"value": crate, "unit": "samples/s", "cores": cores, "kind": "oracle",
                   "sample": cpu_sample_text(cids, args.loops, per, wall, cores, setup, stored)}
        else:
            cpu = {"value": None, "unit": "samples/s", "cores": os.cpu_count(), "kind": "oracle",
                   "sample": NO_ORACLE_SAMPLE}
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    default_workload = (args.loops == 4 and args.graphs == 20 and args.samples == 1 << 21 and learned
                        and args.accept == "paper")
    nominal = 2 * 2 * sms * (ck["sm_mhz"] if ck else 2032.0) * 1e6 / 1e12   # 2 DFMA/SM/clk, FMA = 2 flops
    line = {
        "metric": METRIC, "value": rate, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_dev * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.loops, ngr, N_GRAPHS[args.loops], learned),
                   "canonical_ids": canon if ngr < N_GRAPHS[args.loops] else "all",
                   "samples_per_step": sum(alloc), "seed": "run seed (+ rank offset), counters continue",
                   "acceptance": args.accept, "train_samples_per_graph": args.train if learned else 0,
                   "train_steps": args.train_steps if learned else 0,
                   "refine_rounds": args.refine if learned else 0,
                   "train_cost_ratio": args.cost_ratio if learned else None,
                   "beta": args.beta if learned else None,
                   "init_samples_per_graph": args.init_samples, "pilot_samples_per_graph": args.pilot,
                   "l2": "256 MB buffer written between timed steps", "parallelism": "dp%d" % world},
        "inv_sigma2_per_s": isps,
        "inv_sigma2_per_s_incl_setup": (1.0 / (sigma ** 2 * (t_dev + train_s + pilot_s + init_s))
                                        if sigma > 0 else None),
        "estimate": {"value": val, "sigma_down": sigma, "sigma_up": sigma_up, "samples": total,
                     "dd_reevaluated": int(n_dd), "zeroed": int(zeroed)},
        "dd_pass": {"reevaluated": int(n_dd), "zeroed": int(zeroed), "seconds": dd_s,
                    "share_of_step": (dd_s / step_s) if step_s > 0 else None,
                    "achieved_tflops": dd_fl / dd_s / 1e12 if dd_s > 0 else None,
                    "frac": dd_fl / dd_s / 1e12 / peak if dd_s > 0 and peak else None,
                    "note": "double-double re-evaluation, queue sort and reduction; not credited to the FP64 "
                            "fraction; its own frac counts the double-double tape's FP64 flops (FMA = 2) "
                            "against the same measured peak"},
        "plain_pdf": plain,
        "gain_vs_plain": ({"inv_sigma2_per_s": isps / plain["inv_sigma2_per_s"],
                           "note": "learned+batched over plain+batched, equal device time"}
                          if plain and isps and plain["inv_sigma2_per_s"] else None),
        "other_acceptance": other,
        "setup_seconds": {"compile": compile_s, "train": train_s, "pilot_allocation": pilot_s,
                          "initialisation": init_s},
        "allocation": {"min": min(alloc), "max": max(alloc), "mode": "pilot, n_j ~ sigma_j/sqrt(t_j)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak if peak else None,
                     "traffic": TRAFFIC_DEFAULT_BYTES if default_workload else None,
                     "kernel": "batched_kernel (sampler + FP64 tape)",
                     "peak_source": "measured: own DFMA probe (ae_fp64_peak)",
                     "peak_nominal": nominal, "frac_vs_nominal": achieved / nominal,
                     "frac_method_only": fl_method / kern_s / 1e12 / peak if peak else None,
                     "note": "nominal = 2 DFMA per SM per cycle at the median SM clock; method_only leaves out "
                             "the certified bound's magnitude twins"},
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
