"""A resumable integration campaign over a gauge-invariant class of graphs
(Sec. V, Table I), driven through the library's run calls.

    python -m paper_1909_08015_b300.campaign --loops 5 --klass 5 0 0 \\
        --checkpoint run.ckpt --seconds 900 --summary summary.txt

Every call: load the class's graphs (ae_graph_classes, ae_load_graph_subset),
an initialisation pass of the plain density whose sigma_down sets the widths
of the paper's acceptance test (Eq. eq_interval_accept), train the learned
proposals (fixed seeds: every call rebuilds the same densities), split each
block over the graphs from a pilot (n_j ~ sigma_j / sqrt(t_j), Sec. IV.C),
then resume the run from the checkpoint (if it exists) and add blocks until
the time budget is spent, writing the checkpoint after every block.  The
estimate (value, sigma_down, sigma_up) after each call is appended to the
summary file.  All arithmetic runs in libae; this module only orders calls.
"""
import argparse
import os
import time

from . import Context, accept_widths, default_opts, graph_classes


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--loops", type=int, default=5)
    ap.add_argument("--klass", type=int, nargs=3, default=[5, 0, 0])
    ap.add_argument("--checkpoint", required=True)
    ap.add_argument("--summary", default=None)
    ap.add_argument("--seconds", type=float, default=600.0, help="time budget of the blocks")
    ap.add_argument("--block", type=int, default=1 << 25, help="samples per block (all graphs)")
    ap.add_argument("--seed", type=int, default=2019)
    ap.add_argument("--learned", type=int, default=1, help="1: learned proposals, 0: plain density")
    ap.add_argument("--train", type=int, default=1 << 20)
    ap.add_argument("--train-steps", type=int, default=150)
    ap.add_argument("--deg-max", type=float, default=None, help="cap on Deg(s) (ae_opts.deg_max; default 1)")
    a = ap.parse_args()

    t_start = time.perf_counter()
    klass, _ = graph_classes(a.loops)
    ids = [i for i, k in enumerate(klass.tolist()) if k == list(a.klass)]
    if not ids:
        raise SystemExit("no graph of class %s at %d loops" % (a.klass, a.loops))
    opts = default_opts()
    if a.deg_max is not None:
        opts.deg_max = a.deg_max
    ctx = Context(0, opts)
    n = ctx.load_graph_subset(a.loops, ids)
    loc = list(range(n))
    t_load = time.perf_counter() - t_start
    _, _, per0 = ctx.integrate_batched(loc, [1 << 16] * n, seed=77)
    widths = accept_widths([p["sigma"] for p in per0])
    for i in loc:
        ctx.set_accept_width(i, widths[i])
    if a.learned:
        for i in loc:
            ctx.train_proposal(i, a.train, seed=7, steps=a.train_steps, lr=3e-3, beta=0.1)
    n_j, _ = ctx.allocate(loc, 1 << 16, a.block, seed=99, mode=0)
    alloc = [int(x) for x in n_j]
    ctx.run_reset(a.seed)
    if os.path.exists(a.checkpoint):
        ctx.resume(a.checkpoint)
    t_setup = time.perf_counter() - t_start
    t0 = time.perf_counter()
    blocks = 0
    while time.perf_counter() - t0 < a.seconds:
        ctx.run_step(loc, alloc)
        ctx.checkpoint(a.checkpoint)
        blocks += 1
    t_run = time.perf_counter() - t0
    v, s, su, per = ctx.run_estimate()
    N = sum(p["n"] for p in per)
    heavy = sum(1 for p in per if p["n"] and p["max_y2"] > 0.5 * p["sum_y2"])
    line = ("class %s loops %d graphs %d (%s, deg_max %s): N %d value %.6f sigma_down %.6f sigma_up %.6f "
            "re-evaluated %d zeroed %d, graphs with one sample over half of sum y^2: %d | this call: %d blocks "
            "in %.1f s (%.3g samples/s), set-up %.1f s (load %.1f s)"
            % (tuple(a.klass), a.loops, n, "learned" if a.learned else "plain", opts.deg_max, N, v, s, su,
               sum(p["n_dd"] for p in per), sum(p["n_nonfinite"] for p in per), heavy, blocks, t_run,
               blocks * a.block / max(t_run, 1e-9), t_setup, t_load))
    print(line)
    if a.summary:
        with open(a.summary, "a") as f:
            f.write(line + "\n")
    ctx.close()


if __name__ == "__main__":
    main()
