"""Small, self-contained integration case for profiling the kernels (a
test-suite helper: the ncu summaries under profiles/ name it in their
commands).

    python tests/profile_case.py --loops 4 --graphs 8

loads a seeded subset of graphs (optionally trains a learned proposal for
each), runs one per-graph integration of graph 0 and two batched
integrations of the subset (the first one tunes; the second one runs inside
the NVTX range "measure").  With --no-dd the double-double
re-evaluation is switched off so that the FP64 kernels can be captured alone.
"""
import argparse
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_1909_08015_b300 import Context, default_opts, seeded_subset  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--loops", type=int, default=4)
    ap.add_argument("--graphs", type=int, default=8)
    ap.add_argument("--samples", type=int, default=1 << 17)
    ap.add_argument("--no-dd", action="store_true")
    ap.add_argument("--learned", type=int, default=0,
                    help="train a learned proposal for every graph with this many steps first")
    ap.add_argument("--paper-accept", action="store_true",
                    help="the paper's acceptance widths from an initialisation pass")
    ap.add_argument("--peak", action="store_true", help="also run the FP64 peak probe")
    a = ap.parse_args()
    o = default_opts()
    if a.no_dd:
        o.dd_tol = 0.0
    c = Context(0, o)
    total = {1: 1, 2: 4, 3: 28, 4: 269, 5: 3213}[a.loops]
    ids = seeded_subset(total, min(a.graphs, total), 0)
    n = c.load_graph_subset(a.loops, ids)
    if a.paper_accept:
        from paper_1909_08015_b300 import accept_widths
        _, _, per0 = c.integrate_batched(list(range(n)), [1 << 16] * n, seed=77)
        w = accept_widths([p["sigma"] for p in per0])
        for g in range(n):
            c.set_accept_width(g, w[g])
    if a.learned:
        for g in range(n):
            c.train_proposal(g, 1 << 18, seed=7, steps=a.learned, lr=3e-3, beta=0.1)
    c.integrate([0], a.samples, 1)
    c.integrate_batched(list(range(n)), [a.samples // 2] * n, seed=1)   # tunes
    # the tuned batched launch again, inside the NVTX range "measure" (for
    # profilers that filter by range)
    import torch
    torch.cuda.nvtx.range_push("measure")
    _, _, per = c.integrate_batched(list(range(n)), [a.samples // 2] * n, seed=2)
    torch.cuda.nvtx.range_pop()
    if a.peak:
        print("fp64 peak probe %.4f TFLOP/s" % c.fp64_peak())
    print("ok", n, "samples", sum(p["n"] for p in per), "re-evaluated", sum(p["n_dd"] for p in per),
          "device s %.4f fp64 kernel s %.4f" % (sum(p["seconds"] for p in per), sum(p["kernel_seconds"] for p in per)))


if __name__ == "__main__":
    main()
