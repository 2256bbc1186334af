"""Small, self-contained integration case for profiling the kernels.

    python -m paper_1909_08015_b300.profile_case --loops 4 --graphs 8

loads a seeded subset of graphs, runs one per-graph integration of graph 0
and one batched integration of the subset.  With --no-dd the double-double
re-evaluation is switched off so that the FP64 kernels can be captured alone.
"""
import argparse

from . import Context, default_opts, seeded_subset


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--loops", type=int, default=4)
    ap.add_argument("--graphs", type=int, default=8)
    ap.add_argument("--samples", type=int, default=1 << 17)
    ap.add_argument("--no-dd", action="store_true")
    a = ap.parse_args()
    o = default_opts()
    if a.no_dd:
        o.dd_ratio = 0.0
    c = Context(0, o)
    total = {1: 1, 2: 4, 3: 28, 4: 269, 5: 3213}[a.loops]
    ids = seeded_subset(total, min(a.graphs, total), 0)
    n = c.load_graph_subset(a.loops, ids)
    c.integrate([0], a.samples, 1)
    c.integrate_batched(list(range(n)), [a.samples // 2] * n, seed=1)
    print("ok", n)


if __name__ == "__main__":
    main()
