"""Writes tests/golden/oracle_sums_3loop.txt: the CPU oracle's (and nothing
else's) sums of y over fixed sample ranges of every 3-loop graph, and its
per-sample values around sample index 2^32, for the GPU parity tests of the
staged integration kernels (many rounds per CTA, ranges that straddle the
Philox counter's high word).

    python tests/golden/make_oracle_sums.py

Seed 5.  Ranges per graph: A = samples 0 .. 1499, B = samples
2^32 - 700 .. 2^32 + 647.  Lines
    S graph first count sum_y sum_y2        (math.fsum over the oracle's y)
    P graph index log2g I K                 (B's samples 2^32 - 16 .. 2^32 + 15)
all floats as hexadecimal literals (exact round trip).
"""
import math
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

SEED = 5
RANGES = [(0, 1500), (2 ** 32 - 700, 1348)]
AROUND = (2 ** 32 - 16, 32)


def one(args):
    gi, first, count = args
    from oracle.estimate import GraphOracle
    from oracle.graphs import enumerate_graphs
    o = GraphOracle(enumerate_graphs(3)[gi], gi)
    r = o.samples(first, count, SEED)
    y = r["y"]
    lines = ["S %d %d %d %s %s" % (gi, first, count, math.fsum(y).hex(), math.fsum(y * y).hex())]
    if first == RANGES[1][0]:
        lo = AROUND[0] - first
        for k in range(lo, lo + AROUND[1]):
            lines.append("P %d %d %s %s %s" % (gi, first + k, float(r["log2g"][k]).hex(), float(r["I"][k]).hex(),
                                               float(r["K"][k]).hex()))
    return lines


def main():
    jobs = []
    for gi in range(28):
        for first, count in RANGES:
            jobs.append((gi, first, count))
    with mp.get_context("spawn").Pool(os.cpu_count() or 1) as pool:
        res = pool.map(one, jobs, chunksize=1)
    path = os.path.join(HERE, "oracle_sums_3loop.txt")
    with open(path, "w") as f:
        f.write("# CPU oracle sums of y, 3-loop graphs 0..27, seed %d, ranges %s\n" % (SEED, RANGES))
        f.write("# written by tests/golden/make_oracle_sums.py (calls oracle/ only)\n")
        f.write("# S graph first count sum_y sum_y2 | P graph index log2g I K (hex floats)\n")
        for lines in res:
            f.write("\n".join(lines) + "\n")
    print(path)


if __name__ == "__main__":
    main()
