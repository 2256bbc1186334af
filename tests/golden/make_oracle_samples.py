"""Writes tests/golden/oracle_samples_<n>loop.txt: per-sample values of the
CPU oracle (and nothing else) for a few graphs whose oracle set-up takes
minutes, so that the GPU parity tests can compare against them without
rebuilding the oracle's coefficient tables on every run.

    python tests/golden/make_oracle_samples.py 3 0 1 2 ... 27 --count 24
    python tests/golden/make_oracle_samples.py 4 0 5 30 60 100 134 200 268 --count 12

Each line: graph id, sample index, then z (M values), log2 g, I, K, all as
hexadecimal floating-point literals (exact round trip).  Seed 0.

With --compact the lines hold graph id, sample index, I and K only (the
tests recompute z and log2 g with the oracle's sampler, which is fast), for
samples --first .. --first+count-1, written to oracle_values_<n>loop.txt:

    python tests/golden/make_oracle_samples.py 3 0 1 ... 27 --first 24 --count 256 --compact
"""
import argparse
import multiprocessing as mp
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))


def one(args):
    n, gi, first, count, seed, compact = args
    from oracle.estimate import GraphOracle
    from oracle.graphs import enumerate_graphs
    o = GraphOracle(enumerate_graphs(n)[gi], gi)
    r = o.samples(first, count, seed)
    lines = []
    for k in range(count):
        vals = ([] if compact else list(r["z"][k]) + [r["log2g"][k]]) + [r["I"][k], r["K"][k]]
        lines.append("%d %d %s" % (gi, first + k, " ".join(float(v).hex() for v in vals)))
    return lines


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("loops", type=int)
    ap.add_argument("ids", type=int, nargs="+")
    ap.add_argument("--count", type=int, default=12)
    ap.add_argument("--first", type=int, default=0)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--compact", action="store_true")
    a = ap.parse_args()
    with mp.get_context("spawn").Pool(min(len(a.ids), os.cpu_count() or 1)) as pool:
        res = pool.map(one, [(a.loops, gi, a.first, a.count, a.seed, a.compact) for gi in a.ids], chunksize=1)
    name = "oracle_values_%dloop.txt" if a.compact else "oracle_samples_%dloop.txt"
    path = os.path.join(HERE, name % a.loops)
    with open(path, "w") as f:
        f.write("# CPU oracle per-sample values, %d-loop graphs %s, seed %d, samples %d..%d\n"
                % (a.loops, a.ids, a.seed, a.first, a.first + a.count - 1))
        f.write("# written by tests/golden/make_oracle_samples.py (calls oracle/ only)\n")
        f.write("# columns: graph sample %sI K (hex floats)\n" % ("" if a.compact else "z[0..M-1] log2g "))
        for lines in res:
            f.write("\n".join(lines) + "\n")
    print(path)


if __name__ == "__main__":
    main()
