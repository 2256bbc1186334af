"""A five-loop graph against the CPU oracle.  The oracle's coefficient
tables of canonical graph 878 (a graph whose only UV-divergent subgraph is
itself, so its subtracted integrand is one forest term) are stored
(tests/golden/oracle_tables_5loop_878.json.gz, written by
make_oracle_tables.py from oracle/ alone; their set-up took 4.3 hours on one
core).  Samples [0, 2048) and [2^32 - 64, 2^32 + 64), seed 0, per sample,
with the bars of the three- and four-loop scale tests (tests/oracle_pool.py):
z and log2 g bit for bit; the FP64 and double-double values within their
certified bounds plus the oracle's two-precision uncertainty, the oracle's
exact rational value as referee outside it; the least certain sample of
each chunk against the exact value; the integration kernel over [0, 2048)
against the dumps' counts and sum."""
import math
import multiprocessing as mp
import os

import numpy as np
import pytest

import paper_1909_08015_b300 as ae
from oracle.estimate import weight_many
from tests.oracle_pool import exact_values, graph_values

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CID = 878
PATH = os.path.join(HERE, "golden", "oracle_tables_5loop_%d.json.gz" % CID)
RANGES = [(0, 2048), ((1 << 32) - 64, 128)]
CHUNK = 128
MAX_REFEREED = 64
TOL = 1e-10


def _rejected(y, E, lg):
    with np.errstate(invalid="ignore", over="ignore"):
        Ey = weight_many(E, lg)
        return ~np.isfinite(y) | ~np.isfinite(Ey) | (Ey > TOL * np.abs(y))


def _within_bounds(ex, I64, E64, f64, Idd, Edd):
    slack = 2.0 ** -52 * np.abs(ex)
    assert np.all(np.abs(Idd - ex) <= Edd + slack)
    assert np.all((np.abs(I64 - ex) <= E64 + slack)[f64])


def test_five_loop_graph_against_stored_table_oracle():
    jobs = [(5, CID, lo, min(CHUNK, first + count - lo), 0, 1, PATH)
            for first, count in RANGES for lo in range(first, first + count, CHUNK)]
    pool = mp.get_context("spawn").Pool(max(1, min(len(jobs), os.cpu_count() or 1)))
    try:
        res = pool.map(graph_values, jobs, chunksize=1)
        opts = ae.default_opts()
        opts.grid_ctas = 3
        ctx = ae.Context(0, opts)
        plain = ae.Context(0)
        try:
            assert ctx.load_graph_subset(5, [CID]) == 1
            plain.load_graph_subset(5, [CID])
            refereed = []
            n_miss = 0
            for first, count in RANGES:
                parts = sorted((r for r in res if first <= r["first"] < first + count), key=lambda r: r["first"])
                I = np.concatenate([r["I"] for r in parts])
                scale = np.concatenate([r["scale"] for r in parts])
                z = np.concatenate([r["z"] for r in parts])
                lg = np.concatenate([r["log2g"] for r in parts])
                assert len(I) == count and np.all(np.isfinite(I)) and np.all(np.isfinite(scale))
                d = ctx.eval_samples(0, first, count, seed=0)
                assert np.array_equal(d["z"], z)
                assert np.array_equal(d["log2g"], lg)
                fin = np.isfinite(d["I"]) & np.isfinite(d["E"])
                dd = ctx.eval_samples_dd(0, first, count, seed=0)
                assert np.all(np.isfinite(dd["I"]) & np.isfinite(dd["E"]))
                with np.errstate(invalid="ignore"):
                    out64 = fin & ~(np.abs(d["I"] - I) <= d["E"] + scale)
                outdd = ~(np.abs(dd["I"] - I) <= dd["E"] + scale)
                miss = np.nonzero(out64 | outdd)[0]
                n_miss += len(miss)
                if len(miss):
                    refereed.append((d["I"][miss], d["E"][miss], fin[miss], dd["I"][miss], dd["E"][miss],
                                     pool.apply_async(exact_values, ((5, CID, z[miss], PATH),))))
                for r in parts:
                    k = r["exact_idx"] + (r["first"] - first)
                    _within_bounds(r["exact_I"], d["I"][k], d["E"][k], fin[k], dd["I"][k], dd["E"][k])
                if first == 0:
                    flag = _rejected(d["y"], d["E"], d["log2g"])
                    zero = flag & _rejected(dd["y"], dd["E"], d["log2g"])
                    y = np.where(flag, np.where(zero, 0.0, dd["y"]), d["y"])
                    per = plain.integrate_range(0, 0, count, seed=0)
                    assert per["n"] == count
                    assert per["n_dd"] == int(flag.sum())
                    assert per["n_nonfinite"] == int(zero.sum())
                    assert abs(per["sum_y"] - math.fsum(y)) <= 1e-12 * math.fsum(np.abs(y))
            assert n_miss <= MAX_REFEREED, n_miss
            for I64, E64, f64, Idd, Edd, job in refereed:
                _within_bounds(job.get(timeout=1500), I64, E64, f64, Idd, Edd)
        finally:
            ctx.close()
            plain.close()
    finally:
        pool.close()
        pool.join()
