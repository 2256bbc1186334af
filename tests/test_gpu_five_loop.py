"""Five-loop graphs (a seeded subset of the 3213): the oracle's coefficient
tables take hours per graph at this order (one graph is compared with the
oracle itself, from stored tables, in test_gpu_five_loop_oracle.py), so the
path is pinned here in parts:
sample points and densities bit for bit against the oracle's sampler; the
GPU integrand bit for bit against the host replay of the same compiled tape
(both evaluate the same IEEE operations in the same order); and the
integration kernel (tape staged through shared memory, double-double
re-evaluation) against per-sample values summed on the host."""
import math

import numpy as np
import pytest

import paper_1909_08015_b300 as ae
from oracle.estimate import weight
from oracle.graphs import enumerate_graphs
from oracle.philox import uniforms
from oracle.sampler import Density, sample
from tests.acceptance import rejected

pytestmark = pytest.mark.gpu

CANON = ae.seeded_subset(3213, 200, 0)[:2]


@pytest.fixture(scope="module")
def ctx5():
    c = ae.Context(0)
    n = c.load_graph_subset(5, CANON)
    assert n == len(CANON)
    yield c
    c.close()


def test_five_loop_samples_bit_exact(ctx5):
    gs = enumerate_graphs(5)
    count = 128
    for gi, cid in enumerate(CANON):
        d = ctx5.eval_samples(gi, 0, count, seed=0)
        dens = Density(gs[cid])
        u = uniforms(np.arange(count, dtype=np.uint64), cid, 0, dens.M)
        z, lg, _ = sample(dens, u)
        assert np.array_equal(d["z"], z)
        assert np.array_equal(d["log2g"], lg)
        I, K = ctx5.tape_replay(gi, d["z"])
        assert np.array_equal(d["I"], I, equal_nan=True)
        assert np.array_equal(d["K"], K, equal_nan=True)
        assert np.isfinite(I).mean() > 0.9


def test_five_loop_integration_sums(ctx5):
    """integrate (staged tape) = sum over the same samples of the per-sample
    values (FP64 where kept, double-double where re-evaluated), 1e-9."""
    N = 4096
    _, _, per = ctx5.integrate(list(range(len(CANON))), N, seed=3)
    for gi in range(len(CANON)):
        d = ctx5.eval_samples(gi, 0, N, seed=3)
        dd = ctx5.eval_samples_dd(gi, 0, N, seed=3)
        flagged = rejected(d["y"], d["E"], d["log2g"])
        bad_dd = rejected(dd["y"], dd["E"], d["log2g"])
        y = np.where(flagged, np.where(bad_dd, 0.0, dd["y"]), d["y"])
        assert per[gi]["n"] == N
        assert per[gi]["n_dd"] == int(flagged.sum())
        assert per[gi]["n_nonfinite"] == int((flagged & bad_dd).sum())
        sy = math.fsum(y)
        sy2 = math.fsum(y * y)
        assert abs(per[gi]["sum_y"] - sy) <= 1e-9 * abs(sy)
        assert abs(per[gi]["sum_y2"] - sy2) <= 1e-9 * abs(sy2)
