"""GPU parity: the CUDA path through the C ABI against the CPU oracle on the
same Philox samples, and the integrated values against the closed forms."""
import math

import numpy as np
import pytest

import paper_1909_08015_b300 as ae
from oracle.estimate import GraphOracle, summarize
from oracle.graphs import enumerate_graphs
from oracle.philox import philox4x32_10, philox_np
from tests.acceptance import bound_holds, rejected

pytestmark = pytest.mark.gpu

# 2-loop no-lepton-loop part: A_1^(4) (Sec. I) minus the vacuum-polarisation
# graph 119/36 - pi^2/3.
A4_NO_LEPTON_LOOPS = -0.328478965579193 - (119.0 / 36.0 - math.pi ** 2 / 3.0)

# Per-sample tolerance of the FP64 integrand against the oracle's exactly
# rounded value: relative 1e-10 plus a term proportional to the forest-term
# magnitude K (cancellation between terms costs digits; 2^-40 K allows for
# the rounding of sums of up to ~10^4 monomials each of size <= K).
REL = 1e-10


@pytest.fixture(scope="module")
def ctx():
    c = ae.Context(0)
    yield c
    c.close()


def test_philox_bit_exact(ctx):
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2 ** 32, size=(4096, 4), dtype=np.uint64)
    key = rng.integers(0, 2 ** 32, size=(4096, 2), dtype=np.uint64)
    got = ctx.philox(ctr.astype(np.uint32), key.astype(np.uint32))
    for i in range(0, 4096, 97):
        assert list(got[i]) == list(philox4x32_10(ctr[i], key[i]))
    w = philox_np(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], 0, 0)
    z0 = ctx.philox(ctr.astype(np.uint32), np.zeros((4096, 2), np.uint32))
    assert np.array_equal(z0[:, 0], w[0].astype(np.uint32))


@pytest.mark.parametrize("n,ids,count", [(1, [0], 512), (2, [0, 1, 2, 3], 256), (3, [0, 13, 27], 48)])
def test_samples_and_integrand(ctx, n, ids, count):
    """z and log2 g bit for bit; the certified bound E of the FP64 value
    (and of the double-double one) holds on every sample; samples the
    acceptance test keeps are within 1e-10 of the oracle."""
    ctx.load_graphs(n)
    gs = enumerate_graphs(n)
    for gi in ids:
        ref = GraphOracle(gs[gi], gi).samples(0, count, seed=0)
        d = ctx.eval_samples(gi, 0, count, seed=0)
        assert np.array_equal(d["z"], ref["z"])
        assert np.array_equal(d["log2g"], ref["log2g"])
        assert bound_holds(d["I"], d["E"], ref["I"])
        # K = sum of |forest terms| carries at most the rounding of I's terms
        fin = np.isfinite(d["K"])
        assert np.all(np.abs(d["K"] - ref["K"])[fin] <= d["E"][fin] + 1e-12 * ref["K"][fin])
        keep = ~rejected(d["y"], d["E"], d["log2g"])
        err = np.abs(d["I"] - ref["I"])
        assert np.all(err[keep] <= REL * np.abs(ref["I"][keep]))
        dd = ctx.eval_samples_dd(gi, 0, count, seed=0)
        assert bound_holds(dd["I"], dd["E"], ref["I"])
        ok = ~rejected(dd["y"], dd["E"], d["log2g"])
        assert np.all(np.abs(dd["I"] - ref["I"])[ok] <= REL * np.abs(ref["I"][ok]))


def test_summed_estimate_matches_oracle(ctx):
    """Sum of y over the same 2048 samples: GPU (FP64 + double-double
    re-evaluation) against the oracle within 1e-9 relative."""
    ctx.load_graphs(2)
    gs = enumerate_graphs(2)
    N = 2048
    _, _, per = ctx.integrate([0, 1, 2, 3], N, seed=5)
    for gi in range(4):
        ref = summarize(GraphOracle(gs[gi], gi).samples(0, N, seed=5)["y"], gs[gi].mult)
        assert per[gi]["n"] == N and per[gi]["n_nonfinite"] == 0
        assert abs(per[gi]["sum_y"] - ref["sum_y"]) <= 1e-9 * abs(ref["sum_y"])
        assert abs(per[gi]["sum_y2"] - ref["sum_y2"]) <= 1e-9 * abs(ref["sum_y2"])


@pytest.mark.parametrize("N", [1, 31, 33, 257, 1000])
def test_ragged_sample_counts_match_oracle(ctx, N):
    """Counts that leave a partial warp, round or CTA (and a single sample):
    sums over samples 0..N-1 against the oracle's, per-graph and batched
    (with a zero-count entry beside them)."""
    ctx.load_graphs(2)
    gs = enumerate_graphs(2)
    for gi in (1, 3):
        ref = summarize(GraphOracle(gs[gi], gi).samples(0, N, seed=6)["y"], gs[gi].mult)
        _, _, per = ctx.integrate([gi], N, seed=6)
        assert per[0]["n"] == N
        assert abs(per[0]["sum_y"] - ref["sum_y"]) <= 1e-9 * abs(ref["sum_y"]) + 1e-300
        v, s, pb = ctx.integrate_batched([gi, 0], [N, 0], seed=6)
        assert pb[0]["n"] == N and pb[1]["n"] == 0
        assert pb[1]["value"] == 0.0 and pb[1]["sigma"] == 0.0
        assert abs(pb[0]["sum_y"] - ref["sum_y"]) <= 1e-9 * abs(ref["sum_y"]) + 1e-300
        assert abs(v - pb[0]["value"]) <= 1e-15 * abs(v) + 1e-300


def test_one_loop_value(ctx):
    ctx.load_graphs(1)
    v, s, per = ctx.integrate([0], 10 ** 7, seed=0)
    assert abs(v - 0.5) < 3 * s
    assert s < 1e-3


def test_two_loop_value(ctx):
    """Sum over the four 2-loop graphs (times multiplicity) against the
    closed form, within 3 sigma."""
    ctx.load_graphs(2)
    v, s, per = ctx.integrate([0, 1, 2, 3], 10 ** 7, seed=0)
    assert abs(v - A4_NO_LEPTON_LOOPS) < 3 * s, (v, s)
    assert s < 0.01


def test_deterministic(ctx):
    ctx.load_graphs(2)
    a = ctx.integrate([1, 3], 200000, seed=9)
    b = ctx.integrate([1, 3], 200000, seed=9)
    assert a[0] == b[0] and a[1] == b[1]
    assert [p["sum_y"] for p in a[2]] == [p["sum_y"] for p in b[2]]


def test_errors(ctx):
    ctx.load_graphs(1)
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        ctx.integrate([3], 1000)
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        ctx.integrate([0], 0)
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        ctx.integrate_batched([0], [0])
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        ctx.integrate_batched([1], [100])
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        ctx.integrate_adaptive([0], 0, 2, 4)
