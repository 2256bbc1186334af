"""The entry point that allocates no device memory (ae_integrate_noalloc).

Some callers cannot allocate device memory once they are running (their
device memory is reserved up front by another allocator, or their loop may
not pay for cudaMalloc's device synchronisation).  For them the library keeps
the scratch of one integration in a fixed device array.  This checks, through
the C ABI, that two calls in a row on the same array reproduce what the
allocating entry point ae_integrate returns for the same inputs.
"""
import pytest

import paper_1909_08015_b300 as ae

pytestmark = pytest.mark.gpu

REL = 1e-9   # summed-estimate tolerance used by the other parity tests


@pytest.fixture(scope="module")
def ctx():
    c = ae.Context(0)
    c.load_graphs(2)
    yield c
    c.close()


def _same(a, b):
    assert a["n"] == b["n"]
    assert a["n_dd"] == b["n_dd"]
    assert a["n_nonfinite"] == b["n_nonfinite"]
    for k in ("sum_y", "sum_y2"):
        assert abs(a[k] - b[k]) <= REL * abs(b[k]), (k, a[k], b[k])


def test_two_calls_match_allocating_entry_point(ctx):
    # calls in a row: each reuses the array the previous one filled; the
    # third is smaller than the second, so stale flags and values beyond its
    # own samples are still in the array and must be ignored
    for gid, n, seed in ((1, 300000, 3), (3, 524288, 4), (1, 100003, 5)):
        got = ctx.integrate_noalloc(gid, n, seed)
        _, _, per = ctx.integrate([gid], n, seed)
        _same(got, per[0])
        assert got["n_dd"] > 0          # the double-double pass was exercised


def test_rejects_sizes_beyond_the_limit(ctx):
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        ctx.integrate_noalloc(0, 524289, 0)
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        ctx.integrate_noalloc(0, 0, 0)
