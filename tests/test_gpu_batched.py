"""Batched persistent launch and inter-graph allocation on the GPU."""
import math

import numpy as np
import pytest

import paper_1909_08015_b300 as ae

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ae.Context(0)
    yield c
    c.close()


def test_batched_matches_per_graph(ctx):
    """Same samples (indices 0..n-1 per graph) through the persistent
    work-queue launch and through one launch per graph."""
    ctx.load_graphs(3)
    ids = list(range(28))
    ns = [200000 + 3001 * i for i in ids]          # uneven counts, ragged chunks
    vb, sb, pb = ctx.integrate_batched(ids, ns, seed=8)
    assert sum(p["seconds"] for p in pb) > 0 and sum(p["kernel_seconds"] for p in pb) > 0
    for i in (0, 5, 13, 22, 27):
        _, _, pg = ctx.integrate([i], ns[i], seed=8)
        assert pb[i]["n"] == ns[i]
        assert pb[i]["n_dd"] == pg[0]["n_dd"]
        assert abs(pb[i]["sum_y"] - pg[0]["sum_y"]) <= 1e-9 * abs(pg[0]["sum_y"])
        assert abs(pb[i]["sum_y2"] - pg[0]["sum_y2"]) <= 1e-9 * abs(pg[0]["sum_y2"])


def test_allocation_sums_and_orders(ctx):
    ctx.load_graphs(3)
    ids = list(range(28))
    n, sig = ctx.allocate(ids, 100000, 10 ** 7, seed=2, mode=0)
    assert int(n.sum()) == 10 ** 7
    assert np.all(n >= 1024)
    # the graph with the largest pilot sigma gets more than the smallest
    assert n[int(np.argmax(sig))] > n[int(np.argmin(sig))]
    n1, _ = ctx.allocate(ids, 100000, 10 ** 7, seed=2, mode=1)
    assert int(n1.sum()) == 10 ** 7


def test_four_loop_batched_runs(ctx):
    """All 269 four-loop graphs in one persistent launch (tapes of 21k-95k
    instructions); spot-check three graphs against per-graph launches."""
    N = ctx.load_graphs(4)
    assert N == 269
    ids = list(range(N))
    ns = [1 << 14] * N
    v, s, pb = ctx.integrate_batched(ids, ns, seed=1)
    assert all(p["n"] == 1 << 14 for p in pb)
    assert math.isfinite(v) and math.isfinite(s)
    for i in (0, 134, 268):
        _, _, pg = ctx.integrate([i], 1 << 14, seed=1)
        assert abs(pb[i]["sum_y"] - pg[0]["sum_y"]) <= 1e-9 * abs(pg[0]["sum_y"]) + 1e-300


def test_resume_by_counter_range(ctx):
    """Two consecutive counter ranges add up to the whole range (resume and
    sharding by range draw exactly the samples of an uninterrupted run)."""
    ctx.load_graphs(2)
    whole = ctx.integrate_range(3, 0, 400000, seed=4)
    a = ctx.integrate_range(3, 0, 150000, seed=4)
    b = ctx.integrate_range(3, 150000, 250000, seed=4)
    assert a["n"] + b["n"] == whole["n"]
    assert abs(a["sum_y"] + b["sum_y"] - whole["sum_y"]) <= 1e-12 * abs(whole["sum_y"]) + 1e-12
    assert abs(a["sum_y2"] + b["sum_y2"] - whole["sum_y2"]) <= 1e-12 * whole["sum_y2"]
    _, _, per = ctx.integrate([3], 400000, seed=4)
    assert abs(per[0]["sum_y"] - whole["sum_y"]) <= 1e-9 * abs(whole["sum_y"])


def test_adaptive_controller(ctx):
    """The paper's controller on the 2-loop set: closed form within 3 sigma,
    deterministic, each graph's samples exactly those of integrate_range over
    [0, N_j), and the graph with the largest C_j / sqrt(t_j) sampled most."""
    import math
    ctx.load_graphs(2)
    A4 = -0.328478965579193 - (119.0 / 36.0 - math.pi ** 2 / 3.0)
    v, s, per = ctx.integrate_adaptive([0, 1, 2, 3], 8192, 12, 96, p_floor=0.1, seed=21)
    assert abs(v - A4) < 3 * s, (v, s)
    total = sum(p["n"] for p in per)
    assert total == 8192 * (4 + 11 * 96)
    v2, s2, per2 = ctx.integrate_adaptive([0, 1, 2, 3], 8192, 12, 96, p_floor=0.1, seed=21)
    assert v2 == v and s2 == s
    for gi in (0, 3):
        r = ctx.integrate_range(gi, 0, per[gi]["n"], seed=21)
        assert abs(r["sum_y"] - per[gi]["sum_y"]) <= 1e-10 * abs(r["sum_y"])
    # C_j = sigma_up_j sqrt(N_j), t_j = tape flops + 150 M (Sec. IV.C)
    info = [ctx.graph_info(i) for i in range(4)]
    w = [per[i]["sigma_up"] * math.sqrt(per[i]["n"]) / math.sqrt(info[i]["flops"] + 150 * info[i]["M"])
         for i in range(4)]
    assert int(np.argmax([p["n"] for p in per])) == int(np.argmax(w))
    assert all(p["sigma_up"] >= p["sigma"] for p in per)


def test_allocation_follows_formula(ctx):
    """n_j = floor + largest-remainder share of the rest, shares proportional
    to C_j / sqrt(t_j) = sigma_j sqrt(N_pilot) / sqrt(t_j) (mode 0, Sec. IV.C)
    or to sigma_j^2 (mode 1), from the returned pilot sigmas; floor =
    min(1024, n_total / n_ids); t_j = tape flops + 150 M."""
    ctx.load_graphs(3)
    ids = list(range(28))
    info = [ctx.graph_info(i) for i in ids]
    t = np.array([m["flops"] + 150 * m["M"] for m in info])
    n_pilot, n_total = 100000, 10 ** 7 + 13
    for mode in (0, 1):
        n, sig = ctx.allocate(ids, n_pilot, n_total, seed=2, mode=mode)
        w = sig * math.sqrt(n_pilot) / np.sqrt(t) if mode == 0 else sig ** 2
        floor = min(1024, n_total // len(ids))
        want = floor + (n_total - floor * len(ids)) * w / w.sum()
        assert int(n.sum()) == n_total
        assert np.all(np.abs(n - want) < 1.0 + 1e-9 * want), np.max(np.abs(n - want))


def test_run_steps_checkpoint_resume(ctx, tmp_path):
    """A run of three batched blocks equals a run of two blocks, checkpointed,
    resumed in a new context and continued by one block; and each graph's
    sums equal one launch over [0, 3n) (counter continuity)."""
    n = 100000
    ctx.load_graphs(2)
    ids = [0, 1, 2, 3]
    ctx.run_reset(11)
    for _ in range(3):
        ctx.run_step(ids, [n] * 4)
    v, s, su, whole = ctx.run_estimate()
    ctx.run_reset(11)
    for _ in range(2):
        ctx.run_step(ids, [n] * 4)
    p = str(tmp_path / "run.ckpt")
    ctx.checkpoint(p)
    c2 = ae.Context(0)
    try:
        c2.load_graphs(2)
        c2.resume(p)
        c2.run_step(ids, [n] * 4)
        v2, s2, su2, res = c2.run_estimate()
        st, _ = c2.run_get()
        assert [g.next for g in st] == [3 * n] * 4
    finally:
        c2.close()
    assert abs(v2 - v) <= 1e-10 * abs(v) and abs(s2 - s) <= 1e-9 * s
    for gi in ids:
        assert res[gi]["n"] == 3 * n and res[gi]["n_dd"] == whole[gi]["n_dd"]
        r = ctx.integrate_range(gi, 0, 3 * n, seed=11)
        assert abs(r["sum_y"] - res[gi]["sum_y"]) <= 1e-10 * abs(r["sum_y"])
        assert abs(r["sum_y2"] - res[gi]["sum_y2"]) <= 1e-10 * r["sum_y2"]
    assert su >= s


def test_bounded_wait_runs_out(ctx):
    """The bounded wait for a tape segment (about 2 s in normal use) made to
    run out through the test hook (first copy left out, wait limit 2^20
    cycles): the call returns AE_ERR_TIMEOUT and the context stays usable."""
    ctx.load_graphs(2)
    before = ctx.integrate([2], 50000, seed=3)
    with pytest.raises(ae.AeError, match="AE_ERR_TIMEOUT"):
        ctx.test_stage_timeout(2, 1 << 20)
    after = ctx.integrate([2], 50000, seed=3)
    assert after[0] == before[0] and after[1] == before[1]


def test_run_step_argument_errors(ctx):
    """A graph listed twice in one block, an empty block, an unknown graph and
    a run step on a context without graphs are refused with AE_ERR_* codes."""
    ctx.load_graphs(2)
    ctx.run_reset(0)
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        ctx.run_step([1, 1], [100, 100])
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        ctx.run_step([0, 1], [0, 0])
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        ctx.run_step([7], [100])
    fresh = ae.Context(0)
    try:
        with pytest.raises(ae.AeError, match="AE_ERR_STATE"):
            fresh.run_step([0], [100])
    finally:
        fresh.close()
    st, _ = ctx.run_get()
    assert all(g.next == 0 and g.n == 0 for g in st)   # nothing was added
