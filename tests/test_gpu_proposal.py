"""Learned proposal on the GPU: training kernels against the CPU oracle
(gradients), normalisation of the learned mixture, unbiasedness, and the
variance it gains over the plain density."""
import math

import numpy as np
import pytest

import paper_1909_08015_b300 as ae
from oracle import proposal as pr
from oracle.graphs import enumerate_graphs
from oracle.sampler import Density
from tests import proposal_inputs as pin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = ae.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("n,gi", [(2, 1), (3, 5)])
def test_gradient_matches_oracle(ctx, n, gi):
    g = enumerate_graphs(n)[gi]
    d = Density(g)
    M = d.M
    deg = d.deg[0].copy()
    wplain = np.ones(1 << M)
    wplain[1:-1] = d.phi[0][1:-1] / d.deg[0][1:-1]
    p = pin.params(7)
    order, lt, w = pin.records(7, 600, M)
    loss, grad, lp2, degt = ctx.proposal_eval(M, p, deg, wplain, order, lt, w)
    rl, rg, rlogp, rdegt = pr.loss_and_grad(p, deg, wplain, order, lt, w, M)
    # BF16 activations on the device against float64 activations in the
    # oracle: agreement to about a per cent.
    assert abs(loss - rl) <= 5e-3 * abs(rl)
    cos = float(np.dot(grad, rg) / (np.linalg.norm(grad) * np.linalg.norm(rg)))
    assert cos > 0.998, cos
    assert np.linalg.norm(grad - rg) <= 6e-2 * np.linalg.norm(rg)
    mask = np.isfinite(rlogp)
    assert np.max(np.abs(lp2[mask] - rlogp[mask] / math.log(2))) < 0.05
    assert np.max(np.abs(degt[1:-1] / rdegt[1:-1] - 1)) < 0.02


def test_learned_mixture_normalised_and_unbiased(ctx):
    """E_q[1/q] = 1/(M-1)! for the trained mixture; the learned estimate
    agrees with the plain one; report the variance ratio."""
    ctx.load_graphs(3)
    gid = 3
    rep = ctx.train_proposal(gid, 1 << 18, seed=1, steps=80, lr=3e-3, beta=0.1)
    assert rep["loss_final"] < rep["loss_initial"]
    d = ctx.eval_samples(gid, 0, 1 << 20, seed=2)
    wq = np.exp2(-d["log2g"]) * math.factorial(7)
    assert abs(wq.mean() - 1) < 4 * wq.std() / math.sqrt(len(wq))
    N = 1 << 22
    _, _, pl = ctx.integrate([gid], N, seed=3)
    ctx.set_proposal(gid, 0)
    _, _, pp = ctx.integrate([gid], N, seed=4)
    a, b = pl[0], pp[0]
    assert abs(a["mean"] - b["mean"]) < 4 * math.hypot(a["sigma1"], b["sigma1"])


def test_cost_aware_training_normalised_and_unbiased(ctx):
    """Cost-aware weights (|y| / sqrt(1 + R) where double-double is needed):
    the trained mixture is still normalised and its estimate agrees with the
    plain density's; the ratio returns to 0 afterwards."""
    ctx.load_graphs(3)
    gid = 12
    ctx.set_train_cost_ratio(8.0)
    try:
        ctx.train_proposal(gid, 1 << 18, seed=1, steps=80, lr=3e-3, beta=0.1)
    finally:
        ctx.set_train_cost_ratio(0.0)
    d = ctx.eval_samples(gid, 0, 1 << 20, seed=2)
    wq = np.exp2(-d["log2g"]) * math.factorial(7)
    assert abs(wq.mean() - 1) < 4 * wq.std() / math.sqrt(len(wq))
    N = 1 << 22
    _, _, pl = ctx.integrate([gid], N, seed=3)
    ctx.set_proposal(gid, 0)
    _, _, pp = ctx.integrate([gid], N, seed=4)
    a, b = pl[0], pp[0]
    assert abs(a["mean"] - b["mean"]) < 4 * math.hypot(a["sigma1"], b["sigma1"])


def test_fast_exp2_log2_against_device_library(ctx):
    """The learned sampler's fused-multiply-add exp2/log2 against the device
    library's exp2/log2 (itself within a couple of ulp of the exact value):
    within 4 ulp of it, exp2 on [-1020, 1] (0 below -1074), log2 on
    (1e-300, 1e3); exact at powers of 2."""
    rng = np.random.default_rng(5)
    x = np.concatenate([rng.uniform(-1070, 0, 100000), rng.uniform(-1, 1, 50000), [0.0, -1.0, -3.0, -2000.0]])
    y = np.concatenate([np.exp(rng.uniform(-690, 6.9, 100000)), 1 + rng.uniform(-1e-6, 1e-6, 50000),
                        [1.0, 2.0, 0.5, 0.25]])
    out = ctx.fast_elem(x, y)
    ok = x > -1020
    e2 = np.abs(out[ok, 0] - out[ok, 1]) / np.spacing(np.abs(out[ok, 1]))
    assert e2.max() <= 4, e2.max()
    assert out[-1, 0] == 0.0 and list(out[-4:-1, 0]) == [1.0, 0.5, 0.125]
    err = np.abs(out[:, 2] - out[:, 3]) / np.spacing(np.abs(out[:, 3]))
    assert err.max() <= 4, err.max()
    assert list(out[-4:, 2]) == [0.0, 1.0, -1.0, -2.0]
