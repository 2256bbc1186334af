"""The integration controller's sampling probabilities (Sec. IV.C, "Monte
Carlo integration: details"), on the host: they minimise sigma^2 * time, and
the floor and degenerate cases behave as stated."""
import numpy as np
import pytest

import paper_1909_08015_b300 as ae


def objective(p, C, t):
    """(sum C_j^2 / p_j) (sum p_j t_j): N sigma^2 times the time per sample."""
    return np.sum(C * C / p) * np.sum(p * t)


def test_probabilities_minimise_variance_times_time():
    rng = np.random.default_rng(3)
    for trial in range(20):
        n = rng.integers(2, 12)
        sigma = rng.lognormal(0, 1.5, n)
        N = rng.integers(1, 10 ** 6, n).astype(np.uint64)
        t = rng.lognormal(0, 1.0, n)
        p = ae.schedule_probabilities(sigma, N, t, 0.0)
        assert abs(p.sum() - 1) < 1e-12 and np.all(p > 0)
        C = sigma * np.sqrt(N.astype(float))
        best = objective(p, C, t)
        for _ in range(200):
            q = rng.dirichlet(np.ones(n))
            assert best <= objective(q, C, t) * (1 + 1e-12)
        # small perturbations of the optimum do not improve it either
        for _ in range(50):
            q = p * np.exp(rng.normal(0, 1e-3, n))
            q /= q.sum()
            assert best <= objective(q, C, t) * (1 + 1e-12)


def test_probability_floor_and_degenerate_inputs():
    p = ae.schedule_probabilities([1.0, 2.0, 0.0, 4.0], [100, 100, 100, 400], [1.0, 4.0, 1.0, 1.0], 0.1)
    w = np.array([10.0, 10.0, 0.025 * 100, 80.0])
    assert np.allclose(p, w / w.sum(), rtol=1e-12)
    assert np.allclose(ae.schedule_probabilities([0.0, 0.0], [5, 5], [1.0, 1.0], 0.0), [0.5, 0.5])
    assert np.allclose(ae.schedule_probabilities([np.nan, 1.0], [5, 5], [1.0, 1.0], 0.0), [0.0, 1.0])
    with pytest.raises(ae.AeError):
        ae.schedule_probabilities([1.0], [1], [1.0], 1.5)


def test_accept_widths_of_eq_interval_accept():
    """width_j = (1/4) sigma_j sqrt(sum sigma^2) / sum sigma (Sec. IV.A):
    the widths add up to a quarter of the set's sigma_down, are proportional
    to sigma_j, and graphs without a positive finite sigma get 0."""
    sig = np.array([3.0, 4.0, 0.0, float("nan"), 12.0])
    w = ae.accept_widths(sig)
    good = np.array([3.0, 4.0, 12.0])
    assert w[2] == 0 and w[3] == 0
    assert np.isclose(w[[0, 1, 4]].sum(), 0.25 * 13.0)           # sqrt(9 + 16 + 144) = 13
    assert np.allclose(w[[0, 1, 4]], 0.25 * good * 13.0 / good.sum())
    assert np.all(ae.accept_widths(np.zeros(3)) == 0)
