"""MRG32k3a, the generator of Calc 1 (Sec. V), in the oracle: pinned by the
full period of both components (a property of the published parameters:
A^(m^3 - 1) = I), by jump-ahead against step-by-step recursion, and by the
uniformity of its doubles; and the combination of two calculations."""
import numpy as np
import pytest

import paper_1909_08015_b300 as ae
from oracle import mrg32k3a as mrg


def test_components_have_full_period():
    ident = ((1, 0, 0), (0, 1, 0), (0, 0, 1))
    assert mrg.matpow(mrg.A1, mrg.M1 ** 3 - 1, mrg.M1) == ident
    assert mrg.matpow(mrg.A2, mrg.M2 ** 3 - 1, mrg.M2) == ident
    # and not a shorter obvious one
    assert mrg.matpow(mrg.A1, mrg.M1 - 1, mrg.M1) != ident
    assert mrg.matpow(mrg.A2, mrg.M2 - 1, mrg.M2) != ident


def test_jump_ahead_equals_stepping():
    s1, s2 = mrg.SEED, mrg.SEED
    seq = []
    for _ in range(600):
        s1, s2, z = mrg.step(s1, s2)
        seq.append(z)
    for pos in (0, 1, 2, 63, 64, 200, 511):
        assert mrg.words(pos, 5) == seq[pos:pos + 5]
    assert all(0 <= z < mrg.M1 for z in seq)


def test_uniforms_layout_and_distribution():
    u = mrg.uniforms(np.arange(400, dtype=np.uint64), 3, 7, 4)
    assert u.shape == (400, 8)
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.02
    # sample i's words are outputs 64 i + 1 .. of the stream of (seed, graph)
    w = mrg.words((7 << 96) + (3 << 80) + 64 * 5, 2)
    assert u[5, 0] == ((w[0] >> 5) * 67108864.0 + (w[1] >> 6) + 0.5) * 2.0 ** -53


def test_combine_runs():
    v, s, tot, ts = ae.combine_runs([1.0, 2.0, 5.0], [0.1, 0.2, 0.0], [3.0, 2.5, 4.0], [0.1, 0.1, 1.0])
    assert np.allclose(v, [2.0, (2.0 / 0.04 + 2.5 / 0.01) / (1 / 0.04 + 1 / 0.01), 5.0])
    assert np.allclose(s, [np.sqrt(0.005), np.sqrt(1 / (1 / 0.04 + 1 / 0.01)), 0.0])
    assert abs(tot - v.sum()) < 1e-12 and abs(ts - np.sqrt((s ** 2).sum())) < 1e-12
    with pytest.raises(ae.AeError):
        ae.combine_runs([], [], [], [])
