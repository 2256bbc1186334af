"""Host-side checks of libae (no GPU): the library loads and exports its
ABI, and its graph set, forests, sampling tables and compiled integrand
tapes agree with the independent CPU oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_1909_08015_b300 as ae
from oracle.forest import divergent_subgraphs, terms as forest_terms
from oracle.graphs import enumerate_graphs
from oracle.integrand import Integrand
from oracle.sampler import Density

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_abi_symbols_exported():
    header = open(os.path.join(ROOT, "include", "ae.h")).read()
    names = set(re.findall(r"^\s*(?:int|void|const char \*)\s*\*?\s*(ae\w+|aetest\w+)\s*\(", header, re.M))
    assert {"ae_create", "ae_load_graphs", "ae_integrate", "ae_eval_samples"} <= names
    L = ctypes.CDLL(ae.lib()._name)
    for n in names:
        assert hasattr(L, n), n


@pytest.fixture(scope="module")
def host():
    return ae.Context(-1)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_graph_list_matches_oracle(host, n):
    N = host.load_graphs(n)
    gs = enumerate_graphs(n)
    assert N == len(gs)
    for i, g in enumerate(gs):
        info = host.graph_info(i)
        assert info["word"] == g.word
        assert info["mult"] == g.mult
        assert info["klass"] == g.klass()
        assert info["M"] == 3 * n - 1


def _oracle_terms(g):
    out = []
    for sign, ops in forest_terms(g):
        code = {"A": 0, "U": 1, "L": 2, "L-U": 3}
        els = tuple(sorted((min(S.verts), max(S.verts), code[op]) for S, op in ops))
        out.append((sign, els))
    return sorted(out)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_forests_match_oracle(host, n):
    host.load_graphs(n)
    gs = enumerate_graphs(n)
    step = 1 if n < 4 else 9
    for i in range(0, len(gs), step):
        g = gs[i]
        subs = sorted((min(S.verts), max(S.verts), 0 if S.kind == "SE" else (2 if S.in_J else 1))
                      for S in divergent_subgraphs(g))
        assert sorted(host.subgraphs(i)) == subs
        got = sorted((s, tuple(sorted(els))) for s, els in host.terms(i))
        assert got == _oracle_terms(g)


@pytest.mark.parametrize("n", [1, 2, 3])
def test_density_tables_bit_exact(host, n):
    host.load_graphs(n)
    gs = enumerate_graphs(n)
    for i in range(0, len(gs), 3):
        deg, phi = host.density_tables(i)
        d = Density(gs[i])
        for k in range(3):
            assert np.array_equal(deg[k][1:-1], d.deg[k][1:-1])
            assert np.array_equal(phi[k][1:], d.phi[k][1:])


@pytest.mark.parametrize("n,ids", [(1, [0]), (2, [0, 1, 2, 3]), (3, [0, 9, 13, 27])])
def test_tape_matches_oracle_integrand(host, n, ids):
    """Compiled tape (symbolic graph polynomials, 4-D contraction identities)
    against the oracle (exact rational graph functions, explicit index sums)
    at random simplex points."""
    host.load_graphs(n)
    gs = enumerate_graphs(n)
    rng = np.random.default_rng(n)
    for gi in ids:
        I = Integrand(gs[gi])
        z = rng.dirichlet(np.ones(3 * n - 1), size=3)
        Ic, Kc = host.tape_replay(gi, z)
        ref = np.array([I.evaluate(p) for p in z])
        assert np.all(np.abs(Ic - ref[:, 0]) <= 1e-10 * np.abs(ref[:, 0]) + 1e-12 * ref[:, 1])
        assert np.all(np.abs(Kc - ref[:, 1]) <= 1e-10 * ref[:, 1])


def test_settings_validate_arguments(host):
    host.load_graphs(1)
    host.set_train_cost_ratio(8.0)
    host.set_train_cost_ratio(0.0)
    host.set_accept_floor(0, 0.5)
    host.set_accept_floor(0, 0.0)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
            host.set_train_cost_ratio(bad)
        with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
            host.set_accept_floor(0, bad)
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        host.set_accept_floor(3, 1.0)


def test_host_context_refuses_device_calls(host):
    host.load_graphs(1)
    with pytest.raises(ae.AeError, match="AE_ERR_NODEV"):
        host.integrate([0], 1000, 0)
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        host.graph_info(5)
    with pytest.raises(ae.AeError, match="AE_ERR_ARG"):
        host.load_graphs(7)


@pytest.mark.parametrize("n,ids,worst", [(2, [0, 1, 2, 3], 40), (3, [0, 12], 20)])
def test_error_bound_holds_at_worst_points(host, n, ids, worst):
    """The tape's certified rounding-error bound E (magnitude twins, gamma_D
    times the absolute-value evaluation) against the oracle's exact rational
    integrand, at the sampler's most ill-conditioned points (largest E/|I|
    out of 2048, which reach the sector corners where the forest terms
    cancel): |I_fp64 - I_exact| <= E everywhere.  And E is informative:
    at most 1e-10 |I| on the median point."""
    from oracle.estimate import GraphOracle
    host.load_graphs(n)
    gs = enumerate_graphs(n)
    for gi in ids:
        pts = GraphOracle(gs[gi], gi).points(0, 2048, seed=11)
        I, K, E = host.tape_replay(gi, pts["z"], bound=True)
        r = E / np.abs(I)
        assert np.median(r) < 1e-10
        It = Integrand(gs[gi])
        for k in np.argsort(-r)[:worst]:
            ex = It.evaluate(pts["z"][k])[0]
            assert abs(I[k] - ex) <= E[k] + 2.0 ** -52 * abs(ex), (gi, k, I[k], ex, E[k])


def test_graph_classes_match_table_I_and_oracle():
    """ae_graph_classes (no compilation): the library's class of every
    5-loop graph against the oracle's, graph by graph, and the counts per
    class against Table I's N_diag (Sec. V)."""
    from oracle.graphs import enumerate_graphs as oracle_graphs
    k, m = ae.graph_classes(5)
    gs = oracle_graphs(5)
    assert len(k) == 3213
    assert [tuple(x) for x in k] == [g.klass() for g in gs]
    assert list(m) == [g.mult for g in gs]
    want = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "table1_ndiag.txt")):
        if line.startswith("#") or not line.strip():
            continue
        a, b, c, nd = map(int, line.split())
        want[(a, b, c)] = nd
    got = {}
    for row in k:
        got[tuple(row)] = got.get(tuple(row), 0) + 1
    assert got == want
