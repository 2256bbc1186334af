"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself: a
count or expression printed in the paper, a published test vector, a closed
form, an invariant, or brute force on a tiny input.
"""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import dirac
from oracle.forest import divergent_subgraphs, terms as forest_terms
from oracle.graphs import Graph, enumerate_graphs, class_counts, perfect_matchings, is_1pi, word_of
from oracle.integrand import Integrand, project
from oracle.philox import philox4x32_10, uniforms
from oracle.sampler import Density, sample, log2_series, exp2_series, log2_tab, exp2_tab, deg_table, phi_table
from oracle.estimate import GraphOracle, summarize, weight

GOLD = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------ graph set ---
def test_graph_counts_and_table_I():
    """3213 graphs at 5 loops (Sec. I) and Table I's N_diag per class."""
    gs = enumerate_graphs(5)
    assert len(gs) == 3213
    want = {}
    for line in open(os.path.join(GOLD, "table1_ndiag.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, m, mp, nd = map(int, line.split())
        want[(k, m, mp)] = nd
    assert class_counts(gs) == want


def test_small_counts_by_brute_force():
    """1..4 loops: compare with a direct count of all oriented 1PI graphs
    (no canonical-form machinery): oriented = sum of multiplicities."""
    for n in (1, 2, 3, 4):
        oriented = 0
        for m in perfect_matchings(list(range(2 * n))):
            for s in range(2 * n + 1):
                pos = lambda x: x if x < s else x + 1
                partner = [None] * (2 * n + 1)
                for a, b in m:
                    partner[pos(a)] = pos(b)
                    partner[pos(b)] = pos(a)
                if is_1pi(partner, s):
                    oriented += 1
        gs = enumerate_graphs(n)
        # every labelled matching is a distinct oriented graph
        assert sum(g.mult for g in gs) == oriented
    assert [len(enumerate_graphs(n)) for n in (1, 2, 3, 4)] == [1, 4, 28, 269]


def test_subgraphs_are_intervals():
    for n in (2, 3, 4):
        for g in enumerate_graphs(n)[::7]:
            for S in divergent_subgraphs(g):
                v = sorted(S.verts)
                assert v == list(range(v[0], v[-1] + 1))


def _parse_example():
    lines = [l.split() for l in open(os.path.join(GOLD, "worked_example.txt"))
             if l.strip() and not l.startswith("#")]
    photons = [tuple(map(int, t.split("-"))) for t in lines[0][1:]]
    ext = int(lines[1][1])
    brackets = []
    for l in lines[2:]:
        alts = " ".join(l[1:]).split("|")
        opts = []
        for a in alts:
            a = a.strip()
            sign = -1 if a[0] == "-" else 1
            items = [x for x in a[1:].split(",") if x]
            opts.append((sign, [tuple(x.split("@")) for x in items]))
        brackets.append(opts)
    return photons, ext, brackets


def test_worked_example_expression():
    """R^new of the graph of Sec. II equals the printed expression
    (Eq. eq_example_expression) term by term."""
    photons, ext, brackets = _parse_example()
    partner = [None] * 11
    for a, b in photons:
        partner[a], partner[b] = b, a
    g = Graph(partner, ext)
    name = lambda S: "".join("abcdefghijk"[v] for v in sorted(S.verts))
    got = {}
    for sign, ops in forest_terms(g):
        key = tuple(sorted((op.replace("L-U", "LmU"), name(S)) for S, op in ops))
        got[key] = got.get(key, 0) + sign
    want = {}
    for combo in itertools.product(*brackets):
        sign = 1
        items = []
        for s, its in combo:
            sign *= s
            items += [(op, sub) for op, sub in its]
        key = tuple(sorted(items))
        want[key] = want.get(key, 0) + sign
    assert got == want


# --------------------------------------------------------------- Philox ---
def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert list(philox4x32_10(w[:4], w[4:6])) == w[6:10]


def test_uniforms_open_interval():
    u = uniforms(np.arange(20000), 3, 12345, 4)
    assert u.min() > 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.005


# --------------------------------------------------- elementary functions ---
def test_log2_exp2_series_accuracy():
    rng = np.random.default_rng(0)
    x = np.exp(rng.uniform(-700, 700, 20000))
    l = log2_series(x)
    assert np.all(np.abs(l - np.log2(x)) <= 4 * np.spacing(np.abs(np.log2(x))) + 1e-300)
    t = rng.uniform(-1000, 1000, 20000)
    assert np.all(np.abs(exp2_series(t) / np.exp2(t) - 1) < 4e-16)


def test_log2_exp2_table_accuracy():
    """The table-driven forms used by the sampler: within 4 ulp of libm for
    log2 (including arguments next to 1, where the result is tiny) and 4e-16
    relative for exp2; exact at powers of two."""
    rng = np.random.default_rng(1)
    for x in (np.exp(rng.uniform(-700, 700, 20000)), 1.0 + rng.uniform(-1e-3, 1e-3, 20000),
              rng.uniform(0.3, 3.0, 20000)):
        l = log2_tab(x)
        assert np.all(np.abs(l - np.log2(x)) <= 4 * np.spacing(np.abs(np.log2(x))) + 1e-300)
    assert list(log2_tab(np.array([0.25, 0.5, 1.0, 2.0, 1024.0]))) == [-2.0, -1.0, 0.0, 1.0, 10.0]
    t = np.concatenate([rng.uniform(-1000, 1000, 20000), rng.uniform(-1, 1, 20000)])
    assert np.all(np.abs(exp2_tab(t) / np.exp2(t) - 1) < 4e-16)
    assert list(exp2_tab(np.array([-3.0, 0.0, 1.0, 10.0]))) == [0.125, 1.0, 2.0, 1024.0]


# ---------------------------------------------------------------- pdf -----
@pytest.mark.parametrize("n,gi", [(1, 0), (2, 1), (3, 5)])
def test_density_normalisation(n, gi):
    """E_g[1/g] = simplex volume 1/(M-1)!; E_g[z_0/g] = 1/M!."""
    g = enumerate_graphs(n)[gi]
    d = Density(g)
    M = d.M
    N = 200000
    u = uniforms(np.arange(N), gi, 7, M)
    z, lg, _ = sample(d, u)
    w = np.exp2(-lg)
    m1 = w.mean() * math.factorial(M - 1)
    s1 = w.std() / math.sqrt(N) * math.factorial(M - 1)
    assert abs(m1 - 1) < 4 * s1 + 1e-3
    m2 = (z[:, 0] * w).mean() * math.factorial(M)
    s2 = (z[:, 0] * w).std() / math.sqrt(N) * math.factorial(M)
    assert abs(m2 - 1) < 4 * s2 + 1e-3


def test_sector_probabilities_exact():
    """Sector frequencies of the pure-g1 walk against prod 1/Deg / Phi(all)
    by explicit enumeration of all orderings (M = 5)."""
    g = enumerate_graphs(2)[0]
    d = Density(g, C2=0.0, C3=0.0, C4=0.0)
    M = d.M
    deg = d.deg[0]
    probs = {}
    for perm in itertools.permutations(range(M)):
        T = (1 << M) - 1
        p = 1.0
        for j in perm[:-1]:
            T ^= 1 << j
            p /= deg[T]
        probs[perm] = p
    tot = sum(probs.values())
    assert abs(tot - d.phi[0][(1 << M) - 1]) < 1e-12 * tot
    N = 100000
    u = uniforms(np.arange(N), 0, 3, M)
    z, lg, _ = sample(d, u)
    order = np.argsort(-z, axis=1, kind="stable")
    cnt = {}
    for row in order:
        cnt[tuple(row)] = cnt.get(tuple(row), 0) + 1
    chi2 = sum((cnt.get(k, 0) - N * v / tot) ** 2 / (N * v / tot) for k, v in probs.items())
    dof = len(probs) - 1
    assert chi2 < dof + 5 * math.sqrt(2 * dof)


def _plain_form_points(dens, u):
    """The sampler of Sec. III.A written in its plain form: log2 t =
    log2(u)/Deg and z = 2^lz / sum by quotients, with numpy's log2/exp2
    instead of the table-driven functions (component g1 only)."""
    M = dens.M
    deg, phi = dens.deg[0], dens.phi[0]
    S = u.shape[0]
    lz = np.zeros((S, M))
    for s_ in range(S):
        T = dens.full
        cur = 0.0
        for l in range(M - 1):
            target = u[s_, 1 + 2 * l] * phi[T]
            acc = 0.0
            chosen = -1
            last = 0
            for j in range(M):
                if T >> j & 1:
                    acc = acc + phi[T ^ (1 << j)] / deg[T ^ (1 << j)]
                    if chosen < 0 and target < acc:
                        chosen = j
                    last = j
            chosen = last if chosen < 0 else chosen
            lz[s_, chosen] = cur
            T ^= 1 << chosen
            cur = cur + np.log2(u[s_, 2 + 2 * l]) / deg[T]
        lz[s_, int(math.log2(T))] = cur
    e = np.exp2(lz)
    ssum = e.sum(1)
    return e / ssum[:, None]


def test_sampler_rounding_order_is_a_rounding_choice():
    """The oracle's sampler multiplies by tabulated reciprocals and uses
    table-driven log2/exp2 (the same operation order as the device sampler,
    so that z is reproducible bit for bit).  Written in its plain form
    (quotients, numpy's log2/exp2) the same walk gives the same sector
    choices and z within a few ulp: the order of operations is a rounding
    choice, not a different sampler."""
    g = enumerate_graphs(3)[7]
    d = Density(g)
    idx = np.arange(0, 3000, dtype=np.uint64)
    u = uniforms(idx, 7, 0, d.M)
    z, lg, comp = sample(d, u)
    sel = np.nonzero(comp == 0)[0][:400]
    zp = _plain_form_points(d, u[sel])
    rel = np.abs(zp - z[sel]) / z[sel]
    assert rel.max() < 64 * 2.0 ** -52, rel.max()


# --------------------------------------------------------------- Dirac ----
def test_dirac_identities():
    rng = np.random.default_rng(1)
    sl = lambda v: sum(dirac.METRIC[m] * v[m] * dirac.GAMMA[m] for m in range(4))
    a, b, c, d = (rng.normal(size=4) for _ in range(4))
    dot = lambda x, y: float(np.sum(dirac.METRIC * x * y))
    assert abs(dirac.trace([dirac.ONE]) - 4) < 1e-12
    assert abs(dirac.trace([("g", 1), ("g", 1)]) - 16) < 1e-12
    t4 = dirac.trace([sl(a), sl(b), sl(c), sl(d)])
    assert abs(t4 - 4 * (dot(a, b) * dot(c, d) - dot(a, c) * dot(b, d) + dot(a, d) * dot(b, c))) < 1e-9
    lhs = dirac.trace([("g", 1), sl(a), sl(b), sl(c), ("g", 1), sl(d)])
    rhs = -2 * np.trace(sl(c) @ sl(b) @ sl(a) @ sl(d))
    assert abs(lhs - rhs) < 1e-9


# ------------------------------------------------ projectors (Sec. II) ---
def _chain_of(*els):
    """A synthetic Dirac chain for oracle.integrand.project: 'mu' is the
    external gamma_mu, 'q' the q-slot (qslash), anything else a matrix."""
    def chain(q_elem=None, mu_repl=None):
        out = []
        for e in els:
            if isinstance(e, str) and e == "mu":
                out.append(mu_repl if mu_repl is not None else ("g", "mu"))
            elif isinstance(e, str) and e == "q":
                out.append(q_elem)
            else:
                out.append(e)
        return out
    return chain, any(isinstance(e, str) and e == "q" for e in els)


def _proj(channel, parts):
    """The projection is linear in Gamma: sum of coef * project(chain)."""
    return sum(c * project(channel, *_chain_of(*els)) for c, els in parts)


def test_amm_projector_on_synthetic_vertices():
    """A = F2(0) (Sec. II, the projector of the anomalous magnetic moment),
    with P = (p + p')/2, q = p' - p, m = 1, on structures whose form factors
    are textbook facts:
      gamma_mu -> F2 = 0;  i sigma_{mu nu} q^nu / 2m -> 1;
      P_mu / m -> -1 (Gordon identity: gamma_mu = P_mu/m + i sigma q/2m);
      q_mu -> 0 (the F3 structure, annihilated);
      (pslash' - m) gamma_mu and gamma_mu (pslash - m) -> 0 (vanish on shell).
    i sigma_{mu nu} q^nu = -(gamma_mu qslash - qslash gamma_mu)/2,
    P_mu = (Pslash gamma_mu + gamma_mu Pslash)/2, likewise q_mu."""
    P = dirac.PSLASH
    assert abs(_proj("F2", [(1.0, ("mu",))])) < 1e-13
    assert abs(_proj("F2", [(-0.25, ("mu", "q")), (0.25, ("q", "mu"))]) - 1.0) < 1e-13
    assert abs(_proj("F2", [(0.5, (P, "mu")), (0.5, ("mu", P))]) + 1.0) < 1e-13
    assert abs(_proj("F2", [(0.5, ("q", "mu")), (0.5, ("mu", "q"))])) < 1e-13
    # pslash' = Pslash + qslash/2 on the left, pslash = Pslash - qslash/2 on the right
    assert abs(_proj("F2", [(1.0, (P, "mu")), (-1.0, ("mu",)), (0.5, ("q", "mu"))])) < 1e-13
    assert abs(_proj("F2", [(1.0, ("mu", P)), (-1.0, ("mu",)), (-0.5, ("mu", "q"))])) < 1e-13
    # linearity across the two parts (q-independent and linear in q)
    mix = [(0.3, ("mu",)), (-0.25 * 2.0, ("mu", "q")), (0.25 * 2.0, ("q", "mu")), (0.5 * 0.7, (P, "mu")),
           (0.5 * 0.7, ("mu", P))]
    assert abs(_proj("F2", mix) - (2.0 - 0.7)) < 1e-12


def test_l_u_projectors_recover_abc_and_uv():
    """U and L of Sec. II read a, b, c of Eq. eq_gamma_general_q0 (at q = 0,
    m = 1) off Gamma_mu = a gamma_mu + b P_mu + c Pslash P_mu + d [Pslash,
    gamma_mu]: channel 'a' gives a (U), 'abc' gives a + m b + m^2 c (L), 'bc'
    gives m b + m^2 c (L - U), whatever d; a self-energy Sigma = u + v Pslash
    gives u and v."""
    P = dirac.PSLASH
    rng = np.random.default_rng(11)
    for _ in range(3):
        a, b, c, d = rng.normal(size=4)
        G = [(a, ("mu",)), (b / 2, (P, "mu")), (b / 2, ("mu", P)), (c / 2, (P, P, "mu")), (c / 2, (P, "mu", P)),
             (d, (P, "mu")), (-d, ("mu", P))]
        assert abs(_proj("a", G) - a) < 1e-12
        assert abs(_proj("abc", G) - (a + b + c)) < 1e-12
        assert abs(_proj("bc", G) - (b + c)) < 1e-12
        u, v = rng.normal(size=2)
        S = [(u, (dirac.ONE,)), (v, (P,))]
        assert abs(_proj("u", S) - u) < 1e-12
        assert abs(_proj("v", S) - v) < 1e-12


# ------------------------------------------------------------ estimator ---
def test_summarize_sigma_down_by_hand():
    """Eq. eq_sigma_down on hand-computed cases: y = (1, 2, 3, 4): mean 5/2,
    sigma_down^2 = 30/16 - 100/64 = 5/16; multiplicity scales value and
    sigma; mean |y| of (-1, 3) is 2 with sigma_down^2 = 10/4 - 4/8 = 2."""
    r = summarize([1.0, 2.0, 3.0, 4.0])
    assert r["mean"] == 2.5 and r["n"] == 4
    assert abs(r["sigma1"] - math.sqrt(5.0 / 16.0)) < 1e-15
    assert r["sum_y"] == 10.0 and r["sum_y2"] == 30.0
    r2 = summarize([1.0, 2.0, 3.0, 4.0], mult=2)
    assert r2["value"] == 5.0 and abs(r2["sigma"] - 2 * math.sqrt(5.0 / 16.0)) < 1e-15
    r3 = summarize([-1.0, 3.0])
    assert r3["mean"] == 1.0 and r3["mean_abs"] == 2.0
    assert abs(r3["sigma1"] - math.sqrt(2.0)) < 1e-15
    # a constant sample (binary-exact value) has sigma_down exactly 0
    assert summarize([0.375] * 1000)["sigma1"] == 0.0


# ------------------------------------------------------------ integrand ---
def test_one_loop_quadrature_is_half():
    """A_1^(2) = 1/2 (Sec. I) by Gauss-Legendre on the 1-simplex; the
    1-loop integrand is a polynomial, so the rule is exact."""
    g = enumerate_graphs(1)[0]
    I = Integrand(g)
    x, w = np.polynomial.legendre.leggauss(8)
    t = 0.5 * (x + 1)
    val = sum(0.5 * wi * I.evaluate(np.array([ti, 1 - ti]))[0] for ti, wi in zip(t, w))
    assert abs(val - 0.5) < 1e-14


def _mirror_graph(g):
    N = g.nverts
    p = [None] * N
    for v in range(N):
        if v != g.s:
            p[N - 1 - v] = N - 1 - g.partner[v]
    return Graph(p, N - 1 - g.s)


@pytest.mark.parametrize("n", [2, 3])
def test_mirror_invariance(n):
    """A graph and its arrow-reversed image give the same integrand at
    corresponding points (charge conjugation; graphs that differ only by
    arrow direction are one graph, Sec. I).  Fails if the AMM projector
    picks up the q^mu structure."""
    rng = np.random.default_rng(n)
    for g in enumerate_graphs(n):
        if g.mult != 2:
            continue
        h = _mirror_graph(g)
        Ig, Ih = Integrand(g), Integrand(h)
        ig, ih = g.line_index(), h.line_index()
        N = g.nverts
        for _ in range(2):
            z = rng.dirichlet(np.ones(3 * n - 1))
            zh = np.empty_like(z)
            for key, i in ig.items():
                if key[0] == 'e':
                    mk = ('e', N - key[1])
                else:
                    mk = ('g', N - 1 - key[2], N - 1 - key[1])
                zh[ih[mk]] = z[i]
            a, b = Ig.evaluate(z)[0], Ih.evaluate(zh)[0]
            assert abs(a - b) <= 1e-11 * max(abs(a), 1.0)
        if n == 3:
            break


def test_two_loop_finiteness():
    """Subtracted integrands are integrable: shrinking any subset of lines,
    |I| * lambda^|s| vanishes as a positive power of lambda (UV and IR)."""
    rng = np.random.default_rng(5)
    for g in enumerate_graphs(2):
        I = Integrand(g)
        M = 5
        for r in range(1, M):
            for s in itertools.combinations(range(M), r):
                z0 = rng.dirichlet(np.ones(M))
                vals = []
                for lam in (1e-6, 1e-8):
                    z = z0.copy()
                    z[list(s)] *= lam
                    z /= z.sum()
                    vals.append(abs(I.evaluate(z)[0]) * lam ** r + 1e-300)
                slope = math.log(vals[1] / vals[0]) / math.log(1e-8 / 1e-6)
                assert slope > 0.3, (g.word, s, slope)


def test_three_loop_finiteness():
    """UV and IR finiteness of the subtracted integrand (Sec. II) at three
    loops, for three graphs spread over the canonical list: shrinking any of
    the 254 proper subsets of the 8 lines by lambda, |I| lambda^|s| vanishes
    as a positive power of lambda (measured slope 1.0 on every subset; a
    missing subtraction term leaves a slope near 0)."""
    rng = np.random.default_rng(7)
    gs = enumerate_graphs(3)
    for gi in (0, 12, 27):
        I = Integrand(gs[gi])
        M = 8
        for r in range(1, M):
            for s in itertools.combinations(range(M), r):
                z0 = rng.dirichlet(np.ones(M))
                vals = []
                for lam in (1e-6, 1e-8):
                    z = z0.copy()
                    z[list(s)] *= lam
                    z /= z.sum()
                    vals.append(abs(I.evaluate(z)[0]) * lam ** r + 1e-300)
                slope = math.log(vals[1] / vals[0]) / math.log(1e-8 / 1e-6)
                assert slope > 0.5, (gi, s, slope)


def _two_loop_graph_sums(gi, n):
    """(sum y, sum y^2, N, exactly re-evaluated) of 2-loop graph gi over
    samples 0..n-1 (seed 0): a spawned worker of the closed-form pin."""
    from oracle.estimate import GraphOracle
    g = enumerate_graphs(2)[gi]
    y, n_exact = GraphOracle(g, gi).samples_batched(0, n, 0)
    return math.fsum(y), math.fsum(y * y), len(y), n_exact


def test_two_loop_sum_closed_form():
    """The oracle's own 2-loop sum against the closed form (CPU, no GPU).

    A_1^(4) = 197/144 + pi^2/12 - (pi^2/2) ln 2 + (3/4) zeta(3) (Petermann;
    Sommerfield) = -0.328478965579...; the graphs without lepton loops give it
    minus the vacuum-polarisation graph, 119/36 - pi^2/3, i.e.
    -0.344166387438296.  2^20 samples per graph (Eqs. eq_integral_approx,
    eq_sigma_down, eq_sigma_sum): the estimate must lie within 3 sigma_down,
    with sigma_down below 0.01 (3 % of the value) so that a dropped or
    mis-signed forest term (an O(0.1) change) cannot pass."""
    import concurrent.futures as cf
    import multiprocessing as mp
    zeta3 = 1.2020569031595942854
    a4 = 197 / 144 + math.pi ** 2 / 12 - math.pi ** 2 / 2 * math.log(2) + 0.75 * zeta3
    want = a4 - (119 / 36 - math.pi ** 2 / 3)
    assert abs(want - (-0.344166387438296)) < 1e-14
    gs = enumerate_graphs(2)
    n = 1 << 20
    with cf.ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(_two_loop_graph_sums, range(len(gs)), [n] * len(gs)))
    val = var = 0.0
    for g, (sy, sy2, N, n_exact) in zip(gs, res):
        assert n_exact < N // 100
        val += g.mult * sy / N
        var += g.mult ** 2 * max(sy2 / N ** 2 - sy ** 2 / N ** 3, 0.0)
    sig = math.sqrt(var)
    assert sig < 0.01, sig
    assert abs(val - want) < 3 * sig, (val, sig, want)


def test_batched_integrand_matches_exact():
    """The batched floating-point integrand (statistical pins only) against
    the exact one at 64 sampler points of every 2-loop graph."""
    from oracle.estimate import GraphOracle
    for gi, g in enumerate(enumerate_graphs(2)):
        o = GraphOracle(g, gi)
        r = o.samples(0, 64, 7)
        I, K = o.integrand.evaluate_many(r["z"], np.longdouble)
        assert np.all(np.abs(I.astype(np.float64) - r["I"]) <= 1e-8 * np.abs(r["I"]) + 1e-12 * r["K"])
        assert np.allclose(K.astype(np.float64), r["K"], rtol=1e-12)


def test_batched_long_double_coefficients_are_long_double():
    """The rational coefficients enter the long-double form rounded once to
    long double (numpy would take a Fraction through double); large
    numerators and denominators included."""
    from fractions import Fraction
    from oracle.integrand import _rational_in
    ld = np.longdouble
    assert _rational_in(ld, Fraction(1, 3)) == ld(1) / ld(3)
    assert _rational_in(ld, Fraction(1, 3)) != ld(float(Fraction(1, 3)))
    assert _rational_in(ld, Fraction(-7, 10)) == -ld(7) / ld(10)
    assert _rational_in(ld, 12345) == ld(12345)
    big = Fraction(3 ** 40 + 1, 2 ** 70 + 3)   # parts wider than 64 bits: rounded, not truncated to double
    assert abs(float((Fraction(str(_rational_in(ld, big))) - big) / big)) < 2.0 ** -60
    assert _rational_in(np.float64, Fraction(1, 3)) == 1.0 / 3.0


def test_weight_range_safe():
    assert weight(3.0, 1.0) == 1.5
    assert weight(1.0, 2000.0) == 2.0 ** -2000 or weight(1.0, 2000.0) == 0.0
    assert weight(2.0 ** -1000, -1500.0) == 2.0 ** 500
    # the array form used by the statistical pins is the same function
    from oracle.estimate import weight_many
    rng = np.random.default_rng(2)
    lg = rng.uniform(-900.0, 3000.0, 500)
    I = rng.normal(size=500) * 10.0 ** rng.uniform(-30, 30, 500)
    assert np.array_equal(weight_many(I, lg), np.array([weight(a, b) for a, b in zip(I, lg)]))


# ------------------------------------------------------ learned proposal ---
def test_proposal_gradient_finite_differences():
    """The oracle's backpropagation against central differences of its own
    loss (float64, unrounded weights)."""
    from oracle import proposal as pr
    from tests import proposal_inputs as pin
    g = enumerate_graphs(2)[1]
    d = Density(g)
    M = d.M
    p = pin.params(3).astype(np.float64)
    order, lt, w = pin.records(3, 40, M)
    wplain = np.ones(1 << M)
    wplain[1:-1] = d.phi[0][1:-1] / d.deg[0][1:-1]
    deg = d.deg[0].copy()
    grad = pr.grad_unrounded(p, deg, wplain, order, lt, w, M)
    rng = np.random.default_rng(0)
    idx = list(rng.choice(pr.NPARAM, 12, replace=False)) + [pr.NPARAM - 1, pr.NPARAM - 16 - 5]
    for k in idx:
        h = 1e-5
        pp, pm = p.copy(), p.copy()
        pp[k] += h
        pm[k] -= h
        fd = (pr.loss_only(pp, deg, wplain, order, lt, w, M) - pr.loss_only(pm, deg, wplain, order, lt, w, M)) / (2 * h)
        assert abs(fd - grad[k]) <= 1e-5 * max(1.0, abs(fd)), (k, fd, grad[k])


def test_proposal_zero_output_is_plain_walk():
    """With a zero output layer the learned walk is exactly the plain walk:
    P(j|T) = Phi(T\\j)/Deg(T\\j)/Phi(T) and Deg_theta = Deg."""
    from oracle import proposal as pr
    g = enumerate_graphs(2)[0]
    d = Density(g)
    M = d.M
    p = np.zeros(pr.NPARAM)
    f = pr.forward(p, M)
    wplain = np.ones(1 << M)
    wplain[1:-1] = d.phi[0][1:-1] / d.deg[0][1:-1]
    logp, degt = pr.tables(f["o"], d.deg[0], wplain, M)
    for T in range(1, 1 << M):
        js = [j for j in range(M) if T >> j & 1]
        if len(js) < 2:
            continue
        for j in js:
            want = d.phi[0][T ^ (1 << j)] / d.deg[0][T ^ (1 << j)] / d.phi[0][T]
            assert abs(np.exp(logp[T, j]) - want) < 1e-12
    assert np.allclose(degt[1:-1], d.deg[0][1:-1])


def _random_outputs(M, seed, scale=1.5):
    return np.random.default_rng(seed).normal(0.0, scale, size=(1 << M, 16))


def test_learned_mixture_is_a_density():
    """The oracle's learned mixture density integrates to 1 over the simplex:
    E_g[q/g] = 1 with points drawn from the plain density g (2-loop graph,
    random network outputs); a missing Deg_theta factor or an unnormalised
    choice probability fails it."""
    from oracle import proposal as pr
    g = enumerate_graphs(2)[2]
    d = Density(g)
    M = d.M
    o = _random_outputs(M, 4)
    wplain = np.ones(1 << M)
    wplain[1:-1] = d.phi[0][1:-1] / d.deg[0][1:-1]
    logp, degt = pr.tables(o, d.deg[0], wplain, M)
    idx = np.arange(0, 40000, dtype=np.uint64)
    z, lg, _ = sample(d, uniforms(idx, 2, 3, M))
    lq = pr.log2_mixture(d, logp, degt, 0.1, np.log2(z))
    r = np.exp2(lq - lg)
    assert abs(r.mean() - 1.0) < 4 * r.std() / math.sqrt(len(r)), (r.mean(), r.std())


def test_learned_sampler_matches_its_density():
    """Points drawn by the oracle's learned sampler have E_q[1/q] = 1/(M-1)!
    (the simplex volume): the walk and the density agree."""
    from oracle import proposal as pr
    from oracle.philox import uniforms_fine
    g = enumerate_graphs(2)[1]
    d = Density(g)
    M = d.M
    o = _random_outputs(M, 5)
    u = uniforms_fine(np.arange(0, 20000, dtype=np.uint64), 1, 9, M)
    z, lq, plain = pr.learned_points(d, o, 0.1, u)
    assert np.allclose(z.sum(1), 1.0)
    assert 0.05 < plain.mean() < 0.15
    w = np.exp2(-lq) * math.factorial(M - 1)
    assert abs(w.mean() - 1.0) < 4 * w.std() / math.sqrt(len(w)), (w.mean(), w.std())


def test_fine_uniforms_layout():
    """uniforms_fine: u = (2m + 1) 2^-53 with m the 52 high-order bits of
    (w0, w1); strictly inside (0, 1)."""
    from oracle.philox import philox4x32_10, uniforms_fine
    u = uniforms_fine(np.array([5, 2 ** 33 + 7], dtype=np.uint64), 3, 11, 2)
    for row, idx in enumerate((5, 2 ** 33 + 7)):
        for b in range(2):
            w = philox4x32_10([idx & 0xFFFFFFFF, idx >> 32, 3, b], [11, 0])
            for h in range(2):
                m = (w[2 * h] << 20) | (w[2 * h + 1] >> 12)
                assert u[row, 2 * b + h] == (2 * m + 1) * 2.0 ** -53
    assert np.all((u > 0) & (u < 1))


def test_oracle_pool_values_cover_exact():
    """The scale-test helper (tests/oracle_pool.py): its batched values lie
    within its stated uncertainty of the exact ones at its own least certain
    samples and at random ones, its points are the sampler's, and the exact
    referee returns Integrand.evaluate."""
    from oracle.estimate import GraphOracle
    from tests.oracle_pool import exact_values, graph_values
    g = enumerate_graphs(2)[1]
    r = graph_values((2, 1, 100, 2048, 3, 8))
    assert r["first"] == 100 and len(r["I"]) == 2048
    o = GraphOracle(g, 1)
    p = o.points(100, 2048, 3)
    assert np.array_equal(p["z"], r["z"]) and np.array_equal(p["log2g"], r["log2g"])
    k = r["exact_idx"]
    assert np.all(np.abs(r["I"][k] - r["exact_I"]) <= r["scale"][k])
    pick = np.random.default_rng(4).choice(2048, 24, replace=False)
    ex = exact_values((2, 1, r["z"][pick]))
    assert np.array_equal(ex, np.array([float(o.integrand.evaluate(z)[0]) for z in r["z"][pick]]))
    assert np.all(np.abs(r["I"][pick] - ex) <= r["scale"][pick])
