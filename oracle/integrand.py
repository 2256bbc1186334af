"""Oracle: the divergence-subtracted Feynman-parametric integrand I(z) of one
vertex graph (Sec. II; Sec. III.A, Eq. eq_feyn_integral).

TEST INFRASTRUCTURE ONLY (see the package header).

Reading of the construction (the paper defers it to its earlier work; what
follows is the reading this oracle and the library both implement):

* Every term (F, G') of R^new factorises into one factor per forest element
  S: the reduced graph S/children(S), in which each maximal element of F
  strictly inside S is collapsed to a point.  The operator on a child leaves
  only a simple Dirac structure in the parent:
      U on a self-energy   -> u(m^2) * 1 + v(m^2) * pslash,
      U on a vertex        -> a(m^2) * gamma^nu,
      L on a vertex        -> [a + m b + m^2 c](m^2) * gamma^nu,
      A on a vertex        -> F2(0) * gamma^nu,
      L-U on G             -> [m b + m^2 c](m^2) * gamma^mu,
  with the structures of Eq. eq_gamma_general_q0.  Each factor is a scalar
  Schwinger-parameter integrand over its own lines; the term is the product
  of the factors over the joint parameter space, and every term is put on the
  same simplex by alpha = lambda*z over all lines and integrating lambda.
* Schwinger parameters and Gaussian loop integration (Minkowski metric):
      <kappa_l kappa_l'> = (i/2) Z_ll' g,  Z = eta A^-1 eta^T, U = det A,
      V = -B^T A^-1 B (on shell: p^2 = m^2 makes the constant term vanish);
  the lambda integral of a term with j Wick pairs in all is
      Gamma(n-j) (-W)^-(n-j),   W = sum of the factors' V,
  and the full coefficient of (alpha/pi)^n is
      I(z) = z_e 4^-n (-1)^n sum_terms sign * sum_j (-1)^j 2^-j Gamma(n-j)
             (-W)^-(n-j) * [convolution over factors of U_H^-2 N_H,j].
* The two electron lines at the external vertex are merged (the 3n -> 3n-1
  trick of Sec. III.A): at linear order in q every integrand is linear in the
  split fraction, so the split integral equals the value at alpha1 = alpha2
  = z_e/2, times the measure factor z_e.
* A = F2(0), extracted at linear order in q from Gamma(P +- q/2) with the
  projector F2 = -(1/24) (g_ab - P_a P_b) tau^ba, tau from
  Tr[(P+q/2+m) Gamma (P-q/2+m) q_a Y^a], Y_mu^a = [gamma_mu, gamma^a]
  + 3 gamma_mu Pslash gamma^a + 3 g_mu^a (on shell it returns F2 and
  annihilates the gamma^mu (F1) and q^mu (F3) structures as well as every
  structure that vanishes on shell, so a graph and its mirror image give
  the same value).
* a, b, c from traces: E1 = Tr[Gamma^mu gamma_mu] = 16a + 4c,
  E2 = Tr[Gamma^mu P_mu Pslash] = 4a + 4c, E3 = Tr[Gamma^mu P_mu] = 4b;
  u = Tr[Sigma]/4, v = Tr[Pslash Sigma]/4.

Graph functions are evaluated in exact rational arithmetic at each sample
point (fractions of the double-precision z), then rounded once; the Dirac
part is expanded into monomials whose coefficients come from explicit
numeric traces (``dirac.trace``), computed once per graph.

Pinned by A_1^(2) = 1/2 (1-loop, deterministic quadrature); by the 2-loop
no-lepton-loop sum -0.344166387438296 within 3 sigma (the oracle's own sum,
2^20 samples per graph, on the CPU; evaluate_many with exact re-evaluation
where two precisions disagree); by UV/IR finiteness of the subtracted
integrands (scaling of every line subset: all 2-loop graphs and three-loop
graphs 0, 12, 27); by mirror invariance; and, for the closing projections
(``project``), by textbook form factors of synthetic vertices (F2 of
gamma_mu, i sigma q/2m, P_mu/m (Gordon), q_mu and on-shell-vanishing
structures; a, b, c and u, v read off Eq. eq_gamma_general_q0 structures).
3-, 4-, 5-loop values: parity unpinned beyond these properties.
"""
from fractions import Fraction
from itertools import product
import math
import numpy as np

from . import dirac
from .forest import terms as forest_terms

P = dirac.PSLASH
ONE = dirac.ONE


# ---------------------------------------------------------------- factors --

class Factor:
    """Reduced graph S/children for one forest element S."""

    def __init__(self, g, S, children):
        self.g = g
        self.S = S
        self.kind = S.kind
        verts = sorted(S.verts)
        assert verts == list(range(verts[0], verts[-1] + 1)), "subgraph is not an interval"
        child_of = {}
        for C in children:
            for v in C.verts:
                child_of[v] = C
        self.nodes = []
        seen = set()
        for v in verts:
            C = child_of.get(v)
            if C is None:
                self.nodes.append(('v', v))
            elif id(C) not in seen:
                seen.add(id(C))
                self.nodes.append(('c', C))
        inner = set()
        for C in children:
            inner |= C.lines
        self.node_of = {}
        for k, nd in enumerate(self.nodes):
            if nd[0] == 'v':
                self.node_of[nd[1]] = k
            else:
                for v in nd[1].verts:
                    self.node_of[v] = k
        # electron lines between consecutive nodes: the original line entering
        # the first vertex of the next node
        self.elines = []
        for k in range(len(self.nodes) - 1):
            nd = self.nodes[k + 1]
            first = nd[1] if nd[0] == 'v' else min(nd[1].verts)
            self.elines.append(('e', first))
        self.photons = [l for l in S.lines if l[0] == 'g' and l not in inner]
        self.photons.sort()
        self.loops = len(self.photons)
        self.ext_node = None
        for k, nd in enumerate(self.nodes):
            if self.label(k) == 'mu':
                self.ext_node = k
        assert (self.ext_node is None) == (self.kind == 'SE')

    def label(self, k):
        """Lorentz label of the gamma at node k (None for a self-energy insertion)."""
        nd = self.nodes[k]
        if nd[0] == 'v':
            v = nd[1]
            if v == self.g.s:
                return 'mu'
            pl = ('g', min(v, self.g.partner[v]), max(v, self.g.partner[v]))
            return ('ph', pl) if pl in self.photons else 'mu'
        C = nd[1]
        if C.kind == 'SE':
            return None
        if C.ext_photon == 'ext':
            return 'mu'
        return ('ph', C.ext_photon) if C.ext_photon in self.photons else 'mu'

    # ----------------------------------------------------- graph functions --
    def graph_functions(self, alpha, batch=False):
        """Exact U, Z (electron-line block), flows a, b and V.
        alpha: dict line -> Fraction (or, batch=True, line -> array of
        floating-point values over sample points)."""
        E = len(self.elines)
        Lp = self.loops
        ae = [alpha[l] for l in self.elines]
        # photon c spans elines [lo, hi): cycle = photon plus the path back
        spans = []
        for ph in self.photons:
            na, nb = self.node_of[ph[1]], self.node_of[ph[2]]
            spans.append((min(na, nb), max(na, nb)))
        A = [[(alpha[self.photons[0]] * 0 if batch else Fraction(0))] * Lp for _ in range(Lp)]
        # (x = x + y rather than x += y: batched entries are shared arrays)
        for c in range(Lp):
            A[c][c] = A[c][c] + alpha[self.photons[c]]
            for c2 in range(Lp):
                lo = max(spans[c][0], spans[c2][0])
                hi = min(spans[c][1], spans[c2][1])
                for k in range(lo, hi):
                    A[c][c2] = A[c][c2] + ae[k]
        # eta for electron lines: -1 on the span of each photon
        eta = [[(-1 if spans[c][0] <= k < spans[c][1] else 0) for c in range(Lp)] for k in range(E)]
        det, Ainv = _det_inv_batch(A) if batch else _det_inv(A)
        Z = [[sum(eta[k][c] * Ainv[c][c2] * eta[k2][c2] for c in range(Lp) for c2 in range(Lp))
              for k2 in range(E)] for k in range(E)]
        # particular flow along the path: P on every electron line, q-part d_k
        d = []
        for k in range(E):
            if self.ext_node is None:
                d.append(0.0 if batch else Fraction(0))
            elif batch:
                d.append(-0.5 if k < self.ext_node else 0.5)
            else:
                d.append(Fraction(-1, 2) if k < self.ext_node else Fraction(1, 2))
        a = [1 - sum(Z[k][k2] * ae[k2] for k2 in range(E)) for k in range(E)]
        b = [d[k] - sum(Z[k][k2] * ae[k2] * d[k2] for k2 in range(E)) for k in range(E)]
        # V = -B^T A^-1 B, B_c = sum_k alpha_k eta_kc (coefficient of P)
        Bv = [sum(ae[k] * eta[k][c] for k in range(E)) for c in range(Lp)]
        V = -sum(Bv[c] * Ainv[c][c2] * Bv[c2] for c in range(Lp) for c2 in range(Lp))
        return det, Z, a, b, V

    # ------------------------------------------------------- Dirac sites --
    def sites(self, child_chan):
        """Sites in chain order (left = outgoing end): ('prop', eline index) or
        ('ins', eline index of the line entering the insertion node)."""
        out = []
        for k in range(len(self.nodes) - 1, -1, -1):
            nd = self.nodes[k]
            if nd[0] == 'c' and nd[1].kind == 'SE' and child_chan[id(nd[1])] == 'v':
                out.append(('node', k, 'ins', k - 1))
            else:
                out.append(('node', k, None, None))
            if k > 0:
                out.append(('prop', k - 1))
        return out


def _det_inv(A):
    """Exact determinant and inverse by Gauss-Jordan elimination."""
    n = len(A)
    if n == 0:
        return Fraction(1), []
    M = [row[:] + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(A)]
    det = Fraction(1)
    for c in range(n):
        p = next(r for r in range(c, n) if M[r][c] != 0)
        if p != c:
            M[c], M[p] = M[p], M[c]
            det = -det
        piv = M[c][c]
        det *= piv
        M[c] = [x / piv for x in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return det, [row[n:] for row in M]


def _rational_in(dtype, q):
    """The rational q (int or Fraction) in the floating type dtype.  numpy
    converts a Fraction through a Python float, which would leave a long
    double evaluation with double-rounded coefficients; for wider types the
    numerator and denominator are read from their decimal strings (exact up
    to 64 bits, else rounded once) and divided."""
    q = Fraction(q)
    if np.dtype(dtype) == np.float64:
        return np.float64(float(q))   # correctly rounded
    return dtype(str(q.numerator)) / dtype(str(q.denominator))


def _det_inv_batch(A):
    """Determinant and inverse by Gauss-Jordan elimination for matrices whose
    entries are arrays over sample points (one matrix per point).  The
    matrices here are positive definite (sums of alpha > 0 over the lines of
    the cycles), so no pivot vanishes and rows are taken in order."""
    n = len(A)
    if n == 0:
        return 1.0, []
    one = A[0][0] * 0 + 1
    M = [row[:] + [one * (i == j) for j in range(n)] for i, row in enumerate(A)]
    det = one
    for c in range(n):
        piv = M[c][c]
        det = det * piv
        M[c] = [x / piv for x in M[c]]
        for r in range(n):
            if r != c:
                f = M[r][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return det, [row[n:] for row in M]


# ------------------------------------------------ coefficient expansion --

def _matchings(items):
    if not items:
        yield []
        return
    a = items[0]
    for k in range(1, len(items)):
        rest = items[1:k] + items[k + 1:]
        for m in _matchings(rest):
            yield [(a, items[k])] + m


def _chain(factor, elems, child_chan, mu_repl=None):
    """Chain elements (left = outgoing end) for one configuration.
    elems: dict site-position -> element for sites (prop / ins)."""
    out = []
    seq = factor.sites(child_chan)
    for pos, st in enumerate(seq):
        if st[0] == 'node':
            lab = factor.label(st[1])
            if lab is None:
                if st[2] == 'ins':
                    out.append(elems[pos])
                # u-channel insertion: identity, nothing to add
            elif lab == 'mu':
                out.append(mu_repl if mu_repl is not None else ('g', 'mu'))
            else:
                out.append(('g', lab))
        else:
            out.append(elems[pos])
    return out


def coefficient_table(factor, channel, child_chan):
    """Expand U^-2-weighted numerator of a factor channel into monomials.
    Returns list of (coef, j, a_sites, q_site, pairs) with sites given as
    eline indices (an insertion uses the eline entering it)."""
    seq = factor.sites(child_chan)
    site_pos = [p for p, st in enumerate(seq) if st[0] == 'prop' or st[2] == 'ins']
    line_of = {}
    is_prop = {}
    for p in site_pos:
        st = seq[p]
        if st[0] == 'prop':
            line_of[p], is_prop[p] = st[1], True
        else:
            line_of[p], is_prop[p] = st[3], False
    F2 = channel == 'F2'
    table = []
    nsites = len(site_pos)
    for r in range(0, nsites + 1, 2):
        from itertools import combinations
        for K in combinations(site_pos, r):
            rest = [p for p in site_pos if p not in K]
            for pairs in _matchings(list(K)):
                elk = {}
                for t, (p1, p2) in enumerate(pairs):
                    elk[p1] = ('g', ('k', t))
                    elk[p2] = ('g', ('k', t))
                modes_each = []
                for p in rest:
                    modes_each.append(['m', 'P'] if is_prop[p] else ['P'])
                qchoices = [None] + (rest if F2 else [])
                for qsite in qchoices:
                    for modes in product(*[(['q'] if p == qsite else me)
                                           for p, me in zip(rest, modes_each)]):
                        el = dict(elk)
                        asites = []
                        for p, md in zip(rest, modes):
                            if md == 'm':
                                el[p] = ONE
                            elif md == 'P':
                                el[p] = P
                                asites.append(line_of[p])
                            else:
                                el[p] = 'Q'
                        coef = _project(factor, channel, child_chan, el, qsite)
                        if abs(coef) > 1e-12:
                            table.append((coef, len(pairs), tuple(sorted(asites)),
                                          None if qsite is None else line_of[qsite],
                                          tuple((line_of[a], line_of[b]) for a, b in pairs)))
    return table


def _project(factor, channel, child_chan, el, qsite):
    """Apply the channel's closing projection to one configuration."""
    def chain(q_elem=None, mu_repl=None):
        e = el
        if qsite is not None and q_elem is not None:
            e = dict(el)
            e[qsite] = q_elem
        return _chain(factor, e, child_chan, mu_repl=mu_repl)
    return project(channel, chain, qsite is not None)


def project(channel, chain, has_q):
    """Closing projection of one Dirac chain (linear in the chain).

    chain(q_elem, mu_repl) returns the chain's elements with its q-slot (if
    has_q) holding q_elem and its external gamma_mu replaced by mu_repl
    (None: gamma_mu itself).  Channels (Eq. eq_gamma_general_q0, m = 1):
      'u', 'v'          Sigma = u + v Pslash  ->  u, v;
      'a', 'abc', 'bc'  Gamma_mu = a gamma_mu + b P_mu + c Pslash P_mu
                        + d [Pslash, gamma_mu] at q = 0  ->  a, a+b+c, b+c;
      'F2'              the magnetic form factor F2(0) of Gamma_mu(P+q/2,
                        P-q/2) at linear order in q (the AMM projector A).
    """
    if channel == 'u':
        return (dirac.trace(chain()) / 4).real
    if channel == 'v':
        return (dirac.trace([P] + chain()) / 4).real
    if channel in ('a', 'abc', 'bc'):
        E1 = dirac.trace(chain() + [('g', 'mu')]).real
        E2 = dirac.trace(chain(mu_repl=P) + [P]).real
        E3 = dirac.trace(chain(mu_repl=P)).real
        if channel == 'a':
            return (E1 - E2) / 12
        if channel == 'abc':
            return (E2 + E3) / 4
        return E3 / 4 + (4 * E2 - E1) / 12
    assert channel == 'F2'
    Lam = P + ONE
    tot = 0.0
    for part in ('g', 'P'):
        # the two q-slots: gamma^beta (g part) or Pslash (P part)
        qb = ('g', 'beta') if part == 'g' else P
        if part == 'g':
            Ys = [[('g', 'mu'), ('g', 'beta')], [('g', 'beta'), ('g', 'mu')],
                  [('g', 'mu'), P, ('g', 'beta')]]
        else:
            Ys = [[('g', 'mu'), P], [P, ('g', 'mu')], [('g', 'mu'), P, P]]
        wts = [1.0, -1.0, 3.0]
        sgn = 1.0 if part == 'g' else -1.0
        # the 3 g_mu^a part of Y: the q-slot contracts with the external gamma^mu
        qmu = ('g', 'mu') if part == 'g' else P
        mrep = None if part == 'g' else P
        if has_q:
            ch = chain(qb)
            for Y, w in zip(Ys, wts):
                tot += sgn * w * dirac.trace([Lam] + ch + [Lam] + Y).real
            ch = chain(qmu, mrep)
            tot += sgn * 3.0 * dirac.trace([Lam] + ch + [Lam]).real
        else:
            ch = chain()
            for Y, w in zip(Ys, wts):
                tot += sgn * w * 0.5 * dirac.trace([qb] + ch + [Lam] + Y).real
                tot -= sgn * w * 0.5 * dirac.trace([Lam] + ch + [qb] + Y).real
            ch = chain(mu_repl=mrep)
            tot += sgn * 3.0 * 0.5 * dirac.trace([qmu] + ch + [Lam]).real
            tot -= sgn * 3.0 * 0.5 * dirac.trace([Lam] + ch + [qmu]).real
    return -tot / 24.0


def _listify(x):
    return [_listify(v) for v in x] if isinstance(x, (tuple, list)) else x


def _tuplify(x):
    return tuple(_tuplify(v) for v in x) if isinstance(x, list) else x


# --------------------------------------------------------- the integrand --

CHANNEL_OF_OP = {'A': 'F2', 'L': 'abc', 'L-U': 'bc'}


class Integrand:
    """I(z) of one graph: terms, factors and their coefficient tables.

    tables (optional): the coefficient tables of the factors, keyed as in
    self.tables (as written by table_records()), to skip their computation
    (minutes to hours per graph at four loops and more); the factors and
    terms are rebuilt as usual."""

    def __init__(self, g, tables=None):
        self.g = g
        self.n = g.n
        self.idx = g.line_index()
        self.terms = []           # list of (sign, [assignments])
        cache = {}
        for sign, ops in forest_terms(g):
            F = [S for S, _ in ops]
            opof = {id(S): op for S, op in ops}
            facs = []
            for S in F:
                inner = [C for C in F if C is not S and C.lines < S.lines]
                children = [C for C in inner if not any(C.lines < D.lines for D in inner if D is not C)]
                facs.append((S, children))
            se = [S for S in F if S.kind == 'SE']
            assigns = []
            for chans in product(*[('u', 'v')] * len(se)):
                cc = {id(S): ch for S, ch in zip(se, chans)}
                parts = []
                for S, children in facs:
                    op = opof[id(S)]
                    if S.kind == 'SE':
                        channel = cc[id(S)]
                    elif op == 'U':
                        channel = 'a'
                    else:
                        channel = CHANNEL_OF_OP[op]
                    key = (tuple(sorted(S.verts)), channel,
                           tuple(sorted((tuple(sorted(C.verts)), cc[id(C)]) for C in children if C.kind == 'SE')),
                           tuple(sorted(tuple(sorted(C.verts)) for C in children)))
                    if key not in cache:
                        fac = Factor(g, S, children)
                        tab = tables[key] if tables is not None else coefficient_table(fac, channel, cc)
                        cache[key] = (fac, tab)
                    parts.append(key)
                assigns.append(parts)
            self.terms.append((sign, assigns))
        self.tables = cache

    def table_records(self):
        """The coefficient tables as plain lists (for storing):
        [[key, [[coef, j, asites, qsite, pairs], ...]], ...]."""
        return [[list(_listify(k)), [[c, j, list(a), q, [list(p) for p in pr]] for c, j, a, q, pr in tab]]
                for k, (_, tab) in self.tables.items()]

    @staticmethod
    def tables_from_records(records):
        """Inverse of table_records()."""
        out = {}
        for k, tab in records:
            out[_tuplify(k)] = [(c, j, tuple(a), q, tuple(tuple(p) for p in pr)) for c, j, a, q, pr in tab]
        return out

    def alphas(self, z):
        """Exact Schwinger parameters of every original line at point z."""
        al = {}
        for key, i in self.idx.items():
            zi = Fraction(float(z[i]))
            if key[0] == 'e' and i == 0:
                al[('e', key[1])] = zi / 2
            elif key[0] == 'e':
                al[('e', key[1])] = zi
            else:
                al[key] = zi
        return al

    def evaluate(self, z):
        """Return (I, K) at one point z (array of M doubles):
        I = subtracted integrand, K = sum over terms of |term|."""
        al = self.alphas(z)
        gf = {}
        vals = {}
        for key, (fac, table) in self.tables.items():
            fk = (key[0], key[3])
            if fk not in gf:
                gf[fk] = [x for x in fac.graph_functions(al)]
            U, Z, a, b, V = gf[fk]
            vec = {}
            for coef, j, asites, qsite, pairs in table:
                m = Fraction(coef)
                for s in asites:
                    m *= a[s]
                if qsite is not None:
                    m *= b[qsite]
                for (s1, s2) in pairs:
                    m *= Z[s1][s2]
                vec[j] = vec.get(j, Fraction(0)) + m
            vals[key] = ({j: v / (U * U) for j, v in vec.items()}, V)
        n = self.n
        total = Fraction(0)
        K = Fraction(0)
        for sign, assigns in self.terms:
            tv = Fraction(0)
            for parts in assigns:
                conv = {0: Fraction(1)}
                W = Fraction(0)
                for key in parts:
                    fv, V = vals[key]
                    W += V
                    new = {}
                    for j1, x1 in conv.items():
                        for j2, x2 in fv.items():
                            new[j1 + j2] = new.get(j1 + j2, Fraction(0)) + x1 * x2
                    conv = new
                for j, x in conv.items():
                    if x == 0:
                        continue
                    assert j < n, "divergent lambda integral with nonzero coefficient"
                    tv += x * (-1) ** j * Fraction(1, 2 ** j) * math.factorial(n - j - 1) \
                        / (-W) ** (n - j)
            total += sign * tv
            K += abs(tv)
        pref = Fraction(float(z[0])) * Fraction(1, 4 ** n) * (-1) ** n
        return float(pref * total), float(abs(pref) * K)

    def evaluate_many(self, z, dtype=np.float64):
        """(I, K) at many points z (array S x M) in floating point of the
        given dtype: the same steps as evaluate(), every exact rational
        operation replaced by the floating-point one, vectorised over the
        points.  Coefficients of lambda powers j >= n are left out (evaluate()
        asserts that they vanish exactly).  Not a parity reference: only the
        statistical pin of the 2-loop sum uses it (with exact re-evaluation
        of the points where two precisions disagree).  The rational
        coefficients enter rounded once to the dtype (_rational_in)."""
        z = np.asarray(z, dtype=dtype)
        al = {}
        for key, i in self.idx.items():
            zi = z[:, i]
            if key[0] == 'e' and i == 0:
                al[('e', key[1])] = zi / 2
            elif key[0] == 'e':
                al[('e', key[1])] = zi
            else:
                al[key] = zi
        zero = z[:, 0] * 0
        gf = {}
        vals = {}
        for key, (fac, table) in self.tables.items():
            fk = (key[0], key[3])
            if fk not in gf:
                gf[fk] = fac.graph_functions(al, batch=True)
            U, Z, a, b, V = gf[fk]
            vec = {}
            for coef, j, asites, qsite, pairs in table:
                m = zero + _rational_in(dtype, coef)
                for s_ in asites:
                    m = m * a[s_]
                if qsite is not None:
                    m = m * b[qsite]
                for (s1, s2) in pairs:
                    m = m * Z[s1][s2]
                vec[j] = vec.get(j, zero) + m
            vals[key] = ({j: v / (U * U) for j, v in vec.items()}, V)
        n = self.n
        total = zero
        K = zero
        for sign, assigns in self.terms:
            tv = zero
            for parts in assigns:
                conv = {0: zero + 1}
                W = zero
                for key in parts:
                    fv, V = vals[key]
                    W = W + V
                    new = {}
                    for j1, x1 in conv.items():
                        for j2, x2 in fv.items():
                            new[j1 + j2] = new.get(j1 + j2, zero) + x1 * x2
                    conv = new
                for j, x in conv.items():
                    if j >= n:
                        continue
                    tv = tv + x * (dtype((-1) ** j * math.factorial(n - j - 1)) / dtype(2 ** j)) / (-W) ** (n - j)
            total = total + sign * tv
            K = K + np.abs(tv)
        pref = z[:, 0] * (dtype((-1) ** n) / dtype(4 ** n))
        return pref * total, np.abs(pref) * K
