"""Oracle: the set of QED vertex graphs without lepton loops.

TEST INFRASTRUCTURE ONLY (see the package header).

A graph (Sec. I and its footnote; Sec. V, Table I) is one open electron
path carrying 2n+1 vertices v_0..v_{2n}; exactly one of them, v_s, holds the
external photon, every other vertex holds one end of one of n internal
photons.  Graphs that differ only by the direction of the electron arrows
(reversal of the path) are one graph.

Brute-force definition used here (no interval shortcuts):
  * enumerate every perfect matching of the 2n photon ends and every position
    of the external vertex;
  * keep a graph iff it is one-particle irreducible, tested directly: the
    graph stays connected after deleting any single internal line;
  * canonical word: vertex symbols along the path, -1 for the external
    vertex, photons numbered by first appearance; a graph and its mirror
    (reversed path) share the lexicographically smaller word.

Pinned by: the 5-loop count 3213 (Sec. I) and the nine class counts N_diag
of Table I; 1..4 loops by brute force on tiny inputs.
"""
from itertools import combinations


def perfect_matchings(items):
    """All perfect matchings of a list (recursive definition)."""
    if not items:
        yield []
        return
    a = items[0]
    for k in range(1, len(items)):
        b = items[k]
        rest = items[1:k] + items[k + 1:]
        for m in perfect_matchings(rest):
            yield [(a, b)] + m


def word_of(partner, s):
    """Path word: -1 at the external vertex, photons labelled by first appearance."""
    lab = {}
    w = []
    for v in range(len(partner)):
        if v == s:
            w.append(-1)
            continue
        key = min(v, partner[v])
        if key not in lab:
            lab[key] = len(lab)
        w.append(lab[key])
    return tuple(w)


def mirror(partner, s):
    N = len(partner)
    p2 = [None] * N
    for v in range(N):
        if v != s:
            p2[N - 1 - v] = N - 1 - partner[v]
    return p2, N - 1 - s


def lines_of(partner, s):
    """All internal lines as (kind, u, v): electron lines between consecutive
    path vertices, photon lines between partners."""
    N = len(partner)
    L = [('e', i - 1, i) for i in range(1, N)]
    for v in range(N):
        if v != s and v < partner[v]:
            L.append(('g', v, partner[v]))
    return L


def connected(nverts, edges):
    par = list(range(nverts))

    def f(x):
        while par[x] != x:
            par[x] = par[par[x]]
            x = par[x]
        return x
    for (_, a, b) in edges:
        par[f(a)] = f(b)
    return len({f(x) for x in range(nverts)}) == 1


def is_1pi(partner, s):
    L = lines_of(partner, s)
    N = len(partner)
    if not connected(N, L):
        return False
    for k in range(len(L)):
        if not connected(N, L[:k] + L[k + 1:]):
            return False
    return True


class Graph:
    """One vertex graph: ``partner[v]`` is the other end of the photon at v
    (None at the external vertex ``s``).  The stored orientation is the one
    whose word is the canonical (smaller) word."""

    def __init__(self, partner, s):
        self.partner = list(partner)
        self.s = s
        self.n = (len(partner) - 1) // 2
        self.word = word_of(partner, s)
        pm, sm = mirror(partner, s)
        self.mult = 1 if word_of(pm, sm) == self.word else 2

    @property
    def nverts(self):
        return 2 * self.n + 1

    def photons(self):
        """Photon lines (a, b), a < b, in order of first appearance."""
        return sorted({(min(v, self.partner[v]), max(v, self.partner[v]))
                       for v in range(self.nverts) if v != self.s})

    def klass(self):
        """Gauge-invariant class (k, m, m') of Sec. V: k photons cross the
        external vertex, m and m' lie wholly on either side, m >= m'."""
        left = right = cross = 0
        for a, b in self.photons():
            if b < self.s:
                left += 1
            elif a > self.s:
                right += 1
            else:
                cross += 1
        return (cross, max(left, right), min(left, right))

    def line_index(self):
        """Index of the M = 3n-1 Feynman parameters: 0 = the merged pair of
        electron lines touching the external vertex (the 3n -> 3n-1 trick
        of Sec. III.A), then the other electron lines along the path, then
        the photons in order of first appearance.  Returns a dict mapping
        ('e', i) (line v_{i-1} -> v_i) and ('g', a, b) to the index."""
        idx = {('e', self.s): 0, ('e', self.s + 1): 0}
        k = 1
        for i in range(1, 2 * self.n + 1):
            if i not in (self.s, self.s + 1):
                idx[('e', i)] = k
                k += 1
        for (a, b) in self.photons():
            idx[('g', a, b)] = k
            k += 1
        assert k == 3 * self.n - 1
        return idx


def enumerate_graphs(n):
    """Sorted list of canonical n-loop vertex graphs without lepton loops."""
    seen = {}
    for m in perfect_matchings(list(range(2 * n))):
        for s in range(0, 2 * n + 1):
            # insert the external vertex before photon end number s
            pos = lambda x: x if x < s else x + 1
            partner = [None] * (2 * n + 1)
            for a, b in m:
                partner[pos(a)] = pos(b)
                partner[pos(b)] = pos(a)
            if not is_1pi(partner, s):
                continue
            w = word_of(partner, s)
            pm, sm = mirror(partner, s)
            wm = word_of(pm, sm)
            if wm < w:
                partner, s, w = pm, sm, wm
            if w not in seen:
                seen[w] = Graph(partner, s)
    return [seen[w] for w in sorted(seen)]


def class_counts(graphs):
    out = {}
    for g in graphs:
        out[g.klass()] = out.get(g.klass(), 0) + 1
    return out
