"""Oracle: UV-divergent subgraphs, forests and the terms of R^new (Sec. II).

TEST INFRASTRUCTURE ONLY (see the package header).

Definitions followed (Sec. II):
  * a subgraph is given by a set of vertices and contains every line joining
    two of its vertices; it must be one-particle irreducible (the reading of
    "strongly connected": connected, at least one loop, and no internal line
    whose removal disconnects it);
  * UV-divergent types: self-energy (N_e = 2, N_gamma = 0) and vertexlike
    (N_e = 2, N_gamma = 1); external lines of a subgraph are the lines with
    exactly one end inside plus the graph's own external legs at its vertices;
  * two subgraphs overlap iff neither contains the other and their line sets
    intersect; a forest is a set of pairwise non-overlapping subgraphs;
  * F[G] = forests of UV-divergent subgraphs containing G;
    J[G] = vertexlike subgraphs containing the external-photon vertex;
  * R^new = sum over F in F[G] and G' in J[G] & F of
    (-1)^(|F|-1) prod_{G'' in F} M^{G'}_{G''} with
      M = A    if G'' = G'
          U    if G'' not in J[G] or G'' strictly inside G'
          L    if G'' in J[G], G' strictly inside G'', G'' != G
          L-U  if G'' = G and G' != G.

Subgraphs are found by brute force over ALL vertex subsets (not intervals).
Pinned by the worked example (Sec. II, Eq. eq_example_expression) and by the
brute-force enumeration itself.
"""
from itertools import combinations


class Subgraph:
    def __init__(self, verts, lines, kind, in_J, ext_photon):
        self.verts = frozenset(verts)
        self.lines = frozenset(lines)      # internal lines as ('e', i) / ('g', a, b)
        self.kind = kind                   # 'SE' or 'V'
        self.in_J = in_J
        self.ext_photon = ext_photon       # None (SE), 'ext' (graph's photon) or ('g', a, b)

    def __repr__(self):
        return "Sub(%s,%s%s)" % (sorted(self.verts), self.kind, ",J" if self.in_J else "")


def _connected_1pi(verts, lines):
    verts = list(verts)
    ix = {v: k for k, v in enumerate(verts)}

    def conn(ls):
        par = list(range(len(verts)))

        def f(x):
            while par[x] != x:
                x = par[x]
            return x
        for (a, b) in ls:
            par[f(ix[a])] = f(ix[b])
        return len({f(x) for x in range(len(verts))}) == 1
    if not conn(lines):
        return False
    for k in range(len(lines)):
        if not conn(lines[:k] + lines[k + 1:]):
            return False
    return True


def ends(line):
    if line[0] == 'e':
        return (line[1] - 1, line[1])
    return (line[1], line[2])


def all_lines(g):
    L = [('e', i) for i in range(1, 2 * g.n + 1)]
    L += [('g', a, b) for (a, b) in g.photons()]
    return L


def divergent_subgraphs(g):
    """Every UV-divergent subgraph of g (including g itself), brute force."""
    N = g.nverts
    L = all_lines(g)
    out = []
    for r in range(2, N + 1):
        for vs in combinations(range(N), r):
            V = set(vs)
            internal = [l for l in L if ends(l)[0] in V and ends(l)[1] in V]
            if len(internal) - len(V) + 1 < 1:
                continue
            if not _connected_1pi(V, [ends(l) for l in internal]):
                continue
            ne = ng = 0
            ext_ph = None
            for l in L:
                a, b = ends(l)
                if (a in V) != (b in V):
                    if l[0] == 'e':
                        ne += 1
                    else:
                        ng += 1
                        ext_ph = l
            if 0 in V:
                ne += 1
            if N - 1 in V:
                ne += 1
            if g.s in V:
                ng += 1
                ext_ph = 'ext'
            if ne != 2 or ng > 1:
                continue
            kind = 'SE' if ng == 0 else 'V'
            out.append(Subgraph(V, internal, kind, kind == 'V' and g.s in V,
                                ext_ph if ng == 1 else None))
    return out


def overlap(a, b):
    if a.lines <= b.lines or b.lines <= a.lines:
        return False
    return len(a.lines & b.lines) > 0


def forests_containing_G(g, subs):
    """All forests (pairwise non-overlapping sets) that contain G itself."""
    G = [s for s in subs if len(s.verts) == g.nverts][0]
    others = [s for s in subs if s is not G]
    out = []
    for r in range(len(others) + 1):
        for comb in combinations(others, r):
            if all(not overlap(a, b) for a, b in combinations(comb, 2)):
                out.append([G] + list(comb))
    return G, out


def operator_for(G, Gp, Gpp):
    """M^{G'}_{G''} of Sec. II."""
    if Gpp is Gp:
        return 'A'
    if (not Gpp.in_J) or (Gpp.lines < Gp.lines):
        return 'U'
    if Gpp.in_J and Gp.lines < Gpp.lines and Gpp is not G:
        return 'L'
    if Gpp is G and Gp is not G:
        return 'L-U'
    raise ValueError("no operator")


def terms(g):
    """List of (sign, [(subgraph, operator), ...]) for R^new of graph g."""
    subs = divergent_subgraphs(g)
    G, fs = forests_containing_G(g, subs)
    out = []
    for F in fs:
        for Gp in F:
            if not Gp.in_J:
                continue
            sign = (-1) ** (len(F) - 1)
            out.append((sign, [(S, operator_for(G, Gp, S)) for S in F]))
    return out
