// Graph set, UV-divergent subgraphs, forests and R^new terms (Secs. I, II).
//
// Enumeration here works on chord diagrams directly: an n-loop graph is an
// irreducible pairing of 2n photon ends along the electron path (no proper
// prefix is closed under the pairing, which is one-particle irreducibility)
// with the external vertex in one of the 2n-1 inner slots.  Subgraphs are
// path intervals whose every inner cut is crossed by an internal photon.
#include <algorithm>
#include <functional>
#include <map>
#include <set>

#include "ae_internal.h"

namespace ae {

static std::vector<int> make_word(const std::vector<int> &partner, int s) {
  std::vector<int> lab(partner.size(), -1), w;
  int next = 0;
  for (int v = 0; v < (int)partner.size(); ++v) {
    if (v == s) { w.push_back(-1); continue; }
    int key = std::min(v, partner[v]);
    if (lab[key] < 0) lab[key] = next++;
    w.push_back(lab[key]);
  }
  return w;
}

static void mirror_of(const std::vector<int> &p, int s, std::vector<int> &pm, int &sm) {
  int N = (int)p.size();
  pm.assign(N, -1);
  for (int v = 0; v < N; ++v)
    if (v != s) pm[N - 1 - v] = N - 1 - p[v];
  sm = N - 1 - s;
}

std::vector<Graph> enumerate_graphs(int n) {
  std::map<std::vector<int>, Graph> seen;
  int E = 2 * n;
  std::vector<int> pair(E, -1);
  // recursive generation of irreducible pairings of positions 0..2n-1
  std::function<void()> rec = [&]() {
    int first = -1;
    for (int i = 0; i < E; ++i)
      if (pair[i] < 0) { first = i; break; }
    if (first < 0) {
      // irreducibility: no proper prefix closed under the pairing
      for (int k = 1; k < E; ++k) {
        bool closed = true;
        for (int i = 0; i < k && closed; ++i)
          if (pair[i] >= k) closed = false;
        if (closed) return;
      }
      for (int s = 1; s <= E - 1; ++s) {
        std::vector<int> partner(E + 1, -1);
        auto pos = [&](int x) { return x < s ? x : x + 1; };
        for (int i = 0; i < E; ++i) partner[pos(i)] = pos(pair[i]);
        std::vector<int> w = make_word(partner, s), pm;
        int sm;
        mirror_of(partner, s, pm, sm);
        std::vector<int> wm = make_word(pm, sm);
        Graph g;
        g.n = n;
        if (wm < w) { g.partner = pm; g.s = sm; g.word = wm; }
        else { g.partner = partner; g.s = s; g.word = w; }
        g.mult = (w == wm) ? 1 : 2;
        if (!seen.count(g.word)) seen.emplace(g.word, g);
      }
      return;
    }
    for (int j = first + 1; j < E; ++j) {
      if (pair[j] >= 0) continue;
      pair[first] = j; pair[j] = first;
      rec();
      pair[first] = -1; pair[j] = -1;
    }
  };
  rec();
  std::vector<Graph> out;
  for (auto &kv : seen) {
    Graph g = kv.second;
    int left = 0, right = 0, cross = 0;
    for (int v = 0; v < g.nverts(); ++v) {
      if (v == g.s || v > g.partner[v]) continue;
      int a = v, b = g.partner[v];
      if (b < g.s) ++left; else if (a > g.s) ++right; else ++cross;
    }
    g.klass[0] = cross; g.klass[1] = std::max(left, right); g.klass[2] = std::min(left, right);
    out.push_back(g);
  }
  return out;   // std::map keeps lexicographic word order
}

std::vector<Line> photon_lines(const Graph &g) {
  std::vector<Line> ph;
  for (int v = 0; v < g.nverts(); ++v)
    if (v != g.s && v < g.partner[v]) ph.push_back(Line{true, v, g.partner[v]});
  std::sort(ph.begin(), ph.end());
  return ph;
}

int line_param(const Graph &g, const Line &l) {
  if (!l.photon) {
    int i = l.b;   // e_i
    if (i == g.s || i == g.s + 1) return 0;
    int k = 1;
    for (int j = 1; j < i; ++j)
      if (j != g.s && j != g.s + 1) ++k;
    return k;
  }
  std::vector<Line> ph = photon_lines(g);
  for (size_t k = 0; k < ph.size(); ++k)
    if (ph[k] == l) return 2 * g.n - 1 + (int)k;
  return -1;
}

std::vector<Sub> divergent_subgraphs(const Graph &g) {
  std::vector<Sub> out;
  int N = g.nverts();
  for (int lo = 0; lo < N; ++lo)
    for (int hi = lo + 1; hi < N; ++hi) {
      int ext = 0, extv = -1, internal = 0;
      for (int v = lo; v <= hi; ++v) {
        if (v == g.s) { ++ext; extv = v; continue; }
        int p = g.partner[v];
        if (p < lo || p > hi) { ++ext; extv = v; }
        else if (p > v) ++internal;
      }
      if (internal == 0 || ext > 1) continue;
      // one-particle irreducible: every inner cut crossed by an internal photon
      bool ok = true;
      for (int cut = lo; cut < hi && ok; ++cut) {
        bool crossed = false;
        for (int v = lo; v <= cut && !crossed; ++v) {
          if (v == g.s) continue;
          int p = g.partner[v];
          if (p > cut && p <= hi) crossed = true;
        }
        ok = crossed;
      }
      if (!ok) continue;
      Sub s;
      s.lo = lo; s.hi = hi; s.se = (ext == 0);
      s.inJ = (!s.se) && (lo <= g.s && g.s <= hi);
      s.ext_photon_vertex = s.se ? -1 : extv;
      out.push_back(s);
    }
  // put G first
  std::stable_sort(out.begin(), out.end(), [&](const Sub &a, const Sub &b) {
    return (a.hi - a.lo) > (b.hi - b.lo);
  });
  return out;
}

static bool nested(const Sub &a, const Sub &b) {   // a inside b (lines)
  return b.lo <= a.lo && a.hi <= b.hi;
}
static bool compatible(const Sub &a, const Sub &b) {
  return nested(a, b) || nested(b, a) || a.hi < b.lo || b.hi < a.lo;
}

std::vector<Term> rnew_terms(const Graph &g, const std::vector<Sub> &subs) {
  std::vector<Term> out;
  int K = (int)subs.size();   // subs[0] is G
  for (uint32_t m = 0; m < (1u << (K - 1)); ++m) {
    std::vector<int> F = {0};
    for (int i = 1; i < K; ++i)
      if (m >> (i - 1) & 1) F.push_back(i);
    bool ok = true;
    for (size_t i = 0; i < F.size() && ok; ++i)
      for (size_t j = i + 1; j < F.size() && ok; ++j)
        ok = compatible(subs[F[i]], subs[F[j]]);
    if (!ok) continue;
    for (int gp : F) {
      if (!subs[gp].inJ) continue;
      Term t;
      t.sign = (F.size() % 2 == 1) ? 1 : -1;
      t.elems = F;
      for (int e : F) {
        int op;
        const Sub &S = subs[e];
        bool strictly_in_gp = nested(S, subs[gp]) && e != gp;
        bool gp_strictly_in = nested(subs[gp], S) && e != gp;
        if (e == gp) op = OP_A;
        else if (!S.inJ || strictly_in_gp) op = OP_U;
        else if (e == 0) op = OP_LmU;
        else if (gp_strictly_in) op = OP_L;
        else op = -1;
        t.ops.push_back(op);
      }
      out.push_back(t);
    }
  }
  return out;
}

}  // namespace ae

// The canonical list of one loop order without compiling anything: per graph
// its class (k, m, m') of Sec. V, Table I, and its multiplicity.
extern "C" int ae_graph_classes(int loops, int *klass, int *mult, int cap, int *n_out) {
  if (loops < 1 || loops > 5 || !n_out) return -1;
  try {
    const std::vector<ae::Graph> gs = ae::enumerate_graphs(loops);
    *n_out = (int)gs.size();
    if (!klass && !mult) return 0;
    if (cap < (int)gs.size()) return -1;
    for (size_t i = 0; i < gs.size(); ++i) {
      if (klass)
        for (int k = 0; k < 3; ++k) klass[3 * i + k] = gs[i].klass[k];
      if (mult) mult[i] = gs[i].mult;
    }
  } catch (...) {
    return -1;
  }
  return 0;
}
