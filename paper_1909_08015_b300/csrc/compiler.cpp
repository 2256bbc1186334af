// Integrand compiler: from a graph to a straight-line FP64 tape that
// evaluates the subtracted Feynman-parametric integrand I(z), the sum of
// the absolute values of its forest terms K(z) and a certified bound E(z)
// of the rounding error of I (Sec. II, Eq. eq_feyn_integral; Sec. IV.A on
// round-off control and on splitting integrand code).
//
// Construction (the paper defers the formulas to earlier work; this is the
// library's reading, stated once here):
//  * each term (F, G') of R^new factorises into one factor per element S of
//    F, the reduced graph S/children(S).  A collapsed self-energy child leaves
//    u(m^2) or v(m^2) pslash, a collapsed vertex child a gamma^nu; the factor
//    of S is projected by its own operator: U (u, v or a), L (a + b + c),
//    L - U (b + c) or A (F2(0), the magnetic form factor at q = 0);
//  * graph functions of a factor with loop matrix A (photon cycles closed
//    along the electron path): U = det A, Bbar = eta adj(A) eta^T,
//    flow numerators U*Q_l and U*V = -B^T adj(A) B, all kept as exact
//    polynomials in z so that every cancellation happens symbolically;
//  * Wick expansion of the electron numerators: <kappa_l kappa_l'> =
//    (i/2) Z_ll' g with Z = Bbar/U, external parts a_l P + b_l q;
//  * Dirac traces with contracted indices by the 4-dimensional contraction
//    identities gamma^n X gamma_n (Chisholm), exact integers;
//  * joint lambda integral over all lines: weight (-1)^j 2^-j Gamma(n-j)
//    (-W)^-(n-j), W = sum of the factors' V, overall z_e 4^-n (-1)^n;
//  * the two electron lines at the external vertex are one parameter z_e,
//    each line carrying z_e/2 (the integrand is linear in the split).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <set>
#include <climits>
#include <numeric>
#include <stdexcept>
#include <unordered_map>

#include "ae_internal.h"

namespace ae {

// ================================================================ polys ==
// Sparse polynomial in z_0..z_{M-1} with exact dyadic coefficients.
struct Poly {
  std::map<uint64_t, double> t;   // exponent key (4 bits per variable) -> coef
  static Poly var(int i, double c = 1.0) { Poly p; p.t[1ull << (4 * i)] = c; return p; }
  static Poly cst(double c) { Poly p; if (c != 0) p.t[0] = c; return p; }
  void clean() { for (auto it = t.begin(); it != t.end();) { if (it->second == 0) it = t.erase(it); else ++it; } }
};
static Poly operator+(const Poly &a, const Poly &b) {
  Poly r = a;
  for (auto &kv : b.t) r.t[kv.first] += kv.second;
  r.clean();
  return r;
}
static Poly operator*(double s, const Poly &a) {
  Poly r;
  if (s == 0) return r;
  for (auto &kv : a.t) r.t[kv.first] = s * kv.second;
  return r;
}
static Poly operator-(const Poly &a, const Poly &b) { return a + (-1.0) * b; }
static Poly operator*(const Poly &a, const Poly &b) {
  Poly r;
  for (auto &x : a.t)
    for (auto &y : b.t) r.t[x.first + y.first] += x.second * y.second;
  r.clean();
  return r;
}

static Poly det_poly(const std::vector<std::vector<Poly>> &A) {
  int n = (int)A.size();
  if (n == 0) return Poly::cst(1.0);
  if (n == 1) return A[0][0];
  Poly r;
  for (int c = 0; c < n; ++c) {
    if (A[0][c].t.empty()) continue;
    std::vector<std::vector<Poly>> m;
    for (int i = 1; i < n; ++i) {
      std::vector<Poly> row;
      for (int j = 0; j < n; ++j) if (j != c) row.push_back(A[i][j]);
      m.push_back(row);
    }
    Poly t = A[0][c] * det_poly(m);
    r = (c % 2 == 0) ? r + t : r - t;
  }
  return r;
}

// =============================================================== traces ==
// A gamma string: element -1 = Pslash (P^2 = 1), element >= 0 = gamma^label;
// every label occurs twice and is contracted.  Mass terms are omitted (m = 1).
using GStr = std::vector<int>;

struct TraceMemo {
  std::unordered_map<std::string, double> memo;
};

static std::string key_of(const GStr &s) {
  // relabel by first appearance so equal strings share the memo entry
  int lab_from[64], lab_to[64], nl = 0;
  std::string k;
  k.reserve(s.size());
  for (int e : s) {
    if (e < 0) { k.push_back('P'); continue; }
    int id = -1;
    for (int t = 0; t < nl; ++t)
      if (lab_from[t] == e) { id = lab_to[t]; break; }
    if (id < 0) { lab_from[nl] = e; lab_to[nl] = nl; id = nl; ++nl; }
    k.push_back((char)('a' + id));
  }
  return k;
}

static void simplify(GStr &s) {
  // cancel adjacent Pslash Pslash (P^2 = 1), cyclically
  bool changed = true;
  while (changed && s.size() >= 2) {
    changed = false;
    for (size_t i = 0; i + 1 < s.size(); ++i)
      if (s[i] < 0 && s[i + 1] < 0) { s.erase(s.begin() + i, s.begin() + i + 2); changed = true; break; }
    if (!changed && s.size() >= 2 && s.front() < 0 && s.back() < 0) {
      s.pop_back(); s.erase(s.begin()); changed = true;
    }
  }
}

// gamma^n a_1..a_k gamma_n as a list of (coefficient, string); a dot product
// a.b is returned as the marker pair {-2, -2} meaning "contract a with b".
static void contract(const GStr &a, std::vector<std::pair<double, GStr>> &out, double c) {
  size_t k = a.size();
  if (k == 0) { out.push_back({4.0 * c, {}}); return; }
  if (k == 1) { out.push_back({-2.0 * c, a}); return; }
  if (k == 2) { out.push_back({4.0 * c, {-2, a[0], a[1]}}); return; }
  if (k == 3) { out.push_back({-2.0 * c, {a[2], a[1], a[0]}}); return; }
  if (k == 4) {
    out.push_back({2.0 * c, {a[3], a[0], a[1], a[2]}});
    out.push_back({2.0 * c, {a[2], a[1], a[0], a[3]}});
    return;
  }
  // gamma^n a1 X gamma_n = 2 X a1 - a1 gamma^n X gamma_n
  GStr rot(a.begin() + 1, a.end());
  rot.push_back(a[0]);
  out.push_back({2.0 * c, rot});
  std::vector<std::pair<double, GStr>> sub;
  contract(GStr(a.begin() + 1, a.end()), sub, -c);
  for (auto &p : sub) {
    GStr s = {a[0]};
    if (!p.second.empty() && p.second[0] == -2) {
      // keep the dot marker first, then a1, then the dotted pair
      GStr t = {-2, p.second[1], p.second[2], a[0]};
      t.insert(t.end(), p.second.begin() + 3, p.second.end());
      out.push_back({p.first, t});
    } else {
      s.insert(s.end(), p.second.begin(), p.second.end());
      out.push_back({p.first, s});
    }
  }
}

static double trace_rec(GStr s, TraceMemo &tm) {
  simplify(s);
  if (s.empty()) return 4.0;
  if (s.size() % 2) return 0.0;
  std::string key = key_of(s);
  auto it = tm.memo.find(key);
  if (it != tm.memo.end()) return it->second;
  // pick the label whose two ends are closest (cyclic distance)
  int n = (int)s.size();
  int best = -1, bi = -1, bj = -1;
  for (int i = 0; i < n; ++i) {
    if (s[i] < 0) continue;
    for (int j = i + 1; j < n; ++j)
      if (s[j] == s[i]) {
        int d1 = j - i - 1, d2 = n - (j - i) - 1;
        int d = std::min(d1, d2);
        if (best < 0 || d < best) {
          best = d;
          if (d1 <= d2) { bi = i; bj = j; } else { bi = j; bj = i; }
        }
      }
  }
  double res;
  if (best < 0) {
    res = 4.0;   // only Pslash left, even count: (P^2)^k = 1
  } else {
    GStr inner, rest;
    for (int t = 1; t < n; ++t) {
      int p = (bi + t) % n;
      if (p == bj) {
        for (int u = 1; u < n - t; ++u) rest.push_back(s[(bj + u) % n]);
        break;
      }
      inner.push_back(s[p]);
    }
    std::vector<std::pair<double, GStr>> ex;
    contract(inner, ex, 1.0);
    res = 0.0;
    for (auto &pr : ex) {
      GStr ns;
      double c = pr.first;
      GStr body = pr.second;
      GStr r2 = rest;
      // resolve dot markers {-2, x, y, tail...}: contract the pair (x, y)
      if (!body.empty() && body[0] == -2) {
        int x = body[1], y = body[2];
        GStr tail(body.begin() + 3, body.end());
        body = tail;
        auto replace_other = [&](int lab, int with) {
          for (auto &e : body) if (e == lab) { e = with; return; }
          for (auto &e : r2) if (e == lab) { e = with; return; }
        };
        if (x < 0 && y < 0) { /* P.P = 1 */ }
        else if (x < 0) replace_other(y, -1);
        else if (y < 0) replace_other(x, -1);
        else if (x == y) c *= 4.0;
        else replace_other(y, x);
      }
      ns = body;
      ns.insert(ns.end(), r2.begin(), r2.end());
      if (c != 0) res += c * trace_rec(ns, tm);
    }
  }
  tm.memo.emplace(key, res);
  return res;
}

// ============================================================== factors ==
struct Factor {
  const Graph *g = nullptr;
  int lo = 0, hi = 0;
  bool se = false;
  std::vector<int> child_lo, child_hi;     // collapsed children
  std::vector<char> child_se;
  // nodes in path order: vertex v (>= 0) or child ~c (< 0)
  std::vector<int> nodes;
  std::vector<int> elines;                 // e_i index of the line into node k+1
  std::vector<Line> photons;
  std::vector<std::pair<int, int>> spans;  // node span of each photon
  int ext_node = -1;
  std::vector<int> node_label;             // -2 none(SE child), -1 mu, >= 0 photon index
};

static Factor make_factor(const Graph &g, const std::vector<Sub> &subs, int S,
                          const std::vector<int> &children) {
  Factor f;
  f.g = &g;
  f.lo = subs[S].lo; f.hi = subs[S].hi; f.se = subs[S].se;
  std::vector<int> ch = children;
  std::sort(ch.begin(), ch.end(), [&](int a, int b) { return subs[a].lo < subs[b].lo; });
  for (int c : ch) {
    f.child_lo.push_back(subs[c].lo); f.child_hi.push_back(subs[c].hi);
    f.child_se.push_back(subs[c].se);
  }
  std::vector<int> node_of(g.nverts(), -1);
  for (int v = f.lo; v <= f.hi;) {
    int ci = -1;
    for (size_t c = 0; c < ch.size(); ++c)
      if (f.child_lo[c] == v) ci = (int)c;
    if (ci >= 0) {
      for (int u = f.child_lo[ci]; u <= f.child_hi[ci]; ++u) node_of[u] = (int)f.nodes.size();
      f.nodes.push_back(~ci);
      v = f.child_hi[ci] + 1;
    } else {
      node_of[v] = (int)f.nodes.size();
      f.nodes.push_back(v);
      ++v;
    }
  }
  for (size_t k = 0; k + 1 < f.nodes.size(); ++k) {
    int nd = f.nodes[k + 1];
    int first = nd >= 0 ? nd : f.child_lo[~nd];
    f.elines.push_back(first);   // e_first joins v_{first-1} -> v_first
  }
  auto inside_child = [&](int v) {
    for (size_t c = 0; c < ch.size(); ++c)
      if (f.child_lo[c] <= v && v <= f.child_hi[c]) return true;
    return false;
  };
  for (const Line &l : photon_lines(g)) {
    if (l.a < f.lo || l.b > f.hi) continue;
    bool inner = false;
    for (size_t c = 0; c < ch.size(); ++c)
      if (f.child_lo[c] <= l.a && l.b <= f.child_hi[c]) inner = true;
    if (inner) continue;
    f.photons.push_back(l);
    f.spans.push_back({node_of[l.a], node_of[l.b]});
  }
  (void)inside_child;
  f.node_label.assign(f.nodes.size(), -2);
  for (size_t k = 0; k < f.nodes.size(); ++k) {
    int nd = f.nodes[k];
    int v;   // vertex whose photon the node carries
    if (nd >= 0) v = nd;
    else {
      int c = ~nd;
      if (f.child_se[c]) { f.node_label[k] = -2; continue; }
      v = subs[ch[c]].ext_photon_vertex;
    }
    if (v == g.s) { f.node_label[k] = -1; continue; }
    int a = std::min(v, g.partner[v]), b = std::max(v, g.partner[v]);
    int idx = -1;
    for (size_t p = 0; p < f.photons.size(); ++p)
      if (f.photons[p].a == a && f.photons[p].b == b) idx = (int)p;
    f.node_label[k] = idx >= 0 ? idx : -1;
  }
  for (size_t k = 0; k < f.nodes.size(); ++k)
    if (f.node_label[k] == -1) f.ext_node = (int)k;
  if ((f.ext_node < 0) != f.se) throw std::runtime_error("factor external photon mismatch");
  return f;
}

// ======================================================= Dirac expansion ==
enum Chan { CH_U = 0, CH_V = 1, CH_A = 2, CH_ABC = 3, CH_BC = 4, CH_F2 = 5 };

struct Mono {          // one monomial of a factor numerator
  long long num;       // exact coefficient = num / den
  long long den;
  int j;
  std::vector<int> a_sites;   // eline indices (a_k factors)
  int q_site;                 // eline index of the b_k factor or -1
  std::vector<std::pair<int, int>> pairs;   // Z_kk' factors
};

// Chain sites in matrix order (outgoing end first).
struct Site { int kind; int node; int eline; };  // kind 0 node, 1 prop, 2 insertion

static std::vector<Site> chain_sites(const Factor &f, const std::vector<int> &child_chan) {
  std::vector<Site> out;
  for (int k = (int)f.nodes.size() - 1; k >= 0; --k) {
    int nd = f.nodes[k];
    if (nd < 0 && f.child_se[~nd] && child_chan[~nd] == CH_V)
      out.push_back({2, k, k - 1});
    else
      out.push_back({0, k, -1});
    if (k > 0) out.push_back({1, k, k - 1});
  }
  return out;
}

static long long gcdll(long long a, long long b) { a = std::llabs(a); b = std::llabs(b); while (b) { long long t = a % b; a = b; b = t; } return a; }

static std::vector<Mono> expand_factor(const Factor &f, int chan, const std::vector<int> &child_chan,
                                       TraceMemo &tm) {
  std::vector<Site> seq = chain_sites(f, child_chan);
  std::vector<int> spos;
  for (size_t p = 0; p < seq.size(); ++p)
    if (seq[p].kind != 0) spos.push_back((int)p);
  int ns = (int)spos.size();
  const int MU = 1000, BETA = 1001;   // reserved labels
  std::vector<Mono> out;
  bool F2 = chan == CH_F2;
  // element codes for a configuration: -10 mass, -1 P, label >= 0
  std::vector<int> el(seq.size(), -10);
  auto build = [&](int mu_as, const std::vector<int> &elv) {
    GStr s;
    for (size_t p = 0; p < seq.size(); ++p) {
      const Site &st = seq[p];
      if (st.kind == 0) {
        int lab = f.node_label[st.node];
        if (lab == -2) continue;          // u insertion: identity
        if (lab == -1) s.push_back(mu_as);
        else s.push_back(100 + lab);
      } else {
        int e = elv[p];
        if (e == -10) continue;           // mass term
        s.push_back(e);
      }
    }
    return s;
  };
  auto cat = [](std::initializer_list<GStr> parts) {
    GStr r;
    for (auto &p : parts) r.insert(r.end(), p.begin(), p.end());
    return r;
  };
  // projection value times 24 (all projections have denominators | 24)
  auto project24 = [&](const std::vector<int> &elv, int qpos) -> long long {
    double v = 0;
    if (chan == CH_U) v = 6.0 * trace_rec(build(MU, elv), tm);
    else if (chan == CH_V) v = 6.0 * trace_rec(cat({{-1}, build(MU, elv)}), tm);
    else if (chan == CH_A || chan == CH_ABC || chan == CH_BC) {
      double E1 = trace_rec(cat({build(MU, elv), {MU}}), tm);
      double E2 = trace_rec(cat({build(-1, elv), {-1}}), tm);
      double E3 = trace_rec(build(-1, elv), tm);
      if (chan == CH_A) v = 2.0 * (E1 - E2);
      else if (chan == CH_ABC) v = 6.0 * (E2 + E3);
      else v = 6.0 * E3 + 2.0 * (4.0 * E2 - E1);
    } else {
      // F2 = -(1/24) [tau_g - tau_P]; Lambda = Pslash + 1 expands into two
      // strings; Y^a = gamma_mu gamma^a - gamma^a gamma_mu + 3 gamma_mu P gamma^a
      // + 3 g_mu^a.  Returned value is 24 * F2 = -(tau_g - tau_P).
      double tot = 0;
      for (int part = 0; part < 2; ++part) {
        double sgn = part == 0 ? 1.0 : -1.0;
        int qb = part == 0 ? BETA : -1;
        std::vector<std::pair<double, GStr>> Ys;
        if (part == 0) Ys = {{1.0, {MU, BETA}}, {-1.0, {BETA, MU}}, {3.0, {MU, -1, BETA}}};
        else Ys = {{1.0, {MU, -1}}, {-1.0, {-1, MU}}, {3.0, {MU, -1, -1}}};
        int qmu = part == 0 ? MU : -1;
        int murep = part == 0 ? MU : -1;
        auto lam_tr = [&](const GStr &pre, const GStr &mid, const GStr &post) {
          // Tr[(P+1) pre ... ] helpers are expanded by the caller
          return trace_rec(cat({pre, mid, post}), tm);
        };
        (void)lam_tr;
        if (qpos >= 0) {
          std::vector<int> e2 = elv;
          e2[qpos] = qb;
          GStr ch = build(MU, e2);
          for (auto &Y : Ys)
            for (int l1 = 0; l1 < 2; ++l1)
              for (int l2 = 0; l2 < 2; ++l2) {
                GStr s = cat({l1 ? GStr{-1} : GStr{}, ch, l2 ? GStr{-1} : GStr{}, Y.second});
                tot += sgn * Y.first * trace_rec(s, tm);
              }
          e2[qpos] = qmu;
          GStr ch2 = build(murep, e2);
          for (int l1 = 0; l1 < 2; ++l1)
            for (int l2 = 0; l2 < 2; ++l2) {
              GStr s = cat({l1 ? GStr{-1} : GStr{}, ch2, l2 ? GStr{-1} : GStr{}});
              tot += sgn * 3.0 * trace_rec(s, tm);
            }
        } else {
          GStr ch = build(MU, elv);
          for (auto &Y : Ys)
            for (int l = 0; l < 2; ++l) {
              GStr L = l ? GStr{-1} : GStr{};
              tot += sgn * Y.first * 0.5 * trace_rec(cat({{qb}, ch, L, Y.second}), tm);
              tot -= sgn * Y.first * 0.5 * trace_rec(cat({L, ch, {qb}, Y.second}), tm);
            }
          GStr ch2 = build(murep, elv);
          for (int l = 0; l < 2; ++l) {
            GStr L = l ? GStr{-1} : GStr{};
            tot += sgn * 3.0 * 0.5 * trace_rec(cat({{qmu}, ch2, L}), tm);
            tot -= sgn * 3.0 * 0.5 * trace_rec(cat({L, ch2, {qmu}}), tm);
          }
        }
      }
      v = -tot;
    }
    double r = std::nearbyint(v);
    if (std::fabs(r - v) > 1e-6) throw std::runtime_error("non-integer projection");
    return (long long)r;
  };
  // enumerate kappa subsets and their pairings, then modes of the rest
  std::vector<int> K;
  std::function<void(int)> choose;
  std::vector<std::pair<int, int>> pairs;
  std::function<void(std::vector<int>)> match = [&](std::vector<int> rem) {
    if (!rem.empty()) {
      int a = rem[0];
      for (size_t k = 1; k < rem.size(); ++k) {
        std::vector<int> r2;
        for (size_t t = 1; t < rem.size(); ++t) if (t != k) r2.push_back(rem[t]);
        pairs.push_back({a, rem[k]});
        match(r2);
        pairs.pop_back();
      }
      return;
    }
    std::vector<int> rest;
    for (int p : spos)
      if (std::find(K.begin(), K.end(), p) == K.end()) rest.push_back(p);
    std::vector<int> base(seq.size(), -10);
    for (size_t t = 0; t < pairs.size(); ++t) {
      base[pairs[t].first] = (int)t;
      base[pairs[t].second] = (int)t;
    }
    int nr = (int)rest.size();
    std::vector<int> qopts = {-1};
    if (F2) for (int p : rest) qopts.push_back(p);
    for (int qpos : qopts) {
      // modes: prop -> mass or P; insertion -> P only
      std::vector<int> free;
      for (int p : rest) if (p != qpos) free.push_back(p);
      int nf = (int)free.size();
      for (uint32_t m = 0; m < (1u << nf); ++m) {
        bool ok = true;
        std::vector<int> elv = base;
        std::vector<int> asites;
        for (int t = 0; t < nf; ++t) {
          int p = free[t];
          bool isP = (m >> t & 1) != 0;
          if (!isP && seq[p].kind == 2) { ok = false; break; }
          elv[p] = isP ? -1 : -10;
          if (isP) asites.push_back(seq[p].eline);
        }
        if (!ok) continue;
        if (qpos >= 0) elv[qpos] = 0;   // placeholder, replaced in project24
        long long c24 = project24(elv, qpos);
        if (c24 == 0) continue;
        Mono mo;
        long long gg = gcdll(c24, 24);
        mo.num = c24 / gg; mo.den = 24 / gg;
        mo.j = (int)pairs.size();
        std::sort(asites.begin(), asites.end());
        mo.a_sites = asites;
        mo.q_site = qpos >= 0 ? seq[qpos].eline : -1;
        for (auto &pr : pairs) {
          int x = seq[pr.first].eline, y = seq[pr.second].eline;
          mo.pairs.push_back({std::min(x, y), std::max(x, y)});
        }
        std::sort(mo.pairs.begin(), mo.pairs.end());
        out.push_back(mo);
      }
    }
    (void)nr;
  };
  choose = [&](int idx) {
    if (idx == ns) {
      if (K.size() % 2 == 0) match(K);
      return;
    }
    choose(idx + 1);
    K.push_back(spos[idx]);
    choose(idx + 1);
    K.pop_back();
  };
  choose(0);
  return out;
}

// ========================================================== tape builder ==
struct Builder {
  // value ids; b may be a constant index (T_FMAC, T_MULC, T_CONST, or T_G
  // with G_BK), c a value id or (T_G with G_CK) a constant index
  struct SIns { uint8_t op; int d, a, b; int c = -1; uint8_t fl = 0; };
  std::vector<SIns> prog;
  std::vector<double> khi, klo;
  std::map<std::pair<double, double>, int> kidx;
  int nvals = 0;
  int M = 0;
  std::map<std::tuple<int, int, int>, int> cse;
  double flops = 0, flops_bound = 0;
  bool horner = true;   // Horner trees for sums of monomials (else monomial chains)
  bool share = true;    // reuse identical Horner subtrees emitted recently
  int share_window = 64;   // instructions (set per loop order in compile_integrand)
  std::map<std::vector<long long>, std::pair<int, size_t>> hcse;   // value id, program size after it

  int newval() { return nvals++; }
  int konst(double hi, double lo = 0.0) {
    auto key = std::make_pair(hi, lo);
    auto it = kidx.find(key);
    if (it != kidx.end()) return it->second;
    int k = (int)khi.size();
    khi.push_back(hi); klo.push_back(lo);
    kidx[key] = k;
    return k;
  }
  int konst_rat(long long num, long long den) {
    long double q = (long double)num / (long double)den;
    double hi = (double)q;
    double lo = (double)(q - (long double)hi);
    return konst(hi, lo);
  }
  int bin(uint8_t op, int a, int b) {
    if (op == T_MUL && a > b) std::swap(a, b);
    if (op == T_ADD && a > b) std::swap(a, b);
    auto key = std::make_tuple((int)op, a, b);
    auto it = cse.find(key);
    if (it != cse.end()) return it->second;
    int d = newval();
    prog.push_back({op, d, a, b});
    flops += 1;
    cse[key] = d;
    return d;
  }
  int zero() { int d = newval(); prog.push_back({T_ZERO, d, -1, -1}); return d; }
  int cval(int k) { int d = newval(); prog.push_back({T_CONST, d, -1, k}); return d; }
  void fmac(int acc, int a, int k) { prog.push_back({T_FMAC, acc, a, k}); flops += 2; }
  void fma(int acc, int a, int b) { prog.push_back({T_FMA, acc, a, b}); flops += 2; }
  int mulc(int a, int k) { int d = newval(); prog.push_back({T_MULC, d, a, k}); flops += 1; return d; }
  void addabs(int acc, int a) { prog.push_back({T_ADDABS, acc, a, -1}); flops += 1; }
  void clear_cse() { cse.clear(); hcse.clear(); }
};

// Products of sorted variable lists evaluated in lexicographic order: the
// prefix shared with the previous monomial is reused, so at most (degree)
// partial products are live at any time.
struct ProdStack {
  std::vector<int> vars, vals;
};
static int stack_product(Builder &B, ProdStack &ps, const std::vector<int> &v) {
  size_t common = 0;
  while (common < ps.vars.size() && common < v.size() && ps.vars[common] == v[common]) ++common;
  ps.vars.resize(common);
  ps.vals.resize(common);
  for (size_t i = common; i < v.size(); ++i) {
    int val;
    if (i == 0) val = v[0];
    else {
      val = B.newval();
      B.prog.push_back({T_MUL, val, ps.vals[i - 1], v[i]});
      B.flops += 1;
    }
    ps.vars.push_back(v[i]);
    ps.vals.push_back(val);
  }
  return ps.vals.back();
}

// ------------------------------------------------------------ Horner --
// A sum of monomials  sum_m K[k_m] prod(vars_m)  evaluated by greedy
// multivariate Horner factorisation: at every node the variable that occurs
// in most of the node's monomials is factored out,
//     q = x * q_x + q_rest,
// recursively, so that every edge of the resulting tree costs one fused
// multiply-add and no monomial is multiplied out.  The running sums are
// ordinary values (SSA); the slot allocator gives each update the slot of the
// sum it replaces.
struct HMono { std::vector<int> v; int k; };   // sorted variable multiset, constant index

// Returns the value id of the node's polynomial  K[coef] + sum over ms.
static int horner_node(Builder &B, std::vector<HMono> &ms, int coef, int zero_k) {
  // ms: monomials of this node with at least one variable each; coef: the
  // node's own constant index or -1.  A polynomial already emitted since the
  // last clear_cse (same monomials, same coefficients) is reused.
  std::vector<long long> key;
  if (B.share && ms.size() >= 2) {
    std::vector<std::pair<std::vector<int>, int>> srt;
    srt.reserve(ms.size());
    for (auto &m : ms) srt.push_back({m.v, m.k});
    std::sort(srt.begin(), srt.end());
    key.push_back(coef);
    for (auto &p : srt) {
      key.push_back(-1 - (long long)p.first.size());
      for (int x : p.first) key.push_back(x);
      key.push_back(p.second);
    }
    auto it = B.hcse.find(key);
    // only recent subtrees: reusing one from far back would keep its value
    // live (a slot occupied) across everything in between
    if (it != B.hcse.end() && B.prog.size() - it->second.second <= (size_t)B.share_window) return it->second.first;
  }
  int acc = -1;
  std::vector<HMono> rest;
  rest.swap(ms);
  while (!rest.empty()) {
    std::map<int, int> cnt;
    for (auto &m : rest) {
      int prev = -1;
      for (int x : m.v) if (x != prev) { cnt[x]++; prev = x; }
    }
    int best = -1, bc = -1;
    for (auto &kv : cnt) if (kv.second > bc) { bc = kv.second; best = kv.first; }
    std::vector<HMono> grp, oth;
    int leaf_k = -1;
    for (auto &m : rest) {
      auto it = std::find(m.v.begin(), m.v.end(), best);
      if (it == m.v.end()) { oth.push_back(std::move(m)); continue; }
      m.v.erase(it);
      if (m.v.empty()) leaf_k = m.k;
      else grp.push_back(std::move(m));
    }
    rest.swap(oth);
    // multiplicand: the leaf's coefficient, or the child's polynomial
    int mul = -1;
    uint8_t fl = 0;
    if (grp.empty()) { mul = leaf_k; fl |= G_BK; }
    else mul = horner_node(B, grp, leaf_k, zero_k);
    // addend: the running sum, else the node's own coefficient (or zero)
    int add = acc;
    if (acc < 0) { add = coef >= 0 ? coef : zero_k; fl |= G_CK; }
    int d = B.newval();
    B.prog.push_back({T_G, d, best, mul, add, fl});
    B.flops += (acc < 0 && coef < 0) ? 1 : 2;
    acc = d;
  }
  if (!key.empty()) B.hcse[key] = {acc, B.prog.size()};
  return acc;
}

// Emits the Horner evaluation of ms into a fresh value; monomials must have
// distinct variable lists.
static int emit_horner(Builder &B, std::vector<HMono> ms) {
  int coef = -1;
  std::vector<HMono> inner;
  for (auto &m : ms) {
    std::sort(m.v.begin(), m.v.end());
    if (m.v.empty()) coef = m.k;
    else inner.push_back(std::move(m));
  }
  if (inner.empty()) return coef >= 0 ? B.cval(coef) : B.zero();
  return horner_node(B, inner, coef, B.konst(0.0));
}

// polynomial in z evaluated into a fresh accumulator
static int emit_poly(Builder &B, const Poly &p) {
  std::vector<std::pair<std::vector<int>, double>> ms;
  for (auto &kv : p.t) {
    std::vector<int> vars;
    for (int i = 0; i < B.M; ++i) {
      int e = (int)(kv.first >> (4 * i) & 15);
      for (int t = 0; t < e; ++t) vars.push_back(i);
    }
    ms.push_back({vars, kv.second});
  }
  std::sort(ms.begin(), ms.end());
  if (B.horner) {
    std::vector<HMono> hm;
    for (auto &m : ms) hm.push_back({m.first, B.konst(m.second)});
    int v = emit_horner(B, hm);
    if (v >= 0) return v;
  }
  int acc = B.zero();
  ProdStack ps;
  int one = -1;
  for (auto &m : ms) {
    int k = B.konst(m.second);
    int mv;
    if (m.first.empty()) { if (one < 0) one = B.cval(B.konst(1.0)); mv = one; }
    else mv = stack_product(B, ps, m.first);
    B.fmac(acc, mv, k);
  }
  return acc;
}

struct FactorVals {
  int rU, V;                         // value ids
  std::vector<int> a, b;             // per eline
  std::vector<std::vector<int>> Z;   // per eline pair
};

static FactorVals emit_graph_functions(Builder &B, const Factor &f, bool need_b) {
  const Graph &g = *f.g;
  int E = (int)f.elines.size(), Lp = (int)f.photons.size();
  auto alpha_e = [&](int k) {
    int p = line_param(g, Line{false, f.elines[k] - 1, f.elines[k]});
    return p == 0 ? Poly::var(0, 0.5) : Poly::var(p);
  };
  std::vector<Poly> ae(E);
  for (int k = 0; k < E; ++k) ae[k] = alpha_e(k);
  std::vector<std::vector<Poly>> A(Lp, std::vector<Poly>(Lp));
  for (int c = 0; c < Lp; ++c) {
    A[c][c] = A[c][c] + Poly::var(line_param(g, f.photons[c]));
    for (int c2 = 0; c2 < Lp; ++c2) {
      int lo = std::max(f.spans[c].first, f.spans[c2].first);
      int hi = std::min(f.spans[c].second, f.spans[c2].second);
      for (int k = lo; k < hi; ++k) A[c][c2] = A[c][c2] + ae[k];
    }
  }
  Poly U = det_poly(A);
  std::vector<std::vector<Poly>> adj(Lp, std::vector<Poly>(Lp));
  for (int c = 0; c < Lp; ++c)
    for (int c2 = 0; c2 < Lp; ++c2) {
      std::vector<std::vector<Poly>> m;
      for (int i = 0; i < Lp; ++i) {
        if (i == c2) continue;
        std::vector<Poly> row;
        for (int j = 0; j < Lp; ++j) if (j != c) row.push_back(A[i][j]);
        m.push_back(row);
      }
      Poly d = det_poly(m);
      adj[c][c2] = ((c + c2) % 2 == 0) ? d : (-1.0) * d;
    }
  auto in_span = [&](int k, int c) { return f.spans[c].first <= k && k < f.spans[c].second; };
  std::vector<std::vector<Poly>> Bb(E, std::vector<Poly>(E));
  for (int k = 0; k < E; ++k)
    for (int k2 = k; k2 < E; ++k2) {
      Poly s;
      for (int c = 0; c < Lp; ++c) if (in_span(k, c))
        for (int c2 = 0; c2 < Lp; ++c2) if (in_span(k2, c2)) s = s + adj[c][c2];
      Bb[k][k2] = s;
      Bb[k2][k] = s;
    }
  std::vector<Poly> Bc(Lp);
  for (int c = 0; c < Lp; ++c)
    for (int k = f.spans[c].first; k < f.spans[c].second; ++k) Bc[c] = Bc[c] + ae[k];
  Poly UV;
  for (int c = 0; c < Lp; ++c)
    for (int c2 = 0; c2 < Lp; ++c2) UV = UV - (Bc[c] * Bc[c2]) * adj[c][c2];
  std::vector<Poly> Na(E), Nb(E);
  for (int k = 0; k < E; ++k) {
    Poly s = U;
    for (int k2 = 0; k2 < E; ++k2) s = s - Bb[k][k2] * ae[k2];
    Na[k] = s;
    if (need_b) {
      auto d = [&](int kk) { return kk < f.ext_node ? -0.5 : 0.5; };
      Poly t = d(k) * U;
      for (int k2 = 0; k2 < E; ++k2) t = t - d(k2) * (Bb[k][k2] * ae[k2]);
      Nb[k] = t;
    }
  }
  // emit
  FactorVals fv;
  B.clear_cse();
  int Uv = emit_poly(B, U);
  int one = B.cval(B.konst(1.0));
  fv.rU = B.bin(T_DIV, one, Uv);
  std::map<std::map<uint64_t, double>, int> pcache;
  auto ratio = [&](const Poly &p) {
    auto it = pcache.find(p.t);
    if (it != pcache.end()) return it->second;
    int v;
    if (p.t.empty()) v = B.zero();
    else v = B.bin(T_MUL, emit_poly(B, p), fv.rU);
    pcache[p.t] = v;
    return v;
  };
  fv.V = ratio(UV);
  fv.a.resize(E); fv.b.assign(E, -1);
  fv.Z.assign(E, std::vector<int>(E, -1));
  for (int k = 0; k < E; ++k) fv.a[k] = ratio(Na[k]);
  if (need_b) for (int k = 0; k < E; ++k) fv.b[k] = ratio(Nb[k]);
  for (int k = 0; k < E; ++k)
    for (int k2 = k; k2 < E; ++k2) { fv.Z[k][k2] = ratio(Bb[k][k2]); fv.Z[k2][k] = fv.Z[k][k2]; }
  B.clear_cse();
  return fv;
}

// numerator j-vector of one factor channel: vec[j] = rU^2 sum_monomials
static std::vector<int> emit_numerator(Builder &B, const FactorVals &fv, const std::vector<Mono> &ms) {
  int jmax = -1;
  for (auto &m : ms) jmax = std::max(jmax, m.j);
  std::vector<int> acc(jmax + 1, -1);
  int one = -1;
  std::vector<std::pair<std::vector<int>, const Mono *>> order;
  for (auto &m : ms) {
    std::vector<int> vars;
    for (int s : m.a_sites) vars.push_back(fv.a[s]);
    if (m.q_site >= 0) vars.push_back(fv.b[m.q_site]);
    for (auto &pr : m.pairs) vars.push_back(fv.Z[pr.first][pr.second]);
    std::sort(vars.begin(), vars.end());
    order.push_back({vars, &m});
  }
  // by Wick order j first (one Horner tree, or one contiguous monomial chain,
  // per j), then lexicographically for prefix reuse
  std::sort(order.begin(), order.end(), [](const std::pair<std::vector<int>, const Mono *> &x,
                                           const std::pair<std::vector<int>, const Mono *> &y) {
    if (x.second->j != y.second->j) return x.second->j < y.second->j;
    return x.first < y.first;
  });
  B.clear_cse();
  if (B.horner) {
    // one Horner tree per Wick order j; equal variable lists merged exactly
    std::vector<int> res(jmax + 1, -1);
    bool ok = true;
    for (int j = 0; j <= jmax && ok; ++j) {
      std::map<std::vector<int>, std::pair<long long, long long>> merged;
      for (auto &o : order) {
        if (o.second->j != j) continue;
        auto it = merged.find(o.first);
        if (it == merged.end()) { merged[o.first] = {o.second->num, o.second->den}; continue; }
        long long n1 = it->second.first, d1 = it->second.second;
        long long n2 = o.second->num, d2 = o.second->den;
        long long g = gcdll(d1, d2);
        __int128 num = (__int128)n1 * (d2 / g) + (__int128)n2 * (d1 / g), den = (__int128)(d1 / g) * d2;
        __int128 h = num, b2 = den;
        if (h < 0) h = -h;
        while (b2) { __int128 t = h % b2; h = b2; b2 = t; }
        if (h == 0) h = 1;
        num /= h; den /= h;
        if (num > LLONG_MAX || num < -LLONG_MAX || den > LLONG_MAX) ok = false;
        it->second = {(long long)num, (long long)den};
      }
      if (merged.empty()) continue;
      std::vector<HMono> hm;
      for (auto &kv : merged)
        if (kv.second.first != 0) hm.push_back({kv.first, B.konst_rat(kv.second.first, kv.second.second)});
      if (hm.empty()) { res[j] = B.zero(); continue; }
      int v = emit_horner(B, hm);
      if (v < 0) ok = false;
      res[j] = v;
    }
    if (ok) {
      int rU2 = B.bin(T_MUL, fv.rU, fv.rU);
      for (auto &a : res)
        if (a >= 0) a = B.bin(T_MUL, a, rU2);
      B.clear_cse();
      return res;
    }
  }
  ProdStack ps;
  for (auto &o : order) {
    const Mono &m = *o.second;
    int mv;
    if (o.first.empty()) { if (one < 0) one = B.cval(B.konst(1.0)); mv = one; }
    else mv = stack_product(B, ps, o.first);
    if (acc[m.j] < 0) acc[m.j] = B.zero();
    B.fmac(acc[m.j], mv, B.konst_rat(m.num, m.den));
  }
  int rU2 = B.bin(T_MUL, fv.rU, fv.rU);
  for (auto &a : acc)
    if (a >= 0) a = B.bin(T_MUL, a, rU2);
  B.clear_cse();
  return acc;
}

// ============================================================ integrand ==
Tape compile_integrand(const Graph &g, CompileStats *st) {
  std::vector<Sub> subs = divergent_subgraphs(g);
  std::vector<Term> terms = rnew_terms(g, subs);
  int n = g.n;
  Builder B;
  B.M = g.M();
  // reuse window of Horner subtrees: a wider one saves more instructions but
  // keeps more values live; at four and five loops the slot file limits
  // occupancy, at three it does not (measured: 3 loops -2.8 % instructions
  // at 1024 vs 64 with the same pitch; 5 loops +40 % pitch at 1024)
  B.share_window = g.n <= 3 ? 1024 : g.n == 4 ? 256 : 64;
  B.nvals = B.M;    // z values are 0..M-1
  TraceMemo tm;
  int nmono = 0;
  auto nested = [&](int a, int b) { return subs[b].lo <= subs[a].lo && subs[a].hi <= subs[b].hi; };

  // ---- phase 1: list every factor channel each term needs ------------------
  struct Need { std::string gkey; int S; std::vector<int> ch; int chan; std::vector<int> child_chan; };
  std::map<std::string, Need> needs;                // nkey -> need
  std::map<std::string, std::vector<std::string>> by_graph;   // gkey -> nkeys
  struct Assign { std::vector<std::string> nkeys; std::vector<std::string> gkeys; };
  std::vector<std::vector<Assign>> term_assigns(terms.size());
  for (size_t ti = 0; ti < terms.size(); ++ti) {
    const Term &t = terms[ti];
    const std::vector<int> &F = t.elems;
    std::vector<int> se_elems;
    for (int e : F) if (subs[e].se) se_elems.push_back(e);
    std::vector<std::vector<int>> kids(F.size());
    for (size_t i = 0; i < F.size(); ++i)
      for (size_t j = 0; j < F.size(); ++j) {
        if (i == j || !nested(F[j], F[i])) continue;
        bool maximal = true;
        for (size_t k = 0; k < F.size(); ++k)
          if (k != i && k != j && nested(F[j], F[k]) && nested(F[k], F[i])) maximal = false;
        if (maximal) kids[i].push_back(F[j]);
      }
    for (uint32_t cm = 0; cm < (1u << se_elems.size()); ++cm) {
      auto chan_of_se = [&](int e) {
        for (size_t q = 0; q < se_elems.size(); ++q)
          if (se_elems[q] == e) return (cm >> q & 1) ? (int)CH_V : (int)CH_U;
        return -1;
      };
      Assign as;
      for (size_t i = 0; i < F.size(); ++i) {
        int S = F[i], op = t.ops[i], chan;
        if (subs[S].se) chan = chan_of_se(S);
        else if (op == OP_U) chan = CH_A;
        else if (op == OP_L) chan = CH_ABC;
        else if (op == OP_LmU) chan = CH_BC;
        else chan = CH_F2;
        std::vector<int> ch = kids[i];
        std::sort(ch.begin(), ch.end(), [&](int x, int y) { return subs[x].lo < subs[y].lo; });
        bool need_b = chan == CH_F2;
        std::string gkey = std::to_string(subs[S].lo) + ":" + std::to_string(subs[S].hi);
        for (int c : ch) gkey += "," + std::to_string(subs[c].lo) + "-" + std::to_string(subs[c].hi);
        if (need_b) gkey += "b";
        std::vector<int> child_chan;
        std::string nkey = gkey + "|" + std::to_string(chan);
        for (int c : ch) { int cc = subs[c].se ? chan_of_se(c) : -1; child_chan.push_back(cc); nkey += "/" + std::to_string(cc); }
        if (!needs.count(nkey)) {
          needs[nkey] = Need{gkey, S, ch, chan, child_chan};
          by_graph[gkey].push_back(nkey);
        }
        as.nkeys.push_back(nkey);
        as.gkeys.push_back(gkey);
      }
      term_assigns[ti].push_back(as);
    }
  }
  // ---- phases 2 and 3: factor graphs, and each term as soon as its factors
  // are there (so the numerator values of finished terms die early and the
  // slot file stays small) ----------------------------------------------------
  std::map<std::string, std::vector<int>> numv;   // nkey -> j-vector values
  std::map<std::string, int> Vval;                // gkey -> V value
  int Itot = B.zero(), Ktot = B.zero();
  auto emit_term = [&](size_t ti) {
    int termval = B.zero();
    const std::vector<Assign> &asg = term_assigns[ti];
    // W = sum of the factors' V (same factor graphs for every assignment)
    int Wv = Vval[asg[0].gkeys[0]];
    for (size_t i = 1; i < asg[0].gkeys.size(); ++i) Wv = B.bin(T_ADD, Wv, Vval[asg[0].gkeys[i]]);
    int negW = B.mulc(Wv, B.konst(-1.0));
    int one = B.cval(B.konst(1.0));
    int r = B.bin(T_DIV, one, negW);
    std::vector<int> rp(n + 1, -1);
    rp[1] = r;
    for (int k = 2; k <= n; ++k) rp[k] = B.bin(T_MUL, rp[k - 1], r);
    for (const Assign &as : asg) {
      std::vector<int> conv = {-2};   // -2 = exact one, -1 = zero
      for (const std::string &nk : as.nkeys) {
        const std::vector<int> &v = numv[nk];
        std::vector<int> nc(conv.size() + v.size() - 1, -1);
        for (size_t j1 = 0; j1 < conv.size(); ++j1) {
          if (conv[j1] == -1) continue;
          for (size_t j2 = 0; j2 < v.size(); ++j2) {
            if (v[j2] < 0) continue;
            int prod = conv[j1] == -2 ? v[j2] : B.bin(T_MUL, conv[j1], v[j2]);
            if (nc[j1 + j2] == -1) nc[j1 + j2] = prod;
            else nc[j1 + j2] = B.bin(T_ADD, nc[j1 + j2], prod);
          }
        }
        conv = nc;
      }
      // weights (-1)^j 2^-j (n-j-1)! (-W)^-(n-j)
      for (size_t j = 0; j < conv.size(); ++j) {
        if (conv[j] == -1) continue;
        if ((int)j >= n) throw std::runtime_error("nonzero coefficient of a divergent lambda integral");
        double w = ((j % 2) ? -1.0 : 1.0) * std::ldexp(1.0, -(int)j);
        double fact = 1.0;
        for (int i = 2; i <= n - (int)j - 1; ++i) fact *= i;
        int x = conv[j] == -2 ? one : conv[j];
        int wx = B.bin(T_MUL, x, rp[n - j]);
        B.fmac(termval, wx, B.konst(w * fact));
      }
    }
    B.fmac(Itot, termval, B.konst((double)terms[ti].sign));
    B.addabs(Ktot, termval);
  };
  std::vector<std::set<std::string>> term_g(terms.size());
  for (size_t ti = 0; ti < terms.size(); ++ti)
    for (const Assign &as : term_assigns[ti]) term_g[ti].insert(as.gkeys.begin(), as.gkeys.end());
  std::set<std::string> done_g;
  std::vector<char> term_done(terms.size(), 0);
  std::vector<std::string> left;
  for (auto &kv : by_graph) left.push_back(kv.first);
  while (!left.empty()) {
    // next factor graph: the one that completes most terms, then the one
    // needed by most unfinished terms (first in key order on ties)
    size_t pick = 0;
    int best_c = -1, best_u = -1;
    for (size_t q = 0; q < left.size(); ++q) {
      int c = 0, u = 0;
      for (size_t ti = 0; ti < terms.size(); ++ti) {
        if (term_done[ti] || !term_g[ti].count(left[q])) continue;
        ++u;
        bool complete = true;
        for (const std::string &gk : term_g[ti])
          if (gk != left[q] && !done_g.count(gk)) { complete = false; break; }
        if (complete) ++c;
      }
      if (c > best_c || (c == best_c && u > best_u)) { best_c = c; best_u = u; pick = q; }
    }
    const std::string gkey = left[pick];
    left.erase(left.begin() + pick);
    const std::vector<std::string> &nks = by_graph[gkey];
    const Need &n0 = needs[nks[0]];
    Factor f = make_factor(g, subs, n0.S, n0.ch);
    bool need_b = gkey.back() == 'b';
    FactorVals fv = emit_graph_functions(B, f, need_b);
    Vval[gkey] = fv.V;
    for (const std::string &nk : nks) {
      const Need &nd = needs[nk];
      std::vector<Mono> ms = expand_factor(f, nd.chan, nd.child_chan, tm);
      nmono += (int)ms.size();
      numv[nk] = emit_numerator(B, fv, ms);
    }
    done_g.insert(gkey);
    for (size_t ti = 0; ti < terms.size(); ++ti) {
      if (term_done[ti]) continue;
      bool complete = true;
      for (const std::string &gk : term_g[ti])
        if (!done_g.count(gk)) { complete = false; break; }
      if (complete) { emit_term(ti); term_done[ti] = 1; }
    }
  }
  int nfac = (int)by_graph.size();
  // prefactor z_e 4^-n (-1)^n
  double pref = std::ldexp(1.0, -2 * n) * ((n % 2) ? -1.0 : 1.0);
  int zI = B.bin(T_MUL, Itot, 0);
  int outI = B.mulc(zI, B.konst(pref));
  int zK = B.bin(T_MUL, Ktot, 0);
  int outK = B.mulc(zK, B.konst(std::fabs(pref)));
  // ------------------------------------------------ dead code removal --
  // value operands of an intermediate instruction
  auto b_is_val = [](const Builder::SIns &in) {
    return in.op == T_ADD || in.op == T_SUB || in.op == T_MUL || in.op == T_DIV || in.op == T_FMA ||
           ((in.op == T_G || in.op == T_GA || in.op == T_GAC) && !(in.fl & G_BK));
  };
  auto c_is_val = [](const Builder::SIns &in) { return (in.op == T_G || in.op == T_GA) && !(in.fl & G_CK); };
  auto accum = [](uint8_t op) { return op == T_FMA || op == T_FMAC || op == T_ADDABS || op == T_GAC; };
  const int zk = B.konst(0.0);
  const int k_one = B.konst(1.0), k_mone = B.konst(-1.0);
  auto dce = [&](std::vector<int> roots) {
    std::vector<char> live(B.nvals, 0);
    for (int r : roots) live[r] = 1;
    std::vector<char> keep(B.prog.size(), 0);
    for (int i = (int)B.prog.size() - 1; i >= 0; --i) {
      auto &in = B.prog[i];
      if (!live[in.d]) continue;
      keep[i] = 1;
      if (in.a >= 0) live[in.a] = 1;
      if (b_is_val(in) && in.b >= 0) live[in.b] = 1;
      if (c_is_val(in) && in.c >= 0) live[in.c] = 1;
      if (accum(in.op)) live[in.d] = 1;
    }
    std::vector<Builder::SIns> np;
    for (size_t i = 0; i < B.prog.size(); ++i)
      if (keep[i]) np.push_back(B.prog[i]);
    B.prog.swap(np);
  };
  dce({outI, outK});
  // ------------------------------------------------ running error bound --
  // The paper certifies every FP64 value with an interval whose radius is
  // estimated next to the centres (Sec. IV.A, Eq. eq_interval_accept).  The
  // library's form of that estimate is the classical running bound for
  // straight-line code: a value reached through k roundings on its deepest
  // chain lies within gamma_k * M of the exact one, M being the same
  // computation done on absolute values (products add depths, sums take the
  // larger; a quotient a/b has M = (M_a + |a/b| M_b) / |b| to first order).
  // A value whose operands never meet with opposite signs has M = |value|
  // and costs nothing; only the others get a magnitude twin (T_GA, T_GAC).
  int outE = -1, depth = 0;
  {
    const size_t n0 = B.prog.size();
    const size_t cap = (size_t)B.nvals + 3 * n0 + 8;
    std::vector<uint8_t> sg(cap, 1);   // bit 0: may be > 0, bit 1: may be < 0
    std::vector<int> mv(cap, -1);      // magnitude twin, -1: |value| itself
    std::vector<int> kd(cap, 0);       // roundings on the deepest chain
    auto ksg = [&](int k) -> uint8_t { double v = B.khi[k]; return v > 0 ? 1 : v < 0 ? 2 : 0; };
    auto kdep = [&](int k) { return B.klo[k] != 0.0 ? 1 : 0; };
    auto mulsg = [](uint8_t x, uint8_t y) -> uint8_t {
      uint8_t r = 0;
      if (((x & 1) && (y & 1)) || ((x & 2) && (y & 2))) r |= 1;
      if (((x & 1) && (y & 2)) || ((x & 2) && (y & 1))) r |= 2;
      return r;
    };
    auto mag = [&](int v) { return mv[v] >= 0 ? mv[v] : v; };
    auto tracked = [&](int v) { return mv[v] >= 0; };
    std::vector<Builder::SIns> np;
    np.reserve(2 * n0 + 4);
    auto twin = [&](uint8_t op, int d, int a, int b, int c, uint8_t fl) {
      Builder::SIns t;
      t.op = op; t.d = d; t.a = a; t.b = b; t.c = c; t.fl = fl;
      np.push_back(t);
    };
    // d = A * Bv + Cv, operands given as (is constant, id); C absent: c < 0
    struct Opd { bool k; int id; };
    auto opsg = [&](Opd o) -> uint8_t { return o.id < 0 ? 0 : o.k ? ksg(o.id) : sg[o.id]; };
    auto opdep = [&](Opd o) { return o.id < 0 ? 0 : o.k ? kdep(o.id) : kd[o.id]; };
    auto optr = [&](Opd o) { return o.id >= 0 && !o.k && tracked(o.id); };
    for (size_t i = 0; i < n0; ++i) {
      const Builder::SIns in = B.prog[i];
      Opd A{false, in.a}, Bo{false, -1}, Co{false, -1};
      bool acc = false, special = false;
      switch (in.op) {
        case T_ADD: Bo = {true, k_one}; Co = {false, in.b}; break;
        case T_SUB: A = {false, in.b}; Bo = {true, k_mone}; Co = {false, in.a}; break;
        case T_MUL: Bo = {false, in.b}; break;
        case T_FMA: Bo = {false, in.b}; Co = {false, in.d}; acc = true; break;
        case T_FMAC: Bo = {true, in.b}; Co = {false, in.d}; acc = true; break;
        case T_MULC: Bo = {true, in.b}; break;
        case T_G:
          Bo = (in.fl & G_BK) ? Opd{true, in.b} : Opd{false, in.b};
          Co = (in.fl & G_CK) ? Opd{true, in.c} : Opd{false, in.c};
          break;
        default: special = true; break;
      }
      if (!special) {
        const uint8_t sP = mulsg(opsg(A), opsg(Bo)), sC = opsg(Co);
        const bool cancel = ((sP & 1) && (sC & 2)) || ((sP & 2) && (sC & 1));
        const int kP = opdep(A) + opdep(Bo);
        // magnitude operands
        const int ma = mag(A.id);
        const int mb = Bo.k ? Bo.id : mag(Bo.id);
        const uint8_t fb = Bo.k ? G_BK : 0;
        if (acc) {
          const int d = in.d;
          if (tracked(d)) {
            twin(T_GAC, mv[d], ma, mb, -1, fb);
          } else if (cancel || optr(A) || optr(Bo)) {
            const int md = B.newval();
            twin(T_GA, md, ma, mb, d, fb);   // reads d before the update below
            mv[d] = md;
          }
          np.push_back(in);
          sg[d] = (uint8_t)(sP | sC);
          kd[d] = std::max(kP, kd[d]) + 1;
        } else {
          np.push_back(in);
          const int d = in.d;
          sg[d] = (uint8_t)(sP | sC);
          kd[d] = std::max(kP, opdep(Co)) + 1;
          int ex;
          if (in.op == T_MULC && std::fabs(std::frexp(B.khi[in.b], &ex)) == 0.5) kd[d] = kP;   // exact scaling
          if (cancel || optr(A) || optr(Bo) || optr(Co)) {
            const int md = B.newval();
            int mc; uint8_t fc;
            if (Co.id < 0) { mc = zk; fc = G_CK; }
            else if (Co.k) { mc = Co.id; fc = G_CK; }
            else { mc = mag(Co.id); fc = 0; }
            twin(T_GA, md, ma, mb, mc, (uint8_t)(fb | fc));
            mv[d] = md;
          }
        }
        continue;
      }
      const int d = in.d;
      switch (in.op) {
        case T_DIV: {
          np.push_back(in);
          sg[d] = mulsg(sg[in.a], sg[in.b]);
          kd[d] = kd[in.a] + kd[in.b] + 1;
          if (tracked(in.a) || tracked(in.b)) {
            const int t = B.newval(), md = B.newval();
            twin(T_GA, t, d, mag(in.b), mag(in.a), 0);   // |a/b| M_b + M_a
            twin(T_DIV, md, t, in.b, -1, 0);             // over b (sign dropped by the readers)
            mv[d] = md;
          }
          break;
        }
        case T_CONST:
          np.push_back(in);
          sg[d] = ksg(in.b); kd[d] = kdep(in.b);
          break;
        case T_ZERO:
          np.push_back(in);
          sg[d] = 0; kd[d] = 0;
          break;
        case T_ABS: case T_NEG: {
          np.push_back(in);
          const uint8_t s = sg[in.a];
          sg[d] = in.op == T_ABS ? (uint8_t)(s ? 1 : 0) : (uint8_t)(((s & 1) << 1) | ((s & 2) >> 1));
          kd[d] = kd[in.a];
          if (tracked(in.a)) {   // own copy: the operand may be an accumulator that changes later
            const int md = B.newval();
            twin(T_GA, md, mv[in.a], k_one, zk, G_BK | G_CK);
            mv[d] = md;
          }
          break;
        }
        case T_ADDABS: {   // d = d + |a|
          const uint8_t sP = sg[in.a] ? 1 : 0, sC = sg[d];
          const bool cancel = (sP & 1) && (sC & 2);
          if (tracked(d)) twin(T_GAC, mv[d], mag(in.a), k_one, -1, G_BK);
          else if (cancel || tracked(in.a)) {
            const int md = B.newval();
            twin(T_GA, md, mag(in.a), k_one, d, G_BK);
            mv[d] = md;
          }
          np.push_back(in);
          sg[d] = (uint8_t)(sP | sC);
          kd[d] = std::max(kd[in.a], kd[d]) + 1;
          break;
        }
        default: throw std::runtime_error("error bound: unknown intermediate operation");
      }
    }
    // E = gamma_D * M_I,  gamma_D = D u / (1 - D u),  u = 2^-53, with a 2 %
    // allowance for the rounding of M itself and first-order terms
    depth = kd[outI];
    const double u = std::ldexp(1.0, -53);
    const double gam = 1.02 * depth * u / (1.0 - depth * u);
    outE = B.newval();
    twin(T_GA, outE, mag(outI), B.konst(gam), zk, G_BK | G_CK);
    B.prog.swap(np);
  }
  dce({outI, outK, outE});
  {
    double fl = 0, flb = 0;
    for (const auto &in : B.prog) {
      double f;
      if (in.op == T_G || in.op == T_GA) f = ((in.fl & G_CK) && in.c == zk) ? 1 : 2;
      else f = (in.op == T_FMA || in.op == T_FMAC || in.op == T_GAC) ? 2
             : (in.op == T_CONST || in.op == T_ZERO) ? 0 : 1;
      fl += f;
      if (in.op == T_GA || in.op == T_GAC) flb += f;
    }
    B.flops = fl;
    B.flops_bound = flb;
  }
  // ---------------------------------------------------- slot allocation --
  std::vector<int> last(B.nvals, -1);
  for (size_t i = 0; i < B.prog.size(); ++i) {
    auto &in = B.prog[i];
    if (in.a >= 0) last[in.a] = (int)i;
    if (b_is_val(in) && in.b >= 0) last[in.b] = (int)i;
    if (c_is_val(in) && in.c >= 0) last[in.c] = (int)i;
    if (accum(in.op)) last[in.d] = (int)i;
  }
  last[outI] = last[outK] = last[outE] = (int)B.prog.size();
  std::vector<int> slot(B.nvals, -1);
  std::vector<int> freelist;
  int nslots = B.M;
  for (int i = 0; i < B.M; ++i) slot[i] = i;   // z slots stay reserved
  struct Low { const Builder::SIns *in; int sd, sa, sb, sc; };
  std::vector<Low> low;
  low.reserve(B.prog.size());
  for (size_t i = 0; i < B.prog.size(); ++i) {
    const auto &in = B.prog[i];
    int sa = in.a >= 0 ? slot[in.a] : 0;
    int sb = b_is_val(in) ? slot[in.b] : -1;
    int sc = c_is_val(in) ? slot[in.c] : -1;
    // release operands whose last use is here (before allocating d, so that
    // d may take the slot of the value it replaces)
    bool acc = accum(in.op);
    std::vector<int> rel;
    auto release = [&](int v) {
      if (v >= B.M && last[v] == (int)i && !(acc && v == in.d) &&
          std::find(rel.begin(), rel.end(), v) == rel.end()) rel.push_back(v);
    };
    if (in.a >= 0) release(in.a);
    if (b_is_val(in) && in.b >= 0) release(in.b);
    if (c_is_val(in) && in.c >= 0) release(in.c);
    int sd;
    if (acc) sd = slot[in.d];
    else {
      for (int v : rel) freelist.push_back(slot[v]);
      rel.clear();
      if (!freelist.empty()) { sd = freelist.back(); freelist.pop_back(); }
      else sd = nslots++;
      slot[in.d] = sd;
      if (last[in.d] <= (int)i) freelist.push_back(sd);   // never read
    }
    for (int v : rel) freelist.push_back(slot[v]);
    if (acc && last[in.d] == (int)i && in.d != outI && in.d != outK && in.d != outE) freelist.push_back(sd);
    low.push_back({&in, sd, sa, sb, sc});
  }
  if (nslots > 8191) throw std::runtime_error("tape needs more than 8191 slots");
  // ------------------------------------------- lowering to instructions --
  // every arithmetic operation becomes  d = a * (b | kb) + (c | kc)
  if (B.khi.size() > 65535) throw std::runtime_error("constant pool exceeds 16-bit indices");
  Tape tp;
  tp.M = B.M;
  for (const Low &l : low) {
    const auto &in = *l.in;
    Ins o{};
    auto setb = [&](int k) { o.op |= I_BK; o.kbi = (uint16_t)k; o.kb = B.khi[k]; };
    auto setc = [&](int k) { o.op |= I_CK; o.kci = (uint16_t)k; o.kc = B.khi[k]; };
    int a = l.sa, bb = 0, cc = 0;
    switch (in.op) {
      case T_ADD: bb = 0; setb(k_one); cc = l.sb; break;                 // a * 1 + b
      case T_SUB: a = l.sb; setb(k_mone); cc = l.sa; break;              // b * -1 + a
      case T_MUL: bb = l.sb; setc(zk); break;                            // a * b + 0
      case T_DIV: bb = l.sb; o.op = I_DIV; break;
      case T_FMA: bb = l.sb; cc = l.sd; break;                           // a * b + d
      case T_FMAC: setb(in.b); cc = l.sd; break;                         // a * K + d
      case T_MULC: setb(in.b); setc(zk); break;                          // a * K + 0
      case T_CONST: a = 0; setb(zk); setc(in.b); break;                  // z0 * 0 + K
      case T_ABS: o.op = I_ABS; break;
      case T_NEG: setb(k_mone); setc(zk); break;                         // a * -1 + 0
      case T_ZERO: a = 0; setb(zk); setc(zk); break;                     // z0 * 0 + 0
      case T_ADDABS: o.op = I_ADDABS; cc = l.sd; break;                  // d + |a|
      case T_G:
        if (in.fl & G_BK) setb(in.b); else bb = l.sb;
        if (in.fl & G_CK) setc(in.c); else cc = l.sc;
        break;
      case T_GA:
        o.op = I_AB;
        if (in.fl & G_BK) setb(in.b); else bb = l.sb;
        if (in.fl & G_CK) setc(in.c); else cc = l.sc;
        break;
      case T_GAC:
        o.op = I_AB;
        if (in.fl & G_BK) setb(in.b); else bb = l.sb;
        cc = l.sd;
        break;
      default: throw std::runtime_error("unknown intermediate operation");
    }
    if (!(o.op & 0xff00) && !(o.op & I_AB)) {
      const bool bx = !(o.op & I_BK) || B.klo[o.kbi] == 0.0, cx = !(o.op & I_CK) || B.klo[o.kci] == 0.0;
      if (bx && cx) o.op |= I_KX;
      if ((o.op & I_CK) && o.kc == 0.0 && cx) o.op |= I_C0;
      if ((o.op & I_BK) && (o.kb == 1.0 || o.kb == -1.0) && bx) o.op |= I_B1;
    }
    o.d = (uint16_t)(l.sd * 8);
    o.a = (uint16_t)(a * 8);
    o.b = (uint16_t)(bb * 8);
    o.c = (uint16_t)(cc * 8);
    tp.code.push_back(o);
  }
  // FP64 flops of the double-double evaluation of every instruction, by the
  // form its hints select (FMA = 2; two-sum 6, quick two-sum 3 operations):
  // magnitude twin 2, exact scaling 8, product 10, sum 11, c + exact k*a 16,
  // general 18, quotient 86, |a| 0, c + |a| 11
  for (const Ins &o : tp.code) {
    const uint16_t sp = o.op & 0xff00;
    double f;
    if (o.op & I_AB) f = 2;
    else if (sp == 0) {
      const bool bx = (o.op & (I_BK | I_KX)) == (I_BK | I_KX);
      if (o.op & I_C0) f = bx ? 8 : 10;
      else if (o.op & I_B1) f = 11;
      else f = bx ? 16 : 18;
    } else if (sp == I_DIV) f = 86;
    else if (sp == I_ABS) f = 0;
    else f = 11;
    tp.flops_dd += f;
  }
  tp.khi = B.khi; tp.klo = B.klo;
  tp.nslots = nslots | 1;   // odd row pitch: the rows of a warp fall in distinct banks
  tp.out_I = slot[outI]; tp.out_K = slot[outK]; tp.out_E = slot[outE];
  tp.depth = depth;
  tp.flops = B.flops;
  tp.flops_bound = B.flops_bound;
  tp.n_terms = (int)terms.size();
  if (st) { st->n_terms = (int)terms.size(); st->n_factors = nfac; st->n_monomials = nmono; }
  return tp;
}

// Host replay of a tape: used only by the test suite to check the compiler
// against the oracle without a GPU.  Same operations as the device
// interpreter.
void tape_replay(const Tape &t, const double *z, double *I, double *K, double *E) {
  std::vector<double> s(t.nslots, 0.0);
  for (int i = 0; i < t.M; ++i) s[i] = z[i];
  for (const Ins &in : t.code) {
    const double a = s[in.a / 8];
    const double b = (in.op & I_BK) ? in.kb : s[in.b / 8];
    const double c = (in.op & I_CK) ? in.kc : s[in.c / 8];
    double r;
    switch (in.op >> 8) {   // special code
      case 0: r = (in.op & I_AB) ? std::fma(std::fabs(a), std::fabs(b), std::fabs(c)) : std::fma(a, b, c); break;
      case I_DIV >> 8: r = a / b; break;
      case I_ABS >> 8: r = std::fabs(a); break;
      case I_ADDABS >> 8: r = c + std::fabs(a); break;
      default: throw std::runtime_error("bad opcode");
    }
    s[in.d / 8] = r;
  }
  *I = s[t.out_I];
  *K = s[t.out_K];
  if (E) *E = s[t.out_E];
}

}  // namespace ae
