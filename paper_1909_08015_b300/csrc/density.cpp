// Deg(s) and the sector-density tables of g1, g3, g4 (Sec. III.A,
// Eqs. eq_pdf_final, eq_pdf, eq_mc_settings), and the project's log2/exp2.
//
// Deg(s) (the paper's formula is in a reference that is not available; this
// is the library's reading): power counting in Feynman-parameter units,
//   d0(s) = n_e(s)/2 + n_gamma(s) - 2 L(s) + 1/2 [merged line in s],
// Deg(s) = d0(s) if d0(s) > 0, else 1/2 - C_sub with C_sub = C_subI when s
// holds the merged line, C_subSE when d0 < 0, C_subO when d0 = 0; then
// capped at deg_max.  The cap is needed because d0 counts only ultraviolet
// scaling: when the shrinking set is a forest of electron lines the
// photons of the complement are soft and the integrand decays like
// lambda^1, not lambda^d0, and a steeper density gives infinite variance
// (finite variance needs Deg(s) < 2 * true exponent).
// Phi(T) = sum_{j in T} Phi(T\j)/Deg(T\j), Phi({j}) = 1; the sector
// probability of an ordering is prod 1/Deg(s_l) / Phi(all).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include <array>

#include "ae_internal.h"

namespace ae {

// log2 by the atanh series: x = f 2^k, f in [1/sqrt2, sqrt2),
// ln f = 2 atanh((f-1)/(f+1)) = 2 sum s^(2i+1)/(2i+1), i = 0..12.
// Plain IEEE operations (the file is compiled with -ffp-contract=off).
double ae_log2(double x) {
  int k;
  double f = std::frexp(x, &k);
  if (f < 0.7071067811865476) { f = f * 2.0; k = k - 1; }
  double s = (f - 1.0) / (f + 1.0);
  double s2 = s * s;
  double p = 1.0 / 25.0;
  for (int d = 23; d >= 3; d -= 2) p = p * s2 + 1.0 / (double)d;
  p = p * s2 + 1.0;
  double lnf = (s + s) * p;
  return (double)k + lnf * 1.4426950408889634;
}

// 2^x by the Taylor series of exp on r = (x - round(x)) ln 2, 19 terms.
double ae_exp2(double x) {
  double k = std::floor(x + 0.5);
  double r = (x - k) * 0.6931471805599453;
  double fact = 6402373705728000.0;   // 18!
  double p = 1.0 / fact;
  for (int i = 18; i >= 1; --i) {
    fact = fact / (double)i;
    p = p * r + 1.0 / fact;
  }
  return std::ldexp(p, (int)std::max(-100000.0, std::min(100000.0, k)));
}

// Table-driven log2 / exp2 (Tang's method): the argument is reduced to a
// short interval around a table point and a short series is evaluated there.
//   exp2: x = k/32 + d, |d| <= 1/64: 2^x = 2^(k div 32) 2^((k mod 32)/32) exp(d ln 2),
//         exp by its Taylor polynomial of degree 7.
//   log2: x = F 2^E, F in [3/4, 3/2), c = j/32 nearest to F (j = 24..48):
//         log2 x = E + log2 c + 2 atanh(s)/ln 2, s = (F - c)/(F + c), |s| <= 1/96,
//         atanh s by s (1 + s^2/3 + s^4/5 + s^6/7).
// The tables are ae_exp2 / ae_log2 at the table points.  The device's
// dexp2/dlog2 perform the same IEEE operations on the same tables.
// (function-local statics: initialised once, thread-safe; the graphs are
// compiled on several host threads)
const double *ae_exp2_table() {
  static const std::array<double, 32> t = [] {
    std::array<double, 32> a{};
    for (int j = 0; j < 32; ++j) a[j] = ae_exp2((double)j / 32.0);
    return a;
  }();
  return t.data();
}
const double *ae_log2_table() {
  static const std::array<double, 25> t = [] {
    std::array<double, 25> a{};
    for (int j = 24; j <= 48; ++j) a[j - 24] = ae_log2((double)j / 32.0);
    return a;
  }();
  return t.data();
}

double ae_exp2t(double x) {
  if (!(x >= -1100.0 && x <= 1100.0)) return x > 1100.0 ? HUGE_VAL : (x < -1100.0 ? 0.0 : x);
  const double *T = ae_exp2_table();
  double k = std::floor(x * 32.0 + 0.5);
  double m = std::floor(k * 0.03125);
  int j = (int)(k - m * 32.0);
  double r = (x - k * 0.03125) * 0.6931471805599453;
  double p = 1.0 / 5040.0;
  const double c[7] = {1.0 / 720.0, 1.0 / 120.0, 1.0 / 24.0, 1.0 / 6.0, 0.5, 1.0, 1.0};
  for (int i = 0; i < 7; ++i) p = p * r + c[i];
  return std::ldexp(T[j] * p, (int)m);
}

double ae_log2t(double x) {
  if (!(x > 0.0 && x < HUGE_VAL)) return x == 0.0 ? -HUGE_VAL : (x == HUGE_VAL ? HUGE_VAL : NAN);
  const double *T = ae_log2_table();
  int e;
  double f = std::frexp(x, &e);
  double F = f, E = (double)e;
  if (f < 0.75) { F = f * 2.0; E = (double)(e - 1); }
  double jf = std::floor(F * 32.0 + 0.5);
  double c = jf * 0.03125;
  double s = (F - c) / (F + c);
  double s2 = s * s;
  double p = 1.0 / 7.0;
  p = p * s2 + 1.0 / 5.0;
  p = p * s2 + 1.0 / 3.0;
  p = p * s2 + 1.0;
  double t = ((s + s) * p) * 1.4426950408889634;
  return (E + T[(int)jf - 24]) + t;
}

DensityTables build_density(const Graph &g, const DensityConsts &c) {
  DensityTables t;
  int M = g.M();
  t.M = M;
  // line ends in the merged numbering
  std::vector<int> ea(M), eb(M);
  std::vector<char> isph(M, 0);
  for (int i = 1; i <= 2 * g.n; ++i) {
    Line l{false, i - 1, i};
    int p = line_param(g, l);
    if (p == 0) { ea[0] = g.s - 1; eb[0] = g.s + 1; }
    else { ea[p] = i - 1; eb[p] = i; }
  }
  for (const Line &l : photon_lines(g)) {
    int p = line_param(g, l);
    ea[p] = l.a; eb[p] = l.b; isph[p] = 1;
  }
  uint32_t full = (1u << M) - 1;
  std::vector<double> d1(1u << M, 0.0);
  int N = g.nverts();
  for (uint32_t s = 1; s < full; ++s) {
    int ne = 0, ng = 0, nl = 0;
    std::vector<int> par(N);
    for (int v = 0; v < N; ++v) par[v] = v;
    std::vector<char> touched(N, 0);
    auto find = [&](int x) { while (par[x] != x) x = par[x]; return x; };
    for (int i = 0; i < M; ++i) {
      if (!(s >> i & 1)) continue;
      ++nl;
      if (isph[i]) ++ng; else ++ne;
      touched[ea[i]] = touched[eb[i]] = 1;
      par[find(ea[i])] = find(eb[i]);
    }
    int nv = 0, comps = 0;
    for (int v = 0; v < N; ++v)
      if (touched[v]) { ++nv; if (find(v) == v) ++comps; }
    int loops = nl - nv + comps;
    double d0 = (double)ne / 2.0 + (double)ng - 2.0 * (double)loops + ((s & 1u) ? 0.5 : 0.0);
    double deg;
    if (d0 > 0) deg = d0;
    else if (s & 1u) deg = 0.5 - c.CsubI;
    else if (d0 < 0) deg = 0.5 - c.CsubSE;
    else deg = 0.5 - c.CsubO;
    if (c.deg_max > 0 && deg > c.deg_max) deg = c.deg_max;
    d1[s] = deg;
  }
  for (int k = 0; k < 3; ++k) {
    t.deg[k].assign(1u << M, 0.0);
    for (uint32_t s = 1; s < full; ++s) {
      if (k == 0) t.deg[k][s] = d1[s];
      else if (k == 1) t.deg[k][s] = d1[s] * c.D;
      else t.deg[k][s] = d1[s] < 0.5 ? d1[s] : 0.5;
    }
    t.phi[k].assign(1u << M, 0.0);
    for (uint32_t T = 1; T <= full; ++T) {
      if ((T & (T - 1)) == 0) { t.phi[k][T] = 1.0; continue; }
      double acc = 0.0;
      for (int j = 0; j < M; ++j)
        if (T >> j & 1) {
          uint32_t R = T ^ (1u << j);
          acc = acc + t.phi[k][R] / t.deg[k][R];
        }
      t.phi[k][T] = acc;
    }
  }
  double C1 = 1.0 - c.C2 - c.C3 - c.C4;
  t.C[0] = C1; t.C[1] = c.C2; t.C[2] = c.C3; t.C[3] = c.C4;
  double f = 1.0;
  for (int i = 2; i <= M - 1; ++i) f = f * (double)i;
  t.log2_fact = ae_log2t(f);
  return t;
}

// Host Philox4x32-10 (same definition as the device generator).
void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * c[0], p1 = (uint64_t)M1 * c[2];
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0, n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    c[0] = n0; c[1] = (uint32_t)p1; c[2] = n2; c[3] = (uint32_t)p0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
}

// Tables and coefficients of the fused-multiply-add exp2/log2 of the learned
// sampler (device): 2^(j/64), j = 0..63 and log2(j/64), 64/j, j = 48..96 from
// the series definitions above; Taylor coefficients ln2^i / i! (i = 0..6) of
// 2^r and (-1)^(k+1) / (k ln 2) (k = 1..8) of log2(1 + t), rounded from long
// double.  Layout: 64 + 49 + 49 + 7 + 8 doubles.
const double *ae_fast_tables() {
  static const std::array<double, 177> t = [] {
    std::array<double, 177> a{};
    for (int j = 0; j < 64; ++j) a[j] = ae_exp2((double)j / 64.0);
    for (int j = 48; j <= 96; ++j) {
      a[64 + j - 48] = ae_log2((double)j / 64.0);
      a[113 + j - 48] = 64.0 / (double)j;
    }
    const long double ln2 = 0.693147180559945309417232121458176568L;
    long double c = 1.0L;
    for (int i = 0; i <= 6; ++i) { a[162 + i] = (double)c; c = c * ln2 / (long double)(i + 1); }
    for (int k = 1; k <= 8; ++k) a[169 + k - 1] = (double)(((k % 2) ? 1.0L : -1.0L) / ((long double)k * ln2));
    return a;
  }();
  return t.data();
}

// MRG32k3a (L'Ecuyer 1999): jump matrices A1^(2^k) mod m1, A2^(2^k) mod m2,
// k = 0..159, row-major, 18 words per k (A1 then A2).  Exact 128-bit products.
static void mat3_mul(const uint64_t *A, const uint64_t *B, uint64_t *C, uint64_t m) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      unsigned __int128 acc = 0;
      for (int k = 0; k < 3; ++k) acc += (unsigned __int128)A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = (uint64_t)(acc % m);
    }
}

const uint32_t *mrg_jump_table() {
  static const std::vector<uint32_t> t = [] {
    const uint64_t m1 = 4294967087ull, m2 = 4294944443ull;
    uint64_t P1[9] = {0, 1, 0, 0, 0, 1, m1 - 810728, 1403580, 0};
    uint64_t P2[9] = {0, 1, 0, 0, 0, 1, m2 - 1370589, 0, 527612};
    std::vector<uint32_t> v(160 * 18);
    for (int k = 0; k < 160; ++k) {
      for (int e = 0; e < 9; ++e) { v[18 * k + e] = (uint32_t)P1[e]; v[18 * k + 9 + e] = (uint32_t)P2[e]; }
      uint64_t Q1[9], Q2[9];
      mat3_mul(P1, P1, Q1, m1);
      mat3_mul(P2, P2, Q2, m2);
      std::copy(Q1, Q1 + 9, P1);
      std::copy(Q2, Q2 + 9, P2);
    }
    return v;
  }();
  return t.data();
}

}  // namespace ae

// Seeded subset of k indices out of n_total: Fisher-Yates driven by Philox
// (counter = (i, 0, 0xFFFF, 0x5E1EC7), key = seed); ascending output.
extern "C" int ae_seeded_subset(uint64_t n_total, int k, uint64_t seed, int *out) {
  if (!out || k < 0 || (uint64_t)k > n_total || n_total > (1ull << 31)) return -1;
  std::vector<int> a(n_total);
  for (uint64_t i = 0; i < n_total; ++i) a[i] = (int)i;
  for (uint64_t t = 0; t < (uint64_t)k; ++t) {
    uint64_t i = n_total - 1 - t;
    uint32_t c[4] = {(uint32_t)i, 0u, 0xFFFFu, 0x5E1EC7u};
    ae::philox_host(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    double u = ((double)(c[0] >> 5) * 67108864.0 + (double)(c[1] >> 6)) * (1.0 / 9007199254740992.0);
    uint64_t j = (uint64_t)(u * (double)(i + 1));
    if (j > i) j = i;
    std::swap(a[i], a[j]);
  }
  std::vector<int> sel(a.end() - k, a.end());
  std::sort(sel.begin(), sel.end());
  for (int t = 0; t < k; ++t) out[t] = sel[t];
  return 0;
}
