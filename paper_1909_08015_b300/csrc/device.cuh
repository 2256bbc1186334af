// Device building blocks for sm_103a: Philox4x32-10, the Hepp-sector
// sampler and density, the FP64 tape interpreter and its double-double twin.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <cstdint>

namespace aedev {

// ------------------------------------------------------------ Philox ----
// Philox4x32-10 (Salmon et al., SC'11): ten rounds of the 4x32 S-box with
// multipliers M0, M1 and Weyl key increments W0, W1.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
    uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += W0; k1 += W1;
  }
}

// two words -> uniform double in (0, 1): ((w0>>5) 2^26 + (w1>>6) + 1/2) 2^-53
__device__ __forceinline__ double u01(uint32_t w0, uint32_t w1) {
  double a = (double)(w0 >> 5), b = (double)(w1 >> 6);
  return __dmul_rn(__dadd_rn(__dadd_rn(__dmul_rn(a, 67108864.0), b), 0.5), 1.1102230246251565e-16);
}

// two words -> uniform double in (0, 1) from 52 of their bits, built as the
// double 1.m in [1, 2) and shifted: (2k + 1) 2^-53, two exact additions
// (used where the draw need not match the host operation by operation)
__device__ __forceinline__ double u01_bits(uint32_t w0, uint32_t w1) {
  const double d = __hiloint2double((int)(0x3FF00000u | (w0 >> 12)), (int)((w0 << 20) | (w1 >> 12)));
  return __dadd_rn(__dadd_rn(d, -1.0), 1.1102230246251565e-16);
}

// ---------------------------------------------------------- MRG32k3a ----
// L'Ecuyer's combined multiple recursive generator (the generator of the
// paper's Calc 1): x1_n = (1403580 x1_{n-2} - 810728 x1_{n-3}) mod m1,
// x2_n = (527612 x2_{n-1} - 1370589 x2_{n-3}) mod m2, output (x1 - x2) mod m1.
// Counter-based use: sample i of graph g under seed s starts at output
// position s 2^96 + g 2^80 + 64 i of the stream from the state (12345 x 6),
// reached by the jump matrices A^(2^k) (a host table, k = 0..159).
constexpr uint64_t kMrgM1 = 4294967087ull, kMrgM2 = 4294944443ull;

// x mod m for m = 2^32 - c (c < 2^15): fold the high word twice
__device__ __forceinline__ uint64_t mrg_mod(uint64_t x, uint64_t m, uint64_t c) {
  x = (x >> 32) * c + (x & 0xffffffffull);
  x = (x >> 32) * c + (x & 0xffffffffull);
  return x >= m ? x - m : x;
}

struct MrgState { uint64_t a[3], b[3]; };   // (x_{n-3}, x_{n-2}, x_{n-1}) of both components

__device__ __forceinline__ void mrg_apply(const uint32_t *J, MrgState &s) {
  uint64_t r[3];
  for (int i = 0; i < 3; ++i) {
    uint64_t acc = 0;
    for (int k = 0; k < 3; ++k) acc += mrg_mod((uint64_t)__ldg(J + 3 * i + k) * s.a[k], kMrgM1, 209);
    r[i] = mrg_mod(acc, kMrgM1, 209);
  }
  for (int i = 0; i < 3; ++i) s.a[i] = r[i];
  for (int i = 0; i < 3; ++i) {
    uint64_t acc = 0;
    for (int k = 0; k < 3; ++k) acc += mrg_mod((uint64_t)__ldg(J + 9 + 3 * i + k) * s.b[k], kMrgM2, 22853);
    r[i] = mrg_mod(acc, kMrgM2, 22853);
  }
  for (int i = 0; i < 3; ++i) s.b[i] = r[i];
}

// state at the start of sample idx of graph g under seed (jump over the set
// bits of s 2^96 + g 2^80 + 64 idx)
__device__ __forceinline__ MrgState mrg_start(const uint32_t *jump, uint64_t seed, uint32_t g, uint64_t idx) {
  MrgState s = {{12345, 12345, 12345}, {12345, 12345, 12345}};
  for (int k = 0; k < 64; ++k)
    if (idx >> k & 1) mrg_apply(jump + 18 * (k + 6), s);
  for (int k = 0; k < 16; ++k)
    if (g >> k & 1) mrg_apply(jump + 18 * (k + 80), s);
  for (int k = 0; k < 64; ++k)
    if (seed >> k & 1) mrg_apply(jump + 18 * (k + 96), s);
  return s;
}

__device__ __forceinline__ uint32_t mrg_next(MrgState &s) {
  const uint64_t x1 = mrg_mod(mrg_mod(1403580ull * s.a[1], kMrgM1, 209) +
                              mrg_mod((kMrgM1 - 810728ull) * s.a[0], kMrgM1, 209), kMrgM1, 209);
  const uint64_t x2 = mrg_mod(mrg_mod(527612ull * s.b[2], kMrgM2, 22853) +
                              mrg_mod((kMrgM2 - 1370589ull) * s.b[0], kMrgM2, 22853), kMrgM2, 22853);
  s.a[0] = s.a[1]; s.a[1] = s.a[2]; s.a[2] = x1;
  s.b[0] = s.b[1]; s.b[1] = s.b[2]; s.b[2] = x2;
  return (uint32_t)(x1 >= x2 ? x1 - x2 : x1 + kMrgM1 - x2);
}

// ------------------------------------------------- log2 / exp2 (series) ---
// The same sequence of IEEE operations as the host's ae_log2/ae_exp2.  The
// series coefficients 1/(2i+1) and 1/k! are the exact double quotients of
// those definitions (IEEE division is deterministic), stored as constants.
__device__ __constant__ double kInvOdd[12] = {
    0.04, 0.043478260869565216, 0.047619047619047616, 0.05263157894736842,
    0.058823529411764705, 0.06666666666666667, 0.07692307692307693, 0.09090909090909091,
    0.1111111111111111, 0.14285714285714285, 0.2, 0.3333333333333333};   // 1/25, 1/23, ..., 1/3
__device__ __constant__ double kInvFact[19] = {
    1.5619206968586225e-16, 2.8114572543455206e-15, 4.779477332387385e-14, 7.647163731819816e-13,
    1.1470745597729725e-11, 1.6059043836821613e-10, 2.08767569878681e-09, 2.505210838544172e-08,
    2.755731922398589e-07, 2.7557319223985893e-06, 2.48015873015873e-05, 0.0001984126984126984,
    0.001388888888888889, 0.008333333333333333, 0.041666666666666664, 0.16666666666666666,
    0.5, 1.0, 1.0};   // 1/18!, 1/17!, ..., 1/0!

__device__ __forceinline__ double dlog2(double x) {
  int k;
  double f = frexp(x, &k);
  if (f < 0.7071067811865476) { f = __dmul_rn(f, 2.0); k = k - 1; }
  double s = __ddiv_rn(__dadd_rn(f, -1.0), __dadd_rn(f, 1.0));
  double s2 = __dmul_rn(s, s);
  double p = kInvOdd[0];
#pragma unroll
  for (int i = 1; i < 12; ++i) p = __dadd_rn(__dmul_rn(p, s2), kInvOdd[i]);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0);
  double lnf = __dmul_rn(__dadd_rn(s, s), p);
  return __dadd_rn((double)k, __dmul_rn(lnf, 1.4426950408889634));
}

__device__ __forceinline__ double dexp2(double x) {
  double k = floor(__dadd_rn(x, 0.5));
  double r = __dmul_rn(__dadd_rn(x, -k), 0.6931471805599453);
  double p = kInvFact[0];
#pragma unroll
  for (int i = 1; i < 19; ++i) p = __dadd_rn(__dmul_rn(p, r), kInvFact[i]);
  double kc = fmin(fmax(k, -100000.0), 100000.0);
  return ldexp(p, (int)kc);
}

// --------------------------------------- log2 / exp2 (table-driven) ----
// Tang's table-driven method, the same IEEE operations as the host's
// ae_log2t / ae_exp2t on the same tables (2^(j/32) and log2(j/32), the series
// above at the table points, computed by the host and uploaded when a
// context is created).
//   exp2: x = k/32 + d, |d| <= 1/64; Taylor polynomial of degree 7 for exp(d ln 2).
//   log2: x = F 2^E, F in [3/4, 3/2), c = j/32; 2 atanh((F-c)/(F+c))/ln 2, 4 terms.
// Outside [-1100, 1100] exp2 is 0 or inf; log2 0 = -inf; NaN stays NaN (so a
// table index is always in range).
// (global memory read through L1: each lane indexes its own entry, which the
// constant cache would serialise)
__device__ double kExp2Tab[32];
__device__ double kLog2Tab[25];

// Fused-multiply-add exp2/log2 for the learned sampler (not compared with the
// host operation by operation; checked against the device library's exp2/log2):
//   exp2: x = k/64 + r, |r| <= 1/128: 2^x = 2^(k div 64) 2^((k mod 64)/64) p(r),
//         p the degree-6 Taylor polynomial of 2^r (remainder < 3e-20);
//   log2: x = F 2^E, F in [3/4, 3/2), c = j/64 nearest to F, t = (F - c)(64/j)
//         (F - c exact), log2 x = E + log2 c + t q(t), q of degree 7 from the
//         series of log2(1 + t) (|t| <= 1/96, remainder < 2e-19 t).
// Layout of kFast: 2^(j/64) (64), log2(j/64) (49, j = 48..96), 64/j (49),
// ln2^i / i! (7), (-1)^(k+1)/(k ln 2) (8).
__device__ double kFast[177];

// Each translation unit that launches sampling kernels holds its own copy of
// the tables and uploads it with this function.
static inline cudaError_t upload_elem_tables(const double *exp2_tab, const double *log2_tab, const double *fast) {
  cudaError_t e = cudaMemcpyToSymbol(kExp2Tab, exp2_tab, 32 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kLog2Tab, log2_tab, 25 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(kFast, fast, 177 * sizeof(double));
  return e;
}

// 2^x (0 below -1074, inf above 1023)
__device__ __forceinline__ double fexp2(double x) {
  if (!(x >= -1074.0 && x <= 1023.0)) return x != x ? x : (x > 0.0 ? CUDART_INF : 0.0);
  const double magic = 6755399441055744.0;   // 1.5 * 2^52: rounds x*64 to an integer in the low word
  const double kd = __fma_rn(x, 64.0, magic);
  const int k = __double2loint(kd);
  const double kr = kd - magic;
  const double r = __fma_rn(kr, -0.015625, x);
  const double *c = kFast + 162;
  double p = __ldg(c + 6);
  p = __fma_rn(p, r, __ldg(c + 5));
  p = __fma_rn(p, r, __ldg(c + 4));
  p = __fma_rn(p, r, __ldg(c + 3));
  p = __fma_rn(p, r, __ldg(c + 2));
  p = __fma_rn(p, r, __ldg(c + 1));
  p = __fma_rn(p, r, __ldg(c + 0));
  const int j = k & 63, m = k >> 6;
  const double y = __ldg(kFast + j) * p;
  if (m >= -1022) return y * __hiloint2double((m + 1023) << 20, 0);
  return ldexp(y, m);
}

// log2 x for positive finite x (the sampler's arguments: uniforms, sums >= 1)
__device__ __forceinline__ double flog2(double x) {
  int hi = __double2hiint(x);
  const int lo = __double2loint(x);
  int e = ((hi >> 20) & 0x7ff) - 1023;
  if (e == -1023) return log2(x);   // subnormal: not met by the sampler
  double F = __hiloint2double((hi & 0x000fffff) | 0x3ff00000, lo);   // [1, 2)
  if (F >= 1.5) { F = F * 0.5; e += 1; }
  const int j = __double2int_rn(F * 64.0);   // 48..96
  const double d = F - (double)j * 0.015625;
  const double t = d * __ldg(kFast + 113 + j - 48);
  const double *b = kFast + 169;
  double q = __ldg(b + 7);
  q = __fma_rn(q, t, __ldg(b + 6));
  q = __fma_rn(q, t, __ldg(b + 5));
  q = __fma_rn(q, t, __ldg(b + 4));
  q = __fma_rn(q, t, __ldg(b + 3));
  q = __fma_rn(q, t, __ldg(b + 2));
  q = __fma_rn(q, t, __ldg(b + 1));
  q = __fma_rn(q, t, __ldg(b + 0));
  return __fma_rn(t, q, (double)e + __ldg(kFast + 64 + j - 48));
}

__device__ __forceinline__ double dexp2t(double x) {
  if (!(x >= -1100.0 && x <= 1100.0)) return x > 1100.0 ? CUDART_INF : (x < -1100.0 ? 0.0 : x);
  const double k = floor(__dadd_rn(__dmul_rn(x, 32.0), 0.5));
  const double m = floor(__dmul_rn(k, 0.03125));
  const int j = (int)__dadd_rn(k, -__dmul_rn(m, 32.0));
  const double r = __dmul_rn(__dadd_rn(x, -__dmul_rn(k, 0.03125)), 0.6931471805599453);
  double p = 1.0 / 5040.0;
  p = __dadd_rn(__dmul_rn(p, r), 1.0 / 720.0);
  p = __dadd_rn(__dmul_rn(p, r), 1.0 / 120.0);
  p = __dadd_rn(__dmul_rn(p, r), 1.0 / 24.0);
  p = __dadd_rn(__dmul_rn(p, r), 1.0 / 6.0);
  p = __dadd_rn(__dmul_rn(p, r), 0.5);
  p = __dadd_rn(__dmul_rn(p, r), 1.0);
  p = __dadd_rn(__dmul_rn(p, r), 1.0);
  return ldexp(__dmul_rn(__ldg(kExp2Tab + j), p), (int)m);
}

__device__ __forceinline__ double dlog2t(double x) {
  if (!(x > 0.0 && x < CUDART_INF)) return x == 0.0 ? -CUDART_INF : (x == CUDART_INF ? CUDART_INF : CUDART_NAN);
  int e;
  const double f = frexp(x, &e);
  const bool low = f < 0.75;
  const double F = low ? __dmul_rn(f, 2.0) : f;
  const double E = (double)(low ? e - 1 : e);
  const double jf = floor(__dadd_rn(__dmul_rn(F, 32.0), 0.5));
  const double c = __dmul_rn(jf, 0.03125);
  const double s = __ddiv_rn(__dadd_rn(F, -c), __dadd_rn(F, c));
  const double s2 = __dmul_rn(s, s);
  double p = 1.0 / 7.0;
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 5.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 3.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0);
  const double t = __dmul_rn(__dmul_rn(__dadd_rn(s, s), p), 1.4426950408889634);
  return __dadd_rn(__dadd_rn(E, __ldg(kLog2Tab + (int)jf - 24)), t);
}

// ---------------------------------------------------- double-double ----
struct dd { double hi, lo; };
__device__ __forceinline__ dd two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  double bb = __dadd_rn(s, -a);
  double e = __dadd_rn(__dadd_rn(a, -__dadd_rn(s, -bb)), __dadd_rn(b, -bb));
  return {s, e};
}
__device__ __forceinline__ dd quick_two_sum(double a, double b) {
  double s = __dadd_rn(a, b);
  return {s, __dadd_rn(b, -__dadd_rn(s, -a))};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  dd t = two_sum(a.lo, b.lo);
  s.lo = __dadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __dadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  double p = __dmul_rn(a.hi, b.hi);
  double e = __fma_rn(a.hi, b.hi, -p);
  e = __fma_rn(a.hi, b.lo, e);
  e = __fma_rn(a.lo, b.hi, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  double q1 = __ddiv_rn(a.hi, b.hi);
  dd r = dd_add(a, dd_mul({-q1, 0.0}, b));
  double q2 = __ddiv_rn(r.hi, b.hi);
  r = dd_add(r, dd_mul({-q2, 0.0}, b));
  double q3 = __ddiv_rn(r.hi, b.hi);
  dd q = quick_two_sum(q1, q2);
  return dd_add(q, {q3, 0.0});
}
__device__ __forceinline__ dd dd_abs(dd a) { return a.hi < 0 ? dd{-a.hi, -a.lo} : a; }

// Faster forms for the tape: one two-sum instead of two (relative error about
// 2^-104 times the operands rather than the result; ample for re-evaluating
// cancelling sums), and d + k*a with k a double-double constant.
__device__ __forceinline__ dd dd_add_fast(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  s.lo = __dadd_rn(s.lo, __dadd_rn(a.lo, b.lo));
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_mul_fast(dd a, dd b) {
  double p = __dmul_rn(a.hi, b.hi);
  double e = __fma_rn(a.hi, b.hi, -p);
  e = __fma_rn(a.hi, b.lo, __fma_rn(a.lo, b.hi, e));
  return quick_two_sum(p, e);
}
// k an exact double: k*a (no addend) and d + k*a
__device__ __forceinline__ dd dd_scale_x(double k, dd a) {
  double p = __dmul_rn(k, a.hi);
  double e = __fma_rn(k, a.lo, __fma_rn(k, a.hi, -p));
  return quick_two_sum(p, e);
}
__device__ __forceinline__ dd dd_fma_x(dd d, double k, dd a) {
  double p = __dmul_rn(k, a.hi);
  double e = __fma_rn(k, a.lo, __fma_rn(k, a.hi, -p));
  dd s = two_sum(d.hi, p);
  s.lo = __dadd_rn(s.lo, __dadd_rn(d.lo, e));
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_fma_fast(dd d, dd k, dd a) {
  double p = __dmul_rn(k.hi, a.hi);
  double e = __fma_rn(k.hi, a.hi, -p);
  e = __fma_rn(k.hi, a.lo, __fma_rn(k.lo, a.hi, e));
  dd s = two_sum(d.hi, p);
  s.lo = __dadd_rn(s.lo, __dadd_rn(d.lo, e));
  return quick_two_sum(s.hi, s.lo);
}

}  // namespace aedev
