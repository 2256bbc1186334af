// Device-side pieces shared by the integration and training kernels:
// per-graph device descriptor, sampler and density, the FP64 tape and its
// double-double twin, accumulators and the CTA reduction.
#pragma once
#include <cstdint>

#include "ae_internal.h"
#include "device.cuh"

namespace aek {
using namespace ae;
using namespace aedev;

// ------------------------------------------------------------ structs ----
struct GraphDev {
  const double *deg;      // 3 * 2^M
  const double *phi;      // 3 * 2^M
  const double *wt;       // 3 * 2^M: phi/deg (same IEEE quotient as the walk's definition)
  const uint2 *code;      // tape
  const double *khi, *klo;
  int M, ntape, nslots, outI, outK;
  int graph_id;
  double C1, C2, C3, C4, log2_fact;
  double log2C[4];        // log2 of C1..C4 (g1, g2, g3, g4 order)
  double log2phi_full[3];
  // learned proposal (null lP: plain density only)
  const double *lP = nullptr;    // 2^M x 16: P(j | T)
  const double *lP2 = nullptr;   // log2 P(j | T)
  const double *lD = nullptr;    // Deg_theta(T)
  const double *lD2 = nullptr;   // log2 Deg_theta(T)
  double beta = 0.1;             // weight of the plain density in the mixture
};

struct Partial {
  double sy_hi, sy_lo, sy2_hi, sy2_lo, sa_hi, sa_lo, max_y2;
  unsigned long long n, n_flag, n_overflow;
};


// Draw one sample: z (M), log2 z (M) and log2 g.  Same steps, same order of
// IEEE operations as the host-side definition of the sampler.
static __device__ void draw_sample(const GraphDev &G, uint64_t idx, uint64_t seed, double *z, double *lz,
                            double &log2g) {
  const int M = G.M;
  double u[2 * 14 + 2];
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  int nb = M;
  for (int b = 0; b < nb; ++b) {
    uint32_t c[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), (uint32_t)G.graph_id, (uint32_t)b};
    philox4x32_10(c, k0, k1);
    u[2 * b] = u01(c[0], c[1]);
    u[2 * b + 1] = u01(c[2], c[3]);
  }
  double pick = u[0];
  int comp;
  if (pick < G.C1) comp = 0;
  else if (pick < __dadd_rn(G.C1, G.C2)) comp = 1;
  else if (pick < __dadd_rn(__dadd_rn(G.C1, G.C2), G.C3)) comp = 2;
  else comp = 3;
  const uint32_t full = (1u << M) - 1;
  if (comp != 1) {
    int k = comp == 0 ? 0 : comp - 1;
    const double *deg = G.deg + ((size_t)k << M);
    const double *phi = G.phi + ((size_t)k << M);
    const double *wt = G.wt + ((size_t)k << M);
    uint32_t T = full;
    double cur = 0.0;
    for (int l = 0; l < M - 1; ++l) {
      double uc = u[1 + 2 * l], ut = u[2 + 2 * l];
      double target = __dmul_rn(uc, __ldg(phi + T));
      double acc = 0.0;
      int chosen = -1, last = 0;
      for (int j = 0; j < M; ++j) {
        if (!(T >> j & 1)) continue;
        uint32_t R = T ^ (1u << j);
        acc = __dadd_rn(acc, __ldg(wt + R));
        if (chosen < 0 && target < acc) chosen = j;
        last = j;
      }
      if (chosen < 0) chosen = last;
      lz[chosen] = cur;
      T ^= 1u << chosen;
      cur = __dadd_rn(cur, __ddiv_rn(dlog2(ut), __ldg(deg + T)));
    }
    int lastj = __ffs(T) - 1;
    lz[lastj] = cur;
    double ssum = 0.0;
    for (int i = 0; i < M; ++i) { z[i] = dexp2(lz[i]); ssum = __dadd_rn(ssum, z[i]); }
    double ls = dlog2(ssum);
    for (int i = 0; i < M; ++i) { z[i] = __ddiv_rn(z[i], ssum); lz[i] = __dadd_rn(lz[i], -ls); }
  } else {
    double ssum = 0.0;
    for (int i = 0; i < M; ++i) { z[i] = -dlog2(u[1 + i]); ssum = __dadd_rn(ssum, z[i]); }
    double ls = dlog2(ssum);
    for (int i = 0; i < M; ++i) {
      lz[i] = __dadd_rn(dlog2(z[i]), -ls);
      z[i] = __ddiv_rn(z[i], ssum);
    }
  }
  // density: sector order = descending log2 z, ties by lower index
  int ord[14];
  for (int i = 0; i < M; ++i) {
    int p = i;
    while (p > 0 && lz[ord[p - 1]] < lz[i]) { ord[p] = ord[p - 1]; --p; }
    ord[p] = i;
  }
  double sumlz = 0.0;
  for (int i = 0; i < M; ++i) sumlz = __dadd_rn(sumlz, lz[i]);
  double t[4];
  for (int k = 0; k < 3; ++k) {
    const double *deg = G.deg + ((size_t)k << M);
    double acc = 0.0;
    uint32_t T = full ^ (1u << ord[0]);
    double prev = lz[ord[0]];
    for (int l = 1; l < M; ++l) {
      double cv = lz[ord[l]];
      acc = __dadd_rn(acc, __dmul_rn(__ldg(deg + T), __dadd_rn(cv, -prev)));
      prev = cv;
      T ^= 1u << ord[l];
    }
    int slot = k == 0 ? 0 : k + 1;
    t[slot] = __dadd_rn(__dadd_rn(__dadd_rn(G.log2C[slot], -G.log2phi_full[k]), acc), -sumlz);
  }
  t[1] = __dadd_rn(G.log2C[1], G.log2_fact);
  double m = t[0];
  for (int k = 1; k < 4; ++k) m = fmax(m, t[k]);
  double rel = 0.0;
  for (int k = 0; k < 4; ++k) rel = __dadd_rn(rel, dexp2(__dadd_rn(t[k], -m)));
  log2g = __dadd_rn(m, dlog2(rel));
}

// y = I / g with g = 2^log2g, range-safe: I * 2^(kf - lg) * 2^-kf
__device__ __forceinline__ double weight(double I, double lg) {
  double kf = floor(lg);
  double s = dexp2(__dadd_rn(kf, -lg));
  double kc = fmin(fmax(kf, -100000.0), 100000.0);
  return ldexp(__dmul_rn(I, s), -(int)kc);
}

// Defensive mixture q = (1-beta) q_theta + beta g.  u[0] < beta selects the
// plain density (its component pick rescaled to u[0]/beta), otherwise the
// learned walk; the returned log2 density is that of the mixture.
static __device__ void draw_mix(const GraphDev &G, uint64_t idx, uint64_t seed, double *z, double *lz, double &log2q) {
  const int M = G.M;
  double u[2 * 14 + 2];
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int b = 0; b < M; ++b) {
    uint32_t c[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), (uint32_t)G.graph_id, (uint32_t)b};
    philox4x32_10(c, k0, k1);
    u[2 * b] = u01(c[0], c[1]);
    u[2 * b + 1] = u01(c[2], c[3]);
  }
  const uint32_t full = (1u << M) - 1;
  bool plain = u[0] < G.beta;
  if (plain) {
    double pick = u[0] / G.beta;
    int comp;
    if (pick < G.C1) comp = 0;
    else if (pick < G.C1 + G.C2) comp = 1;
    else if (pick < G.C1 + G.C2 + G.C3) comp = 2;
    else comp = 3;
    if (comp != 1) {
      int k = comp == 0 ? 0 : comp - 1;
      const double *deg = G.deg + ((size_t)k << M);
      const double *wt = G.wt + ((size_t)k << M);
      const double *phi = G.phi + ((size_t)k << M);
      uint32_t T = full;
      double cur = 0.0;
      for (int l = 0; l < M - 1; ++l) {
        double target = u[1 + 2 * l] * __ldg(phi + T);
        double acc = 0.0;
        int chosen = -1, last = 0;
        for (int j = 0; j < M; ++j) {
          if (!(T >> j & 1)) continue;
          acc += __ldg(wt + (T ^ (1u << j)));
          if (chosen < 0 && target < acc) chosen = j;
          last = j;
        }
        if (chosen < 0) chosen = last;
        lz[chosen] = cur;
        T ^= 1u << chosen;
        cur += dlog2(u[2 + 2 * l]) / __ldg(deg + T);
      }
      lz[__ffs(T) - 1] = cur;
    } else {
      for (int i = 0; i < M; ++i) lz[i] = dlog2(-dlog2(u[1 + i]));
    }
  } else {
    uint32_t T = full;
    double cur = 0.0;
    for (int l = 0; l < M - 1; ++l) {
      double uc = u[1 + 2 * l];
      double acc = 0.0;
      int chosen = -1, last = 0;
      for (int j = 0; j < M; ++j) {
        if (!(T >> j & 1)) continue;
        acc += __ldg(G.lP + (size_t)T * 16 + j);
        if (chosen < 0 && uc < acc) chosen = j;
        last = j;
      }
      if (chosen < 0) chosen = last;
      lz[chosen] = cur;
      T ^= 1u << chosen;
      cur += dlog2(u[2 + 2 * l]) / __ldg(G.lD + T);
    }
    lz[__ffs(T) - 1] = cur;
  }
  // normalise: z = 2^lz / sum, log2 z = lz - log2 sum
  double ssum = 0.0;
  for (int i = 0; i < M; ++i) { z[i] = dexp2(lz[i]); ssum += z[i]; }
  double ls = dlog2(ssum);
  for (int i = 0; i < M; ++i) { z[i] = z[i] / ssum; lz[i] = lz[i] - ls; }
  // densities at z
  int ord[14];
  for (int i = 0; i < M; ++i) {
    int p = i;
    while (p > 0 && lz[ord[p - 1]] < lz[i]) { ord[p] = ord[p - 1]; --p; }
    ord[p] = i;
  }
  double sumlz = 0.0;
  for (int i = 0; i < M; ++i) sumlz += lz[i];
  double t[4];
  for (int k = 0; k < 3; ++k) {
    const double *deg = G.deg + ((size_t)k << M);
    double acc = 0.0;
    uint32_t T = full ^ (1u << ord[0]);
    double prev = lz[ord[0]];
    for (int l = 1; l < M; ++l) {
      double cv = lz[ord[l]];
      acc += __ldg(deg + T) * (cv - prev);
      prev = cv;
      T ^= 1u << ord[l];
    }
    int slot = k == 0 ? 0 : k + 1;
    t[slot] = G.log2C[slot] - G.log2phi_full[k] + acc - sumlz;
  }
  t[1] = G.log2C[1] + G.log2_fact;
  double m = fmax(fmax(t[0], t[1]), fmax(t[2], t[3]));
  double rel = 0.0;
  for (int k = 0; k < 4; ++k) rel += dexp2(t[k] - m);
  double lg = m + dlog2(rel);
  // learned density along the same order
  double lq = 0.0;
  {
    uint32_t T = full;
    double prev = 0.0;
    for (int l = 0; l < M - 1; ++l) {
      int j = ord[l];
      lq += __ldg(G.lP2 + (size_t)T * 16 + j);
      T ^= 1u << j;
      double cv = lz[ord[l + 1]];
      double pv = l == 0 ? lz[ord[0]] : prev;
      lq += __ldg(G.lD2 + T) + __ldg(G.lD + T) * (cv - pv);
      prev = cv;
    }
    lq -= sumlz;
  }
  double a = dlog2(1.0 - G.beta) + lq, b = dlog2(G.beta) + lg;
  double mm = fmax(a, b);
  log2q = mm + dlog2(dexp2(a - mm) + dexp2(b - mm));
}

__device__ __forceinline__ void draw_any(const GraphDev &G, uint64_t idx, uint64_t seed, double *z, double *lz,
                                         double &lg) {
  if (G.lP) draw_mix(G, idx, seed, z, lz, lg);
  else draw_sample(G, idx, seed, z, lz, lg);
}

// Horner-stack cases of the interpreters: level k accumulates into R##k and
// reads its child level from R##k1.
#define AE_HCASES(k, k1)                                                             \
  case T_HFL + k: R##k = __fma_rn(S[a * stride], __ldg(K + b), __ldg(K + d)); break; \
  case T_HL + k: R##k = __fma_rn(S[a * stride], __ldg(K + b), R##k); break;          \
  case T_HFU + k: R##k = __fma_rn(S[a * stride], R##k1, __ldg(K + d)); break;        \
  case T_HU + k: R##k = __fma_rn(S[a * stride], R##k1, R##k); break;
#define AE_HCASES_ALL                                                                \
  AE_HCASES(0, 1) AE_HCASES(1, 2) AE_HCASES(2, 3) AE_HCASES(3, 4) AE_HCASES(4, 5)     \
  AE_HCASES(5, 6) AE_HCASES(6, 7) AE_HCASES(7, 8) AE_HCASES(8, 9) AE_HCASES(9, 10)    \
  AE_HCASES(10, 11)
static_assert(kHLevels == 12, "interpreter cases cover Horner levels 0..10 (degree <= 11)");

// FP64 tape interpreter.  S points at this thread's column of the slot file
// (stride = blockDim.x); r is the register accumulator of monomial chains and
// R0..R11 the Horner stack.  The next instruction word is fetched while the
// current one executes.
__device__ __forceinline__ void run_tape(const GraphDev &G, double *S, int stride) {
  const uint2 *code = G.code;
  const double *K = G.khi;
  const int n = G.ntape;
  double r = 0.0;
  double R0 = 0, R1 = 0, R2 = 0, R3 = 0, R4 = 0, R5 = 0, R6 = 0, R7 = 0, R8 = 0, R9 = 0, R10 = 0, R11 = 0;
  uint2 w = __ldg(code);
  for (int pc = 0; pc < n; ++pc) {
    uint2 wn = __ldg(code + min(pc + 1, n - 1));
    int op = w.x & 0xff;
    int d = w.x >> 16;
    int a = w.y & 0xffff;
    int b = w.y >> 16;
    double *D = S + d * stride;
    switch (op) {
      case T_RFMAC: r = __fma_rn(__ldg(K + b), S[a * stride], r); break;
      case T_MUL: *D = __dmul_rn(S[a * stride], S[b * stride]); break;
      case T_RFMA: r = __fma_rn(S[a * stride], S[b * stride], r); break;
      case T_RZERO: r = 0.0; break;
      case T_RST: *D = r; break;
      case T_ADD: *D = __dadd_rn(S[a * stride], S[b * stride]); break;
      case T_SUB: *D = __dadd_rn(S[a * stride], -S[b * stride]); break;
      case T_DIV: *D = __ddiv_rn(S[a * stride], S[b * stride]); break;
      case T_FMA: *D = __fma_rn(S[a * stride], S[b * stride], *D); break;
      case T_FMAC: *D = __fma_rn(__ldg(K + b), S[a * stride], *D); break;
      case T_MULC: *D = __dmul_rn(__ldg(K + b), S[a * stride]); break;
      case T_CONST: *D = __ldg(K + b); break;
      case T_ABS: *D = fabs(S[a * stride]); break;
      case T_NEG: *D = -S[a * stride]; break;
      case T_ZERO: *D = 0.0; break;
      case T_ADDABS: *D = __dadd_rn(*D, fabs(S[a * stride])); break;
      AE_HCASES_ALL
      case T_HST: *D = R0; break;
      default: break;
    }
    w = wn;
  }
}

// Double-double twin of run_tape (slot file holds hi/lo pairs).
static __device__ void run_tape_dd(const GraphDev &G, dd *S, int stride) {
  dd r = {0.0, 0.0};
  dd R[kHLevels];
#pragma unroll
  for (int k = 0; k < kHLevels; ++k) R[k] = {0.0, 0.0};
  for (int pc = 0; pc < G.ntape; ++pc) {
    uint2 w = __ldg(G.code + pc);
    int op = w.x & 0xff, d = w.x >> 16, a = w.y & 0xffff, b = w.y >> 16;
    if (op >= T_HFL && op < T_HST) {
      // Horner stack: unrolled over the levels so that R stays in registers
      const int kind = op & ~15, lvl = op & 15;
      dd x = S[a * stride];
      dd kb = {0, 0}, kd = {0, 0};
      if (kind == T_HFL || kind == T_HL) kb = {__ldg(G.khi + b), __ldg(G.klo + b)};
      if (kind == T_HFL || kind == T_HFU) kd = {__ldg(G.khi + d), __ldg(G.klo + d)};
#pragma unroll
      for (int k = 0; k < kHLevels - 1; ++k) {
        if (k != lvl) continue;
        dd m = (kind == T_HFL || kind == T_HL) ? kb : R[k + 1];
        dd acc = (kind == T_HFL || kind == T_HFU) ? kd : R[k];
        R[k] = dd_fma_fast(acc, m, x);
      }
      continue;
    }
    dd *D = S + d * stride;
    dd kb = {0, 0};
    if (op == T_FMAC || op == T_MULC || op == T_CONST || op == T_RFMAC) kb = {__ldg(G.khi + b), __ldg(G.klo + b)};
    switch (op) {
      case T_RZERO: r = {0.0, 0.0}; break;
      case T_RFMAC: r = dd_fma_fast(r, kb, S[a * stride]); break;
      case T_RFMA: r = dd_fma_fast(r, S[a * stride], S[b * stride]); break;
      case T_RST: *D = r; break;
      case T_ADD: *D = dd_add_fast(S[a * stride], S[b * stride]); break;
      case T_SUB: { dd t = S[b * stride]; *D = dd_add_fast(S[a * stride], {-t.hi, -t.lo}); } break;
      case T_MUL: *D = dd_mul_fast(S[a * stride], S[b * stride]); break;
      case T_DIV: *D = dd_div(S[a * stride], S[b * stride]); break;
      case T_FMA: *D = dd_fma_fast(*D, S[a * stride], S[b * stride]); break;
      case T_FMAC: *D = dd_fma_fast(*D, kb, S[a * stride]); break;
      case T_MULC: *D = dd_mul_fast(kb, S[a * stride]); break;
      case T_CONST: *D = kb; break;
      case T_ABS: *D = dd_abs(S[a * stride]); break;
      case T_NEG: { dd t = S[a * stride]; *D = {-t.hi, -t.lo}; } break;
      case T_ZERO: *D = {0.0, 0.0}; break;
      case T_ADDABS: *D = dd_add_fast(*D, dd_abs(S[a * stride])); break;
      case T_HST: *D = R[0]; break;
      default: break;
    }
  }
}

__device__ __forceinline__ void dd_acc(double &hi, double &lo, double x) {
  dd s = two_sum(hi, x);
  lo = __dadd_rn(lo, s.lo);
  dd r = quick_two_sum(s.hi, lo);
  hi = r.hi; lo = r.lo;
}

__device__ __forceinline__ void dd_merge(double &hi, double &lo, double h2, double l2) {
  dd r = dd_add({hi, lo}, {h2, l2});
  hi = r.hi; lo = r.lo;
}

// Block reduction of the per-thread accumulators into one Partial.
static __device__ void block_reduce(Partial p, Partial *out) {
  __shared__ Partial red[32];
  const unsigned full = 0xffffffffu;
  for (int off = 16; off > 0; off >>= 1) {
    Partial q;
    q.sy_hi = __shfl_down_sync(full, p.sy_hi, off); q.sy_lo = __shfl_down_sync(full, p.sy_lo, off);
    q.sy2_hi = __shfl_down_sync(full, p.sy2_hi, off); q.sy2_lo = __shfl_down_sync(full, p.sy2_lo, off);
    q.sa_hi = __shfl_down_sync(full, p.sa_hi, off); q.sa_lo = __shfl_down_sync(full, p.sa_lo, off);
    q.max_y2 = __shfl_down_sync(full, p.max_y2, off);
    q.n = __shfl_down_sync(full, p.n, off); q.n_flag = __shfl_down_sync(full, p.n_flag, off);
    q.n_overflow = __shfl_down_sync(full, p.n_overflow, off);
    dd_merge(p.sy_hi, p.sy_lo, q.sy_hi, q.sy_lo);
    dd_merge(p.sy2_hi, p.sy2_lo, q.sy2_hi, q.sy2_lo);
    dd_merge(p.sa_hi, p.sa_lo, q.sa_hi, q.sa_lo);
    p.max_y2 = fmax(p.max_y2, q.max_y2);
    p.n += q.n; p.n_flag += q.n_flag; p.n_overflow += q.n_overflow;
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = p;
  __syncthreads();
  if (threadIdx.x == 0) {
    Partial r = red[0];
    int nw = (blockDim.x + 31) >> 5;
    for (int w = 1; w < nw; ++w) {
      dd_merge(r.sy_hi, r.sy_lo, red[w].sy_hi, red[w].sy_lo);
      dd_merge(r.sy2_hi, r.sy2_lo, red[w].sy2_hi, red[w].sy2_lo);
      dd_merge(r.sa_hi, r.sa_lo, red[w].sa_hi, red[w].sa_lo);
      r.max_y2 = fmax(r.max_y2, red[w].max_y2);
      r.n += red[w].n; r.n_flag += red[w].n_flag; r.n_overflow += red[w].n_overflow;
    }
    *out = r;
  }
}


}  // namespace aek
