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
  const double *dinv;     // 3 * 2^M: 1/deg
  const Ins *code;       // tape (32-byte instructions)
  const double *khi, *klo;
  int M, ntape, nslots, outI, outK, outE;
  int graph_id;
  double yfloor = 0;      // absolute floor on |y| in the acceptance of a value
  double ywidth = 0;      // > 0: the paper's acceptance, interval width on y <= ywidth
  double C1, C2, C3, C4, log2_fact;
  double log2C[4];        // log2 of C1..C4 (g1, g2, g3, g4 order)
  double log2phi_full[3];
  // learned proposal (null lP: plain density only)
  const double *lP = nullptr;    // 2^M x 16: P(j | T)
  const double *lP2 = nullptr;   // log2 P(j | T)
  const double *lD = nullptr;    // Deg_theta(T)
  const double *lD2 = nullptr;   // log2 Deg_theta(T)
  const double *lDi = nullptr;   // 1 / Deg_theta(T)
  const double *lPc = nullptr;   // 2^M x 16: sum of P(j' | T) over j' <= j in T
  double beta = 0.1;             // weight of the plain density in the mixture
  double l2beta = 0, l2nbeta = 0;   // log2 beta, log2 (1 - beta)
  const uint32_t *mrg = nullptr;    // MRG32k3a jump table (null: Philox4x32-10)
};

struct Partial {
  double sy_hi, sy_lo, sy2_hi, sy2_lo, sa_hi, sa_lo, max_y2;
  unsigned long long n, n_flag, n_overflow;
};


// The 2M uniforms of sample idx: draw block b gives u[2b] and u[2b+1] from
// four generator words (Philox4x32-10: counter (idx lo, idx hi, graph, b),
// key = seed; MRG32k3a: outputs 4b..4b+3 after the sample's start position).
// exact: the host's word-to-double mapping; else the two-addition form.
__device__ __forceinline__ void draw_uniforms(const GraphDev &G, uint64_t idx, uint64_t seed, double *u, bool fast) {
  const int M = G.M;
  if (G.mrg) {
    MrgState st = mrg_start(G.mrg, seed, (uint32_t)G.graph_id, idx);
    for (int b = 0; b < M; ++b) {
      const uint32_t w0 = mrg_next(st), w1 = mrg_next(st), w2 = mrg_next(st), w3 = mrg_next(st);
      u[2 * b] = fast ? u01_bits(w0, w1) : u01(w0, w1);
      u[2 * b + 1] = fast ? u01_bits(w2, w3) : u01(w2, w3);
    }
    return;
  }
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int b = 0; b < M; ++b) {
    uint32_t c[4] = {(uint32_t)idx, (uint32_t)(idx >> 32), (uint32_t)G.graph_id, (uint32_t)b};
    philox4x32_10(c, k0, k1);
    u[2 * b] = fast ? u01_bits(c[0], c[1]) : u01(c[0], c[1]);
    u[2 * b + 1] = fast ? u01_bits(c[2], c[3]) : u01(c[2], c[3]);
  }
}

// Draw one sample: z (M), log2 z (M) and log2 g.  Same steps, same order of
// IEEE operations as the host-side definition of the sampler.
static __device__ void draw_sample(const GraphDev &G, uint64_t idx, uint64_t seed, double *z, double *lz,
                            double &log2g) {
  const int M = G.M;
  double u[2 * 14 + 2];
  draw_uniforms(G, idx, seed, u, false);
  double pick = u[0];
  int comp;
  if (pick < G.C1) comp = 0;
  else if (pick < __dadd_rn(G.C1, G.C2)) comp = 1;
  else if (pick < __dadd_rn(__dadd_rn(G.C1, G.C2), G.C3)) comp = 2;
  else comp = 3;
  const uint32_t full = (1u << M) - 1;
  if (comp != 1) {
    int k = comp == 0 ? 0 : comp - 1;
    const double *phi = G.phi + ((size_t)k << M);
    const double *wt = G.wt + ((size_t)k << M);
    const double *dinv = G.dinv + ((size_t)k << M);
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
      cur = __dadd_rn(cur, __dmul_rn(dlog2t(ut), __ldg(dinv + T)));   // log2 t = log2(u) (1/Deg)
    }
    int lastj = __ffs(T) - 1;
    lz[lastj] = cur;
    double ssum = 0.0;
    for (int i = 0; i < M; ++i) { z[i] = dexp2t(lz[i]); ssum = __dadd_rn(ssum, z[i]); }
    double ls = dlog2t(ssum), rs = __ddiv_rn(1.0, ssum);
    for (int i = 0; i < M; ++i) { z[i] = __dmul_rn(z[i], rs); lz[i] = __dadd_rn(lz[i], -ls); }
  } else {
    double ssum = 0.0;
    for (int i = 0; i < M; ++i) { z[i] = -dlog2t(u[1 + i]); ssum = __dadd_rn(ssum, z[i]); }
    double ls = dlog2t(ssum), rs = __ddiv_rn(1.0, ssum);
    for (int i = 0; i < M; ++i) {
      lz[i] = __dadd_rn(dlog2t(z[i]), -ls);
      z[i] = __dmul_rn(z[i], rs);
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
  for (int k = 0; k < 4; ++k) rel = __dadd_rn(rel, dexp2t(__dadd_rn(t[k], -m)));
  log2g = __dadd_rn(m, dlog2t(rel));
}

// y = I / g with g = 2^log2g, range-safe: I * 2^(kf - lg) * 2^-kf
__device__ __forceinline__ double weight(double I, double lg) {
  double kf = floor(lg);
  double s = dexp2t(__dadd_rn(kf, -lg));
  double kc = fmin(fmax(kf, -100000.0), 100000.0);
  return ldexp(__dmul_rn(I, s), -(int)kc);
}

// weight() of I and of its error bound E with one exponential
__device__ __forceinline__ void weight2(double I, double E, double lg, double &y, double &Ey) {
  double kf = floor(lg);
  double s = dexp2t(__dadd_rn(kf, -lg));
  int kc = (int)fmin(fmax(kf, -100000.0), 100000.0);
  y = ldexp(__dmul_rn(I, s), -kc);
  Ey = ldexp(__dmul_rn(E, s), -kc);
}

// Acceptance of a value (Sec. IV.A).  The certified rounding-error bound Ey
// of y (the bound of I carried to y = I/g like I) gives the interval
// [y - Ey, y + Ey].  With a graph width set (G.ywidth > 0) the paper's test
// of Eq. eq_interval_accept applies: the interval's width 2 Ey must not
// exceed ywidth.  Otherwise the library's relative test: Ey <= tol *
// max(|y|, yfloor); tol <= 0 accepts every finite value.  For the
// double-double twin the bound is scaled from the FP64 unit 2^-53 to 2^-100
// (the double-double operations' unit with a margin for the non-normalising
// additions).
__device__ __forceinline__ bool fp64_rejected(const GraphDev &G, double y, double Ey, double tol) {
  if (!isfinite(y) || !isfinite(Ey)) return true;
  if (G.ywidth > 0) return 2.0 * Ey > G.ywidth;
  return tol > 0 && Ey > tol * fmax(fabs(y), G.yfloor);
}
__device__ __forceinline__ bool dd_rejected(const GraphDev &G, double y, double Ey, double tol) {
  if (!isfinite(y) || !isfinite(Ey)) return true;
  if (G.ywidth > 0) return 2.0 * (Ey * 0x1p-47) > G.ywidth;
  return tol > 0 && Ey * 0x1p-47 > tol * fmax(fabs(y), G.yfloor);
}

// Defensive mixture q = (1-beta) q_theta + beta g.  u[0] < beta selects the
// plain density (its component pick rescaled to u[0]/beta), otherwise the
// learned walk; the returned log2 density is that of the mixture,
//   log2 q = log2( (1-beta) 2^{log2 q_theta} + sum_k beta C_k 2^{log2 g_k} ),
// one log-sum-exp over five terms.  This path is checked statistically
// (normalisation, unbiasedness), not operation by operation against the
// host, so it uses fused-multiply-add exp2/log2 (fexp2/flog2: faster than
// the forms without fused multiply-adds that draw_sample shares with the
// host) and a reciprocal table of the exponents (products instead of
// quotients).
static __device__ void draw_mix(const GraphDev &G, uint64_t idx, uint64_t seed, double *z, double *lz, double &log2q) {
  const int M = G.M;
  double u[2 * 14 + 2];
  draw_uniforms(G, idx, seed, u, true);
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
        cur += flog2(u[2 + 2 * l]) / __ldg(deg + T);
      }
      lz[__ffs(T) - 1] = cur;
    } else {
      for (int i = 0; i < M; ++i) lz[i] = flog2(-flog2(u[1 + i]));
    }
  } else {
    uint32_t T = full;
    double cur = 0.0;
    for (int l = 0; l < M - 1; ++l) {
      // first j in T whose cumulative probability exceeds the uniform (the
      // cumulative sums are tabulated in the order of j)
      double uc = u[1 + 2 * l];
      int chosen = 31 - __clz(T);   // the last j in T, if rounding leaves uc above every sum
      for (int j = 0; j < M; ++j) {
        if (!(T >> j & 1)) continue;
        if (uc < __ldg(G.lPc + (size_t)T * 16 + j)) { chosen = j; break; }
      }
      lz[chosen] = cur;
      T ^= 1u << chosen;
      cur += flog2(u[2 + 2 * l]) * __ldg(G.lDi + T);
    }
    lz[__ffs(T) - 1] = cur;
  }
  // normalise: z = 2^lz / sum, log2 z = lz - log2 sum
  double ssum = 0.0;
  for (int i = 0; i < M; ++i) { z[i] = fexp2(lz[i]); ssum += z[i]; }
  const double ls = flog2(ssum), rs = 1.0 / ssum;
  for (int i = 0; i < M; ++i) { z[i] = z[i] * rs; lz[i] = lz[i] - ls; }
  // sector order at z (descending log2 z, ties by lower index)
  int ord[14];
  for (int i = 0; i < M; ++i) {
    int p = i;
    while (p > 0 && lz[ord[p - 1]] < lz[i]) { ord[p] = ord[p - 1]; --p; }
    ord[p] = i;
  }
  double sumlz = 0.0;
  for (int i = 0; i < M; ++i) sumlz += lz[i];
  // five log2 terms: beta C_k g_k (k = g1, g2, g3, g4) and (1 - beta) q_theta
  double t[5];
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
    t[slot] = G.log2C[slot] - G.log2phi_full[k] + acc - sumlz + G.l2beta;
  }
  t[1] = G.log2C[1] + G.log2_fact + G.l2beta;
  {
    uint32_t T = full;
    double lq = 0.0, prev = 0.0;
    for (int l = 0; l < M - 1; ++l) {
      int j = ord[l];
      lq += __ldg(G.lP2 + (size_t)T * 16 + j);
      T ^= 1u << j;
      double cv = lz[ord[l + 1]];
      double pv = l == 0 ? lz[ord[0]] : prev;
      lq += __ldg(G.lD2 + T) + __ldg(G.lD + T) * (cv - pv);
      prev = cv;
    }
    t[4] = lq - sumlz + G.l2nbeta;
  }
  double m = fmax(fmax(fmax(t[0], t[1]), fmax(t[2], t[3])), t[4]);
  double rel = 0.0;
  for (int k = 0; k < 5; ++k) rel += fexp2(t[k] - m);
  log2q = m + flog2(rel);
}

__device__ __forceinline__ void draw_any(const GraphDev &G, uint64_t idx, uint64_t seed, double *z, double *lz,
                                         double &lg) {
  if (G.lP) draw_mix(G, idx, seed, z, lz, lg);
  else draw_sample(G, idx, seed, z, lz, lg);
}

// x if flag != 0, else y
__device__ __forceinline__ double sel64(uint32_t flag, double x, double y) {
  double r;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %3, 0;\n\tselp.f64 %0, %1, %2, q;\n\t}"
      : "=d"(r) : "d"(x), "d"(y), "r"(flag));
  return r;
}

// The rare instructions (division, |a|, c + |a|), kept out of the loop body.
static __device__ __noinline__ double special_op(uint32_t sp, double va, double vb, double vc) {
  if (sp == I_DIV) return __ddiv_rn(va, vb);
  if (sp == I_ABS) return fabs(va);
  return __dadd_rn(vc, fabs(va));   // I_ADDABS
}

// Clears the sign bit of x when m = 0x7fffffff (m = 0xffffffff: x unchanged).
__device__ __forceinline__ double absmask(double x, uint32_t m) {
  return __hiloint2double(__double2hiint(x) & (int)m, __double2loint(x));
}

// One tape instruction on this thread's slot row Sb:
//   S[d] = S[a] * (kb | S[b]) + (kc | S[c])   or a special operation;
// with I_AB the operands enter as absolute values (magnitude twins of the
// error bound), by a sign mask rather than a branch.
__device__ __forceinline__ void tape_step(const uint4 &w0, const uint4 &w1, char *Sb) {
  const uint32_t op = w0.x & 0xffffu, d = w0.x >> 16, a = w0.y & 0xffffu, b = w0.y >> 16, c = w0.z & 0xffffu;
  const uint32_t m = ~((op & I_AB) << 29);   // I_AB = 4: bit 31
  const double va = absmask(*reinterpret_cast<const double *>(Sb + a), m);
  const double vb = absmask(sel64(op & I_BK, __hiloint2double((int)w1.y, (int)w1.x), *reinterpret_cast<const double *>(Sb + b)), m);
  const double vc = absmask(sel64(op & I_CK, __hiloint2double((int)w1.w, (int)w1.z), *reinterpret_cast<const double *>(Sb + c)), m);
  const uint32_t sp = op & 0xff00u;
  *reinterpret_cast<double *>(Sb + d) = sp == 0 ? __fma_rn(va, vb, vc) : special_op(sp, va, vb, vc);
}

// FP64 tape interpreter reading instructions from global memory (next one
// prefetched).  Used by the kernels whose threads do not run the tape in step
// (parity dumps, training samples); the integration kernels stream the tape
// through shared memory instead (run_tape_staged).
__device__ __forceinline__ void run_tape(const GraphDev &G, double *S) {
  char *Sb = reinterpret_cast<char *>(S);
  const uint4 *code = reinterpret_cast<const uint4 *>(G.code);
  const int n = G.ntape;
  uint4 w0 = __ldg(code), w1 = __ldg(code + 1);
#pragma unroll 1
  for (int pc = 0; pc < n; ++pc) {
    const int nx = 2 * min(pc + 1, n - 1);
    const uint4 n0 = __ldg(code + nx), n1 = __ldg(code + nx + 1);
    tape_step(w0, w1, Sb);
    w0 = n0; w1 = n1;
  }
}

// ------------------------------------------------ tape staging (TMA) ----
// The integration kernels run the tape CTA-synchronously: every thread of a
// CTA evaluates its own sample, all of them step through the same tape
// segment by segment, and the segments are copied global -> shared memory by
// the bulk-copy engine (cp.async.bulk, completion on an mbarrier), two
// buffers deep, so that instruction fetch is a shared-memory broadcast
// instead of a per-warp L1/L2 round trip.
constexpr int kSeg = 128;                               // instructions per segment
constexpr int kSegBytes = kSeg * (int)sizeof(Ins);      // 4 KB
constexpr int kStageBytes = 2 * kSegBytes;              // both buffers
constexpr long long kWaitCycles = 4000000000ll;         // bound of one wait (~2 s)

struct Stage {
  Ins *buf;             // 2 x kSeg instructions, shared memory
  uint64_t *bar;        // 2 mbarriers, shared memory
  uint32_t issued;      // segments issued (thread 0's view)
  uint32_t used;        // segments consumed (identical in every thread)
  long long wait;       // bound of one wait in clock cycles (kWaitCycles)
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// thread 0; the caller synchronises the CTA afterwards
__device__ __forceinline__ void stage_init(Stage &st) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(st.bar)) : "memory");
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_addr(st.bar + 1)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// thread 0: copy segment seg of G's tape into the next buffer.  The buffer's
// previous contents must have been consumed by every thread (the caller
// issues after a CTA barrier).
__device__ __forceinline__ void stage_issue(Stage &st, const GraphDev &G, int seg) {
  const int k = st.issued & 1;
  const int cnt = min(kSeg, G.ntape - seg * kSeg);
  const uint32_t bytes = (uint32_t)cnt * (uint32_t)sizeof(Ins);
  const uint32_t bar = smem_addr(st.bar + k), dst = smem_addr(st.buf + k * kSeg);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               :: "r"(dst), "l"(G.code + (size_t)seg * kSeg), "r"(bytes), "r"(bar) : "memory");
  ++st.issued;
}

// wait (bounded by st.wait cycles) until segment number k has landed in its
// buffer; false if the wait ran out
__device__ __forceinline__ bool stage_wait_seg(const Stage &st, uint32_t k) {
  const uint32_t bar = smem_addr(st.bar + (k & 1)), parity = (k >> 1) & 1;
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    if (done) return true;
    if (clock64() - t0 > st.wait) return false;
  }
}

// every thread: wait until the next segment to consume has landed
__device__ __forceinline__ bool stage_wait(const Stage &st) { return stage_wait_seg(st, st.used); }

// thread 0, after a wait ran out: wait (again bounded) for the copies it
// issued that were not consumed, so that none is still writing into the
// CTA's shared memory when the CTA leaves
__device__ __forceinline__ void stage_drain(const Stage &st) {
  for (uint32_t k = st.used; k < st.issued; ++k) (void)stage_wait_seg(st, k);
}

// All threads of the CTA together: run G's tape on this thread's row (only
// if active).  Segment 0 must have been issued; if `again` the tape is
// rerun next (the next round of samples), and its segment 0 is issued while
// the last segment executes.  Returns false (in every thread) if a wait ran
// out; *err is set and the caller must leave the kernel.
static __device__ bool run_tape_staged(Stage &st, const GraphDev &G, double *S, bool active, bool again, int *err) {
  char *Sb = reinterpret_cast<char *>(S);
  const int nseg = (G.ntape + kSeg - 1) / kSeg;
  for (int s = 0; s < nseg; ++s) {
    const bool ok = stage_wait(st);
    // after this barrier every thread has finished segment s-1: its buffer
    // may be refilled
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) { atomicExch(err, 1); stage_drain(st); }
      return false;
    }
    if (threadIdx.x == 0) {
      if (s + 1 < nseg) stage_issue(st, G, s + 1);
      else if (again) stage_issue(st, G, 0);
    }
    const uint4 *code = reinterpret_cast<const uint4 *>(st.buf + (st.used & 1) * kSeg);
    const int cnt = min(kSeg, G.ntape - s * kSeg);
    ++st.used;
    if (!active) continue;
    uint4 w0 = code[0], w1 = code[1];
#pragma unroll 1
    for (int k = 0; k < cnt; ++k) {
      const int nx = 2 * min(k + 1, cnt - 1);
      const uint4 n0 = code[nx], n1 = code[nx + 1];
      tape_step(w0, w1, Sb);
      w0 = n0; w1 = n1;
    }
  }
  return true;
}

// One double-double tape instruction on this thread's row Sb (hi/lo pairs;
// the instruction's byte offsets scaled by 2; constants with their low parts
// from the pool).  Magnitude twins stay in FP64 (their low parts are zero);
// the compiler's hints I_KX, I_C0, I_B1 select the shorter exact forms of a
// product, a scaling and a sum.
__device__ __forceinline__ void tape_step_dd(const uint4 &w0, const uint4 &w1, char *Sb, const double *khi,
                                             const double *klo) {
  const uint32_t op = w0.x & 0xffffu, d = (w0.x >> 16) * 2, a = (w0.y & 0xffffu) * 2, b = (w0.y >> 16) * 2,
                 c = (w0.z & 0xffffu) * 2, kbi = w0.z >> 16, kci = w0.w & 0xffffu;
  const dd va = *reinterpret_cast<const dd *>(Sb + a);
  // exact constants (I_KX) come from the instruction's immediates, others
  // with their low parts from the pool
  const dd vb = !(op & I_BK) ? *reinterpret_cast<const dd *>(Sb + b)
                : (op & I_KX) ? dd{__hiloint2double((int)w1.y, (int)w1.x), 0.0}
                              : dd{__ldg(khi + kbi), __ldg(klo + kbi)};
  const dd vc = !(op & I_CK) ? *reinterpret_cast<const dd *>(Sb + c)
                : (op & I_KX) ? dd{__hiloint2double((int)w1.w, (int)w1.z), 0.0}
                              : dd{__ldg(khi + kci), __ldg(klo + kci)};
  dd r;
  const uint32_t sp = op & 0xff00u;
  if (op & I_AB) r = dd{__fma_rn(fabs(va.hi), fabs(vb.hi), fabs(vc.hi)), 0.0};   // magnitudes: FP64 is enough
  else if (sp == 0) {
    // the compiler's hints pick the shortest exact form of c + a*b
    const bool bx = (op & (I_BK | I_KX)) == (I_BK | I_KX);   // b an exact constant
    if (op & I_C0) r = bx ? dd_scale_x(vb.hi, va) : dd_mul_fast(va, vb);
    else if (op & I_B1) r = dd_add_fast(vc, vb.hi > 0 ? va : dd{-va.hi, -va.lo});
    else if (bx) r = dd_fma_x(vc, vb.hi, va);
    else r = dd_fma_fast(vc, vb, va);
  }
  else if (sp == I_DIV) r = dd_div(va, vb);
  else if (sp == I_ABS) r = dd_abs(va);
  else r = dd_add_fast(vc, dd_abs(va));   // I_ADDABS
  *reinterpret_cast<dd *>(Sb + d) = r;
}

// Double-double twin of run_tape, instructions read from global memory (next
// one prefetched): the per-sample dumps.
static __device__ void run_tape_dd(const GraphDev &G, dd *S) {
  char *Sb = reinterpret_cast<char *>(S);
  const uint4 *code = reinterpret_cast<const uint4 *>(G.code);
  const int n = G.ntape;
  if (n <= 0) return;
  uint4 w0 = __ldg(code), w1 = __ldg(code + 1);
  for (int pc = 0; pc < n; ++pc) {
    const int nx = 2 * min(pc + 1, n - 1);
    const uint4 n0 = __ldg(code + nx), n1 = __ldg(code + nx + 1);
    tape_step_dd(w0, w1, Sb, G.khi, G.klo);
    w0 = n0; w1 = n1;
  }
}

// Double-double twin of run_tape_staged: all threads of the CTA step through
// the same tape segments in shared memory (same staging, same bounded waits);
// segment 0 must have been issued.  Returns false (in every thread) if a wait
// ran out; *err is set and the caller must leave the kernel.
static __device__ bool run_tape_dd_staged(Stage &st, const GraphDev &G, dd *S, bool active, int *err) {
  char *Sb = reinterpret_cast<char *>(S);
  const int nseg = (G.ntape + kSeg - 1) / kSeg;
  const double *khi = G.khi, *klo = G.klo;
  for (int s = 0; s < nseg; ++s) {
    const bool ok = stage_wait(st);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) { atomicExch(err, 1); stage_drain(st); }
      return false;
    }
    if (threadIdx.x == 0 && s + 1 < nseg) stage_issue(st, G, s + 1);
    const uint4 *code = reinterpret_cast<const uint4 *>(st.buf + (st.used & 1) * kSeg);
    const int cnt = min(kSeg, G.ntape - s * kSeg);
    ++st.used;
    if (!active) continue;
    uint4 w0 = code[0], w1 = code[1];
#pragma unroll 1
    for (int k = 0; k < cnt; ++k) {
      const int nx = 2 * min(k + 1, cnt - 1);
      const uint4 n0 = code[nx], n1 = code[nx + 1];
      tape_step_dd(w0, w1, Sb, khi, klo);
      w0 = n0; w1 = n1;
    }
  }
  return true;
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

// Warp reduction of the per-lane accumulators (fixed tree: lane 0 holds the
// result, the same for any schedule).
__device__ __forceinline__ void warp_reduce(Partial &p) {
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
}

// Block reduction of the per-thread accumulators into one Partial.
static __device__ void block_reduce(Partial p, Partial *out) {
  __shared__ Partial red[32];
  warp_reduce(p);
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
