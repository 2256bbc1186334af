// Learned proposal: a small MLP that reweights the graph's own sector density.
//
// Reading of the design (the paper has no learned component; this is the
// library's extension, kept unbiased by construction):
//  * the sampler state is the set T of lines not yet ordered; the network
//    maps T (16 indicator bits, |T|/M, a constant) through three hidden
//    layers of width 64 (ReLU) to 16 outputs o_0..o_15;
//  * the learned walk removes line j from T with probability
//    softmax_j( ln[Phi(T\j)/Deg(T\j)] + 3 tanh(o_j(T)/3) ) and draws the next
//    ratio t with exponent Deg_theta(T\j) = Deg(T\j) exp(0.7 tanh(o_15(T\j)/0.7));
//    with o = 0 it is exactly the plain walk of g1;
//  * both are tabulated for all 2^M states once per network update, so the
//    per-sample cost is table look-ups and the density is exact:
//      q_theta(z) = prod_l P(j_l|S_l) prod_{l>=1} Deg_theta(S_l) t_l^Deg_theta(S_l) / prod z;
//  * evaluation uses the defensive mixture q = (1-beta) q_theta + beta g, so
//    y = I/q <= I/(beta g) and the plain density remains the fallback;
//  * training minimises -sum_i w_i ln q_theta(z_i) (forward Kullback-Leibler
//    divergence to |I|), w_i = |I(z_i)|/g(z_i) from plain samples, with Adam on
//    FP32 master weights; GEMM operands in BF16, FP32 accumulation
//    (mma.sync m16n8k16: the network is tiny, about 0.01 % of the step time, so
//    tcgen05 would buy nothing here).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "context.h"

using namespace aek;
using namespace aedev;

namespace {

constexpr int IN = 32, HID = 64, OUT = 16;
constexpr int NW1 = HID * IN, NW2 = HID * HID, NW3 = HID * HID, NW4 = OUT * HID;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NW1, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + NW2;
constexpr int OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + NW3, OFF_W4 = OFF_B3 + HID, OFF_B4 = OFF_W4 + NW4;
constexpr int NPARAM = OFF_B4 + OUT;   // 11472
constexpr double GSCALE = 1099511627776.0;   // 2^40 fixed point for gradient sums
constexpr double LAM = 3.0, KAP = 0.7;   // bounds of the logit and exponent corrections


__device__ __forceinline__ void mma16816(float c[4], const uint32_t a[4], const uint32_t b[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// One warp: Y[16 x N] = A[16 x K] * B^T with A rows in smem (bf16, row stride
// lda elements) and B stored as Bt[N][K] (bf16, row stride ldb).  Results in
// registers acc[N/8][4] with the m16n8 accumulator layout.
template <int N, int K>
__device__ __forceinline__ void warp_gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *Bt, int ldb,
                                          float acc[N / 8][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int nt = 0; nt < N / 8; ++nt)
#pragma unroll
    for (int r = 0; r < 4; ++r) acc[nt][r] = 0.f;
#pragma unroll
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t *>(A + g * lda + k0 + 2 * t);
    a[1] = *reinterpret_cast<const uint32_t *>(A + (g + 8) * lda + k0 + 2 * t);
    a[2] = *reinterpret_cast<const uint32_t *>(A + g * lda + k0 + 2 * t + 8);
    a[3] = *reinterpret_cast<const uint32_t *>(A + (g + 8) * lda + k0 + 2 * t + 8);
#pragma unroll
    for (int nt = 0; nt < N / 8; ++nt) {
      uint32_t b[2];
      b[0] = *reinterpret_cast<const uint32_t *>(Bt + (nt * 8 + g) * ldb + k0 + 2 * t);
      b[1] = *reinterpret_cast<const uint32_t *>(Bt + (nt * 8 + g) * ldb + k0 + 2 * t + 8);
      mma16816(acc[nt], a, b);
    }
  }
}

__device__ __forceinline__ float feature(uint32_t T, int M, int k) {
  if (k < 16) return (k < M && (T >> k & 1)) ? 1.f : 0.f;
  if (k == 16) return (float)__popc(T) / (float)M;
  if (k == 17) return 1.f;
  return 0.f;
}

// Forward over states [tile*64, tile*64+64): 4 warps x 16 rows.  Stores the
// post-ReLU activations (bf16) for the backward pass and the outputs (fp32).
__global__ void mlp_fwd_kernel(int M, const __nv_bfloat16 *Wbf, const float *P, __nv_bfloat16 *H1,
                               __nv_bfloat16 *H2, __nv_bfloat16 *H3, float *O) {
  __shared__ __align__(16) __nv_bfloat16 sW1[NW1], sW2[NW2], sW3[NW3], sW4[NW4];
  __shared__ __align__(16) __nv_bfloat16 sX[64 * IN], sH[2][64 * HID];
  const int S = 1 << M;
  for (int i = threadIdx.x; i < NW1; i += blockDim.x) sW1[i] = Wbf[OFF_W1 + i];
  for (int i = threadIdx.x; i < NW2; i += blockDim.x) sW2[i] = Wbf[OFF_W2 + i];
  for (int i = threadIdx.x; i < NW3; i += blockDim.x) sW3[i] = Wbf[OFF_W3 + i];
  for (int i = threadIdx.x; i < NW4; i += blockDim.x) sW4[i] = Wbf[OFF_W4 + i];
  const int row0 = blockIdx.x * 64;
  for (int i = threadIdx.x; i < 64 * IN; i += blockDim.x) {
    int r = i / IN, k = i % IN;
    uint32_t T = (uint32_t)(row0 + r);
    sX[i] = __float2bfloat16_rn(row0 + r < S ? feature(T, M, k) : 0.f);
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = w * 16;
  float acc[8][4];
  // layer 1
  warp_gemm<64, IN>(sX + r0 * IN, IN, sW1, IN, acc);
#pragma unroll
  for (int nt = 0; nt < 8; ++nt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int c0 = nt * 8 + 2 * t;
      int rr = r0 + g + 8 * h;
      float v0 = fmaxf(acc[nt][2 * h] + P[OFF_B1 + c0], 0.f);
      float v1 = fmaxf(acc[nt][2 * h + 1] + P[OFF_B1 + c0 + 1], 0.f);
      sH[0][rr * HID + c0] = __float2bfloat16_rn(v0);
      sH[0][rr * HID + c0 + 1] = __float2bfloat16_rn(v1);
    }
  __syncwarp();
  for (int i = lane; i < 16 * HID; i += 32) {
    int rr = r0 + i / HID;
    if (row0 + rr < S) H1[(size_t)(row0 + rr) * HID + i % HID] = sH[0][rr * HID + i % HID];
  }
  // layers 2 and 3
  for (int layer = 0; layer < 2; ++layer) {
    const __nv_bfloat16 *Wl = layer == 0 ? sW2 : sW3;
    const float *bl = P + (layer == 0 ? OFF_B2 : OFF_B3);
    __nv_bfloat16 *src = sH[layer & 1], *dst = sH[(layer + 1) & 1];
    warp_gemm<64, HID>(src + r0 * HID, HID, Wl, HID, acc);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int c0 = nt * 8 + 2 * t;
        int rr = r0 + g + 8 * h;
        dst[rr * HID + c0] = __float2bfloat16_rn(fmaxf(acc[nt][2 * h] + bl[c0], 0.f));
        dst[rr * HID + c0 + 1] = __float2bfloat16_rn(fmaxf(acc[nt][2 * h + 1] + bl[c0 + 1], 0.f));
      }
    __syncwarp();
    __nv_bfloat16 *Hout = layer == 0 ? H2 : H3;
    for (int i = lane; i < 16 * HID; i += 32) {
      int rr = r0 + i / HID;
      if (row0 + rr < S) Hout[(size_t)(row0 + rr) * HID + i % HID] = dst[rr * HID + i % HID];
    }
  }
  // layer 4 (outputs), input = sH[0] (layer 3 wrote into sH[0])
  float acc4[2][4];
  warp_gemm<OUT, HID>(sH[0] + r0 * HID, HID, sW4, HID, acc4);
#pragma unroll
  for (int nt = 0; nt < 2; ++nt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int c0 = nt * 8 + 2 * t;
      int rr = row0 + r0 + g + 8 * h;
      if (rr < S) {
        O[(size_t)rr * OUT + c0] = acc4[nt][2 * h] + P[OFF_B4 + c0];
        O[(size_t)rr * OUT + c0 + 1] = acc4[nt][2 * h + 1] + P[OFF_B4 + c0 + 1];
      }
    }
}

// Tables of the learned walk for every state T.
//   lp[T*16+j]  = P(j | T) (0 for j not in T), lp2 = log2 of it;
//   lpc[T*16+j] = sum of P(j' | T) over j' <= j (in the order of j: the
//   sampler's cumulative comparison);
//   ld[T] = Deg_theta(T), ld2 = log2 Deg_theta(T), ldi = 1 / Deg_theta(T)
//   (proper nonempty T).
__global__ void tables_kernel(int M, const float *O, const double *deg, const double *wplain, double *lp,
                              double *lp2, double *lpc, double *ld, double *ld2, double *ldi) {
  uint32_t S = 1u << M, full = S - 1;
  for (uint32_t T = blockIdx.x * blockDim.x + threadIdx.x; T < S; T += gridDim.x * blockDim.x) {
    const float *o = O + (size_t)T * OUT;
    double l[16];
    double mx = -1e300;
    int cnt = __popc(T);
    for (int j = 0; j < 16; ++j) {
      l[j] = -1e300;
      if (j < M && (T >> j & 1) && cnt >= 2) {
        uint32_t R = T ^ (1u << j);
        l[j] = log(wplain[R]) + LAM * tanh((double)o[j] / LAM);
        mx = fmax(mx, l[j]);
      }
    }
    double se = 0;
    for (int j = 0; j < 16; ++j)
      if (l[j] > -1e299) se += exp(l[j] - mx);
    double lse = mx + log(se);
    double cum = 0.0;
    for (int j = 0; j < 16; ++j) {
      bool in = l[j] > -1e299;
      lp[(size_t)T * 16 + j] = in ? exp(l[j] - lse) : 0.0;
      lp2[(size_t)T * 16 + j] = in ? (l[j] - lse) * 1.4426950408889634 : 0.0;
      if (in) cum += lp[(size_t)T * 16 + j];
      lpc[(size_t)T * 16 + j] = cum;
    }
    if (T != 0 && T != full) {
      double dth = deg[T] * exp(KAP * tanh((double)o[15] / KAP));
      ld[T] = dth;
      ld2[T] = log2(dth);
      ldi[T] = 1.0 / dth;
    } else {
      ld[T] = 1.0;
      ld2[T] = 0.0;
      ldi[T] = 1.0;
    }
  }
}

// Training samples from the graph's density (the plain one; the current
// learned mixture when a proposal is refined): order[16] (descending z),
// ln t at levels 1..M-1, and w = |I|/q (q the sampling density), divided by
// sqrt(1 + R) for samples the acceptance test sends to double-double (R = 0:
// the plain weights).
// With per-sample cost c, the density minimising variance x expected cost
// is proportional to |f| / sqrt(c) rather than to |f|.
__global__ void train_gen_kernel(GraphDev G, uint64_t first, uint64_t count, uint64_t seed, uint8_t *order,
                                 float *lt, double *w, double dd_tol, double cost_ratio) {
  extern __shared__ double slots[];
  double *Sl = slots + threadIdx.x * G.nslots;   // this thread's row of the slot file
  for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x; base < count; base += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t i = base + threadIdx.x;
    if (i >= count) continue;
    double z[14], lz[14], lg;
    draw_any(G, first + i, seed, z, lz, lg);   // plain density, or the current mixture when refining
    for (int k = 0; k < G.M; ++k) Sl[k] = z[k];
    run_tape(G, Sl);
    double y, Ey;
    weight2(Sl[G.outI], Sl[G.outE], lg, y, Ey);
    double wi = isfinite(y) ? fabs(y) : 0.0;
    if (cost_ratio > 0 && fp64_rejected(G, y, Ey, dd_tol)) wi /= sqrt(1.0 + cost_ratio);
    w[i] = wi;
    int ord[14];
    for (int a = 0; a < G.M; ++a) {
      int p = a;
      while (p > 0 && lz[ord[p - 1]] < lz[a]) { ord[p] = ord[p - 1]; --p; }
      ord[p] = a;
    }
    for (int l = 0; l < 16; ++l) {
      order[i * 16 + l] = (uint8_t)(l < G.M ? ord[l] : 0);
      lt[i * 16 + l] = (l >= 1 && l < G.M) ? (float)((lz[ord[l]] - lz[ord[l - 1]]) * 0.6931471805599453) : 0.f;
    }
  }
}

// Per-CTA partial sums of w (fixed-order reduction on the host).
__global__ void wsum_kernel(const double *w, uint64_t n, double *part) {
  __shared__ double red[256];
  double s = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    s += w[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// The forward-KL loss -sum_i wn_i ln q_theta(z_i) over fixed training
// samples depends on them only through per-state sums (fixed point, 2^40;
// integer atomics: order-independent, hence deterministic), gathered once
// per training call:
//   acc[T*16+j]  (j < 15)  weight of the samples that choose line j at T,
//   accw[T]                weight of the samples that choose a line at T,
//   bpost[T]               weight of the samples that reach T by a choice,
//   acc[T*16+15]           sum of wn ln t over those samples (signed),
// since ln q_theta(z) = sum over the walk's levels of ln P(j|T) (choice) +
// ln Deg_theta(T') + Deg_theta(T') ln t (the ratio t = u^(1/Deg) drawn at the
// state T' the choice leads to).  Every sample passes through the full line
// set (level 0) and one of its M subsets with one line removed (level 1):
// those 1 + M states are summed per CTA in shared memory first and added to
// the global tables once per CTA.
__device__ __forceinline__ int hot_row(uint32_t full, uint32_t T) {
  const uint32_t gone = full ^ T;
  if (gone == 0) return 0;
  if ((gone & (gone - 1)) == 0) return __ffs(gone);   // 1 + the removed line
  return -1;
}

__global__ void stats_kernel(int M, const uint8_t *order, const float *lt, const double *w, uint64_t n,
                             double inv_wsum, unsigned long long *acc, unsigned long long *accw,
                             unsigned long long *bpost) {
  __shared__ unsigned long long sacc[15 * 16];   // level-0 state (row 0) and level-1 states (row 1 + line)
  __shared__ unsigned long long sw[15], sb[15];
  const uint32_t full = (1u << M) - 1;
  for (int i = threadIdx.x; i < 15 * 16; i += blockDim.x) sacc[i] = 0;
  for (int i = threadIdx.x; i < 15; i += blockDim.x) { sw[i] = 0; sb[i] = 0; }
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const double wn = w[i] * inv_wsum;
    if (wn == 0) continue;
    const unsigned long long qw = (unsigned long long)llrint(wn * GSCALE);
    uint32_t T = full;
    for (int l = 0; l < M - 1; ++l) {
      const int j = order[i * 16 + l];
      if (qw) {
        const int r = hot_row(full, T);
        if (r >= 0) { atomicAdd(sw + r, qw); atomicAdd(sacc + r * 16 + j, qw); }
        else { atomicAdd(accw + T, qw); atomicAdd(acc + (size_t)T * 16 + j, qw); }
      }
      T ^= 1u << j;
      const long long qc = llrint(wn * (double)lt[i * 16 + l + 1] * GSCALE);
      const int r = hot_row(full, T);
      if (qw) {
        if (r >= 0) atomicAdd(sb + r, qw);
        else atomicAdd(bpost + T, qw);
      }
      if (qc) {
        if (r >= 0) atomicAdd(sacc + r * 16 + 15, (unsigned long long)qc);
        else atomicAdd(acc + (size_t)T * 16 + 15, (unsigned long long)qc);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (1 + M) * 16; i += blockDim.x) {
    const unsigned long long v = sacc[i];
    if (!v) continue;
    const int row = i / 16, col = i % 16;
    const uint32_t T = row == 0 ? full : full ^ (1u << (row - 1));
    atomicAdd(acc + (size_t)T * 16 + col, v);
  }
  for (int r = threadIdx.x; r < 1 + M; r += blockDim.x) {
    const uint32_t T = r == 0 ? full : full ^ (1u << (r - 1));
    if (sw[r]) atomicAdd(accw + T, sw[r]);
    if (sb[r]) atomicAdd(bpost + T, sb[r]);
  }
}

// dL/do (fp32) through the tanh bounds: the choice logits take
// P(j|T) W_T - C_{T,j}; the exponent -(B_T + Deg_theta(T) L_T), B = bpost
// and L = acc[.. 15] (d/d ln Deg of -B ln Deg - Deg L).
__global__ void dout_kernel(int M, const unsigned long long *acc, const unsigned long long *accw,
                            const unsigned long long *bpost, const double *lp, const double *ld, const float *O,
                            float *dO) {
  size_t S = (size_t)1 << M;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < S * 16; i += (size_t)gridDim.x * blockDim.x) {
    int j = (int)(i & 15);
    double gq;
    if (j == 15) gq = -(double)bpost[i >> 4] / GSCALE - ld[i >> 4] * ((double)(long long)acc[i] / GSCALE);
    else gq = lp[i] * ((double)accw[i >> 4] / GSCALE) - (double)acc[i] / GSCALE;
    double o = O[i];
    double th = j == 15 ? tanh(o / KAP) : tanh(o / LAM);
    dO[i] = (float)(gq * (1.0 - th * th));
  }
}

// Per-CTA partials of the loss from the same sums:
// -[ln 2 sum C_{T,j} log2 P(j|T) + ln 2 sum B_T log2 Deg_theta(T) + sum Deg_theta(T) L_T].
__global__ void loss_kernel(int M, const unsigned long long *acc, const unsigned long long *bpost,
                            const double *lp2, const double *ld, const double *ld2, double *lossp) {
  __shared__ double red[256];
  const size_t S = (size_t)1 << M;
  double s = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < S * 16; i += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(i & 15);
    const size_t T = i >> 4;
    if (j < 15) {
      if (acc[i]) s += ((double)acc[i] / GSCALE) * lp2[i] * 0.6931471805599453;
    } else {
      if (bpost[T]) s += ((double)bpost[T] / GSCALE) * ld2[T] * 0.6931471805599453;
      if (acc[i]) s += ld[T] * ((double)(long long)acc[i] / GSCALE);
    }
  }
  red[threadIdx.x] = -s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) lossp[blockIdx.x] = red[0];
}

// Backward over a 64-state tile: dH = dZ W (tensor cores), ReLU masks, and
// per-tile partial weight gradients (FP32 on CUDA cores) written to part.
__global__ void mlp_bwd_kernel(int M, const __nv_bfloat16 *Wbf, const __nv_bfloat16 *H1, const __nv_bfloat16 *H2,
                               const __nv_bfloat16 *H3, const float *dO, float *part) {
  __shared__ __align__(16) __nv_bfloat16 sW2t[NW2], sW3t[NW3], sW4t[HID * OUT];
  __shared__ __align__(16) __nv_bfloat16 sD[64 * HID], sHa[64 * HID], sHb[64 * HID];
  __shared__ __align__(16) __nv_bfloat16 sdO[64 * OUT];
  __shared__ __nv_bfloat16 sX[64 * 18];
  const int S = 1 << M;
  const int row0 = blockIdx.x * 64;
  float *gp = part + (size_t)blockIdx.x * NPARAM;
  // transposed weights: Bt[n][k] for dH = dZ * W  (n = input unit, k = output unit)
  for (int i = threadIdx.x; i < NW2; i += blockDim.x) { int o = i / HID, in = i % HID; sW2t[in * HID + o] = Wbf[OFF_W2 + i]; }
  for (int i = threadIdx.x; i < NW3; i += blockDim.x) { int o = i / HID, in = i % HID; sW3t[in * HID + o] = Wbf[OFF_W3 + i]; }
  for (int i = threadIdx.x; i < NW4; i += blockDim.x) { int o = i / HID, in = i % HID; sW4t[in * OUT + o] = Wbf[OFF_W4 + i]; }
  for (int i = threadIdx.x; i < 64 * OUT; i += blockDim.x) {
    int r = i / OUT;
    sdO[i] = __float2bfloat16_rn(row0 + r < S ? dO[(size_t)(row0 + r) * OUT + i % OUT] : 0.f);
  }
  for (int i = threadIdx.x; i < 64 * 18; i += blockDim.x) {
    int r = i / 18, k = i % 18;
    sX[i] = __float2bfloat16_rn(row0 + r < S ? feature((uint32_t)(row0 + r), M, k) : 0.f);
  }
  auto loadH = [&](const __nv_bfloat16 *H, __nv_bfloat16 *dst) {
    for (int i = threadIdx.x; i < 64 * HID; i += blockDim.x) {
      int r = i / HID;
      dst[i] = row0 + r < S ? H[(size_t)(row0 + r) * HID + i % HID] : __float2bfloat16_rn(0.f);
    }
  };
  loadH(H3, sHa);
  __syncthreads();
  // dW4[o][h] = sum_r dO[r][o] H3[r][h]; db4[o] = sum_r dO[r][o]
  for (int i = threadIdx.x; i < NW4; i += blockDim.x) {
    int o = i / HID, h = i % HID;
    float s = 0;
    for (int r = 0; r < 64; ++r) s += __bfloat162float(sdO[r * OUT + o]) * __bfloat162float(sHa[r * HID + h]);
    gp[OFF_W4 + i] = s;
  }
  for (int o = threadIdx.x; o < OUT; o += blockDim.x) {
    float s = 0;
    for (int r = 0; r < 64; ++r) s += __bfloat162float(sdO[r * OUT + o]);
    gp[OFF_B4 + o] = s;
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int r0 = w * 16;
  float acc[8][4];
  // dZ3 = (dO W4) * [H3 > 0]
  warp_gemm<64, OUT>(sdO + r0 * OUT, OUT, sW4t, OUT, acc);
  auto store_masked = [&](const __nv_bfloat16 *Hm) {
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        int c0 = nt * 8 + 2 * t;
        int rr = r0 + g + 8 * h;
        float m0 = __bfloat162float(Hm[rr * HID + c0]) > 0.f ? 1.f : 0.f;
        float m1 = __bfloat162float(Hm[rr * HID + c0 + 1]) > 0.f ? 1.f : 0.f;
        sD[rr * HID + c0] = __float2bfloat16_rn(acc[nt][2 * h] * m0);
        sD[rr * HID + c0 + 1] = __float2bfloat16_rn(acc[nt][2 * h + 1] * m1);
      }
  };
  store_masked(sHa);
  __syncthreads();
  // dW3[o][i] = sum_r dZ3[r][o] H2[r][i]; db3
  loadH(H2, sHb);
  __syncthreads();
  auto dW = [&](int off_w, int off_b, const __nv_bfloat16 *Hin, int nin) {
    for (int i = threadIdx.x; i < HID * nin; i += blockDim.x) {
      int o = i / nin, in = i % nin;
      float s = 0;
      for (int r = 0; r < 64; ++r) s += __bfloat162float(sD[r * HID + o]) * __bfloat162float(Hin[r * HID + in]);
      gp[off_w + i] = s;
    }
    for (int o = threadIdx.x; o < HID; o += blockDim.x) {
      float s = 0;
      for (int r = 0; r < 64; ++r) s += __bfloat162float(sD[r * HID + o]);
      gp[off_b + o] = s;
    }
  };
  dW(OFF_W3, OFF_B3, sHb, HID);
  __syncthreads();
  // dZ2 = (dZ3 W3) * [H2 > 0]
  warp_gemm<64, HID>(sD + r0 * HID, HID, sW3t, HID, acc);
  __syncthreads();
  store_masked(sHb);
  __syncthreads();
  loadH(H1, sHa);
  __syncthreads();
  dW(OFF_W2, OFF_B2, sHa, HID);
  __syncthreads();
  // dZ1 = (dZ2 W2) * [H1 > 0]
  warp_gemm<64, HID>(sD + r0 * HID, HID, sW2t, HID, acc);
  __syncthreads();
  store_masked(sHa);
  __syncthreads();
  // dW1[o][k] = sum_r dZ1[r][o] x[r][k] (x in bf16 as in the forward pass)
  for (int i = threadIdx.x; i < NW1; i += blockDim.x) {
    int o = i / IN, k = i % IN;
    float s = 0;
    if (k < 18)
      for (int r = 0; r < 64; ++r) s += __bfloat162float(sD[r * HID + o]) * __bfloat162float(sX[r * 18 + k]);
    gp[OFF_W1 + i] = s;
  }
  for (int o = threadIdx.x; o < HID; o += blockDim.x) {
    float s = 0;
    for (int r = 0; r < 64; ++r) s += __bfloat162float(sD[r * HID + o]);
    gp[OFF_B1 + o] = s;
  }
}

// Sum of the per-tile partials in tile order.
__global__ void grad_reduce_kernel(const float *part, int ntiles, float *grad) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  float s = 0;
  for (int b = 0; b < ntiles; ++b) s += part[(size_t)b * NPARAM + i];
  grad[i] = s;
}

__global__ void adam_kernel(float *master, float *m, float *v, const float *grad, __nv_bfloat16 *Wbf, float *P,
                            float lr, float b1t, float b2t) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  float gr = grad[i];
  float mi = 0.9f * m[i] + 0.1f * gr;
  float vi = 0.999f * v[i] + 0.001f * gr * gr;
  m[i] = mi; v[i] = vi;
  float mh = mi / (1.f - b1t), vh = vi / (1.f - b2t);
  float x = master[i] - lr * mh / (sqrtf(vh) + 1e-8f);
  master[i] = x;
  Wbf[i] = __float2bfloat16_rn(x);
  P[i] = x;
}

__global__ void to_bf16_kernel(const float *src, __nv_bfloat16 *dst, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

// Device buffers of one proposal (carved from one allocation).
struct Net {
  __nv_bfloat16 *Wbf, *H1, *H2, *H3;
  float *P, *master, *m, *v, *grad, *O, *dO, *part;
  double *lp, *lp2, *lpc, *ld, *ld2, *ldi, *deg, *wplain, *wsum_part, *loss_part;
  unsigned long long *acc, *accw, *bpost;
  int M;
  int ntiles;
};

size_t net_bytes(int M) {
  size_t S = (size_t)1 << M;
  size_t nt = (S + 63) / 64;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  return al(NPARAM * 2) + 3 * al(S * HID * 2) + al(NPARAM * 4) * 5 + al(S * OUT * 4) * 2 + al(nt * NPARAM * 4) +
         al(S * 16 * 8) * 3 + al(S * 8) * 5 + al(1024 * 8) * 2 + al(S * 16 * 8) + al(S * 8) * 2;
}

void carve(Net &n, void *mem, int M) {
  size_t S = (size_t)1 << M;
  n.M = M;
  n.ntiles = (int)((S + 63) / 64);
  char *p = (char *)mem;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  auto take = [&](size_t b) { char *r = p; p += al(b); return (void *)r; };
  n.Wbf = (__nv_bfloat16 *)take(NPARAM * 2);
  n.H1 = (__nv_bfloat16 *)take(S * HID * 2);
  n.H2 = (__nv_bfloat16 *)take(S * HID * 2);
  n.H3 = (__nv_bfloat16 *)take(S * HID * 2);
  n.P = (float *)take(NPARAM * 4);
  n.master = (float *)take(NPARAM * 4);
  n.m = (float *)take(NPARAM * 4);
  n.v = (float *)take(NPARAM * 4);
  n.grad = (float *)take(NPARAM * 4);
  n.O = (float *)take(S * OUT * 4);
  n.dO = (float *)take(S * OUT * 4);
  n.part = (float *)take((size_t)n.ntiles * NPARAM * 4);
  n.lp = (double *)take(S * 16 * 8);
  n.lp2 = (double *)take(S * 16 * 8);
  n.ld = (double *)take(S * 8);
  n.ld2 = (double *)take(S * 8);
  n.ldi = (double *)take(S * 8);
  n.lpc = (double *)take(S * 16 * 8);
  n.deg = (double *)take(S * 8);
  n.wplain = (double *)take(S * 8);
  n.wsum_part = (double *)take(1024 * 8);
  n.loss_part = (double *)take(1024 * 8);
  n.acc = (unsigned long long *)take(S * 16 * 8);
  n.accw = (unsigned long long *)take(S * 8);
  n.bpost = (unsigned long long *)take(S * 8);
}

// forward + tables for the current weights
cudaError_t net_forward(Net &n, cudaStream_t st) {
  size_t S = (size_t)1 << n.M;
  mlp_fwd_kernel<<<n.ntiles, 128, 0, st>>>(n.M, n.Wbf, n.P, n.H1, n.H2, n.H3, n.O);
  tables_kernel<<<(unsigned)((S + 127) / 128), 128, 0, st>>>(n.M, n.O, n.deg, n.wplain, n.lp, n.lp2, n.lpc, n.ld,
                                                             n.ld2, n.ldi);
  return cudaGetLastError();
}

// The training samples' sums (device arrays; see stats_kernel).
cudaError_t net_stats(Net &n, const uint8_t *order, const float *lt, const double *w, uint64_t ns, double inv_wsum,
                      cudaStream_t st) {
  size_t S = (size_t)1 << n.M;
  cudaMemsetAsync(n.acc, 0, S * 16 * 8, st);
  cudaMemsetAsync(n.accw, 0, S * 8, st);
  cudaMemsetAsync(n.bpost, 0, S * 8, st);
  stats_kernel<<<1024, 256, 0, st>>>(n.M, order, lt, w, ns, inv_wsum, n.acc, n.accw, n.bpost);
  return cudaGetLastError();
}

// Parameter gradient of the current weights from the sums (after net_forward).
cudaError_t net_grad(Net &n, cudaStream_t st) {
  size_t S = (size_t)1 << n.M;
  dout_kernel<<<(unsigned)((S * 16 + 255) / 256), 256, 0, st>>>(n.M, n.acc, n.accw, n.bpost, n.lp, n.ld, n.O, n.dO);
  mlp_bwd_kernel<<<n.ntiles, 128, 0, st>>>(n.M, n.Wbf, n.H1, n.H2, n.H3, n.dO, n.part);
  grad_reduce_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(n.part, n.ntiles, n.grad);
  return cudaGetLastError();
}

// Loss of the current weights from the sums (after net_forward); host value.
cudaError_t net_loss(Net &n, cudaStream_t st, double *loss) {
  size_t S = (size_t)1 << n.M;
  const int gb = (int)std::min<size_t>(1024, (S * 16 + 255) / 256);
  loss_kernel<<<gb, 256, 0, st>>>(n.M, n.acc, n.bpost, n.lp2, n.ld, n.ld2, n.loss_part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  std::vector<double> lp(gb);
  e = cudaMemcpyAsync(lp.data(), n.loss_part, gb * 8, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  double s = 0;
  for (double x : lp) s += x;
  *loss = s;
  return e;
}

// Seeded initial weights: He-uniform hidden layers, zero output layer (so the
// untrained proposal is exactly the plain walk).  A small counter-based hash
// keeps the initialisation reproducible.
void init_params(std::vector<float> &p, uint64_t seed) {
  p.assign(NPARAM, 0.f);
  auto uni = [&](uint64_t i) {
    uint64_t x = (seed + 0x9E3779B97F4A7C15ull) ^ (i * 0xBF58476D1CE4E5B9ull);
    x ^= x >> 31; x *= 0x94D049BB133111EBull; x ^= x >> 29;
    return ((x >> 11) * (1.0 / 9007199254740992.0)) * 2.0 - 1.0;
  };
  auto fill = [&](int off, int cnt, int fan_in) {
    double a = std::sqrt(6.0 / fan_in);
    for (int i = 0; i < cnt; ++i) p[off + i] = (float)(a * uni(off + i));
  };
  fill(OFF_W1, NW1, 18);
  fill(OFF_W2, NW2, HID);
  fill(OFF_W3, NW3, HID);
}

}  // namespace

cudaError_t ae_learned_upload_tables() {
  return upload_elem_tables(ae_exp2_table(), ae_log2_table(), ae_fast_tables());
}

// Tables of the current proposal for the sampler (called after training).
static void attach_tables(LoadedGraph &lg, Net &n) {
  lg.dev.lP = n.lp;
  lg.dev.lP2 = n.lp2;
  lg.dev.lD = n.ld;
  lg.dev.lD2 = n.ld2;
  lg.dev.lDi = n.ldi;
  lg.dev.lPc = n.lpc;
}

// Training of a graph's proposal.  refine = false: fresh weights, samples of
// the plain density (indices from 2^40 on).  refine = true: the current
// weights go on training on samples of the current mixture (indices from
// 2^41 on), weighted |I|/q, which concentrates the data where |I| is large.
static int train_impl(ae_ctx *c, int gid, uint64_t n_train, uint64_t seed, int steps, double lr, double beta,
                      ae_train_report *rep, bool refine) {
  if (!c) return AE_ERR_ARG;
  if (c->device < 0) return ae_fail(c, AE_ERR_NODEV, "training needs a CUDA device");
  if (gid < 0 || gid >= (int)c->graphs.size()) return ae_fail(c, AE_ERR_ARG, "graph id out of range");
  if (n_train < 1024 || steps < 0 || !(lr > 0) || !(beta > 0 && beta <= 1))
    return ae_fail(c, AE_ERR_ARG, "need n_train >= 1024, steps >= 0, lr > 0, 0 < beta <= 1");
  cudaSetDevice(c->device);
  LoadedGraph &lg = c->graphs[gid];
  if (refine && (!lg.learned.mem || !lg.learned.active || lg.learned.master.size() != (size_t)NPARAM))
    return ae_fail(c, AE_ERR_STATE, "refining needs an active trained proposal");
  int M = lg.g.M();
  size_t S = (size_t)1 << M;
  cudaStream_t st = c->stream;
  auto t0 = std::chrono::steady_clock::now();
  // network and tables
  if (!refine) {
    if (lg.learned.mem) { cudaFree(lg.learned.mem); lg.learned.mem = nullptr; }
    lg.dev.lP = nullptr;
    size_t nb = net_bytes(M);
    if (cudaMalloc(&lg.learned.mem, nb) != cudaSuccess) return ae_fail(c, AE_ERR_OOM, "proposal buffers");
    lg.learned.bytes = nb;
  }
  Net n;
  carve(n, lg.learned.mem, M);
  if (!refine) {
    std::vector<double> wpl(S, 1.0), dg(S, 1.0);
    for (size_t R = 1; R + 1 < S; ++R) { dg[R] = lg.dens.deg[0][R]; wpl[R] = lg.dens.phi[0][R] / lg.dens.deg[0][R]; }
    cudaMemcpyAsync(n.deg, dg.data(), S * 8, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(n.wplain, wpl.data(), S * 8, cudaMemcpyHostToDevice, st);
  }
  std::vector<float> p;
  if (refine) p = lg.learned.master;
  else init_params(p, seed);
  cudaMemcpyAsync(n.master, p.data(), NPARAM * 4, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(n.P, p.data(), NPARAM * 4, cudaMemcpyHostToDevice, st);
  cudaMemsetAsync(n.m, 0, NPARAM * 4, st);
  cudaMemsetAsync(n.v, 0, NPARAM * 4, st);
  to_bf16_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(n.master, n.Wbf, NPARAM);
  // training data from the plain density
  uint8_t *d_order = nullptr;
  float *d_lt = nullptr;
  double *d_w = nullptr;
  if (cudaMalloc(&d_order, n_train * 16) != cudaSuccess || cudaMalloc(&d_lt, n_train * 16 * 4) != cudaSuccess ||
      cudaMalloc(&d_w, n_train * 8) != cudaSuccess) {
    cudaFree(d_order); cudaFree(d_lt); cudaFree(d_w);
    return ae_fail(c, AE_ERR_OOM, "training sample buffers");
  }
  GraphDev G = lg.dev;   // refining: the current mixture's tables are attached
  if (!refine) G.lP = nullptr;
  int bs = 64;
  while (bs < 256 && (size_t)bs * 2 * G.nslots * 8 <= 96 * 1024) bs *= 2;
  size_t smem = (size_t)bs * G.nslots * 8;
  cudaFuncSetAttribute(train_gen_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  train_gen_kernel<<<(unsigned)std::min<uint64_t>((n_train + bs - 1) / bs, (uint64_t)c->sm_count * 8), bs, smem, st>>>(
      G, refine ? 1ull << 41 : 1ull << 40, n_train, seed, d_order, d_lt, d_w, c->opts.dd_tol, c->train_cost_ratio);
  wsum_kernel<<<1024, 256, 0, st>>>(d_w, n_train, n.wsum_part);
  std::vector<double> wp(1024);
  cudaMemcpyAsync(wp.data(), n.wsum_part, 1024 * 8, cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(d_order); cudaFree(d_lt); cudaFree(d_w);
    return ae_fail(c, AE_ERR_CUDA, std::string("training data: ") + cudaGetErrorString(e));
  }
  double wsum = 0;
  for (double x : wp) wsum += x;
  double inv = wsum > 0 ? 1.0 / wsum : 0.0;
  // the samples enter the loss only through per-state sums: gather them
  // once, release the samples, and take every step on the sums alone
  e = net_stats(n, d_order, d_lt, d_w, n_train, inv, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_order); cudaFree(d_lt); cudaFree(d_w);
  double loss0 = 0, loss = 0;
  for (int s = 0; e == cudaSuccess && s <= steps; ++s) {
    e = net_forward(n, st);
    if (e == cudaSuccess && (s == 0 || s == steps)) e = net_loss(n, st, &loss);
    if (e != cudaSuccess) break;
    if (s == 0) loss0 = loss;
    if (s == steps) break;
    e = net_grad(n, st);
    if (e != cudaSuccess) break;
    float b1t = (float)std::pow(0.9, s + 1), b2t = (float)std::pow(0.999, s + 1);
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(n.master, n.m, n.v, n.grad, n.Wbf, n.P, (float)lr, b1t, b2t);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return ae_fail(c, AE_ERR_CUDA, std::string("training: ") + cudaGetErrorString(e));
  lg.learned.master.resize(NPARAM);
  cudaMemcpy(lg.learned.master.data(), n.master, NPARAM * 4, cudaMemcpyDeviceToHost);
  attach_tables(lg, n);
  lg.dev.beta = beta;
  lg.dev.l2beta = std::log2(beta);
  lg.dev.l2nbeta = beta < 1 ? std::log2(1.0 - beta) : -1e300;
  lg.learned.beta = beta;
  lg.learned.active = true;
  if (rep) {
    rep->loss_initial = loss0;
    rep->loss_final = loss;
    rep->steps = steps;
    rep->n_train = n_train;
    rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return AE_OK;
}

extern "C" int ae_train_proposal(ae_ctx *c, int gid, uint64_t n_train, uint64_t seed, int steps, double lr,
                                 double beta, ae_train_report *rep) {
  return train_impl(c, gid, n_train, seed, steps, lr, beta, rep, false);
}

extern "C" int ae_refine_proposal(ae_ctx *c, int gid, uint64_t n_train, uint64_t seed, int steps, double lr,
                                  ae_train_report *rep) {
  if (!c) return AE_ERR_ARG;
  if (gid < 0 || gid >= (int)c->graphs.size()) return ae_fail(c, AE_ERR_ARG, "graph id out of range");
  return train_impl(c, gid, n_train, seed, steps, lr, c->graphs[gid].learned.beta, rep, true);
}

extern "C" int ae_set_proposal(ae_ctx *c, int gid, int mode, double beta) {
  if (!c) return AE_ERR_ARG;
  if (gid < 0 || gid >= (int)c->graphs.size()) return ae_fail(c, AE_ERR_ARG, "graph id out of range");
  LoadedGraph &lg = c->graphs[gid];
  if (mode == 0) { lg.dev.lP = nullptr; lg.learned.active = false; return AE_OK; }
  if (mode != 1) return ae_fail(c, AE_ERR_ARG, "mode must be 0 (plain) or 1 (learned mixture)");
  if (!lg.learned.mem) return ae_fail(c, AE_ERR_STATE, "no trained proposal for this graph");
  if (!(beta > 0 && beta <= 1)) return ae_fail(c, AE_ERR_ARG, "beta must be in (0, 1]");
  Net n;
  carve(n, lg.learned.mem, lg.g.M());
  attach_tables(lg, n);
  lg.dev.beta = beta;
  lg.dev.l2beta = std::log2(beta);
  lg.dev.l2nbeta = beta < 1 ? std::log2(1.0 - beta) : -1e300;
  lg.learned.beta = beta;
  lg.learned.active = true;
  return AE_OK;
}

extern "C" int ae_set_train_cost_ratio(ae_ctx *c, double ratio) {
  if (!c) return AE_ERR_ARG;
  if (!(ratio >= 0) || !std::isfinite(ratio)) return ae_fail(c, AE_ERR_ARG, "ratio must be finite and >= 0");
  c->train_cost_ratio = ratio;
  return AE_OK;
}

extern "C" int ae_set_accept_floor(ae_ctx *c, int gid, double yfloor) {
  if (!c) return AE_ERR_ARG;
  if (gid < 0 || gid >= (int)c->graphs.size()) return ae_fail(c, AE_ERR_ARG, "graph id out of range");
  if (!(yfloor >= 0) || !std::isfinite(yfloor)) return ae_fail(c, AE_ERR_ARG, "floor must be finite and >= 0");
  c->graphs[gid].dev.yfloor = yfloor;
  return AE_OK;
}

extern "C" int ae_set_accept_width(ae_ctx *c, int gid, double width) {
  if (!c) return AE_ERR_ARG;
  if (gid < 0 || gid >= (int)c->graphs.size()) return ae_fail(c, AE_ERR_ARG, "graph id out of range");
  if (!(width >= 0) || !std::isfinite(width)) return ae_fail(c, AE_ERR_ARG, "width must be finite and >= 0");
  // the width is on the graph's contribution mult * y; the kernels test y
  c->graphs[gid].dev.ywidth = width / c->graphs[gid].g.mult;
  return AE_OK;
}

// The trained proposal: FP32 master weights and the network outputs the
// sampling tables were built from (the last forward pass of training).
extern "C" int ae_proposal_export(ae_ctx *c, int gid, float *params, float *outputs, double *beta) {
  if (!c) return AE_ERR_ARG;
  if (gid < 0 || gid >= (int)c->graphs.size()) return ae_fail(c, AE_ERR_ARG, "graph id out of range");
  LoadedGraph &lg = c->graphs[gid];
  if (!lg.learned.mem || lg.learned.master.size() != (size_t)NPARAM)
    return ae_fail(c, AE_ERR_STATE, "no trained proposal for this graph");
  if (params) std::memcpy(params, lg.learned.master.data(), NPARAM * sizeof(float));
  if (outputs) {
    Net n;
    carve(n, lg.learned.mem, lg.g.M());
    cudaSetDevice(c->device);
    cudaError_t e = cudaMemcpy(outputs, n.O, ((size_t)1 << lg.g.M()) * OUT * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return ae_fail(c, AE_ERR_CUDA, std::string("proposal_export: ") + cudaGetErrorString(e));
  }
  if (beta) *beta = lg.learned.beta;
  return AE_OK;
}

// Test entry: loss, gradient and tables for given parameters and samples
// (host buffers), on the device, without sampling or training.
extern "C" int ae_proposal_eval(ae_ctx *c, int M, const float *params, const double *deg, const double *wplain,
                                const uint8_t *order, const float *lt, const double *w, uint64_t n, double *loss,
                                float *grad, double *lp2_out, double *ld_out) {
  if (!c || !params || !deg || !wplain || !order || !lt || !w || !loss || !grad) return AE_ERR_ARG;
  if (c->device < 0) return ae_fail(c, AE_ERR_NODEV, "needs a CUDA device");
  if (M < 2 || M > 14 || n == 0) return ae_fail(c, AE_ERR_ARG, "M must be 2..14 and n > 0");
  cudaSetDevice(c->device);
  cudaStream_t st = c->stream;
  size_t S = (size_t)1 << M;
  void *mem = nullptr;
  size_t nb = net_bytes(M);
  if (cudaMalloc(&mem, nb + n * (16 + 64 + 8) + 1024) != cudaSuccess) return ae_fail(c, AE_ERR_OOM, "buffers");
  Net net;
  carve(net, mem, M);
  char *extra = (char *)mem + nb;
  uint8_t *d_order = (uint8_t *)extra;
  float *d_lt = (float *)(((uintptr_t)(extra + n * 16) + 255) & ~(uintptr_t)255);
  double *d_w = (double *)(((uintptr_t)(d_lt + n * 16) + 255) & ~(uintptr_t)255);
  cudaMemcpyAsync(net.master, params, NPARAM * 4, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(net.P, params, NPARAM * 4, cudaMemcpyHostToDevice, st);
  to_bf16_kernel<<<(NPARAM + 255) / 256, 256, 0, st>>>(net.master, net.Wbf, NPARAM);
  cudaMemcpyAsync(net.deg, deg, S * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(net.wplain, wplain, S * 8, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_order, order, n * 16, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_lt, lt, n * 16 * 4, cudaMemcpyHostToDevice, st);
  cudaMemcpyAsync(d_w, w, n * 8, cudaMemcpyHostToDevice, st);
  double wsum = 0;
  for (uint64_t i = 0; i < n; ++i) wsum += w[i];
  cudaError_t e = net_forward(net, st);
  if (e == cudaSuccess) e = net_stats(net, d_order, d_lt, d_w, n, wsum > 0 ? 1.0 / wsum : 0.0, st);
  if (e == cudaSuccess) e = net_grad(net, st);
  if (e == cudaSuccess) e = net_loss(net, st, loss);   // ends with a stream synchronisation
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(grad, net.grad, NPARAM * 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && lp2_out) e = cudaMemcpy(lp2_out, net.lp2, S * 16 * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && ld_out) e = cudaMemcpy(ld_out, net.ld, S * 8, cudaMemcpyDeviceToHost);
  cudaFree(mem);
  if (e != cudaSuccess) return ae_fail(c, AE_ERR_CUDA, std::string("proposal_eval: ") + cudaGetErrorString(e));
  return AE_OK;
}

extern "C" int ae_proposal_nparams(void) { return NPARAM; }
