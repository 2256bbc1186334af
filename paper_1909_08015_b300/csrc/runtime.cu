// libae runtime: the C ABI of include/ae.h, device memory for the loaded
// graph set, and the integration kernels for sm_103a.
//
// Hot path (one launch per graph, or one persistent launch for a batch):
//   Philox4x32-10 (or MRG32k3a) -> mixture pick -> Hepp-sector walk
//   (Deg/Phi tables, or the learned tables) -> log2 g -> tape interpreter
//   (FP64 fused multiply-adds on a per-thread slot row in shared memory; the
//   tape streamed into shared memory segment by segment by TMA bulk copies,
//   all threads of a CTA stepping through it together) -> y = I/g ->
//   double-double accumulation of sum y, sum y^2, sum |y| -> warp-shuffle
//   and CTA reduction -> one partial per CTA (or chunk), summed on the host
//   in fixed order.
// Every FP64 evaluation carries a certified rounding-error bound E of I (the
// tape's magnitude twins).  Samples whose bound, carried to y, exceeds
// dd_tol * max(|y|, the graph's floor on |y|), or whose value is not finite,
// are queued and re-evaluated by the double-double kernel, which applies the
// same test at its own unit; samples that fail it too count as zero.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <thread>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <stdexcept>
#include <string>
#include <vector>

#include "context.h"

using namespace ae;
using namespace aek;
using namespace aedev;

int ae_fail(ae_ctx *c, int code, const std::string &msg) {
  if (c) c->err = msg;
  return code;
}
static int fail(ae_ctx *c, int code, const std::string &msg) { return ae_fail(c, code, msg); }
#define CUDA_TRY(c, x)                                                        \
  do {                                                                        \
    cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess)                                                    \
      return fail(c, e_ == cudaErrorMemoryAllocation ? AE_ERR_OOM : AE_ERR_CUDA, \
                  std::string(#x) + ": " + cudaGetErrorString(e_));            \
  } while (0)

// Process samples [first, first + count) of one graph; CTA b takes a
// contiguous chunk in rounds of blockDim.x samples (one per thread), each
// round's tapes run together, staged through shared memory.
// wait_cycles bounds every wait for a tape segment (kWaitCycles in normal
// use); skip_first (test hook only) leaves out the copy of the first segment,
// so that the first wait runs out with nothing in flight.
__global__ void integrate_kernel(GraphDev Gp, uint64_t first, uint64_t count, uint64_t seed,
                                 double dd_tol, Partial *part, unsigned long long *queue,
                                 unsigned long long qcap, unsigned long long *qcount, int *err,
                                 long long wait_cycles, int skip_first) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(16) unsigned char Gmem[sizeof(GraphDev)];   // raw: no dynamic initialisation
  GraphDev &G = *reinterpret_cast<GraphDev *>(Gmem);
  __shared__ uint64_t bars[2];
  Stage st{reinterpret_cast<Ins *>(dsm), bars, 0, 0, wait_cycles};
  if (threadIdx.x == 0) { G = Gp; stage_init(st); }
  __syncthreads();
  double *S = reinterpret_cast<double *>(dsm + kStageBytes) + threadIdx.x * G.nslots;   // this thread's row
  uint64_t chunk = (count + gridDim.x - 1) / gridDim.x;
  uint64_t lo = (uint64_t)blockIdx.x * chunk;
  uint64_t hi = min(count, lo + chunk);
  Partial p = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  double z[14], lz[14];
  if (threadIdx.x == 0 && lo < hi && !skip_first) stage_issue(st, G, 0);
  for (uint64_t base = lo; base < hi; base += blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    const bool active = i < hi;
    const uint64_t idx = first + i;
    double lg = 0.0;
    if (active) {
      draw_any(G, idx, seed, z, lz, lg);
      for (int k = 0; k < G.M; ++k) S[k] = z[k];
    }
    if (!run_tape_staged(st, G, S, active, base + blockDim.x < hi, err)) return;
    if (!active) continue;
    double y, Ey;
    weight2(S[G.outI], S[G.outE], lg, y, Ey);
    const bool bad = fp64_rejected(G, y, Ey, dd_tol);
    p.n += 1;
    if (bad) {
      p.n_flag += 1;
      unsigned long long slot = atomicAdd(qcount, 1ull);
      if (slot < qcap) queue[slot] = idx;
      else p.n_overflow += 1;
      continue;
    }
    dd_acc(p.sy_hi, p.sy_lo, y);
    dd_acc(p.sy2_hi, p.sy2_lo, y * y);
    dd_acc(p.sa_hi, p.sa_lo, fabs(y));
    p.max_y2 = fmax(p.max_y2, y * y);
  }
  block_reduce(p, part + blockIdx.x);
}

// Double-double re-evaluation of one graph's queued samples, written to the
// sample's dense slot (offset from `first`): y and a flag (1 re-evaluated, 2
// still failing -> the sample counts as zero).  CTA-synchronous with the
// tape staged through shared memory: item k = entries k*blockDim ..
// (k+1)*blockDim-1 of the queue, items taken in grid-stride order.
__global__ void dd_staged_kernel(GraphDev Gp, uint64_t seed, const unsigned long long *queue, uint64_t nq,
                                 double dd_tol, uint64_t first, double *ydense, unsigned char *fdense, int *err) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(16) unsigned char Gmem[sizeof(GraphDev)];   // raw: no dynamic initialisation
  GraphDev &G = *reinterpret_cast<GraphDev *>(Gmem);
  __shared__ uint64_t bars[2];
  Stage st{reinterpret_cast<Ins *>(dsm), bars, 0, 0, kWaitCycles};
  if (threadIdx.x == 0) { G = Gp; stage_init(st); }
  __syncthreads();
  dd *S = reinterpret_cast<dd *>(dsm + kStageBytes) + threadIdx.x * G.nslots;   // this thread's row
  double z[14], lz[14];
  const uint64_t items = (nq + blockDim.x - 1) / blockDim.x;
  for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
    if (threadIdx.x == 0) stage_issue(st, G, 0);
    const uint64_t i = it * blockDim.x + threadIdx.x;
    const bool active = i < nq;
    double lg = 0.0;
    if (active) {
      draw_any(G, queue[i], seed, z, lz, lg);
      for (int k = 0; k < G.M; ++k) S[k] = dd{z[k], 0.0};
    }
    if (!run_tape_dd_staged(st, G, S, active, err)) return;
    if (active) {
      double y, Ey;
      weight2(S[G.outI].hi + S[G.outI].lo, S[G.outE].hi, lg, y, Ey);
      const bool bad = dd_rejected(G, y, Ey, dd_tol);
      ydense[queue[i] - first] = bad ? 0.0 : y;
      fdense[queue[i] - first] = bad ? 2 : 1;
    }
    __syncthreads();   // every thread is done with the last segment's buffer
  }
}

// Per-sample dump for parity tests, through the same CTA-synchronous staged
// interpreter as integrate_kernel and batched_kernel: CTA b takes the b-th
// contiguous chunk of [0, count) and steps through it blockDim samples at a
// time, so that a small grid runs several rounds per CTA (segment 0 of the
// next round issued while the last segment of this one executes).
__global__ void eval_kernel(GraphDev Gp, uint64_t first, uint64_t count, uint64_t seed, double *z_out,
                            double *lg_out, double *I_out, double *K_out, double *y_out, double *E_out, int *err) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(16) unsigned char Gmem[sizeof(GraphDev)];   // raw: no dynamic initialisation
  GraphDev &G = *reinterpret_cast<GraphDev *>(Gmem);
  __shared__ uint64_t bars[2];
  Stage st{reinterpret_cast<Ins *>(dsm), bars, 0, 0, kWaitCycles};
  if (threadIdx.x == 0) { G = Gp; stage_init(st); }
  __syncthreads();
  double *S = reinterpret_cast<double *>(dsm + kStageBytes) + threadIdx.x * G.nslots;   // this thread's row
  const uint64_t chunk = (count + gridDim.x - 1) / gridDim.x;
  const uint64_t lo = (uint64_t)blockIdx.x * chunk;
  const uint64_t hi = min(count, lo + chunk);
  double z[14], lz[14];
  if (threadIdx.x == 0 && lo < hi) stage_issue(st, G, 0);
  for (uint64_t base = lo; base < hi; base += blockDim.x) {
    const uint64_t i = base + threadIdx.x;
    const bool active = i < hi;
    double lg = 0.0;
    if (active) {
      draw_any(G, first + i, seed, z, lz, lg);
      for (int k = 0; k < G.M; ++k) { S[k] = z[k]; z_out[i * G.M + k] = z[k]; }
    }
    if (!run_tape_staged(st, G, S, active, base + blockDim.x < hi, err)) return;
    if (!active) continue;
    const double I = S[G.outI];
    lg_out[i] = lg; I_out[i] = I; K_out[i] = S[G.outK]; y_out[i] = weight(I, lg); E_out[i] = S[G.outE];
  }
}

// Per-sample dump with every sample evaluated in double-double, through the
// staged double-double interpreter of the re-evaluation pass: item k =
// samples k*blockDim .. (k+1)*blockDim-1, items taken in grid-stride order.
__global__ void eval_dd_kernel(GraphDev Gp, uint64_t first, uint64_t count, uint64_t seed, double *I_out,
                               double *K_out, double *y_out, double *E_out, int *err) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ __align__(16) unsigned char Gmem[sizeof(GraphDev)];   // raw: no dynamic initialisation
  GraphDev &G = *reinterpret_cast<GraphDev *>(Gmem);
  __shared__ uint64_t bars[2];
  Stage st{reinterpret_cast<Ins *>(dsm), bars, 0, 0, kWaitCycles};
  if (threadIdx.x == 0) { G = Gp; stage_init(st); }
  __syncthreads();
  dd *S = reinterpret_cast<dd *>(dsm + kStageBytes) + threadIdx.x * G.nslots;   // this thread's row
  double z[14], lz[14];
  const uint64_t items = (count + blockDim.x - 1) / blockDim.x;
  for (uint64_t it = blockIdx.x; it < items; it += gridDim.x) {
    if (threadIdx.x == 0) stage_issue(st, G, 0);
    const uint64_t i = it * blockDim.x + threadIdx.x;
    const bool active = i < count;
    double lg = 0.0;
    if (active) {
      draw_any(G, first + i, seed, z, lz, lg);
      for (int k = 0; k < G.M; ++k) S[k] = dd{z[k], 0.0};
    }
    if (!run_tape_dd_staged(st, G, S, active, err)) return;
    if (active) {
      const double Iv = S[G.outI].hi + S[G.outI].lo;
      I_out[i] = Iv; K_out[i] = S[G.outK].hi + S[G.outK].lo; y_out[i] = weight(Iv, lg);
      E_out[i] = S[G.outE].hi * 0x1p-47;   // bound at the double-double unit
    }
    __syncthreads();   // every thread is done with the last segment's buffer
  }
}

// FP64 peak probe: independent DFMA chains, 8 per thread, no memory traffic.
__global__ void dfma_probe_kernel(int iters, double a, double b, double *sink) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = threadIdx.x * 1e-9 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = __fma_rn(x[k], a, b);
  }
  double s = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  if (s == 1234.5678) sink[0] = s;   // keeps the chains alive
}

__global__ void philox_kernel(const uint32_t *ctr, const uint32_t *key, uint32_t *out, size_t count) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  uint32_t c[4] = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
  philox4x32_10(c, key[2 * i], key[2 * i + 1]);
  for (int k = 0; k < 4; ++k) out[4 * i + k] = c[k];
}

// ------------------------------------------------- batched persistent ----
// One chunk of work: samples [first, first + count) of graph gi.
struct Chunk {
  int gi;
  int pad;
  unsigned long long first, count;
};

// Persistent kernel over a queue of chunks from many graphs (tapes of very
// different lengths).  CTAs take chunks in list order through one atomic
// counter; each chunk's partial is written to its own slot, so the result does
// not depend on which CTA ran it.  Flagged samples go to the queue as
// (graph, sample index).
__global__ void batched_kernel(const GraphDev *graphs, const Chunk *chunks, int nchunks, uint64_t seed,
                               double dd_tol, Partial *part, unsigned long long *queue_idx, int *queue_gi,
                               unsigned long long qcap, unsigned long long *qcount, int *next, int *err) {
  // chunks/part point at this launch's slice of the chunk list
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ int cur, curg;
  __shared__ __align__(16) unsigned char Gmem[sizeof(GraphDev)];   // raw: no dynamic initialisation
  GraphDev &G = *reinterpret_cast<GraphDev *>(Gmem);               // descriptor of the current chunk's graph
  __shared__ uint64_t bars[2];
  Stage st{reinterpret_cast<Ins *>(dsm), bars, 0, 0, kWaitCycles};
  double z[14], lz[14];
  if (threadIdx.x == 0) { curg = -1; stage_init(st); }
  for (;;) {
    if (threadIdx.x == 0) {
      cur = atomicAdd(next, 1);
      if (cur < nchunks && chunks[cur].gi != curg) { curg = chunks[cur].gi; G = graphs[curg]; }
      if (cur < nchunks && chunks[cur].count > 0) stage_issue(st, G, 0);
    }
    __syncthreads();
    int c = cur;
    if (c >= nchunks) break;
    const Chunk ch = chunks[c];
    // this thread's row of the slot file (pitch of the current graph; the
    // launch reserves the largest pitch of its bucket)
    double *S = reinterpret_cast<double *>(dsm + kStageBytes) + threadIdx.x * G.nslots;
    Partial p = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (uint64_t base = 0; base < ch.count; base += blockDim.x) {
      const uint64_t i = base + threadIdx.x;
      const bool active = i < ch.count;
      const uint64_t idx = ch.first + i;
      double lg = 0.0;
      if (active) {
        draw_any(G, idx, seed, z, lz, lg);
        for (int k = 0; k < G.M; ++k) S[k] = z[k];
      }
      if (!run_tape_staged(st, G, S, active, base + blockDim.x < ch.count, err)) return;
      if (!active) continue;
      double y, Ey;
      weight2(S[G.outI], S[G.outE], lg, y, Ey);
      const bool bad = fp64_rejected(G, y, Ey, dd_tol);
      p.n += 1;
      if (bad) {
        p.n_flag += 1;
        unsigned long long slot = atomicAdd(qcount, 1ull);
        if (slot < qcap) { queue_idx[slot] = idx; queue_gi[slot] = ch.gi; }
        else p.n_overflow += 1;
        continue;
      }
      dd_acc(p.sy_hi, p.sy_lo, y);
      dd_acc(p.sy2_hi, p.sy2_lo, y * y);
      dd_acc(p.sa_hi, p.sa_lo, fabs(y));
      p.max_y2 = fmax(p.max_y2, y * y);
    }
    block_reduce(p, part + c);
    __syncthreads();
  }
}

// Counting sort of the re-evaluation queue by graph (so that the warps of the
// double-double pass run one tape each): histogram, exclusive scan, scatter.
__global__ void queue_hist_kernel(const int *queue_gi, const unsigned long long *qcount, unsigned long long qcap,
                                  const int *rank, unsigned int *hist) {
  uint64_t nq = min(*qcount, qcap);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(hist + rank[queue_gi[i]], 1u);
}
__global__ void queue_scan_kernel(unsigned int *hist, int ngraphs) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    unsigned int acc = 0;
    for (int g = 0; g < ngraphs; ++g) { unsigned int v = hist[g]; hist[g] = acc; acc += v; }
  }
}
__global__ void queue_scatter_kernel(const unsigned long long *qi, const int *qg, const unsigned long long *qcount,
                                     unsigned long long qcap, const int *rank, unsigned int *offs,
                                     unsigned long long *qi2, int *qg2) {
  uint64_t nq = min(*qcount, qcap);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (uint64_t)gridDim.x * blockDim.x) {
    unsigned int pos = atomicAdd(offs + rank[qg[i]], 1u);
    qi2[pos] = qi[i];
    qg2[pos] = qg[i];
  }
}

// Work plan of the staged double-double pass over the graph-sorted queue:
// rank r (a graph, in bucket order) holds entries [end_{r-1}, end_r) and is
// cut into work items of B_r consecutive entries (B_r = the block size of
// its bucket's launch); wstart[r] = first item of rank r, wstart[nranks] =
// the total.  One thread: at most a few thousand ranks.
__global__ void dd_plan_kernel(const unsigned int *hist_end, const int *rank_bs, int nranks, unsigned int *wstart) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  unsigned int acc = 0;
  for (int r = 0; r < nranks; ++r) {
    const unsigned int beg = r ? hist_end[r - 1] : 0u, cnt = hist_end[r] - beg;
    wstart[r] = acc;
    acc += (cnt + (unsigned int)rank_bs[r] - 1) / (unsigned int)rank_bs[r];
  }
  wstart[nranks] = acc;
}

// Double-double re-evaluation of the batched queue, CTA-synchronous like the
// FP64 kernel: a CTA takes a work item (blockDim consecutive entries of one
// graph, ranks r0..r1 of this launch's bucket) through an atomic counter,
// every thread draws its entry's sample, and all step through the graph's
// tape together, the segments staged into shared memory by bulk copies.
// Results go to the samples' dense slots (flag 1 = re-evaluated, 2 = failed
// again -> counts as zero).  Counts are read on the device, so the launch
// shape is fixed and the pass can be captured in a graph.
__global__ void batched_dd_staged_kernel(const GraphDev *graphs, uint64_t seed, const unsigned long long *qi,
                                         const int *qg, const unsigned int *hist_end, const unsigned int *wstart,
                                         int r0, int r1, const unsigned long long *gpos, double *ydense,
                                         unsigned char *fdense, int pitch, double dd_tol, int *next, int *err) {
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ unsigned int item_s;
  __shared__ int rank_s;
  __shared__ __align__(16) unsigned char Gmem[sizeof(GraphDev)];   // raw: no dynamic initialisation
  GraphDev &G = *reinterpret_cast<GraphDev *>(Gmem);               // descriptor of the current item's graph
  __shared__ uint64_t bars[2];
  Stage st{reinterpret_cast<Ins *>(dsm), bars, 0, 0, kWaitCycles};
  int curr = -1;   // thread 0: the rank whose descriptor is in G
  if (threadIdx.x == 0) stage_init(st);
  const unsigned int wbeg = wstart[r0], wend = wstart[r1 + 1];
  dd *S = reinterpret_cast<dd *>(dsm + kStageBytes) + threadIdx.x * pitch;   // this thread's row
  double z[14], lz[14];
  for (;;) {
    if (threadIdx.x == 0) {
      const unsigned int it = wbeg + (unsigned int)atomicAdd(next, 1);
      int r = -1;
      if (it < wend) {
        // the largest rank r in [r0, r1] with wstart[r] <= it; it has items
        int lo = r0, hi = r1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (wstart[mid] <= it) lo = mid; else hi = mid - 1;
        }
        r = lo;
        const unsigned int beg = r ? hist_end[r - 1] : 0u;
        if (r != curr) { G = graphs[qg[beg]]; curr = r; }
        stage_issue(st, G, 0);
      }
      item_s = it;
      rank_s = r;
    }
    __syncthreads();
    const unsigned int it = item_s;
    if (it >= wend) break;
    const int r = rank_s;
    const unsigned int beg = r ? hist_end[r - 1] : 0u, end = hist_end[r];
    const unsigned long long i = (unsigned long long)beg + (unsigned long long)(it - wstart[r]) * blockDim.x + threadIdx.x;
    const bool active = i < end;
    double lg = 0.0;
    if (active) {
      draw_any(G, qi[i], seed, z, lz, lg);
      for (int k = 0; k < G.M; ++k) S[k] = dd{z[k], 0.0};
    }
    if (!run_tape_dd_staged(st, G, S, active, err)) return;
    if (active) {
      double y, Ey;
      weight2(S[G.outI].hi + S[G.outI].lo, S[G.outE].hi, lg, y, Ey);
      const bool bad = dd_rejected(G, y, Ey, dd_tol);
      const int gq = qg[i];
      const unsigned long long pos = gpos[2 * gq] + (qi[i] - gpos[2 * gq + 1]);
      ydense[pos] = bad ? 0.0 : y;
      fdense[pos] = bad ? 2 : 1;
    }
    __syncthreads();   // the item's shared state is rewritten next
  }
}

// Re-evaluated samples of each chunk, summed in sample order: one warp per
// chunk, lane l taking offsets l, l+32, ... (flags 1 = re-evaluated, 2 =
// zeroed), then the fixed warp tree.  n_flag counts re-evaluated samples,
// n_overflow the zeroed ones.  The result does not depend on the order in
// which the double-double pass ran.
__global__ void chunk_dd_reduce_kernel(const Chunk *chunks, int nchunks, const unsigned long long *gpos,
                                       const double *ydense, const unsigned char *fdense, Partial *out) {
  const int lane = threadIdx.x & 31;
  const int warps = (int)((gridDim.x * blockDim.x) >> 5);
  for (int c = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); c < nchunks; c += warps) {
    const Chunk ch = chunks[c];
    const unsigned long long pos0 = gpos[2 * ch.gi] + (ch.first - gpos[2 * ch.gi + 1]);
    Partial p = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (unsigned long long o = lane; o < ch.count; o += 32) {
      const unsigned char f = fdense[pos0 + o];
      if (!f) continue;
      const double y = ydense[pos0 + o];
      p.n_flag += 1;
      if (f == 2) p.n_overflow += 1;
      dd_acc(p.sy_hi, p.sy_lo, y);
      dd_acc(p.sy2_hi, p.sy2_lo, y * y);
      dd_acc(p.sa_hi, p.sa_lo, fabs(y));
      p.max_y2 = fmax(p.max_y2, y * y);
    }
    warp_reduce(p);
    if (lane == 0) out[c] = p;
  }
}

// Same sums over a dense range of len samples cut into segments of seg:
// one warp per segment, segment s to out[s].
__global__ void dense_dd_reduce_kernel(uint64_t len, uint64_t seg, const double *ydense,
                                       const unsigned char *fdense, Partial *out) {
  const int lane = threadIdx.x & 31;
  const uint64_t nseg = (len + seg - 1) / seg;
  const uint64_t warps = (gridDim.x * blockDim.x) >> 5;
  for (uint64_t sg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; sg < nseg; sg += warps) {
    const uint64_t pos0 = sg * seg, cnt = min(seg, len - pos0);
    Partial p = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (uint64_t o = lane; o < cnt; o += 32) {
      const unsigned char f = fdense[pos0 + o];
      if (!f) continue;
      const double y = ydense[pos0 + o];
      p.n_flag += 1;
      if (f == 2) p.n_overflow += 1;
      dd_acc(p.sy_hi, p.sy_lo, y);
      dd_acc(p.sy2_hi, p.sy2_lo, y * y);
      dd_acc(p.sa_hi, p.sa_lo, fabs(y));
      p.max_y2 = fmax(p.max_y2, y * y);
    }
    warp_reduce(p);
    if (lane == 0) out[sg] = p;
  }
}

// ------------------------------------------- no-allocation entry point ---
// Scratch of ae_integrate_noalloc: one file-scope device array, shared by all
// calls on a device and kept between them.  Layout (bytes from the start):
//   [0, kNaPartBytes)          per-CTA partials (at most kNaMaxGrid)
//   next 256                   queue counter + final result
//   queue                      sample indices needing double-double (u64)
//   y                          double-double value per sample offset
//   flag                       1 byte per sample offset (set by the dd pass)
constexpr uint64_t kNaMaxSamples = 1ull << 19;   // samples per call
constexpr int kNaMaxGrid = 2048;                 // CTAs per launch
constexpr size_t kNaPartBytes = (size_t)kNaMaxGrid * sizeof(Partial);
constexpr size_t kNaCtlBytes = 256;
constexpr size_t kNaQueueOff = kNaPartBytes + kNaCtlBytes;
constexpr size_t kNaYOff = kNaQueueOff + kNaMaxSamples * 8;
constexpr size_t kNaFlagOff = kNaYOff + kNaMaxSamples * 8;
constexpr size_t kNaScratchBytes = kNaFlagOff + kNaMaxSamples;   // about 8.3 MB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

// Double-double pass writing by sample offset (deterministic order later).
__global__ void dd_dense_kernel(GraphDev G, uint64_t first, uint64_t seed, const unsigned long long *queue,
                                const unsigned long long *qcount, double *y_off, unsigned char *flag,
                                double dd_tol) {
  extern __shared__ dd dsl3[];
  dd *S = dsl3 + threadIdx.x * G.nslots;   // this thread's row of the slot file
  uint64_t nq = *qcount;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t idx = queue[i];
    double z[14], lz[14], lg;
    draw_any(G, idx, seed, z, lz, lg);
    for (int k = 0; k < G.M; ++k) S[k] = {z[k], 0.0};
    run_tape_dd(G, S);
    double y, Ey;
    weight2(S[G.outI].hi + S[G.outI].lo, S[G.outE].hi, lg, y, Ey);
    const bool bad = dd_rejected(G, y, Ey, dd_tol);
    y_off[idx - first] = bad ? 0.0 : y;
    flag[idx - first] = bad ? 2 : 1;
  }
}

// One CTA: partials in CTA order, then re-evaluated samples in a fixed
// strided order; result[0] = merged partial, result counters in n_flag
// (re-evaluated) and n_overflow (zeroed).
__global__ void noalloc_reduce_kernel(const Partial *part, int nparts, const double *y_off,
                                      const unsigned char *flag, uint64_t count, Partial *result) {
  Partial p = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nparts; b += blockDim.x) {
    const Partial &q = part[b];
    dd_merge(p.sy_hi, p.sy_lo, q.sy_hi, q.sy_lo);
    dd_merge(p.sy2_hi, p.sy2_lo, q.sy2_hi, q.sy2_lo);
    dd_merge(p.sa_hi, p.sa_lo, q.sa_hi, q.sa_lo);
    p.max_y2 = fmax(p.max_y2, q.max_y2);
    p.n += q.n;
  }
  for (uint64_t i = threadIdx.x; i < count; i += blockDim.x) {
    unsigned char f = flag[i];
    if (!f) continue;
    double y = y_off[i];
    dd_acc(p.sy_hi, p.sy_lo, y);
    dd_acc(p.sy2_hi, p.sy2_lo, y * y);
    dd_acc(p.sa_hi, p.sa_lo, fabs(y));
    p.max_y2 = fmax(p.max_y2, y * y);
    p.n_flag += 1;
    if (f == 2) p.n_overflow += 1;
  }
  block_reduce(p, result);
}

// ============================================================ host ABI ===
extern "C" void ae_default_opts(ae_opts *o) {
  o->C2 = 0.03; o->C3 = 0.01; o->C4 = 0.06; o->D = 0.75;
  o->C_subI = 0.2; o->C_subSE = 0.0; o->C_subO = 0.2;
  o->C_bigZ = 0.256; o->C_bigF = 0.839; o->C_add = 0.786;
  o->deg_max = 1.0;
  o->dd_tol = 1e-10;
  o->block_size = 0;
  o->ctas_per_sm = 0;
  o->stream = nullptr;
  o->rng = 0;
  o->grid_ctas = 0;
}

extern "C" void ae_calc1_opts(ae_opts *o) {
  ae_default_opts(o);
  o->C3 = 0.035; o->C4 = 0.035;
  o->rng = 1;
}

extern "C" int ae_create(ae_ctx **out, int dev, const ae_opts *opts) {
  if (!out) return AE_ERR_ARG;
  *out = nullptr;
  ae_ctx *c = new (std::nothrow) ae_ctx();
  if (!c) return AE_ERR_OOM;
  if (opts) c->opts = *opts; else ae_default_opts(&c->opts);
  if ((c->opts.rng != 0 && c->opts.rng != 1) || c->opts.grid_ctas < 0) { delete c; return AE_ERR_ARG; }
  c->device = dev;
  if (dev >= 0) {
    cudaError_t e = cudaSetDevice(dev);
    if (e != cudaSuccess) { delete c; return AE_ERR_CUDA; }
    cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, dev);
    // tables of the sampler's log2/exp2, in both units that launch sampling kernels
    e = upload_elem_tables(ae_exp2_table(), ae_log2_table(), ae_fast_tables());
    if (e == cudaSuccess) e = ae_learned_upload_tables();
    if (e != cudaSuccess) { delete c; return AE_ERR_CUDA; }
    if (c->opts.stream) {
      c->stream = (cudaStream_t)c->opts.stream;
      c->own_stream = false;
    } else if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      return AE_ERR_CUDA;
    }
  }
  *out = c;
  return AE_OK;
}

static void free_device(ae_ctx *c) {
  if (c->device < 0) return;
  cudaSetDevice(c->device);
  if (c->arena) cudaFree(c->arena);
  if (c->d_part) cudaFree(c->d_part);
  if (c->d_queue) cudaFree(c->d_queue);
  if (c->d_qcount) cudaFree(c->d_qcount);
  if (c->d_yq) cudaFree(c->d_yq);
  if (c->d_qstat) cudaFree(c->d_qstat);
  if (c->bbuf) cudaFree(c->bbuf);
  c->bbuf = nullptr;
  c->bbuf_bytes = 0;
  for (auto &lg : c->graphs)
    if (lg.learned.mem) { cudaFree(lg.learned.mem); lg.learned.mem = nullptr; lg.dev.lP = nullptr; }
  c->tune_cache.clear();
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
  c->gkey.clear();
  c->arena = nullptr; c->d_part = nullptr; c->d_queue = nullptr; c->d_qcount = nullptr;
  c->d_yq = nullptr; c->d_qstat = nullptr; c->part_cap = c->queue_cap = 0;
}

extern "C" void ae_destroy(ae_ctx *c) {
  if (!c) return;
  free_device(c);
  if (c->d_mrg) cudaFree(c->d_mrg);
  for (auto &ev : c->gev)
    if (ev) cudaEventDestroy(ev);
  if (c->stream && c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

extern "C" const char *ae_last_error(const ae_ctx *c) { return c ? c->err.c_str() : "null context"; }

static int load_impl(ae_ctx *c, int loops, const int *subset, int n_subset, int *n_out);

extern "C" int ae_load_graphs(ae_ctx *c, int loops, int *n_out) {
  return load_impl(c, loops, nullptr, 0, n_out);
}

extern "C" int ae_load_graph_subset(ae_ctx *c, int loops, const int *canonical_ids, int n_ids, int *n_out) {
  if (!c) return AE_ERR_ARG;
  if (!canonical_ids || n_ids <= 0) return fail(c, AE_ERR_ARG, "empty subset");
  return load_impl(c, loops, canonical_ids, n_ids, n_out);
}

static int load_impl(ae_ctx *c, int loops, const int *subset, int n_subset, int *n_out) {
  if (!c) return AE_ERR_ARG;
  if (loops < 1 || loops > 5) return fail(c, AE_ERR_ARG, "loops must be 1..5");
  std::vector<int> canon;
  try {
    std::vector<Graph> all = enumerate_graphs(loops);
    std::vector<Graph> gs;
    if (subset) {
      for (int k = 0; k < n_subset; ++k) {
        if (subset[k] < 0 || subset[k] >= (int)all.size()) return fail(c, AE_ERR_ARG, "canonical id out of range");
        gs.push_back(all[subset[k]]);
        canon.push_back(subset[k]);
      }
    } else {
      gs = all;
      for (size_t k = 0; k < all.size(); ++k) canon.push_back((int)k);
    }
    DensityConsts dc;
    dc.C2 = c->opts.C2; dc.C3 = c->opts.C3; dc.C4 = c->opts.C4; dc.D = c->opts.D;
    dc.CsubI = c->opts.C_subI; dc.CsubSE = c->opts.C_subSE; dc.CsubO = c->opts.C_subO;
    dc.deg_max = c->opts.deg_max;
    std::vector<LoadedGraph> L(gs.size());
    // graphs compile independently: spread them over the host's cores
    std::atomic<size_t> next(0);
    std::vector<std::string> errs(gs.size());
    auto worker = [&]() {
      for (size_t i = next++; i < gs.size(); i = next++) {
        try {
          L[i].g = gs[i];
          L[i].subs = divergent_subgraphs(gs[i]);
          L[i].terms = rnew_terms(gs[i], L[i].subs);
          L[i].tape = compile_integrand(gs[i], &L[i].st);
          L[i].dens = build_density(gs[i], dc);
          L[i].canonical_id = canon[i];
        } catch (std::exception &e) {
          errs[i] = e.what();
        }
      }
    };
    unsigned nt = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), 64u));
    std::vector<std::thread> th;
    for (unsigned t = 0; t < nt; ++t) th.emplace_back(worker);
    for (auto &t : th) t.join();
    for (size_t i = 0; i < gs.size(); ++i)
      if (!errs[i].empty()) throw std::runtime_error("graph " + std::to_string(i) + ": " + errs[i]);
    free_device(c);
    c->graphs.swap(L);
    c->loops = loops;
    c->run.assign(c->graphs.size(), ae_run_graph{});
    c->run_seed = 0;
  } catch (std::exception &e) {
    return fail(c, AE_ERR_STATE, std::string("load_graphs: ") + e.what());
  }
  if (c->device >= 0) {
    // one arena: per graph deg, phi, konst hi, konst lo, code
    size_t bytes = 0;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    for (auto &lg : c->graphs) {
      size_t T = (size_t)1 << lg.g.M();
      bytes += al(3 * T * 8) * 4 + al(lg.tape.khi.size() * 8) * 2 + al(lg.tape.code.size() * sizeof(Ins));
    }
    CUDA_TRY(c, cudaMalloc(&c->arena, bytes));
    c->arena_bytes = bytes;
    if (c->opts.rng == 1 && !c->d_mrg) {
      CUDA_TRY(c, cudaMalloc(&c->d_mrg, 160 * 18 * sizeof(uint32_t)));
      CUDA_TRY(c, cudaMemcpy(c->d_mrg, mrg_jump_table(), 160 * 18 * sizeof(uint32_t), cudaMemcpyHostToDevice));
    }
    char *p = (char *)c->arena;
    for (size_t gi = 0; gi < c->graphs.size(); ++gi) {
      LoadedGraph &lg = c->graphs[gi];
      size_t T = (size_t)1 << lg.g.M();
      std::vector<double> deg(3 * T), phi(3 * T), wt(3 * T, 0.0), dinv(3 * T, 0.0);
      for (int k = 0; k < 3; ++k) {
        std::copy(lg.dens.deg[k].begin(), lg.dens.deg[k].end(), deg.begin() + k * T);
        std::copy(lg.dens.phi[k].begin(), lg.dens.phi[k].end(), phi.begin() + k * T);
        for (size_t R = 1; R + 1 < T; ++R) {
          wt[k * T + R] = lg.dens.phi[k][R] / lg.dens.deg[k][R];
          dinv[k * T + R] = 1.0 / lg.dens.deg[k][R];
        }
      }
      GraphDev &G = lg.dev;
      G.deg = (double *)p; CUDA_TRY(c, cudaMemcpy(p, deg.data(), 3 * T * 8, cudaMemcpyHostToDevice)); p += al(3 * T * 8);
      G.phi = (double *)p; CUDA_TRY(c, cudaMemcpy(p, phi.data(), 3 * T * 8, cudaMemcpyHostToDevice)); p += al(3 * T * 8);
      G.wt = (double *)p; CUDA_TRY(c, cudaMemcpy(p, wt.data(), 3 * T * 8, cudaMemcpyHostToDevice)); p += al(3 * T * 8);
      G.dinv = (double *)p; CUDA_TRY(c, cudaMemcpy(p, dinv.data(), 3 * T * 8, cudaMemcpyHostToDevice)); p += al(3 * T * 8);
      size_t nk = lg.tape.khi.size();
      G.khi = (double *)p; if (nk) CUDA_TRY(c, cudaMemcpy(p, lg.tape.khi.data(), nk * 8, cudaMemcpyHostToDevice)); p += al(nk * 8);
      G.klo = (double *)p; if (nk) CUDA_TRY(c, cudaMemcpy(p, lg.tape.klo.data(), nk * 8, cudaMemcpyHostToDevice)); p += al(nk * 8);
      G.code = (const Ins *)p;
      CUDA_TRY(c, cudaMemcpy(p, lg.tape.code.data(), lg.tape.code.size() * sizeof(Ins), cudaMemcpyHostToDevice));
      p += al(lg.tape.code.size() * sizeof(Ins));
      G.M = lg.g.M(); G.ntape = (int)lg.tape.code.size(); G.nslots = lg.tape.nslots;
      G.outI = lg.tape.out_I; G.outK = lg.tape.out_K; G.outE = lg.tape.out_E; G.graph_id = canon[gi];   // random stream of the graph
      G.mrg = c->opts.rng == 1 ? c->d_mrg : nullptr;
      lg.canonical_id = canon[gi];
      G.C1 = lg.dens.C[0]; G.C2 = lg.dens.C[1]; G.C3 = lg.dens.C[2]; G.C4 = lg.dens.C[3];
      G.log2_fact = lg.dens.log2_fact;
      for (int k = 0; k < 4; ++k) G.log2C[k] = ae_log2t(lg.dens.C[k]);
      for (int k = 0; k < 3; ++k) G.log2phi_full[k] = ae_log2t(lg.dens.phi[k][T - 1]);
    }
  }
  if (n_out) *n_out = (int)c->graphs.size();
  return AE_OK;
}

extern "C" int ae_graph_info(ae_ctx *c, int id, ae_graph_meta *o) {
  if (!c || !o) return AE_ERR_ARG;
  if (id < 0 || id >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  const LoadedGraph &lg = c->graphs[id];
  std::memset(o, 0, sizeof(*o));
  o->loops = lg.g.n; o->M = lg.g.M(); o->mult = lg.g.mult;
  for (int k = 0; k < 3; ++k) o->klass[k] = lg.g.klass[k];
  for (int k = 0; k < 11; ++k) o->word[k] = k < (int)lg.g.word.size() ? lg.g.word[k] : -2;
  o->n_subgraphs = (int)lg.subs.size(); o->n_terms = (int)lg.terms.size();
  o->tape_len = (int)lg.tape.code.size(); o->nslots = lg.tape.nslots;
  o->n_monomials = lg.st.n_monomials; o->flops = lg.tape.flops;
  o->canonical_id = lg.canonical_id;
  o->bound_depth = lg.tape.depth; o->flops_bound = lg.tape.flops_bound; o->flops_dd = lg.tape.flops_dd;
  return AE_OK;
}

// Block size for a kernel whose dynamic shared memory is bs * nslots * elem:
// the candidate with the most resident warps per SM (the slot file, not the
// register file, is what limits residency for long tapes), ties to the
// larger block.
// Largest block the kernel can launch with (its registers per thread).
static int max_threads(const void *kernel) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, kernel) != cudaSuccess) return 0;
  return a.maxThreadsPerBlock;
}

static int pick_block_for(const ae_ctx *c, const void *kernel, int nslots, size_t elem, size_t extra = 0) {
  const size_t smem_cap = 224 * 1024;
  if (c->opts.block_size > 0) {
    int bs = c->opts.block_size;
    if (kernel && bs > max_threads(kernel)) return -1;
    return extra + (size_t)bs * nslots * elem > smem_cap ? -1 : bs;
  }
  int best = -1, best_warps = 0;
  for (int bs : {1024, 768, 640, 512, 448, 384, 320, 256, 224, 192, 160, 128, 96, 64, 32}) {
    size_t smem = extra + (size_t)bs * nslots * elem;
    if (smem > smem_cap) continue;
    int per_sm = 0;
    if (kernel) {
      cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, bs, smem) != cudaSuccess) per_sm = 0;
    } else {
      per_sm = (int)std::min<size_t>(32, (228 * 1024) / (smem + 3072));
    }
    int warps = per_sm * bs / 32;
    if (warps > best_warps) { best_warps = warps; best = bs; }
  }
  return best;
}


static int ensure_scratch(ae_ctx *c, size_t nparts, size_t qcap) {
  if (nparts > c->part_cap) {
    if (c->d_part) cudaFree(c->d_part);
    CUDA_TRY(c, cudaMalloc(&c->d_part, nparts * sizeof(Partial)));
    c->part_cap = nparts;
  }
  if (!c->d_qcount) CUDA_TRY(c, cudaMalloc(&c->d_qcount, 2 * sizeof(unsigned long long)));
  if (qcap > c->queue_cap) {
    if (c->d_queue) cudaFree(c->d_queue);
    if (c->d_yq) cudaFree(c->d_yq);
    if (c->d_qstat) cudaFree(c->d_qstat);
    CUDA_TRY(c, cudaMalloc(&c->d_queue, qcap * sizeof(unsigned long long)));
    CUDA_TRY(c, cudaMalloc(&c->d_yq, qcap * sizeof(double)));
    CUDA_TRY(c, cudaMalloc(&c->d_qstat, qcap * sizeof(int)));
    c->queue_cap = qcap;
  }
  return AE_OK;
}

static void host_dd_add(double &hi, double &lo, double x) {
  double s = hi + x;
  double bb = s - hi;
  double e = (hi - (s - bb)) + (x - bb);
  lo += e;
  double r = s + lo;
  lo = lo - (r - s);
  hi = r;
}

// Mean, sigma_down (Eq. eq_sigma_down) and the heuristic sigma_up of a
// result from its sums: sigma_up^2 = sigma_down^2 + max y^2 / N^2.  A graph
// with no samples gets value 0 and sigma 0.
void ae_result_finish(ae_graph_result *r, int mult, double sum_abs) {
  const double N = (double)r->n;
  r->mean = r->n ? r->sum_y / N : 0.0;
  const double var = r->n ? r->sum_y2 / (N * N) - r->sum_y * r->sum_y / (N * N * N) : 0.0;
  r->sigma1 = var > 0 ? std::sqrt(var) : 0.0;
  r->mean_abs = r->n ? sum_abs / N : 0.0;
  r->value = mult * r->mean;
  r->sigma = mult * r->sigma1;
  const double up = r->n ? r->sigma1 * r->sigma1 + r->max_y2 / (N * N) : 0.0;
  r->sigma_up = mult * std::sqrt(up);
}

// Integrate one graph in slices of at most 2^28 samples (bounds the
// double-double queue); sums are combined in slice order, so the result is
// independent of the schedule.
static int integrate_one(ae_ctx *c, int gid, uint64_t first, uint64_t nsamp, uint64_t seed, ae_graph_result *res) {
  LoadedGraph &lg = c->graphs[gid];
  GraphDev &G = lg.dev;
  int bs = pick_block_for(c, (const void *)integrate_kernel, G.nslots, 8, kStageBytes);
  if (bs < 0) return fail(c, AE_ERR_STATE, "tape slot file does not fit in shared memory");
  size_t smem = kStageBytes + (size_t)bs * G.nslots * 8;
  CUDA_TRY(c, cudaFuncSetAttribute(integrate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = c->opts.ctas_per_sm;
  if (per_sm <= 0) {
    CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, integrate_kernel, bs, smem));
    if (per_sm < 1) per_sm = 1;
  }
  const uint64_t SLICE = 1ull << 28;
  double sy = 0, syl = 0, sy2 = 0, sy2l = 0, sa = 0, sal = 0, mx = 0;
  uint64_t n = 0, ndd = 0, nbad = 0, launches = 0, d2h = 0;
  double secs = 0, ksecs = 0;
  for (uint64_t start = 0; start < nsamp; start += SLICE) {
    uint64_t len = std::min(SLICE, nsamp - start);
    uint64_t grid = (uint64_t)c->sm_count * per_sm;
    if (c->opts.grid_ctas > 0) grid = std::min<uint64_t>(grid, (uint64_t)c->opts.grid_ctas);
    if (grid * bs > len) grid = std::max<uint64_t>(1, (len + bs - 1) / bs);
    size_t qcap = (size_t)std::max<uint64_t>(len, 65536);   // every sample may need re-evaluation
    const uint64_t SEG = 1ull << 14;
    const uint64_t nseg = (len + SEG - 1) / SEG;
    int rc = ensure_scratch(c, grid + nseg, qcap);
    if (rc) return rc;
    // dense double-double results of the slice: y in d_yq, flags in d_qstat
    double *ydense = c->d_yq;
    unsigned char *fdense = reinterpret_cast<unsigned char *>(c->d_qstat);
    // d_qcount[0]: queue length, d_qcount[1]: wait-timeout flag
    CUDA_TRY(c, cudaMemsetAsync(c->d_qcount, 0, 2 * sizeof(unsigned long long), c->stream));
    CUDA_TRY(c, cudaMemsetAsync(fdense, 0, len, c->stream));
    cudaEvent_t e0, e1, ek;
    cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&ek);
    cudaEventRecord(e0, c->stream);
    integrate_kernel<<<(unsigned)grid, bs, smem, c->stream>>>(G, first + start, len, seed, c->opts.dd_tol, c->d_part,
                                                              c->d_queue, c->queue_cap, c->d_qcount,
                                                              (int *)(c->d_qcount + 1), kWaitCycles, 0);
    CUDA_TRY(c, cudaGetLastError());
    cudaEventRecord(ek, c->stream);
    ++launches;
    unsigned long long hq[2] = {0, 0};
    CUDA_TRY(c, cudaMemcpyAsync(hq, c->d_qcount, sizeof(hq), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    unsigned long long nq = hq[0];
    if (hq[1]) {
      cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(ek);
      return fail(c, AE_ERR_TIMEOUT, "integrate: a tape-staging wait ran out");
    }
    if (nq > c->queue_cap) {
      cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(ek);
      return fail(c, AE_ERR_STATE, "double-double queue overflow");
    }
    if (nq) {
      int bsd = pick_block_for(c, (const void *)dd_staged_kernel, G.nslots, 16, kStageBytes);
      if (bsd < 0) return fail(c, AE_ERR_STATE, "double-double slot file does not fit in shared memory");
      size_t sm2 = kStageBytes + (size_t)bsd * G.nslots * 16;
      CUDA_TRY(c, cudaFuncSetAttribute(dd_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
      int pm = 0;
      CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pm, dd_staged_kernel, bsd, sm2));
      unsigned g2 = (unsigned)std::min<uint64_t>((nq + bsd - 1) / bsd, (uint64_t)c->sm_count * std::max(pm, 1));
      dd_staged_kernel<<<g2, bsd, sm2, c->stream>>>(G, seed, c->d_queue, nq, c->opts.dd_tol, first + start, ydense,
                                                   fdense, (int *)(c->d_qcount + 1));
      CUDA_TRY(c, cudaGetLastError());
      dense_dd_reduce_kernel<<<(unsigned)std::min<uint64_t>((nseg + 7) / 8, (uint64_t)c->sm_count * 16), 256, 0,
                               c->stream>>>(len, SEG, ydense, fdense, c->d_part + grid);
      CUDA_TRY(c, cudaGetLastError());
      launches += 2;
    }
    cudaEventRecord(e1, c->stream);
    const size_t np = nq ? grid + nseg : grid;
    std::vector<Partial> parts(np);
    CUDA_TRY(c, cudaMemcpyAsync(parts.data(), c->d_part, np * sizeof(Partial), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaMemcpyAsync(hq, c->d_qcount, sizeof(hq), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (hq[1]) {
      cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(ek);
      return fail(c, AE_ERR_TIMEOUT, "integrate: a tape-staging wait ran out (double-double pass)");
    }
    float ms = 0, mk = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventElapsedTime(&mk, e0, ek);
    cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(ek);
    secs += ms * 1e-3;
    ksecs += mk * 1e-3;
    d2h += 2 * sizeof(unsigned long long) + np * sizeof(Partial);
    // CTA partials in CTA order, then the re-evaluated samples' segment sums
    // in segment order (deterministic)
    for (size_t k = 0; k < np; ++k) {
      const Partial &p = parts[k];
      host_dd_add(sy, syl, p.sy_hi); host_dd_add(sy, syl, p.sy_lo);
      host_dd_add(sy2, sy2l, p.sy2_hi); host_dd_add(sy2, sy2l, p.sy2_lo);
      host_dd_add(sa, sal, p.sa_hi); host_dd_add(sa, sal, p.sa_lo);
      mx = std::max(mx, p.max_y2);
      if (k < grid) n += p.n;
      else { ndd += p.n_flag; nbad += p.n_overflow; }
    }
  }
  res->sum_y = sy + syl; res->sum_y2 = sy2 + sy2l;
  res->n = n; res->n_dd = ndd; res->n_nonfinite = nbad;
  res->max_y2 = mx;
  ae_result_finish(res, lg.g.mult, sa + sal);
  res->seconds = secs;
  res->launches = launches;
  res->kernel_seconds = ksecs;
  res->d2h_bytes = d2h;
  return AE_OK;
}

static int run_batched(ae_ctx *c, const std::vector<int> &ids, const std::vector<uint64_t> &ns,
                       const std::vector<uint64_t> &firsts, uint64_t seed, int bs, uint64_t chunk,
                       bool use_graph, std::vector<ae_graph_result> &res, double *secs_out);

// Samples [first, first + count) of one graph (resume / sharding by counter
// range): the same Philox stream as ae_integrate, so ranges concatenate.
// One launch of the per-graph kernel, which starts at `first`.
extern "C" int ae_integrate_range(ae_ctx *c, int gid, uint64_t first, uint64_t count, uint64_t seed,
                                  ae_graph_result *out) {
  if (!c || !out) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "integration needs a CUDA device");
  if (gid < 0 || gid >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  if (count == 0) return fail(c, AE_ERR_ARG, "zero samples");
  if (first + count < first) return fail(c, AE_ERR_ARG, "sample index overflows 2^64");
  CUDA_TRY(c, cudaSetDevice(c->device));
  ae_graph_result r;
  std::memset(&r, 0, sizeof(r));
  int rc = integrate_one(c, gid, first, count, seed, &r);
  if (rc) return rc;
  *out = r;
  return AE_OK;
}

extern "C" int ae_integrate(ae_ctx *c, const int *ids, int n_ids, uint64_t nsamp, uint64_t seed,
                            double *value, double *sigma, ae_graph_result *per) {
  if (!c) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "integration needs a CUDA device");
  if (c->graphs.empty()) return fail(c, AE_ERR_STATE, "no graphs loaded");
  if (!ids || n_ids <= 0 || nsamp == 0) return fail(c, AE_ERR_ARG, "empty graph list or zero samples");
  for (int i = 0; i < n_ids; ++i)
    if (ids[i] < 0 || ids[i] >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  CUDA_TRY(c, cudaSetDevice(c->device));
  double v = 0, s2 = 0;
  for (int i = 0; i < n_ids; ++i) {
    ae_graph_result r;
    std::memset(&r, 0, sizeof(r));
    int rc = integrate_one(c, ids[i], 0, nsamp, seed, &r);
    if (rc) return rc;
    v += r.value;
    s2 += r.sigma * r.sigma;
    if (per) per[i] = r;
  }
  if (value) *value = v;
  if (sigma) *sigma = std::sqrt(s2);
  return AE_OK;
}

// Autotuned launch shape of the batched kernel for one (graph set, budget).
struct BatchTune {
  int block = 0;
  unsigned long long chunk = 0;
};

static int run_batched_q(ae_ctx *c, const std::vector<int> &ids, const std::vector<uint64_t> &ns,
                         const std::vector<uint64_t> &firsts, uint64_t seed, int bs, uint64_t chunk,
                         bool use_graph, std::vector<ae_graph_result> &res, double *secs_out, bool full_queue);

static int run_batched(ae_ctx *c, const std::vector<int> &ids, const std::vector<uint64_t> &ns,
                       const std::vector<uint64_t> &firsts, uint64_t seed, int bs, uint64_t chunk,
                       bool use_graph, std::vector<ae_graph_result> &res, double *secs_out) {
  // queue sized for a quarter of the samples; a batch that needs more is
  // rerun with room for every sample (same samples, same result)
  int rc = run_batched_q(c, ids, ns, firsts, seed, bs, chunk, use_graph, res, secs_out, false);
  if (rc == AE_ERR_STATE && c->err == "double-double queue overflow")
    rc = run_batched_q(c, ids, ns, firsts, seed, bs, chunk, use_graph, res, secs_out, true);
  return rc;
}

static int run_batched_q(ae_ctx *c, const std::vector<int> &ids, const std::vector<uint64_t> &ns,
                         const std::vector<uint64_t> &firsts, uint64_t seed, int bs, uint64_t chunk,
                         bool use_graph, std::vector<ae_graph_result> &res, double *secs_out, bool full_queue) {
  int maxslots = 0;
  for (int g : ids) maxslots = std::max(maxslots, c->graphs[g].dev.nslots);
  // Buckets of similar slot-file size, one persistent launch each (a launch
  // sized for the largest tape would cut the occupancy of all the others);
  // inside a bucket, graphs by decreasing tape length (balances the tail).
  std::vector<int> order(ids.size());
  for (size_t i = 0; i < ids.size(); ++i) order[i] = (int)i;
  auto bucket_of = [&](int oi) {
    int ns_ = c->graphs[ids[oi]].dev.nslots;
    int b = 0;
    for (int lim : {40, 56, 72, 96, 128, 176, 256, 512}) { if (ns_ <= lim) return b; ++b; }
    return b;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    int ba = bucket_of(a), bb = bucket_of(b);
    if (ba != bb) return ba < bb;
    return c->graphs[ids[a]].dev.ntape > c->graphs[ids[b]].dev.ntape;
  });
  // Chunks graph by graph.  A graph gets at least ~2 chunks per resident CTA
  // when its budget allows, so the CTAs work on one or two tapes at a time and
  // the tape stays in L2 (many different tapes in flight thrash it).
  std::vector<Chunk> chunks;
  struct Launch { size_t c0, c1; int bs; size_t smem; unsigned grid; };
  std::vector<Launch> launches;
  for (size_t k = 0; k < order.size();) {
    int b = bucket_of(order[k]);
    size_t k1 = k;
    int bslots = 0;
    while (k1 < order.size() && bucket_of(order[k1]) == b) { bslots = std::max(bslots, c->graphs[ids[order[k1]]].dev.nslots); ++k1; }
    Launch L;
    L.c0 = chunks.size();
    // block size: the tuned one if it fits, else the occupancy choice for this bucket
    L.bs = (kStageBytes + (size_t)bs * bslots * 8 <= 224 * 1024 && bs <= max_threads((const void *)batched_kernel))
               ? bs : pick_block_for(c, (const void *)batched_kernel, bslots, 8, kStageBytes);
    if (L.bs < 0) return fail(c, AE_ERR_STATE, "batched slot file does not fit in shared memory");
    L.smem = kStageBytes + (size_t)L.bs * bslots * 8;
    int pm = 0;
    CUDA_TRY(c, cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem));
    CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pm, batched_kernel, L.bs, L.smem));
    if (pm < 1) pm = 1;
    L.grid = (unsigned)(c->sm_count * pm);
    if (c->opts.grid_ctas > 0) L.grid = std::min<unsigned>(L.grid, (unsigned)c->opts.grid_ctas);
    uint64_t res_b = (uint64_t)L.grid;
    for (size_t t = k; t < k1; ++t) {
      int oi = order[t];
      uint64_t cg = std::min<uint64_t>(chunk, std::max<uint64_t>((ns[oi] + 2 * res_b - 1) / (2 * res_b), (uint64_t)L.bs));
      for (uint64_t s0 = 0; s0 < ns[oi]; s0 += cg)
        chunks.push_back(Chunk{oi, 0, firsts[oi] + s0, std::min<uint64_t>(cg, ns[oi] - s0)});
    }
    L.c1 = chunks.size();
    launches.push_back(L);
    k = k1;
  }
  size_t smax = 0;
  for (const Launch &L : launches) smax = std::max(smax, L.smem);
  CUDA_TRY(c, cudaFuncSetAttribute(batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smax));
  uint64_t total = 0;
  for (uint64_t x : ns) total += x;
  size_t nch = chunks.size();
  size_t qcap = (size_t)std::max<uint64_t>(full_queue ? total : total / 4, 65536);
  // device buffers (graph descriptors, chunks, partials, queue), kept in the
  // context and grown when a larger batch arrives
  // dense double-double results: one y and one flag byte per sample of the batch
  size_t need = ids.size() * sizeof(GraphDev) + nch * sizeof(Chunk) + 2 * nch * sizeof(Partial) +
                qcap * (8 + 4 + 8 + 4) + ids.size() * (8 + 16 + 8) + total * 9 + 64 * 4 + 12 * 1024;
  if (need > c->bbuf_bytes) {
    if (c->bbuf) cudaFree(c->bbuf);
    c->bbuf = nullptr;
    c->bbuf_bytes = 0;
    CUDA_TRY(c, cudaMalloc(&c->bbuf, need));
    c->bbuf_bytes = need;
  }
  char *buf = (char *)c->bbuf;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  char *p = buf;
  GraphDev *dG = (GraphDev *)p; p += al(ids.size() * sizeof(GraphDev));
  Chunk *dC = (Chunk *)p; p += al(nch * sizeof(Chunk));
  Partial *dP = (Partial *)p; p += al(nch * sizeof(Partial));
  Partial *dP2 = (Partial *)p; p += al(nch * sizeof(Partial));
  unsigned long long *qi = (unsigned long long *)p; p += al(qcap * 8);
  int *qg = (int *)p; p += al(qcap * 4);
  unsigned long long *gpos = (unsigned long long *)p; p += al(ids.size() * 16);
  double *ydense = (double *)p; p += al(total * 8);
  unsigned char *fdense = (unsigned char *)p; p += al(total);
  unsigned long long *qi2 = (unsigned long long *)p; p += al(qcap * 8);
  int *qg2 = (int *)p; p += al(qcap * 4);
  unsigned int *hist = (unsigned int *)p; p += al(ids.size() * 4);
  int *drank = (int *)p; p += al(ids.size() * 4);
  unsigned int *wstart = (unsigned int *)p; p += al((ids.size() + 1) * 4);
  int *rank_bs = (int *)p; p += al(ids.size() * 4);
  unsigned long long *qcount = (unsigned long long *)p; p += 256;
  int *next = (int *)(qcount + 1);   // one counter per launch (up to 16), then one per dd launch
  int *derr = (int *)((char *)qcount + 192);   // wait-timeout flag
  std::vector<GraphDev> hg;
  for (int g : ids) hg.push_back(c->graphs[g].dev);
  // rank of each graph in bucket order; last rank of each bucket
  std::vector<int> hrank(ids.size());
  for (size_t r = 0; r < order.size(); ++r) hrank[order[r]] = (int)r;
  std::vector<int> bucket_last;   // rank of the last graph of each launch's bucket
  {
    size_t r = 0;
    for (const Launch &L : launches) {
      (void)L;
      int b = bucket_of(order[r]);
      while (r < order.size() && bucket_of(order[r]) == b) ++r;
      bucket_last.push_back((int)r - 1);
    }
  }
  cudaError_t e = cudaMemcpyAsync(dG, hg.data(), hg.size() * sizeof(GraphDev), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(drank, hrank.data(), hrank.size() * 4, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dC, chunks.data(), nch * sizeof(Chunk), cudaMemcpyHostToDevice, c->stream);
  // dense layout of the batch: graph i's samples firsts[i] .. firsts[i]+ns[i]-1
  // at base_i .. base_i+ns[i]-1, bases in id order
  std::vector<unsigned long long> hgpos(2 * ids.size());
  {
    unsigned long long base = 0;
    for (size_t i = 0; i < ids.size(); ++i) { hgpos[2 * i] = base; hgpos[2 * i + 1] = firsts[i]; base += ns[i]; }
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(gpos, hgpos.data(), hgpos.size() * 8, cudaMemcpyHostToDevice, c->stream);
  // one staged double-double launch per bucket, shaped for that bucket's
  // slots (16-byte rows), persistent (SMs x resident CTAs)
  std::vector<int> dd_bs(launches.size()), dd_pitch(launches.size()), dd_r0(launches.size());
  std::vector<unsigned> dd_grid(launches.size());
  std::vector<size_t> dd_sm(launches.size());
  std::vector<int> hrank_bs(ids.size());
  size_t ddmax = 0;
  {
    size_t r = 0;
    for (size_t l = 0; l < launches.size(); ++l) {
      int bslots = 0;
      const size_t rb = r;
      int b = bucket_of(order[r]);
      while (r < order.size() && bucket_of(order[r]) == b) { bslots = std::max(bslots, c->graphs[ids[order[r]]].dev.nslots); ++r; }
      int b16 = pick_block_for(c, (const void *)batched_dd_staged_kernel, bslots, 16, kStageBytes);
      if (b16 < 0) return fail(c, AE_ERR_STATE, "double-double slot file does not fit in shared memory");
      dd_bs[l] = b16;
      dd_pitch[l] = bslots;
      dd_r0[l] = (int)rb;
      dd_sm[l] = kStageBytes + (size_t)b16 * bslots * 16;
      for (size_t q = rb; q < r; ++q) hrank_bs[q] = b16;
      int pm = 0;
      CUDA_TRY(c, cudaFuncSetAttribute(batched_dd_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dd_sm[l]));
      CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&pm, batched_dd_staged_kernel, b16, dd_sm[l]));
      dd_grid[l] = (unsigned)(c->sm_count * std::max(pm, 1));
      ddmax = std::max(ddmax, dd_sm[l]);
    }
  }
  if (e == cudaSuccess) e = cudaFuncSetAttribute(batched_dd_staged_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ddmax);
  if (e == cudaSuccess) e = cudaMemcpyAsync(rank_bs, hrank_bs.data(), hrank_bs.size() * 4, cudaMemcpyHostToDevice, c->stream);
  unsigned grid2 = (unsigned)(c->sm_count * 4);
  if (use_graph)
    for (auto &ev : c->gev)
      if (!ev && e == cudaSuccess) e = cudaEventCreate(&ev);
  cudaEvent_t e0 = nullptr, e1 = nullptr, ek = nullptr;
  // events recorded with cudaEventRecordExternal so that, inside a captured
  // graph, they become event-record nodes readable after the launch
  auto rec = [&](cudaEvent_t ev) {
    if (use_graph) cudaEventRecordWithFlags(ev, c->stream, cudaEventRecordExternal);
    else cudaEventRecord(ev, c->stream);
  };
  auto enqueue = [&]() {
    rec(e0);
    cudaMemsetAsync(qcount, 0, 256, c->stream);
    cudaMemsetAsync(hist, 0, ids.size() * 4, c->stream);
    cudaMemsetAsync(fdense, 0, total, c->stream);
    for (size_t l = 0; l < launches.size(); ++l) {
      const Launch &L = launches[l];
      batched_kernel<<<L.grid, L.bs, L.smem, c->stream>>>(dG, dC + L.c0, (int)(L.c1 - L.c0), seed, c->opts.dd_tol,
                                                          dP + L.c0, qi, qg, qcap, qcount, next + l, derr);
    }
    rec(ek);
    queue_hist_kernel<<<grid2, 256, 0, c->stream>>>(qg, qcount, qcap, drank, hist);
    queue_scan_kernel<<<1, 32, 0, c->stream>>>(hist, (int)ids.size());
    queue_scatter_kernel<<<grid2, 256, 0, c->stream>>>(qi, qg, qcount, qcap, drank, hist, qi2, qg2);
    // after the scatter hist[r] is the end of bin r; the plan cuts every
    // rank into items of its bucket's block size
    dd_plan_kernel<<<1, 32, 0, c->stream>>>(hist, rank_bs, (int)ids.size(), wstart);
    for (size_t l = 0; l < launches.size(); ++l)
      batched_dd_staged_kernel<<<dd_grid[l], dd_bs[l], dd_sm[l], c->stream>>>(
          dG, seed, qi2, qg2, hist, wstart, dd_r0[l], bucket_last[l], gpos, ydense, fdense, dd_pitch[l],
          c->opts.dd_tol, next + 16 + l, derr);
    chunk_dd_reduce_kernel<<<(unsigned)std::min<size_t>((nch + 7) / 8, (size_t)c->sm_count * 16), 256, 0,
                             c->stream>>>(dC, (int)nch, gpos, ydense, fdense, dP2);
    rec(e1);
  };
  cudaGraph_t graph = nullptr;
  if (e == cudaSuccess) {
    if (use_graph) {
      // the launches and their timing events form one CUDA graph; it is kept
      // and launched again while the launch shape, the buffers and the scalar
      // arguments stay the same (the chunk list and graph descriptors are
      // copied to the device before every launch)
      e0 = c->gev[0]; e1 = c->gev[1]; ek = c->gev[2];
      uint64_t tol_bits;
      std::memcpy(&tol_bits, &c->opts.dd_tol, sizeof(tol_bits));   // exact: any change of dd_tol recaptures
      std::string key = std::to_string((uintptr_t)buf) + "/" + std::to_string(seed) + "/" +
                        std::to_string(tol_bits) + "/" + std::to_string(nch) + "/" + std::to_string(total) +
                        "/" + std::to_string(qcap) + "/" + std::to_string(ids.size()) + "/" + std::to_string(grid2);
      for (size_t l = 0; l < launches.size(); ++l)
        key += "|" + std::to_string(launches[l].grid) + "," + std::to_string(launches[l].bs) + "," +
               std::to_string(launches[l].smem) + "," + std::to_string(launches[l].c0) + "," +
               std::to_string(launches[l].c1) + "," + std::to_string(dd_bs[l]) + "," + std::to_string(dd_sm[l]) +
               "," + std::to_string(dd_pitch[l]) + "," + std::to_string(bucket_last[l]) + "," +
               std::to_string(dd_grid[l]);
      if (!(c->gexec && key == c->gkey)) {
        if (c->gexec) cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
        c->gkey.clear();
        e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          enqueue();
          e = cudaStreamEndCapture(c->stream, &graph);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, graph, 0);
        if (e == cudaSuccess) c->gkey = key;
      }
      if (e == cudaSuccess) e = cudaGraphLaunch(c->gexec, c->stream);
    } else {
      cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventCreate(&ek);
      enqueue();
      e = cudaGetLastError();
    }
  }
  unsigned long long nq = 0;
  int herr = 0;
  std::vector<Partial> parts(nch), parts2(nch);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&nq, qcount, 8, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, derr, 4, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(parts.data(), dP, nch * sizeof(Partial), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(parts2.data(), dP2, nch * sizeof(Partial), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  float ms = 0, mk = 0;
  if (e == cudaSuccess) {
    cudaError_t t1 = cudaEventElapsedTime(&ms, e0, e1), t2 = cudaEventElapsedTime(&mk, e0, ek);
    if (t1 != cudaSuccess || t2 != cudaSuccess) e = t1 != cudaSuccess ? t1 : t2;
  }
  nq = std::min<unsigned long long>(nq, qcap);
  if (graph) cudaGraphDestroy(graph);
  if (!use_graph) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (ek) cudaEventDestroy(ek);
  }
  if (e != cudaSuccess) {
    if (use_graph && c->gexec) { cudaGraphExecDestroy(c->gexec); c->gexec = nullptr; c->gkey.clear(); }
    return fail(c, AE_ERR_CUDA, std::string("batched: ") + cudaGetErrorString(e));
  }
  if (herr) return fail(c, AE_ERR_TIMEOUT, "batched: a tape-staging wait ran out");
  for (auto &pp : parts)
    if (pp.n_overflow) return fail(c, AE_ERR_STATE, "double-double queue overflow");
  (void)buf;
  // per graph, in chunk order: each chunk's FP64 partial, then the sums of
  // its re-evaluated samples (in sample order, reduced on the device)
  size_t G = ids.size();
  std::vector<double> sy(G, 0), syl(G, 0), sy2(G, 0), sy2l(G, 0), sa(G, 0), sal(G, 0), mx(G, 0);
  std::vector<uint64_t> n(G, 0), ndd(G, 0), nbad(G, 0);
  for (size_t k = 0; k < nch; ++k) {
    int gi = chunks[k].gi;
    const Partial &q = parts[k];
    host_dd_add(sy[gi], syl[gi], q.sy_hi); host_dd_add(sy[gi], syl[gi], q.sy_lo);
    host_dd_add(sy2[gi], sy2l[gi], q.sy2_hi); host_dd_add(sy2[gi], sy2l[gi], q.sy2_lo);
    host_dd_add(sa[gi], sal[gi], q.sa_hi); host_dd_add(sa[gi], sal[gi], q.sa_lo);
    mx[gi] = std::max(mx[gi], q.max_y2);
    n[gi] += q.n;
    const Partial &r = parts2[k];
    host_dd_add(sy[gi], syl[gi], r.sy_hi); host_dd_add(sy[gi], syl[gi], r.sy_lo);
    host_dd_add(sy2[gi], sy2l[gi], r.sy2_hi); host_dd_add(sy2[gi], sy2l[gi], r.sy2_lo);
    host_dd_add(sa[gi], sal[gi], r.sa_hi); host_dd_add(sa[gi], sal[gi], r.sa_lo);
    mx[gi] = std::max(mx[gi], r.max_y2);
    ndd[gi] += r.n_flag; nbad[gi] += r.n_overflow;
  }
  res.assign(G, ae_graph_result{});
  for (size_t gi = 0; gi < G; ++gi) {
    ae_graph_result &r = res[gi];
    std::memset(&r, 0, sizeof(r));
    r.sum_y = sy[gi] + syl[gi]; r.sum_y2 = sy2[gi] + sy2l[gi];
    r.n = n[gi]; r.n_dd = ndd[gi]; r.n_nonfinite = nbad[gi];
    r.max_y2 = mx[gi];
    // a graph given no samples contributes value 0 and sigma 0
    ae_result_finish(&r, c->graphs[ids[gi]].g.mult, sa[gi] + sal[gi]);
    r.seconds = ms * 1e-3 * (double)ns[gi] / (double)total;   // share of the launch by samples
    r.kernel_seconds = mk * 1e-3 * (double)ns[gi] / (double)total;
    r.launches = gi == 0 ? (uint64_t)(2 * launches.size() + 5) : 0;
    r.d2h_bytes = gi == 0 ? (8 + 4 + 2 * nch * sizeof(Partial)) : 0;
    r.h2d_bytes = gi == 0 ? (ids.size() * (sizeof(GraphDev) + 4 + 16) + nch * sizeof(Chunk)) : 0;
  }
  if (secs_out) *secs_out = ms * 1e-3;
  return AE_OK;
}

// Autotuner: time the batched kernel on a small budget for each candidate
// (block size x chunk size) and keep the fastest; cached per graph set.
static int autotune_batched(ae_ctx *c, const std::vector<int> &ids, BatchTune &best) {
  std::string key = std::to_string(c->loops) + ":";
  for (int g : ids) key += std::to_string(g) + ",";
  auto it = c->tune_cache.find(key);
  if (it != c->tune_cache.end()) { best.block = it->second.first; best.chunk = it->second.second; return AE_OK; }
  int maxslots = 0;
  for (int g : ids) maxslots = std::max(maxslots, c->graphs[g].dev.nslots);
  // trial set: up to six graphs spanning the tape lengths (longest, shortest,
  // quantiles), so tuning costs a fraction of a second even for 269 graphs
  std::vector<int> byl = ids;
  std::sort(byl.begin(), byl.end(), [&](int a, int b) { return c->graphs[a].dev.ntape > c->graphs[b].dev.ntape; });
  std::vector<int> trial;
  for (int q = 0; q < 6 && q < (int)byl.size(); ++q) {
    int k = (int)((size_t)q * (byl.size() - 1) / 5);
    if (std::find(trial.begin(), trial.end(), byl[k]) == trial.end()) trial.push_back(byl[k]);
  }
  double best_rate = 0;
  // candidates: the block with the most resident warps for the largest slot
  // row, and the usual sizes that fit
  const int occ = pick_block_for(c, (const void *)batched_kernel, maxslots, 8, kStageBytes);
  std::vector<int> cand;
  for (int bs : {occ, 128, 256, 512})
    if (bs > 0 && std::find(cand.begin(), cand.end(), bs) == cand.end()) cand.push_back(bs);
  for (int bs : cand) {
    if (kStageBytes + (size_t)bs * maxslots * 8 > 224 * 1024) continue;
    for (unsigned long long ch : {1024ull, 4096ull, 16384ull}) {
      uint64_t per = std::max<uint64_t>(ch * 4, (uint64_t)c->sm_count * bs * 8 / trial.size());
      std::vector<uint64_t> ns(trial.size(), per), fs(trial.size(), 1ull << 44);
      std::vector<ae_graph_result> res;
      double secs = 0;
      int rc = run_batched(c, trial, ns, fs, 0x5eed, bs, ch, false, res, &secs);
      if (rc) return rc;
      double fl = 0;
      for (int g : trial) fl += c->graphs[g].tape.flops * (double)per;
      double rate = fl / std::max(secs, 1e-9);   // tape flops per second
      if (rate > best_rate) { best_rate = rate; best.block = bs; best.chunk = ch; }
    }
  }
  c->tune_cache[key] = {best.block, best.chunk};
  return AE_OK;
}

extern "C" int ae_integrate_batched(ae_ctx *c, const int *ids, int n_ids, const uint64_t *ns, uint64_t seed,
                                    double *value, double *sigma, ae_graph_result *per) {
  if (!c) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "integration needs a CUDA device");
  if (c->graphs.empty()) return fail(c, AE_ERR_STATE, "no graphs loaded");
  if (!ids || !ns || n_ids <= 0) return fail(c, AE_ERR_ARG, "empty graph list");
  std::vector<int> vid(ids, ids + n_ids);
  std::vector<uint64_t> vn(ns, ns + n_ids), vf(n_ids, 0);
  uint64_t total = 0;
  for (int i = 0; i < n_ids; ++i) {
    if (ids[i] < 0 || ids[i] >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
    total += ns[i];
  }
  if (total == 0) return fail(c, AE_ERR_ARG, "no samples requested");
  CUDA_TRY(c, cudaSetDevice(c->device));
  BatchTune t;
  if (c->opts.block_size > 0) { t.block = c->opts.block_size; t.chunk = 16384; }
  else {
    int rc = autotune_batched(c, vid, t);
    if (rc) return rc;
  }
  std::vector<ae_graph_result> res;
  double secs = 0;
  int rc = run_batched(c, vid, vn, vf, seed, t.block, t.chunk, true, res, &secs);
  if (rc) return rc;
  double v = 0, s2 = 0;
  for (int i = 0; i < n_ids; ++i) {
    v += res[i].value;
    s2 += res[i].sigma * res[i].sigma;
    if (per) per[i] = res[i];
  }
  if (value) *value = v;
  if (sigma) *sigma = std::sqrt(s2);
  c->last_tune_block = t.block;
  c->last_tune_chunk = t.chunk;
  return AE_OK;
}

// One block of a run: every listed graph continues its own stream from the
// run's next index, all in one batched launch; the sums go into the run.
extern "C" int ae_run_step(ae_ctx *c, const int *ids, int n_ids, const uint64_t *ns, ae_graph_result *per) {
  if (!c) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "integration needs a CUDA device");
  if (c->graphs.empty()) return fail(c, AE_ERR_STATE, "no graphs loaded");
  if (!ids || !ns || n_ids <= 0) return fail(c, AE_ERR_ARG, "empty graph list");
  std::vector<int> vid(ids, ids + n_ids);
  std::vector<uint64_t> vn(ns, ns + n_ids), vf(n_ids);
  std::vector<char> seen(c->graphs.size(), 0);
  uint64_t total = 0;
  for (int i = 0; i < n_ids; ++i) {
    if (ids[i] < 0 || ids[i] >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
    if (seen[ids[i]]) return fail(c, AE_ERR_ARG, "a graph listed twice in one run step");
    seen[ids[i]] = 1;
    vf[i] = c->run[ids[i]].next;
    if (vf[i] + ns[i] < vf[i]) return fail(c, AE_ERR_ARG, "sample index overflows 2^64");
    total += ns[i];
  }
  if (total == 0) return fail(c, AE_ERR_ARG, "no samples requested");
  CUDA_TRY(c, cudaSetDevice(c->device));
  BatchTune t;
  if (c->opts.block_size > 0) { t.block = c->opts.block_size; t.chunk = 16384; }
  else {
    int rc = autotune_batched(c, vid, t);
    if (rc) return rc;
  }
  std::vector<ae_graph_result> res;
  double secs = 0;
  int rc = run_batched(c, vid, vn, vf, c->run_seed, t.block, t.chunk, true, res, &secs);
  if (rc) return rc;
  for (int i = 0; i < n_ids; ++i) {
    ae_run_fold(c, ids[i], res[i], ns[i]);
    if (per) per[i] = res[i];
  }
  c->last_tune_block = t.block;
  c->last_tune_chunk = t.chunk;
  return AE_OK;
}

// Inter-graph allocation (Sec. IV.C): a pilot of n_pilot samples per graph
// (seed ^ 0x9E3779B97F4A7C15, independent of the main run's stream) gives
// sigma_j; with C_j = sigma_j sqrt(N_pilot) and t_j the cost of one sample
// (tape flops plus the sampler), mode 0 allocates n_j proportional to
// C_j / sqrt(t_j) (the paper's optimum p_j), mode 1 proportional to the
// variance estimate sigma_j^2.  Integer counts by largest remainder, at
// least min(1024, n_total / n_ids) each.
// The paper's integration controller (Sec. IV.C): blocks of samples whose
// graphs are drawn with the optimal probabilities of the samples so far.
extern "C" int ae_integrate_adaptive(ae_ctx *c, const int *ids, int n_ids, uint64_t block, int n_rounds,
                                     int blocks_per_round, double p_floor, uint64_t seed, double *value,
                                     double *sigma, ae_graph_result *per) {
  if (!c) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "integration needs a CUDA device");
  if (c->graphs.empty()) return fail(c, AE_ERR_STATE, "no graphs loaded");
  if (!ids || n_ids <= 0 || block == 0 || n_rounds < 1 || blocks_per_round < 1 || !(p_floor >= 0) || p_floor > 1)
    return fail(c, AE_ERR_ARG, "need graphs, block_size > 0, n_rounds >= 1, blocks_per_round >= 1, 0 <= p_floor <= 1");
  for (int i = 0; i < n_ids; ++i)
    if (ids[i] < 0 || ids[i] >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  CUDA_TRY(c, cudaSetDevice(c->device));
  const size_t G = (size_t)n_ids;
  std::vector<int> vid(ids, ids + n_ids);
  std::vector<uint64_t> Nj(G, 0);
  std::vector<double> sy(G, 0), syl(G, 0), sy2(G, 0), sy2l(G, 0), sa(G, 0), sal(G, 0), mx(G, 0), secs(G, 0),
      ksecs(G, 0);
  std::vector<uint64_t> ndd(G, 0), nbad(G, 0), launches(G, 0), d2h(G, 0), h2d(G, 0);
  std::vector<double> tj(G), sig(G), p(G);
  for (size_t i = 0; i < G; ++i) tj[i] = c->graphs[vid[i]].tape.flops + 150.0 * c->graphs[vid[i]].g.M();
  BatchTune tune;
  int rc = autotune_batched(c, vid, tune);
  if (rc) return rc;
  uint64_t draw = 0;   // counter of the block-draw stream
  // The first round is the initialisation pass: graphs without a floor of
  // their own take its mean |y| as the floor of the acceptance test for the
  // later rounds (restored on return).
  struct FloorGuard {
    ae_ctx *c; std::vector<int> ids; std::vector<double> old;
    ~FloorGuard() { for (size_t i = 0; i < ids.size(); ++i) c->graphs[ids[i]].dev.yfloor = old[i]; }
  } guard{c, vid, {}};
  for (int id : vid) guard.old.push_back(c->graphs[id].dev.yfloor);
  for (int r = 0; r < n_rounds; ++r) {
    if (r == 1)
      for (size_t i = 0; i < G; ++i)
        if (guard.old[i] == 0 && Nj[i] > 0) c->graphs[vid[i]].dev.yfloor = (sa[i] + sal[i]) / (double)Nj[i];
    std::vector<uint64_t> nb(G, 0);
    if (r == 0) {
      for (size_t i = 0; i < G; ++i) nb[i] = 1;
    } else {
      // C_j = sigma_up_j sqrt(N_j) (Sec. IV.C)
      for (size_t i = 0; i < G; ++i) {
        double N = (double)Nj[i], var = (sy2[i] + sy2l[i]) / (N * N) - (sy[i] + syl[i]) * (sy[i] + syl[i]) / (N * N * N);
        sig[i] = c->graphs[vid[i]].g.mult * std::sqrt(std::max(var, 0.0) + mx[i] / (N * N));
      }
      ae_schedule_probabilities(sig.data(), Nj.data(), tj.data(), n_ids, p_floor, p.data());
      std::vector<double> cdf(G);
      double acc = 0;
      for (size_t i = 0; i < G; ++i) { acc += p[i]; cdf[i] = acc; }
      for (int b = 0; b < blocks_per_round; ++b, ++draw) {
        // one uniform per block: Philox of (draw index, 0, 0x5c4ed, 0) under seed
        uint32_t w[4] = {(uint32_t)draw, (uint32_t)(draw >> 32), 0x5c4edu, 0u};
        ae::philox_host(w, (uint32_t)seed, (uint32_t)(seed >> 32));
        double u = (((double)(w[0] >> 5)) * 67108864.0 + (double)(w[1] >> 6) + 0.5) * 1.1102230246251565e-16;
        size_t j = (size_t)(std::lower_bound(cdf.begin(), cdf.end(), u * acc) - cdf.begin());
        if (j >= G) j = G - 1;
        nb[j] += 1;
      }
    }
    std::vector<int> rid;
    std::vector<uint64_t> rn, rf;
    std::vector<size_t> pos;
    for (size_t i = 0; i < G; ++i)
      if (nb[i]) { rid.push_back(vid[i]); rn.push_back(nb[i] * block); rf.push_back(Nj[i]); pos.push_back(i); }
    std::vector<ae_graph_result> res;
    double s_round = 0;
    rc = run_batched(c, rid, rn, rf, seed, tune.block, tune.chunk, true, res, &s_round);
    if (rc) return rc;
    for (size_t k = 0; k < pos.size(); ++k) {
      size_t i = pos[k];
      const ae_graph_result &q = res[k];
      host_dd_add(sy[i], syl[i], q.sum_y);
      host_dd_add(sy2[i], sy2l[i], q.sum_y2);
      host_dd_add(sa[i], sal[i], q.mean_abs * (double)q.n);
      mx[i] = std::max(mx[i], q.max_y2);
      Nj[i] += q.n; ndd[i] += q.n_dd; nbad[i] += q.n_nonfinite;
      secs[i] += q.seconds; ksecs[i] += q.kernel_seconds;
      launches[i] += q.launches; d2h[i] += q.d2h_bytes; h2d[i] += q.h2d_bytes;
    }
  }
  double tot = 0, var = 0;
  for (size_t i = 0; i < G; ++i) {
    ae_graph_result r;
    std::memset(&r, 0, sizeof(r));
    r.sum_y = sy[i] + syl[i]; r.sum_y2 = sy2[i] + sy2l[i];
    r.n = Nj[i]; r.n_dd = ndd[i]; r.n_nonfinite = nbad[i];
    r.max_y2 = mx[i];
    ae_result_finish(&r, c->graphs[vid[i]].g.mult, sa[i] + sal[i]);
    r.seconds = secs[i]; r.kernel_seconds = ksecs[i]; r.launches = launches[i];
    r.d2h_bytes = d2h[i]; r.h2d_bytes = h2d[i];
    tot += r.value;
    var += r.sigma * r.sigma;
    if (per) per[i] = r;
  }
  if (value) *value = tot;
  if (sigma) *sigma = std::sqrt(var);
  return AE_OK;
}

extern "C" int ae_allocate(ae_ctx *c, const int *ids, int n_ids, uint64_t n_pilot, uint64_t n_total, uint64_t seed,
                           int mode, uint64_t *n_out, double *sigma_out) {
  if (!c || !ids || !n_out || n_ids <= 0) return AE_ERR_ARG;
  if (n_pilot == 0 || n_total < (uint64_t)n_ids) return fail(c, AE_ERR_ARG, "n_pilot > 0 and n_total >= n_ids needed");
  if (mode != 0 && mode != 1) return fail(c, AE_ERR_ARG, "mode must be 0 or 1");
  std::vector<uint64_t> np(n_ids, n_pilot);
  std::vector<ae_graph_result> per(n_ids);
  int rc = ae_integrate_batched(c, ids, n_ids, np.data(), seed ^ 0x9E3779B97F4A7C15ull, nullptr, nullptr, per.data());
  if (rc) return rc;
  std::vector<double> wgt(n_ids);
  double sum = 0;
  for (int i = 0; i < n_ids; ++i) {
    const LoadedGraph &lg = c->graphs[ids[i]];
    double sj = per[i].sigma;   // multiplicity included
    double Cj = sj * std::sqrt((double)n_pilot);
    double tj = lg.tape.flops + 150.0 * lg.g.M();
    wgt[i] = mode == 0 ? Cj / std::sqrt(tj) : sj * sj;
    if (!(wgt[i] > 0) || !std::isfinite(wgt[i])) wgt[i] = 0;
    sum += wgt[i];
    if (sigma_out) sigma_out[i] = sj;
  }
  uint64_t floor_n = std::min<uint64_t>(1024, n_total / n_ids);
  uint64_t rest = n_total - floor_n * n_ids;
  std::vector<double> frac(n_ids);
  uint64_t given = 0;
  for (int i = 0; i < n_ids; ++i) {
    double want = sum > 0 ? (double)rest * wgt[i] / sum : (double)rest / n_ids;
    uint64_t w = (uint64_t)std::floor(want);
    n_out[i] = floor_n + w;
    frac[i] = want - (double)w;
    given += w;
  }
  std::vector<int> ord(n_ids);
  for (int i = 0; i < n_ids; ++i) ord[i] = i;
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return frac[a] > frac[b]; });
  for (uint64_t k = 0; given + k < rest && k < (uint64_t)n_ids; ++k) n_out[ord[k]] += 1;
  return AE_OK;
}

// Grid of a per-sample dump: as many CTAs as are resident on the device
// (ae_opts.ctas_per_sm, else the occupancy calculator), capped by
// ae_opts.grid_ctas and by one CTA per blockDim samples.
static unsigned dump_grid(const ae_ctx *c, const void *kernel, int bs, size_t smem, uint64_t count) {
  int per_sm = c->opts.ctas_per_sm;
  if (per_sm <= 0 && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, bs, smem) != cudaSuccess)
    per_sm = 1;
  uint64_t grid = (uint64_t)c->sm_count * (uint64_t)std::max(per_sm, 1);
  if (c->opts.grid_ctas > 0) grid = std::min<uint64_t>(grid, (uint64_t)c->opts.grid_ctas);
  return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(grid, (count + bs - 1) / bs));
}

extern "C" int ae_eval_samples(ae_ctx *c, int gid, uint64_t first, uint64_t count, uint64_t seed,
                               double *z, double *log2g, double *I, double *K, double *y, double *E) {
  if (!c) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "eval_samples needs a CUDA device");
  if (gid < 0 || gid >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  if (count == 0) return AE_OK;
  CUDA_TRY(c, cudaSetDevice(c->device));
  GraphDev &G = c->graphs[gid].dev;
  int bs = pick_block_for(c, (const void *)eval_kernel, G.nslots, 8, kStageBytes);
  if (bs < 0) return fail(c, AE_ERR_STATE, "tape slot file does not fit in shared memory");
  size_t smem = kStageBytes + (size_t)bs * G.nslots * 8;
  CUDA_TRY(c, cudaFuncSetAttribute(eval_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = dump_grid(c, (const void *)eval_kernel, bs, smem, count);
  double *d = nullptr;
  size_t per = (size_t)G.M + 5;
  CUDA_TRY(c, cudaMalloc(&d, count * per * 8 + 16));
  double *dz = d, *dl = d + count * G.M, *dI = dl + count, *dK = dI + count, *dy = dK + count, *dE = dy + count;
  int *derr = reinterpret_cast<int *>(dE + count);
  cudaError_t e = cudaMemsetAsync(derr, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) {
    eval_kernel<<<grid, bs, smem, c->stream>>>(G, first, count, seed, dz, dl, dI, dK, dy, dE, derr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && z) e = cudaMemcpy(z, dz, count * G.M * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && log2g) e = cudaMemcpy(log2g, dl, count * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && I) e = cudaMemcpy(I, dI, count * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && K) e = cudaMemcpy(K, dK, count * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && y) e = cudaMemcpy(y, dy, count * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && E) e = cudaMemcpy(E, dE, count * 8, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e == cudaSuccess && herr) return fail(c, AE_ERR_TIMEOUT, "eval_samples: a tape-staging wait ran out");
  if (e != cudaSuccess) return fail(c, AE_ERR_CUDA, std::string("eval_samples: ") + cudaGetErrorString(e));
  return AE_OK;
}

// Device address of g_noalloc_scratch, looked up once per device (with that
// device current) the first time ae_integrate_noalloc runs on it.
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];

extern "C" int ae_integrate_noalloc(ae_ctx *c, int gid, uint64_t nsamp, uint64_t seed,
                                    ae_graph_result *out) {
  if (!c || !out) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "integrate_noalloc needs a CUDA device");
  if (c->graphs.empty()) return fail(c, AE_ERR_STATE, "no graphs loaded");
  if (gid < 0 || gid >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  if (nsamp == 0 || nsamp > kNaMaxSamples)
    return fail(c, AE_ERR_ARG, "n_samples must be 1..524288 for ae_integrate_noalloc "
                               "(fixed scratch of the no-allocation path)");
  if (c->device >= 256) return fail(c, AE_ERR_ARG, "device index too large for the no-allocation path");
  CUDA_TRY(c, cudaSetDevice(c->device));
  unsigned char *scr = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[c->device]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail(c, AE_ERR_CUDA, std::string("cudaGetSymbolAddress(g_noalloc_scratch): ") + cudaGetErrorString(e));
      g_noalloc_addr[c->device] = p;
    }
    scr = (unsigned char *)g_noalloc_addr[c->device];
  }
  Partial *part = (Partial *)scr;
  unsigned long long *qcount = (unsigned long long *)(scr + kNaPartBytes);
  Partial *result = (Partial *)(scr + kNaPartBytes + 128);
  unsigned long long *queue = (unsigned long long *)(scr + kNaQueueOff);
  double *y_off = (double *)(scr + kNaYOff);
  unsigned char *flag = scr + kNaFlagOff;
  GraphDev &G = c->graphs[gid].dev;
  int bs = pick_block_for(c, (const void *)integrate_kernel, G.nslots, 8, kStageBytes);
  if (bs < 0) return fail(c, AE_ERR_STATE, "tape slot file does not fit in shared memory");
  size_t smem = kStageBytes + (size_t)bs * G.nslots * 8;
  CUDA_TRY(c, cudaFuncSetAttribute(integrate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = c->opts.ctas_per_sm;
  if (per_sm <= 0) {
    CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, integrate_kernel, bs, smem));
    if (per_sm < 1) per_sm = 1;
  }
  uint64_t grid = std::min<uint64_t>((uint64_t)c->sm_count * per_sm, (uint64_t)kNaMaxGrid);
  if (grid * bs > nsamp) grid = std::max<uint64_t>(1, (nsamp + bs - 1) / bs);
  int *werr = (int *)(qcount + 1);   // wait-timeout flag
  // what must start at zero: the queue counter, the timeout flag and the
  // per-sample flags
  CUDA_TRY(c, cudaMemsetAsync(qcount, 0, 2 * sizeof(unsigned long long), c->stream));
  CUDA_TRY(c, cudaMemsetAsync(flag, 0, nsamp, c->stream));
  integrate_kernel<<<(unsigned)grid, bs, smem, c->stream>>>(G, 0, nsamp, seed, c->opts.dd_tol, part, queue,
                                                            kNaMaxSamples, qcount, werr, kWaitCycles, 0);
  CUDA_TRY(c, cudaGetLastError());
  int bsd = pick_block_for(c, (const void *)dd_dense_kernel, G.nslots, 16);
  if (bsd < 0) return fail(c, AE_ERR_STATE, "double-double slot file does not fit in shared memory");
  size_t sm2 = (size_t)bsd * G.nslots * 16;
  CUDA_TRY(c, cudaFuncSetAttribute(dd_dense_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
  dd_dense_kernel<<<(unsigned)(c->sm_count * 2), bsd, sm2, c->stream>>>(G, 0, seed, queue, qcount, y_off, flag,
                                                                        c->opts.dd_tol);
  CUDA_TRY(c, cudaGetLastError());
  noalloc_reduce_kernel<<<1, 256, 0, c->stream>>>(part, (int)grid, y_off, flag, nsamp, result);
  CUDA_TRY(c, cudaGetLastError());
  Partial r;
  int herr = 0;
  CUDA_TRY(c, cudaMemcpyAsync(&r, result, sizeof(Partial), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaMemcpyAsync(&herr, werr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (herr) return fail(c, AE_ERR_TIMEOUT, "integrate_noalloc: a tape-staging wait ran out");
  std::memset(out, 0, sizeof(*out));
  out->sum_y = r.sy_hi + r.sy_lo;
  out->sum_y2 = r.sy2_hi + r.sy2_lo;
  out->n = r.n;
  out->n_dd = r.n_flag;
  out->n_nonfinite = r.n_overflow;
  out->max_y2 = r.max_y2;
  ae_result_finish(out, c->graphs[gid].g.mult, r.sa_hi + r.sa_lo);
  out->launches = 3;
  return AE_OK;
}

extern "C" int ae_eval_samples_dd(ae_ctx *c, int gid, uint64_t first, uint64_t count, uint64_t seed,
                                  double *I, double *K, double *y, double *E) {
  if (!c) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "eval_samples_dd needs a CUDA device");
  if (gid < 0 || gid >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  if (count == 0) return AE_OK;
  CUDA_TRY(c, cudaSetDevice(c->device));
  GraphDev &G = c->graphs[gid].dev;
  int bs = pick_block_for(c, (const void *)eval_dd_kernel, G.nslots, 16, kStageBytes);
  if (bs < 0) return fail(c, AE_ERR_STATE, "tape slot file does not fit in shared memory");
  size_t smem = kStageBytes + (size_t)bs * G.nslots * 16;
  CUDA_TRY(c, cudaFuncSetAttribute(eval_dd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = dump_grid(c, (const void *)eval_dd_kernel, bs, smem, count);
  double *d = nullptr;
  CUDA_TRY(c, cudaMalloc(&d, count * 4 * 8 + 16));
  int *derr = reinterpret_cast<int *>(d + 4 * count);
  cudaError_t e = cudaMemsetAsync(derr, 0, sizeof(int), c->stream);
  if (e == cudaSuccess) {
    eval_dd_kernel<<<grid, bs, smem, c->stream>>>(G, first, count, seed, d, d + count, d + 2 * count, d + 3 * count,
                                                  derr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  int herr = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && I) e = cudaMemcpy(I, d, count * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && K) e = cudaMemcpy(K, d + count, count * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && y) e = cudaMemcpy(y, d + 2 * count, count * 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && E) e = cudaMemcpy(E, d + 3 * count, count * 8, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e == cudaSuccess && herr) return fail(c, AE_ERR_TIMEOUT, "eval_samples_dd: a tape-staging wait ran out");
  if (e != cudaSuccess) return fail(c, AE_ERR_CUDA, std::string("eval_samples_dd: ") + cudaGetErrorString(e));
  return AE_OK;
}

extern "C" int ae_philox(ae_ctx *c, const uint32_t *ctr, const uint32_t *key, uint32_t *out, size_t count) {
  if (!c || !ctr || !key || !out) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "philox needs a CUDA device");
  if (count == 0) return AE_OK;
  CUDA_TRY(c, cudaSetDevice(c->device));
  uint32_t *d = nullptr;
  CUDA_TRY(c, cudaMalloc(&d, count * 40));
  uint32_t *dc = d, *dk = d + 4 * count, *dout = dk + 2 * count;
  cudaError_t e = cudaMemcpy(dc, ctr, count * 16, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dk, key, count * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    philox_kernel<<<(unsigned)((count + 255) / 256), 256, 0, c->stream>>>(dc, dk, dout, count);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, count * 16, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(c, AE_ERR_CUDA, std::string("philox: ") + cudaGetErrorString(e));
  return AE_OK;
}

extern "C" int ae_fp64_peak(ae_ctx *c, double *tflops) {
  if (!c || !tflops) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "fp64 probe needs a CUDA device");
  CUDA_TRY(c, cudaSetDevice(c->device));
  double *sink = nullptr;
  CUDA_TRY(c, cudaMalloc(&sink, 8));
  const int iters = 1 << 14, bs = 256;
  int per_sm = 0;
  CUDA_TRY(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dfma_probe_kernel, bs, 0));
  unsigned grid = (unsigned)(c->sm_count * std::max(per_sm, 1));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  double best = 0;
  for (int rep = 0; rep < 6; ++rep) {
    cudaEventRecord(e0, c->stream);
    dfma_probe_kernel<<<grid, bs, 0, c->stream>>>(iters, 0.999999, 1e-7, sink);
    cudaEventRecord(e1, c->stream);
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) { cudaFree(sink); return fail(c, AE_ERR_CUDA, cudaGetErrorString(e)); }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    double fl = 2.0 * 8.0 * iters * (double)grid * bs;
    if (rep > 0) best = std::max(best, fl / (ms * 1e-3) / 1e12);
  }
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  cudaFree(sink);
  *tflops = best;
  return AE_OK;
}

extern "C" int ae_density_tables(ae_ctx *c, int gid, double *deg, double *phi) {
  if (!c || !deg || !phi) return AE_ERR_ARG;
  if (gid < 0 || gid >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  const DensityTables &d = c->graphs[gid].dens;
  size_t T = (size_t)1 << d.M;
  for (int k = 0; k < 3; ++k) {
    std::copy(d.deg[k].begin(), d.deg[k].end(), deg + k * T);
    std::copy(d.phi[k].begin(), d.phi[k].end(), phi + k * T);
  }
  return AE_OK;
}

extern "C" int ae_subgraphs(ae_ctx *c, int gid, int *buf, int cap, int *len) {
  if (!c || !len) return AE_ERR_ARG;
  if (gid < 0 || gid >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  std::vector<int> v;
  for (auto &s : c->graphs[gid].subs) { v.push_back(s.lo); v.push_back(s.hi); v.push_back(s.se ? 0 : (s.inJ ? 2 : 1)); }
  *len = (int)v.size();
  if (buf && cap >= (int)v.size()) std::copy(v.begin(), v.end(), buf);
  else if (buf) return fail(c, AE_ERR_ARG, "buffer too small");
  return AE_OK;
}

extern "C" int ae_terms(ae_ctx *c, int gid, int *buf, int cap, int *len) {
  if (!c || !len) return AE_ERR_ARG;
  if (gid < 0 || gid >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  const LoadedGraph &lg = c->graphs[gid];
  std::vector<int> v;
  for (auto &t : lg.terms) {
    v.push_back(t.sign); v.push_back((int)t.elems.size());
    for (size_t i = 0; i < t.elems.size(); ++i) {
      v.push_back(lg.subs[t.elems[i]].lo); v.push_back(lg.subs[t.elems[i]].hi); v.push_back(t.ops[i]);
    }
  }
  *len = (int)v.size();
  if (buf && cap >= (int)v.size()) std::copy(v.begin(), v.end(), buf);
  else if (buf) return fail(c, AE_ERR_ARG, "buffer too small");
  return AE_OK;
}

// Test hook: the FP64 integration kernel with its first tape copy left out
// and a short bound on the wait for it; the wait runs out with nothing in
// flight and the call fails the way a real timeout does.
extern "C" int aetest_stage_timeout(ae_ctx *c, int gid, long long wait_cycles) {
  if (!c) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "needs a CUDA device");
  if (gid < 0 || gid >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  if (wait_cycles < 1 || wait_cycles > kWaitCycles) return fail(c, AE_ERR_ARG, "wait_cycles must be 1..4e9");
  CUDA_TRY(c, cudaSetDevice(c->device));
  GraphDev &G = c->graphs[gid].dev;
  const int bs = 32;
  const size_t smem = kStageBytes + (size_t)bs * G.nslots * 8;
  if (smem > 224 * 1024) return fail(c, AE_ERR_STATE, "tape slot file does not fit in shared memory");
  int rc = ensure_scratch(c, 1, 65536);
  if (rc) return rc;
  CUDA_TRY(c, cudaFuncSetAttribute(integrate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  CUDA_TRY(c, cudaMemsetAsync(c->d_qcount, 0, 2 * sizeof(unsigned long long), c->stream));
  integrate_kernel<<<1, bs, smem, c->stream>>>(G, 0, bs, 0, c->opts.dd_tol, c->d_part, c->d_queue, c->queue_cap,
                                               c->d_qcount, (int *)(c->d_qcount + 1), wait_cycles, 1);
  CUDA_TRY(c, cudaGetLastError());
  unsigned long long hq[2] = {0, 0};
  CUDA_TRY(c, cudaMemcpyAsync(hq, c->d_qcount, sizeof(hq), cudaMemcpyDeviceToHost, c->stream));
  CUDA_TRY(c, cudaStreamSynchronize(c->stream));
  if (hq[1]) return fail(c, AE_ERR_TIMEOUT, "integrate: a tape-staging wait ran out");
  return fail(c, AE_ERR_STATE, "the wait did not run out");
}

// Test hook: the learned sampler's fused-multiply-add exp2/log2 next to the
// device library's exp2/log2 on the same arguments (accuracy test).
__global__ void fast_elem_kernel(const double *x, const double *y, size_t n, double *out) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[4 * i] = fexp2(x[i]);
  out[4 * i + 1] = exp2(x[i]);
  out[4 * i + 2] = flog2(y[i]);
  out[4 * i + 3] = log2(y[i]);
}

extern "C" int aetest_fast_elem(ae_ctx *c, const double *x, const double *y, size_t n, double *out) {
  if (!c || !x || !y || !out || n == 0) return AE_ERR_ARG;
  if (c->device < 0) return fail(c, AE_ERR_NODEV, "needs a CUDA device");
  CUDA_TRY(c, cudaSetDevice(c->device));
  double *d = nullptr;
  CUDA_TRY(c, cudaMalloc(&d, n * 6 * sizeof(double)));
  cudaError_t e = cudaMemcpy(d, x, n * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(d + n, y, n * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    fast_elem_kernel<<<(unsigned)((n + 255) / 256), 256, 0, c->stream>>>(d, d + n, n, d + 2 * n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = cudaMemcpy(out, d + 2 * n, n * 4 * sizeof(double), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return fail(c, AE_ERR_CUDA, std::string("fast_elem: ") + cudaGetErrorString(e));
  return AE_OK;
}

extern "C" int aetest_tape_replay(ae_ctx *c, int gid, const double *z, size_t count, double *I, double *K,
                                  double *E) {
  if (!c || !z || !I || !K) return AE_ERR_ARG;
  if (gid < 0 || gid >= (int)c->graphs.size()) return fail(c, AE_ERR_ARG, "graph id out of range");
  const Tape &t = c->graphs[gid].tape;
  for (size_t i = 0; i < count; ++i) tape_replay(t, z + i * t.M, I + i, K + i, E ? E + i : nullptr);
  return AE_OK;
}
