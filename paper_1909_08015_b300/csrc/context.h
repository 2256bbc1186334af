// Host-side context of libae (the object behind the opaque ae_ctx handle).
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/ae.h"
#include "ae_internal.h"
#include "kernels.cuh"

using namespace ae;
using aek::GraphDev;
using aek::Partial;

// Learned proposal state of one graph (device tables and network).
struct LearnedState {
  bool active = false;
  double beta = 0.1;
  void *mem = nullptr;      // device block holding tables and weights
  size_t bytes = 0;
  std::vector<float> master;   // FP32 master weights (host copy after training)
};

struct LoadedGraph {
  Graph g;
  std::vector<Sub> subs;
  std::vector<Term> terms;
  Tape tape;
  DensityTables dens;
  CompileStats st;
  GraphDev dev{};
  LearnedState learned;
  int canonical_id = 0;     // index in the full canonical list of its loop order
};

struct ae_ctx {
  int device = -1;
  ae_opts opts;
  std::string err;
  std::vector<LoadedGraph> graphs;
  int loops = 0;
  void *arena = nullptr;
  size_t arena_bytes = 0;
  int sm_count = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = true;
  // scratch
  Partial *d_part = nullptr; size_t part_cap = 0;
  uint32_t *d_mrg = nullptr;    // MRG32k3a jump table on the device (opts.rng == 1)
  double train_cost_ratio = 0;  // R of the proposal's training weights |y| / sqrt(1 + R [re-evaluated])
  unsigned long long *d_queue = nullptr; size_t queue_cap = 0;
  unsigned long long *d_qcount = nullptr;
  double *d_yq = nullptr;
  int *d_qstat = nullptr;
  // autotuner cache: graph-set key -> (block size, chunk size)
  std::map<std::string, std::pair<int, unsigned long long>> tune_cache;
  void *bbuf = nullptr;         // batched-launch buffers (grow only)
  size_t bbuf_bytes = 0;
  int last_tune_block = 0;
  unsigned long long last_tune_chunk = 0;
  // the batched launch captured as a CUDA graph, kept for the next call with
  // the same launch shape, buffers and scalar arguments (a run's steps)
  std::string gkey;
  cudaGraphExec_t gexec = nullptr;
  cudaEvent_t gev[3] = {nullptr, nullptr, nullptr};
  // run state (ae_run_*): one entry per loaded graph
  uint64_t run_seed = 0;
  std::vector<ae_run_graph> run;
};


int ae_fail(ae_ctx *c, int code, const std::string &msg);
// mean, sigma_down and sigma_up of a result from its sums (runtime.cu)
void ae_result_finish(ae_graph_result *r, int mult, double sum_abs);
// fold a result of `count` samples of one graph into the run (runstate.cu)
void ae_run_fold(ae_ctx *c, int gid, const ae_graph_result &r, uint64_t count);
// uploads the sampler's log2/exp2 tables into learned.cu's constant memory
cudaError_t ae_learned_upload_tables();
