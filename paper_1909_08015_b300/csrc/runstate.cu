// Run state of a long integration (Sec. IV.C: the integrals of all graphs
// are computed simultaneously, block after block, over a campaign): per
// loaded graph the next sample index of its counter-based stream and the
// running sums, the run's estimate (Eqs. eq_integral_approx, eq_sigma_down,
// eq_sigma_sum), checkpoints and the merge of several ranks' runs.  Host
// code; ae_run_step (runtime.cu) adds one batched launch to the run.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "context.h"

namespace {

// sum (hi, lo) += x: Knuth's two-sum, then renormalisation
void dd_add_host(double *p, double x) {
  const double s = p[0] + x;
  const double bb = s - p[0];
  const double e = (p[0] - (s - bb)) + (x - bb);
  const double lo = p[1] + e;
  const double r = s + lo;
  p[1] = lo - (r - s);
  p[0] = r;
}

// CRC-64/XZ (ECMA-182 polynomial, reflected, initial value and final xor
// all ones), bitwise
uint64_t crc64(const unsigned char *p, size_t n) {
  uint64_t c = ~0ull;
  for (size_t i = 0; i < n; ++i) {
    c ^= p[i];
    for (int k = 0; k < 8; ++k) c = (c >> 1) ^ (0xC96C5795D7870F42ull & (0ull - (c & 1)));
  }
  return ~c;
}

constexpr char kMagic[8] = {'A', 'E', 'R', 'U', 'N', 'C', 'K', '1'};

struct CkptHead {
  char magic[8];
  uint32_t loops, ngraphs, rng, reserved;
  uint64_t seed;
};
struct CkptGraph {
  int32_t canonical_id, mult;
  ae_run_graph st;
};

}  // namespace

void ae_run_fold(ae_ctx *c, int gid, const ae_graph_result &r, uint64_t count) {
  ae_run_graph &s = c->run[gid];
  dd_add_host(s.sum_y, r.sum_y);
  dd_add_host(s.sum_y2, r.sum_y2);
  dd_add_host(s.sum_abs, r.mean_abs * (double)r.n);
  if (r.max_y2 > s.max_y2) s.max_y2 = r.max_y2;
  s.n += r.n;
  s.n_dd += r.n_dd;
  s.n_zero += r.n_nonfinite;
  s.next += count;
}

extern "C" int ae_run_reset(ae_ctx *c, uint64_t seed) {
  if (!c) return AE_ERR_ARG;
  if (c->graphs.empty()) return ae_fail(c, AE_ERR_STATE, "no graphs loaded");
  c->run.assign(c->graphs.size(), ae_run_graph{});
  c->run_seed = seed;
  return AE_OK;
}

extern "C" int ae_run_add(ae_ctx *c, int gid, const ae_graph_result *r, uint64_t count) {
  if (!c || !r) return AE_ERR_ARG;
  if (gid < 0 || gid >= (int)c->graphs.size()) return ae_fail(c, AE_ERR_ARG, "graph id out of range");
  if (!std::isfinite(r->sum_y) || !std::isfinite(r->sum_y2) || !std::isfinite(r->mean_abs))
    return ae_fail(c, AE_ERR_NONFINITE, "result sums must be finite");
  if (c->run[gid].next + count < c->run[gid].next) return ae_fail(c, AE_ERR_ARG, "sample index overflows 2^64");
  ae_run_fold(c, gid, *r, count);
  return AE_OK;
}

extern "C" int ae_run_get(ae_ctx *c, ae_run_graph *out, int n, uint64_t *seed) {
  if (!c || !out) return AE_ERR_ARG;
  if (n != (int)c->graphs.size()) return ae_fail(c, AE_ERR_ARG, "n must be the number of loaded graphs");
  for (int i = 0; i < n; ++i) out[i] = c->run[i];
  if (seed) *seed = c->run_seed;
  return AE_OK;
}

extern "C" int ae_run_merge(ae_ctx *c, const ae_run_graph *o, int n) {
  if (!c || !o) return AE_ERR_ARG;
  if (n != (int)c->graphs.size()) return ae_fail(c, AE_ERR_ARG, "n must be the number of loaded graphs");
  for (int i = 0; i < n; ++i) {
    ae_run_graph &s = c->run[i];
    dd_add_host(s.sum_y, o[i].sum_y[0]); dd_add_host(s.sum_y, o[i].sum_y[1]);
    dd_add_host(s.sum_y2, o[i].sum_y2[0]); dd_add_host(s.sum_y2, o[i].sum_y2[1]);
    dd_add_host(s.sum_abs, o[i].sum_abs[0]); dd_add_host(s.sum_abs, o[i].sum_abs[1]);
    if (o[i].max_y2 > s.max_y2) s.max_y2 = o[i].max_y2;
    s.n += o[i].n;
    s.n_dd += o[i].n_dd;
    s.n_zero += o[i].n_zero;
  }
  return AE_OK;
}

extern "C" int ae_run_estimate(ae_ctx *c, double *value, double *sigma, double *sigma_up, ae_graph_result *per) {
  if (!c) return AE_ERR_ARG;
  if (c->graphs.empty()) return ae_fail(c, AE_ERR_STATE, "no graphs loaded");
  double v = 0, s2 = 0, u2 = 0;
  for (size_t i = 0; i < c->graphs.size(); ++i) {
    const ae_run_graph &s = c->run[i];
    ae_graph_result r;
    std::memset(&r, 0, sizeof(r));
    r.sum_y = s.sum_y[0] + s.sum_y[1];
    r.sum_y2 = s.sum_y2[0] + s.sum_y2[1];
    r.n = s.n;
    r.n_dd = s.n_dd;
    r.n_nonfinite = s.n_zero;
    r.max_y2 = s.max_y2;
    ae_result_finish(&r, c->graphs[i].g.mult, s.sum_abs[0] + s.sum_abs[1]);
    v += r.value;
    s2 += r.sigma * r.sigma;
    u2 += r.sigma_up * r.sigma_up;
    if (per) per[i] = r;
  }
  if (value) *value = v;
  if (sigma) *sigma = std::sqrt(s2);
  if (sigma_up) *sigma_up = std::sqrt(u2);
  return AE_OK;
}

extern "C" int ae_checkpoint(ae_ctx *c, const char *path) {
  if (!c || !path) return AE_ERR_ARG;
  if (c->graphs.empty()) return ae_fail(c, AE_ERR_STATE, "no graphs loaded");
  std::vector<unsigned char> buf(sizeof(CkptHead) + c->graphs.size() * sizeof(CkptGraph) + 8, 0);
  CkptHead h;
  std::memset(&h, 0, sizeof(h));
  std::memcpy(h.magic, kMagic, 8);
  h.loops = (uint32_t)c->loops;
  h.ngraphs = (uint32_t)c->graphs.size();
  h.rng = (uint32_t)c->opts.rng;
  h.seed = c->run_seed;
  std::memcpy(buf.data(), &h, sizeof(h));
  for (size_t i = 0; i < c->graphs.size(); ++i) {
    CkptGraph g;
    std::memset(&g, 0, sizeof(g));
    g.canonical_id = c->graphs[i].canonical_id;
    g.mult = c->graphs[i].g.mult;
    g.st = c->run[i];
    std::memcpy(buf.data() + sizeof(CkptHead) + i * sizeof(CkptGraph), &g, sizeof(g));
  }
  const size_t body = buf.size() - 8;
  const uint64_t crc = crc64(buf.data(), body);
  std::memcpy(buf.data() + body, &crc, 8);
  const std::string tmp = std::string(path) + ".tmp";
  FILE *f = std::fopen(tmp.c_str(), "wb");
  if (!f) return ae_fail(c, AE_ERR_ARG, "checkpoint: cannot open " + tmp);
  const size_t w = std::fwrite(buf.data(), 1, buf.size(), f);
  const int cl = std::fclose(f);
  if (w != buf.size() || cl != 0) {
    std::remove(tmp.c_str());
    return ae_fail(c, AE_ERR_ARG, "checkpoint: write failed");
  }
  if (std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return ae_fail(c, AE_ERR_ARG, std::string("checkpoint: cannot rename to ") + path);
  }
  return AE_OK;
}

extern "C" int ae_resume(ae_ctx *c, const char *path) {
  if (!c || !path) return AE_ERR_ARG;
  if (c->graphs.empty()) return ae_fail(c, AE_ERR_STATE, "no graphs loaded");
  FILE *f = std::fopen(path, "rb");
  if (!f) return ae_fail(c, AE_ERR_ARG, std::string("resume: cannot open ") + path);
  std::vector<unsigned char> buf;
  unsigned char tmp[4096];
  size_t r;
  while ((r = std::fread(tmp, 1, sizeof(tmp), f)) > 0) buf.insert(buf.end(), tmp, tmp + r);
  std::fclose(f);
  const size_t want = sizeof(CkptHead) + c->graphs.size() * sizeof(CkptGraph) + 8;
  if (buf.size() < sizeof(CkptHead) + 8 || std::memcmp(buf.data(), kMagic, 8) != 0)
    return ae_fail(c, AE_ERR_STATE, "resume: not a run checkpoint (or truncated)");
  if (buf.size() != want) return ae_fail(c, AE_ERR_STATE, "resume: truncated or of another graph set");
  uint64_t crc;
  std::memcpy(&crc, buf.data() + want - 8, 8);
  if (crc != crc64(buf.data(), want - 8)) return ae_fail(c, AE_ERR_STATE, "resume: checksum mismatch (corrupt file)");
  CkptHead h;
  std::memcpy(&h, buf.data(), sizeof(h));
  if ((int)h.loops != c->loops || h.ngraphs != c->graphs.size())
    return ae_fail(c, AE_ERR_STATE, "resume: the checkpoint holds another graph set");
  if ((int)h.rng != c->opts.rng) return ae_fail(c, AE_ERR_STATE, "resume: the checkpoint used another generator");
  std::vector<ae_run_graph> st(c->graphs.size());
  for (size_t i = 0; i < c->graphs.size(); ++i) {
    CkptGraph g;
    std::memcpy(&g, buf.data() + sizeof(CkptHead) + i * sizeof(CkptGraph), sizeof(g));
    if (g.canonical_id != c->graphs[i].canonical_id || g.mult != c->graphs[i].g.mult)
      return ae_fail(c, AE_ERR_STATE, "resume: the checkpoint holds another graph set");
    st[i] = g.st;
  }
  c->run.swap(st);
  c->run_seed = h.seed;
  return AE_OK;
}
