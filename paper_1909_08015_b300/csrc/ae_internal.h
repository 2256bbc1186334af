// Internal declarations of libae: graph set, forests, densities, integrand
// compiler and tapes.  Not part of the public C ABI (see include/ae.h).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace ae {

// ------------------------------------------------------------- graphs ----
// One vertex graph without lepton loops (Sec. I): an electron path with
// vertices 0..2n; vertex s holds the external photon, every other vertex one
// end of an internal photon (partner[v]).  The stored orientation is the one
// whose path word is the canonical (lexicographically smaller) word.
struct Graph {
  int n = 0;
  int s = 0;
  std::vector<int> partner;   // -1 at s
  std::vector<int> word;      // -1 at s, photons numbered by first appearance
  int mult = 1;               // 2 unless the graph equals its mirror image
  int klass[3] = {0, 0, 0};   // (k, m, m') of Sec. V
  int nverts() const { return 2 * n + 1; }
  int M() const { return 3 * n - 1; }
};

std::vector<Graph> enumerate_graphs(int n);

// A line of the graph: electron line e_i joins v_{i-1} -> v_i (i = 1..2n);
// photon line joins a < b.
struct Line {
  bool photon;
  int a, b;   // electron: a = i-1, b = i ; photon: a < b
  bool operator<(const Line &o) const {
    if (photon != o.photon) return !photon;
    if (a != o.a) return a < o.a;
    return b < o.b;
  }
  bool operator==(const Line &o) const { return photon == o.photon && a == o.a && b == o.b; }
};

// Index of the M = 3n-1 Feynman parameters: 0 = merged pair of electron lines
// at the external vertex, then the other electron lines along the path, then
// photons in order of first appearance.
int line_param(const Graph &g, const Line &l);
std::vector<Line> photon_lines(const Graph &g);

// ------------------------------------------------------------ forests ----
// UV-divergent subgraph = a path interval [lo..hi] (Sec. II).
struct Sub {
  int lo = 0, hi = 0;
  bool se = false;       // self-energy (N_gamma = 0) or vertexlike
  bool inJ = false;      // contains the external-photon vertex
  int ext_photon_vertex = -1;  // vertex inside holding its external photon
};
enum Op : int { OP_A = 0, OP_U = 1, OP_L = 2, OP_LmU = 3 };
struct Term {
  int sign = 1;
  std::vector<int> elems;   // indices into subgraph list; elems[0] = G
  std::vector<int> ops;     // operator per element
};
std::vector<Sub> divergent_subgraphs(const Graph &g);
std::vector<Term> rnew_terms(const Graph &g, const std::vector<Sub> &subs);

// ------------------------------------------------------------ density ----
struct DensityConsts {
  double C2 = 0.03, C3 = 0.01, C4 = 0.06, D = 0.75;  // Calc 2
  double CsubI = 0.2, CsubSE = 0.0, CsubO = 0.2;
  double CbigZ = 0.256, CbigF = 0.839, Cadd = 0.786;  // kept, unused
  double deg_max = 1.0;                                 // cap on Deg(s); <= 0: none
};
// deg[k][mask], phi[k][mask] for the three sector densities g1, g3, g4.
struct DensityTables {
  int M = 0;
  std::vector<double> deg[3], phi[3];
  double C[4] = {0, 0, 0, 0};   // weights of g1, g2, g3, g4
  double log2_fact = 0;         // log2 (M-1)!
};
DensityTables build_density(const Graph &g, const DensityConsts &c);

// Elementary functions shared by host code and device code bit for bit:
// plain IEEE add/multiply, series from their published definitions.
double ae_log2(double x);
double ae_exp2(double x);

// ------------------------------------------------------------- tapes -----
// One tape instruction (8 bytes).  Slots hold FP64 values; z occupies slots
// 0..M-1 on entry.  Constants live in a per-graph pool (hi, lo) pairs.
enum TapeOp : uint8_t {
  T_ADD = 1,   // d = a + b
  T_SUB = 2,   // d = a - b
  T_MUL = 3,   // d = a * b
  T_DIV = 4,   // d = a / b
  T_FMA = 5,   // d = d + a * b        (accumulate)
  T_FMAC = 6,  // d = d + K[b] * a     (accumulate with constant)
  T_MULC = 7,  // d = K[b] * a
  T_CONST = 8, // d = K[b]
  T_ABS = 9,   // d = |a|
  T_NEG = 10,  // d = -a
  T_ZERO = 11, // d = 0
  T_ADDABS = 12, // d = d + |a|
  // register accumulator r (one per thread): accumulation chains without a
  // shared-memory round trip per step
  T_RZERO = 13,  // r = 0
  T_RFMAC = 14,  // r = r + K[b] * a
  T_RFMA = 15,   // r = r + a * b
  T_RST = 16,    // d = r
  // Horner form of a sum of monomials: a stack of register accumulators
  // R[0..kHLevels-1]; the level k of an instruction is op - base.  Each op is
  // one FMA; "first" ops start R[k] from the node's own coefficient K[d].
  T_HFL = 32,    // R[k] = a * K[b] + K[d]      (first edge, leaf child)
  T_HL = 48,     // R[k] = a * K[b] + R[k]      (leaf child)
  T_HFU = 64,    // R[k] = a * R[k+1] + K[d]    (first edge, inner child)
  T_HU = 80,     // R[k] = a * R[k+1] + R[k]    (inner child)
  T_HST = 96,    // d = R[0]
};
constexpr int kHLevels = 12;   // register accumulators of the Horner stack
inline bool is_horner(int op) { return op >= T_HFL && op < T_HST; }
inline int horner_kind(int op) { return op & ~15; }
inline int horner_level(int op) { return op & 15; }
struct Ins {
  uint8_t op;
  uint8_t pad;
  uint16_t d, a, b;
};
static_assert(sizeof(Ins) == 8, "Ins must be 8 bytes");

struct Tape {
  std::vector<Ins> code;
  std::vector<double> khi, klo;  // constant pool
  int nslots = 0;
  int out_I = -1, out_K = -1;     // output slots
  double flops = 0;               // FP64 flops per evaluation (FMA = 2)
  int M = 0;
  int n_terms = 0;
};

struct CompileStats {
  int n_terms = 0, n_factors = 0, n_monomials = 0;
};
Tape compile_integrand(const Graph &g, CompileStats *st);

// Host replay of a tape (test harness only; not an evaluation path of the
// library's integration calls).
void tape_replay(const Tape &t, const double *z, double *I, double *K);

}  // namespace ae
