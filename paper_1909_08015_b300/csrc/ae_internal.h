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
// table-driven forms used by the sampler and density (tables from the series)
double ae_log2t(double x);
double ae_exp2t(double x);
const double *ae_exp2_table();   // 2^(j/32), j = 0..31
// host Philox4x32-10 (same definition as the device generator)
void philox_host(uint32_t c[4], uint32_t k0, uint32_t k1);
// MRG32k3a jump matrices A1^(2^k), A2^(2^k), k = 0..159 (18 words per k)
const uint32_t *mrg_jump_table();
// tables and coefficients of the device's fused-multiply-add exp2/log2
const double *ae_fast_tables();
constexpr int kFastTabs = 177;
const double *ae_log2_table();   // log2(j/32), j = 24..48

// ------------------------------------------------------------- tapes -----
// Operations of the integrand compiler's intermediate program (value ids,
// constants in a per-graph pool).  They are lowered to the device instruction
// format Ins below.
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
  T_G = 13,    // d = a * (b or K[b]) + (c or K[c]); flags G_BK, G_CK
  T_GA = 14,   // d = |a| * |b or K[b]| + |c or K[c]|   (magnitude twin)
  T_GAC = 15,  // d = |d| + |a| * |b or K[b]|           (accumulating twin)
};
enum : uint8_t { G_BK = 1, G_CK = 2 };

// One device instruction (32 bytes).  Almost every instruction is the same
// fused multiply-add
//     S[d] = S[a] * (I_BK ? kb : S[b]) + (I_CK ? kc : S[c]),
// so the interpreter needs no dispatch beyond one test of the special code
// (division, absolute value, accumulated absolute value).  With I_AB the
// three operands enter the fused multiply-add as absolute values; those
// instructions carry the magnitudes of the running error bound.  Slot fields are
// byte offsets (slot * 8) into the thread's row of the slot file; a field
// that names an immediate holds 0 (a valid slot).  kbi/kci index the
// constant pool (hi, lo) so that the double-double evaluation can use the
// constants' low parts.
struct Ins {
  uint16_t op;          // flags I_* | special code << 8
  uint16_t d, a, b, c;  // byte offsets in the slot row
  uint16_t kbi, kci;    // constant-pool indices of kb, kc
  uint16_t pad;
  double kb, kc;
};
static_assert(sizeof(Ins) == 32, "Ins must be 32 bytes");
enum : uint16_t {
  I_BK = 1, I_CK = 2,
  I_AB = 4,           // S[d] = |S[a]| * |kb or S[b]| + |kc or S[c]|
  // hints for the double-double evaluation (the FP64 interpreter ignores them)
  I_KX = 8,           // every constant operand is an exact double (no low part)
  I_C0 = 16,          // c is the constant 0: a product
  I_B1 = 32,          // b is the constant +1 or -1: a sum
  I_DIV = 1 << 8,     // S[d] = S[a] / S[b]
  I_ABS = 2 << 8,     // S[d] = |S[a]|
  I_ADDABS = 3 << 8,  // S[d] = S[c] + |S[a]|
};

struct Tape {
  std::vector<Ins> code;
  std::vector<double> khi, klo;  // constant pool
  int nslots = 0;                 // row pitch of the slot file (odd: conflict-free rows)
  int out_I = -1, out_K = -1;     // output slots
  int out_E = -1;                 // slot of the rounding-error bound of I
  int depth = 0;                  // roundings along the deepest chain into I
  double flops = 0;               // FP64 flops per evaluation (FMA = 2)
  double flops_bound = 0;         // of which the error bound's magnitude twins
  double flops_dd = 0;            // FP64 flops of one double-double evaluation (FMA = 2)
  int M = 0;
  int n_terms = 0;
};

struct CompileStats {
  int n_terms = 0, n_factors = 0, n_monomials = 0;
};
Tape compile_integrand(const Graph &g, CompileStats *st);

// Host replay of a tape (test harness only; not an evaluation path of the
// library's integration calls).
void tape_replay(const Tape &t, const double *z, double *I, double *K, double *E = nullptr);

}  // namespace ae
