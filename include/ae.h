/* libae: B300-native Monte Carlo integration of the divergence-subtracted
 * Feynman-parametric integrands of QED vertex graphs without lepton loops
 * (S. Volkov, arXiv:1909.08015).
 *
 * C ABI.  Plain pointers and sizes only.  Every entry point returns 0 on
 * success or a negative AE_ERR_* code; no exception crosses the boundary and
 * the message of the last failure is read with ae_last_error().
 *
 * Ownership: output buffers are caller-owned HOST memory unless stated
 * otherwise.  Device memory, streams and compiled integrand tapes are owned
 * by the context.  One context per host thread.
 */
#ifndef AE_H
#define AE_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AE_OK 0
#define AE_ERR_ARG (-1)       /* invalid argument (graph id, size, pointer) */
#define AE_ERR_CUDA (-2)      /* a CUDA runtime call failed                  */
#define AE_ERR_OOM (-3)       /* device or host allocation failed            */
#define AE_ERR_TIMEOUT (-4)   /* a bounded device wait ran out               */
#define AE_ERR_NONFINITE (-5) /* non-finite result where one is not allowed  */
#define AE_ERR_STATE (-6)     /* call out of order (e.g. no graphs loaded)   */
#define AE_ERR_NODEV (-7)     /* the call needs a CUDA device, none bound    */

typedef struct ae_ctx ae_ctx;

/* Options.  Defaults (ae_default_opts) are the Calc 2 settings of Sec. V:
 * C2 = 0.03, C3 = 0.01, C4 = 0.06, D = 0.75 (C1 = 1 - C2 - C3 - C4), and the
 * six Deg constants of Eq. eq_mc_settings. */
typedef struct ae_opts {
  double C2, C3, C4, D;              /* mixture weights of g2, g3, g4; g3 flattening */
  double C_subI, C_subSE, C_subO;    /* Deg(s) constants used by the library      */
  double C_bigZ, C_bigF, C_add;      /* Deg(s) constants kept, not used           */
  double deg_max;                    /* cap on Deg(s) (library reading: power
                                        counting sees only ultraviolet scaling,
                                        and infrared-type sets decay like
                                        lambda^1); <= 0 means no cap              */
  double dd_tol;                     /* acceptance of an FP64 value: its certified
                                        rounding-error bound, carried to y = I/g,
                                        at most dd_tol * max(|y|, the graph's
                                        floor, ae_set_accept_floor); others are
                                        re-evaluated in double-double under the
                                        same test, and count as zero if they fail
                                        it again.  Default 1e-10; <= 0: accept
                                        every finite value */
  int block_size;                    /* threads per CTA, 0 = automatic            */
  int ctas_per_sm;                   /* CTAs per SM for the grid, 0 = automatic   */
  void *stream;                      /* cudaStream_t to launch on; NULL = a stream
                                        owned by the context                      */
  int rng;                           /* 0 = Philox4x32-10 (Calc 2), 1 = MRG32k3a
                                        (Calc 1, L'Ecuyer 1999): sample i of graph
                                        g under seed s starts at output
                                        s 2^96 + g 2^80 + 64 i of the stream from
                                        the state (12345 x 6); set before loading */
  int grid_ctas;                     /* CTAs per FP64 integration launch, 0 =
                                        automatic (SMs x resident CTAs).  A small
                                        value makes every CTA run many rounds of
                                        samples (used by the parity tests); the
                                        results do not depend on it beyond the
                                        summation order */
} ae_opts;

/* The settings of the paper's second calculation (Sec. V, Calc 1):
 * MRG32k3a, C2 = 0.03, C3 = 0.035, C4 = 0.035, D = 0.75; the rest as in
 * ae_default_opts. */
void ae_calc1_opts(ae_opts *opts);

void ae_default_opts(ae_opts *opts);

/* Create a context.  cuda_device >= 0 binds that device; -1 creates a
 * host-only context (graph enumeration, compilation and table export work;
 * integration calls return AE_ERR_NODEV).  opts may be NULL (defaults). */
int ae_create(ae_ctx **out, int cuda_device, const ae_opts *opts);
void ae_destroy(ae_ctx *ctx);
const char *ae_last_error(const ae_ctx *ctx);

/* Enumerate every n-loop vertex graph without lepton loops (Sec. I: graphs
 * differing only in arrow direction count once), find its UV-divergent
 * subgraphs and forests (Sec. II), compile its subtracted integrand to a
 * tape and build its sampling tables (Sec. III.A).  Graph ids are 0..N-1 in
 * lexicographic order of the canonical path word.  Replaces any previously
 * loaded set.  1 <= loops <= 5. */
int ae_load_graphs(ae_ctx *ctx, int loops, int *n_graphs_out);

/* Load only the listed graphs (indices into the canonical list of `loops`
 * loops); the loaded graphs get ids 0..n_ids-1 in the given order, and each
 * keeps its canonical index as its Philox stream (graph word of the counter),
 * so a graph draws the same samples whichever set it is loaded with. */
int ae_load_graph_subset(ae_ctx *ctx, int loops, const int *canonical_ids, int n_ids, int *n_graphs_out);

/* Seeded choice of k graph indices out of n_total (Fisher-Yates driven by
 * Philox4x32-10, key = seed): the "seeded random subsets" of graphs used by
 * the 4- and 5-loop workloads.  Ascending output; returns 0, or -1 on bad
 * arguments.  No context needed. */
int ae_seeded_subset(uint64_t n_total, int k, uint64_t seed, int *out);

/* The canonical list of `loops` loops without compiling: *n_out = number of
 * graphs; klass (3 ints per graph: (k, m, m') of Sec. V, Table I) and mult
 * (1 int per graph) are filled when non-NULL and cap >= *n_out.  Returns 0,
 * or -1 on bad arguments.  No context needed. */
int ae_graph_classes(int loops, int *klass, int *mult, int cap, int *n_out);

typedef struct ae_graph_meta {
  int loops, M, mult;
  int klass[3];          /* (k, m, m') of Sec. V, Table I */
  int word[11];          /* path word, -1 = external vertex; 2n+1 entries */
  int n_subgraphs, n_terms, tape_len, nslots, n_monomials;
  double flops;          /* FP64 flops of one tape evaluation (FMA = 2), the
                            error bound's magnitude twins included */
  int canonical_id;      /* index in the full canonical list */
  int bound_depth;       /* D: roundings on the deepest chain into I; the
                            bound is gamma_D M_I (Sec. IV.A, library reading) */
  double flops_bound;    /* of flops, those of the magnitude twins */
  double flops_dd;       /* FP64 flops of one double-double evaluation of the
                            tape (FMA = 2), by the form each instruction takes */
} ae_graph_meta;
int ae_graph_info(ae_ctx *ctx, int graph_id, ae_graph_meta *out);

typedef struct ae_graph_result {
  double value;          /* mult * mean of y = I/g (Eq. eq_integral_approx)       */
  double sigma;          /* mult * sigma_down (Eq. eq_sigma_down)                  */
  double mean;           /* mean of y for one orientation                         */
  double sigma1;         /* sigma_down for one orientation                        */
  double mean_abs;       /* mean |y|, estimate of the integral of |I|            */
  double sum_y, sum_y2;  /* raw sums                                               */
  double max_y2;         /* largest single y^2                                     */
  uint64_t n;            /* samples                                               */
  uint64_t n_dd;         /* samples re-evaluated in double-double                 */
  uint64_t n_nonfinite;  /* samples that failed the acceptance test in double-double
                            too (or stayed non-finite): counted as zero          */
  double seconds;        /* device time of the graph's launches                    */
  uint64_t launches;     /* kernels launched for this graph                        */
  double kernel_seconds; /* device time of the FP64 integrand kernel alone         */
  uint64_t d2h_bytes;    /* bytes read back to the host for this graph's result     */
  uint64_t h2d_bytes;    /* bytes copied to the device for this call (batched: on
                            the first graph's entry)                                */
  double sigma_up;       /* mult * sigma_up: heuristic upper estimate of the
                            standard deviation (Sec. III.B; the paper's own
                            heuristic is in a reference that is not available,
                            this is the library's): sigma_up^2 = sigma_down^2 +
                            max y^2 / N^2, i.e. room for one more sample as large
                            as the largest seen.  sigma_up / sigma_down is near 1
                            when many samples carry sum y^2 and grows when one
                            sample dominates it                                 */
} ae_graph_result;

/* Integrate the listed graphs with n_samples samples each, Philox seed
 * `seed`.  value = sum_j mult_j mean_j, sigma^2 = sum_j (mult_j sigma_j)^2
 * (Eq. eq_sigma_sum).  per_graph may be NULL, else n_ids entries.  One
 * launch per graph.  Deterministic for given (ids, n_samples, seed, opts). */
int ae_integrate(ae_ctx *ctx, const int *graph_ids, int n_ids, uint64_t n_samples,
                 uint64_t seed, double *value, double *sigma, ae_graph_result *per_graph);

/* Samples first .. first+count-1 of one graph (the same Philox stream as
 * ae_integrate): resuming a run or sharding a graph by counter range.  The
 * sums of consecutive ranges add up to the sums of the whole range (up to
 * summation order). */
int ae_integrate_range(ae_ctx *ctx, int graph_id, uint64_t first, uint64_t count, uint64_t seed,
                       ae_graph_result *out);

/* Batched form: all listed graphs with their own sample counts in ONE
 * persistent launch: a work queue of (graph, counter range) chunks, longest
 * tapes first, taken by CTAs through one atomic counter; the flagged samples
 * of every graph are re-evaluated by one double-double launch; both launches
 * are captured in a CUDA graph.  Block and chunk size come from an
 * autotuner (timed trial runs on sample indices from 2^44 on, cached per
 * graph set) unless opts.block_size is set.  Per-graph `seconds` are the
 * launch time apportioned by sample count.  Same samples (indices 0..n-1) and
 * the same result as ae_integrate up to summation order.  A graph given 0
 * samples contributes value 0 and sigma 0. */
int ae_integrate_batched(ae_ctx *ctx, const int *graph_ids, int n_ids,
                         const uint64_t *n_samples, uint64_t seed, double *value,
                         double *sigma, ae_graph_result *per_graph);

/* Integration of one graph that allocates nothing.
 *
 * For callers that cannot allocate device memory once they are running:
 * for example a host process whose device memory is entirely reserved up
 * front by another framework's caching allocator, or a service loop that
 * must not call cudaMalloc/cudaFree after start-up because those calls
 * synchronise the device and have unbounded latency.  The paper has no
 * counterpart; this is a property of the library, not of the method.
 *
 * Same computation as ae_integrate for a single graph (FP64 integrand,
 * double-double re-evaluation of the samples that fail the acceptance test
 * of ae_opts.dd_tol, fixed-order
 * reduction), but every intermediate lives in one fixed device array of
 * about 8.3 MB that the library declares statically; each GPU that loads the
 * library holds that array until the process exits.  The caller passes the
 * inputs (graph id, sample count, seed) and receives the result in *out
 * (host memory); value, sigma, mean, sigma1, mean_abs, sum_y, sum_y2, max_y2,
 * n, n_dd and n_nonfinite are filled, seconds and the byte counters are 0.
 *
 * Limits and behaviour:
 *  - n_samples must be 1..524288 (every sample may need the double-double
 *    pass, and the array holds one slot per sample); larger values return
 *    AE_ERR_ARG without launching anything;
 *  - the first call on a device looks up the array's device address (with
 *    that device current); make that first call before any stream capture;
 *  - every call on a device uses the same array and it keeps the previous
 *    call's contents; the call clears what must start at zero.  Calls whose
 *    work overlaps on the GPU (two host threads, or two streams) race on the
 *    array and give wrong results: serialise them.
 * The result equals ae_integrate's for the same (graph, n_samples, seed) up
 * to the summation order of the re-evaluated samples. */
int ae_integrate_noalloc(ae_ctx *ctx, int graph_id, uint64_t n_samples, uint64_t seed,
                         ae_graph_result *out);

/* Learned proposal (an extension the paper does not have; unbiased by
 * construction).  A three-hidden-layer MLP (width 64, BF16 weights, FP32
 * accumulation) maps the sampler state (the set of lines not yet ordered) to
 * corrections of the walk's choice logits and of the exponent of the next
 * ratio t; it is tabulated over all 2^M states.  Training: n_train plain
 * samples (indices from 2^40 on, disjoint from integration samples),
 * w = |I|/g, loss -sum w ln q_theta / sum w, `steps` full-batch Adam steps with
 * learning rate lr, all on the device.  Afterwards the graph integrates with
 * the defensive mixture (1-beta) q_theta + beta g (beta in (0,1]).
 * Reallocates the graph's proposal buffers (not for the no-allocation path). */
typedef struct ae_train_report {
  double loss_initial, loss_final;   /* -sum w ln q_theta / sum w (nats), first/last step */
  int steps;
  uint64_t n_train;
  double seconds;                    /* wall time of data generation and training */
} ae_train_report;
int ae_train_proposal(ae_ctx *ctx, int graph_id, uint64_t n_train, uint64_t seed, int steps,
                      double lr, double beta, ae_train_report *report);

/* Refine a graph's trained proposal (library extension, like the proposal
 * itself): the current weights go on training for `steps` Adam steps on
 * n_train samples drawn from the current mixture (indices from 2^41 on),
 * weighted w = |I|/q with q the mixture's density, so that the training data
 * concentrate where |I| is large; the loss and its estimate of the forward
 * Kullback-Leibler divergence to |I| stay the same.  beta is kept.
 * AE_ERR_STATE if the graph has no active trained proposal. */
int ae_refine_proposal(ae_ctx *ctx, int graph_id, uint64_t n_train, uint64_t seed, int steps, double lr,
                       ae_train_report *report);

/* Select a graph's density: mode 0 = plain g, 1 = learned mixture with weight
 * beta on g (needs a trained proposal). */
int ae_set_proposal(ae_ctx *ctx, int graph_id, int mode, double beta);

/* Absolute floor on |y| in the acceptance of a graph's values (see
 * ae_opts.dd_tol): a value is kept when its bound is at most
 * dd_tol * max(|y|, yfloor).  0 (the default) makes the test relative to
 * each sample.  The paper fixes its tolerance from an initialisation pass
 * (Sec. IV.A, Eq. eq_interval_accept: a quarter of the graph's expected
 * sigma); the library leaves the scale to the caller, e.g. the mean |y| of
 * a pilot, which keeps the summed rounding error of N samples below
 * 2 dd_tol N mean|y|.  yfloor finite and >= 0. */
int ae_set_accept_floor(ae_ctx *ctx, int graph_id, double yfloor);

/* The paper's acceptance of a value (Sec. IV.A, Eq. eq_interval_accept): a
 * value of graph j is kept when the width of its certified interval on y,
 * 2 * (rounding-error bound of I carried to y), is at most
 *     width_j = (1/4) sigma_down_j sqrt(sum_l sigma_down_l^2) / sum_l sigma_down_l,
 * sigma_down from an initialisation pass over the graph set, so that the
 * summed round-off error of the set stays below a quarter of its sigma_down.
 * Values that fail are re-evaluated in double-double under the same width;
 * those failing again count as zero.  ae_accept_widths computes width_j from
 * n sigma_down values (host, no context; sigma_down_l <= 0 or not finite
 * contribute nothing and get width 0); ae_set_accept_width sets one graph's
 * width (width > 0: this test replaces the relative test of ae_opts.dd_tol
 * for the graph; 0: back to the relative test).  Widths and sigma_down are
 * those of each graph's contribution, multiplicity included (ae_graph_result
 * .sigma); the library tests y against width / mult. */
int ae_accept_widths(const double *sigma_down, int n, double *width);   /* AE_ERR_ARG: NULL or n <= 0 */
int ae_set_accept_width(ae_ctx *ctx, int graph_id, double width);   /* AE_ERR_ARG: unknown graph,
                                                                       width < 0 or not finite */

/* Cost-aware training weights of the learned proposal (library design; the
 * paper has no learned part): with ratio R > 0, a training sample that the
 * acceptance test would send to double-double has its weight |y| divided by
 * sqrt(1 + R), R being the cost of a re-evaluation in units of an FP64
 * evaluation.  The proposal then approaches |f| / sqrt(cost), the density
 * that minimises variance x expected cost, instead of |f|.  0 (default): the
 * plain weights |y|.  Applies to later ae_train_proposal calls; uses each
 * graph's acceptance floor as set at that time. */
int ae_set_train_cost_ratio(ae_ctx *ctx, double ratio);

/* Test entry: loss and gradient of the proposal for given parameters
 * (ae_proposal_nparams() floats: W1[64][32], b1, W2[64][64], b2, W3[64][64],
 * b3, W4[16][64], b4) and given samples (order: n*16 bytes, descending lines;
 * lt: n*16 floats, ln t at levels 1..M-1; w: n weights), with the plain
 * tables deg and wplain = Phi/Deg (2^M each).  Outputs: loss, grad
 * (nparams), optionally log2 P(j|T) (2^M*16) and Deg_theta (2^M). */
int ae_proposal_eval(ae_ctx *ctx, int M, const float *params, const double *deg,
                     const double *wplain, const uint8_t *order, const float *lt,
                     const double *w, uint64_t n, double *loss, float *grad,
                     double *log2p_out, double *degt_out);
int ae_proposal_nparams(void);

/* The trained proposal of a graph, for checking it outside the library:
 * params (ae_proposal_nparams() floats, nullable) = the FP32 master weights
 * (layout as in ae_proposal_eval); outputs (2^M * 16 floats, nullable) = the
 * network outputs o(T) for every state T from which the sampling tables were
 * built (BF16 weights and activations, FP32 accumulation); *beta (nullable)
 * = the weight of the plain density in the mixture.  AE_ERR_STATE if the
 * graph has no trained proposal. */
int ae_proposal_export(ae_ctx *ctx, int graph_id, float *params, float *outputs, double *beta);

/* Inter-graph allocation (Sec. IV.C).  A pilot of n_pilot samples per graph
 * (independent stream) estimates sigma_j; n_total samples are split into
 * n_out[i]: mode 0 proportional to C_j / sqrt(t_j), C_j = sigma_j sqrt(N_pilot)
 * and t_j the per-sample cost (the paper's optimal probabilities), mode 1
 * proportional to sigma_j^2.  sigma_out (nullable) receives the pilot sigmas. */
int ae_allocate(ae_ctx *ctx, const int *graph_ids, int n_ids, uint64_t n_pilot, uint64_t n_total,
                uint64_t seed, int mode, uint64_t *n_out, double *sigma_out);

/* The paper's sampling probabilities of its integration controller
 * (Sec. IV.C, "Monte Carlo integration: details"): with C_j = sigma_j sqrt(N_j)
 * and t_j the time of one integrand evaluation, the total sigma^2 * time is
 * smallest for p_j = (C_j / sqrt(t_j)) / sum_l (C_l / sqrt(t_l)).  p_floor in
 * [0, 1] raises every p_j below p_floor / n to that value, then renormalises
 * (the paper gives extra
 * attention to graphs with a large sigma_up/sigma_down, a quantity this
 * library does not estimate, so a floor is its stabilisation).  Graphs with
 * no finite positive weight get the floor only; if no graph has one, p is
 * uniform.  Pure host function: sigma, N, t, p are n-element host arrays. */
int ae_schedule_probabilities(const double *sigma, const uint64_t *N, const double *t, int n,
                              double p_floor, double *p);

/* The paper's integration controller: rounds of blocks_per_round blocks of
 * block_size samples; the graph of every block is drawn at random (a host
 * Philox stream of `seed`) with ae_schedule_probabilities(p_floor) from the
 * samples processed so far; round 0 gives each graph one block.  One batched
 * launch per round; each graph continues its own Philox counter, so its
 * samples are exactly those of ae_integrate over [0, N_j).  per_graph (n_ids
 * entries, nullable) holds the accumulated per-graph results (n = N_j). */
int ae_integrate_adaptive(ae_ctx *ctx, const int *graph_ids, int n_ids, uint64_t block_size,
                          int n_rounds, int blocks_per_round, double p_floor, uint64_t seed,
                          double *value, double *sigma, ae_graph_result *per_graph);

/* ------------------------------------------------------------ run state
 * A run (Sec. IV.C: integration in blocks over a long campaign) keeps, per
 * loaded graph, the next sample index of the graph's stream and the running
 * sums below, so that a run can be continued, checkpointed, resumed and
 * merged across ranks.  Because the generator is counter-based, a resumed
 * run draws exactly the samples of an uninterrupted one. */
typedef struct ae_run_graph {
  uint64_t next;             /* next sample index of the graph's stream        */
  uint64_t n, n_dd, n_zero;  /* samples, re-evaluated, zeroed (failed twice)    */
  double sum_y[2];           /* sum of y, double-double (hi, lo)               */
  double sum_y2[2];          /* sum of y^2                                     */
  double sum_abs[2];         /* sum of |y|                                     */
  double max_y2;             /* largest single y^2                             */
} ae_run_graph;

/* Start a run over all loaded graphs with the given seed: zero sums, next
 * sample index 0 for every graph.  Loading graphs clears the run.
 * AE_ERR_STATE if no graphs are loaded. */
int ae_run_reset(ae_ctx *ctx, uint64_t seed);

/* One block of the run: graph_ids[i] gets samples next .. next+n_samples[i]-1
 * of its stream, all graphs in one batched launch (ae_integrate_batched's
 * kernels, captured in a CUDA graph that later steps of the same shape
 * launch again); the sums are added to the run and next advances.  per
 * (nullable, n_ids entries) receives this block's own per-graph results
 * (device seconds, launches, bytes copied included).  Errors (the run is
 * then unchanged): AE_ERR_ARG for an unknown graph, a graph listed twice, no
 * samples at all or a sample index past 2^64; AE_ERR_NODEV on a host-only
 * context; AE_ERR_STATE with no graphs loaded; AE_ERR_CUDA / AE_ERR_TIMEOUT
 * from the launch. */
int ae_run_step(ae_ctx *ctx, const int *graph_ids, int n_ids, const uint64_t *n_samples,
                ae_graph_result *per);

/* Add an integration result of `count` samples of one graph (e.g. from
 * ae_integrate_range at the graph's next index) to the run; next advances by
 * count.  Host only.  AE_ERR_ARG for an unknown graph or an index past 2^64,
 * AE_ERR_NONFINITE if r's sums are not finite. */
int ae_run_add(ae_ctx *ctx, int graph_id, const ae_graph_result *r, uint64_t count);

/* Copy the run state of all loaded graphs into out (caller-owned, n = the
 * number of loaded graphs, else AE_ERR_ARG), and the seed (nullable). */
int ae_run_get(ae_ctx *ctx, ae_run_graph *out, int n, uint64_t *seed);

/* Add another run's sums (e.g. another rank's, on its own stream) to this
 * run, graph by graph in order, double-double; this run's next indices stay.
 * n = number of loaded graphs, else AE_ERR_ARG. */
int ae_run_merge(ae_ctx *ctx, const ae_run_graph *other, int n);

/* The run's estimate: value = sum_j mult_j mean_j, sigma^2 = sum_j (mult_j
 * sigma_down_j)^2 (Eqs. eq_integral_approx, eq_sigma_down, eq_sigma_sum),
 * sigma_up likewise with the heuristic sigma_up_j (nullable outputs).  per
 * (nullable) receives one result per loaded graph (graphs with no samples:
 * value 0, sigma 0).  AE_ERR_STATE if no graphs are loaded. */
int ae_run_estimate(ae_ctx *ctx, double *value, double *sigma, double *sigma_up, ae_graph_result *per);

/* Write the run (graph set identity: loop order, canonical ids, generator;
 * seed; per-graph state) to `path` as a binary file closed by a CRC-64
 * checksum; written to path + ".tmp" and renamed, so a crash leaves the old
 * file.  ae_resume reads it back into a context holding the same graph set:
 * AE_ERR_STATE (nothing changed) if the file is truncated, corrupt (checksum),
 * of another format or of another graph set or generator. */
int ae_checkpoint(ae_ctx *ctx, const char *path);
int ae_resume(ae_ctx *ctx, const char *path);

/* Two independent calculations (e.g. Calc 1 and Calc 2) combined as in
 * Sec. V: per graph by inverse-variance weighting (v = sum w v / sum w,
 * w = 1/sigma^2, sigma = (sum w)^-1/2), then summed with Eq. eq_sigma_sum.
 * v1, s1, v2, s2: per-graph values (multiplicity included) and sigmas;
 * v_out, s_out (nullable): combined per graph; total, total_sigma
 * (nullable): the sum.  A graph with one sigma 0 takes that exact value. */
int ae_combine_runs(const double *v1, const double *s1, const double *v2, const double *s2, int n,
                    double *v_out, double *s_out, double *total, double *total_sigma);

/* Per-sample dump for parity tests: samples first .. first+count-1 of
 * graph_id under `seed`, evaluated in FP64 by the same staged tape
 * interpreter as the integration kernels (each CTA takes a contiguous chunk
 * in rounds of one sample per thread; ae_opts.grid_ctas caps the grid, so a
 * small cap makes many rounds per CTA).  z: count*M, log2g, I, K, y, E:
 * count each (any may be NULL); E is the certified bound on |I - exact I|
 * (rounding only: gamma_D times the magnitude evaluation of I).  Host
 * buffers.  AE_ERR_TIMEOUT if a tape-staging wait ran out (outputs then
 * undefined); AE_ERR_CUDA on a CUDA error. */
int ae_eval_samples(ae_ctx *ctx, int graph_id, uint64_t first, uint64_t count,
                    uint64_t seed, double *z, double *log2g, double *I, double *K,
                    double *y, double *E);

/* Same samples, every one evaluated by the double-double (about 106-bit)
 * twin of the integrand tape, through the staged interpreter of the
 * re-evaluation pass.  I, K, y, E: count each (any may be NULL); E is the
 * bound at the double-double unit.  Errors as ae_eval_samples. */
int ae_eval_samples_dd(ae_ctx *ctx, int graph_id, uint64_t first, uint64_t count,
                       uint64_t seed, double *I, double *K, double *y, double *E);

/* Philox4x32-10 on the device: count (counter[4], key[2]) -> word[4]. */
int ae_philox(ae_ctx *ctx, const uint32_t *ctr, const uint32_t *key, uint32_t *out,
              size_t count);

/* Measured FP64 throughput of this device (TFLOP/s, FMA = 2 flops): eight
 * independent DFMA chains per thread on every SM, best of five launches.
 * The roofline denominator of the integrand kernel. */
int ae_fp64_peak(ae_ctx *ctx, double *tflops);

/* Host copies of a graph's sampling tables: deg and phi are 3 * 2^M doubles
 * each (densities g1, g3, g4). */
int ae_density_tables(ae_ctx *ctx, int graph_id, double *deg, double *phi);

/* Structure export for tests: the UV-divergent subgraphs as (lo, hi, kind)
 * with kind 0 = self-energy, 1 = vertexlike, 2 = vertexlike in J[G]; and
 * the R^new terms as a flat list: sign, count, then count * (lo, hi, op) with
 * op 0 = A, 1 = U, 2 = L, 3 = L-U.  *len receives the number of ints. */
int ae_subgraphs(ae_ctx *ctx, int graph_id, int *buf, int cap, int *len);
int ae_terms(ae_ctx *ctx, int graph_id, int *buf, int cap, int *len);

/* Test hook (host, no device): replay a graph's tape at count points z
 * (count*M doubles): I, K and (E non-NULL) the rounding-error bound of I.
 * Used only by the test suite to check the compiler against the oracle on
 * machines without a GPU; no integration call uses it. */
int aetest_tape_replay(ae_ctx *ctx, int graph_id, const double *z, size_t count,
                       double *I, double *K, double *E);

/* Test hook (device): runs the FP64 integration kernel on one graph with
 * the tape copy for the first segment left out and the bounded wait for it
 * shortened to about `wait_cycles` clock cycles, so that the wait runs out
 * (nothing is in flight).  Returns what the integration entry points return
 * in that case: AE_ERR_TIMEOUT, with the context still usable. */
int aetest_stage_timeout(ae_ctx *ctx, int graph_id, long long wait_cycles);

/* Test hook (device): the learned sampler's fused-multiply-add exp2 and log2
 * next to the device library's exp2 and log2, on n arguments x (exp2) and y
 * (log2, positive).  out: n*4 doubles (fexp2 x, exp2 x, flog2 y, log2 y). */
int aetest_fast_elem(ae_ctx *ctx, const double *x, const double *y, size_t n, double *out);

#ifdef __cplusplus
}
#endif
#endif /* AE_H */
