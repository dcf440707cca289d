/*
 * afc.h -- C ABI of the GB300 (sm_103a) absorbing-frequency-centrality engine.
 *
 * The engine estimates, by Monte Carlo over sampled network realizations, the absorbing
 * Markov chain whose states are the reported local betweenness centres of a stochastic
 * network, and from it the absorbing-frequency centrality (AFC) and its sensitivity to
 * row-wise perturbations of the estimated kernel ("Betweenness-Central Nodes Under
 * Uncertainty: An Absorbing Markov Chain Approach", Bao, Kontou, Vogiatzis).
 *
 * Conventions for every entry point:
 *   - Return value: AFC_OK (0) or one of the AFC_E* codes below; afc_last_error() gives a
 *     thread-local message for the last failure on the calling thread.  No C++ exception
 *     crosses this boundary.
 *   - "device" pointers are CUDA global-memory addresses on the current device; "host"
 *     pointers are ordinary CPU memory.  The caller owns every buffer it passes in; the
 *     library keeps no pointer after the call returns.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Device entry points only
 *     enqueue work on it unless their comment says they synchronise it.
 *   - Node ids are 0..n-1; undirected edge e joins eu[e] and ev[e]; the absorbing state is
 *     column n of the transition-count matrix.
 */
#ifndef AFC_H_
#define AFC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AFC_OK 0
#define AFC_EINVAL 1       /* invalid argument (sizes, ranges, malformed graph)           */
#define AFC_ENOMEM 2       /* a device or host allocation failed, or workspace too small   */
#define AFC_EOVERFLOW 3    /* a shortest-path count exceeded 2^64 - 1 in some realization  */
#define AFC_ESINGULAR 4    /* I - Q was numerically singular                               */
#define AFC_ETIMEOUT 5     /* a bounded wait for device work expired (afc_server_poll)     */
#define AFC_ECUDA 6        /* a CUDA runtime call failed                                   */
#define AFC_EUNSUPPORTED 7 /* the problem exceeds an implementation limit                  */
#define AFC_EDEVICE 8      /* a device-side consistency check failed (see message)        */
#define AFC_EBUSY 9        /* serving: refused for now (over budget, queue full) or pending */
#define AFC_ECANCELED 10   /* serving: the query was cancelled (afc_server_cancel)           */

#define AFC_FP64 0          /* dependencies delta accumulated in FP64                        */
#define AFC_FP32_RECHECK 1  /* delta in FP32, realizations with a near-tied top two in FP64 */

#define AFC_PATH_AUTO 0     /* counting path chosen by what fits in shared memory            */
                            /* (a CTA must hold at least six source slots)                   */
#define AFC_PATH_SHARED 1   /* realization and source state in shared memory (small graphs)  */
#define AFC_PATH_GLOBAL 2   /* realized graph and source state in device memory (any size)   */

const char *afc_last_error(void);
int afc_version(void);

/* ------------------------------------------------------------------------------------ */
/* Host helpers                                                                          */
/* ------------------------------------------------------------------------------------ */

/* Base topology G(V, E) (Sec. 3.1) as a symmetric CSR.  Host in: eu, ev [m] (int32), each
 * edge once, no self loops, no duplicates, 0 <= eu, ev < n.  Host out (caller-allocated):
 * row_ptr [n+1], col [2m], eid [2m] (undirected edge id of each arc), rows sorted by col.
 * Returns AFC_EINVAL on a malformed edge list (nothing is written in that case except
 * possibly partial row_ptr). */
int afc_csr_from_edges(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev,
                       int32_t *row_ptr, int32_t *col, int32_t *eid);

/* Survival threshold T = floor(p * 2^32) of an edge that survives with probability p
 * (T = 2^32 for p >= 1, 0 for p <= 0); a realization keeps the edge iff its 32-bit draw
 * u0 < T (Sec. 3.1 network state; independent edge availability as in Sec. 9.1). */
uint64_t afc_survival_threshold(double p);

/* ------------------------------------------------------------------------------------ */
/* A1-A7: Monte Carlo transition counts (Alg. 1 SampleNext, Alg. 2 row-wise construction) */
/* ------------------------------------------------------------------------------------ */

/* One stochastic base graph and its one-step simulator.  All pointers are DEVICE pointers
 * except where noted.  Realization r of graph `graph_tag` draws, for each undirected edge e,
 * (u0, u1) = Philox4x32-10(counter = (e, r, graph_tag, 0), key = seed): the edge survives
 * iff u0 < thresh[e] and has integer length w = w_lo[e] + floor(u1 (w_hi[e]-w_lo[e]+1) / 2^32).
 * From realization r every anchor i moves to the tie-broken betweenness centre of its
 * component K(i; H_r) (Sec. 3.2 eq. local-center) or to the absorbing state when
 * |K(i; H_r)| < k_min or K(i; H_r) holds no admissible candidate (Sec. 7.1 Sel_W). */
typedef struct {
  int32_t n;                 /* nodes, 1 <= n <= 65535                                   */
  int64_t m;                 /* undirected edges                                          */
  const int32_t *row_ptr;    /* [n+1] device symmetric CSR (afc_csr_from_edges layout)   */
  const int32_t *col;        /* [2m]  device                                              */
  const int32_t *eid;        /* [2m]  device                                              */
  uint64_t seed;             /* Philox key (low word, high word)                          */
  uint32_t graph_tag;        /* third Philox counter word                                 */
  const uint64_t *thresh;    /* [m] device survival thresholds, or NULL -> thresh_all     */
  uint64_t thresh_all;
  const uint32_t *w_lo;      /* [m] device, or NULL -> w_lo_all (lengths >= 1)            */
  const uint32_t *w_hi;      /* [m] device, or NULL -> w_hi_all (w_hi >= w_lo, <= 65535)  */
  uint32_t w_lo_all, w_hi_all;
  uint32_t k_min;            /* component-size threshold (Sec. 3.2), >= 1                 */
  const uint8_t *in_w;       /* [n] device candidate-pool mask W, or NULL = all nodes     */
  uint32_t top_k;            /* 0: centre = tie-broken argmax over K cap W; k > 0: that    */
                             /* centre must also rank within the first k of K (Sec. 7.1)  */
  double tie_rel;            /* relative tie band: v ties the maximum B* iff              */
                             /* B_v >= B* - tie_rel * B*; ties go to the smallest id       */
  int32_t precision;         /* AFC_FP64 or AFC_FP32_RECHECK                              */
  double recheck_margin;     /* FP32 mode: recompute a realization in FP64 when some valid */
                             /* component's top-two gap (B1 - B2) / B1 < recheck_margin    */
  uint32_t bucket_width;     /* SSSP bucket width Delta, rounded up per realization to a    */
                             /* power of two >= ceil(max length / 14); 0 = automatic       */
  int32_t block_threads;     /* threads per CTA of the counting kernel: 256, 512 or 1024;  */
                             /* 0 = automatic                                              */
  int32_t team_threads;      /* threads of one team (32 .. block_threads, a power of two); */
                             /* each team advances its own batch of sources; 0 = auto      */
  int32_t slots_per_team;    /* sources a team advances in lockstep (1..16); 0 = as many   */
                             /* as shared memory holds                                     */
  int32_t memory_path;       /* AFC_PATH_AUTO: realizations of graphs whose CTA holds the  */
                             /* realization and at least six source slots in shared memory */
                             /* run there, others on the global-memory path;               */
                             /* AFC_PATH_SHARED / AFC_PATH_GLOBAL force one                 */
                             /* (AFC_EUNSUPPORTED if the shared path does not fit)          */
  /* Simulator-level rewards (Sec. 6) and rank-r reports.  The ordering pi of a valid        */
  /* component K repeats the centre rule on the nodes of K not yet listed (B* over the rest, */
  /* the tie_rel band, smallest id), so pi(1) is the centre (Sec. 2.3 eq. topk-comp).        */
  uint32_t reward_k;         /* 0: off.  k > 0: every anchor of a valid component adds the  */
                             /* valued Top-k step reward sum_{t <= min(k,|K|)} gamma[pi(t)]  */
                             /* over pi(t) in reward_pool (Sec. 6.2-6.3) to psi_sum[anchor]  */
  const double *reward_gamma;  /* [n] DEVICE node values gamma >= 0, or NULL = 1           */
  const uint8_t *reward_pool;  /* [n] DEVICE pool mask W, or NULL = every node             */
  double *psi_sum;           /* [n] DEVICE accumulator (not cleared); required with reward_k */
  uint32_t report_rank;      /* 0 or 1: report the centre; r > 1: report pi(r), the rank-r   */
                             /* centre (bottom if |K| < r).  reward_k > 0 or report_rank > 1 */
                             /* needs AFC_FP64, in_w NULL, top_k 0 and at most 256 ranks      */
  /* Fallback selector Sel_{W,fb} (Sec. 7.3).  With use_fallback 0 a valid component whose     */
  /* candidate set (in_w, top_k) admits no centre absorbs: the hard-filtered kernel P^W of     */
  /* Sec. 7.1.  With 1 it reports fallback_node instead; invalid components still absorb.      */
  int32_t use_fallback;
  int32_t fallback_node;     /* v_fb in [0, n) (inside or outside W)                          */
  uint32_t *fallback_count;  /* [n] DEVICE u32, accumulated (not cleared), or NULL: draws of  */
                             /* anchor i redirected to v_fb (afc_feasibility needs them)       */
  int32_t tie_random;        /* 0: ties of the centre rule go to the smallest id.  1: drawn   */
                             /* uniformly (Remark on randomized tie-breaking, Sec. 4.1): the   */
                             /* floor(u t / 2^32)-th of the t tied candidates by id, u =       */
                             /* Philox4x32-10(counter (root, r, graph_tag, 3), key = seed)[0], */
                             /* root = the smallest id of the component.  Not with reward_k or */
                             /* report_rank > 1                                                */
  /* Discrete length law (Sec. 9 weighted-network experiment).  With wtab_ptr non-NULL edge e's */
  /* length is lo_e + #{k : wtab[wtab_ptr[e] + k] <= u1}, capped at hi_e, u1 the same Philox     */
  /* word that the uniform law uses (thresholds non-decreasing per edge; afc_weight_table_normal */
  /* builds them for the rounded and clipped normal law).  DEVICE [m+1] and thresholds.        */
  const uint32_t *wtab_ptr;
  const uint32_t *wtab;
  /* Row-wise mode (Alg. 2 taken literally: every row i gets its own independent draws, no      */
  /* realization shared between rows).  per_row 1: a call over realizations [r_begin, r_begin   */
  /* + r_count) makes r_count draws for every row, draw m of row i on realization m n + i      */
  /* ((r_begin + r_count) n < 2^32); only row i is counted, from the betweenness of i's         */
  /* component (r_count x n items: n times the work of the shared mode; stats count items).     */
  /* hop_radius r > 0 (row-wise mode only): the working graph is the realization induced on    */
  /* S_r(i), the nodes within r hops of i in the base graph, and K is i's component there      */
  /* (Sec. 9 weighted-network experiment).  No dump_bc / dump_next, rewards or rank-r reports. */
  int32_t per_row;
  uint32_t hop_radius;
} afc_mc_problem;

/* Device-side counters of one or more afc_transition_counts calls (caller zeroes them). */
typedef struct {
  uint64_t realizations;     /* realizations processed                                    */
  uint64_t sources;          /* single-source shortest-path problems solved               */
  uint64_t edge_visits;      /* sum over solved sources of the alive edges of the source's */
                             /* component (Graph500 TEPS numerator, edges once)            */
  uint64_t overflow;         /* realizations with a path count above 2^64 - 1              */
  uint64_t rechecked;        /* FP32 mode: realizations recomputed in FP64                */
  uint64_t device_error;     /* bit mask of device consistency failures (0 = none)         */
  uint64_t vertex_visits;    /* sum over solved sources of the size of the source's component */
  uint64_t wide_redone;      /* shared-memory path: realizations redone with 64-bit path-count */
                             /* slots because a count exceeded 2^32 - 1 (results unchanged)   */
} afc_mc_stats;

/* AFC_PATH_SHARED or AFC_PATH_GLOBAL: where afc_transition_counts runs this problem (the
 * problem's memory_path, or for AFC_PATH_AUTO the rule given at memory_path); a negative error
 * code for an invalid problem. */
int afc_counts_path(const afc_mc_problem *prob);

/* Bytes of device workspace afc_transition_counts needs for this problem, for any realization
 * count (0 for an invalid problem): on the shared-memory path one region per CTA (components,
 * source list, selection scratch, betweenness accumulators), on the global path the
 * realizations in flight and the source-slot arena. */
size_t afc_transition_counts_workspace(const afc_mc_problem *prob);

/* Adds the outcomes of realizations r_begin .. r_begin + r_count - 1 to counts, a DEVICE
 * uint32 matrix [n][n+1] in row-major order (column n = absorption).  counts is accumulated,
 * not cleared, so disjoint realization ranges (shards, resumed runs) sum bit-exactly.
 * stats: DEVICE afc_mc_stats (accumulated), or NULL.  dump_bc: DEVICE double [r_count][n]
 * receiving each realization's betweenness B_v(H_r) over ordered pairs for nodes of valid
 * components (0 elsewhere), or NULL; dump_next: DEVICE int32 [r_count][n] receiving each
 * anchor's next state (n = absorbed), or NULL.  workspace: DEVICE, at least
 * afc_transition_counts_workspace(prob) bytes (may be NULL when that is 0).
 * Asynchronous on `stream`; argument errors are returned before anything is enqueued. */
int afc_transition_counts(const afc_mc_problem *prob, uint32_t r_begin, uint32_t r_count,
                          uint32_t *counts, afc_mc_stats *stats, double *dump_bc,
                          int32_t *dump_next, void *workspace, size_t workspace_bytes,
                          void *stream);

/* Autotuner of the counting launch (an engineering layer; the paper has no counterpart).  Times
 * a small grid of launch configurations on `sample` realizations of the problem (r_begin .. r_begin
 * + sample - 1) and writes the fastest into prob->block_threads, team_threads, bucket_width and,
 * when prob->memory_path is AFC_PATH_AUTO, memory_path.  Grid: bucket widths {1/2, 1, 2} x the
 * automatic one; on the shared-memory path the block/team pairs (1024,32), (1024,128),
 * (1024,256), (1024,1024), (512,64), (512,512), (256,256) that fit; on the global path (1024,128),
 * (1024,256), (1024,512) (tried also for AUTO problems that fit in shared memory).  The automatic
 * configuration is timed too, so the winner is never slower on the sample.  The configuration
 * never changes the results, only the speed.  Allocates and frees its own device scratch (stream
 * ordered) and SYNCHRONISES `stream`.  sample 0 = ceil(2000 x SMs / n) realizations, clamped to
 * [2, 2 x SMs].  Errors: those of afc_transition_counts (the problem is left unchanged). */
typedef struct {
  int32_t block_threads, team_threads;
  uint32_t bucket_width;
  double realizations_per_s;  /* of the winner on the sample                                 */
  double default_per_s;       /* of the automatic configuration on the same sample           */
  int32_t candidates;         /* configurations timed                                         */
} afc_tune_result;
int afc_autotune(afc_mc_problem *prob, uint32_t r_begin, uint32_t sample, void *stream,
                 afc_tune_result *out);

/* Threshold tables of the rounded and clipped normal length law of the paper's weighted-network
 * experiment (Sec. 9): x ~ N(mu_e, sigma_e^2) with mu_e = w0_e + rho_mu (wmax - w0_e), sigma_e =
 * rho_sigma (wmax - w0_e), length round(x) clipped to [w0_e, wmax].  Edge e gets wmax - w0_e
 * thresholds t_k = min(floor(2^32 F(w0_e + k)), 2^32 - 1), F(x) = Phi((x + 1/2 - mu_e) /
 * sigma_e), indexed by ptr[e] .. ptr[e+1]-1 (a law quantised to 2^-32).  HOST in: w0 [m] (each
 * in [1, wmax]); HOST out: ptr [m+1], tab [capacity]; *used = thresholds written.  Use with
 * afc_mc_problem.w_lo = w0 and w_hi_all = wmax.  Errors: AFC_EINVAL for bad arguments,
 * AFC_EUNSUPPORTED when sum_e (wmax - w0_e) >= 2^32 (32-bit offsets), AFC_ENOMEM when
 * capacity < sum_e (wmax - w0_e). */
int afc_weight_table_normal(int64_t m, const uint32_t *w0, uint32_t wmax, double rho_mu,
                            double rho_sigma, uint32_t *ptr, uint32_t *tab, size_t capacity,
                            size_t *used);

/* Measured FMA throughput of the current GPU (a diagnostic; the paper has no counterpart):
 * *tflops = 2 x FMAs per second / 1e12 of a register-resident FMA loop over 4 CTAs of 256
 * threads per SM, in FP64 (fp64 != 0) or FP32.  The FP64 figure is the denominator of the
 * FP64-bound kernels' rooflines (GB300's FP64 rate is a small fraction of its FP32 rate).
 * Allocates 8 bytes (stream ordered) and SYNCHRONISES `stream`. */
int afc_measure_fma_rate(int32_t fp64, double *tflops, void *stream);

/* Several base graphs in one persistent launch (the batched mix).  probs: HOST array of
 * nprob problems; r_count: HOST [nprob]; counts: HOST array of nprob DEVICE count matrices;
 * stats: DEVICE afc_mc_stats [nprob] or NULL.  workspace: DEVICE, at least
 * afc_transition_counts_batched_workspace(...) bytes.  Realization r of problem g is exactly
 * the realization r of afc_transition_counts on that problem alone. */
size_t afc_transition_counts_batched_workspace(int32_t nprob, const afc_mc_problem *probs,
                                               const uint32_t *r_count);
int afc_transition_counts_batched(int32_t nprob, const afc_mc_problem *probs,
                                  const uint32_t *r_count, uint32_t *const *counts,
                                  afc_mc_stats *stats, void *workspace, size_t workspace_bytes,
                                  void *stream);

/* Parity hooks for single steps of the same kernels (DEVICE outputs):
 *   afc_debug_realize: alive [r_count][m] (uint8), w [r_count][m] (uint32) for A1.
 *   afc_debug_components: comp [r_count][n] (smallest id of the component), csize.
 *   afc_debug_sssp: realization r, sources[nsrc] (DEVICE int32): dist [nsrc][n] (uint32,
 *     0xFFFFFFFF = unreachable) and sigma [nsrc][n] (uint64) from the production SSSP and
 *     path-counting code, run on every source's whole component. */
int afc_debug_realize(const afc_mc_problem *prob, uint32_t r_begin, uint32_t r_count,
                      uint8_t *alive, uint32_t *w, void *stream);
int afc_debug_components(const afc_mc_problem *prob, uint32_t r_begin, uint32_t r_count,
                         int32_t *comp, int32_t *csize, void *stream);
int afc_debug_sssp(const afc_mc_problem *prob, uint32_t r, const int32_t *sources, int32_t nsrc,
                   uint32_t *dist, uint64_t *sigma, afc_mc_stats *stats, void *stream);

/* ------------------------------------------------------------------------------------ */
/* A8: kernel assembly and the absorbing-chain solve (Sec. 4 eqs. fundamental, visits,    */
/* expected-length, afc-def; Sec. 6.4 eq. mr-inner-product; Sec. 8.2 stabilisation)        */
/* ------------------------------------------------------------------------------------ */

/* Q_ij = (1 - alpha) counts_ij / R and r_i = alpha + (1 - alpha) counts_i,n / R; a row with
 * r_i = 0 (possible only for alpha = 0) gets r_i = absorb_floor and its transient part
 * rescaled to 1 - absorb_floor. */
typedef struct {
  int32_t n;
  uint32_t realizations;     /* R: the row sum of every count row                         */
  double alpha;              /* exogenous per-step stop probability (Sec. 4)               */
  double absorb_floor;       /* eta                                                        */
  const double *s_init;      /* [n] DEVICE initial law, or NULL = uniform                  */
  const double *reward;      /* [n] DEVICE node values f, or NULL                          */
} afc_chain;

/* Observed centre states C = {j : counts_ij > 0 for some i} (DEVICE outputs c_index [n]:
 * position of j in C or -1; c_list [n]: the members of C in increasing id).  Writes |C| to
 * *c_host (HOST) and SYNCHRONISES `stream`. */
int afc_observed_states(int32_t n, const uint32_t *counts, int32_t *c_index, int32_t *c_list,
                        int32_t *c_host, void *stream);

/* Device workspace of afc_absorbing_solve / afc_perturb_sweep / afc_certificates. */
size_t afc_solve_workspace(int32_t n, int32_t c);

/* AFC from the counts by the reduced solve on C: with the columns of U = V \ C zero,
 * mu_U = s_U and mu_C (I - Q_CC) = s_C + s_U Q_UC, solved by FP64 LU with partial pivoting.
 * DEVICE outputs: mu [n], b [n] = mu / (mu 1), scalars [4] = {E_s[T], b_f = b.f (0 without a
 * reward), max_i (N 1)_i (largest expected absorption time over start nodes), |C|},
 * lu [c*c] and piv [c]: the LU factors of (I - Q_CC) (kept for afc_perturb_sweep and
 * afc_certificates).  Returns AFC_ESINGULAR (after synchronising) if a pivot vanished. */
int afc_absorbing_solve(const afc_chain *chain, const uint32_t *counts, const int32_t *c_index,
                        const int32_t *c_list, int32_t c, double *mu, double *b, double *scalars,
                        double *lu, int32_t *piv, void *workspace, size_t workspace_bytes,
                        void *stream);

/* Reward-AFC of the simulator-level rewards (Prop. reward-afc-general: s N psi / s N 1 =
 * b . psi for an expected one-step reward psi).  DEVICE out [2]: out[0] = b . psi_topk with
 * psi_topk_i = (1 - alpha) psi_sum[i] / R (the exogenous stop ends a step without reward; 0
 * when psi_sum is NULL); out[1] = b . psi_sw, the switching count of Sec. 6.4 (eta_sw(i, j) = 1
 * for j in V, j != i), psi_sw_i = sum_{j != i} Q_ij with Q assembled as afc_absorbing_solve
 * does.  DEVICE in: counts [n][n+1], b [n] (afc_absorbing_solve), psi_sum [n] or NULL.
 * Asynchronous on `stream`. */
int afc_reward_afc(const afc_chain *chain, const uint32_t *counts, const double *b,
                   const double *psi_sum, double *out, void *stream);

/* Realization-level bootstrap of b (Sec. 8: nonparametric bootstrap intervals by resampling
 * the draws with replacement; every anchor's draws come from the same realizations, so whole
 * realizations are resampled).  Replicate b (0 <= b < B) draws R = chain->realizations indices
 * k = 0 .. R-1 with u = Philox4x32-10(counter (k, b, 0, 2), key = seed)[0], realization
 * floor(u R / 2^32); it re-counts the next-state records with those multiplicities and solves
 * the reduced chain on the nominal observed states exactly as afc_absorbing_solve (states not
 * re-drawn into keep only their initial mass, as they would as unobserved states).
 * DEVICE in: next_states [R][n] int32 (the dump_next records of afc_transition_counts over the
 * same realizations; n = absorption), c_index / c_list / c of afc_observed_states on the
 * nominal counts.  DEVICE out: b_rep [B][n] (or NULL: kept in the workspace), T_rep [B] E_s[T]
 * per replicate (or NULL), b_lo / b_hi [n] (or NULL): per node the replicates at sorted
 * positions floor(q (B-1)) and ceil((1-q) (B-1)), q = (1 - level) / 2 (ties by replicate index).
 * Workspace: afc_bootstrap_workspace bytes (fewer work with fewer resident replicates).
 * SYNCHRONISES `stream`.  Errors: AFC_EINVAL for a record outside absorption and the observed
 * states, AFC_ESINGULAR for a zero pivot. */
size_t afc_bootstrap_workspace(int32_t n, int32_t c, uint32_t R, uint32_t B);
int afc_bootstrap(const afc_chain *chain, const int32_t *next_states, const int32_t *c_index,
                  const int32_t *c_list, int32_t c, uint32_t B, uint64_t seed, double level,
                  double *b_rep, double *T_rep, double *b_lo, double *b_hi, void *workspace,
                  size_t workspace_bytes, void *stream);

/* Row-wise robust inner problem (Sec. 8 post-processing, over the uncertainty set of Sec. 5.1):
 * T[i] = inf over q_i in U_i of sum_j q_ij v_j + (1 - sum_j q_ij) v_bot, with U_i the box
 * [(Q_ij - eps)_+, min(Q_ij + eps, 1)] around the kernel assembled from `counts` (as
 * afc_absorbing_solve assembles it) and sum_j q_ij <= 1 - r_min.  support_only 1: the box on
 * the row's observed support (q_ij = 0 elsewhere); 0: on every j (new transitions up to eps).
 * Solved exactly per row (lower bounds, then the budget to the most negative coefficients
 * v_j - v_bot first, ties by j).  DEVICE in: counts [n][n+1], v [n].  DEVICE out: T [n],
 * Qstar [n][n] a minimising kernel (or NULL).  Workspace: 256 bytes.  SYNCHRONISES `stream`.
 * Errors: AFC_EINVAL when some U_i is empty (its lower bounds exceed 1 - r_min). */
int afc_robust_inner(const afc_chain *chain, const uint32_t *counts, double eps, double r_min,
                     int32_t support_only, const double *v, double v_bot, double *T, double *Qstar,
                     void *workspace, size_t workspace_bytes, void *stream);

/* Robust value and its scenario kernel (Sec. 8: a kernel P* in U chosen by a robust Bellman
 * operator; Remark on the robust optimisation viewpoint in Sec. 5): V = f + T_sense(V) with
 * v_bot = 0, f = chain->reward (NULL = 1: the robust expected length), sense -1 the adversary
 * minimises, +1 maximises.  Policy iteration: the inner problem's optimiser at V, V of that
 * kernel by an FP64 LU of I - Q*, until V changes by at most 1e-13 relative (at most 100
 * rounds).  DEVICE out: V [n], Qstar [n][n] (or NULL), b_star [n] = the AFC of P*, scalars [2]
 * = {E_s[T] under P*, b* . f}; HOST out: *iterations (or NULL).  n <= 4096 (dense solve in one
 * CTA).  Workspace: afc_robust_value_workspace(n).  SYNCHRONISES `stream`.  Errors as
 * afc_robust_inner, AFC_ESINGULAR for a zero pivot. */
size_t afc_robust_value_workspace(int32_t n);
int afc_robust_value(const afc_chain *chain, const uint32_t *counts, double eps, double r_min,
                     int32_t support_only, int32_t sense, double *V, double *Qstar, double *b_star,
                     double *scalars, int32_t *iterations, void *workspace, size_t workspace_bytes,
                     void *stream);

/* Envelopes of AFC coordinates over the row-wise uncertainty set (Remark on the robust
 * optimisation viewpoint in Sec. 5: inf / sup over P in U of b_v(s; P)), with U the set of
 * afc_robust_inner (box of radius eps around the kernel assembled from `counts`, transient row
 * sums at most 1 - r_min, support_only as there).  b_v = (s N)_v / (s N 1) is linear-fractional
 * in the visits, so its extremes are the roots of F(lambda) = opt over U of s N (e_v - lambda 1),
 * a robust value that policy iteration computes exactly on a rectangular set (afc_robust_value
 * with that reward); Dinkelbach's iteration lambda <- b_v(argopt) from lambda = 0 reaches the
 * root (until lambda moves by at most 1e-13 relative, at most 60 steps).  The 2k problems (the
 * supremum and the infimum for each of the k HOST nodes) run as one batch: one CTA each for the
 * dense FP64 LU of I - Q*.  HOST out: b_lo [k], b_hi [k], iterations [2k] (or NULL: Dinkelbach
 * steps of the supremum, then the infimum, per node).  n <= 4096.  Workspace:
 * afc_robust_envelope_workspace(n, k) (2 n^2 + O(n) doubles per problem).  SYNCHRONISES
 * `stream`.  Errors as afc_robust_value; AFC_EDEVICE when Dinkelbach does not settle. */
size_t afc_robust_envelope_workspace(int32_t n, int32_t k);
int afc_robust_envelope(const afc_chain *chain, const uint32_t *counts, double eps, double r_min,
                        int32_t support_only, int32_t k, const int32_t *nodes, double *b_lo,
                        double *b_hi, int32_t *iterations, void *workspace,
                        size_t workspace_bytes, void *stream);

/* Wasserstein-1 distances under the base graph's shortest-path (hop) metric, the second
 * discrepancy of the paper's robust search (Sec. 9): out[k] = W1(x_k, y) for the `count` HOST
 * rows x_k = x + k n (each summing to sum y), over the HOST edge lists eu, ev (as
 * afc_csr_from_edges).  Exact (successive shortest paths on the graph; masses settled to a
 * relative 1e-14).  Host code; the rows run on parallel host threads.  Errors: AFC_EINVAL for
 * bad edges. */
int afc_w1_graph(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, const double *x,
                 const double *y, int32_t count, double *out);

/* The same distances on the device (Sec. 9 robust experiment): out[k] = W1(x_k, y) for the
 * `count` DEVICE rows x_k = x + k n against DEVICE y [n], over the graph's DEVICE symmetric CSR
 * (row_ptr [n+1], col [2m], eid [2m], afc_csr_from_edges layout).  Exact: the min-cost flow of
 * unit edge costs, solved per row by one warp with the primal-dual method (Dijkstra phases on
 * reduced costs, then a blocking flow on the zero-reduced-cost arcs); masses settled to a
 * relative 1e-14 of max_v |x_kv - y_v|; out[k] = sum over edges of |flow| in a fixed order.
 * DEVICE out [count].  Workspace: afc_w1_batch_workspace(n, m, count) bytes (256 when a row's
 * state fits in shared memory).  SYNCHRONISES `stream`.  Errors: AFC_EINVAL for bad arguments
 * or when more than 1e-9 of some row's excess mass reaches no deficit (x_k and y differ in total
 * on a connected component), AFC_EDEVICE when an iteration bound or a flow invariant fails. */
size_t afc_w1_batch_workspace(int32_t n, int64_t m, int32_t count);
int afc_w1_batch(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col,
                 const int32_t *eid, const double *x, const double *y, int32_t count, double *out,
                 void *workspace, size_t workspace_bytes, void *stream);

/* Ranking under the tie band (the ordering the sweep and the centre rule use, Sec. 5.5 and
 * Sec. 2.3): rank[v] = #{u != v : b_u - b_v > tie_rel max b, or |b_u - b_v| <= tie_rel max b and
 * u < v}; the band is not transitive, so equal counts are ordered by node id: topk[p] = the node
 * at position p < k of the order (rank[v], v).  The Top-k of the rank-stability check (Sec. 8:
 * estimates from M and from 2M realizations) compares two such lists.  DEVICE in b [n]; DEVICE
 * out rank [n], topk [k] (may be NULL when k = 0).  O(n^2) work.  Asynchronous on `stream`. */
int afc_rank_order(int32_t n, const double *b, double tie_rel, int32_t k, int32_t *rank,
                   int32_t *topk, void *stream);

/* Reductions of the sampled robust search (Sec. 9; Remark on the robust optimisation viewpoint
 * in Sec. 5): arg[0] / arg[1] = the sample maximising d1 / d2 (DEVICE [count] each, e.g. the KL
 * values of afc_perturb_params.kl_out and the afc_w1_batch distances; NULL gives -1), ties to
 * the smaller index and NaN above every number (numpy's argmax); b_low / b_high [n] = per node
 * the smallest / largest of b0 and the sampled rows b_rows [count][n] (the sampled envelopes,
 * an inner approximation of the inf / sup over the whole uncertainty set).  All DEVICE; any
 * output may be NULL.  Asynchronous on `stream`. */
int afc_robust_summary(int32_t n, int32_t count, const double *b_rows, const double *b0,
                       const double *d1, const double *d2, int32_t *arg, double *b_low,
                       double *b_high, void *stream);

/* Set-constrained kernels (Sec. 7).  Counts of the hard-filtered kernel P^W come from
 * afc_transition_counts with in_w / top_k; of the fallback kernel P^{W,fb} with use_fallback,
 * which also fills fallback_count.  b^W, b^{W,fb} and b^W . f come from afc_absorbing_solve on
 * those counts (Sec. 7.2: the same linear-algebraic pipeline).
 *
 * afc_feasibility: xi[i] = sum_{j in W} P^W_ij (Sec. 7.1 eq. settopk-xi), the probability that
 * a step from anchor i reaches the target pool directly, estimated on the kernel assembled from
 * `counts` as afc_absorbing_solve assembles it: the row's transient mass times the share of its
 * non-absorbed draws that were not redirected to v_fb.  DEVICE in: counts [n][n+1],
 * fallback_count [n] (or NULL: no fallback).  DEVICE out: xi [n].  Asynchronous on `stream`. */
int afc_feasibility(const afc_chain *chain, const uint32_t *counts, const uint32_t *fallback_count,
                    double *xi, void *stream);

/* afc_pool_summaries: mass[0] = m_W = sum_{v in W} b_v (Sec. 7.2 eq. settopk-bPsi; m_W^fb for
 * the fallback kernel's b), mass[1] = c_fb = sum_{u not in V_fb} b_u (Sec. 7.4); b_pool[v] =
 * b_v / m_W on W (the within-pool profile), b_censored[v] = b_v / c_fb off V_fb (fallback visits
 * censored); both 0 elsewhere, and everywhere when their mass is 0.  DEVICE in: b [n], in_w [n]
 * (pool mask W), fallback_set [n] (mask of V_fb, or NULL = empty).  DEVICE out: mass [2], b_pool
 * [n] and b_censored [n] (each may be NULL).  One CTA; asynchronous on `stream`. */
int afc_pool_summaries(int32_t n, const double *b, const uint8_t *in_w, const uint8_t *fallback_set,
                       double *b_pool, double *b_censored, double *mass, void *stream);

/* afc_clique_pool (host): the 3-clique target pool of the paper's structure-constrained
 * experiment (Sec. 9): every triangle of the base graph (HOST edge lists eu, ev of length m, as
 * afc_csr_from_edges), scored by the sum of its nodes' base degrees; the S best kept (score
 * descending, ties by the ascending node triple).  HOST out: in_w [n] = their union,
 * *fallback_node = smallest id of the first kept triangle (-1 if none), triangles [3 S] the kept
 * (u < v < w) triples (or NULL), *kept = how many (or NULL).  Errors: AFC_EINVAL for bad edges. */
int afc_clique_pool(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, int32_t S,
                    uint8_t *in_w, int32_t *fallback_node, int32_t *triangles, int32_t *kept);

/* Allocation-free variant of afc_absorbing_solve (the paper has no counterpart: this exists for
 * callers that cannot allocate device memory themselves, e.g. code embedded in a host framework
 * that hands out all device memory up front, or a plugin that may only use the buffers it is
 * given).  It computes the observed states, assembles and solves the reduced system exactly as
 * afc_absorbing_solve, but its whole workspace is one file-scope device array of about 0.6 MB
 * inside the library; it allocates nothing and calls no allocating routine.
 * In: chain, counts (DEVICE [n][n+1]).  Out (DEVICE): mu [n], b [n], scalars [4] as in
 * afc_absorbing_solve.  Limits: n <= 4096 (else AFC_EUNSUPPORTED before any work) and at most
 * 256 observed states (else AFC_EUNSUPPORTED after the states are counted).  SYNCHRONISES
 * `stream` (it reads the state count and status back before returning).  The first call on a
 * device looks up the array's device address (once per device; make that first call before any
 * stream capture).  The CUDA driver places the array when it loads the library's device code:
 * under lazy module loading (the default) that happens at the first use of that code, so a
 * caller that reserves all device memory up front should make one call (or load modules
 * eagerly, CUDA_MODULE_LOADING=EAGER) before doing so.  Every call on a device shares the array and
 * it keeps the last call's contents; calls whose work overlaps on the GPU (other streams or host
 * threads) race on it, so serialise them. */
int afc_absorbing_solve_noalloc(const afc_chain *chain, const uint32_t *counts, double *mu,
                                double *b, double *scalars, void *stream);

/* ------------------------------------------------------------------------------------ */
/* A9: row-wise perturbation sweep (Sec. 5.1 uncertainty set, Sec. 5.4 first-order        */
/* sensitivity, Sec. 5.5 ranking reversals and certificates)                               */
/* ------------------------------------------------------------------------------------ */

/* Perturbation p (p_begin <= p < p_begin + p_count) moves every row i of the estimated kernel
 * on its support J_i = {j : Q_ij > 0} plus the absorbing column: z_j = 2u - 1 with
 * u = Philox4x32-10(counter = (j, i, p, 1), key = seed)[0] / 2^32 (j = n for absorption),
 * d = z - mean(z), d <- l1_radius d / ||d||_1, q' = max(q + d, 0), q' <- q' / sum(q'), and
 * if q'_abs < r_min the transient part is scaled to 1 - r_min.  The perturbed AFC b' is then
 * ranked (u before v iff b'_u - b'_v > tie_rel max b', or within that band and u < v) and
 * compared with the nominal ranking. */
typedef struct {
  uint32_t p_begin, p_count;
  double l1_radius;          /* 0.05 */
  double r_min;              /* leak lower bound r_min (Sec. 5.1)                          */
  uint64_t seed;
  int32_t top_k;             /* k of the Top-k set / order statistics (5)                  */
  int32_t k2;                /* nominal top-k2 nodes tracked for pair flips / shifts (10)  */
  int32_t hist_bins;         /* bins of the rank-shift histogram (16)                      */
  double tie_rel;
  /* Row model.  0: the l1 model above.  1: the multiplicative model of the paper's robust   */
  /* experiment (Sec. 9): every transient entry with Q_ij > 0 becomes                         */
  /* min(max(Q_ij (1 + rel_radius z_j), 0), 1) (z_j as above, no draw for absorption); a     */
  /* transient sum above 1 - r_min is scaled to 1 - r_min; the absorption is the remainder.  */
  int32_t model;
  double rel_radius;         /* model 1: relative radius (0.5 in the experiment)            */
  double *kl_out;            /* [p_count] DEVICE or NULL: KL(b' || b0) = sum_v b'_v          */
                             /* log(b'_v / b0_v) per perturbation (the robust search's       */
                             /* discrepancy; pair it with b_out to pick the maximiser)        */
  uint64_t *solve_stats;     /* [2] DEVICE or NULL, accumulated: perturbations whose reduced  */
                             /* systems were solved by defect correction on the nominal     */
                             /* factors, and by factoring I - Q'_CC (large c only: c x c     */
                             /* matrices that do not fit in shared memory; small c always   */
                             /* factors in shared memory and counts neither)                 */
} afc_perturb_params;

/* DEVICE outputs (accumulated, caller zeroes): counters [3] = {top-1 changes, top-k set
 * changes, top-k order changes}; pair_flips [k2*k2] (entry a*k2+b, a<b: perturbations where
 * nominal ranks a and b swap); shift_hist [hist_bins] (|rank' - rank| of the nominal top-k2
 * nodes, last bin open); maxima [3] = {max ||b' - b||_inf, max ||b' - (b + db_lin)||_inf with
 * the first-order prediction db_lin, max_i (N' 1)_i} as non-negative doubles (updated with
 * an integer max on their bit patterns).  b_out: DEVICE [p_count][n] or NULL.  b0, mu0, lu0,
 * piv0: the nominal afc_absorbing_solve outputs. */
int afc_perturb_sweep(const afc_chain *chain, const afc_perturb_params *pp,
                      const uint32_t *counts, const int32_t *c_index, const int32_t *c_list,
                      int32_t c, const double *mu0, const double *b0, const double *lu0,
                      const int32_t *piv0, uint64_t *counters, uint64_t *pair_flips,
                      uint64_t *shift_hist, double *maxima, double *b_out, void *workspace,
                      size_t workspace_bytes, void *stream);

/* Ranking certificates (Sec. 5.5): for pairs (pu[k], pv[k]) (DEVICE int32 [npairs]) writes
 * gap[k] = mu_u - mu_v (eq. pm-gap) and sharp[k] = (eps_bar / r_min) max_i |N_iu - N_iv|
 * (eq. sharp-gap) to DEVICE arrays; the crude threshold is 2 eps_bar / r_min^2. */
int afc_certificates(const afc_chain *chain, const uint32_t *counts, const int32_t *c_index,
                     const int32_t *c_list, int32_t c, const double *mu0, const double *lu0,
                     const int32_t *piv0, double eps_bar, double r_min, int32_t npairs,
                     const int32_t *pu, const int32_t *pv, double *gap, double *sharp,
                     void *workspace, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------------------------------------ */
/* End-to-end query from HOST memory                                                      */
/* ------------------------------------------------------------------------------------ */

typedef struct {
  int32_t n; int64_t m;
  const int32_t *eu, *ev;            /* HOST edge list                                     */
  const double *p_survive;           /* HOST [m] or NULL -> p_survive_all                   */
  double p_survive_all;
  const uint32_t *w_lo, *w_hi;       /* HOST [m] or NULL -> the scalars                     */
  uint32_t w_lo_all, w_hi_all;
  uint64_t seed; uint32_t graph_tag; uint32_t realizations;
  uint32_t k_min; double alpha; double absorb_floor;
  const double *s_init;              /* HOST [n] or NULL                                    */
  const double *reward;              /* HOST [n] or NULL                                    */
  const int32_t *candidates; int32_t n_candidates;   /* HOST W or NULL                      */
  uint32_t top_k; double tie_rel; int32_t precision; double recheck_margin;
  uint32_t n_perturb; double l1_radius; double r_min; uint64_t perturb_seed;
  uint32_t r_begin;                  /* first realization index: the query draws realizations */
                                     /* r_begin .. r_begin + realizations - 1 (shards of one    */
                                     /* query on several GPUs take disjoint ranges); 0 usually */
} afc_host_query;

typedef struct {
  uint32_t *counts;                  /* HOST [n][n+1] or NULL                               */
  double *mu, *b;                    /* HOST [n] (b required)                               */
  double expected_T, b_f, max_rowsum_N;
  int32_t c;                         /* |C|                                                 */
  afc_mc_stats stats;
  uint64_t perturb_counters[3];      /* as afc_perturb_sweep with top_k 5, k2 10, 16 bins   */
  double perturb_maxima[3];
  double device_ms;                  /* device time of the query (CUDA events)              */
} afc_host_result;

/* Runs the whole query: CSR build, host-to-device copies, counts, solve and (n_perturb > 0)
 * the perturbation sweep, then device-to-host copies.  Allocates and frees its own device
 * memory (stream-ordered) and SYNCHRONISES `stream` before returning. */
int afc_run_host(const afc_host_query *q, afc_host_result *res, void *stream);

/* ------------------------------------------------------------------------------------ */
/* Serving loop: continuous batching of queries that arrive at any time                   */
/* ------------------------------------------------------------------------------------ */
/* The paper defines one query (a base graph, its failure and weight laws, the sampling
 * budget M and the chain parameters: Sec. 3 and Alg. 2); serving many of them at once is an
 * engineering layer with no counterpart there.  Queries are admitted in arrival order while
 * the device-memory footprint of the admitted ones stays within hbm_budget and at most
 * max_active are admitted.  Every admitted query keeps its graph, parameters and partial
 * counts on the device; a scheduler thread advances the admitted queries with the least
 * remaining work (up to slice_queries of them) by one batched counting launch per slice, so a
 * query that arrives while others run joins a slice as soon as it is among the shortest.  A query whose realizations are
 * all counted is finished (observed states, absorbing-chain solve, perturbation sweep,
 * device-to-host copy) on a second stream by a finisher thread while counting goes on, and
 * its device memory is released.  Realization r of a query is the same draw whatever else
 * runs beside it, so its counts equal those of afc_run_host exactly and its visit shares
 * agree up to the rounding order of the solve's accumulations. */
typedef struct afc_server afc_server;

typedef struct {
  uint64_t hbm_budget;         /* bytes admitted queries may hold (graph, parameters, count */
                               /* matrix); 0 = 80% of free memory.  The finisher's solve    */
                               /* workspace (one query at a time) comes from outside it     */
  uint32_t max_active;         /* queries admitted at once; 0 = 64                          */
  uint32_t max_waiting;        /* queue length beyond which submissions are refused         */
                               /* (AFC_EBUSY, counted as shed); 0 = unbounded               */
  uint32_t slice_realizations; /* realizations per query per slice; 0 = automatic (about   */
                               /* four waves of 1000-node realizations of work per slice)  */
  int32_t keep_counts;         /* 1: results include the [n][n+1] count matrix              */
  uint32_t slice_queries;      /* queries advanced per slice, least remaining work first;   */
                               /* 0 = 4                                                     */
} afc_server_cfg;

typedef struct {
  uint64_t submitted, admitted, completed, shed, failed;
  uint64_t cancelled;          /* queries cancelled before they were counted                 */
  uint64_t realizations;       /* realizations of completed queries                          */
  uint64_t edge_visits;        /* Graph500 edge count of completed queries                   */
  uint64_t slices;             /* batched counting launches                                  */
  uint64_t peak_bytes;         /* largest admitted footprint                                 */
  double p50_ms, p99_ms, mean_ms, max_ms;   /* submit -> result ready, completed queries    */
  double wait_p50_ms, wait_p99_ms;          /* submit -> admission                          */
  double wall_s;               /* first submission -> last completion                       */
  double realizations_per_s;   /* realizations / wall_s                                     */
} afc_serving_stats;

/* Starts the scheduler and finisher threads on the current device. */
int afc_server_create(const afc_server_cfg *cfg, afc_server **out);

/* Copies the query (all HOST arrays are read during the call) and queues it.  AFC_EBUSY:
 * the query alone exceeds hbm_budget, or max_waiting queries are already queued.  Argument
 * errors as afc_run_host. */
int afc_server_submit(afc_server *s, const afc_host_query *q, uint64_t *ticket);

/* Waits up to wait_ms (negative: no limit, 0: just look) for the query's result.  While the
 * query is pending: AFC_EBUSY for a look (wait_ms 0), AFC_ETIMEOUT when a wait of wait_ms > 0
 * ran out (the ticket stays valid; poll again).  Otherwise the query's status, its result
 * copied into res (res->b required, res->mu and res->counts optional; counts only with
 * keep_counts) and, when latency_ms is not NULL, its submit-to-ready time.  A ticket can be
 * collected once. */
int afc_server_poll(afc_server *s, uint64_t ticket, int32_t wait_ms, afc_host_result *res,
                    double *latency_ms);

int afc_server_stats(afc_server *s, afc_serving_stats *out);

/* Cancels the query `ticket`, or every query not yet counted when ticket is 0.  A queued
 * query leaves the queue at once; an admitted one leaves at the next slice boundary (the slice
 * already on the GPU completes) and its device memory is freed; a query already counted
 * finishes normally.  Polling a cancelled ticket returns AFC_ECANCELED.  Returns AFC_OK, or
 * AFC_EINVAL for an unknown or already collected ticket. */
int afc_server_cancel(afc_server *s, uint64_t ticket);

/* Finishes every admitted and queued query, then stops the threads and frees everything. */
void afc_server_destroy(afc_server *s);

/* ------------------------------------------------------------------------------------ */
/* Query handles: graph, parameters, result (all HOST-side; the device is used inside)      */
/* ------------------------------------------------------------------------------------ */
/* The problem statement of Sec. 3 (a base graph and the law of its random realizations) and
 * of Alg. 2 (the sampling budget and the chain parameters) as opaque handles; afc_run is
 * afc_run_host on them, and the result keeps the counts as a sparse matrix. */

typedef struct afc_graph afc_graph;    /* library-owned, immutable after creation            */

/* Undirected edge list (edge id = position, 0 <= eu, ev < n, no self loops or duplicates);
 * copied during the call. */
int afc_graph_create(int32_t n, int64_t m, const int32_t *eu, const int32_t *ev, afc_graph **out);
/* Symmetric CSR over HOST arrays: row_ptr [n+1], col [row_ptr[n]], eid [row_ptr[n]]; every
 * edge id 0..m-1 must appear on exactly the two arcs (u, v) and (v, u), m = row_ptr[n] / 2. */
int afc_graph_create_csr(int32_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *eid,
                         afc_graph **out);
int32_t afc_graph_nodes(const afc_graph *g);
int64_t afc_graph_edges(const afc_graph *g);
void afc_graph_destroy(afc_graph *g);

typedef struct {
  uint64_t seed; uint32_t graph_tag;   /* Philox key and third counter word                 */
  uint32_t realizations;               /* R = M samples per anchor row                      */
  const double *p_survive; double p_survive_all;       /* HOST [m] or NULL -> the scalar    */
  const uint32_t *w_lo, *w_hi; uint32_t w_lo_all, w_hi_all;   /* HOST [m] or the scalars   */
  uint32_t k_min; double alpha; double absorb_floor;
  const double *s_init;                /* HOST [n] or NULL = uniform                        */
  const double *reward;                /* HOST [n] node reward f or NULL                    */
  const int32_t *candidates; int32_t n_candidates;   /* HOST pool W or NULL = all nodes     */
  uint32_t top_k;                      /* 0 = no rank cutoff                                */
  int32_t precision;                   /* AFC_FP64 | AFC_FP32_RECHECK                       */
  double recheck_margin;
  double tie_rel;
  void *cuda_stream;                   /* cudaStream_t, or NULL = the default stream        */
} afc_params;

/* Fills the defaults: p_survive_all 1, lengths 1..1, k_min 5, alpha 0.15, absorb_floor 1e-6,
 * FP64, recheck_margin 1e-4, tie_rel 1e-9, everything else 0 / NULL. */
void afc_params_default(afc_params *p);

typedef struct afc_result afc_result;  /* library-owned; free with afc_result_destroy        */

/* Counts (A1-A7) and the absorbing-chain solve (A8) of one query; SYNCHRONISES the stream. */
int afc_run(const afc_graph *g, const afc_params *p, afc_result **out);

/* Transition counts as a sparse matrix: row i has the columns col[row_ptr[i] .. row_ptr[i+1])
 * (ascending node ids) with counts cnt[...], and absorb[i] absorptions; every row sums to R.
 * The arrays belong to the result. */
int afc_result_counts(const afc_result *r, const int64_t **row_ptr, const int32_t **col,
                      const uint32_t **cnt, const uint32_t **absorb);
/* b [n] (belongs to the result), E_s[T] and b_f = b.f (0 without a reward). */
int afc_result_afc(const afc_result *r, const double **b, double *expected_T, double *b_reward);
/* Realizations recomputed in FP64 (FP32 mode) and a bound on ||b - b_exact||_1 from the FP64
 * solve's residual: 2 ||s - mu (I - Q)||_1 max_i (N 1)_i / ||mu||_1, the residual taken in
 * extended precision on the host. */
int afc_result_diag(const afc_result *r, uint64_t *rechecked, double *fp_err_bound);
void afc_result_destroy(afc_result *r);

typedef struct {
  uint64_t top1_changes, topk_set_changes, topk_order_changes;
  uint64_t pair_flips[100];            /* nominal top-10 pairs a < b swapped: entry a*10+b  */
  uint64_t shift_hist[16];             /* |rank shift| of the nominal top 10, last bin open  */
  double max_shift_inf;                /* max ||b' - b||_inf                                */
  double max_linear_err_inf;           /* max ||b' - (b + db_lin)||_inf (Sec. 5.4)          */
  double max_rowsum_N;                 /* max_i (N' 1)_i over the perturbations             */
} afc_perturb_stats;

/* The perturbation sweep (A9, see afc_perturb_sweep) of a result's kernel: n_perturb
 * perturbations 0 .. n_perturb-1, k2 = 10, 16 histogram bins, the result's tie_rel.  Runs on
 * the stream of the afc_params the result came from and SYNCHRONISES it. */
int afc_perturb(const afc_result *r, uint32_t n_perturb, double l1_radius, double r_min,
                uint64_t seed, uint32_t top_k, afc_perturb_stats *out);

/* Serving with handles: the query (g, p) is copied and queued like afc_server_submit (its
 * counts are kept for the result); afc_poll does not wait: AFC_EBUSY while pending, else the
 * query's status and, on AFC_OK, a result to free with afc_result_destroy. */
int afc_submit(afc_server *s, const afc_graph *g, const afc_params *p, uint64_t *ticket);
int afc_poll(afc_server *s, uint64_t ticket, afc_result **out);

/* Internals of one realization r of (g, p) for bit-exact checks, HOST outputs (each may be
 * NULL): dist [n] and sigma [n] from source s (dist 0xFFFFFFFF and sigma 0 where unreachable;
 * shared-memory path only, else AFC_EUNSUPPORTED), and B [n], the realization's betweenness
 * over ordered pairs for nodes of valid components (0 elsewhere).  SYNCHRONISES the stream. */
int afc_debug_realization(const afc_graph *g, const afc_params *p, uint32_t r, int32_t s,
                          uint32_t *dist, uint64_t *sigma, double *B);

#ifdef __cplusplus
}
#endif
#endif /* AFC_H_ */
