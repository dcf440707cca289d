// afc_internal.h -- structures shared by the library's host code and kernels.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "afc.h"
#include "mc_types.h"

namespace afc {

// bytes of one group's arrays and of one source slot (global path)
size_t big_group_bytes(uint32_t n, uint64_t arcs);
uint32_t big_slot_bytes(uint32_t n);
// bytes of one warp's region of the arena on the settle-step global path (path counts, settle
// order, pending list, and the distances when they are not kept on chip)
size_t big_step_slot_bytes(uint32_t n, bool dist_in_arena);
void big_group_carve(BigGroup &G, unsigned char *base, uint32_t n, uint64_t arcs);
bool big_config_supported(int block, int team);
// Runs realizations [0, r_count) of the problem *Pd (device copy) through the global path in
// batches of ngroups realizations.
// slots_on_chip 0: source slots in the arena; 1: their distance arrays in shared memory
// (smem_bytes = big_dist_smem_bytes); 2: the whole slots in shared memory (smem_bytes =
// big_slots_smem_bytes, the arena unused).
// Shared memory of a Brandes CTA that keeps its slots' distance arrays on chip.
uint32_t big_dist_smem_bytes(uint32_t n, uint32_t nslots);
// Shared memory of a Brandes CTA that keeps its whole slots (stride big_slot_bytes) on chip.
uint32_t big_slots_smem_bytes(uint32_t n, uint32_t nslots);
cudaError_t launch_mc_global(int block, int team, const McDev *Pd, int precision,
                             BigGroup *groups_d, uint32_t ngroups, uint32_t r_count,
                             unsigned char *arena, size_t slot_stride, uint32_t spt,
                             uint32_t smem_bytes, int slots_on_chip, uint32_t grid,
                             cudaStream_t stream);

// abi.cu: counting over per-problem realization ranges (the batched launch of the serving
// loop) and the thread-local error message of the C ABI
int counts_ranges(int nprob, const afc_mc_problem *probs, const uint32_t *r_begin,
                  const uint32_t *r_count, uint32_t *const *counts, afc_mc_stats *const *stats,
                  void *workspace, size_t ws_bytes, cudaStream_t stream);
size_t counts_ranges_workspace(int nprob, const afc_mc_problem *probs, const uint32_t *r_count);
int report_error(int code, const char *msg);

// api.cu: result handle from dense counts and solve outputs; host query of a graph handle
afc_result *build_result(int32_t n, uint32_t R, const uint32_t *dense, const double *b,
                         const double *mu, double expected_T, double b_f, double max_rowsum_N,
                         int32_t c, const afc_mc_stats &stats, double alpha, double eta,
                         const double *s, const double *f, double tie_rel, void *stream);
afc_host_query host_query_of(const afc_graph *g, const afc_params *p, uint32_t n_perturb);

// mc_kernel.cu: the shared-memory path (one warp per source, settle steps)
// Shared memory of a counting CTA of the shared-memory path: a graph of n nodes and `arcs`
// arcs, and `nsw` warps that each own one source slot.
uint32_t mc_layout_bytes(uint32_t n, uint64_t arcs, uint32_t nsw);
// Compact source slots that fit next to the realization within `bytes` (0 unless at least one
// wide slot fits).
uint32_t mc_slots_within(uint32_t n, uint64_t arcs, uint32_t bytes);
// Device memory of one counting CTA of the shared-memory path (graphs of up to n nodes):
// components, source list, selection scratch and betweenness accumulators.
size_t mc_cta_scratch_bytes(uint32_t n);
cudaError_t launch_mc_counts(int block, const McDev *probs_dev, int nprob,
                             const uint64_t *prefix_dev, uint64_t total_items,
                             uint32_t source_warps, uint32_t smem_bytes, uint32_t grid,
                             unsigned char *scratch, size_t scratch_stride, cudaStream_t stream);
cudaError_t launch_debug_realize(const McDev &P, uint32_t r_count, uint8_t *alive, uint32_t *w,
                                 cudaStream_t stream);
cudaError_t launch_debug_components(const McDev &P, uint32_t r_count, int32_t *comp,
                                    int32_t *csize, cudaStream_t stream);
cudaError_t launch_debug_sssp(int block, const McDev &P, uint32_t r, const int32_t *sources,
                              int32_t nsrc, uint32_t source_warps, uint32_t smem, uint32_t *dist,
                              uint64_t *sigma, cudaStream_t stream);

// solve.cu / perturb.cu
struct ChainDev {
  int32_t n;
  uint32_t R;
  double alpha, eta;
  const double *s;       // [n] or null (uniform)
  const double *f;       // [n] or null
  const uint32_t *counts;
  const int32_t *c_index, *c_list;
  int32_t c;
};

// Workspace carve-up of the solve path (byte offsets), shared by solve and perturb.
struct SolveWs {
  size_t off_y, off_t, off_rowscale, off_nzptr, off_nzcol, off_nzval, off_flags, off_tmp, off_csc,
      off_slab, total;
  size_t nnz_cap;
  size_t csc_cap;   // entries of the column-wise pattern of Q_CC the large-c sweep builds (0: none)
};
SolveWs solve_ws_layout(int32_t n, int32_t c, size_t nnz_cap, uint32_t perturb_slabs,
                        size_t slab_bytes, size_t csc_cap);

cudaError_t launch_observed_states(int32_t n, const uint32_t *counts, int32_t *c_index,
                                   int32_t *c_list, int32_t *c_dev, cudaStream_t stream);
cudaError_t launch_solve(const ChainDev &C, double *mu, double *b, double *scalars, double *lu,
                         int32_t *piv, unsigned char *ws, const SolveWs &L, uint32_t *status_dev,
                         cudaStream_t stream);
cudaError_t launch_perturb(const ChainDev &C, const afc_perturb_params &pp, const double *mu0,
                           const double *b0, const double *lu0, const int32_t *piv0,
                           uint64_t *counters, uint64_t *pair_flips, uint64_t *shift_hist,
                           double *maxima, double *b_out, unsigned char *ws, const SolveWs &L,
                           uint32_t *status_dev, int num_sms, cudaStream_t stream);
cudaError_t launch_certificates(const ChainDev &C, const double *mu0, const double *lu0,
                                const int32_t *piv0, double eps_bar, double r_min, int32_t npairs,
                                const int32_t *pu, const int32_t *pv, double *gap, double *sharp,
                                unsigned char *ws, const SolveWs &L, cudaStream_t stream);
size_t perturb_slab_bytes(int32_t n, int32_t c);
// true when the sweep keeps a perturbation's c x c matrix in shared memory (else: device slabs)
bool perturb_on_chip(int32_t c, int smem_optin);
// bootstrap.cu: realization-level bootstrap replicates of b and their percentile intervals
size_t bootstrap_slab_bytes(int32_t n, int32_t c, uint32_t R);
cudaError_t launch_bootstrap(const ChainDev &C, const int32_t *rec, uint32_t R, uint32_t B,
                             uint64_t seed, double level, double *b_rep, double *T_rep,
                             double *lo, double *hi, unsigned char *slabs, size_t slab_space,
                             uint32_t *status, int num_sms, cudaStream_t stream);

// robust.cu: row-wise robust inner problem, policy evaluation and scenario AFC; Wasserstein-1
// distance of two node distributions on the graph's hop metric
cudaError_t launch_robust_inner(int32_t n, uint32_t R, double alpha, double eta,
                                const uint32_t *counts, double eps, double r_min,
                                int support_only, const double *v, double v_bot, double vsign,
                                double *T, double *Qstar, uint32_t *status, cudaStream_t stream);
cudaError_t launch_robust_eval(int32_t n, const double *Qstar, double *A, int32_t *piv,
                               const double *f, double *V, double *x, double *diff,
                               uint32_t *status, cudaStream_t stream);
cudaError_t launch_robust_star(int32_t n, const double *A, const int32_t *piv, const double *s,
                               const double *f, double *mu, double *b, double *out,
                               cudaStream_t stream);
double w1_graph_host(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *eid,
                     const double *x, const double *y);

// w1.cu: the same distances on the device, one warp per row; status bits 1 = excess left that
// reaches no deficit, 2 = an iteration bound, 4 = a broken invariant
// (mode 2: row state and graph in shared memory, 1: row state only, 0: both in the slab)
size_t w1_slot_bytes(int32_t n, int64_t m);
size_t w1_graph_bytes(int32_t n, int64_t m);
cudaError_t launch_w1(int32_t n, int64_t m, const int32_t *rp, const int32_t *col,
                      const int32_t *eid, const double *x, const double *y, int32_t count,
                      double *out, unsigned char *slab, int mode, int grid, uint32_t *status,
                      cudaStream_t stream);
// perturb.cu: ranking under the tie band (rank [n]) and the first k nodes in rank order
cudaError_t launch_rank(int32_t n, const double *b, double tie_rel, int32_t k, int32_t *rank,
                        int32_t *topk, cudaStream_t stream);
// robust.cu: a batch of robust problems on one estimated kernel, each with its own node v,
// sense and Dinkelbach parameter lambda (the envelopes of b_v over the row-wise set); problem
// p's n-vectors at p * vstride, its n x n matrices at p * n * n
struct EnvBatch {
  double *Qs, *A;                 // [P][n][n] the inner problem's kernel; I - Q* then its LU
  double *V, *x, *T, *f;          // [P][vstride]
  int32_t *piv;                   // [P][vstride]
  size_t vstride;
  const uint32_t *active;         // [P] 1 while the problem iterates
  const double *vsign;            // [P] 1: the adversary minimises, -1: it maximises
  const double *lambda;           // [P]
  const int32_t *node;            // [P]
  double *diff, *ratio;           // [P] policy-evaluation change; b_v of the current kernel
};
cudaError_t launch_env_reward(int32_t n, uint32_t P, const EnvBatch &B, cudaStream_t stream);
cudaError_t launch_env_round(int32_t n, uint32_t R, double alpha, double eta,
                             const uint32_t *counts, double eps, double r_min, int support_only,
                             uint32_t P, const EnvBatch &B, uint32_t *status,
                             cudaStream_t stream);
cudaError_t launch_env_ratio(int32_t n, const double *s, uint32_t P, const EnvBatch &B,
                             cudaStream_t stream);
// robust.cu: maximisers of two discrepancies and the sampled envelopes of a robust search
cudaError_t launch_robust_summary(int32_t n, int32_t count, const double *rows, const double *b0,
                                  const double *d1, const double *d2, int32_t *arg, double *lo,
                                  double *hi, cudaStream_t stream);

// constrained.cu: feasibility xi per row, pool mass / censoring summaries, 3-clique pools
cudaError_t launch_feasibility(int32_t n, uint32_t R, double alpha, double eta,
                               const uint32_t *counts, const uint32_t *fb_count, double *xi,
                               cudaStream_t stream);
cudaError_t launch_pool_summaries(int32_t n, const double *b, const uint8_t *in_w,
                                  const uint8_t *fb_set, double *b_pool, double *b_censored,
                                  double *mass, cudaStream_t stream);
// Sets tri to the kept triangles as consecutive (u, v, w) triples (min(S, number of
// triangles) of them).
void clique_pool_host(int32_t n, const int32_t *row_ptr, const int32_t *col, int32_t S,
                      std::vector<int32_t> &tri);

cudaError_t launch_reward_afc(int32_t n, uint32_t R, double alpha, double eta,
                              const uint32_t *counts, const double *b, const double *psi_sum,
                              double *out, cudaStream_t stream);

// solve_static.cu (allocation-free solve; scratch is a file-scope device array)
cudaError_t launch_solve_static(int32_t n, uint32_t R, double alpha, double eta, const double *s,
                                const double *f, const uint32_t *counts, double *mu, double *b,
                                double *scalars, uint32_t *status_host, int32_t *c_host,
                                cudaStream_t stream);
size_t solve_static_bytes();
uint32_t perturb_smem_bytes(int32_t n, int32_t c);

}  // namespace afc
