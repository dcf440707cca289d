// perturb.cu -- A9: row-wise perturbation sweep of the estimated kernel (Sec. 5.1 row-wise
// uncertainty, Sec. 5.4 first-order sensitivity, Sec. 5.5 ranking reversals), with the l1 row
// model or the multiplicative one of the robust experiment (Sec. 9), and KL(b' || b0) per
// perturbation for the sampled robust search (Remark on the robust optimisation viewpoint).
//
// One CTA handles one perturbation p at a time (persistent over p).  The perturbation is
// regenerated from Philox (counter (column, row, p, 1)), never stored: every row i is moved on
// its support J_i (transient columns in C plus the absorbing column), the perturbed reduced
// system (I - Q'_CC)^T mu'_C = s_C + s_U Q'_UC is factored and solved in FP64, and the ranking
// of the perturbed AFC b' is compared with the nominal one.
#include <cstdint>
#include <cuda_runtime.h>

#include "afc_device.cuh"
#include "afc_internal.h"
#include "linalg.cuh"

namespace afc {

// 256 threads and two resident CTAs per SM: the factorisation and the triangular solves of one
// perturbation are barrier-bound, so two perturbations per SM overlap their barrier waits.
constexpr int kPerturbThreads = 256;
constexpr int kPerturbCtasPerSm = 2;
constexpr int kMaxK2 = 32;
constexpr int kMaxHist = 64;

struct PerturbArena {
  double *A;    // [c*c]
  double *y;    // [c]  rhs, then mu'_C
  double *x;    // [c]  first-order rhs, then y_lin
  double *t;    // [c]  (N' 1)_C
  int32_t *piv; // [c]
};

// Bytes of one perturbation's arena, a multiple of 256: the perturbed rows (doubles) follow it
// in the device slab, so its size must keep them 8-byte aligned whatever the parity of c.
__host__ __device__ inline size_t arena_bytes(int32_t c) {
  const size_t cc = (size_t)(c > 0 ? c : 1);
  return (8 * cc * cc + 3 * 8 * cc + 4 * cc + 64 + 255) & ~size_t(255);
}

// Device-slab path (large c): after the arena, an FP32 copy of the matrix for the factors and
// two FP64 vectors of refinement scratch.
__host__ __device__ inline size_t mixed_bytes(int32_t c) {
  const size_t cc = (size_t)(c > 0 ? c : 1);
  return ((4 * cc * cc + 255) & ~size_t(255)) + 2 * ((8 * cc + 255) & ~size_t(255));
}

__device__ inline PerturbArena carve(unsigned char *base, int32_t c) {
  const size_t cc = (size_t)(c > 0 ? c : 1);
  PerturbArena a;
  a.A = reinterpret_cast<double *>(base);
  a.y = a.A + cc * cc;
  a.x = a.y + cc;
  a.t = a.x + cc;
  a.piv = reinterpret_cast<int32_t *>(a.t + cc);
  return a;
}

// Nominal ranking: rank0[v] = #{u : u precedes v}; byrank0[a] = node of nominal rank a < k2.
__global__ void nominal_rank_kernel(int32_t n, const double *b0, double tie_rel, int32_t k2,
                                    int32_t *rank0, int32_t *byrank0) {
  __shared__ double red[33];
  double mx = 0.0;
  for (int32_t v = threadIdx.x; v < n; v += blockDim.x) mx = fmax(mx, b0[v]);
  mx = block_max(mx, red);
  const double tau = tie_rel * mx;
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    int32_t r = 0;
    const double bv = b0[v];
    for (int32_t u = 0; u < n; ++u) {
      if (u == v) continue;
      const double d = b0[u] - bv;
      if (d > tau || (fabs(d) <= tau && u < v)) ++r;
    }
    rank0[v] = r;
    if (r < k2) atomicMax(&byrank0[r], v);
  }
}

__device__ __forceinline__ uint32_t draw_u32(uint32_t j, uint32_t i, uint32_t p, uint32_t k0,
                                              uint32_t k1) {
  return philox4x32_10(make_uint4(j, i, p, 1u), k0, k1).x;
}

constexpr double kTwoM31 = 1.0 / 2147483648.0;   // 2^-31, exact

__device__ __forceinline__ double uniform_draw(uint32_t j, uint32_t i, uint32_t p, uint32_t k0,
                                               uint32_t k1) {
  const uint4 u = philox4x32_10(make_uint4(j, i, p, 1u), k0, k1);
  return (double)u.x * (1.0 / 4294967296.0);
}

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

__device__ __forceinline__ long long warp_sum_ll(long long x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xFFFFFFFFu, x, o);
  return x;
}

// FP64 iterative refinement with FP32 factors: x <- x + F^-1 (b - op(A) x) until the update
// is below 1e-15 of x (op(A) = A^T when TRANS); b = NULL means all ones.  Since every admissible
// kernel has ||N||_inf <= 1 / r_min, I - Q' is well conditioned and each round gains about
// seven digits.  Returns false when 12 rounds do not get there.
template <bool TRANS>
__device__ bool refine(const double *A, const float *Af, const int32_t *piv, int32_t c,
                       const double *b, double *x, double *r, LinScratch ls, double *red) {
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int it = 0; it < 12; ++it) {
    if (TRANS) {
      for (int32_t j = threadIdx.x; j < c; j += blockDim.x) {
        double acc = b ? b[j] : 1.0;
        for (int32_t i = 0; i < c; ++i) acc = fma(-A[(size_t)i * c + j], x[i], acc);
        r[j] = acc;
      }
    } else {
      for (int32_t i = warp; i < c; i += nw) {
        double acc = 0.0;
        for (int32_t j = lane; j < c; j += 32) acc = fma(A[(size_t)i * c + j], x[j], acc);
        acc = warp_sum(acc);
        if (lane == 0) r[i] = (b ? b[i] : 1.0) - acc;
      }
    }
    __syncthreads();
    if (TRANS) lu_solve_transposed_blocked_t(Af, c, c, piv, r);
    else lu_solve_blocked_t(Af, c, c, piv, r);
    double dm = 0.0, xm = 0.0;
    for (int32_t k = threadIdx.x; k < c; k += blockDim.x) {
      x[k] += r[k];
      dm = fmax(dm, fabs(r[k]));
      xm = fmax(xm, fabs(x[k]));
    }
    dm = block_max(dm, red);
    xm = block_max(xm, red);
    if (dm <= 1e-15 * xm) return true;
  }
  return false;
}

// Column-wise pattern of Q_CC for the large-c sweep: column j of the C rows' entries as
// ptr[j] .. ptr[j+1]-1, each giving the entry's index in the sparse rows (e) and its row's
// position in C (a), rows ascending.  Built once per launch: every perturbed kernel keeps the
// nominal support.
struct CscPattern {
  const int32_t *ptr, *e, *a;
};

// Position of column j in the sparse-row entries [lo, hi) (columns ascending), or -1.
__device__ __forceinline__ int32_t find_col(const int32_t *nzcol, int32_t lo, int32_t hi,
                                            int32_t j) {
  while (lo < hi) {
    const int32_t mid = (lo + hi) >> 1;
    const int32_t v = nzcol[mid];
    if (v == j) return mid;
    if (v < j) lo = mid + 1;
    else hi = mid;
  }
  return -1;
}

// One warp per column; fill = 0 counts its entries into cnt[j], fill = 1 writes them at ptr[j].
__global__ void csc_kernel(ChainDev C, const int32_t *nzptr, const int32_t *nzcol, int fill,
                           int32_t *cnt, const int32_t *ptr, int32_t *ce, int32_t *ca) {
  const int32_t c = C.c;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int32_t j = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); j < c;
       j += (int32_t)nwarps) {
    int32_t at = fill ? ptr[j] : 0;
    for (int32_t a0 = 0; a0 < c; a0 += 32) {
      const int32_t a = a0 + (int32_t)lane;
      int32_t e = -1;
      if (a < c) {
        const int32_t i = C.c_list[a];
        e = find_col(nzcol, nzptr[i], nzptr[i + 1] - 1, j);   // the last entry is absorption
      }
      const uint32_t hit = __ballot_sync(0xFFFFFFFFu, e >= 0);
      if (fill && e >= 0) {
        const int32_t pos = at + __popc(hit & ((1u << lane) - 1u));
        ce[pos] = e;
        ca[pos] = a;
      }
      at += __popc(hit);
    }
    if (!fill && lane == 0) cnt[j] = at;
  }
}

// ptr[j] = cnt[0] + ... + cnt[j-1] for j <= c (one CTA of whole warps).
__global__ void csc_scan_kernel(int32_t c, const int32_t *cnt, int32_t *ptr) {
  __shared__ int32_t wt[32];
  __shared__ int32_t base;
  if (threadIdx.x == 0) base = 0;
  __syncthreads();
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  for (int32_t s0 = 0; s0 < c; s0 += blockDim.x) {
    const int32_t j = s0 + threadIdx.x;
    const int32_t x = j < c ? cnt[j] : 0;
    int32_t inc = x;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
      if ((int)lane >= o) inc += y;
    }
    if (lane == 31) wt[warp] = inc;
    __syncthreads();
    int32_t off = base;
    for (uint32_t w = 0; w < warp; ++w) off += wt[w];
    if (j < c) ptr[j] = off + inc - x;
    __syncthreads();
    if (threadIdx.x == 0)
      for (uint32_t w = 0; w < blockDim.x / 32u; ++w) base += wt[w];
    __syncthreads();
  }
  if (threadIdx.x == 0) ptr[c] = base;
}

// Defect correction on the nominal factors (large c): solves op(I - Q'_CC) x = b (op = the
// transpose when TRANS; b NULL = all ones) by x <- x + op(M)^-1 (b - op(I - Q'_CC) x), with
// M = I - Q_CC the nominal matrix the solve factored once.  The residual is sparse (the
// perturbed C rows, qp) and summed in a fixed order; the correction is two triangular solves
// with M's factors, which every CTA of the launch reads (they stay in L2).  The error shrinks
// by the spectral radius of M^-1 (Q' - Q)_CC each round -- about 0.004 for l1 moves of 0.05 on
// a chain whose rows absorb 10%, two to three digits a round.  Starts from x = op(M)^-1 b;
// returns false (the caller then factors I - Q'_CC) when an update shrinks by less than 5x
// from the third round on, or 40 rounds do not bring it below 1e-15 of x.
template <bool TRANS>
__device__ bool defect_solve(const ChainDev &Cd, const double *lu0, const int32_t *piv0,
                             const int32_t *nzptr, const int32_t *nzcol, const double *qp,
                             const CscPattern &P, const double *b, double *x, double *r,
                             double *red) {
  const int32_t c = Cd.c;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int32_t k = threadIdx.x; k < c; k += blockDim.x) x[k] = b ? b[k] : 1.0;
  __syncthreads();
  if (TRANS) lu_solve_transposed_blocked_t(lu0, c, c, piv0, x);
  else lu_solve_blocked_t(lu0, c, c, piv0, x);
  double prev = 0.0;
  for (int it = 0; it < 40; ++it) {
    if (TRANS) {
      // r_j = b_j - x_j + sum_a Q'_aj x_a, gathered down column j
      for (int32_t j = (int32_t)warp; j < c; j += (int32_t)nw) {
        double acc = 0.0;
        for (int32_t k = P.ptr[j] + (int32_t)lane; k < P.ptr[j + 1]; k += 32)
          acc = fma(qp[P.e[k]], x[P.a[k]], acc);
        acc = warp_sum(acc);
        if (lane == 0) r[j] = (b ? b[j] : 1.0) - x[j] + acc;
      }
    } else {
      // r_a = b_a - x_a + sum_j Q'_aj x_j along row a
      for (int32_t a = (int32_t)warp; a < c; a += (int32_t)nw) {
        const int32_t i = Cd.c_list[a];
        double acc = 0.0;
        for (int32_t e = nzptr[i] + (int32_t)lane; e < nzptr[i + 1]; e += 32) {
          const int32_t pj = nzcol[e];
          if (pj < c) acc = fma(qp[e], x[pj], acc);
        }
        acc = warp_sum(acc);
        if (lane == 0) r[a] = (b ? b[a] : 1.0) - x[a] + acc;
      }
    }
    __syncthreads();
    if (TRANS) lu_solve_transposed_blocked_t(lu0, c, c, piv0, r);
    else lu_solve_blocked_t(lu0, c, c, piv0, r);
    double dm = 0.0, xm = 0.0;
    for (int32_t k = threadIdx.x; k < c; k += blockDim.x) {
      x[k] += r[k];
      dm = fmax(dm, fabs(r[k]));
      xm = fmax(xm, fabs(x[k]));
    }
    dm = block_max(dm, red);
    xm = block_max(xm, red);
    if (dm <= 1e-15 * xm) return true;
    if (it >= 2 && !(dm < 0.2 * prev)) return false;
    prev = dm;
  }
  return false;
}

// Entries per lane a perturbed row keeps in registers (rows of up to 32 * kRowRegs entries).
constexpr int kRowRegs = 4;

__device__ __forceinline__ void atomic_max_pos(double *addr, double v) {
  atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

__global__ void __launch_bounds__(kPerturbThreads, kPerturbCtasPerSm)
perturb_kernel(ChainDev C, afc_perturb_params pp, const double *mu0, const double *b0,
               const double *lu0, const int32_t *piv0, const int32_t *nzptr, const int32_t *nzcol,
               const double *nzval, const int32_t *byrank0, uint64_t *counters,
               uint64_t *pair_flips, uint64_t *shift_hist, double *maxima, double *b_out,
               unsigned char *slabs, size_t slab_bytes, int use_smem, int use_priv,
               CscPattern csc, unsigned long long *solve_stats, uint32_t *status) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sval[33];
  __shared__ int32_t sidx[32];
  __shared__ double sb[2];
  __shared__ int32_t sflag[1];
  __shared__ double red[33];
  __shared__ int32_t rk[kMaxK2];
  __shared__ uint32_t loc_pair[kMaxK2 * kMaxK2];
  __shared__ uint32_t loc_hist[kMaxHist];
  __shared__ uint32_t loc_cnt[3];
  LinScratch ls{sval, sidx, sb, sflag};
  const int32_t n = C.n, c = C.c;
  const double s_unif = 1.0 / (double)n;   // the uniform initial law, divided once
  const int32_t k2 = min(pp.k2, min(kMaxK2, n));
  const int32_t kk = min(pp.top_k, n);
  const int32_t H = min(pp.hist_bins, kMaxHist);
  unsigned char *slab = slabs + (size_t)blockIdx.x * slab_bytes;
  PerturbArena ar = carve(use_smem ? smem : slab, c);
  // device-slab path: [arena | FP32 copy of A | refinement vectors | perturbed rows]
  unsigned char *mx = slab + arena_bytes(c);
  float *af = reinterpret_cast<float *>(mx);
  double *by = reinterpret_cast<double *>(mx + (((size_t)4 * c * c + 255) & ~size_t(255)));
  double *rv = by + (((size_t)8 * c + 255) & ~size_t(255)) / 8;
  double *qp = reinterpret_cast<double *>(slab + (use_smem ? 0 : arena_bytes(c) + mixed_bytes(c)));
  const uint32_t k0 = (uint32_t)pp.seed, k1 = (uint32_t)(pp.seed >> 32);
  const uint32_t warp = threadIdx.x >> 5, lane = threadIdx.x & 31u, nw = blockDim.x >> 5;
  // warp-private column sums of the perturbed rows (shared memory, after the arena): a warp
  // handles one row at a time and a row's columns are distinct, so they need no atomics
  double *wy = use_priv ? reinterpret_cast<double *>(smem + arena_bytes(c)) : nullptr;
  double *wx = use_priv ? wy + (size_t)nw * c : nullptr;
  for (int32_t k = threadIdx.x; k < kMaxK2 * kMaxK2; k += blockDim.x) loc_pair[k] = 0;
  for (int32_t k = threadIdx.x; k < kMaxHist; k += blockDim.x) loc_hist[k] = 0;
  if (threadIdx.x < 3) loc_cnt[threadIdx.x] = 0;
  // nominal E[T]
  double part = 0.0;
  for (int32_t i = threadIdx.x; i < n; i += blockDim.x) part += mu0[i];
  const double T0 = block_sum(part, red);
  double loc_db = 0.0, loc_lin = 0.0, loc_t = 0.0;

  // large c: defect correction on the nominal factors; I - Q'_CC is assembled only where it
  // is factored (small c, or a perturbation the correction does not settle)
  const bool defect = !use_smem && csc.ptr != nullptr;
  const bool dense = !defect;
  uint32_t loc_defect = 0, loc_factored = 0;
  const uint32_t p_end = pp.p_begin + pp.p_count;
  for (uint32_t p = pp.p_begin + blockIdx.x; p < p_end; p += gridDim.x) {
    // (1) A' = I (where factored), y' = 0, x = 0
    if (dense)
      for (size_t k = threadIdx.x; k < (size_t)c * c; k += blockDim.x)
        ar.A[k] = (k / c == k % c) ? 1.0 : 0.0;
    for (int32_t k = threadIdx.x; k < c; k += blockDim.x) { ar.y[k] = 0.0; ar.x[k] = 0.0; }
    if (use_priv)
      for (int32_t k = threadIdx.x; k < 2 * (int32_t)nw * c; k += blockDim.x) wy[k] = 0.0;
    __syncthreads();
    // (2) perturb every row (warp per row).  The row lives in registers (kRowRegs entries per
    // lane) through its five passes: draws, mean, l1 norm, clipped shift and total,
    // normalisation; the draw sum is exact integer arithmetic (z = (u - 2^31) / 2^31 exactly,
    // and so is their sum) and one reciprocal replaces the per-entry divisions.  Longer rows
    // go through the slab.
    for (int32_t i = warp; i < n; i += nw) {
      const int32_t e0 = nzptr[i], e1 = nzptr[i + 1];
      const int32_t supp = e1 - e0;
      const int32_t pi = C.c_index[i];
      const double si = C.s ? C.s[i] : s_unif;
      const double mi = mu0[i];
      double *py = use_priv ? wy + (size_t)warp * c : ar.y;
      double *px = use_priv ? wx + (size_t)warp * c : ar.x;
      auto add_y = [&](int32_t j, double v) { if (use_priv) py[j] += v; else atomicAdd(&py[j], v); };
      auto add_x = [&](int32_t j, double v) { if (use_priv) px[j] += v; else atomicAdd(&px[j], v); };
      if (supp <= 32 * kRowRegs) {
        double q0[kRowRegs], qv[kRowRegs];
        int32_t col[kRowRegs], zi_raw[kRowRegs];
        long long isum = 0;
#pragma unroll
        for (int t = 0; t < kRowRegs; ++t) {
          const int32_t e = e0 + (int32_t)lane + 32 * t;
          col[t] = -1; zi_raw[t] = 0; q0[t] = 0.0; qv[t] = 0.0;
          if (e < e1) {
            const int32_t pj = nzcol[e];
            col[t] = pj;
            q0[t] = nzval[e];
            if (pp.model == 0 || pj < c) {
              const uint32_t node = pj < c ? (uint32_t)C.c_list[pj] : (uint32_t)n;
              const int32_t zi = (int32_t)(draw_u32(node, (uint32_t)i, p, k0, k1) - 0x80000000u);
              isum += zi;
              zi_raw[t] = zi;
            }
          }
        }
        double rfin = 0.0;   // the perturbed absorption of the row
        if (pp.model == 1) {
          // multiplicative: q' = clamp(q (1 + rel z), 0, 1) on the transient entries, scaled to
          // 1 - r_min when above it; the absorption is the remainder
          double ts = 0.0;
#pragma unroll
          for (int t = 0; t < kRowRegs; ++t)
            if (col[t] >= 0 && col[t] < c) {
              qv[t] = fmin(fmax(q0[t] * (1.0 + pp.rel_radius * ((double)zi_raw[t] * kTwoM31)), 0.0), 1.0);
              ts += qv[t];
            }
          ts = warp_sum(ts);
          if (ts > 1.0 - pp.r_min) {
            const double f = (1.0 - pp.r_min) / ts;
            ts = 0.0;
#pragma unroll
            for (int t = 0; t < kRowRegs; ++t)
              if (col[t] >= 0 && col[t] < c) { qv[t] *= f; ts += qv[t]; }
            ts = warp_sum(ts);
          }
          rfin = 1.0 - ts;
        } else {
          // l1 model with integer draws: with d_j = z_j supp - sum_k z_k (exact integers, z_j =
          // zi_j 2^-31), the shift is (z_j - mean) l1_radius / ||z - mean||_1 = d_j l1_radius /
          // sum_k |d_k|, so the mean and the l1 norm need no FP64 sums.  The shifts sum to 0 and
          // the nominal row sums to 1, so the perturbed row sums to 1 plus what clipping at 0
          // adds; the absorbing entry (always the row's last) then gives ts = 1 - ra.  Same
          // values as the per-entry FP64 form up to rounding, with far fewer FP64 operations
          // (the sweep is bound by GB300's FP64 pipe).
          const long long S = warp_sum_ll(isum);
          long long dab = 0;
          long long dv[kRowRegs];
#pragma unroll
          for (int t = 0; t < kRowRegs; ++t) {
            dv[t] = 0;
            if (col[t] >= 0) {
              dv[t] = (long long)(int32_t)zi_raw[t] * (long long)supp - S;
              dab += dv[t] < 0 ? -dv[t] : dv[t];
            }
          }
          dab = warp_sum_ll(dab);
          const double coef = dab > 0 ? pp.l1_radius / (double)dab : 0.0;
          double clip = 0.0;
#pragma unroll
          for (int t = 0; t < kRowRegs; ++t)
            if (col[t] >= 0) {
              double v = fma((double)dv[t], coef, q0[t]);
              if (v < 0.0) { clip -= v; v = 0.0; }
              qv[t] = v;
            }
          const bool clipped = __any_sync(0xFFFFFFFFu, clip != 0.0);
          if (clipped) {
            const double inv_tot = 1.0 / (1.0 + warp_sum(clip));
#pragma unroll
            for (int t = 0; t < kRowRegs; ++t) qv[t] *= inv_tot;
          }
          // the absorbing entry: position supp - 1 of the row
          const int32_t la = (supp - 1) & 31, ta = (supp - 1) >> 5;
          double mine = 0.0;
#pragma unroll
          for (int t = 0; t < kRowRegs; ++t)
            if (t == ta) mine = qv[t];
          const double ra = __shfl_sync(0xFFFFFFFFu, mine, la);
          const double ts = 1.0 - ra;
          if (ra < pp.r_min && ts > 0.0) {
            const double f = (1.0 - pp.r_min) / ts;
#pragma unroll
            for (int t = 0; t < kRowRegs; ++t)
              if (col[t] >= 0 && col[t] < c) qv[t] *= f;
          }
          rfin = ra < pp.r_min ? pp.r_min : ra;
        }
#pragma unroll
        for (int t = 0; t < kRowRegs; ++t) {
          const int32_t pj = col[t];
          if (pj < 0) continue;
          const int32_t e = e0 + (int32_t)lane + 32 * t;
          if (pj < c) {
            const double v = qv[t];
            qp[e] = v;
            if (pi >= 0) { if (dense) ar.A[(size_t)pi * c + pj] -= v; }
            else add_y(pj, si * v);
            add_x(pj, mi * (v - q0[t]));
          } else {
            qp[e] = rfin;
          }
        }
      } else if (pp.model == 1) {
        double ts = 0.0;
        for (int32_t e = e0 + lane; e < e1; e += 32) {
          const int32_t pj = nzcol[e];
          if (pj >= c) continue;
          const double z = 2.0 * uniform_draw((uint32_t)C.c_list[pj], (uint32_t)i, p, k0, k1) - 1.0;
          const double v = fmin(fmax(nzval[e] * (1.0 + pp.rel_radius * z), 0.0), 1.0);
          qp[e] = v;
          ts += v;
        }
        ts = warp_sum(ts);
        if (ts > 1.0 - pp.r_min) {
          const double f = (1.0 - pp.r_min) / ts;
          ts = 0.0;
          for (int32_t e = e0 + lane; e < e1; e += 32)
            if (nzcol[e] < c) { qp[e] *= f; ts += qp[e]; }
          ts = warp_sum(ts);
        }
        for (int32_t e = e0 + lane; e < e1; e += 32) {
          const int32_t pj = nzcol[e];
          if (pj < c) {
            const double q = qp[e];
            if (pi >= 0) { if (dense) ar.A[(size_t)pi * c + pj] -= q; }
            else add_y(pj, si * q);
            add_x(pj, mi * (q - nzval[e]));
          } else {
            qp[e] = 1.0 - ts;
          }
        }
      } else {
        // the integer form of the register path (see there), through the slab
        long long isum = 0;
        for (int32_t e = e0 + lane; e < e1; e += 32) {
          const int32_t pj = nzcol[e];
          const uint32_t node = pj < c ? (uint32_t)C.c_list[pj] : (uint32_t)n;
          const int32_t zi = (int32_t)(draw_u32(node, (uint32_t)i, p, k0, k1) - 0x80000000u);
          qp[e] = (double)zi;   // exact
          isum += zi;
        }
        const long long S = warp_sum_ll(isum);
        long long dab = 0;
        for (int32_t e = e0 + lane; e < e1; e += 32) {
          const long long d = (long long)qp[e] * (long long)supp - S;
          dab += d < 0 ? -d : d;
        }
        dab = warp_sum_ll(dab);
        const double coef = dab > 0 ? pp.l1_radius / (double)dab : 0.0;
        double clip = 0.0;
        for (int32_t e = e0 + lane; e < e1; e += 32) {
          const long long d = (long long)qp[e] * (long long)supp - S;
          double v = fma((double)d, coef, nzval[e]);
          if (v < 0.0) { clip -= v; v = 0.0; }
          qp[e] = v;
        }
        if (__any_sync(0xFFFFFFFFu, clip != 0.0)) {
          const double inv_tot = 1.0 / (1.0 + warp_sum(clip));
          for (int32_t e = e0 + lane; e < e1; e += 32) qp[e] *= inv_tot;
        }
        __syncwarp();
        const double ra = qp[e1 - 1];   // the absorbing entry is the row's last
        const double ts = 1.0 - ra;
        const double f = (ra < pp.r_min && ts > 0.0) ? (1.0 - pp.r_min) / ts : 1.0;
        for (int32_t e = e0 + lane; e < e1; e += 32) {
          const int32_t pj = nzcol[e];
          double q = qp[e];
          if (pj < c) {
            if (ra < pp.r_min) q *= f;
            qp[e] = q;
            if (pi >= 0) { if (dense) ar.A[(size_t)pi * c + pj] -= q; }
            else add_y(pj, si * q);
            add_x(pj, mi * (q - nzval[e]));
          } else {
            qp[e] = (ra < pp.r_min) ? pp.r_min : q;
          }
        }
      }
      __syncwarp();
      if (lane == 0 && pi >= 0) add_y(pi, si);
    }
    __syncthreads();
    if (use_priv) {
      for (int32_t k = threadIdx.x; k < c; k += blockDim.x) {
        double sy = 0.0, sx = 0.0;
        for (uint32_t w = 0; w < nw; ++w) { sy += wy[w * c + k]; sx += wx[w * c + k]; }
        ar.y[k] += sy;
        ar.x[k] += sx;
      }
      __syncthreads();
    }
    // (3) factor, mu'_C, (N' 1)_C, first-order y_lin = x N0
    bool ok = true;
    if (c > 0 && use_smem) {
      // A in shared memory: the column-by-column FP64 LU
      ok = lu_factor(ar.A, c, c, ar.piv, ls);
      if (ok) {
        lu_solve_transposed(ar.A, c, c, ar.piv, ar.y, ls);
        for (int32_t k = threadIdx.x; k < c; k += blockDim.x) ar.t[k] = 1.0;
        __syncthreads();
        lu_solve(ar.A, c, c, ar.piv, ar.t, ls);
      }
    } else if (c > 0 && defect &&
               [&] {
                 for (int32_t k = threadIdx.x; k < c; k += blockDim.x) by[k] = ar.y[k];
                 __syncthreads();
                 return defect_solve<true>(C, lu0, piv0, nzptr, nzcol, qp, csc, by, ar.y, rv, red) &&
                        defect_solve<false>(C, lu0, piv0, nzptr, nzcol, qp, csc, nullptr, ar.t, rv,
                                            red);
               }()) {
      ++loc_defect;
    } else if (c > 0) {
      ++loc_factored;
      if (defect) {
        // the correction did not settle: assemble I - Q'_CC from the perturbed C rows
        for (size_t k = threadIdx.x; k < (size_t)c * c; k += blockDim.x)
          ar.A[k] = (k / c == k % c) ? 1.0 : 0.0;
        for (int32_t k = threadIdx.x; k < c; k += blockDim.x) ar.y[k] = by[k];
        __syncthreads();
        for (int32_t a = (int32_t)warp; a < c; a += (int32_t)nw) {
          const int32_t i = C.c_list[a];
          for (int32_t e = nzptr[i] + (int32_t)lane; e < nzptr[i + 1]; e += 32) {
            const int32_t pj = nzcol[e];
            if (pj < c) ar.A[(size_t)a * c + pj] -= qp[e];
          }
        }
        __syncthreads();
      }
      // A in the device slab (large c): blocked LU of an FP32 copy (GB300's FP32 rate is many
      // times its FP64 rate), then FP64 iterative refinement against the FP64 matrix; if the
      // refinement stalls, the FP64 blocked LU of A itself
      const size_t cc = (size_t)c * c;
      for (size_t k = threadIdx.x; k < cc; k += blockDim.x) af[k] = (float)ar.A[k];
      for (int32_t k = threadIdx.x; k < c; k += blockDim.x) { by[k] = ar.y[k]; ar.t[k] = 1.0; }
      __syncthreads();
      bool mixed = lu_factor_blocked_t<float>(af, c, c, ar.piv, ls, reinterpret_cast<float *>(smem));
      if (mixed) {
        lu_solve_transposed_blocked_t(af, c, c, ar.piv, ar.y);
        mixed = refine<true>(ar.A, af, ar.piv, c, by, ar.y, rv, ls, red);
      }
      if (mixed) {
        lu_solve_blocked_t(af, c, c, ar.piv, ar.t);
        mixed = refine<false>(ar.A, af, ar.piv, c, nullptr, ar.t, rv, ls, red);
      }
      if (!mixed) {
        for (int32_t k = threadIdx.x; k < c; k += blockDim.x) { ar.y[k] = by[k]; ar.t[k] = 1.0; }
        __syncthreads();
        ok = lu_factor_blocked(ar.A, c, c, ar.piv, ls, reinterpret_cast<double *>(smem));
        if (ok) {
          lu_solve_transposed(ar.A, c, c, ar.piv, ar.y, ls);
          lu_solve(ar.A, c, c, ar.piv, ar.t, ls);
        }
      }
    }
    if (ok && c > 0) {
      if (use_smem) lu_solve_transposed(lu0, c, c, piv0, ar.x, ls);
      else lu_solve_transposed_blocked_t(lu0, c, c, piv0, ar.x);   // large c: blocked
    }
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(status, kErrSolve);
      continue;
    }
    // (4) E'[T], max b', y_lin . 1
    double pT = 0.0, pY = 0.0, pm = 0.0;
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
      const int32_t pv = C.c_index[v];
      pT += pv >= 0 ? ar.y[pv] : (C.s ? C.s[v] : s_unif);
      if (pv >= 0) pY += ar.x[pv];
    }
    const double T = block_sum(pT, red);
    const double Y1 = block_sum(pY, red);
    const double invT = 1.0 / T;
    for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
      const int32_t pv = C.c_index[v];
      const double bv = (pv >= 0 ? ar.y[pv] : (C.s ? C.s[v] : s_unif)) * invT;
      pm = fmax(pm, bv);
      const double lin = b0[v] + (pv >= 0 ? ar.x[pv] : 0.0) / T0 - b0[v] * Y1 / T0;
      loc_db = fmax(loc_db, fabs(bv - b0[v]));
      loc_lin = fmax(loc_lin, fabs(bv - lin));
      if (b_out) b_out[(size_t)(p - pp.p_begin) * n + v] = bv;
    }
    if (pp.kl_out) {   // KL(b' || b0), the discrepancy the robust search maximises
      double kl = 0.0;
      for (int32_t v = threadIdx.x; v < n; v += blockDim.x) {
        const int32_t pv = C.c_index[v];
        const double bv = (pv >= 0 ? ar.y[pv] : (C.s ? C.s[v] : s_unif)) * invT;
        if (bv > 0.0) kl += bv * log(bv / b0[v]);
      }
      kl = block_sum(kl, red);
      if (threadIdx.x == 0) pp.kl_out[p - pp.p_begin] = kl;
    }
    const double bmax = block_max(pm, red);
    const double tau = pp.tie_rel * bmax;
    // (N' 1) over all rows
    for (int32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const int32_t pi = C.c_index[i];
      double ti;
      if (pi >= 0) {
        ti = ar.t[pi];
      } else {
        ti = 1.0;
        for (int32_t e = nzptr[i]; e < nzptr[i + 1]; ++e)
          if (nzcol[e] < c) ti += qp[e] * ar.t[nzcol[e]];
      }
      loc_t = fmax(loc_t, ti);
    }
    // (5) ranks of the nominal top-k2 nodes under b'
    for (int32_t a = warp; a < k2; a += nw) {
      const int32_t v = byrank0[a];
      const int32_t pv = C.c_index[v];
      const double bv = (pv >= 0 ? ar.y[pv] : (C.s ? C.s[v] : s_unif)) * invT;
      int32_t r = 0;
      for (int32_t u = lane; u < n; u += 32) {
        if (u == v) continue;
        const int32_t pu = C.c_index[u];
        const double bu = (pu >= 0 ? ar.y[pu] : (C.s ? C.s[u] : s_unif)) * invT;
        const double d = bu - bv;
        if (d > tau || (fabs(d) <= tau && u < v)) ++r;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xFFFFFFFFu, r, o);
      if (lane == 0) rk[a] = r;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      bool set_changed = false, order_changed = false;
      for (int32_t a = 0; a < kk && a < k2; ++a) {
        if (rk[a] >= kk) set_changed = true;
        if (rk[a] != a) order_changed = true;
      }
      if (k2 > 0 && rk[0] != 0) loc_cnt[0]++;
      if (set_changed) loc_cnt[1]++;
      if (order_changed) loc_cnt[2]++;
      for (int32_t a = 0; a < k2; ++a) {
        int32_t sh = abs(rk[a] - a);
        if (sh > H - 1) sh = H - 1;
        loc_hist[sh]++;
      }
    }
    for (int32_t q = threadIdx.x; q < k2 * k2; q += blockDim.x) {
      const int32_t a = q / k2, b = q % k2;
      if (a < b && rk[a] > rk[b]) loc_pair[a * kMaxK2 + b]++;
    }
    __syncthreads();
  }
  // flush
  loc_db = block_max(loc_db, red);
  loc_lin = block_max(loc_lin, red);
  loc_t = block_max(loc_t, red);
  if (threadIdx.x == 0 && solve_stats && !use_smem) {
    if (loc_defect) atomicAdd(&solve_stats[0], (unsigned long long)loc_defect);
    if (loc_factored) atomicAdd(&solve_stats[1], (unsigned long long)loc_factored);
  }
  if (threadIdx.x == 0) {
    atomic_max_pos(&maxima[0], loc_db);
    atomic_max_pos(&maxima[1], loc_lin);
    atomic_max_pos(&maxima[2], loc_t);
    for (int k = 0; k < 3; ++k)
      if (loc_cnt[k]) atomicAdd(reinterpret_cast<unsigned long long *>(&counters[k]), (unsigned long long)loc_cnt[k]);
  }
  for (int32_t q = threadIdx.x; q < k2 * k2; q += blockDim.x) {
    const int32_t a = q / k2, b = q % k2;
    const uint32_t v = loc_pair[a * kMaxK2 + b];
    if (v) atomicAdd(reinterpret_cast<unsigned long long *>(&pair_flips[a * pp.k2 + b]), (unsigned long long)v);
  }
  for (int32_t h = threadIdx.x; h < H; h += blockDim.x)
    if (loc_hist[h]) atomicAdd(reinterpret_cast<unsigned long long *>(&shift_hist[h]), (unsigned long long)loc_hist[h]);
}

size_t perturb_slab_bytes(int32_t n, int32_t c) {
  (void)n;
  return (arena_bytes(c) + mixed_bytes(c) + 255) & ~size_t(255);
}

// Position of every node in the order (rank, id) -- rank counts of a tie-band ranking need
// not be distinct, the band is not transitive -- and topk[pos] = v for positions below k.
__global__ void rank_order_kernel(int32_t n, const int32_t *rank, int32_t k, int32_t *topk) {
  for (int32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int32_t rv = rank[v];
    int32_t pos = 0;
    for (int32_t u = 0; u < n; ++u) {
      const int32_t ru = rank[u];
      pos += (ru < rv || (ru == rv && u < v)) ? 1 : 0;
    }
    if (pos < k) topk[pos] = v;
  }
}

cudaError_t launch_rank(int32_t n, const double *b, double tie_rel, int32_t k, int32_t *rank,
                        int32_t *topk, cudaStream_t stream) {
  const int grid = (n + 255) / 256;
  nominal_rank_kernel<<<grid, 256, 0, stream>>>(n, b, tie_rel, 0, rank, nullptr);
  if (topk && k > 0) rank_order_kernel<<<grid, 256, 0, stream>>>(n, rank, k, topk);
  return cudaGetLastError();
}

bool perturb_on_chip(int32_t c, int smem_optin) {
  return (int)arena_bytes(c) + 16 * 1024 <= smem_optin;
}

uint32_t perturb_smem_bytes(int32_t n, int32_t c) {
  (void)n;
  return (uint32_t)arena_bytes(c);
}

cudaError_t launch_perturb(const ChainDev &C, const afc_perturb_params &pp, const double *mu0,
                           const double *b0, const double *lu0, const int32_t *piv0,
                           uint64_t *counters, uint64_t *pair_flips, uint64_t *shift_hist,
                           double *maxima, double *b_out, unsigned char *ws, const SolveWs &L,
                           uint32_t *status_dev, int num_sms, cudaStream_t stream) {
  if (pp.p_count == 0) return cudaSuccess;
  const int32_t n = C.n, c = C.c;
  const int32_t *nzptr = reinterpret_cast<const int32_t *>(ws + L.off_nzptr);
  const int32_t *nzcol = reinterpret_cast<const int32_t *>(ws + L.off_nzcol);
  const double *nzval = reinterpret_cast<const double *>(ws + L.off_nzval);
  int32_t *rank0 = reinterpret_cast<int32_t *>(ws + L.off_flags);
  int32_t *byrank0 = reinterpret_cast<int32_t *>(ws + L.off_tmp);
  cudaMemsetAsync(byrank0, 0, sizeof(int32_t) * kMaxK2, stream);
  nominal_rank_kernel<<<(n + 255) / 256, 256, 0, stream>>>(n, b0, pp.tie_rel, min(pp.k2, kMaxK2),
                                                           rank0, byrank0);
  // per-CTA slab: arena (unless in shared memory) + the perturbed rows
  const uint32_t smem = perturb_smem_bytes(n, c);
  int max_optin = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int use_smem = perturb_on_chip(c, max_optin) ? 1 : 0;
  const uint32_t priv = 2u * (kPerturbThreads / 32) * (uint32_t)(c > 0 ? c : 1) * 8u;
  const int use_priv = (use_smem && (int)(smem + priv) + 16 * 1024 <= max_optin) ? 1 : 0;
  // the slab path takes the blocked LU's tiles as dynamic shared memory
  const uint32_t dyn = use_smem ? smem + (use_priv ? priv : 0u)
                                : (uint32_t)(sizeof(double) * lu_blocked_smem_doubles());   // >= the FP32 tiles
  const size_t nnz_bytes = L.nnz_cap * 8;
  const size_t slab_bytes =
      ((use_smem ? 0 : arena_bytes(c) + mixed_bytes(c)) + nnz_bytes + 255) & ~size_t(255);
  const size_t avail = L.total - L.off_slab;
  size_t fit = avail / (slab_bytes ? slab_bytes : 1);
  if (fit > (size_t)num_sms * kPerturbCtasPerSm) fit = (size_t)num_sms * kPerturbCtasPerSm;
  if (fit > (size_t)pp.p_count) fit = (size_t)pp.p_count;
  const int grid = (int)fit;
  if (grid <= 0) return cudaErrorMemoryAllocation;
  // large c: the column-wise pattern of Q_CC for the defect correction (none: always factor)
  CscPattern csc{nullptr, nullptr, nullptr};
  if (!use_smem && c > 0 && L.csc_cap >= (size_t)c * (size_t)c) {
    int32_t *ptr = reinterpret_cast<int32_t *>(ws + L.off_csc);
    int32_t *ce = ptr + (((size_t)c + 1 + 63) & ~size_t(63));
    int32_t *ca = ce + L.csc_cap;
    const int cgrid = (int)(((size_t)c * 32 + 255) / 256);
    csc_kernel<<<cgrid, 256, 0, stream>>>(C, nzptr, nzcol, 0, ptr, nullptr, nullptr, nullptr);
    csc_scan_kernel<<<1, 1024, 0, stream>>>(c, ptr, ptr);
    csc_kernel<<<cgrid, 256, 0, stream>>>(C, nzptr, nzcol, 1, nullptr, ptr, ce, ca);
    csc = CscPattern{ptr, ce, ca};
  }
  // set on every launch: the attribute is the kernel's limit, and an earlier launch may have
  // left it below what this one needs
  cudaFuncSetAttribute(perturb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn);
  perturb_kernel<<<grid, kPerturbThreads, dyn, stream>>>(
      C, pp, mu0, b0, lu0, piv0, nzptr, nzcol, nzval, byrank0, counters, pair_flips, shift_hist,
      maxima, b_out, ws + L.off_slab, slab_bytes, use_smem, use_priv, csc,
      reinterpret_cast<unsigned long long *>(pp.solve_stats), status_dev);
  return cudaGetLastError();
}

}  // namespace afc
