// server.cu -- the serving loop (continuous batching) behind afc_server_*.
//
// Threads and streams:
//   submit    (caller)   copies the query, builds its CSR on the host, sizes its device
//                        footprint and queues it (or refuses it: over budget, queue full)
//   scheduler (thread 1) admits queued queries in arrival order while the footprint of the
//                        admitted ones fits the budget, uploads each admitted query to the
//                        device once (graph, thresholds, candidate mask, zeroed counts), and
//                        then loops: one batched counting launch per slice advancing the
//                        admitted queries with the least remaining work by their next chunk
//                        of realizations, on the counting stream; a query whose last chunk is
//                        enqueued gets an event and goes to the finisher.  At most two slices
//                        are in flight.
//   finisher  (thread 2) per counted query, on the finishing stream (waits on its event):
//                        observed states, absorbing-chain solve, perturbation sweep,
//                        device-to-host copies; then frees the query's device memory and
//                        releases its footprint, which lets the scheduler admit more.
// Realization r of a query is drawn from (seed, r, edge, graph_tag) alone, so batching never
// changes a query's counts.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "afc_internal.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

enum JobState { kWaiting = 0, kActive = 1, kFinishing = 2, kDone = 3 };

struct Job {
  uint64_t ticket = 0;
  afc_host_query q{};
  int32_t n = 0;
  int64_t m = 0;
  std::vector<int32_t> rp, col, eid;
  std::vector<uint64_t> th;
  std::vector<uint32_t> wlo, whi;
  std::vector<uint8_t> inw;
  std::vector<double> s, f;
  size_t footprint = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  // device state (counting stream allocations, freed by the finisher)
  std::vector<void *> allocs;
  afc_mc_problem prob{};
  uint32_t *counts = nullptr;
  afc_mc_stats *stats = nullptr;
  int32_t *cidx = nullptr, *clist = nullptr;
  double *s_d = nullptr, *f_d = nullptr;
  uint32_t next_r = 0;
  cudaEvent_t counted = nullptr;
  // result
  std::vector<double> b, mu;
  std::vector<uint32_t> counts_h;
  afc_host_result res{};
  int status = AFC_OK;
  std::string err;
  int state = kWaiting;
  bool want_counts = false;   // submitted through afc_submit: the result carries the counts
  bool cancel = false;        // cancelled while admitted: leaves at the next slice boundary
};

using JobP = std::shared_ptr<Job>;

// Device memory an admitted query holds until it is finished: its graph, parameters, count
// matrix and observed-state maps.  The finisher's solve workspace is transient and needed for
// one query at a time; it comes out of the memory left outside the budget.
size_t footprint_of(const Job &j) {
  const size_t n = (size_t)j.n, m = (size_t)j.m;
  size_t b = 4 * (n + 1) + 16 * m + 8 * j.th.size() + 4 * (j.wlo.size() + j.whi.size()) +
             j.inw.size() + 8 * (j.s.size() + j.f.size());
  b += 4 * n * (n + 1) + sizeof(afc_mc_stats) + 8 * n;   // counts, stats, observed-state maps
  return b;
}

// Work of one realization of a query: n single-source problems over its n nodes and 2m arcs.
double realization_work(const Job &j) {
  return (double)j.n * ((double)j.n + 2.0 * (double)j.m);
}
double remaining_work(const Job &j) {
  return realization_work(j) * (double)(j.q.realizations - j.next_r);
}
// Reference work: one realization of a 1000-node graph with 3000 edges.
constexpr double kUnitWork = 1000.0 * 7000.0;

}  // namespace

struct afc_server {
  afc_server_cfg cfg{};
  int device = 0, sms = 1;
  cudaStream_t cs = nullptr, fs = nullptr;
  std::mutex mu;
  std::condition_variable cv_sched, cv_fin, cv_done;
  std::deque<JobP> waiting;
  std::vector<JobP> active;
  std::deque<JobP> finishing;
  std::map<uint64_t, JobP> jobs;
  uint64_t next_ticket = 1;
  size_t used = 0;
  bool stop = false;
  std::thread sched, fin;
  void *ws = nullptr;
  size_t ws_bytes = 0;
  // statistics
  afc_serving_stats st{};
  std::vector<double> lat_ms, wait_ms;
  double t_first = -1.0, t_last = 0.0;
};

namespace {

bool admissible(const afc_server *S) {
  return !S->waiting.empty() && S->active.size() < S->cfg.max_active &&
         S->used + S->waiting.front()->footprint <= S->cfg.hbm_budget;
}

// Device copies of an admitted query (counting stream).
int upload(afc_server *S, Job &j) {
  cudaStream_t s = S->cs;
  auto dalloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s) != cudaSuccess) return nullptr;
    j.allocs.push_back(p);
    return p;
  };
  const size_t n = (size_t)j.n, m = (size_t)j.m;
  int32_t *rp = (int32_t *)dalloc(4 * (n + 1));
  int32_t *col = (int32_t *)dalloc(4 * std::max<size_t>(2 * m, 1));
  int32_t *eid = (int32_t *)dalloc(4 * std::max<size_t>(2 * m, 1));
  uint64_t *th = j.th.empty() ? nullptr : (uint64_t *)dalloc(8 * m);
  uint32_t *wlo = j.wlo.empty() ? nullptr : (uint32_t *)dalloc(4 * m);
  uint32_t *whi = j.whi.empty() ? nullptr : (uint32_t *)dalloc(4 * m);
  uint8_t *inw = j.inw.empty() ? nullptr : (uint8_t *)dalloc(n);
  j.s_d = j.s.empty() ? nullptr : (double *)dalloc(8 * n);
  j.f_d = j.f.empty() ? nullptr : (double *)dalloc(8 * n);
  j.counts = (uint32_t *)dalloc(4 * n * (n + 1));
  j.stats = (afc_mc_stats *)dalloc(sizeof(afc_mc_stats));
  j.cidx = (int32_t *)dalloc(4 * n);
  j.clist = (int32_t *)dalloc(4 * n);
  if (!rp || !col || !eid || !j.counts || !j.stats || !j.cidx || !j.clist ||
      (!j.th.empty() && !th) || (!j.wlo.empty() && !wlo) || (!j.whi.empty() && !whi) ||
      (!j.inw.empty() && !inw) || (!j.s.empty() && !j.s_d) || (!j.f.empty() && !j.f_d)) {
    j.err = "device allocation failed";
    return AFC_ENOMEM;
  }
  cudaMemcpyAsync(rp, j.rp.data(), 4 * (n + 1), cudaMemcpyHostToDevice, s);
  if (m) {
    cudaMemcpyAsync(col, j.col.data(), 8 * m, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(eid, j.eid.data(), 8 * m, cudaMemcpyHostToDevice, s);
  }
  if (th) cudaMemcpyAsync(th, j.th.data(), 8 * m, cudaMemcpyHostToDevice, s);
  if (wlo) cudaMemcpyAsync(wlo, j.wlo.data(), 4 * m, cudaMemcpyHostToDevice, s);
  if (whi) cudaMemcpyAsync(whi, j.whi.data(), 4 * m, cudaMemcpyHostToDevice, s);
  if (inw) cudaMemcpyAsync(inw, j.inw.data(), n, cudaMemcpyHostToDevice, s);
  if (j.s_d) cudaMemcpyAsync(j.s_d, j.s.data(), 8 * n, cudaMemcpyHostToDevice, s);
  if (j.f_d) cudaMemcpyAsync(j.f_d, j.f.data(), 8 * n, cudaMemcpyHostToDevice, s);
  cudaMemsetAsync(j.counts, 0, 4 * n * (n + 1), s);
  cudaMemsetAsync(j.stats, 0, sizeof(afc_mc_stats), s);
  afc_mc_problem &p = j.prob;
  p.row_ptr = rp; p.col = col; p.eid = eid;
  p.thresh = th; p.w_lo = wlo; p.w_hi = whi; p.in_w = inw;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    j.err = cudaGetErrorString(e);
    return AFC_ECUDA;
  }
  return AFC_OK;
}

void mark_failed(Job &j, int code) {
  j.status = code;
  if (j.err.empty()) j.err = afc_last_error();
}

void scheduler_main(afc_server *S) {
  cudaSetDevice(S->device);
  std::deque<cudaEvent_t> inflight;
  for (;;) {
    std::vector<JobP> admit, batch;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_sched.wait(lk, [&] { return S->stop || admissible(S) || !S->active.empty(); });
      if (S->stop) break;
      while (admissible(S)) {
        JobP j = S->waiting.front();
        S->waiting.pop_front();
        S->used += j->footprint;
        S->st.peak_bytes = std::max<uint64_t>(S->st.peak_bytes, S->used);
        S->st.admitted++;
        j->t_admit = now_s();
        S->wait_ms.push_back(1e3 * (j->t_admit - j->t_submit));
        j->state = kActive;
        admit.push_back(j);
      }
    }
    std::vector<JobP> failed;
    for (JobP &j : admit) {
      const int rc = upload(S, *j);
      if (rc) {
        mark_failed(*j, rc);
        failed.push_back(j);
      }
    }
    std::vector<JobP> done;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (JobP &j : admit)
        if (j->status == AFC_OK) S->active.push_back(j);
      // cancelled queries leave here (their slices so far are already on the stream)
      for (JobP &j : S->active)
        if (j->cancel) {
          j->status = AFC_ECANCELED;
          j->err = "query cancelled";
          done.push_back(j);
        } else {
          batch.push_back(j);
        }
    }
    // The next slice: the admitted queries with the least remaining work first (at most
    // slice_queries of them), each advanced by a chunk of realizations sized so that the slice
    // holds about four waves of 1000-node realizations of work: small queries finish within a
    // few slices and every slice stays short, so new arrivals join quickly.
    std::sort(batch.begin(), batch.end(), [](const JobP &a, const JobP &b) {
      const double ca = remaining_work(*a), cb = remaining_work(*b);
      return ca < cb || (ca == cb && a->ticket < b->ticket);
    });
    if (batch.size() > S->cfg.slice_queries) batch.resize(S->cfg.slice_queries);
    if (!batch.empty()) {
      const double share = 4.0 * (double)S->sms * kUnitWork / (double)batch.size();
      std::vector<afc_mc_problem> probs;
      std::vector<uint32_t> rb, rc;
      std::vector<uint32_t *> cnt;
      std::vector<afc_mc_stats *> sts;
      for (JobP &j : batch) {
        const uint32_t left = j->q.realizations - j->next_r;
        const double per = std::max(1.0, std::floor(share / realization_work(*j)));
        const uint32_t slice = S->cfg.slice_realizations
                                   ? S->cfg.slice_realizations
                                   : (uint32_t)std::min<double>(per, 4096.0);
        const uint32_t k = std::min(left, slice);
        probs.push_back(j->prob);
        rb.push_back(j->q.r_begin + j->next_r);
        rc.push_back(k);
        cnt.push_back(j->counts);
        sts.push_back(j->stats);
      }
      const size_t need = afc::counts_ranges_workspace((int)probs.size(), probs.data(), rc.data());
      int rcode = AFC_OK;
      if (need > S->ws_bytes) {
        if (S->ws) cudaFreeAsync(S->ws, S->cs);
        S->ws = nullptr;
        S->ws_bytes = 0;
        const size_t want = need + need / 4;
        if (cudaMallocAsync(&S->ws, want, S->cs) == cudaSuccess) S->ws_bytes = want;
        else rcode = afc::report_error(AFC_ENOMEM, "serving workspace allocation failed");
      }
      if (rcode == AFC_OK)
        rcode = afc::counts_ranges((int)probs.size(), probs.data(), rb.data(), rc.data(),
                                   cnt.data(), sts.data(), S->ws, S->ws_bytes, S->cs);
      cudaEvent_t ev = nullptr;
      cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      cudaEventRecord(ev, S->cs);
      inflight.push_back(ev);
      for (size_t k = 0; k < batch.size(); ++k) {
        Job &j = *batch[k];
        if (rcode != AFC_OK) {
          mark_failed(j, rcode);
          done.push_back(batch[k]);
          continue;
        }
        j.next_r += rc[k];
        if (j.next_r >= j.q.realizations) {
          cudaEventCreateWithFlags(&j.counted, cudaEventDisableTiming);
          cudaEventRecord(j.counted, S->cs);
          done.push_back(batch[k]);
        }
      }
      std::lock_guard<std::mutex> lk(S->mu);
      S->st.slices++;
    }
    // every query handed to the finisher carries an event after its last counting work, so
    // that its device memory is freed only once the counting stream is done with it
    for (std::vector<JobP> *v : {&failed, &done})
      for (JobP &j : *v)
        if (!j->counted) {
          cudaEventCreateWithFlags(&j->counted, cudaEventDisableTiming);
          cudaEventRecord(j->counted, S->cs);
        }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      for (JobP &j : failed) {
        j->state = kFinishing;
        S->finishing.push_back(j);
      }
      for (JobP &j : done) {
        S->active.erase(std::find(S->active.begin(), S->active.end(), j));
        j->state = kFinishing;
        S->finishing.push_back(j);
      }
    }
    if (!failed.empty() || !done.empty()) S->cv_fin.notify_one();
    while (inflight.size() > 2) {
      cudaEventSynchronize(inflight.front());
      cudaEventDestroy(inflight.front());
      inflight.pop_front();
    }
  }
  for (cudaEvent_t e : inflight) {
    cudaEventSynchronize(e);
    cudaEventDestroy(e);
  }
}

// Solve, perturbation sweep and copies of one counted query (finishing stream).
int finish(afc_server *S, Job &j) {
  cudaStream_t s = S->fs;
  if (j.counted) cudaStreamWaitEvent(s, j.counted, 0);
  std::vector<void *> tmp;
  auto dalloc = [&](size_t bytes) -> void * {
    void *p = nullptr;
    if (cudaMallocAsync(&p, std::max<size_t>(bytes, 16), s) != cudaSuccess) return nullptr;
    tmp.push_back(p);
    return p;
  };
  auto release = [&]() {
    for (void *p : tmp) cudaFreeAsync(p, s);
  };
  const int32_t n = j.n;
  int32_t c = 0;
  int rc = afc_observed_states(n, j.counts, j.cidx, j.clist, &c, s);
  if (rc) { release(); return rc; }
  afc_chain ch{n, j.q.realizations, j.q.alpha, j.q.absorb_floor, j.s_d, j.f_d};
  const size_t wss = afc_solve_workspace(n, c);
  void *ws = dalloc(wss);
  double *mu = (double *)dalloc(8 * (size_t)n);
  double *b = (double *)dalloc(8 * (size_t)n);
  double *sc = (double *)dalloc(8 * 4);
  double *lu = (double *)dalloc(8 * (size_t)std::max(c, 1) * (size_t)std::max(c, 1));
  int32_t *piv = (int32_t *)dalloc(4 * (size_t)std::max(c, 1));
  uint64_t *pc = (uint64_t *)dalloc(8 * (3 + 100 + 16));
  double *pm = (double *)dalloc(8 * 3);
  if (!ws || !mu || !b || !sc || !lu || !piv || !pc || !pm) {
    release();
    return afc::report_error(AFC_ENOMEM, "finisher allocation failed");
  }
  rc = afc_absorbing_solve(&ch, j.counts, j.cidx, j.clist, c, mu, b, sc, lu, piv, ws, wss, s);
  if (!rc && j.q.n_perturb > 0) {
    cudaMemsetAsync(pc, 0, 8 * (3 + 100 + 16), s);
    cudaMemsetAsync(pm, 0, 8 * 3, s);
    afc_perturb_params pp{0, j.q.n_perturb, j.q.l1_radius, j.q.r_min, j.q.perturb_seed, 5, 10, 16,
                          j.q.tie_rel};
    rc = afc_perturb_sweep(&ch, &pp, j.counts, j.cidx, j.clist, c, mu, b, lu, piv, pc, pc + 3,
                           pc + 103, pm, nullptr, ws, wss, s);
  }
  double scal[4] = {0, 0, 0, 0};
  if (!rc) {
    j.b.resize((size_t)n);
    j.mu.resize((size_t)n);
    cudaMemcpyAsync(j.b.data(), b, 8 * (size_t)n, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(j.mu.data(), mu, 8 * (size_t)n, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(scal, sc, sizeof(scal), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&j.res.stats, j.stats, sizeof(afc_mc_stats), cudaMemcpyDeviceToHost, s);
    if (S->cfg.keep_counts || j.want_counts) {
      j.counts_h.resize((size_t)n * ((size_t)n + 1));
      cudaMemcpyAsync(j.counts_h.data(), j.counts, 4 * j.counts_h.size(), cudaMemcpyDeviceToHost, s);
    }
    if (j.q.n_perturb > 0) {
      cudaMemcpyAsync(j.res.perturb_counters, pc, 8 * 3, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(j.res.perturb_maxima, pm, 8 * 3, cudaMemcpyDeviceToHost, s);
    }
  }
  release();
  const cudaError_t e = cudaStreamSynchronize(s);
  if (!rc && e != cudaSuccess) rc = afc::report_error(AFC_ECUDA, cudaGetErrorString(e));
  if (!rc) {
    j.res.expected_T = scal[0];
    j.res.b_f = scal[1];
    j.res.max_rowsum_N = scal[2];
    j.res.c = c;
    if (j.res.stats.device_error) rc = afc::report_error(AFC_EDEVICE, "device consistency check failed");
    else if (j.res.stats.overflow) rc = afc::report_error(AFC_EOVERFLOW, "path count overflow");
  }
  return rc;
}

void finisher_main(afc_server *S) {
  cudaSetDevice(S->device);
  for (;;) {
    JobP j;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      S->cv_fin.wait(lk, [&] { return S->stop || !S->finishing.empty(); });
      if (S->finishing.empty()) break;   // stop requested and nothing left
      j = S->finishing.front();
      S->finishing.pop_front();
    }
    if (j->status == AFC_OK) {
      const int rc = finish(S, *j);
      if (rc) mark_failed(*j, rc);
    } else if (j->counted) {
      cudaStreamWaitEvent(S->fs, j->counted, 0);
    }
    for (void *p : j->allocs) cudaFreeAsync(p, S->fs);
    j->allocs.clear();
    cudaStreamSynchronize(S->fs);
    if (j->counted) {
      cudaEventDestroy(j->counted);
      j->counted = nullptr;
    }
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->used -= j->footprint;
      j->t_done = now_s();
      j->res.device_ms = 1e3 * (j->t_done - j->t_admit);
      j->state = kDone;
      if (j->status == AFC_OK) {
        S->st.completed++;
        S->st.realizations += j->q.realizations;
        S->st.edge_visits += j->res.stats.edge_visits;
        S->lat_ms.push_back(1e3 * (j->t_done - j->t_submit));
      } else if (j->status == AFC_ECANCELED) {
        S->st.cancelled++;
      } else {
        S->st.failed++;
      }
      S->t_last = std::max(S->t_last, j->t_done);
    }
    S->cv_done.notify_all();
    S->cv_sched.notify_one();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t lo = (size_t)pos;
  const size_t hi = std::min(lo + 1, v.size() - 1);
  return v[lo] + (pos - (double)lo) * (v[hi] - v[lo]);
}

}  // namespace

extern "C" {

int afc_server_create(const afc_server_cfg *cfg, afc_server **out) {
  if (!out) return afc::report_error(AFC_EINVAL, "null output");
  *out = nullptr;
  auto S = std::make_unique<afc_server>();
  if (cfg) S->cfg = *cfg;
  if (cudaGetDevice(&S->device) != cudaSuccess)
    return afc::report_error(AFC_ECUDA, "no CUDA device");
  cudaDeviceGetAttribute(&S->sms, cudaDevAttrMultiProcessorCount, S->device);
  if (S->cfg.max_active == 0) S->cfg.max_active = 64;
  if (S->cfg.slice_queries == 0) S->cfg.slice_queries = 4;
  if (S->cfg.hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return afc::report_error(AFC_ECUDA, "cudaMemGetInfo");
    S->cfg.hbm_budget = (uint64_t)(0.8 * (double)fr);
  }
  if (cudaStreamCreateWithFlags(&S->cs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&S->fs, cudaStreamNonBlocking) != cudaSuccess)
    return afc::report_error(AFC_ECUDA, "stream creation failed");
  afc_server *raw = S.get();
  raw->sched = std::thread(scheduler_main, raw);
  raw->fin = std::thread(finisher_main, raw);
  *out = S.release();
  return AFC_OK;
}

}  // extern "C"

namespace {

int submit_job(afc_server *S, const afc_host_query *q, bool want_counts, uint64_t *ticket) {
  if (!S || !q || !ticket) return afc::report_error(AFC_EINVAL, "null argument");
  auto j = std::make_shared<Job>();
  j->want_counts = want_counts;
  j->t_submit = now_s();
  j->q = *q;
  j->n = q->n;
  j->m = q->m;
  const int32_t n = q->n;
  const int64_t m = q->m;
  if (n < 1 || m < 0) return afc::report_error(AFC_EINVAL, "bad n/m");
  j->rp.resize((size_t)n + 1);
  j->col.resize((size_t)std::max<int64_t>(2 * m, 1));
  j->eid.resize(j->col.size());
  int st = afc_csr_from_edges(n, m, q->eu, q->ev, j->rp.data(), j->col.data(), j->eid.data());
  if (st) return st;
  if (q->p_survive) {
    j->th.resize((size_t)m);
    for (int64_t e = 0; e < m; ++e) j->th[e] = afc_survival_threshold(q->p_survive[e]);
  }
  if (q->w_lo) j->wlo.assign(q->w_lo, q->w_lo + m);
  if (q->w_hi) j->whi.assign(q->w_hi, q->w_hi + m);
  if (q->candidates) {
    j->inw.assign((size_t)n, 0);
    for (int32_t k = 0; k < q->n_candidates; ++k) {
      if (q->candidates[k] < 0 || q->candidates[k] >= n)
        return afc::report_error(AFC_EINVAL, "candidate out of range");
      j->inw[q->candidates[k]] = 1;
    }
  }
  if (q->s_init) j->s.assign(q->s_init, q->s_init + n);
  if (q->reward) j->f.assign(q->reward, q->reward + n);
  j->q.eu = j->q.ev = nullptr;
  j->q.p_survive = nullptr;
  j->q.w_lo = j->q.w_hi = nullptr;
  j->q.s_init = j->q.reward = nullptr;
  j->q.candidates = nullptr;
  afc_mc_problem &p = j->prob;
  p.n = n; p.m = m;
  p.seed = q->seed; p.graph_tag = q->graph_tag;
  p.thresh_all = afc_survival_threshold(q->p_survive_all);
  p.w_lo_all = q->w_lo_all; p.w_hi_all = q->w_hi_all;
  p.k_min = q->k_min; p.top_k = q->top_k; p.tie_rel = q->tie_rel;
  p.precision = q->precision; p.recheck_margin = q->recheck_margin;
  p.block_threads = 1024;   // one block size for every query of a batched launch
  {
    // argument checks of the counting path, with placeholders for the device arrays
    afc_mc_problem chk = p;
    static const int32_t dummy[1] = {0};
    static const uint32_t dummy_u[1] = {1};
    static const uint64_t dummy_t[1] = {0};
    chk.row_ptr = chk.col = chk.eid = dummy;
    if (!j->wlo.empty()) chk.w_lo = dummy_u;
    if (!j->whi.empty()) chk.w_hi = dummy_u;
    if (!j->th.empty()) chk.thresh = dummy_t;
    if (afc_transition_counts_workspace(&chk) == 0) return AFC_EINVAL;
  }
  j->footprint = footprint_of(*j);
  std::lock_guard<std::mutex> lk(S->mu);
  if (j->footprint > S->cfg.hbm_budget) {
    S->st.shed++;
    return afc::report_error(AFC_EBUSY, "query footprint exceeds the serving budget");
  }
  if (S->cfg.max_waiting && S->waiting.size() >= S->cfg.max_waiting) {
    S->st.shed++;
    return afc::report_error(AFC_EBUSY, "serving queue full");
  }
  j->ticket = S->next_ticket++;
  *ticket = j->ticket;
  S->jobs[j->ticket] = j;
  S->waiting.push_back(j);
  S->st.submitted++;
  if (S->t_first < 0) S->t_first = j->t_submit;
  S->cv_sched.notify_one();
  return AFC_OK;
}

}  // namespace

extern "C" {

int afc_server_submit(afc_server *S, const afc_host_query *q, uint64_t *ticket) {
  return submit_job(S, q, false, ticket);
}

int afc_submit(afc_server *S, const afc_graph *g, const afc_params *p, uint64_t *ticket) {
  if (!g || !p) return afc::report_error(AFC_EINVAL, "null argument");
  const afc_host_query q = afc::host_query_of(g, p, 0);
  return submit_job(S, &q, true, ticket);
}

int afc_poll(afc_server *S, uint64_t ticket, afc_result **out) {
  if (!S || !out) return afc::report_error(AFC_EINVAL, "null argument");
  *out = nullptr;
  JobP j;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return afc::report_error(AFC_EINVAL, "unknown or collected ticket");
    if (it->second->state != kDone) return AFC_EBUSY;
    j = it->second;
    S->jobs.erase(it);
  }
  if (j->status != AFC_OK) return afc::report_error(j->status, j->err.c_str());
  if (j->counts_h.empty()) return afc::report_error(AFC_EINVAL, "query was not submitted with afc_submit");
  *out = afc::build_result(j->n, j->q.realizations, j->counts_h.data(), j->b.data(), j->mu.data(),
                           j->res.expected_T, j->res.b_f, j->res.max_rowsum_N, j->res.c,
                           j->res.stats, j->q.alpha, j->q.absorb_floor,
                           j->s.empty() ? nullptr : j->s.data(),
                           j->f.empty() ? nullptr : j->f.data(), j->q.tie_rel, nullptr);
  return AFC_OK;
}

int afc_server_poll(afc_server *S, uint64_t ticket, int32_t wait_ms, afc_host_result *res,
                    double *latency_ms) {
  if (!S || !res || !res->b) return afc::report_error(AFC_EINVAL, "null argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->jobs.find(ticket);
  if (it == S->jobs.end()) return afc::report_error(AFC_EINVAL, "unknown or collected ticket");
  JobP j = it->second;
  auto ready = [&] { return j->state == kDone; };
  if (wait_ms < 0) S->cv_done.wait(lk, ready);
  else if (wait_ms > 0) S->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
  // a look (wait_ms 0) at a pending query: busy; a bounded wait that ran out: timeout
  if (!ready()) return wait_ms == 0 ? AFC_EBUSY : AFC_ETIMEOUT;
  S->jobs.erase(it);
  lk.unlock();
  if (latency_ms) *latency_ms = 1e3 * (j->t_done - j->t_submit);
  if (j->status != AFC_OK) return afc::report_error(j->status, j->err.c_str());
  uint32_t *counts = res->counts;
  double *mu = res->mu, *b = res->b;
  *res = j->res;
  res->counts = counts; res->mu = mu; res->b = b;
  std::memcpy(b, j->b.data(), 8 * j->b.size());
  if (mu) std::memcpy(mu, j->mu.data(), 8 * j->mu.size());
  if (counts && !j->counts_h.empty()) std::memcpy(counts, j->counts_h.data(), 4 * j->counts_h.size());
  return AFC_OK;
}

int afc_server_stats(afc_server *S, afc_serving_stats *out) {
  if (!S || !out) return afc::report_error(AFC_EINVAL, "null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  *out = S->st;
  out->p50_ms = percentile(S->lat_ms, 0.50);
  out->p99_ms = percentile(S->lat_ms, 0.99);
  out->max_ms = S->lat_ms.empty() ? 0.0 : *std::max_element(S->lat_ms.begin(), S->lat_ms.end());
  double sum = 0.0;
  for (double x : S->lat_ms) sum += x;
  out->mean_ms = S->lat_ms.empty() ? 0.0 : sum / (double)S->lat_ms.size();
  out->wait_p50_ms = percentile(S->wait_ms, 0.50);
  out->wait_p99_ms = percentile(S->wait_ms, 0.99);
  out->wall_s = S->t_first < 0 ? 0.0 : std::max(0.0, S->t_last - S->t_first);
  out->realizations_per_s = out->wall_s > 0 ? (double)out->realizations / out->wall_s : 0.0;
  return AFC_OK;
}

int afc_server_cancel(afc_server *S, uint64_t ticket) {
  if (!S) return afc::report_error(AFC_EINVAL, "null server");
  std::vector<JobP> targets;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (ticket) {
      auto it = S->jobs.find(ticket);
      if (it == S->jobs.end()) return afc::report_error(AFC_EINVAL, "unknown or collected ticket");
      targets.push_back(it->second);
    } else {
      for (auto &kv : S->jobs) targets.push_back(kv.second);
    }
    const double t = now_s();
    for (JobP &j : targets) {
      if (j->state == kWaiting) {
        S->waiting.erase(std::find(S->waiting.begin(), S->waiting.end(), j));
        j->status = AFC_ECANCELED;
        j->err = "query cancelled";
        j->state = kDone;
        j->t_done = t;
        S->st.cancelled++;
      } else if (j->state == kActive) {
        j->cancel = true;
      }
    }
  }
  S->cv_done.notify_all();
  S->cv_sched.notify_one();
  return AFC_OK;
}

void afc_server_destroy(afc_server *S) {
  if (!S) return;
  {
    std::unique_lock<std::mutex> lk(S->mu);
    // drain: everything queued or admitted completes first
    S->cv_done.wait(lk, [&] {
      return S->waiting.empty() && S->active.empty() && S->finishing.empty() &&
             std::all_of(S->jobs.begin(), S->jobs.end(),
                         [](const std::pair<const uint64_t, JobP> &kv) { return kv.second->state == kDone; });
    });
    S->stop = true;
  }
  S->cv_sched.notify_all();
  S->cv_fin.notify_all();
  if (S->sched.joinable()) S->sched.join();
  if (S->fin.joinable()) S->fin.join();
  if (S->ws) cudaFreeAsync(S->ws, S->cs);
  cudaStreamSynchronize(S->cs);
  cudaStreamSynchronize(S->fs);
  cudaStreamDestroy(S->cs);
  cudaStreamDestroy(S->fs);
  delete S;
}

}  // extern "C"
