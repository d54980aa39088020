// Served counting: a request loop with continuous batching.
//
// kmc_server_submit copies a job's reads into host memory and queues it.
// Worker threads, each owning a batch handle (its own CUDA stream and its
// resident, graph-captured engines), loop: take from the head of the queue
// as many jobs as fit one batch (bases, reads, sets) and the device-memory
// budget (the predicted footprint of every job in flight), count them as one
// batch, publish each job's result and latency, and come back for more.  A
// job that arrives while batches run is admitted into the next batch whose
// capacity and memory allow it; two workers keep one batch's host work
// (copies, result split) overlapped with another's kernels.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace kmc {
namespace {

// Predicted device bytes per input byte while a job is counted: the
// distribution and sort buffers scale with the input (2-bit codes and
// masks, super k-mer list and bins about 2, the two key arrays 16 per k-mer
// position, survivors and result up to 24 per distinct k-mer), rounded up.
constexpr uint64_t kFootprintPerBase = 32;

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Job {
  uint64_t id = 0;
  uint32_t k = 0;
  std::vector<char> bases;        // the job's own copy of its reads (kmc_server_submit) ...
  std::vector<uint64_t> offsets;
  const char *bp = nullptr;       // ... or the caller's buffers (kmc_server_submit_ref)
  const uint64_t *op = nullptr;
  uint64_t n_bases = 0;
  uint64_t n_reads = 0;
  uint64_t footprint = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  int status = 0;  // 0 queued, 1 running, 2 done, < 0 error code
  BatchSetResult res;  // the k-mers and counts of a batched job (copied out of the batch)
  // ... or of a job counted on the single-set path: a pinned buffer of the
  // server's pool, written by the device and given back at release
  uint64_t *pk = nullptr;
  uint32_t *pc = nullptr;
  uint64_t pcap = 0, pn = 0;
};

// Page-locked result buffers, recycled between jobs (no allocation and no
// page faults once the pool has grown to the load).
struct ResultPool {
  struct Buf {
    uint64_t *k;
    uint32_t *c;
    uint64_t cap;
  };
  std::mutex mu;
  std::vector<Buf> free;
  int take(uint64_t n, Buf *out) {
    {
      std::lock_guard<std::mutex> g(mu);
      size_t best = free.size();
      for (size_t i = 0; i < free.size(); ++i)
        if (free[i].cap >= n && (best == free.size() || free[i].cap < free[best].cap)) best = i;
      if (best < free.size()) {
        *out = free[best];
        free.erase(free.begin() + (long)best);
        kept -= out->cap * 12;
        return KMC_OK;
      }
    }
    const uint64_t cap = std::max<uint64_t>(n + n / 4, 1u << 16);
    void *k = nullptr, *c = nullptr;
    if (host_alloc(&k, cap * 8, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return KMC_ENOMEM;
    }
    if (host_alloc(&c, cap * 4, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      cudaFreeHost(k);
      return KMC_ENOMEM;
    }
    *out = Buf{static_cast<uint64_t *>(k), static_cast<uint32_t *>(c), cap};
    return KMC_OK;
  }
  // Buffers given back are kept for reuse up to kKeepBytes in all; beyond
  // that they are freed, so that the pool does not keep the host memory of a
  // burst of large results.
  static constexpr uint64_t kKeepBytes = 8ull << 30;
  uint64_t kept = 0;
  void give(uint64_t *k, uint32_t *c, uint64_t cap) {
    if (!k) return;
    {
      std::lock_guard<std::mutex> g(mu);
      if (kept + cap * 12 <= kKeepBytes) {
        free.push_back(Buf{k, c, cap});
        kept += cap * 12;
        return;
      }
    }
    cudaFreeHost(k);
    cudaFreeHost(c);
  }
  ~ResultPool() {
    for (Buf &b : free) {
      cudaFreeHost(b.k);
      cudaFreeHost(b.c);
    }
  }
};

}  // namespace
}  // namespace kmc

using namespace kmc;

struct kmc_server {
  kmc_server_cfg cfg{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job *> queue;
  std::unordered_map<uint64_t, std::unique_ptr<Job>> jobs;
  uint64_t next_id = 1;
  uint64_t inflight = 0;        // predicted bytes of jobs being counted
  uint64_t inflight_jobs = 0;
  bool stop = false;
  std::vector<std::thread> workers;
  std::vector<kmc_batch *> batches;
  // jobs of kSingleMinBases or more: each worker's own handle per k (own
  // stream, kept open, its bin map built once), results into the pool
  std::vector<std::map<uint32_t, kmc_handle *>> singles;
  std::vector<std::map<uint32_t, std::vector<uint32_t>>> single_maps;
  ResultPool pool;
  // statistics
  std::vector<double> lat_ms;
  uint64_t done = 0, n_batches = 0, max_batch_jobs = 0, max_inflight_jobs = 0;
  double t_first = 0, t_last = 0;
  int error = 0;
  uint32_t ready = 0;  // workers done warming up
};

namespace {

bool fits(const kmc_server &s, const std::vector<Job *> &take, uint64_t nb, uint64_t nr, uint64_t fp,
          const Job &j) {
  const kmc_server_cfg &c = s.cfg;
  const uint64_t jb = j.n_bases;
  if (s.inflight + fp + j.footprint > c.mem_budget && !(take.empty() && s.inflight == 0)) return false;
  if (take.empty()) return true;  // a job always fits an empty batch (large ones run alone)
  if (take.size() >= c.batch_sets || jb >= kSingleMinBases) return false;
  return nb + jb + 64 <= c.batch_bases && nr + j.n_reads + 1 <= c.batch_reads;
}

// Builds (and captures) the worker's engine of every k in warm_k_mask by
// counting a small synthetic read set with it.
int warm_up(kmc_batch *b, uint64_t mask) {
  std::vector<char> bases(4000 * 150);
  uint64_t x = 0x2545F4914F6CDD1Dull;
  for (char &c : bases) {
    x ^= x << 13;
    x ^= x >> 7;
    x ^= x << 17;
    c = "ACGT"[x & 3];
  }
  std::vector<uint64_t> offs(4001);
  for (int i = 0; i <= 4000; ++i) offs[i] = (uint64_t)i * 150;
  for (uint32_t k = 1; k <= 32; ++k) {
    if (!((mask >> k) & 1)) continue;
    const char *bp = bases.data();
    const uint64_t *op = offs.data();
    const uint64_t nr = 4000;
    int rc = kmc_batch_run(b, 1, &bp, &op, &nr, &k);
    if (rc) return rc;
  }
  return KMC_OK;
}

// A job on the single-set path, counted on the worker's own open handle for
// its k; the result goes from the device straight into a pooled pinned buffer.
void run_single(kmc_server *s, int w, Job *j, uint64_t fp) {
  kmc_handle *&hh = s->singles[w][j->k];
  std::vector<uint32_t> &map = s->single_maps[w][j->k];
  int rc = KMC_OK;
  if (!hh) {
    kmc_params sp = s->cfg.base;
    sp.k = j->k;
    sp.x = 0;
    sp.cuda_stream = nullptr;
    rc = kmc_open(&hh, &sp);
    if (rc) hh = nullptr;
  } else {
    rc = kmc_reset(hh);
    if (!rc && !map.empty() && !hh->h.map_user) rc = kmc_set_bin_map(hh, map.data(), map.size());
  }
  if (!rc) rc = kmc_add_reads(hh, j->bp, j->op, j->n_reads);
  if (!rc && map.empty()) {
    map.resize(hh->h.n_sig);
    rc = kmc_get_bin_map(hh, map.data(), map.size());
    if (rc) map.clear();
  }
  if (!rc) rc = kmc_count(hh);
  uint64_t n = 0;
  if (!rc) rc = kmc_result_size(hh, &n);
  ResultPool::Buf buf{nullptr, nullptr, 0};
  if (!rc) rc = s->pool.take(n, &buf);
  if (!rc) rc = kmc_result(hh, buf.k, buf.c, n, &n);
  if (!rc && j->n_bases >= kTrimMinBases) rc = handle_trim(hh);  // big buffers back to the device pool
  if (rc && hh) {
    kmc_close(hh);
    hh = nullptr;
    map.clear();
  }
  if (rc && buf.k) {
    s->pool.give(buf.k, buf.c, buf.cap);
    buf = ResultPool::Buf{nullptr, nullptr, 0};
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    const double t = now_s();
    j->t_done = t;
    if (rc == KMC_OK) {
      j->pk = buf.k;
      j->pc = buf.c;
      j->pcap = buf.cap;
      j->pn = n;
      j->status = 2;
      s->lat_ms.push_back((j->t_done - j->t_submit) * 1e3);
      s->done += 1;
    } else {
      j->status = rc;
      s->error = rc;
    }
    std::vector<char>().swap(j->bases);
    std::vector<uint64_t>().swap(j->offsets);
    j->bp = nullptr;
    j->op = nullptr;
    s->inflight -= fp;
    s->inflight_jobs -= 1;
    s->n_batches += 1;
    s->max_batch_jobs = std::max<uint64_t>(s->max_batch_jobs, 1);
    s->t_last = t;
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();
}

void worker(kmc_server *s, int w) {
  kmc_batch *b = s->batches[w];
  cudaSetDevice(s->cfg.base.device);
  const int wrc = warm_up(b, s->cfg.warm_k_mask);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (wrc) s->error = wrc;
    s->ready += 1;
  }
  s->cv_done.notify_all();
  for (;;) {
    std::vector<Job *> take;
    uint64_t fp = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
      if (s->queue.empty()) {
        if (s->stop) return;
        continue;
      }
      // continuous batching: admit queued jobs in arrival order while they fit
      uint64_t nb = 0, nr = 0;
      while (!s->queue.empty()) {
        Job *j = s->queue.front();
        if (!fits(*s, take, nb, nr, fp, *j)) break;
        take.push_back(j);
        s->queue.pop_front();
        nb += j->n_bases;
        nr += j->n_reads;
        fp += j->footprint;
        // a job counted on the single-set path runs alone, so that a worker
        // comes back for more as soon as it is done (the workers run such
        // jobs side by side)
        if (nb + 64 > s->cfg.batch_bases || j->n_bases >= kSingleMinBases) break;
      }
      if (take.empty()) {
        // the head job does not fit the memory budget beside the batches in
        // flight: wait until one of them finishes (or the queue changes),
        // then check again
        const uint64_t seen = s->n_batches;
        const Job *head = s->queue.front();
        s->cv_work.wait(lk, [&] {
          return s->stop || s->n_batches != seen || s->queue.empty() || s->queue.front() != head;
        });
        continue;
      }
      s->inflight += fp;
      s->inflight_jobs += take.size();
      s->max_inflight_jobs = std::max(s->max_inflight_jobs, s->inflight_jobs);
      const double t = now_s();
      for (Job *j : take) {
        j->status = 1;
        j->t_start = t;
      }
    }
    if (take.size() == 1 && take[0]->n_bases >= kSingleMinBases) {
      run_single(s, w, take[0], fp);
      continue;
    }
    std::vector<const char *> bp;
    std::vector<const uint64_t *> op;
    std::vector<uint64_t> nr;
    std::vector<uint32_t> ks;
    for (Job *j : take) {
      bp.push_back(j->bp);
      op.push_back(j->op);
      nr.push_back(j->n_reads);
      ks.push_back(j->k);
    }
    int rc = kmc_batch_run(b, (uint32_t)take.size(), bp.data(), op.data(), nr.data(), ks.data());
    std::vector<BatchSetResult> res(take.size());
    if (rc == KMC_OK)
      for (uint32_t i = 0; i < take.size() && rc == KMC_OK; ++i) rc = batch_take_result(b, i, &res[i]);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      const double t = now_s();
      for (uint32_t i = 0; i < take.size(); ++i) {
        Job *j = take[i];
        j->t_done = t;
        if (rc == KMC_OK) {
          j->res = std::move(res[i]);
          j->status = 2;
          s->lat_ms.push_back((j->t_done - j->t_submit) * 1e3);
          s->done += 1;
        } else {
          j->status = rc;
          s->error = rc;
        }
        std::vector<char>().swap(j->bases);  // the reads are no longer needed
        std::vector<uint64_t>().swap(j->offsets);
        j->bp = nullptr;
        j->op = nullptr;
      }
      s->inflight -= fp;
      s->inflight_jobs -= take.size();
      s->n_batches += 1;
      s->max_batch_jobs = std::max<uint64_t>(s->max_batch_jobs, take.size());
      s->t_last = t;
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0;
  std::sort(v.begin(), v.end());
  const double pos = q * (double)(v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - (double)i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

}  // namespace

extern "C" {

int kmc_server_open(kmc_server **out, const kmc_server_cfg *cfg) {
  if (!out || !cfg) return KMC_EINVAL;
  *out = nullptr;
  kmc_server_cfg c = *cfg;
  if (c.n_workers == 0) c.n_workers = 2;
  if (c.n_workers > 8) return KMC_EINVAL;
  if (c.batch_sets == 0) c.batch_sets = 256;
  if (c.batch_bases == 0) c.batch_bases = 128ull << 20;
  if (c.batch_reads == 0) c.batch_reads = c.batch_bases / 64;
  if (c.mem_budget == 0) c.mem_budget = (uint64_t)c.n_workers * kFootprintPerBase * c.batch_bases;
  auto *s = new kmc_server();
  s->cfg = c;
  for (uint32_t w = 0; w < c.n_workers; ++w) {
    kmc_params p = c.base;
    p.cuda_stream = nullptr;  // every worker runs on a stream of its own
    kmc_batch *b = nullptr;
    int rc = kmc_batch_open(&b, &p, c.batch_bases, c.batch_reads, c.batch_sets, c.batch_flags);
    if (rc) {
      for (kmc_batch *x : s->batches) kmc_batch_close(x);
      delete s;
      return rc;
    }
    s->batches.push_back(b);
  }
  s->singles.resize(c.n_workers);
  s->single_maps.resize(c.n_workers);
  for (uint32_t w = 0; w < c.n_workers; ++w) s->workers.emplace_back(worker, s, (int)w);
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->ready == c.n_workers; });
    if (s->error) {
      const int rc = s->error;
      lk.unlock();
      kmc_server_close(s);
      return rc;
    }
  }
  *out = s;
  return KMC_OK;
}

namespace {
int submit_job(kmc_server *s, uint32_t k, const char *bases, const uint64_t *offsets, uint64_t n_reads,
               uint64_t *job_id, bool copy) {
  if (!s || !offsets || !job_id || k < 1 || k > 32) return KMC_EINVAL;
  if (offsets[0] != 0) return KMC_EINPUT;
  for (uint64_t r = 0; r < n_reads; ++r)
    if (offsets[r + 1] < offsets[r]) return KMC_EINPUT;
  const uint64_t nb = offsets[n_reads];
  if (nb && !bases) return KMC_EINVAL;
  auto j = std::make_unique<Job>();
  j->k = k;
  if (copy) {
    j->bases.assign(bases, bases + nb);
    j->offsets.assign(offsets, offsets + n_reads + 1);
    j->bp = j->bases.data();
    j->op = j->offsets.data();
  } else {
    j->bp = bases;
    j->op = offsets;
  }
  j->n_bases = nb;
  j->n_reads = n_reads;
  j->footprint = kFootprintPerBase * (nb + 64);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return KMC_ESTATE;
    j->id = s->next_id++;
    j->t_submit = now_s();
    if (s->t_first == 0) s->t_first = j->t_submit;
    *job_id = j->id;
    s->queue.push_back(j.get());
    s->jobs[j->id] = std::move(j);
  }
  s->cv_work.notify_one();
  return KMC_OK;
}
}  // namespace

int kmc_server_submit(kmc_server *s, uint32_t k, const char *bases, const uint64_t *offsets,
                      uint64_t n_reads, uint64_t *job_id) {
  return submit_job(s, k, bases, offsets, n_reads, job_id, true);
}

int kmc_server_submit_ref(kmc_server *s, uint32_t k, const char *bases, const uint64_t *offsets,
                          uint64_t n_reads, uint64_t *job_id) {
  return submit_job(s, k, bases, offsets, n_reads, job_id, false);
}

int kmc_server_wait(kmc_server *s, uint64_t job_id, double timeout_s) {
  if (!s) return KMC_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return KMC_EINVAL;
  Job *j = it->second.get();
  const auto pred = [&] { return j->status == 2 || j->status < 0; };
  if (timeout_s < 0) s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return KMC_EAGAIN;
  return j->status < 0 ? j->status : KMC_OK;
}

int kmc_server_result(kmc_server *s, uint64_t job_id, const uint64_t **kmers, const uint32_t **counts,
                      uint64_t *n, double *latency_ms) {
  if (!s) return KMC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return KMC_EINVAL;
  Job *j = it->second.get();
  if (j->status < 0) return j->status;
  if (j->status != 2) return KMC_EAGAIN;
  if (kmers) *kmers = j->pk ? j->pk : j->res.k.get();
  if (counts) *counts = j->pk ? j->pc : j->res.c.get();
  if (n) *n = j->pk ? j->pn : j->res.n;
  if (latency_ms) *latency_ms = (j->t_done - j->t_submit) * 1e3;
  return KMC_OK;
}

int kmc_server_release(kmc_server *s, uint64_t job_id) {
  if (!s) return KMC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(job_id);
  if (it == s->jobs.end()) return KMC_EINVAL;
  if (it->second->status < 2 && it->second->status >= 0) return KMC_ESTATE;
  s->pool.give(it->second->pk, it->second->pc, it->second->pcap);
  s->jobs.erase(it);
  return KMC_OK;
}

int kmc_server_cancel(kmc_server *s, uint64_t job_id) {
  if (!s) return KMC_EINVAL;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return KMC_EINVAL;
    Job *j = it->second.get();
    if (j->status != 0) return KMC_ESTATE;  // admitted, finished or failed
    auto q = std::find(s->queue.begin(), s->queue.end(), j);
    if (q == s->queue.end()) return KMC_ESTATE;
    s->queue.erase(q);
    j->status = KMC_ECANCELED;
    j->t_done = now_s();
    std::vector<char>().swap(j->bases);
    std::vector<uint64_t>().swap(j->offsets);
    j->bp = nullptr;
    j->op = nullptr;
  }
  s->cv_done.notify_all();
  s->cv_work.notify_all();  // a worker may wait on this job as the queue's head
  return KMC_OK;
}

int kmc_server_stats_get(kmc_server *s, kmc_server_stats *st) {
  if (!s || !st) return KMC_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  memset(st, 0, sizeof(*st));
  st->jobs_done = s->done;
  st->jobs_queued = s->queue.size();
  st->batches = s->n_batches;
  st->max_batch_jobs = s->max_batch_jobs;
  st->max_inflight_jobs = s->max_inflight_jobs;
  st->p50_ms = percentile(s->lat_ms, 0.50);
  st->p99_ms = percentile(s->lat_ms, 0.99);
  double sum = 0;
  for (double v : s->lat_ms) sum += v;
  st->mean_ms = s->lat_ms.empty() ? 0 : sum / (double)s->lat_ms.size();
  st->wall_s = s->t_last > s->t_first ? s->t_last - s->t_first : 0;
  st->error = s->error;
  return KMC_OK;
}

void kmc_server_close(kmc_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (std::thread &t : s->workers) t.join();
  for (kmc_batch *b : s->batches) kmc_batch_close(b);
  for (auto &m : s->singles)
    for (auto &kv : m) kmc_close(kv.second);
  for (auto &kv : s->jobs) s->pool.give(kv.second->pk, kv.second->pc, kv.second->pcap);
  delete s;
}

}  // extern "C"
