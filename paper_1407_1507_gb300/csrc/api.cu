// C ABI of the k-mer counter (include/kmc.h): handles, parameter checks,
// memory, staging of host reads, and the two phases of the paper's
// algorithm (Sect. 2.4): distribution (at kmc_add_reads*) and sorting (at
// kmc_count).
#include <atomic>
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"
#include "common.cuh"

namespace kmc {

namespace {
constexpr uint64_t kDefaultPieceBytes = 1ull << 28;  // distribution works on pieces of ~256 MiB
constexpr uint64_t kSampleReads = 1ull << 20;   // bin-map sample (Sect. 2.4)
constexpr uint64_t kSampleBytes = 1ull << 28;

thread_local char g_last_err[256];

cudaMemPool_t pool_for(int dev) {
  static std::mutex mu;
  static std::vector<cudaMemPool_t> pools;
  std::lock_guard<std::mutex> g(mu);
  if ((int)pools.size() <= dev) pools.resize(dev + 1, nullptr);
  if (!pools[dev]) {
    cudaMemPoolProps pr{};
    pr.allocType = cudaMemAllocationTypePinned;
    pr.handleTypes = cudaMemHandleTypeNone;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &pr) != cudaSuccess) return nullptr;
    uint64_t thr = ~0ull;  // keep freed memory in the pool for reuse
    cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr);
    pools[dev] = p;
  }
  return pools[dev];
}

__global__ void find_bounds_kernel(const uint64_t *offsets, uint64_t n_reads, const uint64_t *targets,
                                   uint32_t n_t, uint64_t *out_read, uint64_t *out_off) {
  const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_t) return;
  const uint64_t t = targets[j];
  uint64_t lo = 0, hi = n_reads;  // first read r with offsets[r] >= t (r <= n_reads)
  while (lo < hi) {
    uint64_t mid = (lo + hi) / 2;
    if (offsets[mid] < t) lo = mid + 1; else hi = mid;
  }
  out_read[j] = lo;
  out_off[j] = offsets[lo];
}
}  // namespace

thread_local uint64_t g_launches = 0;

cudaEvent_t StageTimer::get() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
size_t StageTimer::begin(int stage, cudaStream_t st) {
  Rec r{stage, get(), nullptr};
  cudaEventRecord(r.a, st);
  pending.push_back(r);
  return pending.size() - 1;
}
void StageTimer::end(size_t idx, cudaStream_t st) {
  if (idx >= pending.size()) return;
  pending[idx].b = get();
  cudaEventRecord(pending[idx].b, st);
}
void StageTimer::resolve() {
  for (Rec &r : pending) {
    float t = 0;
    if (r.a && r.b && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) ms[r.stage] += t;
    if (r.a) pool.push_back(r.a);
    if (r.b) pool.push_back(r.b);
  }
  pending.clear();
  cudaGetLastError();
}
void StageTimer::clear() {
  resolve();
  for (float &x : ms) x = 0;
  launches = 0;
}
void StageTimer::destroy() {
  resolve();
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
  pool.clear();
}

int cuda_fail(cudaError_t e, const char *what) {
  snprintf(g_last_err, sizeof(g_last_err), "%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return KMC_ENOMEM;
  return KMC_ECUDA;
}

// Allocations left before the injected failure (< 0: none is injected).
std::atomic<int64_t> g_fail_alloc{-1};

bool alloc_fault_injected() {
  int64_t v = g_fail_alloc.load();
  while (v >= 0) {
    if (g_fail_alloc.compare_exchange_weak(v, v - 1)) {
      if (v == 0) {
        snprintf(g_last_err, sizeof(g_last_err), "allocation failed (injected by kmc_debug_fail_alloc)");
        return true;
      }
      return false;
    }
  }
  return false;
}

cudaError_t host_alloc(void **p, size_t bytes, unsigned flags) {
  *p = nullptr;
  if (alloc_fault_injected()) return cudaErrorMemoryAllocation;
  return cudaHostAlloc(p, bytes, flags);
}

int dev_ensure(DevBuf &b, size_t bytes, cudaStream_t st) {
  if (bytes <= b.cap && b.p) return 0;
  if (alloc_fault_injected()) {  // the buffer is left as it is: released by its owner
    return 1;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  if (b.p) cudaFreeAsync(b.p, st);
  b.p = nullptr;
  b.cap = 0;
  size_t want = std::max<size_t>(bytes, 256);
  want = (want + 4095) & ~(size_t)4095;
  cudaMemPool_t pool = pool_for(dev);
  cudaError_t e = pool ? cudaMallocFromPoolAsync(&b.p, want, pool, st) : cudaMallocAsync(&b.p, want, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return 1;
  }
  b.cap = want;
  return 0;
}

void dev_release(DevBuf &b, cudaStream_t st) {
  if (b.p) cudaFreeAsync(b.p, st);
  b.p = nullptr;
  b.cap = 0;
}

int check_device_error(Handle &h) {
  uint32_t e = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&e, h.err.p, 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  if (!e) return KMC_OK;
  KMC_CUDA_TRY(cudaMemsetAsync(h.err.p, 0, 4, h.st));
  if (e & ERR_INPUT) return KMC_EINPUT;
  if (e & ERR_OVERFLOW) return KMC_EOVERFLOW;
  if (e & ERR_TIMEOUT) return KMC_ETIMEOUT;
  snprintf(g_last_err, sizeof(g_last_err), "internal capacity bound exceeded (0x%x)", e);
  return KMC_ECUDA;
}

namespace {

void free_piece(Piece *pc, cudaStream_t st) {
  dev_release(pc->index, st);
  dev_release(pc->words, st);
  if (pc->host) {  // spilled bins: no kernel may still read them
    cudaStreamSynchronize(st);
    cudaFreeHost(pc->host);
    pc->host = nullptr;
  }
  dev_release(pc->rec_base, st);
  dev_release(pc->dbg_list, st);
  dev_release(pc->dbg_read, st);
  dev_release(pc->dbg_rel, st);
  delete pc;
}

void release_all(Handle &h) {
  for (Piece *pc : h.pieces) free_piece(pc, h.st);
  h.pieces.clear();
  h.ds.abm_ready = false;
  DevBuf *bufs[] = {&h.err, &h.map, &h.ds.abm, &h.out_kmers, &h.out_counts, &h.ds.packed, &h.ds.inval,
                    &h.ds.starts, &h.ds.list, &h.ds.counters, &h.ds.hist, &h.ds.scan_tmp,
                    &h.ds.bin_scan, &h.ds.stage_dev[0], &h.ds.stage_dev[1], &h.ds.offs_dev[0],
                    &h.ds.offs_dev[1], &h.ss.hist, &h.ss.bucket_base, &h.ss.cursor, &h.ss.flags,
                    &h.ss.flag_scan, &h.ss.tile_first, &h.ss.scan_tmp, &h.ss.keys, &h.ss.keys_gen, &h.ss.tile_desc,
                    &h.ss.sorted_keys, &h.ss.big_list, &h.ss.big_scratch, &h.ss.sv_keys,
                    &h.ss.sv_counts, &h.ss.acc_keys, &h.ss.acc_counts, &h.ss.counters, &h.ss.o_hist, &h.ss.o_base, &h.ss.o_cursor,
                    &h.ss.o_flags, &h.ss.o_flag_scan, &h.ss.o_tile_first, &h.ss.o_scan_tmp,
                    &h.ss.o_big_list, &h.ss.o_big_k, &h.ss.o_big_v, &h.ds.fq_raw, &h.ds.fq_cnt,
                    &h.ds.fq_base, &h.ds.fq_tmp, &h.ds.fq_small, &h.ds.fq_hdr, &h.ds.fq_bases,
                    &h.ds.fq_offsets};
  for (DevBuf *b : bufs) dev_release(*b, h.st);
  for (int i = 0; i < 2; ++i) {
    if (h.ds.stage_host[i]) cudaFreeHost(h.ds.stage_host[i]);
    h.ds.stage_host[i] = nullptr;
    if (h.ds.stage_free[i]) cudaEventDestroy(h.ds.stage_free[i]);
    h.ds.stage_free[i] = nullptr;
    if (h.ds.copy_done[i]) cudaEventDestroy(h.ds.copy_done[i]);
    if (h.ds.buf_free[i]) cudaEventDestroy(h.ds.buf_free[i]);
    h.ds.copy_done[i] = h.ds.buf_free[i] = nullptr;
  }
  if (h.ss.meta_done) cudaEventSynchronize(h.ss.meta_done);
  if (h.ss.meta_host) cudaFreeHost(h.ss.meta_host);
  h.ss.meta_host = nullptr;
  h.ss.meta_host_cap = 0;
  if (h.ss.meta_done) cudaEventDestroy(h.ss.meta_done);
  h.ss.meta_done = nullptr;
  if (h.ds.go) cudaEventDestroy(h.ds.go);
  h.ds.go = nullptr;
  if (h.ds.copy_st) {
    cudaStreamSynchronize(h.ds.copy_st);
    cudaStreamDestroy(h.ds.copy_st);
  }
  h.ds.copy_st = nullptr;
}

// Returns the handle's device buffers that scale with the input to the
// stream-ordered pool (where any handle of the device can reuse them), keeping
// the small ones and the pinned host staging buffers.  The reads and the
// result are dropped: the handle is as after kmc_reset.
void trim_device(Handle &h) {
  for (Piece *pc : h.pieces) free_piece(pc, h.st);
  h.pieces.clear();
  DevBuf *bufs[] = {&h.out_kmers, &h.out_counts, &h.ds.packed, &h.ds.inval, &h.ds.starts, &h.ds.list,
                    &h.ds.stage_dev[0], &h.ds.stage_dev[1], &h.ds.offs_dev[0], &h.ds.offs_dev[1],
                    &h.ss.keys, &h.ss.keys_gen, &h.ss.sorted_keys, &h.ss.big_scratch, &h.ss.sv_keys,
                    &h.ss.sv_counts, &h.ss.acc_keys, &h.ss.acc_counts, &h.ss.o_big_k, &h.ss.o_big_v,
                    &h.ds.fq_raw, &h.ds.fq_bases, &h.ds.fq_offsets};
  for (DevBuf *b : bufs) dev_release(*b, h.st);
}

int validate(const kmc_params *p) {
  if (!p) return KMC_EINVAL;
  if (p->k < 1 || p->k > KMC_MAX_K) return KMC_EINVAL;
  if (p->m < 1 || p->m > KMC_MAX_M) return KMC_EINVAL;
  if (p->n_bins < 1 || p->n_bins > 65536) return KMC_EINVAL;
  if (p->x != KMC_AUTO && p->x > 3) return KMC_EINVAL;
  if (p->cutoff_min > p->cutoff_max) return KMC_EINVAL;
  if (p->canonical > 1) return KMC_EINVAL;
  if (!p->canonical && p->x != 0 && p->x != KMC_AUTO) return KMC_EINVAL;  // (k,x)-mers are canonical
  if (p->reserved0) return KMC_EINVAL;
  if (p->debug_flags & ~(KMC_DEBUG_KEEP_SUPERKMERS | KMC_DEBUG_KEEP_KEYS | KMC_DEBUG_NARROW_SORT |
                         KMC_DEBUG_SIG_TILE | KMC_DEBUG_MINIMIZER | KMC_DEBUG_WAIT_TIMEOUT))
    return KMC_EINVAL;
  return KMC_OK;
}

// Distributes device-resident reads [0, n) (offsets absolute, offsets[0] ==
// first byte): splits into pieces of about kPieceBytes at read boundaries.
int add_device(Handle &h, const char *d_bases, const uint64_t *d_offsets, uint64_t n_reads,
               uint64_t n_bases, uint64_t read_base) {
  // piece boundaries and the sample end, searched on the device
  const uint64_t kPieceBytes = h.piece_bytes;
  const uint32_t n_p = (uint32_t)((n_bases + kPieceBytes - 1) / kPieceBytes);
  std::vector<uint64_t> targets;
  for (uint32_t j = 1; j < n_p; ++j) targets.push_back((uint64_t)j * kPieceBytes);
  targets.push_back(std::min<uint64_t>(n_bases, kSampleBytes));
  const uint32_t nt = (uint32_t)targets.size();
  if (dev_ensure(h.ds.offs_dev[1], (size_t)nt * 24 + 64, h.st)) return KMC_ENOMEM;
  auto *dt = as<uint64_t>(h.ds.offs_dev[1]);
  KMC_CUDA_TRY(cudaMemcpyAsync(dt, targets.data(), nt * 8, cudaMemcpyHostToDevice, h.st));
  find_bounds_kernel<<<(nt + 127) / 128, 128, 0, h.st>>>(d_offsets, n_reads, dt, nt, dt + nt, dt + 2 * nt); KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  std::vector<uint64_t> res(2 * nt + 2);
  KMC_CUDA_TRY(cudaMemcpyAsync(res.data(), dt + nt, 2 * nt * 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(res.data() + 2 * nt, d_offsets, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(res.data() + 2 * nt + 1, d_offsets + n_reads, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  const uint64_t off0 = res[2 * nt], offn = res[2 * nt + 1];
  if (off0 != 0 || offn != n_bases) return KMC_EINPUT;
  std::vector<uint64_t> rb{0}, ob{0};
  for (uint32_t j = 0; j + 1 < nt; ++j) {
    if (res[j] > rb.back() && res[j] < n_reads) {
      rb.push_back(res[j]);
      ob.push_back(res[nt + j]);
    }
  }
  rb.push_back(n_reads);
  ob.push_back(n_bases);
  if (!h.map_ready) {
    uint64_t s_end = std::min<uint64_t>(std::max<uint64_t>(res[nt - 1], 1), n_reads);
    s_end = std::min<uint64_t>(s_end, kSampleReads);
    if (s_end == 0) s_end = std::min<uint64_t>(n_reads, 1);
    uint64_t s_bytes;
    KMC_CUDA_TRY(cudaMemcpyAsync(&s_bytes, d_offsets + s_end, 8, cudaMemcpyDeviceToHost, h.st));
    KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
    int rc = build_bin_map(h, d_bases, d_offsets, s_end, 0, s_bytes, read_base);
    if (rc) return rc;
  }
  for (size_t p = 0; p + 1 < rb.size(); ++p) {
    const uint64_t r0 = rb[p], r1 = rb[p + 1];
    int rc = distribute_device_piece(h, d_bases + ob[p], d_offsets + r0, r1 - r0, ob[p], ob[p + 1],
                                     read_base + r0);
    if (rc) return rc;
  }
  return KMC_OK;
}

}  // namespace

}  // namespace kmc

namespace kmc {
namespace {
constexpr uint64_t kHostPieceBytes = 256ull << 20;  // pieces of pinned host input

// Pinned host reads: pieces are copied on a copy stream into two device
// buffers in turn, the copy of piece i+1 overlapping the distribution of
// piece i on the handle's stream.
int add_pinned(Handle &h, const char *bases, const uint64_t *offsets, uint64_t n_reads) {
  DistScratch &ds = h.ds;
  const uint64_t piece = std::min<uint64_t>(h.piece_bytes, kHostPieceBytes);
  std::vector<uint64_t> cut{0};
  uint64_t max_nb = 0, max_nr = 0;
  while (cut.back() < n_reads) {
    const uint64_t r0 = cut.back(), b0 = offsets[r0];
    const uint64_t *it = std::upper_bound(offsets + r0 + 1, offsets + n_reads + 1, b0 + piece);
    uint64_t r1 = (uint64_t)(it - offsets) - 1;
    if (r1 <= r0) r1 = r0 + 1;
    if (offsets[r1] < b0) return KMC_EINPUT;
    max_nb = std::max(max_nb, offsets[r1] - b0);
    max_nr = std::max(max_nr, r1 - r0);
    cut.push_back(r1);
  }
  const size_t n_pieces = cut.size() - 1;
  const int n_buf = n_pieces > 1 ? 2 : 1;
  for (int i = 0; i < n_buf; ++i)
    if (dev_ensure(ds.stage_dev[i], max_nb + 64, h.st) || dev_ensure(ds.offs_dev[i], (max_nr + 1) * 8, h.st))
      return KMC_ENOMEM;
  if (!ds.copy_st) {
    KMC_CUDA_TRY(cudaStreamCreateWithFlags(&ds.copy_st, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      KMC_CUDA_TRY(cudaEventCreateWithFlags(&ds.copy_done[i], cudaEventDisableTiming));
      KMC_CUDA_TRY(cudaEventCreateWithFlags(&ds.buf_free[i], cudaEventDisableTiming));
    }
    KMC_CUDA_TRY(cudaEventCreateWithFlags(&ds.go, cudaEventDisableTiming));
  }
  // copies start after everything queued so far (buffer allocations included)
  KMC_CUDA_TRY(cudaEventRecord(ds.go, h.st));
  KMC_CUDA_TRY(cudaStreamWaitEvent(ds.copy_st, ds.go, 0));
  auto copy = [&](size_t i) -> int {
    const int b = (int)(i & 1);
    const uint64_t r0 = cut[i], r1 = cut[i + 1], b0 = offsets[r0];
    if (i >= 2) KMC_CUDA_TRY(cudaStreamWaitEvent(ds.copy_st, ds.buf_free[b], 0));
    KMC_CUDA_TRY(cudaMemcpyAsync(ds.stage_dev[b].p, bases + b0, offsets[r1] - b0, cudaMemcpyHostToDevice,
                                 ds.copy_st));
    KMC_CUDA_TRY(cudaMemcpyAsync(ds.offs_dev[b].p, offsets + r0, (r1 - r0 + 1) * 8, cudaMemcpyHostToDevice,
                                 ds.copy_st));
    KMC_CUDA_TRY(cudaEventRecord(ds.copy_done[b], ds.copy_st));
    return KMC_OK;
  };
  int rc = copy(0);
  if (rc) return rc;
  for (size_t i = 0; i < n_pieces; ++i) {
    if (i + 1 < n_pieces && (rc = copy(i + 1))) return rc;
    const int b = (int)(i & 1);
    KMC_CUDA_TRY(cudaStreamWaitEvent(h.st, ds.copy_done[b], 0));
    const uint64_t r0 = cut[i], r1 = cut[i + 1], nr = r1 - r0, b0 = offsets[r0];
    const char *pbase = static_cast<const char *>(ds.stage_dev[b].p);
    const uint64_t *poff = as<uint64_t>(ds.offs_dev[b]);
    if (!h.map_ready) {
      const uint64_t se = std::min<uint64_t>(nr, kSampleReads);
      if ((rc = build_bin_map(h, pbase, poff, se, b0, offsets[r0 + se], h.stats.n_reads + r0))) return rc;
    }
    if ((rc = distribute_device_piece(h, pbase, poff, nr, b0, offsets[r1], h.stats.n_reads + r0))) return rc;
    KMC_CUDA_TRY(cudaEventRecord(ds.buf_free[b], h.st));
  }
  // later work on the handle's stream may reuse the buffers
  KMC_CUDA_TRY(cudaEventRecord(ds.copy_done[0], ds.copy_st));
  KMC_CUDA_TRY(cudaStreamWaitEvent(h.st, ds.copy_done[0], 0));
  return KMC_OK;
}
}  // namespace
}  // namespace kmc

namespace kmc {
void set_error_text(const char *msg) { snprintf(g_last_err, sizeof(g_last_err), "%s", msg); }
}  // namespace kmc

using namespace kmc;

extern "C" {

void kmc_default_params(kmc_params *p) {
  if (!p) return;
  memset(p, 0, sizeof(*p));
  p->k = 25;
  p->m = 7;
  p->n_bins = 512;
  p->x = KMC_AUTO;
  p->cutoff_min = 2;
  p->cutoff_max = 1000000000ull;
  p->canonical = 1;
  p->device = 0;
  p->cuda_stream = nullptr;
}

const char *kmc_strerror(int code) {
  switch (code) {
    case KMC_OK: return "ok";
    case KMC_EINVAL: return "invalid argument";
    case KMC_ESTATE: return "call out of order";
    case KMC_ENOMEM: return "out of device or pinned host memory";
    case KMC_ECUDA: return g_last_err[0] ? g_last_err : "CUDA error";
    case KMC_EOVERFLOW: return "a count exceeds UINT32_MAX";
    case KMC_ETRUNC: return "output capacity too small";
    case KMC_ETIMEOUT: return "device-side wait timed out";
    case KMC_EAGAIN: return "not ready";
    case KMC_EINPUT: return "malformed read offsets";
    case KMC_EIO: return g_last_err[0] ? g_last_err : "file error";
    case KMC_ECANCELED: return "job cancelled";
    default: return "unknown error";
  }
}

int kmc_debug_fail_alloc(int64_t after) {
  g_fail_alloc.store(after < 0 ? -1 : after);
  return KMC_OK;
}

int kmc_open(kmc_handle **out, const kmc_params *p) {
  if (!out) return KMC_EINVAL;
  *out = nullptr;
  int rc = validate(p);
  if (rc) return rc;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev) {
    cudaGetLastError();
    snprintf(g_last_err, sizeof(g_last_err), "no CUDA device %d", p->device);
    return KMC_ECUDA;
  }
  DeviceGuard g(p->device);
  kmc_handle *kh = new (std::nothrow) kmc_handle();
  if (!kh) return KMC_ENOMEM;
  Handle &h = kh->h;
  h.p = *p;
  h.m_used = std::min(p->m, p->k);
  h.n_sig = (1u << (2 * h.m_used)) + 1u;
  h.key_words = (int)((p->k + 31) / 32);
  h.bin_kmers.assign(p->n_bins, 0);
  h.piece_bytes = p->piece_bytes ? p->piece_bytes : kDefaultPieceBytes;
  if (h.piece_bytes > (1ull << 31)) h.piece_bytes = 1ull << 31;  // stream positions are 32-bit
  if (p->cuda_stream) {
    h.st = static_cast<cudaStream_t>(p->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&h.st, cudaStreamNonBlocking) != cudaSuccess) {
      delete kh;
      return cuda_fail(cudaGetLastError(), "cudaStreamCreate");
    }
    h.own_stream = true;
  }
  cudaDeviceGetAttribute(&h.sm_count, cudaDevAttrMultiProcessorCount, p->device);
  for (auto &e : h.ev) cudaEventCreate(&e);
  if (dev_ensure(h.err, 64, h.st)) {
    kmc_close(kh);
    return KMC_ENOMEM;
  }
  cudaMemsetAsync(h.err.p, 0, 64, h.st);
  *out = kh;
  return KMC_OK;
}

int kmc_set_bin_map(kmc_handle *kh, const uint32_t *map, uint64_t n_entries) {
  if (!kh || !map) return KMC_EINVAL;
  Handle &h = kh->h;
  if (!h.pieces.empty() || h.map_ready) return KMC_ESTATE;
  if (n_entries != h.n_sig) return KMC_EINVAL;
  for (uint64_t i = 0; i < n_entries; ++i)
    if (map[i] >= h.p.n_bins) return KMC_EINVAL;
  DeviceGuard g(h.p.device);
  if (dev_ensure(h.map, n_entries * 4, h.st)) return KMC_ENOMEM;
  KMC_CUDA_TRY(cudaMemcpyAsync(h.map.p, map, n_entries * 4, cudaMemcpyHostToDevice, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  h.map_ready = true;
  h.map_user = true;
  return KMC_OK;
}

int kmc_get_bin_map(const kmc_handle *kh, uint32_t *map, uint64_t n_entries) {
  if (!kh || !map) return KMC_EINVAL;
  const Handle &h = kh->h;
  if (!h.map_ready) return KMC_ESTATE;
  if (n_entries != h.n_sig) return KMC_EINVAL;
  DeviceGuard g(h.p.device);
  KMC_CUDA_TRY(cudaMemcpyAsync(map, h.map.p, n_entries * 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  return KMC_OK;
}

int kmc_add_reads_device(kmc_handle *kh, const char *d_bases, const uint64_t *d_offsets,
                         uint64_t n_reads, uint64_t n_bases) {
  if (!kh) return KMC_EINVAL;
  Handle &h = kh->h;
  if (h.counted) return KMC_ESTATE;
  if (n_reads == 0) return KMC_OK;
  if (!d_offsets || (n_bases && !d_bases)) return KMC_EINVAL;
  DeviceGuard g(h.p.device);
  LaunchScope ls(h);
  KMC_CUDA_TRY(cudaEventRecord(h.ev[0], h.st));
  int rc = add_device(h, d_bases, d_offsets, n_reads, n_bases, h.stats.n_reads);
  if (rc) return rc;
  KMC_CUDA_TRY(cudaEventRecord(h.ev[1], h.st));
  rc = check_device_error(h);
  if (rc) return rc;
  h.timer.resolve();
  float ms = 0;
  cudaEventElapsedTime(&ms, h.ev[0], h.ev[1]);
  h.stats.ms_distribute += ms;
  h.stats.n_reads += n_reads;
  h.stats.n_bases += n_bases;
  return KMC_OK;
}

// FASTQ / FASTA bytes in device memory: parsed on the device into reads,
// then distributed like kmc_add_reads_device.
static int add_file_device(Handle &h, const char *d_bytes, uint64_t n_bytes, uint32_t format) {
  const char *d_bases = nullptr;
  const uint64_t *d_offsets = nullptr;
  uint64_t n_reads = 0, n_bases = 0;
  KMC_CUDA_TRY(cudaEventRecord(h.ev[0], h.st));
  int rc = parse_reads(h, reinterpret_cast<const uint8_t *>(d_bytes), n_bytes, format == KMC_FORMAT_FASTQ,
                       &d_bases, &d_offsets, &n_reads, &n_bases);
  if (rc) return rc;
  if (n_reads == 0) return KMC_OK;
  rc = add_device(h, d_bases, d_offsets, n_reads, n_bases, h.stats.n_reads);
  if (rc) return rc;
  KMC_CUDA_TRY(cudaEventRecord(h.ev[1], h.st));
  rc = check_device_error(h);
  if (rc) return rc;
  h.timer.resolve();
  float ms = 0;
  cudaEventElapsedTime(&ms, h.ev[0], h.ev[1]);
  h.stats.ms_distribute += ms;
  h.stats.n_reads += n_reads;
  h.stats.n_bases += n_bases;
  return KMC_OK;
}

int kmc_add_file_bytes_device(kmc_handle *kh, const char *d_bytes, uint64_t n_bytes, uint32_t format) {
  if (!kh) return KMC_EINVAL;
  Handle &h = kh->h;
  if (h.counted) return KMC_ESTATE;
  if (format != KMC_FORMAT_FASTQ && format != KMC_FORMAT_FASTA) return KMC_EINVAL;
  if (n_bytes == 0) return KMC_OK;
  if (!d_bytes) return KMC_EINVAL;
  DeviceGuard g(h.p.device);
  LaunchScope ls(h);
  return add_file_device(h, d_bytes, n_bytes, format);
}

int kmc_add_file_bytes(kmc_handle *kh, const char *bytes, uint64_t n_bytes, uint32_t format) {
  if (!kh) return KMC_EINVAL;
  Handle &h = kh->h;
  if (h.counted) return KMC_ESTATE;
  if (format != KMC_FORMAT_FASTQ && format != KMC_FORMAT_FASTA) return KMC_EINVAL;
  if (n_bytes == 0) return KMC_OK;
  if (!bytes) return KMC_EINVAL;
  DeviceGuard g(h.p.device);
  LaunchScope ls(h);
  // the raw file goes to the device as it is; nothing is parsed on the host
  if (dev_ensure(h.ds.fq_raw, n_bytes + 64, h.st)) return KMC_ENOMEM;
  KMC_CUDA_TRY(cudaMemcpyAsync(h.ds.fq_raw.p, bytes, n_bytes, cudaMemcpyHostToDevice, h.st));
  return add_file_device(h, static_cast<const char *>(h.ds.fq_raw.p), n_bytes, format);
}

int kmc_add_reads(kmc_handle *kh, const char *bases, const uint64_t *offsets, uint64_t n_reads) {
  if (!kh) return KMC_EINVAL;
  Handle &h = kh->h;
  if (h.counted) return KMC_ESTATE;
  if (n_reads == 0) return KMC_OK;
  if (!offsets) return KMC_EINVAL;
  if (offsets[0] != 0) return KMC_EINPUT;
  // offsets that decrease are found by the device (ERR_INPUT) while the
  // reads are marked; the host only checks the piece bounds it copies by
  const uint64_t n_bases = offsets[n_reads];
  if (n_bases && !bases) return KMC_EINVAL;
  DeviceGuard g(h.p.device);
  LaunchScope ls(h);
  DistScratch &ds = h.ds;
  // stage pieces of about kPieceBytes (bytes + offsets) on the device
  cudaPointerAttributes at{};
  const bool pinned_b = cudaPointerGetAttributes(&at, bases) == cudaSuccess && at.type == cudaMemoryTypeHost;
  cudaGetLastError();
  KMC_CUDA_TRY(cudaEventRecord(h.ev[0], h.st));
  if (pinned_b) {
    int rc = add_pinned(h, bases, offsets, n_reads);
    if (rc) return rc;
  }
  const uint64_t kPieceBytes = h.piece_bytes;
  uint64_t r0 = pinned_b ? n_reads : 0;
  while (r0 < n_reads) {
    // reads [r0, r1) with at most kPieceBytes bytes (at least one read)
    const uint64_t b0 = offsets[r0];
    const uint64_t* it = std::upper_bound(offsets + r0 + 1, offsets + n_reads + 1, b0 + kPieceBytes);
    uint64_t r1 = (uint64_t)(it - offsets) - 1;
    if (r1 <= r0) r1 = r0 + 1;
    const uint64_t b1 = offsets[r1];
    if (b1 < b0) return KMC_EINPUT;
    const uint64_t nb = b1 - b0, nr = r1 - r0;
    if (dev_ensure(ds.stage_dev[0], nb + 64, h.st) || dev_ensure(ds.offs_dev[0], (nr + 1) * 8, h.st))
      return KMC_ENOMEM;
    if (pinned_b) {
      KMC_CUDA_TRY(cudaMemcpyAsync(ds.stage_dev[0].p, bases + b0, nb, cudaMemcpyHostToDevice, h.st));
    } else {
      // copy through a pinned staging buffer in slices
      const size_t slice = 64ull << 20;
      for (int i = 0; i < 2; ++i) {
        if (!ds.stage_host[i]) {
          if (host_alloc(&ds.stage_host[i], slice, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            return KMC_ENOMEM;
          }
          cudaEventCreateWithFlags(&ds.stage_free[i], cudaEventDisableTiming);
          cudaEventRecord(ds.stage_free[i], h.st);
        }
      }
      for (uint64_t o = 0, s = 0; o < nb; o += slice, s ^= 1) {
        const size_t len = (size_t)std::min<uint64_t>(slice, nb - o);
        KMC_CUDA_TRY(cudaEventSynchronize(ds.stage_free[s]));
        memcpy(ds.stage_host[s], bases + b0 + o, len);
        KMC_CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(ds.stage_dev[0].p) + o, ds.stage_host[s], len,
                                     cudaMemcpyHostToDevice, h.st));
        KMC_CUDA_TRY(cudaEventRecord(ds.stage_free[s], h.st));
      }
    }
    KMC_CUDA_TRY(cudaMemcpyAsync(ds.offs_dev[0].p, offsets + r0, (nr + 1) * 8, cudaMemcpyHostToDevice, h.st));
    const char *pbase = static_cast<const char *>(ds.stage_dev[0].p);
    const uint64_t *poff = as<uint64_t>(ds.offs_dev[0]);
    if (!h.map_ready) {
      const uint64_t s_end = std::min<uint64_t>(nr, kSampleReads);
      uint64_t s_bytes = offsets[r0 + s_end] - b0;
      if (s_bytes > kSampleBytes) {
        const uint64_t *jt = std::upper_bound(offsets + r0 + 1, offsets + r0 + s_end + 1, b0 + kSampleBytes);
        uint64_t e = (uint64_t)(jt - offsets) - 1 - r0;
        if (e == 0) e = 1;
        s_bytes = offsets[r0 + e] - b0;
        (void)s_bytes;
      }
      const uint64_t se = std::min<uint64_t>(s_end, nr);
      int rc = build_bin_map(h, pbase, poff, se, b0, offsets[r0 + se], h.stats.n_reads + r0);
      if (rc) return rc;
    }
    int rc = distribute_device_piece(h, pbase, poff, nr, b0, b1, h.stats.n_reads + r0);
    if (rc) return rc;
    r0 = r1;
  }
  KMC_CUDA_TRY(cudaEventRecord(h.ev[1], h.st));
  int rc = check_device_error(h);
  if (rc) return rc;
  h.timer.resolve();
  float ms = 0;
  cudaEventElapsedTime(&ms, h.ev[0], h.ev[1]);
  h.stats.ms_distribute += ms;
  h.stats.n_reads += n_reads;
  h.stats.n_bases += n_bases;
  return KMC_OK;
}

int kmc_count(kmc_handle *kh) {
  if (!kh) return KMC_EINVAL;
  Handle &h = kh->h;
  DeviceGuard g(h.p.device);
  LaunchScope ls(h);
  KMC_CUDA_TRY(cudaEventRecord(h.ev[3], h.st));
  h.counted = false;
  if (h.stats.n_kmer_positions == 0) {
    h.n_out = 0;
    h.stats.n_out = 0;
    h.stats.n_distinct = 0;
    h.counted = true;
    return KMC_OK;
  }
  int rc = sort_phase(h);
  if (rc) return rc;
  KMC_CUDA_TRY(cudaEventRecord(h.ev[4], h.st));
  KMC_CUDA_TRY(cudaEventSynchronize(h.ev[4]));
  float ms = 0;
  cudaEventElapsedTime(&ms, h.ev[3], h.ev[4]);
  h.stats.ms_total = ms;
  cudaEventElapsedTime(&ms, h.ev[3], h.ev[2]);
  h.stats.ms_sort = ms;
  cudaEventElapsedTime(&ms, h.ev[2], h.ev[4]);
  h.stats.ms_order = ms;
  h.timer.resolve();
  h.counted = true;
  return KMC_OK;
}

int kmc_result_size(const kmc_handle *kh, uint64_t *n) {
  if (!kh || !n) return KMC_EINVAL;
  if (!kh->h.counted) return KMC_ESTATE;
  *n = kh->h.n_out;
  return KMC_OK;
}

int kmc_result(kmc_handle *kh, uint64_t *kmers, uint32_t *counts, uint64_t capacity, uint64_t *n_out) {
  if (!kh) return KMC_EINVAL;
  Handle &h = kh->h;
  if (!h.counted) return KMC_ESTATE;
  if (n_out) *n_out = h.n_out;
  if (capacity < h.n_out) return KMC_ETRUNC;
  if (h.n_out == 0) return KMC_OK;
  DeviceGuard g(h.p.device);
  if (kmers)
    KMC_CUDA_TRY(cudaMemcpyAsync(kmers, h.out_kmers.p, h.n_out * 8 * h.key_words, cudaMemcpyDeviceToHost, h.st));
  if (counts)
    KMC_CUDA_TRY(cudaMemcpyAsync(counts, h.out_counts.p, h.n_out * 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  return KMC_OK;
}

int kmc_result_device(kmc_handle *kh, const uint64_t **d_kmers, const uint32_t **d_counts, uint64_t *n) {
  if (!kh) return KMC_EINVAL;
  Handle &h = kh->h;
  if (!h.counted) return KMC_ESTATE;
  if (d_kmers) *d_kmers = static_cast<const uint64_t *>(h.out_kmers.p);
  if (d_counts) *d_counts = static_cast<const uint32_t *>(h.out_counts.p);
  if (n) *n = h.n_out;
  return KMC_OK;
}

int kmc_stats_get(const kmc_handle *kh, kmc_stats *s) {
  if (!kh || !s) return KMC_EINVAL;
  *s = kh->h.stats;
  s->m_used = kh->h.m_used;
  for (int i = 0; i < KMC_N_STAGES && i < 12; ++i) s->ms_stage[i] = kh->h.timer.ms[i];
  s->n_launches = kh->h.timer.launches;
  return KMC_OK;
}

int kmc_reset(kmc_handle *kh) {
  if (!kh) return KMC_EINVAL;
  Handle &h = kh->h;
  DeviceGuard g(h.p.device);
  for (Piece *pc : h.pieces) free_piece(pc, h.st);
  h.pieces.clear();
  h.counted = false;
  h.n_out = 0;
  std::fill(h.bin_kmers.begin(), h.bin_kmers.end(), 0);
  h.stats = kmc_stats{};
  h.dev_bin_bytes = 0;
  h.timer.clear();
  if (!h.map_user) h.map_ready = false;
  return KMC_OK;
}

}  // extern "C"

namespace kmc {
int handle_trim(kmc_handle *kh) {
  if (!kh) return KMC_EINVAL;
  DeviceGuard g(kh->h.p.device);
  const int rc = kmc_reset(kh);
  trim_device(kh->h);
  return rc;
}
}  // namespace kmc

extern "C" {

void kmc_close(kmc_handle *kh) {
  if (!kh) return;
  Handle &h = kh->h;
  {
    DeviceGuard g(h.p.device);
    release_all(h);
    cudaStreamSynchronize(h.st);
    h.timer.destroy();
    for (auto &e : h.ev)
      if (e) cudaEventDestroy(e);
    if (h.own_stream) cudaStreamDestroy(h.st);
  }
  delete kh;
}

int kmc_debug_superkmers(kmc_handle *kh, uint64_t *read_index, uint32_t *pos, uint32_t *n_kmers,
                         uint32_t *sig, uint64_t capacity, uint64_t *n_out) {
  if (!kh || !n_out) return KMC_EINVAL;
  DeviceGuard g(kh->h.p.device);
  return debug_superkmers(kh->h, read_index, pos, n_kmers, sig, capacity, n_out);
}

int kmc_debug_bin_keys(kmc_handle *kh, uint32_t bin, uint64_t *keys, uint64_t capacity,
                       uint64_t *n_out, uint32_t *words_per_key) {
  if (!kh || !n_out) return KMC_EINVAL;
  if (bin >= kh->h.p.n_bins) return KMC_EINVAL;
  if (!kh->h.counted) return KMC_ESTATE;
  DeviceGuard g(kh->h.p.device);
  return debug_bin_keys(kh->h, bin, keys, capacity, n_out, words_per_key);
}

}  // extern "C"
