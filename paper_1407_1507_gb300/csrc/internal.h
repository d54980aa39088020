// Host-side internals shared by the translation units of libkmc.
#pragma once
#include <memory>
#include <atomic>
#include <cstdint>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/kmc.h"

namespace kmc {

int cuda_fail(cudaError_t e, const char *what);
void set_error_text(const char *msg);  // the text kmc_strerror gives for KMC_EIO

// "Done once" per CUDA device: kernel attributes (shared-memory limits) are
// per device, so a process that uses several devices sets them on each.
struct DeviceOnce {
  std::atomic<uint64_t> mask{0};
  static int dev() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
  }
  bool done() const {
    const int d = dev();
    return d < 64 && ((mask.load() >> d) & 1ull);
  }
  void set() {
    const int d = dev();
    if (d < 64) mask.fetch_or(1ull << d);
  }
};

// Restores the caller's current device on scope exit.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};
extern thread_local uint64_t g_launches;

// Stream-ordered device buffer that only grows (reused across calls).
struct DevBuf {
  void *p = nullptr;
  size_t cap = 0;
};
int dev_ensure(DevBuf &b, size_t bytes, cudaStream_t st);
// Pinned host allocation (cudaHostAlloc) through the allocation-failure hook
// of kmc_debug_fail_alloc; returns cudaErrorMemoryAllocation when the hook
// fires.
cudaError_t host_alloc(void **p, size_t bytes, unsigned flags);
// True (once) when kmc_debug_fail_alloc asked this allocation to fail.
bool alloc_fault_injected();
void dev_release(DevBuf &b, cudaStream_t st);

template <typename T>
inline T *as(DevBuf &b) { return static_cast<T *>(b.p); }

// One piece of input after the distribution phase: its super k-mer records,
// grouped by bin.  index[i] = word offset (bits 63..32) | n_kmers-1 (bits
// 31..25) | signature (bits 24..0); words = packed bases of the records.
struct Piece {
  DevBuf index;        // uint64[n_records]
  DevBuf words;        // uint64[n_words + pad]
  // where kernels read the bins: index/words above, or (spilled) a pinned
  // host copy, mapped into the device's address space
  const uint64_t *d_index = nullptr, *d_words = nullptr;
  void *host = nullptr;  // the pinned host copy (index, then words)
  DevBuf rec_base;     // uint64[B+1]: first record of each bin
  std::vector<uint64_t> rec_base_host;
  uint64_t n_records = 0;
  uint64_t n_words = 0;
  uint64_t n_kmers = 0;
  // kept only with KMC_DEBUG_KEEP_SUPERKMERS: the raw super k-mer list
  DevBuf dbg_list;     // uint64[n_records]: stream position (hi 32) | n_sig (lo 32)
  DevBuf dbg_read;     // uint64[n_records]: read index
  DevBuf dbg_rel;      // uint32[n_records]: position in read
};

// Per-call scratch of the distribution phase (reused).
struct DistScratch {
  DevBuf packed, inval, starts;  // bit streams of the current piece
  DevBuf abm;                    // allowed m-mers (Sect. 2.2), one bit each, built once
  bool abm_ready = false;
  DevBuf list;                   // uint64 super k-mer list
  DevBuf counters;               // device counters
  DevBuf hist;                   // per-bin histograms (records, words, kmers)
  DevBuf scan_tmp, bin_scan;
  DevBuf stage_dev[2];           // device staging of host reads
  DevBuf offs_dev[2];
  void *stage_host[2] = {nullptr, nullptr};
  size_t stage_host_cap[2] = {0, 0};
  cudaEvent_t stage_free[2] = {nullptr, nullptr};
  // pinned host input: pieces are copied on their own stream, one ahead of
  // the piece being distributed
  cudaStream_t copy_st = nullptr;
  cudaEvent_t copy_done[2] = {nullptr, nullptr}, buf_free[2] = {nullptr, nullptr}, go = nullptr;
  // FASTQ / FASTA input: the raw file (host input), per-chunk counts and
  // their scans, header flags per line, the reads' bases and offsets
  DevBuf fq_raw, fq_cnt, fq_base, fq_tmp, fq_small, fq_hdr, fq_bases, fq_offsets;
};

// Per-call scratch of the sorting phase.
struct SortScratch {
  DevBuf hist, bucket_base, cursor, flags, flag_scan, tile_first, scan_tmp;
  DevBuf keys, keys_gen, sorted_keys, big_list, big_scratch, tile_desc;
  DevBuf sv_keys, sv_counts;  // survivors before global order
  DevBuf acc_keys, acc_counts;  // survivors of all waves (sort in waves)
  DevBuf counters;
  // global-order pass
  DevBuf o_hist, o_base, o_cursor, o_flags, o_flag_scan, o_tile_first, o_scan_tmp, o_big_list,
      o_big_k, o_big_v;
  // second level of the (k,x)-mer path: expanded, weighted k-mers
  DevBuf l2_hist, l2_base, l2_flags, l2_fscan, l2_tfirst, l2_tmp, l2_keys, l2_wts, l2_big,
      l2_big_k, l2_big_v, l2_grp, l2_counters, l2_out_keys, l2_out_counts;
  // pinned staging of the sort metadata (chunks, units, bin tables)
  void *meta_host = nullptr;
  size_t meta_host_cap = 0;
  cudaEvent_t meta_done = nullptr;
  // what kmc_debug_bin_keys needs to find and decode one bin's keys
  std::vector<uint32_t> dbg_group_base;
  int dbg_key_bytes = 0;
  uint64_t dbg_mix[8] = {};  // c lo/hi, cinv lo/hi, mask lo/hi, bits | s1 << 16 | s2 << 32
};

// Device time per stage: events recorded around launches on the handle's
// stream, resolved after the stream has been synchronised.
struct StageTimer {
  struct Rec { int stage; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  float ms[KMC_N_STAGES] = {};
  uint64_t launches = 0;
  cudaEvent_t get();
  size_t begin(int stage, cudaStream_t st);
  void end(size_t idx, cudaStream_t st);
  void resolve();   // call after a stream synchronise
  void destroy();
  void clear();
};

struct Handle {
  kmc_params p{};
  uint32_t m_used = 0;
  uint64_t piece_bytes = 0;
  uint32_t n_sig = 0;          // 4^m_used + 1 signatures (the last is "none")
  int key_words = 1;           // 64-bit words per k-mer in the result
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int sm_count = 0;
  DevBuf err;                  // uint32 device error word
  DevBuf map;                  // uint32[n_sig] signature -> bin
  bool map_ready = false;
  bool map_user = false;
  std::vector<Piece *> pieces;
  DistScratch ds;
  SortScratch ss;
  // result
  DevBuf out_kmers, out_counts;
  uint64_t n_out = 0;
  bool counted = false;
  // statistics
  kmc_stats stats{};
  std::vector<uint64_t> bin_kmers;   // k-mer positions per bin (all pieces)
  uint64_t dev_bin_bytes = 0;        // bin bytes of the pieces kept on the device
  cudaEvent_t ev[8] = {};
  StageTimer timer;
};

// Brackets a launch: STAGE(h, KMC_STAGE_X) { kernel<<<...>>>(...); }
struct StageScope {
  Handle &h;
  size_t idx;
  StageScope(Handle &hh, int stage) : h(hh), idx(hh.timer.begin(stage, hh.st)) {}
  ~StageScope() { h.timer.end(idx, h.st); }
};

// Adds the kernels launched by this thread during a call to the handle.
struct LaunchScope {
  Handle &h;
  uint64_t l0;
  explicit LaunchScope(Handle &hh) : h(hh), l0(g_launches) {}
  ~LaunchScope() { h.timer.launches += g_launches - l0; }
};

// parse.cu: FASTQ / FASTA bytes in device memory -> reads (handle scratch)
int parse_reads(Handle &h, const uint8_t *d_raw, uint64_t n, bool fastq, const char **d_bases,
                const uint64_t **d_offsets, uint64_t *n_reads, uint64_t *n_bases);

// distribute.cu
int distribute_device_piece(Handle &h, const char *piece_ptr, const uint64_t *d_offsets,
                            uint64_t n_reads, uint64_t byte_start, uint64_t byte_end,
                            uint64_t read_base);
int build_bin_map(Handle &h, const char *piece_ptr, const uint64_t *d_offsets, uint64_t n_reads,
                  uint64_t byte_start, uint64_t byte_end, uint64_t read_base);
int debug_superkmers(Handle &h, uint64_t *read_index, uint32_t *pos, uint32_t *n_kmers,
                     uint32_t *sig, uint64_t capacity, uint64_t *n_out);

// count.cu
int sort_phase(Handle &h);
int debug_bin_keys(Handle &h, uint32_t bin, uint64_t *keys, uint64_t capacity, uint64_t *n_out,
                   uint32_t *words_per_key);

// order.cu: sort (key, value) pairs in place by key bits [0, key_bits)
// Read sets of at least this many bases are counted on the single-set path
// by the batch and server calls (the batch engine builds every key twice and
// pays for itself only while per-set launches and host steps dominate, i.e.
// for sets of a few MB).
constexpr uint64_t kSingleMinBases = 4ull << 20;
// Open single-set handles of the batch and server calls give their
// input-sized device buffers back to the pool after a set of at least this
// many bases (smaller sets leave them for the next set).
constexpr uint64_t kTrimMinBases = 256ull << 20;

// One set's result of a batch run, in host memory.
struct BatchSetResult {
  std::unique_ptr<uint64_t[]> k;
  std::unique_ptr<uint32_t[]> c;
  uint64_t n = 0;
};
// kmc_reset, and the handle's input-sized device buffers go back to the
// stream-ordered pool (for handles kept open between large jobs).
int handle_trim(kmc_handle *kh);
// Copies set `set`'s result out of the batch handle.
int batch_take_result(kmc_batch *b, uint32_t set, BatchSetResult *out);

int sort_pairs_u64(Handle &h, uint64_t *keys, uint32_t *vals, uint64_t n, int key_bits);
int sort_pairs_u128(Handle &h, unsigned __int128 *keys, uint32_t *vals, uint64_t n, int key_bits);
// Out of place: the sorted pairs go to (out_k, out_v); the input arrays are
// used as scratch and left unspecified.
int sort_pairs_to_u64(Handle &h, uint64_t *keys, uint32_t *vals, uint64_t n, int key_bits, uint64_t *out_k,
                      uint32_t *out_v);
int sort_pairs_to_u128(Handle &h, unsigned __int128 *keys, uint32_t *vals, uint64_t n, int key_bits,
                       unsigned __int128 *out_k, uint32_t *out_v);

int check_device_error(Handle &h);

}  // namespace kmc

// The object behind the C ABI's kmc_handle.
struct kmc_handle {
  kmc::Handle h;
};
