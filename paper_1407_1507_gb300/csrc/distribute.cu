// Distribution phase (paper Sect. 2.4, Fig. 1, Fig. 3): reads -> 2-bit
// stream -> signatures of every k-mer (Sect. 2.2) -> super k-mers -> bins.
//
// A piece of input is a run of whole reads.  Its bytes are viewed as a
// "stream" starting at the 16-byte aligned address at or before the first
// read, so stream position q is byte (aligned + q); the `mis` bytes before
// the first read are marked invalid.
#include <algorithm>
#include <cstdio>

#include "internal.h"
#include "sortlib.cuh"
#include "dist_kernels.cuh"

namespace kmc {

namespace {

inline unsigned grid_for(uint64_t n, int threads, int cap = 1 << 20) {
  uint64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (unsigned)std::min<uint64_t>(g, (uint64_t)cap);
}

// Stages a piece: pack + read starts.  Returns stream length etc.
struct StreamInfo {
  const uint8_t *aligned;
  uint32_t mis;
  uint64_t n_stream, n_mwords, n_pwords;
};

int stage_stream(Handle &h, const char *piece_ptr, const uint64_t *d_offsets, uint64_t n_reads,
                 uint64_t byte_start, uint64_t byte_end, StreamInfo *si) {
  DistScratch &ds = h.ds;
  const uintptr_t ptr = reinterpret_cast<uintptr_t>(piece_ptr);
  si->mis = (uint32_t)(ptr & 15u);
  si->aligned = reinterpret_cast<const uint8_t *>(ptr - si->mis);
  si->n_stream = si->mis + (byte_end - byte_start);
  si->n_mwords = (si->n_stream + 63) / 64 + STREAM_PAD_WORDS;
  si->n_pwords = 2 * si->n_mwords;
  if (dev_ensure(ds.packed, si->n_pwords * 8, h.st) || dev_ensure(ds.inval, si->n_mwords * 8, h.st) ||
      dev_ensure(ds.starts, si->n_mwords * 8, h.st))
    return KMC_ENOMEM;
  StageScope sc(h, KMC_STAGE_PACK);
  KMC_CUDA_TRY(cudaMemsetAsync(ds.starts.p, 0, si->n_mwords * 8, h.st));
  pack_kernel<<<grid_for(si->n_mwords, PACK_THREADS, 1 << 30), PACK_THREADS, 0, h.st>>>(
      si->aligned, si->n_stream, si->mis, as<uint64_t>(ds.packed), as<uint64_t>(ds.inval),
      si->n_mwords); KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  if (n_reads) {
    starts_kernel<<<grid_for(n_reads, 256, 65535), 256, 0, h.st>>>(
        d_offsets, 0, n_reads, byte_start, si->mis, si->n_stream,
        as<unsigned long long>(ds.starts), as<uint32_t>(h.err)); KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  return KMC_OK;
}

SigArgs sig_args(Handle &h, const StreamInfo &si, const uint64_t *d_offsets, uint64_t n_reads,
                 uint64_t byte_start) {
  SigArgs a{};
  a.no_filter = (h.p.debug_flags & KMC_DEBUG_MINIMIZER) ? 1u : 0u;
  a.packed = as<uint64_t>(h.ds.packed);
  a.inval = as<uint64_t>(h.ds.inval);
  a.smask = as<uint64_t>(h.ds.starts);
  a.n_pwords = si.n_pwords;
  a.n_mwords = si.n_mwords;
  a.n_stream = si.n_stream;
  a.offsets = d_offsets;
  a.r0 = 0;
  a.r1 = n_reads;
  a.byte_start = byte_start;
  a.mis = si.mis;
  a.k = (int)h.p.k;
  a.m = (int)h.m_used;
  a.map = as<uint32_t>(h.map);
  a.n_bins = h.p.n_bins;
  a.err = as<uint32_t>(h.err);
  a.abm = h.ds.abm_ready ? as<uint32_t>(h.ds.abm) : nullptr;
  a.n_stream_dyn = nullptr;
  a.n_reads_dyn = nullptr;
  a.set_starts = nullptr;
  a.n_slots = 1;
  a.bins_per_slot = 0;
  return a;
}

int launch_sig(Handle &h, const SigArgs &a0, uint64_t n_stream, int stage) {
  KMC_CUDA_TRY(sig_prepare());
  if (n_stream == 0) return KMC_OK;
  SigArgs a = a0;
  if (!h.ds.abm_ready) {
    if (dev_ensure(h.ds.abm, (size_t)mmer_bm_words(a.m) * 4, h.st)) return KMC_ENOMEM;
    KMC_CUDA_TRY(build_mmer_bm(as<uint32_t>(h.ds.abm), a.m, h.st));
    KMC_COUNT_LAUNCH();
    h.ds.abm_ready = true;
  }
  a.abm = as<uint32_t>(h.ds.abm);
  StageScope sc(h, stage);
  if (sig_launch(a, n_stream, (h.p.debug_flags & KMC_DEBUG_SIG_TILE) != 0, h.st)) KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  return KMC_OK;
}

}  // namespace

// Sect. 2.4: "in a preprocessing stage KMC 2 reads a small fraction of the
// input data, builds a histogram of found signatures, and finally merges the
// least frequent signatures".  Sample = the n_reads reads given (the caller
// passes at most 2^20 reads of its first call).
int build_bin_map(Handle &h, const char *piece_ptr, const uint64_t *d_offsets, uint64_t n_reads,
                  uint64_t byte_start, uint64_t byte_end, uint64_t read_base) {
  (void)read_base;
  const uint32_t n_sig = h.n_sig;
  if (dev_ensure(h.map, (size_t)n_sig * 4, h.st)) return KMC_ENOMEM;
  DistScratch &ds = h.ds;
  // scratch: weights (u64), keys (u64) x2, vals (u32) x2, prefix (u64)
  const size_t need = (size_t)n_sig * 8 * 5 + 64;
  if (dev_ensure(ds.hist, need, h.st)) return KMC_ENOMEM;
  auto *wt = as<unsigned long long>(ds.hist);
  auto *keys = reinterpret_cast<uint64_t *>(wt + n_sig);
  auto *keys2 = keys + n_sig;
  auto *pref = keys2 + n_sig;
  auto *vals = reinterpret_cast<uint32_t *>(pref + n_sig + 1);
  auto *vals2 = vals + n_sig;
  KMC_CUDA_TRY(cudaMemsetAsync(wt, 0, (size_t)n_sig * 8, h.st));
  StreamInfo si;
  int rc = stage_stream(h, piece_ptr, d_offsets, n_reads, byte_start, byte_end, &si);
  if (rc) return rc;
  SigArgs a = sig_args(h, si, d_offsets, n_reads, byte_start);
  a.sig_weight = wt;
  a.map = nullptr;
  rc = launch_sig(h, a, si.n_stream, KMC_STAGE_BIN_MAP);
  if (rc) return rc;
  StageScope sc(h, KMC_STAGE_BIN_MAP);
  if (n_sig <= MAP_DIRECT_MAX) {
    // keys/keys2 hold the preceding weights and the total
    auto *before = reinterpret_cast<unsigned long long *>(keys);
    auto *total = reinterpret_cast<unsigned long long *>(keys2);
    KMC_CUDA_TRY(cudaMemsetAsync(before, 0, (size_t)n_sig * 8 + 8, h.st));
    map_prefix_kernel<<<dim3((n_sig + 255) / 256, MAP_DIRECT_SLICES), 256, 0, h.st>>>(wt, n_sig, before, total);
    KMC_COUNT_LAUNCH();
    map_direct_assign_kernel<<<grid_for(n_sig, 256, 4096), 256, 0, h.st>>>(wt, before, total, n_sig, h.p.n_bins,
                                                                          as<uint32_t>(h.map));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
    h.map_ready = true;
    return KMC_OK;
  }
  map_keys_kernel<<<grid_for(n_sig, 256, 4096), 256, 0, h.st>>>(wt, n_sig, keys, vals); KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  rc = sort_pairs_u64(h, keys, vals, n_sig, 56);
  if (rc) return rc;
  (void)keys2;
  (void)vals2;
  map_weights_kernel<<<grid_for(n_sig, 256, 4096), 256, 0, h.st>>>(keys, n_sig,
                                                                   reinterpret_cast<uint64_t *>(wt)); KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  if (dev_ensure(ds.scan_tmp, scan_tmp_words(n_sig) * 8, h.st)) return KMC_ENOMEM;
  KMC_CUDA_TRY(device_excl_scan_u64(reinterpret_cast<uint64_t *>(wt), pref, n_sig,
                                    as<uint64_t>(ds.scan_tmp), h.st));
  map_assign_kernel<<<grid_for(n_sig, 256, 4096), 256, 0, h.st>>>(keys, pref, n_sig, h.p.n_bins,
                                                                  as<uint32_t>(h.map)); KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  h.map_ready = true;
  return KMC_OK;
}

// Distributes n_reads reads into a new piece of bins.  piece_ptr is the
// device address of the first read's first byte; d_offsets[0..n_reads] are
// the reads' offsets (absolute: d_offsets[0] == byte_start); read_base is the
// global index of the first read (for inspection).
int distribute_device_piece(Handle &h, const char *piece_ptr, const uint64_t *d_offsets,
                            uint64_t n_reads, uint64_t byte_start, uint64_t byte_end,
                            uint64_t read_base) {
  DistScratch &ds = h.ds;
  const uint32_t B = h.p.n_bins;
  StreamInfo si;
  int rc = stage_stream(h, piece_ptr, d_offsets, n_reads, byte_start, byte_end, &si);
  if (rc) return rc;
  // list capacity: at most one super k-mer per k-mer position
  const uint64_t list_cap = si.n_stream + 1;
  if (dev_ensure(ds.list, list_cap * 8, h.st)) return KMC_ENOMEM;
  // counters: [0] n_list; hist: rec[B], words[B], kmers[B]; bases for scans
  if (dev_ensure(ds.counters, 64, h.st)) return KMC_ENOMEM;
  if (dev_ensure(ds.hist, (size_t)B * 8 * 3, h.st)) return KMC_ENOMEM;
  auto *cnt = as<unsigned long long>(ds.counters);
  auto *h_rec = as<unsigned long long>(ds.hist);
  auto *h_words = h_rec + B;
  auto *h_kmers = h_words + B;
  KMC_CUDA_TRY(cudaMemsetAsync(cnt, 0, 64, h.st));
  KMC_CUDA_TRY(cudaMemsetAsync(h_rec, 0, (size_t)B * 8 * 3, h.st));
  SigArgs a = sig_args(h, si, d_offsets, n_reads, byte_start);
  a.list = as<uint64_t>(ds.list);
  a.n_list = cnt;
  a.list_cap = list_cap;
  a.bin_rec = h_rec;
  a.bin_words = h_words;
  a.bin_kmers = h_kmers;
  rc = launch_sig(h, a, si.n_stream, KMC_STAGE_SIGNATURE);
  if (rc) return rc;
  // bin bases (exclusive scans) and cursors
  if (dev_ensure(ds.bin_scan, ((size_t)B + 1) * 8 * 2, h.st)) return KMC_ENOMEM;
  if (dev_ensure(ds.scan_tmp, scan_tmp_words(B) * 8, h.st)) return KMC_ENOMEM;
  auto *rec_base = as<uint64_t>(ds.bin_scan);
  auto *word_base = rec_base + B + 1;
  KMC_CUDA_TRY(device_excl_scan_u64(reinterpret_cast<uint64_t *>(h_rec), rec_base, B,
                                    as<uint64_t>(ds.scan_tmp), h.st));
  KMC_CUDA_TRY(device_excl_scan_u64(reinterpret_cast<uint64_t *>(h_words), word_base, B,
                                    as<uint64_t>(ds.scan_tmp), h.st));
  // read back sizes: n_list, total words, per-bin k-mers (host keeps the maximum)
  std::vector<unsigned long long> hk(B);
  std::vector<uint64_t> rbh(B + 1);
  uint64_t tot[2];
  KMC_CUDA_TRY(cudaMemcpyAsync(&tot[0], cnt, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(&tot[1], word_base + B, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(hk.data(), h_kmers, (size_t)B * 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(rbh.data(), rec_base, ((size_t)B + 1) * 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  rc = check_device_error(h);
  if (rc) return rc;
  const uint64_t n_rec = tot[0], n_words = tot[1];
  Piece *pc = new Piece();
  pc->rec_base_host = std::move(rbh);
  pc->n_records = n_rec;
  pc->n_words = n_words;
  for (uint32_t b = 0; b < B; ++b) {
    h.bin_kmers[b] += hk[b];
    pc->n_kmers += hk[b];
    if (h.bin_kmers[b] > h.stats.max_bin_kmers) h.stats.max_bin_kmers = h.bin_kmers[b];
  }
  if (dev_ensure(pc->index, (n_rec + 1) * 8, h.st) ||
      dev_ensure(pc->words, (n_words + STREAM_PAD_WORDS) * 8, h.st) ||
      dev_ensure(pc->rec_base, ((size_t)B + 1) * 8, h.st)) {
    delete pc;
    return KMC_ENOMEM;
  }
  h.pieces.push_back(pc);
  KMC_CUDA_TRY(cudaMemcpyAsync(pc->rec_base.p, rec_base, ((size_t)B + 1) * 8,
                               cudaMemcpyDeviceToDevice, h.st));
  KMC_CUDA_TRY(cudaMemsetAsync(static_cast<uint64_t *>(pc->words.p) + n_words, 0,
                               STREAM_PAD_WORDS * 8, h.st));
  // cursors start at the bin bases (reuse the histogram arrays)
  KMC_CUDA_TRY(cudaMemcpyAsync(h_rec, rec_base, (size_t)B * 8, cudaMemcpyDeviceToDevice, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(h_words, word_base, (size_t)B * 8, cudaMemcpyDeviceToDevice, h.st));
  if (n_rec) {
    static DeviceOnce attr_set;
    if (!attr_set.done()) {
      KMC_CUDA_TRY(cudaFuncSetAttribute(scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)scat_smem_bytes(SIG_SMEM_BINS)));
      attr_set.set();
    }
    StageScope sc(h, KMC_STAGE_BIN_SCATTER);
    scatter_kernel<<<(unsigned)((n_rec + SCAT_PER_CTA - 1) / SCAT_PER_CTA), SCAT_THREADS,
                     scat_smem_bytes(B), h.st>>>(as<uint64_t>(ds.list), n_rec, as<uint32_t>(h.map), B,
                                               (int)h.p.k, as<uint64_t>(ds.packed), h_rec, h_words,
                                               static_cast<uint64_t *>(pc->index.p),
                                               static_cast<uint64_t *>(pc->words.p)); KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  if (h.p.debug_flags & KMC_DEBUG_KEEP_SUPERKMERS) {
    if (dev_ensure(pc->dbg_list, (n_rec + 1) * 8, h.st) || dev_ensure(pc->dbg_read, (n_rec + 1) * 8, h.st) ||
        dev_ensure(pc->dbg_rel, (n_rec + 1) * 4, h.st))
      return KMC_ENOMEM;
    KMC_CUDA_TRY(cudaMemcpyAsync(pc->dbg_list.p, ds.list.p, n_rec * 8, cudaMemcpyDeviceToDevice, h.st));
    if (n_rec) {
      dbg_locate_kernel<<<grid_for(n_rec, 256, 65535), 256, 0, h.st>>>(
          as<uint64_t>(pc->dbg_list), n_rec, d_offsets, 0, n_reads, byte_start, si.mis,
          read_base, as<uint64_t>(pc->dbg_read), as<uint32_t>(pc->dbg_rel)); KMC_COUNT_LAUNCH();
      KMC_CUDA_TRY(cudaGetLastError());
    }
  }
  pc->d_index = static_cast<const uint64_t *>(pc->index.p);
  pc->d_words = static_cast<const uint64_t *>(pc->words.p);
  const uint64_t bytes = (n_rec + 1 + n_words + STREAM_PAD_WORDS) * 8;
  if (h.p.device_budget && h.dev_bin_bytes + bytes > h.p.device_budget / 2) {
    // over the device share of the budget: the bins go to pinned host memory
    // (copied after the scatter on this stream), the sort reads them there
    void *host = nullptr;
    if (host_alloc(&host, bytes, cudaHostAllocMapped) != cudaSuccess) {
      cudaGetLastError();
      return KMC_ENOMEM;
    }
    pc->host = host;
    uint64_t *hi = static_cast<uint64_t *>(host), *hw = hi + n_rec + 1;
    KMC_CUDA_TRY(cudaMemcpyAsync(hi, pc->index.p, (n_rec + 1) * 8, cudaMemcpyDeviceToHost, h.st));
    KMC_CUDA_TRY(cudaMemcpyAsync(hw, pc->words.p, (n_words + STREAM_PAD_WORDS) * 8, cudaMemcpyDeviceToHost,
                                 h.st));
    void *dp = nullptr;
    KMC_CUDA_TRY(cudaHostGetDevicePointer(&dp, host, 0));
    pc->d_index = static_cast<const uint64_t *>(dp);
    pc->d_words = static_cast<const uint64_t *>(dp) + n_rec + 1;
    dev_release(pc->index, h.st);  // stream-ordered: after the copies
    dev_release(pc->words, h.st);
    h.stats.spilled_bytes += bytes;
  } else {
    h.dev_bin_bytes += bytes;
  }
  h.stats.n_superkmers += n_rec;
  h.stats.n_kmer_positions += pc->n_kmers;
  h.stats.bin_bytes += (n_words + n_rec) * 8;
  return KMC_OK;
}

int debug_superkmers(Handle &h, uint64_t *read_index, uint32_t *pos, uint32_t *n_kmers,
                     uint32_t *sig, uint64_t capacity, uint64_t *n_out) {
  if (!(h.p.debug_flags & KMC_DEBUG_KEEP_SUPERKMERS)) return KMC_ESTATE;
  uint64_t n = 0;
  for (Piece *pc : h.pieces) n += pc->n_records;
  *n_out = n;
  if (capacity < n) return KMC_ETRUNC;
  uint64_t o = 0;
  for (Piece *pc : h.pieces) {
    const uint64_t r = pc->n_records;
    if (!r) continue;
    std::vector<uint64_t> lst(r), rd(r);
    std::vector<uint32_t> rel(r);
    KMC_CUDA_TRY(cudaMemcpyAsync(lst.data(), pc->dbg_list.p, r * 8, cudaMemcpyDeviceToHost, h.st));
    KMC_CUDA_TRY(cudaMemcpyAsync(rd.data(), pc->dbg_read.p, r * 8, cudaMemcpyDeviceToHost, h.st));
    KMC_CUDA_TRY(cudaMemcpyAsync(rel.data(), pc->dbg_rel.p, r * 4, cudaMemcpyDeviceToHost, h.st));
    KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
    for (uint64_t i = 0; i < r; ++i) {
      if (read_index) read_index[o + i] = rd[i];
      if (pos) pos[o + i] = rel[i];
      if (n_kmers) n_kmers[o + i] = (uint32_t)((lst[i] >> 25) & 127u) + 1;
      if (sig) sig[o + i] = (uint32_t)(lst[i] & 0x1FFFFFFu);
    }
    o += r;
  }
  return KMC_OK;
}

}  // namespace kmc
