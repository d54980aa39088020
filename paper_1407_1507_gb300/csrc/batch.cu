// Batched counting: many independent read sets per launch sequence.
//
// A sub-batch packs whole read sets into one input stream; set s owns bins
// [s*B, (s+1)*B), so the distribution, the sort and the counting treat the
// whole sub-batch as one job and the sets never mix.  Every buffer is sized
// from the engine's capacity (not from the data) and every kernel reads the
// sizes only the device knows from device memory, so the launch sequence
// needs no host synchronisation: it is captured once into a CUDA graph and
// replayed for every sub-batch.  The survivors are ordered by (set, k-mer)
// and split per set at the end.  Sets larger than the engine's capacity
// take the single-set path.  An autotuner times a few settings (bins per
// set, bucket width, tile size) on the first sub-batch and keeps the fastest.
#include <new>
#include <algorithm>
#include <chrono>
#include <cstring>
#include <map>
#include <memory>
#include <vector>
#include <atomic>
#include <mutex>
#include <shared_mutex>
#include <thread>

#include "internal.h"
#include "sortlib.cuh"
#include "dist_kernels.cuh"
#include "kx_kernels.cuh"

namespace kmc {

namespace {

inline unsigned gfor(uint64_t n, int threads, uint64_t cap = 1u << 30) {
  uint64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (unsigned)std::min<uint64_t>(g, cap);
}

struct Tuning {
  uint32_t bins;        // bins per set
  uint32_t bucket_div;  // target keys per bucket = tile / bucket_div
  uint32_t ipt;         // keys per thread in a tile (tile = 256 * ipt)
};

// Per set bin count -> digits for about tile/div keys per bucket.
__global__ void batch_groups_kernel(const unsigned long long *bin_kmers, uint32_t n_bins,
                                    uint32_t key_bits, uint32_t target, uint8_t *group_D,
                                    uint32_t *group_sz) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_bins; b += gridDim.x * blockDim.x) {
    const unsigned long long n = bin_kmers[b];
    uint32_t D = 0;
    while (D < 20 && D < key_bits && (n >> D) > target) ++D;
    group_D[b] = (uint8_t)D;
    group_sz[b] = 1u << D;
  }
}

__global__ void to_u32_kernel(const uint64_t *in, uint32_t n, uint32_t *out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[i] = (uint32_t)in[i];
}

// Chunks of at most `per` records of every bin: counts, then descriptors.
__global__ void chunk_count_kernel(const uint64_t *rec_base, uint32_t n_bins, uint32_t per,
                                   uint32_t *cnt) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_bins; b += gridDim.x * blockDim.x)
    cnt[b] = (uint32_t)((rec_base[b + 1] - rec_base[b] + per - 1) / per);
}
__global__ void chunk_emit_kernel(const uint64_t *rec_base, const uint64_t *chunk_base,
                                  uint32_t n_bins, uint32_t per, Chunk *chunks,
                                  unsigned long long *n_chunks) {
  for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n_bins; b += gridDim.x * blockDim.x) {
    const uint64_t r0 = rec_base[b], r1 = rec_base[b + 1];
    uint64_t c = chunk_base[b];
    for (uint64_t r = r0; r < r1; r += per, ++c)
      chunks[c] = Chunk{r, (uint32_t)(r1 - r < per ? r1 - r : per), 0u, b, 0u};
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_chunks = chunk_base[n_bins];
}

// Order keys (set slot above the k-mer) for the final per-set ordering.
template <typename KO>
__global__ void order_keys_kernel(const uint64_t *kmers, const uint32_t *slots,
                                  const unsigned long long *n_dyn, int k, KO *okeys) {
  const uint64_t n = *n_dyn;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    okeys[i] = ((KO)slots[i] << (2 * k)) | (KO)kmers[i];
}

template <typename KO>
__global__ void order_hist_kernel(const KO *keys, const unsigned long long *n_dyn, int key_bits,
                                  int D, uint32_t *hist) {
  const uint64_t n = *n_dyn;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&hist[top_digit<KO>(keys[i], key_bits, D)], 1u);
}

template <typename KO>
__global__ void order_scatter_kernel(const KO *keys, const uint32_t *vals,
                                     const unsigned long long *n_dyn, int key_bits, int D,
                                     const uint64_t *base, uint32_t *cursor, KO *out_k,
                                     uint32_t *out_v) {
  const uint64_t n = *n_dyn;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t d = top_digit<KO>(keys[i], key_bits, D);
    const uint64_t p = base[d] + atomicAdd(&cursor[d], 1u);
    out_k[p] = keys[i];
    out_v[p] = vals[i];
  }
}

// Splits the ordered (set, k-mer) keys into the result arrays and counts
// the k-mers of each set.
template <typename KO>
__global__ void order_split_kernel(const KO *okeys, const unsigned long long *n_dyn, int k,
                                   uint64_t *kmers, uint32_t *set_hist) {
  const uint64_t n = *n_dyn;
  const KO mask = (KO(1) << (2 * k)) - 1;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    kmers[i] = (uint64_t)(okeys[i] & mask);
    atomicAdd(&set_hist[(uint32_t)(okeys[i] >> (2 * k))], 1u);
  }
}

constexpr int B_THREADS = 256;
constexpr int B_BIG_IPT = 16;

}  // namespace

// One engine: fixed k (<= 32), capacity and tuning; all buffers allocated
// once at construction.
struct BatchEngine {
  kmc_params p{};
  Tuning tune{};
  cudaStream_t st = nullptr;
  int sm_count = 0;
  uint64_t cap_bases = 0, cap_reads = 0;
  uint32_t max_sets = 0;
  uint32_t m_used = 0, n_sig = 0;
  uint32_t B_total = 0;
  uint64_t n_stream_max = 0, n_mwords = 0, list_cap = 0, words_cap = 0, chunk_cap = 0, NB_max = 0;
  uint64_t sv_cap = 0, ond = 0;
  int o_D = 0;
  bool order128 = false;
  // device
  DevBuf in, offs, set_starts, dyn, err, map, abm;
  DevBuf packed, inval, starts, list, hist3, rec_base, word_base, cursors, index, words;
  DevBuf chunk_cnt, chunk_base, chunks, group_D, group_sz, group_base64, group_base, pieces;
  DevBuf hist, bucket_base, flags, fscan, tfirst, tdesc, scan_tmp, keys, sv_keys, sv_counts, sv_slots,
      big_list, big_scratch, counters;
  DevBuf okeys, okeys2, ovals2, o_hist, o_base, o_flags, o_fscan, o_tfirst, o_grp, o_big_list,
      o_big_k, o_big_v, o_counters, res_kmers, set_hist, set_base;
  // pinned host staging
  char *h_in = nullptr;
  uint64_t *h_offs = nullptr, *h_set_starts = nullptr;
  BatchDyn *h_dyn = nullptr;
  // graph
  cudaGraphExec_t exec = nullptr;
  bool use_graph = true;
  // map built from the first sub-batch's sample
  bool map_ready = false;

  ~BatchEngine() { release(); }
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    DevBuf *bufs[] = {&in, &offs, &set_starts, &dyn, &err, &map, &abm, &packed, &inval, &starts, &list,
                      &hist3, &rec_base, &word_base, &cursors, &index, &words, &chunk_cnt,
                      &chunk_base, &chunks, &group_D, &group_sz, &group_base64, &group_base,
                      &pieces, &hist, &bucket_base, &flags, &fscan, &tfirst, &tdesc, &scan_tmp, &keys,
                      &sv_keys, &sv_counts, &sv_slots, &big_list, &big_scratch, &counters, &okeys,
                      &okeys2, &ovals2, &o_hist, &o_base, &o_flags, &o_fscan, &o_tfirst, &o_grp,
                      &o_big_list, &o_big_k, &o_big_v, &o_counters, &res_kmers, &set_hist, &set_base};
    for (DevBuf *b : bufs) dev_release(*b, st);
    if (st) cudaStreamSynchronize(st);
    if (h_in) cudaFreeHost(h_in);
    if (h_offs) cudaFreeHost(h_offs);
    if (h_set_starts) cudaFreeHost(h_set_starts);
    if (h_dyn) cudaFreeHost(h_dyn);
    h_in = nullptr;
    h_offs = h_set_starts = nullptr;
    h_dyn = nullptr;
  }

  int alloc() {
    const uint32_t k = p.k;
    m_used = std::min(p.m, p.k);
    n_sig = (1u << (2 * m_used)) + 1u;
    B_total = max_sets * tune.bins;
    n_stream_max = cap_bases;
    n_mwords = (n_stream_max + 63) / 64 + 8;
    list_cap = n_stream_max + 1;
    // record words: 2(n+k-1) bits rounded up per record, at most one record per position
    words_cap = (2 * n_stream_max + (uint64_t)(2 * k + 62) * list_cap) / 64 + 16;
    chunk_cap = list_cap / KX_RECORDS_PER_CHUNK + B_total + 1;
    const uint64_t tile = 256ull * tune.ipt;
    const uint64_t target = std::max<uint64_t>(1, tile / tune.bucket_div);
    NB_max = 2 * (n_stream_max / target + 1) + B_total;
    sv_cap = n_stream_max / std::max<uint64_t>(1, p.cutoff_min) + tile + 1;
    // per-set order: slot above the 2k k-mer bits
    int slot_bits = 0;
    while ((1u << slot_bits) < max_sets) ++slot_bits;
    order128 = 2 * (int)k + slot_bits > 64;
    o_D = 0;
    while (o_D < 22 && (sv_cap >> o_D) > 1024) ++o_D;
    ond = 1ull << o_D;
    const size_t ok = order128 ? 16 : 8;
    auto E = [&](DevBuf &b, size_t bytes) { return dev_ensure(b, bytes, st); };
    if (E(in, cap_bases + 64) || E(offs, (cap_reads + 2) * 8) || E(set_starts, (max_sets + 2) * 8) ||
        E(dyn, sizeof(BatchDyn)) || E(err, 64) || E(map, (size_t)n_sig * 4) ||
        E(abm, (size_t)mmer_bm_words((int)m_used) * 4) ||
        E(packed, 2 * n_mwords * 8) || E(inval, n_mwords * 8) || E(starts, n_mwords * 8) ||
        E(list, list_cap * 8) || E(hist3, (size_t)B_total * 24) || E(rec_base, ((size_t)B_total + 1) * 8) ||
        E(word_base, ((size_t)B_total + 1) * 8) || E(cursors, (size_t)B_total * 16) ||
        E(index, list_cap * 8) || E(words, words_cap * 8) || E(chunk_cnt, (size_t)B_total * 4) ||
        E(chunk_base, ((size_t)B_total + 1) * 8) || E(chunks, chunk_cap * sizeof(Chunk)) ||
        E(group_D, B_total + 16) || E(group_sz, (size_t)B_total * 4) ||
        E(group_base64, ((size_t)B_total + 1) * 8) || E(group_base, ((size_t)B_total + 1) * 4) ||
        E(pieces, 64) || E(hist, NB_max * 4) || E(bucket_base, (NB_max + 1) * 8) ||
        E(flags, NB_max * 4) || E(fscan, (NB_max + 1) * 8) || E(tfirst, NB_max * 4 + 16) ||
        E(tdesc, (NB_max + 1) * sizeof(TileDesc)) ||
        E(scan_tmp, scan_tmp_words(std::max<uint64_t>(NB_max, std::max<uint64_t>(B_total, ond))) * 8) ||
        E(keys, (list_cap + 2) * 8) || E(sv_keys, sv_cap * 8) || E(sv_counts, sv_cap * 4) ||
        E(sv_slots, sv_cap * 4) || E(big_list, (list_cap / (tile + 1) + 2) * 4) ||
        E(big_scratch, list_cap * 8) || E(counters, 128) || E(okeys, sv_cap * ok) ||
        E(okeys2, sv_cap * ok) || E(ovals2, sv_cap * 4) || E(o_hist, ond * 4) ||
        E(o_base, (ond + 1) * 8) || E(o_flags, ond * 4 + 4) || E(o_fscan, (ond + 1) * 8) ||
        E(o_tfirst, ond * 4 + 16) || E(o_grp, 64) || E(o_big_list, ond * 4 + 4) ||
        E(o_big_k, sv_cap * ok) || E(o_big_v, sv_cap * 4) || E(o_counters, 128) ||
        E(res_kmers, sv_cap * 8) || E(set_hist, (size_t)max_sets * 4 + 4) ||
        E(set_base, ((size_t)max_sets + 2) * 8))
      return KMC_ENOMEM;
    if (host_alloc((void **)&h_in, cap_bases + 64, cudaHostAllocDefault) != cudaSuccess ||
        host_alloc((void **)&h_offs, (cap_reads + 2) * 8, cudaHostAllocDefault) != cudaSuccess ||
        host_alloc((void **)&h_set_starts, (max_sets + 2) * 8, cudaHostAllocDefault) != cudaSuccess ||
        host_alloc((void **)&h_dyn, sizeof(BatchDyn), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return KMC_ENOMEM;
    }
    // kernel attributes and occupancies are set here, outside any capture
    KMC_CUDA_TRY(sig_prepare());
    KMC_CUDA_TRY(build_mmer_bm(as<uint32_t>(abm), (int)m_used, st));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaFuncSetAttribute(scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)scat_smem_bytes(SIG_SMEM_BINS)));
    KMC_CUDA_TRY(cudaFuncSetAttribute(kx0_scatter_kernel<uint64_t>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(KxScatterSmem<uint64_t>)));
    int rc = tune.ipt == 8 ? prepare_count<8>() : prepare_count<16>();
    if (!rc) rc = order128 ? prepare_order<u128>() : prepare_order<uint64_t>();
    if (rc) return rc;
    PieceDesc pd{as<uint64_t>(index), as<uint64_t>(words)};
    KMC_CUDA_TRY(cudaMemcpyAsync(pieces.p, &pd, sizeof(pd), cudaMemcpyHostToDevice, st));
    uint32_t og[4] = {0u, (uint32_t)ond, (uint32_t)o_D, 0u};
    KMC_CUDA_TRY(cudaMemcpyAsync(o_grp.p, og, 16, cudaMemcpyHostToDevice, st));
    KMC_CUDA_TRY(cudaMemsetAsync(err.p, 0, 64, st));
    KMC_CUDA_TRY(cudaStreamSynchronize(st));
    return KMC_OK;
  }

  int occ_count = 1, occ_order = 1, occ_hash = 1;
  template <int IPT>
  int prepare_count() {
    constexpr int GIPT = B_THREADS * IPT / GRP_THREADS;
    using GSM = TileGroupSmem<uint64_t, GRP_THREADS, GIPT>;
    using BSM = BigSmem<uint64_t, NoVal, B_THREADS, B_BIG_IPT>;
    KMC_CUDA_TRY(cudaFuncSetAttribute(tile_group_kernel<uint64_t, GRP_THREADS, GIPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GSM)));
    KMC_CUDA_TRY(cudaFuncSetAttribute(big_count_kernel<uint64_t, B_THREADS, B_BIG_IPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BSM)));
    KMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ_count, tile_group_kernel<uint64_t, GRP_THREADS, GIPT>, GRP_THREADS, sizeof(GSM)));
    constexpr int HIPT = B_THREADS * IPT / HASH_THREADS;
    using HSM = TileHashSmem<HASH_THREADS, HIPT>;
    KMC_CUDA_TRY(cudaFuncSetAttribute(tile_hash_kernel<HASH_THREADS, HIPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(HSM)));
    KMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ_hash, tile_hash_kernel<HASH_THREADS, HIPT>, HASH_THREADS, sizeof(HSM)));
    return KMC_OK;
  }
  template <typename KO>
  int prepare_order() {
    constexpr int IPT = sizeof(KO) == 8 ? 16 : 8;
    using SM = TilePairsSmem<KO, uint32_t, B_THREADS, IPT>;
    using BSM = BigSmem<KO, uint32_t, B_THREADS, 8>;
    KMC_CUDA_TRY(cudaFuncSetAttribute(tile_pairs_kernel<KO, uint32_t, B_THREADS, IPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM)));
    KMC_CUDA_TRY(cudaFuncSetAttribute(big_pairs_kernel<KO, uint32_t, B_THREADS, 8>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BSM)));
    KMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ_order, tile_pairs_kernel<KO, uint32_t, B_THREADS, IPT>, B_THREADS, sizeof(SM)));
    return KMC_OK;
  }
  template <int IPT>
  int count_stage(const TilePlan &plan, const Mixer<uint64_t> &mixer);
  template <typename KO>
  int order_stage();
  int sequence();
};

template <int IPT>
int BatchEngine::count_stage(const TilePlan &plan, const Mixer<uint64_t> &mixer) {
  using K = uint64_t;
  constexpr int GIPT = B_THREADS * IPT / GRP_THREADS;
  using GSM = TileGroupSmem<K, GRP_THREADS, GIPT>;
  using BSM = BigSmem<K, NoVal, B_THREADS, B_BIG_IPT>;
  auto *c32 = as<uint32_t>(counters);
  auto *c64 = reinterpret_cast<unsigned long long *>(c32 + 4);
  KMC_CUDA_TRY(cudaMemsetAsync(c32, 0, 64, st));
  CountOut<K> out;
  out.keys = as<K>(sv_keys);
  out.counts = as<uint32_t>(sv_counts);
  out.n = &as<BatchDyn>(dyn)->n_sv;
  out.cap = sv_cap;
  out.ci = p.cutoff_min ? p.cutoff_min : 1;
  out.cx = p.cutoff_max;
  out.n_distinct = c64 + 1;
  out.mixer = mixer;
  out.sort_bits = kCountSortBits;
  out.slots = as<uint32_t>(sv_slots);
  out.bins_per_slot = tune.bins;
  const int occ = occ_count;
  const uint32_t big_cap = (uint32_t)(list_cap / (256ull * IPT + 1) + 2);
  TilePlan gplan = plan;
  gplan.desc = as<TileDesc>(tdesc);
  tile_desc_kernel<<<(unsigned)std::min<uint64_t>((plan.NB + 255) / 256, 4096), 256, 0, st>>>(plan,
                                                                                           as<TileDesc>(tdesc));
  KMC_COUNT_LAUNCH();
  if (2 * (int)p.k <= 62) {  // keys below 2^62: hashed tiles
    constexpr int HIPT = B_THREADS * IPT / HASH_THREADS;
    tile_hash_kernel<HASH_THREADS, HIPT><<<(unsigned)std::max(1, occ_hash) * sm_count, HASH_THREADS,
                                           sizeof(TileHashSmem<HASH_THREADS, HIPT>), st>>>(
        as<K>(keys), gplan, c32 + 0, out, as<uint32_t>(big_list), c32 + 1, c64 + 2, big_cap, as<uint32_t>(err));
  } else {
    tile_group_kernel<K, GRP_THREADS, GIPT><<<(unsigned)std::max(1, occ) * sm_count, GRP_THREADS, sizeof(GSM),
                                              st>>>(
        as<K>(keys), gplan, c32 + 0, out, as<uint32_t>(big_list), c32 + 1, c64 + 2, big_cap, as<uint32_t>(err));
  }
  KMC_COUNT_LAUNCH();
  big_count_kernel<K, B_THREADS, B_BIG_IPT><<<sm_count, B_THREADS, sizeof(BSM), st>>>(
      as<K>(keys), plan, as<uint32_t>(big_list), c32 + 1, as<K>(big_scratch), c64 + 3, out,
      as<uint32_t>(err), (K *)nullptr);
  KMC_COUNT_LAUNCH();
  return cudaGetLastError() == cudaSuccess ? KMC_OK : KMC_ECUDA;
}

template <typename KO>
int BatchEngine::order_stage() {
  using V = uint32_t;
  constexpr int IPT = sizeof(KO) == 8 ? 16 : 8;
  using SM = TilePairsSmem<KO, V, B_THREADS, IPT>;
  using BSM = BigSmem<KO, V, B_THREADS, 8>;
  const int k = (int)p.k;
  int slot_bits = 0;
  while ((1u << slot_bits) < max_sets) ++slot_bits;
  const int key_bits = 2 * k + slot_bits;
  auto *n_sv = &as<BatchDyn>(dyn)->n_sv;
  const unsigned grid = (unsigned)sm_count * 4;
  order_keys_kernel<KO><<<grid, 256, 0, st>>>(as<uint64_t>(sv_keys), as<uint32_t>(sv_slots), n_sv, k, as<KO>(okeys));
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaMemsetAsync(o_hist.p, 0, ond * 4, st));
  order_hist_kernel<KO><<<grid, 256, 0, st>>>(as<KO>(okeys), n_sv, key_bits, o_D, as<uint32_t>(o_hist));
  KMC_COUNT_LAUNCH();
  const uint32_t *grp = as<uint32_t>(o_grp);
  KMC_CUDA_TRY(device_excl_scan_u32(as<uint32_t>(o_hist), as<uint64_t>(o_base), ond, as<uint64_t>(scan_tmp), st));
  plan_flags_kernel<<<gfor(ond, 256, 65535), 256, 0, st>>>(as<uint32_t>(o_hist), as<uint64_t>(o_base), ond, grp,
                                                          1, (uint32_t)(256 * IPT), as<uint32_t>(o_flags));
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(device_excl_scan_u32(as<uint32_t>(o_flags), as<uint64_t>(o_fscan), ond, as<uint64_t>(scan_tmp), st));
  uint32_t *n_tiles = as<uint32_t>(o_tfirst) + ond + 1;
  plan_emit_kernel<<<gfor(ond, 256, 65535), 256, 0, st>>>(as<uint32_t>(o_flags), as<uint64_t>(o_fscan), ond,
                                                         as<uint32_t>(o_tfirst), n_tiles);
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaMemsetAsync(o_hist.p, 0, ond * 4, st));
  order_scatter_kernel<KO><<<grid, 256, 0, st>>>(as<KO>(okeys), as<uint32_t>(sv_counts), n_sv, key_bits, o_D,
                                                 as<uint64_t>(o_base), as<uint32_t>(o_hist), as<KO>(okeys2),
                                                 as<uint32_t>(ovals2));
  KMC_COUNT_LAUNCH();
  TilePlan plan;
  plan.bucket_base = as<uint64_t>(o_base);
  plan.tile_first = as<uint32_t>(o_tfirst);
  plan.n_tiles = n_tiles;
  plan.group_base = grp;
  plan.group_D = reinterpret_cast<const uint8_t *>(grp + 2);
  plan.n_groups = 1;
  plan.NB = (uint32_t)ond;
  plan.key_bits = key_bits;
  auto *c32 = as<uint32_t>(o_counters);
  auto *c64 = reinterpret_cast<unsigned long long *>(c32 + 4);
  KMC_CUDA_TRY(cudaMemsetAsync(c32, 0, 64, st));
  const int occ = occ_order;
  tile_pairs_kernel<KO, V, B_THREADS, IPT><<<(unsigned)std::max(1, occ) * sm_count, B_THREADS, sizeof(SM), st>>>(
      as<KO>(okeys2), as<uint32_t>(ovals2), plan, c32 + 0, as<uint32_t>(o_big_list), c32 + 1, c64 + 0,
      (uint32_t)ond, as<uint32_t>(err));
  KMC_COUNT_LAUNCH();
  big_pairs_kernel<KO, V, B_THREADS, 8><<<sm_count, B_THREADS, sizeof(BSM), st>>>(
      as<KO>(okeys2), as<uint32_t>(ovals2), plan, as<uint32_t>(o_big_list), c32 + 1, as<KO>(o_big_k),
      as<uint32_t>(o_big_v), c64 + 1);
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaMemsetAsync(set_hist.p, 0, (size_t)max_sets * 4 + 4, st));
  order_split_kernel<KO><<<grid, 256, 0, st>>>(as<KO>(okeys2), n_sv, k, as<uint64_t>(res_kmers),
                                               as<uint32_t>(set_hist));
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(device_excl_scan_u32(as<uint32_t>(set_hist), as<uint64_t>(set_base), max_sets,
                                    as<uint64_t>(scan_tmp), st));
  return cudaGetLastError() == cudaSuccess ? KMC_OK : KMC_ECUDA;
}

// The whole launch sequence of one sub-batch (no host synchronisation).
int BatchEngine::sequence() {
  const int k = (int)p.k;
  BatchDyn *d = as<BatchDyn>(dyn);
  // a1: pack + read starts
  KMC_CUDA_TRY(cudaMemsetAsync(starts.p, 0, n_mwords * 8, st));
  pack_kernel<<<gfor(n_mwords, 256), 256, 0, st>>>(reinterpret_cast<const uint8_t *>(in.p), n_stream_max, 0,
                                                  as<uint64_t>(packed), as<uint64_t>(inval), n_mwords,
                                                  &d->n_stream);
  KMC_COUNT_LAUNCH();
  starts_kernel<<<gfor(cap_reads, 256, 65535), 256, 0, st>>>(as<uint64_t>(offs), 0, cap_reads, 0, 0, n_stream_max,
                                                            as<unsigned long long>(starts), as<uint32_t>(err),
                                                            &d->n_reads);
  KMC_COUNT_LAUNCH();
  // a2: signatures and super k-mers, per (set, bin) histograms
  KMC_CUDA_TRY(cudaMemsetAsync(hist3.p, 0, (size_t)B_total * 24, st));
  auto *h_rec = as<unsigned long long>(hist3);
  auto *h_words = h_rec + B_total;
  auto *h_kmers = h_words + B_total;
  SigArgs a{};
  a.packed = as<uint64_t>(packed);
  a.inval = as<uint64_t>(inval);
  a.smask = as<uint64_t>(starts);
  a.n_pwords = 2 * n_mwords;
  a.n_mwords = n_mwords;
  a.n_stream = n_stream_max;
  a.offsets = as<uint64_t>(offs);
  a.r0 = 0;
  a.r1 = cap_reads;
  a.byte_start = 0;
  a.mis = 0;
  a.k = k;
  a.m = (int)m_used;
  a.map = as<uint32_t>(map);
  a.abm = as<uint32_t>(abm);
  a.n_bins = B_total;
  a.list = as<uint64_t>(list);
  a.n_list = &d->n_list;
  a.list_cap = list_cap;
  a.bin_rec = h_rec;
  a.bin_words = h_words;
  a.bin_kmers = h_kmers;
  a.err = as<uint32_t>(err);
  a.n_stream_dyn = &d->n_stream;
  a.n_reads_dyn = &d->n_reads;
  a.set_starts = as<uint64_t>(set_starts);
  a.n_slots = max_sets;
  a.bins_per_slot = tune.bins;
  if (sig_launch(a, n_stream_max, false, st)) KMC_COUNT_LAUNCH();
  // a3: bins
  KMC_CUDA_TRY(device_excl_scan_u64(reinterpret_cast<uint64_t *>(h_rec), as<uint64_t>(rec_base), B_total,
                                    as<uint64_t>(scan_tmp), st));
  KMC_CUDA_TRY(device_excl_scan_u64(reinterpret_cast<uint64_t *>(h_words), as<uint64_t>(word_base), B_total,
                                    as<uint64_t>(scan_tmp), st));
  auto *cur = as<unsigned long long>(cursors);
  KMC_CUDA_TRY(cudaMemcpyAsync(cur, rec_base.p, (size_t)B_total * 8, cudaMemcpyDeviceToDevice, st));
  KMC_CUDA_TRY(cudaMemcpyAsync(cur + B_total, word_base.p, (size_t)B_total * 8, cudaMemcpyDeviceToDevice, st));
  scatter_kernel<<<gfor(list_cap, SCAT_PER_CTA), SCAT_THREADS, scat_smem_bytes(B_total), st>>>(
      as<uint64_t>(list), 0, as<uint32_t>(map), B_total, k, as<uint64_t>(packed), cur, cur + B_total,
      as<uint64_t>(index), as<uint64_t>(words), &d->n_list, as<uint64_t>(set_starts), max_sets, tune.bins);
  KMC_COUNT_LAUNCH();
  // a4 setup: record chunks and per-bin bucket groups, all on the device
  chunk_count_kernel<<<gfor(B_total, 256), 256, 0, st>>>(as<uint64_t>(rec_base), B_total, KX_RECORDS_PER_CHUNK,
                                                         as<uint32_t>(chunk_cnt));
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(device_excl_scan_u32(as<uint32_t>(chunk_cnt), as<uint64_t>(chunk_base), B_total,
                                    as<uint64_t>(scan_tmp), st));
  chunk_emit_kernel<<<gfor(B_total, 256), 256, 0, st>>>(as<uint64_t>(rec_base), as<uint64_t>(chunk_base), B_total,
                                                        KX_RECORDS_PER_CHUNK, as<Chunk>(chunks), &d->n_chunks);
  KMC_COUNT_LAUNCH();
  const uint32_t tile = 256u * tune.ipt;
  batch_groups_kernel<<<gfor(B_total, 256), 256, 0, st>>>(h_kmers, B_total, 2 * k,
                                                          std::max<uint32_t>(1, tile / tune.bucket_div),
                                                          as<uint8_t>(group_D), as<uint32_t>(group_sz));
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(device_excl_scan_u32(as<uint32_t>(group_sz), as<uint64_t>(group_base64), B_total,
                                    as<uint64_t>(scan_tmp), st));
  to_u32_kernel<<<gfor(B_total + 1, 256), 256, 0, st>>>(as<uint64_t>(group_base64), B_total + 1,
                                                        as<uint32_t>(group_base));
  KMC_COUNT_LAUNCH();
  KxArgs<uint64_t> ka;
  ka.chunks = as<Chunk>(chunks);
  ka.pieces = as<PieceDesc>(pieces);
  ka.k = k;
  ka.key_bits = 2 * k;
  ka.group_base = as<uint32_t>(group_base);
  ka.group_D = as<uint8_t>(group_D);
  ka.mixer = Mixer<uint64_t>{};
  {
    // same constants as the single-set path
    const int bits = 2 * k;
    Mixer<uint64_t> &m = ka.mixer;
    m.bits = bits;
    m.mask = bits >= 64 ? ~0ull : ((1ull << bits) - 1);
    uint64_t c = 0x9E3779B97F4A7C15ull | 1ull, inv = c;
    for (int i = 0; i < 7; ++i) inv *= 2 - c * inv;
    m.c = c & m.mask;
    m.cinv = inv & m.mask;
    m.s1 = (bits + 1) / 2;
    m.s2 = bits / 3 + 1;
    m.on = true;
  }
  ka.n_chunks_dyn = &d->n_chunks;
  KMC_CUDA_TRY(cudaMemsetAsync(hist.p, 0, NB_max * 4, st));
  kx0_count_kernel<uint64_t><<<(unsigned)chunk_cap, KX_THREADS, 0, st>>>(ka, as<uint32_t>(hist));
  KMC_COUNT_LAUNCH();
  // plan over all possible buckets (the tail past the last bin holds no keys)
  KMC_CUDA_TRY(device_excl_scan_u32(as<uint32_t>(hist), as<uint64_t>(bucket_base), NB_max, as<uint64_t>(scan_tmp), st));
  const uint64_t n_seg = (NB_max + kGreedySegment - 1) / kGreedySegment;
  plan_greedy_flags_kernel<<<(unsigned)((n_seg + 7) / 8), 256, 0, st>>>(as<uint32_t>(hist), as<uint32_t>(group_base),
                                                                       B_total, NB_max, tile, as<uint32_t>(flags));
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(device_excl_scan_u32(as<uint32_t>(flags), as<uint64_t>(fscan), NB_max, as<uint64_t>(scan_tmp), st));
  uint32_t *n_tiles = as<uint32_t>(tfirst) + NB_max + 1;
  plan_emit_kernel<<<gfor(NB_max, 256, 65535), 256, 0, st>>>(as<uint32_t>(flags), as<uint64_t>(fscan), NB_max,
                                                            as<uint32_t>(tfirst), n_tiles);
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaMemsetAsync(hist.p, 0, NB_max * 4, st));
  kx0_scatter_kernel<uint64_t><<<(unsigned)chunk_cap, KX_THREADS, sizeof(KxScatterSmem<uint64_t>), st>>>(
      ka, as<uint64_t>(bucket_base), as<uint32_t>(hist), as<uint64_t>(keys), list_cap, as<uint32_t>(err));
  KMC_COUNT_LAUNCH();
  // a5/a6: sort and count every tile; survivors carry their set
  TilePlan plan;
  plan.bucket_base = as<uint64_t>(bucket_base);
  plan.tile_first = as<uint32_t>(tfirst);
  plan.n_tiles = n_tiles;
  plan.group_base = as<uint32_t>(group_base);
  plan.group_D = as<uint8_t>(group_D);
  plan.n_groups = B_total;
  plan.NB = (uint32_t)NB_max;
  plan.key_bits = 2 * k;
  int rc = tune.ipt == 8 ? count_stage<8>(plan, ka.mixer) : count_stage<16>(plan, ka.mixer);
  if (rc) return rc;
  // a7: per-set order
  return order128 ? order_stage<u128>() : order_stage<uint64_t>();
}

}  // namespace kmc

// ------------------------------------------------------------------ C ABI

using namespace kmc;

namespace kmc {
namespace {
// Sets of kSingleMinBases or more (internal.h) are counted one at a time on
// the single-set path, by this many host threads (lanes) at once.
constexpr int kSingleLanes = 2;
}  // namespace
}  // namespace kmc

struct kmc_batch {
  kmc_params base{};
  uint64_t cap_bases = 0, cap_reads = 0;
  uint32_t max_sets = 0;
  uint32_t flags = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  int sm_count = 0;
  std::map<uint32_t, std::unique_ptr<BatchEngine>> engines;  // one per k, kept resident
  std::map<uint32_t, Tuning> tuned;   // tuning chosen per k
  // results of the last run: every set's k-mers and counts in one pinned host
  // arena (reused across runs, grown when a run needs more), set s at
  // [res_off[s], res_off[s] + res_n[s])
  uint64_t *ak = nullptr;
  uint32_t *ac = nullptr;
  uint64_t acap = 0, aused = 0;
  std::vector<uint64_t> res_off, res_n;
  // sets counted one at a time: per lane, one handle per k, kept open and
  // reset per set
  std::map<uint32_t, kmc_handle *> single[kSingleLanes];
  // the bin map each of those handles built from its first set, reused for the
  // sets after it (the result does not depend on the map; this saves the
  // sample scan per set, as the batch engine's one map per k does)
  std::map<uint32_t, std::vector<uint32_t>> single_map[kSingleLanes];
  std::mutex single_mu;
  std::shared_mutex arena_mu;  // growth (exclusive) against copies into the arena (shared)
  kmc_batch_stats stats{};
};

namespace {

// Room for n more results in the arena (growing it keeps what is there).
int arena_reserve(kmc_batch *b, uint64_t n) {
  if (b->aused + n <= b->acap) return KMC_OK;
  const uint64_t cap = std::max<uint64_t>(b->aused + n, 2 * b->acap) + (1u << 16);
  void *nk = nullptr, *nc = nullptr;
  if (host_alloc(&nk, cap * 8, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    return KMC_ENOMEM;
  }
  if (host_alloc(&nc, cap * 4, cudaHostAllocDefault) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(nk);
    return KMC_ENOMEM;
  }
  if (b->aused) {
    memcpy(nk, b->ak, b->aused * 8);
    memcpy(nc, b->ac, b->aused * 4);
  }
  if (b->ak) cudaFreeHost(b->ak);
  if (b->ac) cudaFreeHost(b->ac);
  b->ak = static_cast<uint64_t *>(nk);
  b->ac = static_cast<uint32_t *>(nc);
  b->acap = cap;
  return KMC_OK;
}

int make_engine(kmc_batch *b, uint32_t k, const Tuning &t, std::unique_ptr<BatchEngine> *out) {
  auto e = std::make_unique<BatchEngine>();
  e->p = b->base;
  e->p.k = k;
  e->tune = t;
  e->st = b->st;
  e->sm_count = b->sm_count;
  e->cap_bases = b->cap_bases;
  e->cap_reads = b->cap_reads;
  e->max_sets = b->max_sets;
  int rc = e->alloc();
  if (rc) return rc;
  *out = std::move(e);
  return KMC_OK;
}

// Copies sub-batch sets [s0, s1) into the engine's input and runs it.
int run_sub(kmc_batch *b, BatchEngine &e, const uint32_t *idx, uint32_t s0, uint32_t s1,
            const char *const *bases, const uint64_t *const *offsets, const uint64_t *n_reads,
            bool graph, float *ms) {
  // Reads in page-locked host memory (every set of the sub-batch) are copied
  // to the device set by set, without the host copy into the staging buffer
  // (the first sub-batch of an engine still stages them: its bin map is built
  // from the staged reads).
  bool direct = e.map_ready;
  for (uint32_t j = s0; j < s1 && direct; ++j) {
    const uint32_t s = idx[j];
    if (!offsets[s][n_reads[s]]) continue;
    cudaPointerAttributes at{};
    direct = cudaPointerGetAttributes(&at, bases[s]) == cudaSuccess && at.type == cudaMemoryTypeHost;
  }
  cudaGetLastError();  // a pageable pointer may leave an error behind on some drivers
  uint64_t pos = 0, rd = 0;
  for (uint32_t j = s0; j < s1; ++j) {
    const uint32_t s = idx[j];
    const uint64_t nb = offsets[s][n_reads[s]];
    e.h_set_starts[j - s0] = pos;
    if (direct) {
      if (nb)
        KMC_CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(e.in.p) + pos, bases[s], nb, cudaMemcpyHostToDevice, e.st));
    } else {
      memcpy(e.h_in + pos, bases[s], nb);
    }
    for (uint64_t r = 0; r < n_reads[s]; ++r) e.h_offs[rd + r] = pos + offsets[s][r];
    pos += nb;
    rd += n_reads[s];
  }
  for (uint32_t j = s1 - s0; j <= e.max_sets; ++j) e.h_set_starts[j] = ~0ull;
  e.h_offs[rd] = pos;
  const uint64_t n_stream = pos;
  memset(e.h_dyn, 0, sizeof(BatchDyn));
  e.h_dyn->n_stream = n_stream;
  e.h_dyn->n_reads = rd;
  e.h_dyn->n_sets = s1 - s0;
  if (!direct) KMC_CUDA_TRY(cudaMemcpyAsync(e.in.p, e.h_in, n_stream, cudaMemcpyHostToDevice, e.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(e.offs.p, e.h_offs, (rd + 1) * 8, cudaMemcpyHostToDevice, e.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(e.set_starts.p, e.h_set_starts, (e.max_sets + 1) * 8, cudaMemcpyHostToDevice, e.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(e.dyn.p, e.h_dyn, sizeof(BatchDyn), cudaMemcpyHostToDevice, e.st));
  if (!e.map_ready) {
    // bin map from the first sub-batch: signatures of its first reads
    kmc_params mp = b->base;
    mp.k = e.p.k;
    mp.n_bins = e.tune.bins;
    mp.cuda_stream = e.st;
    mp.debug_flags = 0;
    kmc_handle *hh = nullptr;
    int rc = kmc_open(&hh, &mp);
    if (rc) return rc;
    const uint64_t sample = std::min<uint64_t>(rd, 1u << 18);
    std::vector<uint64_t> so(e.h_offs, e.h_offs + sample + 1);
    // the sample's reads are contiguous from stream position 0
    rc = kmc_add_reads(hh, e.h_in, so.data(), sample);
    std::vector<uint32_t> mapv(e.n_sig);
    if (!rc) rc = kmc_get_bin_map(hh, mapv.data(), e.n_sig);
    kmc_close(hh);
    if (rc) return rc;
    KMC_CUDA_TRY(cudaMemcpyAsync(e.map.p, mapv.data(), (size_t)e.n_sig * 4, cudaMemcpyHostToDevice, e.st));
    KMC_CUDA_TRY(cudaStreamSynchronize(e.st));
    e.map_ready = true;
  }
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  cudaEventRecord(t0, e.st);
  if (graph) {
    if (!e.exec) {
      cudaGraph_t g = nullptr;
      KMC_CUDA_TRY(cudaStreamBeginCapture(e.st, cudaStreamCaptureModeThreadLocal));
      int rc = e.sequence();
      cudaError_t ce = cudaStreamEndCapture(e.st, &g);
      if (rc) return rc;
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
      ce = cudaGraphInstantiate(&e.exec, g, 0);
      cudaGraphDestroy(g);
      if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
    }
    KMC_CUDA_TRY(cudaGraphLaunch(e.exec, e.st));
    KMC_COUNT_LAUNCH();
  } else {
    int rc = e.sequence();
    if (rc) return rc;
  }
  cudaEventRecord(t1, e.st);
  // results: per-set bases and the k-mers / counts
  BatchDyn dy;
  std::vector<uint64_t> sb(e.max_sets + 1);
  KMC_CUDA_TRY(cudaMemcpyAsync(&dy, e.dyn.p, sizeof(BatchDyn), cudaMemcpyDeviceToHost, e.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(sb.data(), e.set_base.p, (e.max_sets + 1) * 8, cudaMemcpyDeviceToHost, e.st));
  uint32_t errw = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&errw, e.err.p, 4, cudaMemcpyDeviceToHost, e.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(e.st));
  if (ms) cudaEventElapsedTime(ms, t0, t1);
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  if (errw) {
    cudaMemsetAsync(e.err.p, 0, 4, e.st);
    return (errw & ERR_INPUT) ? KMC_EINPUT : (errw & ERR_OVERFLOW) ? KMC_EOVERFLOW : KMC_ECUDA;
  }
  const uint64_t n_sv = dy.n_sv;
  // the sub-batch's results (set after set) into the pinned arena, one copy
  int rc = arena_reserve(b, n_sv);
  if (rc) return rc;
  const uint64_t at = b->aused;
  if (n_sv) {
    KMC_CUDA_TRY(cudaMemcpyAsync(b->ak + at, e.res_kmers.p, n_sv * 8, cudaMemcpyDeviceToHost, e.st));
    KMC_CUDA_TRY(cudaMemcpyAsync(b->ac + at, e.ovals2.p, n_sv * 4, cudaMemcpyDeviceToHost, e.st));
    KMC_CUDA_TRY(cudaStreamSynchronize(e.st));
  }
  for (uint32_t j = s0; j < s1; ++j) {
    const uint32_t s = idx[j];
    b->res_off[s] = at + sb[j - s0];
    b->res_n[s] = sb[j - s0 + 1] - sb[j - s0];
  }
  b->aused += n_sv;
  b->stats.n_kmers_out += n_sv;
  return KMC_OK;
}

}  // namespace

extern "C" {

int kmc_batch_open(kmc_batch **out, const kmc_params *p, uint64_t max_bases, uint64_t max_reads,
                   uint32_t max_sets, uint32_t flags) {
  if (!out || !p) return KMC_EINVAL;
  *out = nullptr;
  if (max_bases < 1024 || max_reads < 1 || max_sets < 1 || max_sets > (1u << 16)) return KMC_EINVAL;
  if (max_bases > (1ull << 31)) return KMC_EINVAL;
  if (p->cutoff_min > p->cutoff_max || p->canonical != 1 || p->counter_max || p->m < 1 || p->m > KMC_MAX_M)
    return KMC_EINVAL;
  if (flags & ~(KMC_BATCH_AUTOTUNE | KMC_BATCH_NO_GRAPH)) return KMC_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || p->device < 0 || p->device >= ndev) {
    cudaGetLastError();
    return KMC_ECUDA;
  }
  cudaSetDevice(p->device);
  kmc_batch *b = new kmc_batch();
  b->base = *p;
  b->cap_bases = max_bases;
  b->cap_reads = max_reads;
  b->max_sets = max_sets;
  b->flags = flags;
  if (p->cuda_stream) {
    b->st = static_cast<cudaStream_t>(p->cuda_stream);
  } else {
    cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking);
    b->own_stream = true;
  }
  cudaDeviceGetAttribute(&b->sm_count, cudaDevAttrMultiProcessorCount, p->device);
  *out = b;
  return KMC_OK;
}

int kmc_batch_run(kmc_batch *b, uint32_t n_sets, const char *const *bases,
                  const uint64_t *const *offsets, const uint64_t *n_reads, const uint32_t *k) {
  if (!b || (n_sets && (!bases || !offsets || !n_reads || !k))) return KMC_EINVAL;
  cudaSetDevice(b->base.device);
  for (uint32_t s = 0; s < n_sets; ++s) {
    if (k[s] < 1 || k[s] > 32) return KMC_EINVAL;
    if (!offsets[s] || offsets[s][0] != 0) return KMC_EINPUT;
    for (uint64_t r = 0; r < n_reads[s]; ++r)
      if (offsets[s][r + 1] < offsets[s][r]) return KMC_EINPUT;
  }
  b->res_off.assign(n_sets, 0);
  b->res_n.assign(n_sets, 0);
  b->aused = 0;
  b->stats = kmc_batch_stats{};
  const auto t_start = std::chrono::steady_clock::now();
  // sets grouped by k; large sets go through the single-set path
  std::map<uint32_t, std::vector<uint32_t>> by_k;
  std::vector<uint32_t> single;
  for (uint32_t s = 0; s < n_sets; ++s) {
    const uint64_t nb = offsets[s][n_reads[s]];
    if (nb + 64 > b->cap_bases || n_reads[s] + 1 > b->cap_reads || nb >= kSingleMinBases) single.push_back(s);
    else by_k[k[s]].push_back(s);
  }
  const bool graph = !(b->flags & KMC_BATCH_NO_GRAPH);
  for (auto &kv : by_k) {
    const uint32_t kk = kv.first;
    std::vector<uint32_t> &idx = kv.second;
    // sub-batches: consecutive sets while they fit the capacity
    std::vector<std::pair<uint32_t, uint32_t>> subs;
    for (uint32_t j = 0; j < idx.size();) {
      uint64_t nb = 0, nr = 0;
      uint32_t e = j;
      while (e < idx.size() && e - j < b->max_sets) {
        const uint64_t sb = offsets[idx[e]][n_reads[idx[e]]], sr = n_reads[idx[e]];
        if (nb + sb + 64 > b->cap_bases || nr + sr + 1 > b->cap_reads) break;
        nb += sb;
        nr += sr;
        ++e;
      }
      subs.push_back({j, e});
      j = e;
    }
    size_t first = 0;
    if (!b->tuned.count(kk)) {
      Tuning best{64, 2, 16};
      if (b->flags & KMC_BATCH_AUTOTUNE) {
        // time each candidate on the first sub-batch (direct launches), keep the fastest
        const Tuning cands[] = {{64, 2, 16}, {16, 2, 16}, {256, 2, 16}, {64, 4, 16}, {64, 2, 8}};
        float best_ms = 1e30f;
        for (const Tuning &t : cands) {
          std::unique_ptr<BatchEngine> trial;
          int rc = make_engine(b, kk, t, &trial);
          if (rc) return rc;
          float ms = 0;
          rc = run_sub(b, *trial, idx.data(), subs[0].first, subs[0].second, bases, offsets, n_reads,
                       false, nullptr);  // warm
          if (!rc) rc = run_sub(b, *trial, idx.data(), subs[0].first, subs[0].second, bases, offsets,
                                n_reads, false, &ms);
          if (rc) return rc;
          if (ms < best_ms) { best_ms = ms; best = t; }
        }
        b->stats.tuning_runs += 2 * (uint32_t)(sizeof(cands) / sizeof(cands[0]));
      }
      b->tuned[kk] = best;
      b->engines.erase(kk);
    }
    const Tuning t = b->tuned[kk];
    std::unique_ptr<BatchEngine> &eng = b->engines[kk];
    if (!eng) {
      int rc = make_engine(b, kk, t, &eng);
      if (rc) return rc;
    }
    for (size_t q = first; q < subs.size(); ++q) {
      float ms = 0;
      int rc = run_sub(b, *eng, idx.data(), subs[q].first, subs[q].second, bases, offsets, n_reads,
                       graph, &ms);
      if (rc) return rc;
      b->stats.ms_device += ms;
      b->stats.n_sub_batches += 1;
    }
    b->stats.bins_per_set = t.bins;
    b->stats.tile_keys = 256 * t.ipt;
    b->stats.bucket_keys = 256 * t.ipt / t.bucket_div;
  }
  // Sets counted one at a time on open handles (a handle per k and lane, each
  // on its own stream): kSingleLanes host threads take them in turn, so that
  // one set's host steps overlap another's kernels.
  std::atomic<uint32_t> next{0};
  std::atomic<int> first_err{KMC_OK};
  std::atomic<uint64_t> kmers_out{0};
  auto lane = [&](int li) {
    for (;;) {
      const uint32_t q = next.fetch_add(1);
      if (q >= single.size() || first_err.load() != KMC_OK) return;
      const uint32_t s = single[q];
      kmc_handle *hh = nullptr;
      std::vector<uint32_t> *map = nullptr;
      {
        std::lock_guard<std::mutex> g(b->single_mu);
        hh = b->single[li][k[s]];
        map = &b->single_map[li][k[s]];
      }
      int rc = KMC_OK;
      if (!hh) {
        kmc_params sp = b->base;
        sp.k = k[s];
        sp.cuda_stream = nullptr;  // a stream of its own
        sp.x = 0;
        rc = kmc_open(&hh, &sp);
        if (rc) {
          first_err.store(rc);
          return;
        }
        std::lock_guard<std::mutex> g(b->single_mu);
        b->single[li][k[s]] = hh;
      } else {
        rc = kmc_reset(hh);
        // once set, the map stays with the handle across resets
        if (!rc && !map->empty() && !hh->h.map_user) rc = kmc_set_bin_map(hh, map->data(), map->size());
      }
      if (!rc) rc = kmc_add_reads(hh, bases[s], offsets[s], n_reads[s]);
      if (!rc && map->empty()) {
        map->resize(hh->h.n_sig);
        rc = kmc_get_bin_map(hh, map->data(), map->size());
        if (rc) map->clear();
      }
      if (!rc) rc = kmc_count(hh);
      uint64_t n = 0, off = 0;
      if (!rc) rc = kmc_result_size(hh, &n);
      if (!rc) {  // room in the arena (growing it waits for the copies into it)
        std::unique_lock<std::shared_mutex> g(b->arena_mu);
        rc = arena_reserve(b, n);
        off = b->aused;
        b->aused += rc ? 0 : n;
      }
      if (!rc) {
        std::shared_lock<std::shared_mutex> g(b->arena_mu);
        b->res_off[s] = off;
        b->res_n[s] = n;
        rc = kmc_result(hh, b->ak + off, b->ac + off, n, &n);
      }
      // after a very large set its sort buffers go back to the pool (the
      // handle keeps its pinned staging and stream-ordered state)
      if (!rc && offsets[s][n_reads[s]] >= kTrimMinBases) rc = handle_trim(hh);
      if (rc) {  // a failed handle is not reused
        kmc_close(hh);
        std::lock_guard<std::mutex> g(b->single_mu);
        b->single[li].erase(k[s]);
        b->single_map[li].erase(k[s]);
        first_err.store(rc);
        return;
      }
      kmers_out += n;
    }
  };
  if (!single.empty()) {
    const int n_lanes = (int)std::min<size_t>(kSingleLanes, single.size());
    std::vector<std::thread> th;
    for (int li = 1; li < n_lanes; ++li) th.emplace_back(lane, li);
    lane(0);
    for (std::thread &t : th) t.join();
    if (first_err.load() != KMC_OK) return first_err.load();
    b->stats.n_kmers_out += kmers_out.load();
    b->stats.n_single += (uint32_t)single.size();
  }
  b->stats.ms_wall = std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  return KMC_OK;
}

int kmc_batch_result(kmc_batch *b, uint32_t set, const uint64_t **kmers, const uint32_t **counts,
                     uint64_t *n) {
  if (!b || set >= b->res_n.size()) return KMC_EINVAL;
  if (kmers) *kmers = b->ak ? b->ak + b->res_off[set] : nullptr;
  if (counts) *counts = b->ac ? b->ac + b->res_off[set] : nullptr;
  if (n) *n = b->res_n[set];
  return KMC_OK;
}

}  // extern "C"

namespace kmc {
int batch_take_result(kmc_batch *b, uint32_t set, BatchSetResult *out) {
  if (!b || set >= b->res_n.size()) return KMC_EINVAL;
  const uint64_t n = b->res_n[set], o = b->res_off[set];
  out->n = n;
  out->k.reset(new (std::nothrow) uint64_t[n ? n : 1]);
  out->c.reset(new (std::nothrow) uint32_t[n ? n : 1]);
  if (!out->k || !out->c) return KMC_ENOMEM;
  if (n) {
    memcpy(out->k.get(), b->ak + o, n * 8);
    memcpy(out->c.get(), b->ac + o, n * 4);
  }
  return KMC_OK;
}
}  // namespace kmc

extern "C" {

int kmc_batch_stats_get(const kmc_batch *b, kmc_batch_stats *s) {
  if (!b || !s) return KMC_EINVAL;
  *s = b->stats;
  return KMC_OK;
}

void kmc_batch_close(kmc_batch *b) {
  if (!b) return;
  cudaSetDevice(b->base.device);
  b->engines.clear();
  for (auto &m : b->single) {
    for (auto &kv : m) kmc_close(kv.second);
    m.clear();
  }
  if (b->ak) cudaFreeHost(b->ak);
  if (b->ac) cudaFreeHost(b->ac);
  if (b->own_stream) cudaStreamDestroy(b->st);
  delete b;
}

}  // extern "C"
