// Sorting phase (paper Sect. 2.3, 2.4, Fig. 2): bins of super k-mers ->
// keys -> radix sort -> run-length counting with the cutoffs -> survivors,
// then the survivors of all bins are put in global order.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "internal.h"
#include "sortlib.cuh"

namespace kmc {

namespace {

constexpr int KX_THREADS = 256;
constexpr int KX_RECORDS_PER_CHUNK = 512;
constexpr int CNT_THREADS = 256;
constexpr int CNT_IPT64 = 16;   // tile = 4096 64-bit keys
constexpr int CNT_IPT128 = 8;   // tile = 2048 128-bit keys
constexpr int BIG_IPT = 16;

struct PieceDesc {
  const uint64_t *index;
  const uint64_t *words;
};
struct Chunk {
  uint64_t r0;     // first record (in the piece's index)
  uint32_t n_rec;  // records
  uint32_t piece;
  uint32_t bin;
  uint32_t pad;
};

// Warp-cooperative expansion of a batch of up to 32 super k-mer records into
// their k-mers: lane r holds record r; iteration `it` gives lane l the k-mer
// number 32*it + l of the batch, found by locating the record whose k-mer
// range contains it (ballot of the record starts that fall in the window).
struct RecBatch {
  uint32_t n_rec;   // records in the batch (<= 32)
  uint32_t kst;     // this lane's record: index of its first k-mer in the batch
  uint32_t n;       // k-mers of this lane's record
  uint64_t woff;    // word offset of this lane's record
  uint32_t total;   // k-mers in the batch
};

__device__ __forceinline__ RecBatch load_batch(const uint64_t *index, uint64_t r, uint64_t r_end) {
  RecBatch b;
  const unsigned lane = lane_id();
  const uint64_t ri = r + lane;
  uint64_t e = ri < r_end ? index[ri] : 0ull;
  b.n = ri < r_end ? (uint32_t)((e >> 25) & 127u) + 1u : 0u;
  b.woff = e >> 32;
  uint32_t inc = b.n;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t o = __shfl_up_sync(FULL, inc, d);
    if (lane >= (unsigned)d) inc += o;
  }
  b.kst = inc - b.n;
  b.total = __shfl_sync(FULL, inc, 31);
  b.n_rec = r_end > r ? (uint32_t)(r_end - r < 32 ? r_end - r : 32) : 0u;
  return b;
}

// For k-mer number g = 32*it + lane of the batch: the record (lane index)
// holding it and the k-mer's index inside that record.
__device__ __forceinline__ void locate(const RecBatch &b, uint32_t it, uint32_t *rec,
                                       uint32_t *j) {
  const unsigned lane = lane_id();
  const uint32_t lo = 32 * it;
  const bool mine = lane < b.n_rec && b.n > 0;
  const unsigned before = __ballot_sync(FULL, mine && b.kst < lo);
  const unsigned bit = (mine && b.kst >= lo && b.kst < lo + 32) ? (1u << (b.kst - lo)) : 0u;
  const unsigned starts = __reduce_or_sync(FULL, bit);
  const unsigned upto = lane == 31 ? 0xFFFFFFFFu : ((2u << lane) - 1u);
  const int r = (int)__popc(before) + (int)__popc(starts & upto) - 1;
  const int rr = r < 0 ? 0 : r;
  const uint32_t ks = __shfl_sync(FULL, b.kst, rr);
  *rec = (uint32_t)rr;
  *j = lo + lane - ks;
}

template <typename K>
__device__ __forceinline__ K canonical_kmer(const uint64_t *wds, uint32_t j, int k);
template <>
__device__ __forceinline__ uint64_t canonical_kmer<uint64_t>(const uint64_t *wds, uint32_t j, int k) {
  uint64_t f = get_kmer<uint64_t>(wds, j, k);
  uint64_t r = revcomp64(f, k);
  return f < r ? f : r;
}
template <>
__device__ __forceinline__ u128 canonical_kmer<u128>(const uint64_t *wds, uint32_t j, int k) {
  u128 f = get_kmer<u128>(wds, j, k);
  u128 r = revcomp128(f, k);
  return f < r ? f : r;
}

// Shared arguments of the key-building kernels.
template <typename K>
struct KxArgs {
  const Chunk *chunks;
  const PieceDesc *pieces;
  int k;
  int key_bits;
  const uint32_t *group_base;  // first bucket of each bin
  const uint8_t *group_D;      // digit bits of each bin
  Mixer<K> mixer;
};

constexpr int KX_SMEM_D = 12;            // digits aggregated in shared memory up to 2^12
constexpr int KX_STASH = 1024;           // keys stashed per warp between the two sweeps

// Visits the k-mers of a chunk: warp w takes record batches w, w+8, ...;
// f(lane_ok, key) is called once per 32-k-mer step with the canonical,
// mixed key of this lane's k-mer (all lanes call f).
template <typename K, typename F>
__device__ __forceinline__ void for_chunk_keys(const KxArgs<K> &a, const Chunk &c, F f) {
  const PieceDesc pd = a.pieces[c.piece];
  const unsigned w = threadIdx.x >> 5, lane = lane_id();
  const uint64_t r_end = c.r0 + c.n_rec;
  for (uint64_t r = c.r0 + 32ull * w; r < r_end; r += 32ull * (KX_THREADS / 32)) {
    RecBatch b = load_batch(pd.index, r, r_end);
    for (uint32_t it = 0; 32 * it < b.total; ++it) {
      uint32_t rec, j;
      locate(b, it, &rec, &j);
      const uint64_t woff = __shfl_sync(FULL, b.woff, rec);
      const bool ok = 32 * it + lane < b.total;
      K key = K(0);
      if (ok) key = a.mixer.mix(canonical_kmer<K>(pd.words + woff, j, a.k));
      f(ok, key);
    }
  }
}

// a4, count pass (x = 0): per-bin histogram of the top D bits of every mixed
// canonical k-mer of the chunk's super k-mers.
template <typename K>
__global__ void __launch_bounds__(KX_THREADS)
kx0_count_kernel(KxArgs<K> a, uint32_t *__restrict__ hist) {
  __shared__ uint32_t h[1 << KX_SMEM_D];
  const Chunk c = a.chunks[blockIdx.x];
  const int D = a.group_D[c.bin];
  const uint32_t ND = 1u << D;
  uint32_t *hb = hist + a.group_base[c.bin];
  const bool in_smem = D <= KX_SMEM_D;
  if (in_smem) {
    for (uint32_t i = threadIdx.x; i < ND; i += KX_THREADS) h[i] = 0;
    __syncthreads();
  }
  const unsigned lane = lane_id();
  for_chunk_keys<K>(a, c, [&](bool ok, K key) {
    const uint32_t d = ok ? top_digit<K>(key, a.key_bits, D) : 0xFFFFFFFFu;
    if (in_smem) {
      if (ok) atomicAdd(&h[d], 1u);  // mixed keys: lanes rarely share a digit
    } else {
      const unsigned peers = __match_any_sync(FULL, d);
      if (ok && (int)lane == __ffs(peers) - 1) atomicAdd(&hb[d], (uint32_t)__popc(peers));
    }
  });
  if (in_smem) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < ND; i += KX_THREADS)
      if (h[i]) atomicAdd(&hb[i], h[i]);
  }
}

template <typename K>
struct KxScatterSmem {
  uint32_t h[1 << KX_SMEM_D];      // chunk count per digit, then running rank
  uint32_t gb[1 << KX_SMEM_D];     // chunk base per digit, relative to the bin's first key
  K stash[KX_THREADS / 32][KX_STASH];
};

// a4, scatter pass (x = 0): mixed canonical k-mers written into their (bin,
// digit) buckets.  Sweep 1 computes the keys (stashed in shared memory) and
// counts the chunk's digits; one global atomic per digit reserves space;
// sweep 2 writes every key at its place.
template <typename K>
__global__ void __launch_bounds__(KX_THREADS)
kx0_scatter_kernel(KxArgs<K> a, const uint64_t *__restrict__ bucket_base,
                   uint32_t *__restrict__ cursor, K *__restrict__ keys, uint64_t n_keys,
                   uint32_t *err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  KxScatterSmem<K> &s = *reinterpret_cast<KxScatterSmem<K> *>(smem_raw);
  const Chunk c = a.chunks[blockIdx.x];
  const int D = a.group_D[c.bin];
  const uint32_t ND = 1u << D;
  const uint32_t g0 = a.group_base[c.bin];
  const uint64_t bin_base = bucket_base[g0];
  const bool in_smem = D <= KX_SMEM_D;
  const unsigned w = threadIdx.x >> 5, lane = lane_id();
  if (in_smem) {
    for (uint32_t i = threadIdx.x; i < ND; i += KX_THREADS) s.h[i] = 0;
    __syncthreads();
  }
  uint32_t n_stashed = 0;  // per warp (uniform inside the warp)
  for_chunk_keys<K>(a, c, [&](bool ok, K key) {
    if (n_stashed < KX_STASH) s.stash[w][n_stashed + lane] = key;  // KX_STASH % 32 == 0
    n_stashed += 32;
    if (in_smem && ok) atomicAdd(&s.h[top_digit<K>(key, a.key_bits, D)], 1u);
  });
  if (in_smem) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < ND; i += KX_THREADS) {
      if (s.h[i]) s.gb[i] = (uint32_t)(bucket_base[g0 + i] - bin_base) + atomicAdd(&cursor[g0 + i], s.h[i]);
      s.h[i] = 0;
    }
    __syncthreads();
  }
  __syncwarp();
  // sweep 2: keys from the stash (recomputed past its capacity)
  const PieceDesc pd = a.pieces[c.piece];
  const uint64_t r_end = c.r0 + c.n_rec;
  uint32_t idx = 0;
  for (uint64_t r = c.r0 + 32ull * w; r < r_end; r += 32ull * (KX_THREADS / 32)) {
    RecBatch b = load_batch(pd.index, r, r_end);
    for (uint32_t it = 0; 32 * it < b.total; ++it, idx += 32) {
      const bool ok = 32 * it + lane < b.total;
      K key;
      if (idx < KX_STASH) {
        key = s.stash[w][idx + lane];
      } else {
        uint32_t rec, j;
        locate(b, it, &rec, &j);
        const uint64_t woff = __shfl_sync(FULL, b.woff, rec);
        key = ok ? a.mixer.mix(canonical_kmer<K>(pd.words + woff, j, a.k)) : K(0);
      }
      const uint32_t d = ok ? top_digit<K>(key, a.key_bits, D) : 0xFFFFFFFFu;
      uint64_t p = 0;
      if (in_smem) {
        if (ok) p = bin_base + s.gb[d] + atomicAdd(&s.h[d], 1u);
      } else {
        const unsigned peers = __match_any_sync(FULL, d);
        const int leader = __ffs(peers) - 1;
        uint64_t base = 0;
        if (ok && (int)lane == leader)
          base = bucket_base[g0 + d] + atomicAdd(&cursor[g0 + d], (uint32_t)__popc(peers));
        base = __shfl_sync(FULL, base, leader);
        p = base + __popc(peers & lanemask_lt());
      }
      if (ok) {
        if (p < n_keys) keys[p] = key; else atomicOr(err, ERR_CAPACITY);
      }
    }
  }
}

__global__ void swap_words_kernel(u128 *v, uint64_t n) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    u128 x = v[i];
    v[i] = (x << 64) | (x >> 64);  // little-endian u128 -> (high word, low word)
  }
}

inline unsigned grid_for(uint64_t n, int threads, int cap = 1 << 20) {
  uint64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (unsigned)std::min<uint64_t>(g, (uint64_t)cap);
}

// Host-side constants of the bijective key mix for key_bits-bit keys.
template <typename K>
Mixer<K> make_mixer(int key_bits) {
  Mixer<K> m;
  m.bits = key_bits;
  m.mask = key_bits >= (int)(8 * sizeof(K)) ? ~K(0) : ((K(1) << key_bits) - 1);
  K c = (K)0x9E3779B97F4A7C15ull;
  if (sizeof(K) > 8) c = (c << 64) | (K)0xD1B54A32D192ED03ull;
  c |= 1;
  K inv = c;  // Newton iteration for the inverse modulo 2^(8 sizeof K)
  for (int i = 0; i < 7; ++i) inv *= K(2) - c * inv;
  m.c = c & m.mask;
  m.cinv = inv & m.mask;
  m.s1 = (key_bits + 1) / 2;
  m.s2 = key_bits / 3 + 1;
  m.on = true;
  return m;
}

template <typename K, int IPT>
int count_tiles(Handle &h, SortScratch &ss, const TilePlan &plan, uint64_t n_keys, K *keys,
                const Mixer<K> &mixer, uint64_t *n_sv_out) {
  using SM = TileCountSmem<K, CNT_THREADS, IPT>;
  using BSM = BigSmem<K, NoVal, CNT_THREADS, BIG_IPT>;
  constexpr int TILE = CNT_THREADS * IPT;
  const uint64_t ci = h.p.cutoff_min ? h.p.cutoff_min : 1;
  const uint64_t sv_cap = n_keys / ci + TILE + 1;
  const uint32_t big_cap = (uint32_t)std::min<uint64_t>(n_keys / (TILE + 1) + 1, 0xFFFFFFF0ull);
  if (dev_ensure(ss.sv_keys, sv_cap * sizeof(K), h.st) || dev_ensure(ss.sv_counts, sv_cap * 4, h.st) ||
      dev_ensure(ss.big_list, (size_t)big_cap * 4, h.st))
    return KMC_ENOMEM;
  // counters: [0] work u32, [1] n_big u32, [2..3] pad, then u64: n_sv, n_distinct, big_keys, scratch cursor
  auto *c32 = as<uint32_t>(ss.counters);
  auto *c64 = reinterpret_cast<unsigned long long *>(c32 + 4);
  KMC_CUDA_TRY(cudaMemsetAsync(c32, 0, 64, h.st));
  CountOut<K> out;
  out.keys = as<K>(ss.sv_keys);
  out.counts = as<uint32_t>(ss.sv_counts);
  out.n = c64 + 0;
  out.cap = sv_cap;
  out.ci = ci;
  out.cx = h.p.cutoff_max;
  out.n_distinct = c64 + 1;
  out.mixer = mixer;
  out.sort_bits = (h.p.debug_flags & KMC_DEBUG_NARROW_SORT) ? 8 : kCountSortBits;
  static bool attr = false;
  if (!attr) {
    KMC_CUDA_TRY(cudaFuncSetAttribute(tile_count_kernel<K, CNT_THREADS, IPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM)));
    KMC_CUDA_TRY(cudaFuncSetAttribute(big_count_kernel<K, CNT_THREADS, BIG_IPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BSM)));
    attr = true;
  }
  int occ = 0;
  KMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, tile_count_kernel<K, CNT_THREADS, IPT>, CNT_THREADS, sizeof(SM)));
  const unsigned grid = (unsigned)std::max(1, occ) * (unsigned)h.sm_count;
  {
    StageScope sc(h, KMC_STAGE_TILE_SORT);
    tile_count_kernel<K, CNT_THREADS, IPT><<<grid, CNT_THREADS, sizeof(SM), h.st>>>(
        keys, plan, c32 + 0, out, as<uint32_t>(ss.big_list), c32 + 1, c64 + 2, big_cap,
        as<uint32_t>(h.err), (K *)nullptr); KMC_COUNT_LAUNCH();
  }
  KMC_CUDA_TRY(cudaGetLastError());
  uint32_t nbig = 0;
  unsigned long long bigk = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&nbig, c32 + 1, 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(&bigk, c64 + 2, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  h.stats.n_big_tiles = nbig;
  if (nbig) {
    if (dev_ensure(ss.big_scratch, (bigk + 1) * sizeof(K), h.st)) return KMC_ENOMEM;
    StageScope sc(h, KMC_STAGE_BIG_SORT);
    big_count_kernel<K, CNT_THREADS, BIG_IPT><<<nbig, CNT_THREADS, sizeof(BSM), h.st>>>(
        keys, plan, as<uint32_t>(ss.big_list), as<K>(ss.big_scratch), c64 + 3, out,
        as<uint32_t>(h.err)); KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  unsigned long long vals[2];
  KMC_CUDA_TRY(cudaMemcpyAsync(vals, c64, 16, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  *n_sv_out = vals[0];
  h.stats.n_distinct = vals[1];
  return check_device_error(h);
}

// Tile plan over hist[NB] (u32 counts per bucket, grouped by bin).
int plan_tiles(Handle &h, const uint32_t *hist, uint64_t NB, const uint32_t *group_base,
               uint32_t n_groups, int tile_cap, DevBuf &base, DevBuf &flags, DevBuf &fscan,
               DevBuf &tfirst, DevBuf &tmp, uint32_t **n_tiles_dev) {
  if (dev_ensure(base, (NB + 1) * 8, h.st) || dev_ensure(flags, NB * 4 + 4, h.st) ||
      dev_ensure(fscan, (NB + 1) * 8, h.st) || dev_ensure(tfirst, NB * 4 + 8, h.st) ||
      dev_ensure(tmp, scan_tmp_words(NB) * 8, h.st))
    return KMC_ENOMEM;
  KMC_CUDA_TRY(device_excl_scan_u32(hist, as<uint64_t>(base), NB, as<uint64_t>(tmp), h.st));
  const uint64_t n_seg = (NB + kGreedySegment - 1) / kGreedySegment;
  plan_greedy_flags_kernel<<<(unsigned)((n_seg + 7) / 8), 256, 0, h.st>>>(
      hist, group_base, n_groups, NB, (uint32_t)tile_cap, as<uint32_t>(flags));
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  KMC_CUDA_TRY(device_excl_scan_u32(as<uint32_t>(flags), as<uint64_t>(fscan), NB, as<uint64_t>(tmp), h.st));
  uint32_t *nt = as<uint32_t>(tfirst) + NB + 1;
  plan_emit_kernel<<<grid_for(NB, 256, 65535), 256, 0, h.st>>>(
      as<uint32_t>(flags), as<uint64_t>(fscan), NB, as<uint32_t>(tfirst), nt);
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  *n_tiles_dev = nt;
  return KMC_OK;
}

// Digit bits of a bin with n keys: about TILE/2 keys per bucket.
int digits_for(uint64_t n, int key_bits, int tile) {
  int D = 0;
  while (D < 20 && D < key_bits && (n >> D) > (uint64_t)tile / 2) ++D;
  return D;
}

template <typename K, int IPT>
int sort_phase_x0(Handle &h) {
  SortScratch &ss = h.ss;
  constexpr int TILE = CNT_THREADS * IPT;
  const uint32_t B = h.p.n_bins;
  const int k = (int)h.p.k;
  const int key_bits = 2 * k;
  const uint64_t n_keys = h.stats.n_kmer_positions;
  uint64_t max_bin = 0;
  for (uint64_t v : h.bin_kmers) max_bin = std::max(max_bin, v);
  h.stats.max_bin_kmers = max_bin;
  h.stats.n_sorted_keys = n_keys;
  // per-bin digit widths and bucket groups
  std::vector<uint32_t> gbase(B + 1);
  std::vector<uint8_t> gD(B);
  uint64_t NB = 0;
  for (uint32_t b = 0; b < B; ++b) {
    gD[b] = (uint8_t)digits_for(h.bin_kmers[b], key_bits, TILE);
    gbase[b] = (uint32_t)NB;
    NB += 1ull << gD[b];
  }
  gbase[B] = (uint32_t)NB;
  if (NB >= 0xFFFFFFF0ull) return KMC_EINVAL;
  // chunk list: per piece and bin, runs of KX_RECORDS_PER_CHUNK records
  std::vector<Chunk> chunks;
  std::vector<PieceDesc> pds;
  for (size_t p = 0; p < h.pieces.size(); ++p) {
    Piece *pc = h.pieces[p];
    pds.push_back({static_cast<const uint64_t *>(pc->index.p), static_cast<const uint64_t *>(pc->words.p)});
    const std::vector<uint64_t> &rb = pc->rec_base_host;
    for (uint32_t b = 0; b < B; ++b)
      for (uint64_t r = rb[b]; r < rb[b + 1]; r += KX_RECORDS_PER_CHUNK)
        chunks.push_back({r, (uint32_t)std::min<uint64_t>(KX_RECORDS_PER_CHUNK, rb[b + 1] - r),
                          (uint32_t)p, b, 0});
  }
  const size_t meta_bytes = (chunks.size() + 1) * sizeof(Chunk) + (pds.size() + 1) * sizeof(PieceDesc) +
                            (B + 1) * 4 + B + 64;
  if (dev_ensure(ss.counters, 64, h.st) || dev_ensure(ss.cursor, meta_bytes, h.st) ||
      dev_ensure(ss.hist, NB * 4 + 4, h.st))
    return KMC_ENOMEM;
  std::vector<uint8_t> meta(meta_bytes);
  Chunk *d_chunks = as<Chunk>(ss.cursor);
  size_t o_pd = (chunks.size() + 1) * sizeof(Chunk);
  size_t o_gb = o_pd + (pds.size() + 1) * sizeof(PieceDesc);
  size_t o_gd = o_gb + (B + 1) * 4;
  memcpy(meta.data(), chunks.data(), chunks.size() * sizeof(Chunk));
  memcpy(meta.data() + o_pd, pds.data(), pds.size() * sizeof(PieceDesc));
  memcpy(meta.data() + o_gb, gbase.data(), (B + 1) * 4);
  memcpy(meta.data() + o_gd, gD.data(), B);
  KMC_CUDA_TRY(cudaMemcpyAsync(ss.cursor.p, meta.data(), meta_bytes, cudaMemcpyHostToDevice, h.st));
  KxArgs<K> a;
  a.chunks = d_chunks;
  a.pieces = reinterpret_cast<const PieceDesc *>(static_cast<char *>(ss.cursor.p) + o_pd);
  a.k = k;
  a.key_bits = key_bits;
  a.group_base = reinterpret_cast<const uint32_t *>(static_cast<char *>(ss.cursor.p) + o_gb);
  a.group_D = reinterpret_cast<const uint8_t *>(static_cast<char *>(ss.cursor.p) + o_gd);
  a.mixer = make_mixer<K>(key_bits);
  uint32_t *hist = as<uint32_t>(ss.hist);
  KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, NB * 4, h.st));
  if (!chunks.empty()) {
    StageScope sc(h, KMC_STAGE_KX_COUNT);
    kx0_count_kernel<K><<<(unsigned)chunks.size(), KX_THREADS, 0, h.st>>>(a, hist);
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  uint32_t *n_tiles_dev = nullptr;
  int rc;
  {
    StageScope sc_plan(h, KMC_STAGE_PLAN);
    rc = plan_tiles(h, hist, NB, a.group_base, B, TILE, ss.bucket_base, ss.flags, ss.flag_scan,
                    ss.tile_first, ss.scan_tmp, &n_tiles_dev);
  }
  if (rc) return rc;
  // hist becomes the per-bucket cursor
  KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, NB * 4, h.st));
  if (dev_ensure(ss.keys, (n_keys + 1) * sizeof(K), h.st)) return KMC_ENOMEM;
  K *keys = as<K>(ss.keys);
  if (!chunks.empty()) {
    static bool attr = false;
    if (!attr) {
      KMC_CUDA_TRY(cudaFuncSetAttribute(kx0_scatter_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(KxScatterSmem<K>)));
      attr = true;
    }
    StageScope sc(h, KMC_STAGE_KX_SCATTER);
    kx0_scatter_kernel<K><<<(unsigned)chunks.size(), KX_THREADS, sizeof(KxScatterSmem<K>), h.st>>>(
        a, as<uint64_t>(ss.bucket_base), hist, keys, n_keys, as<uint32_t>(h.err));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  TilePlan plan;
  plan.bucket_base = as<uint64_t>(ss.bucket_base);
  plan.tile_first = as<uint32_t>(ss.tile_first);
  plan.n_tiles = n_tiles_dev;
  plan.group_base = a.group_base;
  plan.group_D = a.group_D;
  plan.n_groups = B;
  plan.NB = (uint32_t)NB;
  plan.key_bits = key_bits;
  uint64_t n_sv = 0;
  rc = count_tiles<K, IPT>(h, ss, plan, n_keys, keys, a.mixer, &n_sv);
  if (rc) return rc;
  uint32_t nt = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&nt, n_tiles_dev, 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaEventRecord(h.ev[2], h.st));
  // global order of the survivors (result arrays)
  if (dev_ensure(h.out_kmers, (n_sv + 1) * sizeof(K), h.st) ||
      dev_ensure(h.out_counts, (n_sv + 1) * 4, h.st))
    return KMC_ENOMEM;
  if (n_sv) {
    StageScope sc(h, KMC_STAGE_ORDER);
    KMC_CUDA_TRY(cudaMemcpyAsync(h.out_kmers.p, ss.sv_keys.p, n_sv * sizeof(K), cudaMemcpyDeviceToDevice, h.st));
    KMC_CUDA_TRY(cudaMemcpyAsync(h.out_counts.p, ss.sv_counts.p, n_sv * 4, cudaMemcpyDeviceToDevice, h.st));
    if constexpr (sizeof(K) == 8) {
      rc = sort_pairs_u64(h, as<uint64_t>(h.out_kmers), as<uint32_t>(h.out_counts), n_sv, key_bits);
    } else {
      rc = sort_pairs_u128(h, as<u128>(h.out_kmers), as<uint32_t>(h.out_counts), n_sv, key_bits);
      if (!rc) {
        swap_words_kernel<<<grid_for(n_sv, 256, 65535), 256, 0, h.st>>>(as<u128>(h.out_kmers), n_sv);
        KMC_COUNT_LAUNCH();
        KMC_CUDA_TRY(cudaGetLastError());
      }
    }
    if (rc) return rc;
  }
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  h.n_out = n_sv;
  h.stats.n_out = n_sv;
  h.stats.n_tiles = nt;
  h.stats.x_used = 0;
  return check_device_error(h);
}

}  // namespace

int sort_phase(Handle &h) {
  if (h.p.k <= 32) return sort_phase_x0<uint64_t, CNT_IPT64>(h);
  return sort_phase_x0<u128, CNT_IPT128>(h);
}

int debug_bin_keys(Handle &h, uint32_t bin, uint64_t *keys, uint64_t capacity, uint64_t *n_out,
                   uint32_t *words_per_key) {
  (void)h; (void)bin; (void)keys; (void)capacity; (void)n_out; (void)words_per_key;
  return KMC_ESTATE;
}

}  // namespace kmc
