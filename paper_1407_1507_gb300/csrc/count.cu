// Sorting phase (paper Sect. 2.3, 2.4, Fig. 2): bins of super k-mers ->
// keys -> radix sort -> run-length counting with the cutoffs -> survivors,
// then the survivors of all bins are put in global order.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "internal.h"
#include "sortlib.cuh"
#include "kx_kernels.cuh"

namespace kmc {

namespace {

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
  if constexpr (sizeof(K) > 8) c = (c << 64) | (K)0xD1B54A32D192ED03ull;
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

// scratch: NULL, or a buffer of n_keys + 2 keys free for the big tiles
template <typename K, int IPT>
int count_tiles(Handle &h, const TilePlan &plan, uint64_t n_keys, K *keys, const Mixer<K> &mixer,
                uint64_t ci, uint64_t cx, DevBuf &out_k, DevBuf &out_c, uint64_t *n_sv_out,
                K *sorted_out, K *scratch = nullptr, const SuperArgs *sup = nullptr) {
  SortScratch &ss = h.ss;
  using SM = TileCountSmem<K, CNT_THREADS, IPT>;
  using BSM = BigSmem<K, NoVal, CNT_THREADS, BIG_IPT>;
  constexpr int TILE = CNT_THREADS * IPT;
  if (ci == 0) ci = 1;
  const uint64_t sv_cap = n_keys / ci + TILE + 1;
  const uint32_t big_cap = (uint32_t)std::min<uint64_t>(n_keys / (TILE + 1) + 1, 0xFFFFFFF0ull);
  if (dev_ensure(out_k, sv_cap * sizeof(K), h.st) || dev_ensure(out_c, sv_cap * 4, h.st) ||
      dev_ensure(ss.big_list, (size_t)big_cap * 4, h.st))
    return KMC_ENOMEM;
  // counters: [0] work u32, [1] n_big u32, [2..3] pad, then u64: n_sv, n_distinct, big_keys, scratch cursor
  auto *c32 = as<uint32_t>(ss.counters);
  auto *c64 = reinterpret_cast<unsigned long long *>(c32 + 4);
  KMC_CUDA_TRY(cudaMemsetAsync(c32, 0, 64, h.st));
  CountOut<K> out;
  out.keys = as<K>(out_k);
  out.counts = as<uint32_t>(out_c);
  out.n = c64 + 0;
  out.cap = sv_cap;
  out.ci = ci;
  out.cx = cx;
  out.n_distinct = c64 + 1;
  out.mixer = mixer;
  out.sort_bits = (h.p.debug_flags & KMC_DEBUG_NARROW_SORT) ? 8 : kCountSortBits;
  out.slots = nullptr;
  out.bins_per_slot = 1;
  // tiles are grouped (one radix step + grouping by value) unless the sorted
  // keys are asked for or the narrow-sort check is on
  constexpr int GIPT = TILE / GRP_THREADS;
  using GSM = TileGroupSmem<K, GRP_THREADS, GIPT>;
  const bool grouped = !sorted_out && out.sort_bits == kCountSortBits;
  static DeviceOnce attr;
  if (!attr.done()) {
    KMC_CUDA_TRY(cudaFuncSetAttribute(tile_count_kernel<K, CNT_THREADS, IPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM)));
    KMC_CUDA_TRY(cudaFuncSetAttribute(tile_group_kernel<K, GRP_THREADS, GIPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(GSM)));
    KMC_CUDA_TRY(cudaFuncSetAttribute(big_count_kernel<K, CNT_THREADS, BIG_IPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BSM)));
    attr.set();
  }
  int occ = 0;
  // 64-bit keys below 2^62 are counted through a hash table per tile
  constexpr int HTHREADS = HASH_THREADS, HIPT = TILE / HTHREADS;
  using HSM = TileHashSmem<HTHREADS, HIPT>;
  const bool hashed = grouped && sizeof(K) == 8 && plan.key_bits <= 62;
  if constexpr (sizeof(K) == 8) if (hashed) {
    static DeviceOnce hattr;
    if (!hattr.done()) {
      KMC_CUDA_TRY(cudaFuncSetAttribute(tile_hash_kernel<HTHREADS, HIPT>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(HSM)));
      hattr.set();
    }
    if (dev_ensure(ss.tile_desc, ((size_t)plan.NB + 1) * sizeof(TileDesc), h.st)) return KMC_ENOMEM;
    TilePlan gplan = plan;
    gplan.desc = as<TileDesc>(ss.tile_desc);
    StageScope sc(h, KMC_STAGE_TILE_SORT);
    tile_desc_kernel<<<(unsigned)std::min<uint64_t>((plan.NB + 255) / 256, 4096), 256, 0, h.st>>>(
        plan, as<TileDesc>(ss.tile_desc));
    KMC_COUNT_LAUNCH();
    int hocc = 0;
    KMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&hocc, tile_hash_kernel<HTHREADS, HIPT>,
                                                               HTHREADS, sizeof(HSM)));
    tile_hash_kernel<HTHREADS, HIPT><<<(unsigned)std::max(1, hocc) * h.sm_count, HTHREADS, sizeof(HSM), h.st>>>(
        keys, gplan, c32 + 0, out, as<uint32_t>(ss.big_list), c32 + 1, c64 + 2, big_cap,
        as<uint32_t>(h.err)); KMC_COUNT_LAUNCH();
    if (sup && sup->n_list) {
      // the fused bins: one pass over each super bucket (same survivor list)
      static DeviceOnce sattr;
      if (!sattr.done()) {
        KMC_CUDA_TRY(cudaFuncSetAttribute(super_hash_kernel<SUPER_THREADS>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)sizeof(SuperHashSmem)));
        sattr.set();
      }
      int socc = 0;
      KMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&socc, super_hash_kernel<SUPER_THREADS>,
                                                                 SUPER_THREADS, sizeof(SuperHashSmem)));
      SuperArgs sa = *sup;
      sa.work = c32 + 2;
      const unsigned grid = (unsigned)std::min<uint64_t>((uint64_t)std::max(1, socc) * h.sm_count, sa.n_list);
      super_hash_kernel<SUPER_THREADS><<<grid, SUPER_THREADS, sizeof(SuperHashSmem), h.st>>>(
          sa, out, as<uint32_t>(h.err));
      KMC_COUNT_LAUNCH();
    }
  }
  if (!hashed && grouped) {
    KMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, tile_group_kernel<K, GRP_THREADS, GIPT>, GRP_THREADS, sizeof(GSM)));
    // tile ranges first: a CTA then takes a tile with one load
    if (dev_ensure(ss.tile_desc, ((size_t)plan.NB + 1) * sizeof(TileDesc), h.st)) return KMC_ENOMEM;
    TilePlan gplan = plan;
    gplan.desc = as<TileDesc>(ss.tile_desc);
    gplan.debug = (h.p.debug_flags & KMC_DEBUG_WAIT_TIMEOUT) ? 1u : 0u;
    StageScope sc(h, KMC_STAGE_TILE_SORT);
    tile_desc_kernel<<<(unsigned)std::min<uint64_t>((plan.NB + 255) / 256, 4096), 256, 0, h.st>>>(
        plan, as<TileDesc>(ss.tile_desc));
    KMC_COUNT_LAUNCH();
    tile_group_kernel<K, GRP_THREADS, GIPT><<<(unsigned)std::max(1, occ) * h.sm_count, GRP_THREADS,
                                              sizeof(GSM), h.st>>>(
        keys, gplan, c32 + 0, out, as<uint32_t>(ss.big_list), c32 + 1, c64 + 2, big_cap,
        as<uint32_t>(h.err)); KMC_COUNT_LAUNCH();
  } else if (!hashed) {
    KMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ, tile_count_kernel<K, CNT_THREADS, IPT>, CNT_THREADS, sizeof(SM)));
    StageScope sc(h, KMC_STAGE_TILE_SORT);
    tile_count_kernel<K, CNT_THREADS, IPT><<<(unsigned)std::max(1, occ) * h.sm_count, CNT_THREADS,
                                             sizeof(SM), h.st>>>(
        keys, plan, c32 + 0, out, as<uint32_t>(ss.big_list), c32 + 1, c64 + 2, big_cap,
        as<uint32_t>(h.err), sorted_out); KMC_COUNT_LAUNCH();
  }
  KMC_CUDA_TRY(cudaGetLastError());
  uint32_t nbig = 0;
  unsigned long long bigk = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&nbig, c32 + 1, 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(&bigk, c64 + 2, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  h.stats.n_big_tiles += nbig;
  if (nbig && grouped) {
    // big tiles: split into sub-buckets at their own positions in scratch
    using BGS = BigGroupSmem<K, GRP_THREADS, GIPT, GIPT>;
    if (!scratch) {
      if (dev_ensure(ss.big_scratch, (n_keys + 2) * sizeof(K), h.st)) return KMC_ENOMEM;
      scratch = as<K>(ss.big_scratch);
    }
    static DeviceOnce battr;
    if (!battr.done()) {
      KMC_CUDA_TRY(cudaFuncSetAttribute(big_group_kernel<K, GRP_THREADS, GIPT, GIPT>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BGS)));
      battr.set();
    }
    StageScope sc(h, KMC_STAGE_BIG_SORT);
    big_group_kernel<K, GRP_THREADS, GIPT, GIPT><<<std::min<uint32_t>(nbig, (uint32_t)h.sm_count), GRP_THREADS,
                                                   sizeof(BGS), h.st>>>(
        keys, plan, as<uint32_t>(ss.big_list), c32 + 1, scratch, out, plan.key_bits, as<uint32_t>(h.err));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  } else if (nbig) {
    if (dev_ensure(ss.big_scratch, (bigk + 1) * sizeof(K), h.st)) return KMC_ENOMEM;
    StageScope sc(h, KMC_STAGE_BIG_SORT);
    big_count_kernel<K, CNT_THREADS, BIG_IPT><<<nbig, CNT_THREADS, sizeof(BSM), h.st>>>(
        keys, plan, as<uint32_t>(ss.big_list), c32 + 1, as<K>(ss.big_scratch), c64 + 3, out,
        as<uint32_t>(h.err), sorted_out); KMC_COUNT_LAUNCH();
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

template <typename K>
void save_debug_mixer(Handle &h, const Mixer<K> &m) {
  h.ss.dbg_key_bytes = (int)sizeof(K);
  h.ss.dbg_mix[0] = (uint64_t)m.c;
  h.ss.dbg_mix[1] = (uint64_t)((u128)m.c >> 64);
  h.ss.dbg_mix[2] = (uint64_t)m.cinv;
  h.ss.dbg_mix[3] = (uint64_t)((u128)m.cinv >> 64);
  h.ss.dbg_mix[4] = (uint64_t)m.mask;
  h.ss.dbg_mix[5] = (uint64_t)((u128)m.mask >> 64);
  h.ss.dbg_mix[6] = (uint64_t)m.bits | ((uint64_t)m.s1 << 16) | ((uint64_t)m.s2 << 32);
}

// Per-bin bucket groups and the chunk list of the bins' records; uploads
// both with the piece table.  keys_per_kmer scales the bins' k-mer counts
// to the expected number of keys (1 for k-mers, ~0.6 for (k,x)-mers).
struct SortMeta {
  KxArgs<uint64_t> dummy;
  size_t n_chunks = 0;
  uint64_t NB = 0;
  const Chunk *chunks = nullptr;
  const PieceDesc *pieces = nullptr;
  const uint32_t *group_base = nullptr;
  const uint8_t *group_D = nullptr;
  // generate + sweep path (x = 0)
  bool gen = false;
  size_t n_units = 0;
  const PartUnit *units = nullptr;
  const uint64_t *bin_key_base = nullptr;  // first key of each bin in the generated array
  const uint32_t *sgroup_base = nullptr;   // first super bucket of each bin [bins + 1]
  uint32_t n_super = 0;
  // device scratch (zeroed by the caller where noted)
  unsigned long long *bin_fill = nullptr;      // keys written per bin (zeroed)
  uint32_t *super_hist = nullptr;              // keys per super bucket (zeroed)
  unsigned long long *super_base = nullptr;    // scan of super_hist [n_super + 1]
  unsigned long long *super_cursor = nullptr;  // keys placed per super bucket (zeroed)
  // bins counted straight from their super buckets (super_hash_kernel)
  const uint8_t *fused = nullptr;    // per bin, 1 if fused [bins]
  const uint32_t *fused_list = nullptr;  // their super buckets, biggest bins first
  uint32_t n_fused_list = 0;
};

// Bins whose super buckets hold at most kFuseMaxKeys keys (expected, 256 of
// them) are counted by super_hash_kernel; a fused bin gets the fewest upper
// digit bits that leave about kFuseTargetKeys keys per super bucket.
#ifndef KMC_FUSE_MAX_KEYS
#define KMC_FUSE_MAX_KEYS 32768
#endif
#ifndef KMC_FUSE_TARGET_KEYS
#define KMC_FUSE_TARGET_KEYS 4096
#endif
constexpr uint64_t kFuseMaxKeys = KMC_FUSE_MAX_KEYS;
constexpr uint64_t kFuseTargetKeys = KMC_FUSE_TARGET_KEYS;

// unit_keys > 0 asks for the generate + sweep path (x = 0, units of
// unit_keys keys); it is taken when the bins' k-mers add up.
// Largest i in [0, n) with first[i] <= x (first[0] <= x < first[n]).
__device__ __forceinline__ uint32_t meta_find(const uint32_t *first, uint32_t n, uint32_t x) {
  uint32_t lo = 0, hi = n;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (first[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Chunk c of the (piece, bin) pair i with cpos[i] <= c < cpos[i+1]: records
// from rec_base[p][b] + (c - cpos[i]) * KX_RECORDS_PER_CHUNK on.
__global__ void meta_chunks_kernel(const uint64_t *const *rec_base, const uint32_t *cpos, uint32_t P,
                                   uint32_t B, uint32_t n_chunks, Chunk *chunks) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < n_chunks; c += gridDim.x * blockDim.x) {
    const uint32_t i = meta_find(cpos, P * B, c);
    const uint32_t p = i / B, b = i % B;
    const uint64_t r = rec_base[p][b] + (uint64_t)(c - cpos[i]) * KX_RECORDS_PER_CHUNK;
    const uint64_t r1 = rec_base[p][b + 1];
    chunks[c] = Chunk{r, (uint32_t)(r1 - r < KX_RECORDS_PER_CHUNK ? r1 - r : KX_RECORDS_PER_CHUNK), p, b, 0u};
  }
}

// Unit u of bin b with ubase[b] <= u < ubase[b+1]: keys from
// kbase[b] + (u - ubase[b]) * unit_keys on.
__global__ void meta_units_kernel(const uint64_t *kbase, const uint32_t *ubase, uint32_t B,
                                  uint32_t unit_keys, uint32_t n_units, PartUnit *units) {
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < n_units; u += gridDim.x * blockDim.x) {
    const uint32_t b = meta_find(ubase, B, u);
    const uint64_t o = kbase[b] + (uint64_t)(u - ubase[b]) * unit_keys, k1 = kbase[b + 1];
    units[u] = PartUnit{o, (uint32_t)(k1 - o < unit_keys ? k1 - o : unit_keys), b};
  }
}

// Only the bins of the wave [wb0, wb1) take part (the others are empty).
int build_meta(Handle &h, int key_bits, int tile, double keys_per_kmer, SortMeta *m,
               uint32_t unit_keys = 0, uint32_t wb0 = 0, uint32_t wb1 = ~0u, bool fuse = false) {
  SortScratch &ss = h.ss;
  const uint32_t B = h.p.n_bins;
  if (wb1 > B) wb1 = B;
  std::vector<uint64_t> bk(B, 0);
  for (uint32_t b = wb0; b < wb1; ++b) bk[b] = h.bin_kmers[b];
  std::vector<uint32_t> gbase(B + 1);
  std::vector<uint8_t> gD(B);
  uint64_t NB = 0;
  std::vector<uint8_t> fused(B, 0);
  uint64_t bk_sum = 0;
  for (uint32_t b = 0; b < B; ++b) bk_sum += bk[b];
  // the generate + sweep path needs every k-mer position in the bins' counts
  bool gen = unit_keys > 0 && !(wb0 == 0 && wb1 == B && bk_sum != h.stats.n_kmer_positions);
  const bool may_fuse = fuse && gen;
  for (uint32_t b = 0; b < B; ++b) {
    gD[b] = (uint8_t)digits_for((uint64_t)(bk[b] * keys_per_kmer), key_bits, tile);
    // the two sweeps place at most SWEEP_BITS_MAX digit bits; bigger bins
    // get bigger buckets, which the big-tile pass splits further
    if (unit_keys) gD[b] = (uint8_t)std::min<int>(gD[b], SWEEP_BITS_MAX);
    if (may_fuse && bk[b] && (bk[b] + 255) / 256 <= kFuseMaxKeys) {
      int S = 0;
      while (S < SWEEP_UPPER && S < key_bits && (bk[b] + (1ull << S) - 1) >> S > kFuseTargetKeys) ++S;
      gD[b] = (uint8_t)S;
      fused[b] = 1;
    }
    gbase[b] = (uint32_t)NB;
    NB += 1ull << gD[b];
  }
  gbase[B] = (uint32_t)NB;
  if (NB >= 0xFFFFFFF0ull) return KMC_EINVAL;
  // per bin: first key, first super bucket, first unit; per (piece, bin):
  // first chunk.  The chunks and units themselves are written on the device.
  std::vector<uint64_t> kbase(B + 1, 0);
  std::vector<uint32_t> sbase(B + 1, 0), ubase(B + 1, 0);
  if (gen) {
    for (uint32_t b = 0; b < B; ++b) {
      kbase[b + 1] = kbase[b] + bk[b];
      sbase[b + 1] = sbase[b] + (1u << std::min<int>(gD[b], SWEEP_UPPER));
      ubase[b + 1] = ubase[b] + (uint32_t)((bk[b] + unit_keys - 1) / unit_keys);
    }
  }
  const uint32_t n_units = gen ? ubase[B] : 0;
  const uint32_t n_super = gen ? sbase[B] : 0;
  // super buckets of the fused bins, the biggest bins first (balance)
  std::vector<uint32_t> flist;
  if (gen && may_fuse) {
    std::vector<uint32_t> order;
    for (uint32_t b = 0; b < B; ++b)
      if (fused[b]) order.push_back(b);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return bk[x] > bk[y]; });
    for (uint32_t b : order) {
      for (uint32_t q = sbase[b]; q < sbase[b + 1]; ++q) flist.push_back(q);
      h.stats.n_fused_keys += bk[b];
    }
  }
  const uint32_t n_flist = (uint32_t)flist.size();
  const size_t P = h.pieces.size();
  std::vector<PieceDesc> pds;
  std::vector<const uint64_t *> rbp;
  std::vector<uint32_t> cpos(P * B + 1, 0);
  for (size_t p = 0; p < P; ++p) {
    Piece *pc = h.pieces[p];
    pds.push_back({pc->d_index, pc->d_words});
    rbp.push_back(static_cast<const uint64_t *>(pc->rec_base.p));
    const std::vector<uint64_t> &rb = pc->rec_base_host;
    for (uint32_t b = 0; b < B; ++b) {
      const uint64_t nr = (b >= wb0 && b < wb1) ? rb[b + 1] - rb[b] : 0;
      cpos[p * B + b + 1] = cpos[p * B + b] + (uint32_t)((nr + KX_RECORDS_PER_CHUNK - 1) / KX_RECORDS_PER_CHUNK);
    }
  }
  const uint32_t n_chunks = cpos[P * B];
  auto up16 = [](size_t x) { return (x + 15) & ~(size_t)15; };
  // uploaded part
  const size_t o_pd = 0;
  const size_t o_gb = o_pd + up16((P + 1) * sizeof(PieceDesc));
  const size_t o_gd = o_gb + up16((B + 1) * 4);
  const size_t o_kb = o_gd + up16(B + 1);
  const size_t o_sg = o_kb + up16((B + 1) * 8);
  const size_t o_ub = o_sg + up16((B + 1) * 4);
  const size_t o_cp = o_ub + up16((B + 1) * 4);
  const size_t o_rb = o_cp + up16((P * B + 1) * 4);
  const size_t o_fu = o_rb + up16((P + 1) * 8);
  const size_t o_fl = o_fu + up16(B + 1);
  const size_t o_up = o_fl + up16(((size_t)n_flist + 1) * 4);  // device-only from here on
  const size_t o_ch = o_up;
  const size_t o_un = o_ch + up16(((size_t)n_chunks + 1) * sizeof(Chunk));
  const size_t o_bf = o_un + up16(((size_t)n_units + 1) * sizeof(PartUnit));
  const size_t o_sh = o_bf + up16((B + 1) * 8);
  const size_t o_sc = o_sh + up16((n_super + 1) * 4);
  const size_t o_sb = o_sc + up16((n_super + 1) * 8);
  const size_t meta_bytes = o_sb + up16((n_super + 2) * 8);
  if (dev_ensure(ss.counters, 64, h.st) || dev_ensure(ss.cursor, meta_bytes, h.st) ||
      dev_ensure(ss.hist, NB * 4 + 4, h.st))
    return KMC_ENOMEM;
  // staged in a pinned buffer; the previous upload from it has finished
  // before it is rewritten
  if (ss.meta_done) KMC_CUDA_TRY(cudaEventSynchronize(ss.meta_done));
  if (ss.meta_host_cap < o_up) {
    if (ss.meta_host) cudaFreeHost(ss.meta_host);
    ss.meta_host = nullptr;
    ss.meta_host_cap = 0;
    if (host_alloc(&ss.meta_host, o_up + (o_up >> 2), cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      return KMC_ENOMEM;
    }
    ss.meta_host_cap = o_up + (o_up >> 2);
  }
  if (!ss.meta_done) KMC_CUDA_TRY(cudaEventCreateWithFlags(&ss.meta_done, cudaEventDisableTiming));
  uint8_t *meta = static_cast<uint8_t *>(ss.meta_host);
  memcpy(meta + o_pd, pds.data(), P * sizeof(PieceDesc));
  memcpy(meta + o_gb, gbase.data(), (B + 1) * 4);
  memcpy(meta + o_gd, gD.data(), B);
  memcpy(meta + o_kb, kbase.data(), (B + 1) * 8);
  memcpy(meta + o_sg, sbase.data(), (B + 1) * 4);
  memcpy(meta + o_ub, ubase.data(), (B + 1) * 4);
  memcpy(meta + o_cp, cpos.data(), (P * B + 1) * 4);
  memcpy(meta + o_rb, rbp.data(), P * 8);
  memcpy(meta + o_fu, fused.data(), B);
  if (n_flist) memcpy(meta + o_fl, flist.data(), (size_t)n_flist * 4);
  KMC_CUDA_TRY(cudaMemcpyAsync(ss.cursor.p, meta, o_up, cudaMemcpyHostToDevice, h.st));
  KMC_CUDA_TRY(cudaEventRecord(ss.meta_done, h.st));
  char *base = static_cast<char *>(ss.cursor.p);
  m->n_chunks = n_chunks;
  m->NB = NB;
  m->chunks = reinterpret_cast<const Chunk *>(base + o_ch);
  m->pieces = reinterpret_cast<const PieceDesc *>(base + o_pd);
  m->group_base = reinterpret_cast<const uint32_t *>(base + o_gb);
  m->group_D = reinterpret_cast<const uint8_t *>(base + o_gd);
  m->gen = gen;
  m->n_units = n_units;
  m->units = reinterpret_cast<const PartUnit *>(base + o_un);
  m->bin_key_base = reinterpret_cast<const uint64_t *>(base + o_kb);
  m->sgroup_base = reinterpret_cast<const uint32_t *>(base + o_sg);
  m->n_super = n_super;
  m->bin_fill = reinterpret_cast<unsigned long long *>(base + o_bf);
  m->super_hist = reinterpret_cast<uint32_t *>(base + o_sh);
  m->super_cursor = reinterpret_cast<unsigned long long *>(base + o_sc);
  m->super_base = reinterpret_cast<unsigned long long *>(base + o_sb);
  m->fused = n_flist ? reinterpret_cast<const uint8_t *>(base + o_fu) : nullptr;
  m->fused_list = reinterpret_cast<const uint32_t *>(base + o_fl);
  m->n_fused_list = n_flist;
  if (n_chunks) {
    meta_chunks_kernel<<<std::min<uint32_t>((n_chunks + 255) / 256, 4096), 256, 0, h.st>>>(
        reinterpret_cast<const uint64_t *const *>(base + o_rb), reinterpret_cast<const uint32_t *>(base + o_cp),
        (uint32_t)P, B, n_chunks, reinterpret_cast<Chunk *>(base + o_ch));
    KMC_COUNT_LAUNCH();
  }
  if (n_units) {
    meta_units_kernel<<<std::min<uint32_t>((n_units + 255) / 256, 4096), 256, 0, h.st>>>(
        reinterpret_cast<const uint64_t *>(base + o_kb), reinterpret_cast<const uint32_t *>(base + o_ub), B,
        unit_keys, n_units, reinterpret_cast<PartUnit *>(base + o_un));
    KMC_COUNT_LAUNCH();
  }
  KMC_CUDA_TRY(cudaGetLastError());
  if (gen)  // fill counters, super histogram and cursors start at zero
    KMC_CUDA_TRY(cudaMemsetAsync(base + o_bf, 0, o_sb - o_bf, h.st));
  ss.dbg_group_base = gbase;
  return KMC_OK;
}

// a7: survivors (canonical k-mers of type K0, counts) into the result arrays,
// ordered by k-mer value.
template <typename K0>
int order_result(Handle &h, DevBuf &sv_k, DevBuf &sv_c, uint64_t n_sv, int k) {
  KMC_CUDA_TRY(cudaEventRecord(h.ev[2], h.st));
  if (dev_ensure(h.out_kmers, (n_sv + 1) * sizeof(K0), h.st) ||
      dev_ensure(h.out_counts, (n_sv + 1) * 4, h.st))
    return KMC_ENOMEM;
  int rc = KMC_OK;
  if (n_sv) {
    StageScope sc(h, KMC_STAGE_ORDER);
    // survivors -> result arrays in k-mer order (the survivor arrays are scratch then)
    if constexpr (sizeof(K0) == 8) {
      rc = sort_pairs_to_u64(h, as<uint64_t>(sv_k), as<uint32_t>(sv_c), n_sv, 2 * k, as<uint64_t>(h.out_kmers),
                             as<uint32_t>(h.out_counts));
    } else {
      rc = sort_pairs_to_u128(h, as<u128>(sv_k), as<uint32_t>(sv_c), n_sv, 2 * k, as<u128>(h.out_kmers),
                              as<uint32_t>(h.out_counts));
      if (!rc) {
        swap_words_kernel<<<grid_for(n_sv, 256, 65535), 256, 0, h.st>>>(as<u128>(h.out_kmers), n_sv);
        KMC_COUNT_LAUNCH();
        KMC_CUDA_TRY(cudaGetLastError());
      }
    }
  }
  if (rc) return rc;
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  h.n_out = n_sv;
  h.stats.n_out = n_sv;
  return check_device_error(h);
}

// One wave: the bins [wb0, wb1) with n_keys k-mers, counted into
// (ss.sv_keys, ss.sv_counts); *n_sv receives the survivors.
template <typename K, int IPT>
int sort_wave_x0(Handle &h, uint32_t wb0, uint32_t wb1, uint64_t n_keys, uint64_t *n_sv_out) {
  SortScratch &ss = h.ss;
  constexpr int TILE = CNT_THREADS * IPT;
  const int k = (int)h.p.k;
  const int key_bits = 2 * k;
  SortMeta meta;
  // keys below 2^62 counted by hashing (not when the sorted keys are kept or
  // the narrow-sort check is on) may skip the lower sweep
  const bool fuse = sizeof(K) == 8 && key_bits <= 62 &&
                    !(h.p.debug_flags & (KMC_DEBUG_KEEP_KEYS | KMC_DEBUG_NARROW_SORT));
  int rc = build_meta(h, key_bits, TILE, 1.0, &meta, SweepTraits<K>::TILE, wb0, wb1, fuse);
  if (rc) return rc;
  KxArgs<K> a;
  a.n_chunks_dyn = nullptr;
  a.noncanonical = h.p.canonical ? 0 : 1;
  a.chunks = meta.chunks;
  a.pieces = meta.pieces;
  a.k = k;
  a.key_bits = key_bits;
  a.group_base = meta.group_base;
  a.group_D = meta.group_D;
  a.mixer = make_mixer<K>(key_bits);
  save_debug_mixer(h, a.mixer);
  const uint64_t NB = meta.NB;
  uint32_t *hist = as<uint32_t>(ss.hist);
  if (dev_ensure(ss.keys, (n_keys + 2) * sizeof(K), h.st)) return KMC_ENOMEM;  // 16 B slack
  K *keys = as<K>(ss.keys);    // the keys the tiles are counted from
  K *scratch = nullptr;        // free space for the big tiles
  if (meta.n_chunks && meta.gen) {
    // keys built once, into their bins' ranges; upper digits counted
    if (dev_ensure(ss.keys_gen, (n_keys + 2) * sizeof(K), h.st)) return KMC_ENOMEM;
    K *gen_keys = as<K>(ss.keys_gen);
    {
      StageScope sc(h, KMC_STAGE_KX_COUNT);
      if (a.noncanonical)
        kx0_gen_kernel<K, true><<<(unsigned)meta.n_chunks, KX_THREADS, 0, h.st>>>(
            a, meta.sgroup_base, meta.super_hist, meta.bin_key_base, meta.bin_fill, gen_keys, n_keys,
            as<uint32_t>(h.err));
      else
        kx0_gen_kernel<K, false><<<(unsigned)meta.n_chunks, KX_THREADS, 0, h.st>>>(
            a, meta.sgroup_base, meta.super_hist, meta.bin_key_base, meta.bin_fill, gen_keys, n_keys,
            as<uint32_t>(h.err));
      KMC_COUNT_LAUNCH();
      KMC_CUDA_TRY(cudaGetLastError());
    }
    if (dev_ensure(ss.scan_tmp, scan_tmp_words(meta.n_super) * 8, h.st)) return KMC_ENOMEM;
    KMC_CUDA_TRY(device_excl_scan_u32(meta.super_hist, reinterpret_cast<uint64_t *>(meta.super_base),
                                      meta.n_super, as<uint64_t>(ss.scan_tmp), h.st));
    SweepArgs<K> sa;
    sa.key_bits = key_bits;
    sa.n_keys = n_keys;
    sa.group_D = meta.group_D;
    sa.group_base = meta.group_base;
    sa.sgroup_base = meta.sgroup_base;
    sa.n_bins = h.p.n_bins;
    sa.super_base = meta.super_base;
    sa.super_cursor = meta.super_cursor;
    sa.fine_hist = hist;
    sa.units = meta.units;
    sa.n_units = (uint32_t)meta.n_units;
    sa.n_super = meta.n_super;
    sa.err = as<uint32_t>(h.err);
    sa.fused = meta.fused;
    static DeviceOnce attr;
    if (!attr.done()) {
      KMC_CUDA_TRY(cudaFuncSetAttribute(kx0_sweep_kernel<K, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(SweepSmem<K>)));
      KMC_CUDA_TRY(cudaFuncSetAttribute(kx0_sweep_kernel<K, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(SweepSmem<K>)));
      attr.set();
    }
    StageScope sc(h, KMC_STAGE_KX_SCATTER);
    // upper digits: generated keys -> super buckets (in ss.keys)
    sa.in = gen_keys;
    sa.out = keys;
    kx0_sweep_kernel<K, 0><<<(unsigned)std::min<uint64_t>(2ull * h.sm_count, meta.n_units), SWEEP_THREADS,
                             sizeof(SweepSmem<K>), h.st>>>(sa);
    KMC_COUNT_LAUNCH();
    // lower digits: super buckets -> final buckets (back in keys_gen)
    sa.in = keys;
    sa.out = gen_keys;
    kx0_sweep_kernel<K, 1><<<meta.n_super, SWEEP_THREADS, sizeof(SweepSmem<K>), h.st>>>(sa);
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
    scratch = keys;
    keys = gen_keys;
  } else if (meta.n_chunks) {
    KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, NB * 4, h.st));
    StageScope sc(h, KMC_STAGE_KX_COUNT);
    kx0_count_kernel<K><<<(unsigned)meta.n_chunks, KX_THREADS, 0, h.st>>>(a, hist);
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  uint32_t *n_tiles_dev = nullptr;
  {
    StageScope sc_plan(h, KMC_STAGE_PLAN);
    rc = plan_tiles(h, hist, NB, a.group_base, h.p.n_bins, TILE, ss.bucket_base, ss.flags,
                    ss.flag_scan, ss.tile_first, ss.scan_tmp, &n_tiles_dev);
  }
  if (rc) return rc;
  if (meta.n_chunks && !meta.gen) {
    KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, NB * 4, h.st));  // hist becomes the per-bucket cursor
    static DeviceOnce attr;
    if (!attr.done()) {
      KMC_CUDA_TRY(cudaFuncSetAttribute(kx0_scatter_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(KxScatterSmem<K>)));
      attr.set();
    }
    StageScope sc(h, KMC_STAGE_KX_SCATTER);
    kx0_scatter_kernel<K><<<(unsigned)meta.n_chunks, KX_THREADS, sizeof(KxScatterSmem<K>), h.st>>>(
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
  plan.n_groups = h.p.n_bins;
  plan.NB = (uint32_t)NB;
  plan.key_bits = key_bits;
  plan.skip_group = meta.fused;
  K *sorted_out = nullptr;
  if (h.p.debug_flags & KMC_DEBUG_KEEP_KEYS) {
    if (dev_ensure(ss.sorted_keys, (n_keys + 1) * sizeof(K), h.st)) return KMC_ENOMEM;
    sorted_out = as<K>(ss.sorted_keys);
  }
  SuperArgs sup{};
  if (meta.gen && meta.n_fused_list) {
    // the fused bins' keys stay where the upper sweep put them (scratch)
    sup.keys = reinterpret_cast<const uint64_t *>(scratch);
    sup.super_base = meta.super_base;
    sup.list = meta.fused_list;
    sup.n_list = meta.n_fused_list;
  }
  rc = count_tiles<K, IPT>(h, plan, n_keys, keys, a.mixer, h.p.cutoff_min, h.p.cutoff_max,
                           ss.sv_keys, ss.sv_counts, n_sv_out, sorted_out, scratch,
                           sup.n_list ? &sup : nullptr);
  if (rc) return rc;
  uint32_t nt = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&nt, n_tiles_dev, 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  h.stats.n_tiles += nt;
  return KMC_OK;
}

// x = 0.  Without a device budget the bins form one wave; with one, waves
// of consecutive bins whose keys fit a quarter of the budget per key buffer
// are sorted one after the other and their survivors gathered.
template <typename K, int IPT>
int sort_phase_x0(Handle &h) {
  SortScratch &ss = h.ss;
  constexpr int TILE = CNT_THREADS * IPT;
  const uint32_t B = h.p.n_bins;
  h.stats.n_sorted_keys = h.stats.n_kmer_positions;
  h.stats.n_fused_keys = 0;
  h.stats.n_big_tiles = 0;
  h.stats.n_tiles = 0;
  h.stats.x_used = 0;
  std::vector<uint32_t> cut{0};
  std::vector<uint64_t> wkeys;
  {
    const uint64_t cap = h.p.device_budget ? std::max<uint64_t>(1, h.p.device_budget / 4 / sizeof(K))
                                           : ~0ull;
    uint64_t acc = 0;
    for (uint32_t b = 0; b < B; ++b) {
      if (b > cut.back() && acc + h.bin_kmers[b] > cap) {
        cut.push_back(b);
        wkeys.push_back(acc);
        acc = 0;
      }
      acc += h.bin_kmers[b];
    }
    cut.push_back(B);
    wkeys.push_back(acc);
  }
  const size_t n_waves = wkeys.size();
  h.stats.n_waves = (uint32_t)n_waves;
  if (n_waves == 1) {
    uint64_t n_sv = 0;
    int rc = sort_wave_x0<K, IPT>(h, 0, B, wkeys[0], &n_sv);
    if (rc) return rc;
    return order_result<K>(h, ss.sv_keys, ss.sv_counts, n_sv, (int)h.p.k);
  }
  // gather the waves' survivors
  const uint64_t ci = h.p.cutoff_min ? h.p.cutoff_min : 1;
  const uint64_t acc_cap = h.stats.n_kmer_positions / ci + n_waves * (TILE + 1) + 1;
  if (dev_ensure(ss.acc_keys, acc_cap * sizeof(K), h.st) || dev_ensure(ss.acc_counts, acc_cap * 4, h.st))
    return KMC_ENOMEM;
  uint64_t total = 0, distinct = 0;
  for (size_t w = 0; w < n_waves; ++w) {
    if (!wkeys[w]) continue;
    uint64_t n_sv = 0;
    int rc = sort_wave_x0<K, IPT>(h, cut[w], cut[w + 1], wkeys[w], &n_sv);
    if (rc) return rc;
    distinct += h.stats.n_distinct;
    if (total + n_sv > acc_cap) return KMC_ENOMEM;
    KMC_CUDA_TRY(cudaMemcpyAsync(as<K>(ss.acc_keys) + total, ss.sv_keys.p, n_sv * sizeof(K),
                                 cudaMemcpyDeviceToDevice, h.st));
    KMC_CUDA_TRY(cudaMemcpyAsync(as<uint32_t>(ss.acc_counts) + total, ss.sv_counts.p, n_sv * 4,
                                 cudaMemcpyDeviceToDevice, h.st));
    total += n_sv;
  }
  h.stats.n_distinct = distinct;
  return order_result<K>(h, ss.acc_keys, ss.acc_counts, total, (int)h.p.k);
}

constexpr int WCNT_IPT64 = 16;
constexpr int WCNT_IPT128 = 8;

// x > 0: level 1 sorts and counts the (k,x)-mers of every bin (keys of type
// K1); level 2 expands the distinct (k,x)-mers into weighted k-mers (type
// K0), sorts them and counts with the cutoffs.
template <typename K1, typename K0>
int sort_phase_kx(Handle &h, int x) {
  SortScratch &ss = h.ss;
  constexpr int IPT1 = sizeof(K1) == 8 ? CNT_IPT64 : CNT_IPT128;
  constexpr int TILE1 = CNT_THREADS * IPT1;
  constexpr int IPT2 = sizeof(K0) == 8 ? WCNT_IPT64 : WCNT_IPT128;
  constexpr int TILE2 = CNT_THREADS * IPT2;
  const int k = (int)h.p.k;
  const int key_bits1 = 2 + 2 * (k + x);
  SortMeta meta;
  int rc = build_meta(h, key_bits1, TILE1, 0.6, &meta);
  if (rc) return rc;
  KxxArgs<K1> a;
  a.chunks = meta.chunks;
  a.pieces = meta.pieces;
  a.k = k;
  a.x = x;
  a.key_bits = key_bits1;
  a.group_base = meta.group_base;
  a.group_D = meta.group_D;
  a.mixer = make_mixer<K1>(key_bits1);
  save_debug_mixer(h, a.mixer);
  const uint64_t NB = meta.NB;
  uint32_t *hist = as<uint32_t>(ss.hist);
  KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, NB * 4, h.st));
  if (meta.n_chunks) {
    StageScope sc(h, KMC_STAGE_KX_COUNT);
    kxx_count_kernel<K1, K0><<<(unsigned)meta.n_chunks, KX_THREADS, 0, h.st>>>(a, hist);
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  uint32_t *n_tiles_dev = nullptr;
  {
    StageScope sc_plan(h, KMC_STAGE_PLAN);
    rc = plan_tiles(h, hist, NB, a.group_base, h.p.n_bins, TILE1, ss.bucket_base, ss.flags,
                    ss.flag_scan, ss.tile_first, ss.scan_tmp, &n_tiles_dev);
  }
  if (rc) return rc;
  uint64_t n_keys1 = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&n_keys1, as<uint64_t>(ss.bucket_base) + NB, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, NB * 4, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  h.stats.n_sorted_keys = n_keys1;
  if (dev_ensure(ss.keys, (n_keys1 + 2) * sizeof(K1), h.st)) return KMC_ENOMEM;  // 16 B slack
  K1 *keys = as<K1>(ss.keys);
  if (meta.n_chunks) {
    StageScope sc(h, KMC_STAGE_KX_SCATTER);
    kxx_scatter_kernel<K1, K0><<<(unsigned)meta.n_chunks, KX_THREADS, 0, h.st>>>(
        a, as<uint64_t>(ss.bucket_base), hist, keys, n_keys1, as<uint32_t>(h.err));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  TilePlan plan;
  plan.bucket_base = as<uint64_t>(ss.bucket_base);
  plan.tile_first = as<uint32_t>(ss.tile_first);
  plan.n_tiles = n_tiles_dev;
  plan.group_base = a.group_base;
  plan.group_D = a.group_D;
  plan.n_groups = h.p.n_bins;
  plan.NB = (uint32_t)NB;
  plan.key_bits = key_bits1;
  K1 *sorted_out = nullptr;
  if (h.p.debug_flags & KMC_DEBUG_KEEP_KEYS) {
    if (dev_ensure(ss.sorted_keys, (n_keys1 + 1) * sizeof(K1), h.st)) return KMC_ENOMEM;
    sorted_out = as<K1>(ss.sorted_keys);
  }
  // level 1: distinct (k,x)-mers with their multiplicities (no cutoffs)
  uint64_t n1 = 0;
  h.stats.n_big_tiles = 0;
  rc = count_tiles<K1, IPT1>(h, plan, n_keys1, keys, a.mixer, 1, ~0ull, ss.sv_keys, ss.sv_counts,
                             &n1, sorted_out);
  if (rc) return rc;
  uint32_t nt = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&nt, n_tiles_dev, 4, cudaMemcpyDeviceToHost, h.st));
  // level 2: expand, bucket by the mixed k-mer's top bits (one group), count
  const uint64_t n2_max = n1 * (uint64_t)(x + 1);
  int D2 = 0;
  while (D2 < 22 && D2 < 2 * k && (n2_max >> D2) > (uint64_t)TILE2 / 2) ++D2;
  const uint32_t ND2 = 1u << D2;
  if (dev_ensure(ss.l2_hist, (size_t)ND2 * 4 + 4, h.st) || dev_ensure(ss.l2_grp, 64, h.st) ||
      dev_ensure(ss.l2_keys, (n2_max + 1) * sizeof(K0), h.st) ||
      dev_ensure(ss.l2_wts, (n2_max + 1) * 4, h.st) || dev_ensure(ss.l2_counters, 64, h.st))
    return KMC_ENOMEM;
  Mixer<K0> mix0 = make_mixer<K0>(2 * k);
  uint32_t *h2 = as<uint32_t>(ss.l2_hist);
  KMC_CUDA_TRY(cudaMemsetAsync(h2, 0, (size_t)ND2 * 4, h.st));
  {
    uint32_t gh[4] = {0u, ND2, (uint32_t)D2, 0u};
    KMC_CUDA_TRY(cudaMemcpyAsync(ss.l2_grp.p, gh, 16, cudaMemcpyHostToDevice, h.st));
  }
  const uint32_t *grp = as<uint32_t>(ss.l2_grp);
  uint32_t *n_tiles2 = nullptr;
  {
    StageScope sc(h, KMC_STAGE_KX_COUNT);
    if (n1)
      expand_kernel<K1, K0><<<grid_for(n1, 256, 65535), 256, 0, h.st>>>(
          as<K1>(ss.sv_keys), as<uint32_t>(ss.sv_counts), n1, k, x, mix0, D2, 0, h2, nullptr,
          nullptr, nullptr, 0, as<uint32_t>(h.err));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  {
    StageScope sc(h, KMC_STAGE_PLAN);
    rc = plan_tiles(h, h2, ND2, grp, 1, TILE2, ss.l2_base, ss.l2_flags, ss.l2_fscan, ss.l2_tfirst,
                    ss.l2_tmp, &n_tiles2);
  }
  if (rc) return rc;
  uint64_t n2 = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&n2, as<uint64_t>(ss.l2_base) + ND2, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemsetAsync(h2, 0, (size_t)ND2 * 4, h.st));
  {
    StageScope sc(h, KMC_STAGE_KX_SCATTER);
    if (n1)
      expand_kernel<K1, K0><<<grid_for(n1, 256, 65535), 256, 0, h.st>>>(
          as<K1>(ss.sv_keys), as<uint32_t>(ss.sv_counts), n1, k, x, mix0, D2, 1, h2,
          as<uint64_t>(ss.l2_base), as<K0>(ss.l2_keys), as<uint32_t>(ss.l2_wts), n2_max,
          as<uint32_t>(h.err));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  TilePlan plan2;
  plan2.bucket_base = as<uint64_t>(ss.l2_base);
  plan2.tile_first = as<uint32_t>(ss.l2_tfirst);
  plan2.n_tiles = n_tiles2;
  plan2.group_base = grp;
  plan2.group_D = reinterpret_cast<const uint8_t *>(grp + 2);
  plan2.n_groups = 1;
  plan2.NB = ND2;
  plan2.key_bits = 2 * k;
  using WSM = TileWCountSmem<K0, CNT_THREADS, IPT2>;
  using BWSM = BigSmem<K0, uint32_t, CNT_THREADS, BIG_IPT>;
  const uint64_t ci = h.p.cutoff_min ? h.p.cutoff_min : 1;
  const uint64_t sv_cap = n2 / ci + TILE2 + 1;
  const uint32_t big_cap = (uint32_t)std::min<uint64_t>(n2 / (TILE2 + 1) + 1, ND2);
  if (dev_ensure(ss.l2_out_keys, sv_cap * sizeof(K0), h.st) ||
      dev_ensure(ss.l2_out_counts, sv_cap * 4, h.st) || dev_ensure(ss.l2_big, (size_t)big_cap * 4 + 4, h.st))
    return KMC_ENOMEM;
  auto *c32 = as<uint32_t>(ss.l2_counters);
  auto *c64 = reinterpret_cast<unsigned long long *>(c32 + 4);
  KMC_CUDA_TRY(cudaMemsetAsync(c32, 0, 64, h.st));
  CountOut<K0> out;
  out.keys = as<K0>(ss.l2_out_keys);
  out.counts = as<uint32_t>(ss.l2_out_counts);
  out.n = c64 + 0;
  out.cap = sv_cap;
  out.ci = ci;
  out.cx = h.p.cutoff_max;
  out.n_distinct = c64 + 1;
  out.mixer = mix0;
  out.sort_bits = (h.p.debug_flags & KMC_DEBUG_NARROW_SORT) ? 8 : kCountSortBits;
  out.slots = nullptr;
  out.bins_per_slot = 1;
  static DeviceOnce attr;
  if (!attr.done()) {
    KMC_CUDA_TRY(cudaFuncSetAttribute(tile_wcount_kernel<K0, CNT_THREADS, IPT2>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(WSM)));
    KMC_CUDA_TRY(cudaFuncSetAttribute(big_wcount_kernel<K0, CNT_THREADS, BIG_IPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BWSM)));
    attr.set();
  }
  int occ = 0;
  KMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, tile_wcount_kernel<K0, CNT_THREADS, IPT2>, CNT_THREADS, sizeof(WSM)));
  {
    StageScope sc(h, KMC_STAGE_TILE_SORT);
    tile_wcount_kernel<K0, CNT_THREADS, IPT2><<<(unsigned)std::max(1, occ) * h.sm_count, CNT_THREADS,
                                                 sizeof(WSM), h.st>>>(
        as<K0>(ss.l2_keys), as<uint32_t>(ss.l2_wts), plan2, c32 + 0, out, as<uint32_t>(ss.l2_big),
        c32 + 1, c64 + 2, big_cap, as<uint32_t>(h.err));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  uint32_t nbig = 0;
  unsigned long long bigk = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&nbig, c32 + 1, 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(&bigk, c64 + 2, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  if (nbig) {
    h.stats.n_big_tiles += nbig;
    if (dev_ensure(ss.l2_big_k, (bigk + 1) * sizeof(K0), h.st) ||
        dev_ensure(ss.l2_big_v, (bigk + 1) * 4, h.st))
      return KMC_ENOMEM;
    StageScope sc(h, KMC_STAGE_BIG_SORT);
    big_wcount_kernel<K0, CNT_THREADS, BIG_IPT><<<nbig, CNT_THREADS, sizeof(BWSM), h.st>>>(
        as<K0>(ss.l2_keys), as<uint32_t>(ss.l2_wts), plan2, as<uint32_t>(ss.l2_big),
        as<K0>(ss.l2_big_k), as<uint32_t>(ss.l2_big_v), c64 + 3, out, as<uint32_t>(h.err));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  unsigned long long vals[2];
  uint32_t nt2 = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(vals, c64, 16, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(&nt2, n_tiles2, 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  rc = check_device_error(h);
  if (rc) return rc;
  h.stats.n_distinct = vals[1];
  h.stats.n_tiles = nt + nt2;
  h.stats.x_used = (uint32_t)x;
  return order_result<K0>(h, ss.l2_out_keys, ss.l2_out_counts, vals[0], k);
}

}  // namespace

// x used for a k: the requested x (KMC_AUTO: 0, the fastest on the GPU),
// limited so that a (k,x)-mer key fits 128 bits (2 + 2(k+x) <= 128).
uint32_t resolve_x(uint32_t k, uint32_t x) {
  if (x == KMC_AUTO) x = 0;
  if (x > 3) x = 3;
  if (k + x > 63) x = k >= 63 ? 0 : 63 - k;
  return x;
}

namespace {
int sort_phase_any(Handle &h) {
  const uint32_t k = h.p.k;
  const int x = (int)resolve_x(k, h.p.x);
  h.stats.n_waves = 1;
  if (x == 0) {
    if (k <= 32) return sort_phase_x0<uint64_t, CNT_IPT64>(h);
    return sort_phase_x0<u128, CNT_IPT128>(h);
  }
  const bool key64 = 2 + 2 * ((int)k + x) <= 64;
  if (k <= 32) {
    if (key64) return sort_phase_kx<uint64_t, uint64_t>(h, x);
    return sort_phase_kx<u128, uint64_t>(h, x);
  }
  return sort_phase_kx<u128, u128>(h, x);
}

// Suppl. S1 -cs: counts above the counter's maximal value are reported as it.
__global__ void saturate_kernel(uint32_t *__restrict__ c, uint64_t n, uint32_t cmax) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    if (c[i] > cmax) c[i] = cmax;
}
}  // namespace

int sort_phase(Handle &h) {
  const int rc = sort_phase_any(h);
  if (rc || !h.p.counter_max || !h.n_out) return rc;
  const uint32_t cmax = (uint32_t)std::min<uint64_t>(h.p.counter_max, 0xFFFFFFFFull);
  saturate_kernel<<<grid_for(h.n_out, 256, 65535), 256, 0, h.st>>>(as<uint32_t>(h.out_counts), h.n_out, cmax);
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  return KMC_OK;
}

namespace {
template <typename K>
int debug_keys_impl(Handle &h, uint32_t bin, uint64_t *keys, uint64_t capacity, uint64_t *n_out,
                    uint32_t *words_per_key) {
  SortScratch &ss = h.ss;
  const int words = (int)sizeof(K) / 8;
  if (words_per_key) *words_per_key = (uint32_t)words;
  const uint32_t g0 = ss.dbg_group_base[bin], g1 = ss.dbg_group_base[bin + 1];
  uint64_t r[2];
  KMC_CUDA_TRY(cudaMemcpyAsync(&r[0], as<uint64_t>(ss.bucket_base) + g0, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(&r[1], as<uint64_t>(ss.bucket_base) + g1, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  const uint64_t n = r[1] - r[0];
  *n_out = n;
  if (capacity < n) return KMC_ETRUNC;
  if (!n) return KMC_OK;
  Mixer<K> m;
  m.c = (K)ss.dbg_mix[0] | (sizeof(K) > 8 ? (K)((u128)ss.dbg_mix[1] << 64) : K(0));
  m.cinv = (K)ss.dbg_mix[2] | (sizeof(K) > 8 ? (K)((u128)ss.dbg_mix[3] << 64) : K(0));
  m.mask = (K)ss.dbg_mix[4] | (sizeof(K) > 8 ? (K)((u128)ss.dbg_mix[5] << 64) : K(0));
  m.bits = (int)(ss.dbg_mix[6] & 0xFFFF);
  m.s1 = (int)((ss.dbg_mix[6] >> 16) & 0xFFFF);
  m.s2 = (int)((ss.dbg_mix[6] >> 32) & 0xFFFF);
  m.on = true;
  DevBuf tmp;
  if (dev_ensure(tmp, n * 8 * words, h.st)) return KMC_ENOMEM;
  unmix_words_kernel<K><<<grid_for(n, 256, 65535), 256, 0, h.st>>>(
      as<K>(ss.sorted_keys) + r[0], n, m, as<uint64_t>(tmp));
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  KMC_CUDA_TRY(cudaMemcpyAsync(keys, tmp.p, n * 8 * words, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  dev_release(tmp, h.st);
  return KMC_OK;
}
}  // namespace

int debug_bin_keys(Handle &h, uint32_t bin, uint64_t *keys, uint64_t capacity, uint64_t *n_out,
                   uint32_t *words_per_key) {
  if (!(h.p.debug_flags & KMC_DEBUG_KEEP_KEYS) || h.ss.dbg_group_base.size() <= bin + 1)
    return KMC_ESTATE;
  if (h.ss.dbg_key_bytes == 8) return debug_keys_impl<uint64_t>(h, bin, keys, capacity, n_out, words_per_key);
  return debug_keys_impl<u128>(h, bin, keys, capacity, n_out, words_per_key);
}

}  // namespace kmc
