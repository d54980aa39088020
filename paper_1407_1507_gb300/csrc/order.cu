// Sort of (key, value) pairs by the low `key_bits` bits of the key: an MSD
// scatter on the top D bits into digit buckets, then the shared-memory LSD
// tile sort of sortlib.cuh.  Used for the global order of the counted
// k-mers (the bins are signature ordered; the result is ordered by k-mer)
// and for ordering signatures by sample weight when building the bin map.
#include <algorithm>

#include "internal.h"
#include "sortlib.cuh"

namespace kmc {

namespace {

constexpr int PAIR_THREADS = 256;
constexpr int PAIR_IPT = 8;   // tile = 2048 pairs (three CTAs per SM)
constexpr int PAIR_BIG_IPT = 8;
constexpr int PAIR_MAX_D = 22;

template <typename K>
__global__ void pair_hist_kernel(const K *__restrict__ keys, uint64_t n, int key_bits, int D,
                                 uint32_t *__restrict__ hist) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n_up = (n + 31) & ~31ull;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_up; i += stride) {
    const bool ok = i < n;
    const uint32_t d = ok ? top_digit<K>(keys[i], key_bits, D) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(FULL, d);
    if (ok && (int)lane_id() == __ffs(peers) - 1) atomicAdd(&hist[d], (uint32_t)__popc(peers));
  }
}

template <typename K, typename V>
__global__ void pair_scatter_kernel(const K *__restrict__ keys, const V *__restrict__ vals,
                                    uint64_t n, int key_bits, int D,
                                    const uint64_t *__restrict__ base, uint32_t *__restrict__ cursor,
                                    K *__restrict__ out_k, V *__restrict__ out_v) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t n_up = (n + 31) & ~31ull;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_up; i += stride) {
    const bool ok = i < n;
    K key = ok ? keys[i] : K(0);
    const uint32_t d = ok ? top_digit<K>(key, key_bits, D) : 0xFFFFFFFFu;
    const unsigned peers = __match_any_sync(FULL, d);
    const int leader = __ffs(peers) - 1;
    uint32_t b = 0;
    if (ok && (int)lane_id() == leader) b = atomicAdd(&cursor[d], (uint32_t)__popc(peers));
    b = __shfl_sync(FULL, b, leader);
    if (ok) {
      const uint64_t p = base[d] + b + __popc(peers & lanemask_lt());
      out_k[p] = key;
      out_v[p] = vals[i];
    }
  }
}

inline unsigned grid_for(uint64_t n, int threads, int cap = 1 << 20) {
  uint64_t g = (n + threads - 1) / threads;
  if (g < 1) g = 1;
  return (unsigned)std::min<uint64_t>(g, (uint64_t)cap);
}

// Sorts (keys, vals)[0, n) into (out_k, out_v); with out_k == keys the sort
// is in place (through the handle's scratch).  When distinct, the input
// arrays are clobbered (they serve as the scratch of the big buckets).
template <typename K>
int sort_pairs_impl(Handle &h, K *keys, uint32_t *vals, uint64_t n, int key_bits, K *out_k,
                    uint32_t *out_v) {
  using V = uint32_t;
  using SM = TilePairsSmem<K, V, PAIR_THREADS, PAIR_IPT>;
  using BSM = BigSmem<K, V, PAIR_THREADS, PAIR_BIG_IPT>;
  constexpr int TILE = PAIR_THREADS * PAIR_IPT;
  SortScratch &ss = h.ss;
  const bool in_place = out_k == keys;
  if (n <= 1) {
    if (n == 1 && !in_place) {
      KMC_CUDA_TRY(cudaMemcpyAsync(out_k, keys, sizeof(K), cudaMemcpyDeviceToDevice, h.st));
      KMC_CUDA_TRY(cudaMemcpyAsync(out_v, vals, sizeof(V), cudaMemcpyDeviceToDevice, h.st));
    }
    return KMC_OK;
  }
  // many small buckets (about TILE/64 keys each): the top bits of canonical
  // k-mers are skewed, and the tile plan packs small buckets back together,
  // while a bucket above a tile would take the slow path
  int D = 0;
  while (D < PAIR_MAX_D && D < key_bits && (n >> D) > (uint64_t)TILE / 64) ++D;
  const uint32_t ND = 1u << D;
  if (dev_ensure(ss.o_hist, (size_t)ND * 4 + 4, h.st) || dev_ensure(ss.o_base, ((size_t)ND + 1) * 8, h.st) ||
      dev_ensure(ss.o_flags, (size_t)ND * 4 + 4, h.st) ||
      dev_ensure(ss.o_flag_scan, ((size_t)ND + 1) * 8, h.st) ||
      dev_ensure(ss.o_tile_first, (size_t)ND * 4 + 16, h.st) ||
      dev_ensure(ss.o_scan_tmp, scan_tmp_words(ND) * 8, h.st) ||
      (in_place && (dev_ensure(ss.o_big_k, (n + 1) * sizeof(K), h.st) ||
                    dev_ensure(ss.o_big_v, (n + 1) * 4, h.st))) ||
      dev_ensure(ss.o_cursor, 128, h.st))
    return KMC_ENOMEM;
  uint32_t *hist = as<uint32_t>(ss.o_hist);
  KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)ND * 4, h.st));
  pair_hist_kernel<K><<<grid_for(n, 256, 65535), 256, 0, h.st>>>(keys, n, key_bits, D, hist); KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  KMC_CUDA_TRY(device_excl_scan_u32(hist, as<uint64_t>(ss.o_base), ND, as<uint64_t>(ss.o_scan_tmp), h.st));
  // one group of ND buckets: group_base = {0, ND}, D
  uint32_t *grp = as<uint32_t>(ss.o_cursor) + 8;
  {
    uint32_t gh[4] = {0u, ND, (uint32_t)D, 0u};
    KMC_CUDA_TRY(cudaMemcpyAsync(grp, gh, 16, cudaMemcpyHostToDevice, h.st));
  }
  plan_flags_kernel<<<grid_for(ND, 256, 65535), 256, 0, h.st>>>(hist, as<uint64_t>(ss.o_base), ND, grp, 1,
                                                                 (uint32_t)TILE, as<uint32_t>(ss.o_flags)); KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  KMC_CUDA_TRY(device_excl_scan_u32(as<uint32_t>(ss.o_flags), as<uint64_t>(ss.o_flag_scan), ND,
                                    as<uint64_t>(ss.o_scan_tmp), h.st));
  uint32_t *n_tiles = as<uint32_t>(ss.o_tile_first) + ND + 1;
  plan_emit_kernel<<<grid_for(ND, 256, 65535), 256, 0, h.st>>>(
      as<uint32_t>(ss.o_flags), as<uint64_t>(ss.o_flag_scan), ND, as<uint32_t>(ss.o_tile_first), n_tiles); KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)ND * 4, h.st));
  K *tk = in_place ? as<K>(ss.o_big_k) : out_k;
  V *tv = in_place ? as<V>(ss.o_big_v) : out_v;
  pair_scatter_kernel<K, V><<<grid_for(n, 256, 65535), 256, 0, h.st>>>(
      keys, vals, n, key_bits, D, as<uint64_t>(ss.o_base), hist, tk, tv); KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  TilePlan plan;
  plan.bucket_base = as<uint64_t>(ss.o_base);
  plan.tile_first = as<uint32_t>(ss.o_tile_first);
  plan.n_tiles = n_tiles;
  plan.group_base = grp;
  plan.group_D = reinterpret_cast<const uint8_t *>(grp + 2);
  plan.n_groups = 1;
  plan.NB = ND;
  plan.key_bits = key_bits;
  static DeviceOnce attr;
  if (!attr.done()) {
    KMC_CUDA_TRY(cudaFuncSetAttribute(tile_pairs_kernel<K, V, PAIR_THREADS, PAIR_IPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SM)));
    KMC_CUDA_TRY(cudaFuncSetAttribute(big_pairs_kernel<K, V, PAIR_THREADS, PAIR_BIG_IPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BSM)));
    attr.set();
  }
  auto *c32 = as<uint32_t>(ss.o_cursor);
  auto *c64 = reinterpret_cast<unsigned long long *>(c32 + 4);  // c64[0..1] = bytes 16..31
  KMC_CUDA_TRY(cudaMemsetAsync(c32, 0, 32, h.st));
  const uint32_t big_cap = (uint32_t)std::min<uint64_t>(n / (TILE + 1) + 1, ND);
  if (dev_ensure(ss.o_flags, (size_t)std::max<uint64_t>(ND, big_cap) * 4 + 4, h.st)) return KMC_ENOMEM;
  int occ = 0;
  KMC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, tile_pairs_kernel<K, V, PAIR_THREADS, PAIR_IPT>, PAIR_THREADS, sizeof(SM)));
  const unsigned grid = (unsigned)std::max(1, occ) * (unsigned)h.sm_count;
  tile_pairs_kernel<K, V, PAIR_THREADS, PAIR_IPT><<<grid, PAIR_THREADS, sizeof(SM), h.st>>>(
      tk, tv, plan, c32 + 0, as<uint32_t>(ss.o_flags), c32 + 1, c64 + 0, big_cap, as<uint32_t>(h.err)); KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  uint32_t nbig = 0;
  unsigned long long bigk = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&nbig, c32 + 1, 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(&bigk, c64 + 0, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  if (nbig) {
    // the original arrays serve as the scratch of the big buckets
    big_pairs_kernel<K, V, PAIR_THREADS, PAIR_BIG_IPT><<<nbig, PAIR_THREADS, sizeof(BSM), h.st>>>(
        tk, tv, plan, as<uint32_t>(ss.o_flags), c32 + 1, keys, vals, c64 + 1); KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  if (in_place) {
    KMC_CUDA_TRY(cudaMemcpyAsync(keys, tk, n * sizeof(K), cudaMemcpyDeviceToDevice, h.st));
    KMC_CUDA_TRY(cudaMemcpyAsync(vals, tv, n * sizeof(V), cudaMemcpyDeviceToDevice, h.st));
  }
  return KMC_OK;
}

}  // namespace

int sort_pairs_u64(Handle &h, uint64_t *keys, uint32_t *vals, uint64_t n, int key_bits) {
  return sort_pairs_impl<uint64_t>(h, keys, vals, n, key_bits, keys, vals);
}
int sort_pairs_u128(Handle &h, u128 *keys, uint32_t *vals, uint64_t n, int key_bits) {
  return sort_pairs_impl<u128>(h, keys, vals, n, key_bits, keys, vals);
}
int sort_pairs_to_u64(Handle &h, uint64_t *keys, uint32_t *vals, uint64_t n, int key_bits, uint64_t *out_k,
                      uint32_t *out_v) {
  return sort_pairs_impl<uint64_t>(h, keys, vals, n, key_bits, out_k, out_v);
}
int sort_pairs_to_u128(Handle &h, u128 *keys, uint32_t *vals, uint64_t n, int key_bits, u128 *out_k,
                       uint32_t *out_v) {
  return sort_pairs_impl<u128>(h, keys, vals, n, key_bits, out_k, out_v);
}

}  // namespace kmc
