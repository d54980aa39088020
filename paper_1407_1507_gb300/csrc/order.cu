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

// ----------------------------------------- two-level radix partition of pairs
// The survivors' global order (large result lists): the pairs are moved by
// two coalesced partition sweeps on the top 8 + E bits of the k-mer value,
// then every final bucket (about 1 k pairs) is sorted by the shared-memory
// LSD tile sort.  Level 1 works on tiles of the whole array: a tile is
// ranked by its top-8-bit digit in shared memory, one global atomic per digit
// reserves the tile's runs in the 256 super buckets, and the runs go out in
// order (consecutive threads write consecutive addresses).  Level 2 gives
// each super bucket to one CTA, which counts its E-bit digits, keeps the
// bucket cursors in shared memory and sweeps the bucket tile by tile; the
// canonical k-mers' top bits are skewed by at most a few times the average,
// so the largest super bucket sets the tail.
constexpr int PSW_THREADS = 512;
constexpr uint64_t kPswMinPairs = 1ull << 22;
constexpr int PSW_UPPER = 8;
constexpr int PSW_LOWER_MAX = 12;

template <typename K>
struct PswTraits {
  static_assert(PSW_THREADS * (sizeof(K) == 8 ? 8 : 4) <= 4096, "tile starts are 16-bit");
  static constexpr int IPT = sizeof(K) == 8 ? 8 : 4;
  static constexpr int TILE = PSW_THREADS * IPT;  // 4096 pairs of 64-bit keys, 2048 of 128-bit
};

template <typename K>
struct PswSmem {
  K sk[PswTraits<K>::TILE];
  uint32_t sv[PswTraits<K>::TILE];
  uint32_t h[1 << PSW_LOWER_MAX];       // tile digit counts
  uint16_t lstart[1 << PSW_LOWER_MAX];  // tile digit starts (a tile holds at most 4096 pairs)
  uint32_t cur[1 << PSW_LOWER_MAX];     // level 2: bucket cursors (relative to the super bucket)
  uint32_t run[1 << PSW_LOWER_MAX];     // level 2: where this tile's run of each digit starts
  unsigned long long gpos[1 << PSW_UPPER];  // level 1: global start of each digit's run
  uint32_t ws[PSW_THREADS / 32 + 1];
};

template <typename K>
__device__ __forceinline__ uint32_t psw_upper(K key, int key_bits) {
  return (uint32_t)(uint64_t)(key >> (key_bits - PSW_UPPER)) & ((1u << PSW_UPPER) - 1u);
}
template <typename K>
__device__ __forceinline__ uint32_t psw_lower(K key, int key_bits, int E) {
  return E ? (uint32_t)(uint64_t)(key >> (key_bits - PSW_UPPER - E)) & ((1u << E) - 1u) : 0u;
}

// Exclusive scan of cnt[0, nd) into out[0, nd) by the whole block (nd a
// power of two, at most 2^PSW_LOWER_MAX).
template <typename K, typename T>
__device__ void psw_block_scan(const uint32_t *cnt, T *out, int nd, PswSmem<K> &s) {
  const int tid = threadIdx.x;
  const int per = nd >= PSW_THREADS ? nd / PSW_THREADS : 1;
  const int i0 = tid * per;
  uint32_t sum = 0;
  if (i0 < nd)
    for (int j = 0; j < per; ++j) sum += cnt[i0 + j];
  uint32_t tot;
  uint32_t run = block_excl_scan<uint32_t, PSW_THREADS>(i0 < nd ? sum : 0u, s.ws, &tot);
  if (i0 < nd)
    for (int j = 0; j < per; ++j) {
      out[i0 + j] = (T)run;
      run += cnt[i0 + j];
    }
}

// Level-1 histogram of the top 8 bits.
template <typename K>
__global__ void __launch_bounds__(256) psw_hist_kernel(const K *__restrict__ keys, uint64_t n, int key_bits,
                                                       uint32_t *__restrict__ hist) {
  __shared__ uint32_t h[1 << PSW_UPPER];
  for (int i = threadIdx.x; i < (1 << PSW_UPPER); i += blockDim.x) h[i] = 0;
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[psw_upper<K>(keys[i], key_bits)], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < (1 << PSW_UPPER); i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

// One tile of n pairs at (ik, iv)[st ..]: ranked by digit (level 1: upper,
// level 2: lower E bits), placed in digit order in shared memory, and each
// digit's run written from its reserved place: reserve(d, count), called
// once per non-empty digit by one thread, records it in s.gpos[d] (level 1,
// absolute) or s.run[d] (level 2, relative to wbase).
template <typename K, int LEVEL, typename R>
__device__ __forceinline__ void psw_tile(const K *__restrict__ ik, const uint32_t *__restrict__ iv, uint64_t st,
                                         uint32_t n, int key_bits, int E, uint64_t wbase, K *__restrict__ ok,
                                         uint32_t *__restrict__ ov, PswSmem<K> &s, R reserve) {
  constexpr int IPT = PswTraits<K>::IPT;
  const int tid = threadIdx.x;
  const int nd = LEVEL == 1 ? (1 << PSW_UPPER) : (1 << E);
  for (int i = tid; i < nd; i += PSW_THREADS) s.h[i] = 0;
  __syncthreads();
  K key[IPT];
  uint32_t val[IPT], rk[IPT];
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t e = tid + i * PSW_THREADS;
    if (e < n) {
      key[i] = ik[st + e];
      val[i] = iv[st + e];
    }
  }
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t e = tid + i * PSW_THREADS;
    rk[i] = 0;
    if (e < n) {
      const uint32_t d = LEVEL == 1 ? psw_upper<K>(key[i], key_bits) : psw_lower<K>(key[i], key_bits, E);
      rk[i] = atomicAdd(&s.h[d], 1u);
    }
  }
  __syncthreads();
  psw_block_scan<K, uint16_t>(s.h, s.lstart, nd, s);
  for (int d = tid; d < nd; d += PSW_THREADS)
    if (s.h[d]) reserve(d, s.h[d]);
  __syncthreads();
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t e = tid + i * PSW_THREADS;
    if (e < n) {
      const uint32_t d = LEVEL == 1 ? psw_upper<K>(key[i], key_bits) : psw_lower<K>(key[i], key_bits, E);
      s.sk[s.lstart[d] + rk[i]] = key[i];
      s.sv[s.lstart[d] + rk[i]] = val[i];
    }
  }
  __syncthreads();
  for (uint32_t i = tid; i < n; i += PSW_THREADS) {
    const K k = s.sk[i];
    const uint32_t d = LEVEL == 1 ? psw_upper<K>(k, key_bits) : psw_lower<K>(k, key_bits, E);
    const uint64_t p = (LEVEL == 1 ? s.gpos[d] : wbase + s.run[d]) + (i - s.lstart[d]);
    ok[p] = k;
    ov[p] = s.sv[i];
  }
  __syncthreads();
}

// Level 1: persistent CTAs over the tiles of the whole array.
template <typename K>
__global__ void __launch_bounds__(PSW_THREADS, 2)
psw_level1_kernel(const K *__restrict__ ik, const uint32_t *__restrict__ iv, uint64_t n, int key_bits,
                  const uint64_t *__restrict__ base1, unsigned long long *__restrict__ cur1,
                  K *__restrict__ ok, uint32_t *__restrict__ ov) {
  constexpr int TILE = PswTraits<K>::TILE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PswSmem<K> &s = *reinterpret_cast<PswSmem<K> *>(smem_raw);
  const uint64_t n_tiles = (n + TILE - 1) / TILE;
  for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const uint64_t st = t * TILE;
    const uint32_t m = (uint32_t)(n - st < (uint64_t)TILE ? n - st : (uint64_t)TILE);
    psw_tile<K, 1>(ik, iv, st, m, key_bits, 0, 0, ok, ov, s, [&](uint32_t d, uint32_t c) {
      s.gpos[d] = base1[d] + atomicAdd(&cur1[d], (unsigned long long)c);
    });
  }
}

// Level 2: one CTA per super bucket; final bucket sizes into fine_hist
// [(super bucket << E) + digit].
template <typename K>
__global__ void __launch_bounds__(PSW_THREADS, 2)
psw_level2_kernel(const K *__restrict__ ik, const uint32_t *__restrict__ iv, int key_bits, int E,
                  const uint64_t *__restrict__ base1, uint32_t *__restrict__ fine_hist, K *__restrict__ ok,
                  uint32_t *__restrict__ ov) {
  constexpr int TILE = PswTraits<K>::TILE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  PswSmem<K> &s = *reinterpret_cast<PswSmem<K> *>(smem_raw);
  const int tid = threadIdx.x;
  const uint32_t sb = blockIdx.x;
  const uint64_t st = base1[sb], en = base1[sb + 1];
  const int nd = 1 << E;
  for (int i = tid; i < nd; i += PSW_THREADS) s.h[i] = 0;
  __syncthreads();
  for (uint64_t e = st + tid; e < en; e += PSW_THREADS) atomicAdd(&s.h[psw_lower<K>(ik[e], key_bits, E)], 1u);
  __syncthreads();
  for (int i = tid; i < nd; i += PSW_THREADS) fine_hist[((uint64_t)sb << E) + i] = s.h[i];
  psw_block_scan<K, uint32_t>(s.h, s.cur, nd, s);
  __syncthreads();
  for (uint64_t t0 = st; t0 < en; t0 += TILE) {
    const uint32_t m = (uint32_t)(en - t0 < (uint64_t)TILE ? en - t0 : (uint64_t)TILE);
    psw_tile<K, 2>(ik, iv, t0, m, key_bits, E, st, ok, ov, s, [&](uint32_t d, uint32_t c) {
      s.run[d] = s.cur[d];  // only the thread of digit d touches its cursor
      s.cur[d] += c;
    });
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
  // Large lists: the two-level partition on 8 + E top bits (buckets of about
  // 1 k pairs).  Others: one scatter into many small buckets (about TILE/64
  // keys each: the top bits of canonical k-mers are skewed, and the tile plan
  // packs small buckets back together, while a bucket above a tile would take
  // the slow path).
  const bool two = n >= kPswMinPairs && key_bits >= PSW_UPPER + 2;
  int D = 0, E = 0;
  if (two) {
    while (E < PSW_LOWER_MAX && E + PSW_UPPER < key_bits && (n >> (PSW_UPPER + E)) > 1024) ++E;
    if (E < 2) E = 2;
    D = PSW_UPPER + E;
  } else {
    while (D < PAIR_MAX_D && D < key_bits && (n >> D) > (uint64_t)TILE / 64) ++D;
  }
  const uint32_t ND = 1u << D;
  if (dev_ensure(ss.o_hist, (size_t)ND * 4 + 4, h.st) || dev_ensure(ss.o_base, ((size_t)ND + 1) * 8, h.st) ||
      dev_ensure(ss.o_flags, (size_t)ND * 4 + 4, h.st) ||
      dev_ensure(ss.o_flag_scan, ((size_t)ND + 1) * 8, h.st) ||
      dev_ensure(ss.o_tile_first, (size_t)ND * 4 + 16, h.st) ||
      dev_ensure(ss.o_scan_tmp, scan_tmp_words(ND) * 8, h.st) ||
      ((in_place || two) && (dev_ensure(ss.o_big_k, (n + 1) * sizeof(K), h.st) ||
                             dev_ensure(ss.o_big_v, (n + 1) * 4, h.st))) ||
      dev_ensure(ss.o_cursor, 128, h.st))
    return KMC_ENOMEM;
  uint32_t *hist = as<uint32_t>(ss.o_hist);
  K *tk = in_place ? as<K>(ss.o_big_k) : out_k;  // where the partitioned pairs end up
  V *tv = in_place ? as<V>(ss.o_big_v) : out_v;
  K *big_k = keys;                               // free space for the big buckets
  V *big_v = vals;
  if (two) {
    // level 1: keys -> scratch (o_big); level 2: scratch -> the result arrays
    // (the input arrays themselves when sorting in place)
    static DeviceOnce pattr;
    if (!pattr.done()) {
      KMC_CUDA_TRY(cudaFuncSetAttribute(psw_level1_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(PswSmem<K>)));
      KMC_CUDA_TRY(cudaFuncSetAttribute(psw_level2_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(PswSmem<K>)));
      pattr.set();
    }
    K *mk = as<K>(ss.o_big_k);
    V *mv = as<V>(ss.o_big_v);
    tk = in_place ? keys : out_k;
    tv = in_place ? vals : out_v;
    if (in_place) {
      big_k = mk;
      big_v = mv;
    }
    uint32_t *hist1 = as<uint32_t>(ss.o_flags);                       // [256]
    uint64_t *base1 = as<uint64_t>(ss.o_flag_scan);                   // [257]
    auto *cur1 = reinterpret_cast<unsigned long long *>(base1 + 300);  // [256] (ND + 1 >= 1025 words)
    KMC_CUDA_TRY(cudaMemsetAsync(hist1, 0, 256 * 4, h.st));
    KMC_CUDA_TRY(cudaMemsetAsync(cur1, 0, 256 * 8, h.st));
    psw_hist_kernel<K><<<std::min<unsigned>(grid_for(n, 256, 65535), 8u * (unsigned)h.sm_count), 256, 0, h.st>>>(
        keys, n, key_bits, hist1); KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(device_excl_scan_u32(hist1, base1, 256, as<uint64_t>(ss.o_scan_tmp), h.st));
    psw_level1_kernel<K><<<2u * (unsigned)h.sm_count, PSW_THREADS, sizeof(PswSmem<K>), h.st>>>(
        keys, vals, n, key_bits, base1, cur1, mk, mv); KMC_COUNT_LAUNCH();
    psw_level2_kernel<K><<<256, PSW_THREADS, sizeof(PswSmem<K>), h.st>>>(mk, mv, key_bits, E, base1, hist, tk, tv);
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  } else {
    KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)ND * 4, h.st));
    pair_hist_kernel<K><<<grid_for(n, 256, 65535), 256, 0, h.st>>>(keys, n, key_bits, D, hist); KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
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
  if (!two) {
    KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, (size_t)ND * 4, h.st));
    pair_scatter_kernel<K, V><<<grid_for(n, 256, 65535), 256, 0, h.st>>>(
        keys, vals, n, key_bits, D, as<uint64_t>(ss.o_base), hist, tk, tv); KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
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
    big_pairs_kernel<K, V, PAIR_THREADS, PAIR_BIG_IPT><<<nbig, PAIR_THREADS, sizeof(BSM), h.st>>>(
        tk, tv, plan, as<uint32_t>(ss.o_flags), c32 + 1, big_k, big_v, c64 + 1); KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  if (in_place && !two) {
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
