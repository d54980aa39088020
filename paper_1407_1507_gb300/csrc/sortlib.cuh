// Sorting and counting machinery of the sorting phase (paper Sect. 2.4: the
// bin's k-mers are radix sorted and equal ones counted).
//
// Design (GB300-first).  A bin's keys (mixed by a bijection, so that their
// top bits are uniform) are first partitioned by their top D bits into
// digit buckets of about 2 k keys (the radix sweeps of kx_kernels.cuh);
// consecutive buckets are packed into tiles of at most TILE keys, and equal
// keys are brought together per tile in shared memory:
//  * tile_hash_kernel (keys below 2^62, i.e. k <= 31): an open-addressing
//    hash table per tile (64-bit CAS to claim a slot, an add to count);
//  * tile_group_kernel (wider keys): the tile arrives by a bulk copy, one
//    more radix step on 11 low key bits, then parallel value rounds;
//  * tile_count_kernel: a full LSD radix sort of the tile with 8-bit digits
//    (kept for the sorted-keys inspection and the narrow-sort check).
// The order inside a bin does not matter: only survivors are put in global
// order, by sort_pairs (order.cu) with the LSD tile sort below.  Ranking
// inside an LSD pass uses warp match (lanes with equal digits find each
// other in one instruction) and per-warp digit counters in shared memory,
// scanned block-wide in (digit, warp) order, which keeps every pass stable.
// A bucket larger than a tile (e.g. one k-mer repeated millions of times)
// takes a slower path: split once more (big_group_kernel) or sorted by one
// CTA with LSD passes through global memory (big_count_kernel).
#pragma once
#include <type_traits>
#include "common.cuh"

namespace kmc {

struct NoVal {};

// ---------------------------------------------------------------- scans

// Inclusive warp scan.
template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const unsigned lane = lane_id();
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T o = __shfl_up_sync(FULL, v, d);
    if (lane >= (unsigned)d) v += o;
  }
  return v;
}

// Exclusive block scan of one value per thread; returns the exclusive prefix
// and writes the block total to *total.  `ws` holds THREADS/32 + 1 entries.
template <typename T, int THREADS>
__device__ __forceinline__ T block_excl_scan(T v, T *ws, T *total) {
  constexpr int NW = THREADS / 32;
  const unsigned lane = lane_id(), w = threadIdx.x >> 5;
  T inc = warp_incl_scan(v);
  if (lane == 31) ws[w] = inc;
  __syncthreads();
  if (w == 0) {
    T x = lane < (unsigned)NW ? ws[lane] : T(0);
    T xi = warp_incl_scan(x);
    if (lane < (unsigned)NW) ws[lane] = xi - x;
    if (lane == NW - 1) ws[NW] = xi;
  }
  __syncthreads();
  T r = ws[w] + inc - v;
  *total = ws[NW];
  __syncthreads();
  return r;
}

// ------------------------------------------------------ block radix sort

// Sorts THREADS*IPT keys (plus optional payload) held in registers in the
// warp-striped arrangement: element e = warp*32*IPT + i*32 + lane sits in
// keys[i] of that lane.  Sorts on bits [0, nbits).  On return the sorted
// keys are in smem.keys (and smem.vals), in order.
template <typename K, typename V, int THREADS, int IPT>
struct BlockSort {
  static constexpr int NW = THREADS / 32;
  static constexpr int TILE = THREADS * IPT;
  static constexpr bool HAS_V = !std::is_same<V, NoVal>::value;
  static_assert(NW >= 8 && (NW % 8) == 0, "THREADS must be a multiple of 256");
  struct Smem {
    K keys[TILE];
    typename std::conditional<HAS_V, V, char>::type vals[HAS_V ? TILE : 1];
    uint32_t cnt[NW][256];
    uint32_t ws[NW + 1];
  };

  // Element layout: the n keys are split evenly over the warps, warp w
  // holding elements [w*chunk, (w+1)*chunk) with chunk = n/NW rounded up to
  // a multiple of 32 (at most 32*IPT); slot i of lane l is element
  // w*chunk + 32*i + l.  Elements past n are neither counted nor written,
  // so the cost follows the number of keys, not the tile capacity.
  __device__ static int chunk_of(int n) {
    int c = (n + NW - 1) / NW;
    c = (c + 31) & ~31;
    return c < 32 * IPT ? c : 32 * IPT;
  }
  __device__ static int elem(int n, int i) {
    return (int)(threadIdx.x >> 5) * chunk_of(n) + 32 * i + (int)lane_id();
  }
  __device__ static bool valid(int n, int i) {
    return 32 * i < chunk_of(n) && elem(n, i) < n;
  }

  __device__ static void sort(K (&k)[IPT], V (&v)[IPT], int nbits, int n, Smem &s) {
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const int chunk = chunk_of(n);
    const int e_warp = (int)w * chunk;
    const bool warp_live = e_warp < n;
    for (int bit = 0; bit < nbits; bit += 8) {
      const int nb = nbits - bit < 8 ? nbits - bit : 8;
      for (int i = lane; i < 256; i += 32) s.cnt[w][i] = 0;
      __syncwarp();
      uint32_t rank[IPT];
      if (warp_live) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
          if (32 * i >= chunk) break;
          const bool ok = e_warp + i * 32 + (int)lane < n;
          const unsigned d = ok ? KeyTraits<K>::digit(k[i], bit, nb) : 256u;
          const unsigned peers = __match_any_sync(FULL, d);
          const int leader = __ffs(peers) - 1;
          uint32_t base = 0;
          if (ok && (int)lane == leader) {
            base = s.cnt[w][d];
            s.cnt[w][d] = base + __popc(peers);
          }
          base = __shfl_sync(FULL, base, leader);
          rank[i] = base + __popc(peers & lanemask_lt());
          __syncwarp();
        }
      }
      __syncthreads();
      // Exclusive scan of the counters in (digit, warp) order: thread t owns
      // digit t/(NW/8) and warps (t%(NW/8))*8 .. +8.
      {
        const int d = threadIdx.x / (NW / 8);
        const int w0 = (threadIdx.x % (NW / 8)) * 8;
        uint32_t c[8], sum = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) { c[j] = s.cnt[w0 + j][d]; sum += c[j]; }
        uint32_t total;
        uint32_t pre = block_excl_scan<uint32_t, THREADS>(sum, s.ws, &total);
#pragma unroll
        for (int j = 0; j < 8; ++j) { s.cnt[w0 + j][d] = pre; pre += c[j]; }
      }
      __syncthreads();
      if (warp_live) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
          if (32 * i >= chunk) break;
          if (e_warp + i * 32 + (int)lane < n) {
            const unsigned d = KeyTraits<K>::digit(k[i], bit, nb);
            const uint32_t pos = s.cnt[w][d] + rank[i];
            s.keys[pos] = k[i];
            if constexpr (HAS_V) s.vals[pos] = v[i];
          }
        }
      }
      __syncthreads();
      if (bit + 8 < nbits) {
        if (warp_live) {
#pragma unroll
          for (int i = 0; i < IPT; ++i) {
            if (32 * i >= chunk) break;
            const int e = e_warp + i * 32 + lane;
            if (e < n) {
              k[i] = s.keys[e];
              if constexpr (HAS_V) v[i] = s.vals[e];
            }
          }
        }
        __syncthreads();
      }
    }
    if (nbits <= 0) {  // nothing to sort: still leave the keys in smem, in order
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        if (valid(n, i)) {
          const int e = elem(n, i);
          s.keys[e] = k[i];
          if constexpr (HAS_V) s.vals[e] = v[i];
        }
      }
      __syncthreads();
    }
  }
};

// Bits that vary inside a tile whose keys share the top `D` digit bits in
// [d_first, d_last] and have `key_bits` significant bits.
__host__ __device__ __forceinline__ int tile_sort_bits(int key_bits, int D, uint32_t d_first,
                                                       uint32_t d_last) {
  uint32_t x = d_first ^ d_last;
  int diff = 0;
  while (x) { ++diff; x >>= 1; }
  return key_bits - D + diff;
}

// ------------------------------------------------------ tile descriptors
// A tile plan over digit buckets.  Buckets are grouped (one group per bin;
// a single group for a plain pair sort); group g has 2^D[g] buckets, the
// first at flattened index group_base[g].  bucket_base[i] = first key of
// bucket i (exclusive scan of the counts; bucket_base[NB] = total).
// tile_first[t] = flattened index of the first bucket of tile t; a tile
// never crosses a group boundary and ends where tile t+1 begins.
// Key range and group of one tile, precomputed so that a CTA takes its next
// tile with one load.
struct TileDesc {
  uint64_t st;     // first key
  uint32_t n;      // keys
  uint32_t group;  // group (bin) of the tile
};

struct TilePlan {
  const uint64_t *bucket_base;  // [NB + 1]
  const uint32_t *tile_first;   // [n_tiles]
  const uint32_t *n_tiles;      // device scalar
  const uint32_t *group_base;   // [n_groups + 1]
  const uint8_t *group_D;       // [n_groups]
  uint32_t n_groups;
  uint32_t NB;                  // total buckets
  int key_bits;
  const TileDesc *desc = nullptr;  // optional: [n_tiles] ranges (tile_desc_kernel)
  uint32_t debug = 0;              // 1: tile_group_kernel times out on purpose (failure-path check)
  const uint8_t *skip_group = nullptr;  // optional: groups counted elsewhere (their tiles get n = 0)
};

// Group holding bucket i (largest g with group_base[g] <= i).
__device__ __forceinline__ uint32_t group_of(const uint32_t *group_base, uint32_t n_groups,
                                             uint32_t i) {
  uint32_t lo = 0, hi = n_groups;  // invariant: group_base[lo] <= i < group_base[hi]
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) / 2;
    if (group_base[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// Key range of tile t and the number of low key bits that vary inside it.
__device__ __forceinline__ void tile_range(const TilePlan &p, uint32_t t, uint32_t nt,
                                           uint64_t *start, uint64_t *end, int *nbits,
                                           uint32_t *group = nullptr) {
  const uint32_t i = p.tile_first[t];
  const uint32_t j = (t + 1 < nt) ? p.tile_first[t + 1] : p.NB;  // one past the last bucket
  *start = p.bucket_base[i];
  *end = p.bucket_base[j];
  const uint32_t g = group_of(p.group_base, p.n_groups, i);
  const uint32_t d0 = i - p.group_base[g], d1 = j - 1 - p.group_base[g];
  *nbits = tile_sort_bits(p.key_bits, p.group_D[g], d0, d1);
  if (group) *group = g;
}

// desc[t] for every tile t < *plan.n_tiles (grid-stride).
static __global__ void tile_desc_kernel(TilePlan plan, TileDesc *desc) {
  const uint32_t nt = *plan.n_tiles;
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    uint64_t st, en;
    int nbits;
    uint32_t group;
    tile_range(plan, t, nt, &st, &en, &nbits, &group);
    uint64_t n = en - st;
    if (plan.skip_group && plan.skip_group[group]) n = 0;  // counted by super_hash_kernel
    desc[t] = {st, n > 0xFFFFFFFFull ? 0xFFFFFFFFu : (uint32_t)n, group};
  }
}

// Optional bijective mix of the keys (2^bits values onto themselves): the
// digit buckets use the top bits of mix(key), which spreads keys evenly
// whatever their structure; equal keys still share a bucket and a tile.
// x -> x ^ (x >> s1) -> x * c (mod 2^bits) -> x ^ (x >> s2), c odd.
template <typename K>
struct Mixer {
  K c, cinv, mask;
  int bits, s1, s2;
  bool on;
  __device__ __forceinline__ K mix(K x) const {
    if (!on) return x;
    x ^= x >> s1;
    x = (x * c) & mask;
    x ^= x >> s2;
    return x;
  }
  __device__ __forceinline__ K unmix(K y) const {
    if (!on) return y;
    for (int t = s2; t < bits; t <<= 1) y ^= y >> t;
    y = (y * cinv) & mask;
    for (int t = s1; t < bits; t <<= 1) y ^= y >> t;
    return y;
  }
};

// ---------------------------------------------------------------- tile kernels

// Grabs the next tile index for the whole CTA (persistent-CTA work loop).
__device__ __forceinline__ uint32_t next_tile(uint32_t *work, uint32_t *s_tile) {
  if (threadIdx.x == 0) *s_tile = atomicAdd(work, 1u);
  __syncthreads();
  uint32_t t = *s_tile;
  __syncthreads();
  return t;
}

__device__ __forceinline__ void push_big(uint32_t t, uint64_t n, uint32_t *big_list,
                                         uint32_t *n_big, unsigned long long *big_keys,
                                         uint32_t big_cap, uint32_t *err) {
  uint32_t idx = atomicAdd(n_big, 1u);
  if (idx < big_cap) {
    big_list[idx] = t;
    atomicAdd(big_keys, (unsigned long long)n);
  } else {
    atomicOr(err, ERR_CAPACITY);
  }
}

// Output of run-length counting: the survivors of a tile, sorted.
template <typename K>
struct CountOut {
  K *keys;                     // survivor k-mers
  uint32_t *counts;            // their counts
  unsigned long long *n;       // survivors written so far (device counter)
  uint64_t cap;                // capacity of keys/counts
  uint64_t ci, cx;             // inclusive cutoffs (Sect. 2.5)
  unsigned long long *n_distinct;
  Mixer<K> mixer;              // keys in the tiles are mixed; survivors are not
  int sort_bits;               // tiles are sorted on this many low bits (<= 24)
  uint32_t *slots;             // batches: set of each survivor (group / bins_per_slot), else NULL
  uint32_t bins_per_slot;
};

// Sect. 2.4 "calculates the statistics": run-length count of the sorted keys
// s_keys[0..n) of one tile, keep counts in [ci, cx], append to `out`.
template <typename K, int THREADS, int IPT>
__device__ void tile_rle(const K *s_keys, int n, uint16_t *heads, uint32_t *ws,
                         unsigned long long *s_base, const CountOut<K> &out, uint32_t *err,
                         uint32_t group) {
  const int e0 = threadIdx.x * IPT;
  uint32_t nh = 0;
#pragma unroll 4
  for (int j = 0; j < IPT; ++j) {
    int e = e0 + j;
    if (e < n && (e == 0 || s_keys[e] != s_keys[e - 1])) ++nh;
  }
  uint32_t U;
  uint32_t hb = block_excl_scan<uint32_t, THREADS>(nh, ws, &U);
#pragma unroll 4
  for (int j = 0; j < IPT; ++j) {
    int e = e0 + j;
    if (e < n && (e == 0 || s_keys[e] != s_keys[e - 1])) heads[hb++] = (uint16_t)e;
  }
  if (threadIdx.x == 0) heads[U] = (uint16_t)n;
  __syncthreads();
  const uint32_t Q = (U + THREADS - 1) / THREADS;
  const uint32_t u0 = threadIdx.x * Q;
  uint32_t keep = 0;
  for (uint32_t j = 0; j < Q; ++j) {
    uint32_t u = u0 + j;
    if (u < U) {
      uint32_t c = (uint32_t)heads[u + 1] - heads[u];
      keep += (c >= out.ci && c <= out.cx);
    }
  }
  uint32_t ktot;
  uint32_t kb = block_excl_scan<uint32_t, THREADS>(keep, ws, &ktot);
  if (threadIdx.x == 0) {
    *s_base = ktot ? atomicAdd(out.n, (unsigned long long)ktot) : 0ull;
    atomicAdd(out.n_distinct, (unsigned long long)U);
  }
  __syncthreads();
  const uint64_t base = *s_base;
  if (base + ktot > out.cap) {
    if (threadIdx.x == 0) atomicOr(err, ERR_CAPACITY);
  } else {
    for (uint32_t j = 0; j < Q; ++j) {
      uint32_t u = u0 + j;
      if (u < U) {
        uint32_t h = heads[u];
        uint32_t c = (uint32_t)heads[u + 1] - h;
        if (c >= out.ci && c <= out.cx) {
          out.keys[base + kb] = out.mixer.unmix(s_keys[h]);
          out.counts[base + kb] = c;
          if (out.slots) out.slots[base + kb] = group / out.bins_per_slot;
          ++kb;
        }
      }
    }
  }
  __syncthreads();
}

// Count mode sorts a tile on the low kCountSortBits bits of its (mixed,
// uniformly spread) keys only, which already puts equal keys next to each
// other unless two different keys of the tile share those bits.  Such runs
// are rare (about t^2/2^25 per tile of t distinct keys) and are repaired by
// group_equal_runs before counting.
constexpr int kCountSortBits = 24;

template <typename K>
__device__ __forceinline__ uint32_t low_bits(K x, int bits) {
  return (uint32_t)(uint64_t)x & ((1u << bits) - 1u);
}

// In s[0..n), sorted on the low kCountSortBits bits: every maximal run of
// equal low bits that holds more than one key value is regrouped so that
// equal keys are adjacent (one thread per dirty run; O(run x values)).
template <typename K, int THREADS>
__device__ void group_equal_runs(K *s, int n, int bits) {
  bool dirty = false;
  for (int e = threadIdx.x + 1; e < n; e += THREADS)
    dirty |= (low_bits(s[e], bits) == low_bits(s[e - 1], bits)) && (s[e] != s[e - 1]);
  if (!__syncthreads_or(dirty)) return;
  // thread t handles the dirty runs that start in its stride positions
  for (int e = threadIdx.x; e < n; e += THREADS) {
    const bool starts_run = e == 0 || low_bits(s[e], bits) != low_bits(s[e - 1], bits);
    if (!starts_run) continue;
    int b = e + 1;
    bool mixed = false;
    while (b < n && low_bits(s[b], bits) == low_bits(s[e], bits)) {
      mixed |= s[b] != s[e];
      ++b;
    }
    if (!mixed) continue;
    for (int i = e; i < b;) {  // move every copy of s[i] next to it
      const K key = s[i];
      int j = i + 1;
      for (int q = i + 1; q < b; ++q) {
        if (s[q] == key) {
          const K t = s[q];
          s[q] = s[j];
          s[j] = t;
          ++j;
        }
      }
      i = j;
    }
  }
  __syncthreads();
}

// group_equal_runs for (key, value) pairs: values move with their keys.
template <typename K, typename V, int THREADS>
__device__ void group_equal_runs_kv(K *s, V *v, int n, int bits) {
  bool dirty = false;
  for (int e = threadIdx.x + 1; e < n; e += THREADS)
    dirty |= (low_bits(s[e], bits) == low_bits(s[e - 1], bits)) && (s[e] != s[e - 1]);
  if (!__syncthreads_or(dirty)) return;
  for (int e = threadIdx.x; e < n; e += THREADS) {
    const bool starts_run = e == 0 || low_bits(s[e], bits) != low_bits(s[e - 1], bits);
    if (!starts_run) continue;
    int b = e + 1;
    bool mixed = false;
    while (b < n && low_bits(s[b], bits) == low_bits(s[e], bits)) {
      mixed |= s[b] != s[e];
      ++b;
    }
    if (!mixed) continue;
    for (int i = e; i < b;) {
      const K key = s[i];
      int j = i + 1;
      for (int q = i + 1; q < b; ++q) {
        if (s[q] == key) {
          const K tk = s[q];
          s[q] = s[j];
          s[j] = tk;
          const V tv = v[q];
          v[q] = v[j];
          v[j] = tv;
          ++j;
        }
      }
      i = j;
    }
  }
  __syncthreads();
}

template <typename K, int THREADS, int IPT>
struct TileCountSmem {
  typename BlockSort<K, NoVal, THREADS, IPT>::Smem bs;
  uint16_t heads[THREADS * IPT + 1];
  uint32_t tile;
  unsigned long long base;
};

// Count mode: sort every tile of the plan and run-length count it (x = 0:
// the keys are canonical k-mers).  Tiles above one CTA's capacity are put on
// the big list.  If `sorted_out` is not NULL the sorted keys are also
// written back there (inspection).
template <typename K, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS, (THREADS * IPT * sizeof(K) <= 32768) ? 3 : 1)
tile_count_kernel(const K *__restrict__ keys, TilePlan plan, uint32_t *work, CountOut<K> out,
                  uint32_t *big_list, uint32_t *n_big, unsigned long long *big_keys,
                  uint32_t big_cap, uint32_t *err, K *sorted_out) {
  using BS = BlockSort<K, NoVal, THREADS, IPT>;
  using SM = TileCountSmem<K, THREADS, IPT>;
  static_assert(BS::TILE < 65536, "heads are 16-bit");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &sm = *reinterpret_cast<SM *>(smem_raw);
  const uint32_t nt = *plan.n_tiles;
  const unsigned lane = lane_id();
  for (;;) {
    const uint32_t t = next_tile(work, &sm.tile);
    if (t >= nt) break;
    uint64_t st, en;
    int nbits;
    uint32_t group;
    tile_range(plan, t, nt, &st, &en, &nbits, &group);
    const uint64_t n64 = en - st;
    if (n64 == 0) continue;
    if (n64 > (uint64_t)BS::TILE) {
      if (threadIdx.x == 0) push_big(t, n64, big_list, n_big, big_keys, big_cap, err);
      continue;
    }
    const int n = (int)n64;
    K k[IPT];
    NoVal v[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i)
      if (BS::valid(n, i)) k[i] = keys[st + BS::elem(n, i)];
    BS::sort(k, v, nbits < out.sort_bits ? nbits : out.sort_bits, n, sm.bs);
    if (nbits > out.sort_bits) group_equal_runs<K, THREADS>(sm.bs.keys, n, out.sort_bits);
    if (sorted_out)
      for (int e = threadIdx.x; e < n; e += THREADS) sorted_out[st + e] = sm.bs.keys[e];
    tile_rle<K, THREADS, IPT>(sm.bs.keys, n, sm.heads, sm.bs.ws, &sm.base, out, err, group);
  }
}

// ----------------------------------------------------- grouping count tiles
// Count mode without a full sort.  Counting needs equal keys side by side,
// not the keys in order: the survivors are put in k-mer order afterwards
// anyway, and the keys of a tile are mixed.  So a tile takes one more radix
// partition step, on the low kGroupBits bits of its keys (one shared-memory
// atomic per key gives both the digit histogram and the key's rank in its
// digit).  A digit bucket then mostly holds copies of one key (at 60x
// coverage a genomic k-mer has dozens), sometimes a few values.  The values
// of a bucket are separated in rounds: each round every unsettled key
// compares itself with the bucket's representative (first the bucket's
// first key, then any unsettled key); the equal ones settle, and the rest
// count themselves, so the representative's group size is the drop of that
// count.  Rounds = most values in one bucket; heavy keys cost no serial work.
// The tile's keys are staged in shared memory by a bulk copy started while
// the previous tile is still being counted.
constexpr int kGroupBits = 11;
constexpr int kGroupDigits = 1 << kGroupBits;

template <typename K, int THREADS, int IPT>
struct TileGroupSmem {
  static constexpr int TILE = THREADS * IPT;
  static constexpr int PAD = 16 / sizeof(K);  // the staged range starts on a 16-byte boundary
  K a[TILE + 2 * PAD];            // staged keys (bulk copy target)
  K b[TILE];                      // keys partitioned by their low digit
  // digit counts, then bucket offsets (off[kGroupDigits] = n); after the
  // scatter: per digit, keys left unsettled by the last two rounds (16-bit halves)
  uint32_t off[kGroupDigits + 4];
  uint16_t rep[kGroupDigits];     // position in b of each bucket's current representative
  // keys left after the first round: position (bits 0-11), group count
  // (bits 12-24), settled (bit 30), group head (bit 31)
  uint32_t wl[THREADS * IPT];
  uint32_t ws[THREADS / 32 + 1];
  uint64_t ws64[THREADS / 32 + 1];
  uint64_t bar;                   // mbarrier of the bulk copies
  uint64_t bar_never;             // an mbarrier nothing arrives on (failure-path check)
  unsigned long long base;
  // the tile whose copy is in flight (t_next = number of tiles when none is)
  uint32_t t_next, n_next, lead_next, group_next;
};

// Thread 0: takes tiles until one fits (bigger ones go to the big list,
// empty ones are skipped), starts its bulk copy and records it.
// SM: shared-memory layout with a (copy target), bar, t_next, n_next,
// lead_next, group_next and the tile capacity TILE.
template <typename K, typename SM>
__device__ void tile_fetch(const K *keys, const TilePlan &plan, uint32_t nt, uint32_t *work, SM &s,
                           uint32_t *big_list, uint32_t *n_big, unsigned long long *big_keys,
                           uint32_t big_cap, uint32_t *err) {
  for (;;) {
    const uint32_t t = atomicAdd(work, 1u);
    if (t >= nt) {
      s.t_next = nt;
      return;
    }
    const TileDesc d = plan.desc[t];
    if (d.n == 0) continue;
    if (d.n > (uint32_t)SM::TILE) {
      push_big(t, d.n, big_list, n_big, big_keys, big_cap, err);
      continue;
    }
    // copy the 16-byte aligned cover of keys[st, st + n) (the key buffers
    // keep 16 bytes of slack past their last key)
    const uintptr_t src = reinterpret_cast<uintptr_t>(keys + d.st);
    const uintptr_t src0 = src & ~(uintptr_t)15;
    const uint32_t bytes = (uint32_t)((src + (uint64_t)d.n * sizeof(K) - src0 + 15) & ~(uintptr_t)15);
    s.t_next = t;
    s.n_next = d.n;
    s.lead_next = (uint32_t)((src - src0) / sizeof(K));
    s.group_next = d.group;
    fence_proxy_async_smem();
    bulk_load(s.a, reinterpret_cast<const void *>(src0), bytes, &s.bar);
    return;
  }
}

// Counts the n keys at s.a[lead ..] of one tile (all threads; the caller
// has passed a barrier after the previous tile's output).  Thread 0 calls
// after_load() once the keys are in registers and s.a may be refilled.
template <typename K, int THREADS, int IPT, typename F>
__device__ __forceinline__ void group_core(TileGroupSmem<K, THREADS, IPT> &s, int n, int lead, uint32_t group,
                                           const CountOut<K> &out, uint32_t *err, F after_load) {
  constexpr int DPT = kGroupDigits / THREADS;  // digit counters scanned per thread
  static_assert(DPT == 4 || DPT == 8 || DPT == 16, "scan uses 16-byte loads");
  static_assert(TileGroupSmem<K, THREADS, IPT>::TILE <= 4096, "positions and counts are 12/13-bit fields");
  // per-key state: position in b (bits 0-12), group count (bits 13-25),
  // settled (bit 30), group head (bit 31)
  constexpr uint32_t POS = 0x1FFFu, SETTLED = 1u << 30, HEAD = 1u << 31;
  const int tid = threadIdx.x;
  for (int i = tid; i < kGroupDigits + 4; i += THREADS) s.off[i] = 0;
  K key[IPT];
  uint32_t st[IPT];
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const int e = tid + i * THREADS;
    st[i] = SETTLED;  // keys past n take no part
    if (e < n) key[i] = s.a[lead + e];
  }
  __syncthreads();  // s.a consumed, s.off zeroed
  if (tid == 0) after_load();
  // digit histogram; the returned old count is the key's rank in its digit
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const int e = tid + i * THREADS;
    if (e < n) st[i] = atomicAdd(&s.off[(uint32_t)(uint64_t)key[i] & (kGroupDigits - 1)], 1u);
  }
  __syncthreads();
  // exclusive scan of the digit counts (thread t: counters [DPT t, DPT t + DPT))
  {
    uint32_t c[DPT];
#pragma unroll
    for (int q = 0; q < DPT; q += 4) {
      const uint4 v = *reinterpret_cast<const uint4 *>(&s.off[DPT * tid + q]);
      c[q] = v.x; c[q + 1] = v.y; c[q + 2] = v.z; c[q + 3] = v.w;
    }
    uint32_t sum = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) sum += c[q];
    uint32_t tot;
    uint32_t run = block_excl_scan<uint32_t, THREADS>(sum, s.ws, &tot);
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const uint32_t x = c[q];
      c[q] = run;
      run += x;
    }
#pragma unroll
    for (int q = 0; q < DPT; q += 4)
      *reinterpret_cast<uint4 *>(&s.off[DPT * tid + q]) = make_uint4(c[q], c[q + 1], c[q + 2], c[q + 3]);
    if (tid == 0) s.off[kGroupDigits] = (uint32_t)n;
  }
  __syncthreads();
  // scatter; a bucket's first key becomes its representative and carries
  // the bucket size
  uint32_t bsize[IPT];
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const int e = tid + i * THREADS;
    bsize[i] = 0;
    if (e < n) {
      const uint32_t d = (uint32_t)(uint64_t)key[i] & (kGroupDigits - 1);
      const uint32_t lo = s.off[d], p = lo + st[i];
      s.b[p] = key[i];
      if (st[i] == 0) {
        s.rep[d] = (uint16_t)p;
        bsize[i] = s.off[d + 1] - lo;
      }
      st[i] = p;  // unsettled
    }
  }
  __syncthreads();  // s.off (offsets) no longer needed: it now holds the unsettled counts
#pragma unroll
  for (int i = 0; i < IPT; ++i)
    if (bsize[i]) s.off[(uint32_t)(uint64_t)key[i] & (kGroupDigits - 1)] = bsize[i];
  __syncthreads();
  // rounds: count j of unsettled keys sits in half j & 1 of the digit's
  // word.  Round 1 (each bucket's first key represents it) runs on the keys
  // in registers; the few keys it leaves go to a work list for the rest.
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    if (st[i] & SETTLED) continue;
    const uint32_t d = (uint32_t)(uint64_t)key[i] & (kGroupDigits - 1);
    const uint32_t r = s.rep[d];
    if (s.b[r] == key[i]) st[i] |= SETTLED | (r == (st[i] & POS) ? HEAD : 0u);
    else atomicAdd(&s.off[d], 0x10000u);
  }
  __syncthreads();
  uint32_t left = 0;
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    if (st[i] & HEAD) {
      const uint32_t d = (uint32_t)(uint64_t)key[i] & (kGroupDigits - 1);
      const uint32_t w = s.off[d];
      st[i] |= ((w & 0xFFFFu) - (w >> 16)) << 13;
      s.off[d] = w & 0xFFFF0000u;
    }
    left += !(st[i] & SETTLED);
  }
  uint32_t n_wl;
  uint32_t wo = block_excl_scan<uint32_t, THREADS>(left, s.ws, &n_wl);
  if (left) {
#pragma unroll
    for (int i = 0; i < IPT; ++i)
      if (!(st[i] & SETTLED)) s.wl[wo++] = st[i] & POS;
  }
  constexpr uint32_t WPOS = 0xFFFu;
  if (n_wl) {
    __syncthreads();
    for (uint32_t round = 2;; ++round) {
      // representatives: any unsettled key of the bucket
      for (uint32_t e = tid; e < n_wl; e += THREADS) {
        const uint32_t x = s.wl[e];
        if (!(x & SETTLED)) s.rep[(uint32_t)(uint64_t)s.b[x & WPOS] & (kGroupDigits - 1)] = (uint16_t)(x & WPOS);
      }
      __syncthreads();
      const uint32_t inc = (round & 1) ? 0x10000u : 1u;
      for (uint32_t e = tid; e < n_wl; e += THREADS) {
        const uint32_t x = s.wl[e];
        if (x & SETTLED) continue;
        const uint32_t p = x & WPOS;
        const K kk = s.b[p];
        const uint32_t d = (uint32_t)(uint64_t)kk & (kGroupDigits - 1);
        const uint32_t r = s.rep[d];
        if (s.b[r] == kk) s.wl[e] = x | SETTLED | (r == p ? HEAD : 0u);
        else atomicAdd(&s.off[d], inc);
      }
      __syncthreads();
      bool more = false;
      for (uint32_t e = tid; e < n_wl; e += THREADS) {
        const uint32_t x = s.wl[e];
        if ((x & HEAD) && ((x >> 12) & 0x1FFFu) == 0) {
          // this round's representative: its group is the drop of the count
          const uint32_t d = (uint32_t)(uint64_t)s.b[x & WPOS] & (kGroupDigits - 1);
          const uint32_t w = s.off[d];
          const uint32_t prev = (round & 1) ? (w & 0xFFFFu) : (w >> 16);
          const uint32_t cur = (round & 1) ? (w >> 16) : (w & 0xFFFFu);
          s.wl[e] = x | ((prev - cur) << 12);
          s.off[d] = (round & 1) ? (w & 0xFFFF0000u) : (w & 0xFFFFu);
        }
        more |= !(x & SETTLED);
      }
      if (!__syncthreads_or(more)) break;
    }
  }
  // survivors, in key order per thread; one scan gives both the survivor
  // offsets (low half) and the group total (high half)
  uint32_t n_groups = 0, n_keep = 0;
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    if (!(st[i] & HEAD)) continue;
    const uint32_t c = (st[i] >> 13) & 0x1FFFu;
    ++n_groups;
    n_keep += c >= out.ci && c <= out.cx;
  }
  for (uint32_t e = tid; e < n_wl; e += THREADS) {
    const uint32_t x = s.wl[e];
    if (!(x & HEAD)) continue;
    const uint32_t c = (x >> 12) & 0x1FFFu;
    ++n_groups;
    n_keep += c >= out.ci && c <= out.cx;
  }
  uint64_t tot2;
  const uint64_t pre = block_excl_scan<uint64_t, THREADS>(((uint64_t)n_groups << 32) | n_keep,
                                                          s.ws64, &tot2);
  uint32_t kb = (uint32_t)pre;
  const uint32_t ktot = (uint32_t)tot2;
  if (tid == 0) {
    s.base = ktot ? atomicAdd(out.n, (unsigned long long)ktot) : 0ull;
    atomicAdd(out.n_distinct, tot2 >> 32);
  }
  __syncthreads();
  const uint64_t base = s.base;
  if (base + ktot > out.cap) {
    if (tid == 0) atomicOr(err, ERR_CAPACITY);
  } else if (n_keep) {
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      if (!(st[i] & HEAD)) continue;
      const uint32_t c = (st[i] >> 13) & 0x1FFFu;
      if (c >= out.ci && c <= out.cx) {
        out.keys[base + kb] = out.mixer.unmix(key[i]);
        out.counts[base + kb] = c;
        if (out.slots) out.slots[base + kb] = group / out.bins_per_slot;
        ++kb;
      }
    }
    for (uint32_t e = tid; e < n_wl; e += THREADS) {
      const uint32_t x = s.wl[e];
      if (!(x & HEAD)) continue;
      const uint32_t c = (x >> 12) & 0x1FFFu;
      if (c >= out.ci && c <= out.cx) {
        out.keys[base + kb] = out.mixer.unmix(s.b[x & WPOS]);
        out.counts[base + kb] = c;
        if (out.slots) out.slots[base + kb] = group / out.bins_per_slot;
        ++kb;
      }
    }
  }
}

template <typename K, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS, 2)
tile_group_kernel(const K *__restrict__ keys, TilePlan plan, uint32_t *work, CountOut<K> out,
                  uint32_t *big_list, uint32_t *n_big, unsigned long long *big_keys, uint32_t big_cap,
                  uint32_t *err) {
  // plan.desc is required; tiles are claimed from *work (zero at launch)
  using SM = TileGroupSmem<K, THREADS, IPT>;
  static_assert(offsetof(SM, off) % 16 == 0 && offsetof(SM, a) == 0, "16-byte aligned arrays");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const uint32_t nt = *plan.n_tiles;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&s.bar, 1);
    mbar_init(&s.bar_never, 1);
    tile_fetch<K>(keys, plan, nt, work, s, big_list, n_big, big_keys, big_cap, err);
  }
  __syncthreads();
  uint32_t parity = 0;
  for (;;) {
    if (s.t_next >= nt) break;
    const int n = (int)s.n_next, lead = (int)s.lead_next;
    const uint32_t group = s.group_next;
    // thread 0 waits for the copy; the barrier passes its result (and the
    // copied data) on to the others, and ends the previous tile.  The
    // failure-path check waits (200 us at most) on a barrier that never
    // completes instead, so that the code below runs.
    const bool ok = tid != 0 || ((plan.debug & 1u) ? mbar_wait(&s.bar_never, 0u, 200000ull)
                                                   : mbar_wait(&s.bar, parity));
    if (!__syncthreads_and(ok)) {
      // the copy did not land in time: report, give it one more bounded
      // wait so that no copy is left in flight, and stop
      if (tid == 0) {
        atomicOr(err, ERR_TIMEOUT);
        mbar_wait(&s.bar, parity);
      }
      return;
    }
    parity ^= 1u;
    group_core<K, THREADS, IPT>(s, n, lead, group, out, err, [&]() {
      tile_fetch<K>(keys, plan, nt, work, s, big_list, n_big, big_keys, big_cap, err);
    });
  }
}

// ------------------------------------------------------- hashed count tiles
// Count mode for 64-bit keys below 2^62 (k <= 31): the keys of a tile go
// into an open-addressing table in shared memory (1.25 slots per key of a
// full tile, linear probing from the key's low bits, one 64-bit CAS to claim
// a slot and one atomic add to count), and the occupied slots are the tile's
// distinct keys.  Same input and output as tile_group_kernel with far fewer
// steps per key; copies of one key meet at one slot whatever their number.
// The tile's keys are read straight into registers (coalesced 8-byte
// loads): without a staging buffer three CTAs fit an SM and hide the load
// latency of one another (measured faster than bulk-copy staging, which
// leaves room for two).
constexpr int HASH_THREADS = 512;
constexpr int HASH_SLOTS = 5120;
constexpr unsigned long long kHashEmpty = ~0ull;

template <int THREADS, int IPT>
struct TileHashSmem {
  static constexpr int TILE = THREADS * IPT;
  static constexpr int SLOTS = HASH_SLOTS;
  unsigned long long tk[SLOTS];    // slot keys (kHashEmpty when free)
  uint32_t tc[SLOTS];              // slot counts
  unsigned long long start[2];     // tiles, alternately: first key, index, keys, group
  uint32_t t[2], n[2], group[2];
};

// Thread 0: claims the next tile that fits (bigger ones go to the big list)
// and records it in slot q of s.start/t/n/group (t = number of tiles when
// none is left).
template <typename SM>
__device__ void hash_claim(SM &s, int q, const TilePlan &plan, uint32_t nt, uint32_t *work, uint32_t *big_list,
                           uint32_t *n_big, unsigned long long *big_keys, uint32_t big_cap, uint32_t *err) {
  for (;;) {
    const uint32_t t = atomicAdd(work, 1u);
    s.t[q] = t;
    if (t >= nt) return;
    const TileDesc d = plan.desc[t];
    if (d.n == 0) continue;
    if (d.n > (uint32_t)SM::TILE) {
      push_big(t, d.n, big_list, n_big, big_keys, big_cap, err);
      continue;
    }
    s.start[q] = d.st;
    s.n[q] = d.n;
    s.group[q] = d.group;
    return;
  }
}

// Two barriers per tile: inserts | emission (which also clears the slots
// for the next tile) |.  Each warp reserves its survivors' places with one
// global atomic, so no block-wide scan is needed; the tile record is double
// buffered so that thread 0 claims the next tile while this one is counted.
template <int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS, 3)
tile_hash_kernel(const uint64_t *__restrict__ keys, TilePlan plan, uint32_t *work, CountOut<uint64_t> out,
                 uint32_t *big_list, uint32_t *n_big, unsigned long long *big_keys, uint32_t big_cap,
                 uint32_t *err) {
  using SM = TileHashSmem<THREADS, IPT>;
  constexpr int SPT = SM::SLOTS / THREADS;  // slots per thread
  static_assert(SM::SLOTS % THREADS == 0 && SM::SLOTS > SM::TILE, "layout");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  const uint32_t nt = *plan.n_tiles;
  const int tid = threadIdx.x;
  const unsigned lane = lane_id();
  // clear the table (thread t owns slots t, t + THREADS, ...)
#pragma unroll
  for (int q = 0; q < SPT; ++q) {
    s.tk[q * THREADS + tid] = kHashEmpty;
    s.tc[q * THREADS + tid] = 0;
  }
  if (tid == 0) hash_claim(s, 0, plan, nt, work, big_list, n_big, big_keys, big_cap, err);
  __syncthreads();
  unsigned long long n_distinct = 0;
  for (int it = 0;; ++it) {
    const int cur = it & 1;
    if (s.t[cur] >= nt) break;
    const int n = (int)s.n[cur];
    const uint64_t *src = keys + s.start[cur];
    const uint32_t group = s.group[cur];
    // the next tile is claimed while this one is counted
    if (tid == 0) hash_claim(s, cur ^ 1, plan, nt, work, big_list, n_big, big_keys, big_cap, err);
    uint64_t key[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      const int e = tid + i * THREADS;
      key[i] = e < n ? src[e] : kHashEmpty;
    }
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      if (key[i] == kHashEmpty) continue;
      // first slot: the key's low 32 bits scaled to [0, SLOTS)
      uint32_t h = (uint32_t)(((uint64_t)(uint32_t)key[i] * SM::SLOTS) >> 32);
      for (;;) {  // at most n < SLOTS probes: the table is never full
        const unsigned long long old = atomicCAS(&s.tk[h], kHashEmpty, key[i]);
        if (old == kHashEmpty || old == key[i]) break;
        h = h + 1 == (uint32_t)SM::SLOTS ? 0u : h + 1;
      }
      atomicAdd(&s.tc[h], 1u);
    }
    __syncthreads();
    // occupied slots are the tile's distinct keys; read and clear them
    uint32_t keep = 0;  // bit q: slot q * THREADS + tid survives
    uint32_t cc[SPT];
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
      cc[q] = s.tc[q * THREADS + tid];
      n_distinct += cc[q] != 0;
      if (cc[q] >= out.ci && cc[q] <= out.cx) keep |= 1u << q;  // ci >= 1
    }
    const uint32_t nk = (uint32_t)__popc(keep);
    const uint32_t incl = warp_incl_scan(nk);
    const uint32_t wtot = __shfl_sync(FULL, incl, 31);
    unsigned long long wbase = 0;
    if (lane == 31 && wtot) wbase = atomicAdd(out.n, (unsigned long long)wtot);
    wbase = __shfl_sync(FULL, wbase, 31);
    const bool fits = wbase + wtot <= out.cap;
    if (!fits && lane == 0) atomicOr(err, ERR_CAPACITY);
    uint64_t p = wbase + incl - nk;
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
      if (cc[q]) {
        const int e = q * THREADS + tid;
        if (fits && ((keep >> q) & 1u)) {
          out.keys[p] = out.mixer.unmix(s.tk[e]);
          out.counts[p] = cc[q];
          if (out.slots) out.slots[p] = group / out.bins_per_slot;
          ++p;
        }
        s.tk[e] = kHashEmpty;
        s.tc[e] = 0;
      }
    }
    __syncthreads();  // the slots are clear and the next tile is claimed
  }
  const unsigned long long nd = __reduce_add_sync(FULL, (unsigned)n_distinct);
  if (lane == 0 && nd) atomicAdd(out.n_distinct, nd);
}

// ------------------------------------------------ hashed count of super buckets
// For bins whose super buckets (the upper radix sweep's output) hold at most
// a few ten thousand keys, the lower sweep and the tile count are replaced
// by one pass over each super bucket: a CTA claims a super bucket and counts
// its keys (mixed, below 2^62) in an open-addressing table in shared memory
// (linear probing from the key's low bits, a 64-bit CAS to claim a slot, an
// add to count), then emits the slots whose count is inside the cutoffs.
// Every key is read once from HBM and nothing is written but the survivors.
// Keys go in in batches of SUPER_BATCH; a batch starts only while at most
// SUPER_LIMIT slots are taken, so the table never fills (SUPER_LIMIT +
// SUPER_BATCH < SUPER_SLOTS) and every probe ends.  A super bucket with more
// distinct keys is counted in P passes instead (P = 2, 4, ...; pass p takes
// the keys whose multiplicative hash selects p, so all copies of a key fall
// in one pass), re-reading it, mostly from L2; a pass that overflows is split
// in two without recounting the passes already emitted.
#ifndef KMC_SUPER_SLOTS
#define KMC_SUPER_SLOTS 8192
#endif
#ifndef KMC_SUPER_UNROLL
#define KMC_SUPER_UNROLL 4
#endif
#ifndef KMC_SUPER_MINB
#define KMC_SUPER_MINB 2
#endif
constexpr int SUPER_THREADS = 512;
constexpr int SUPER_SLOTS = KMC_SUPER_SLOTS;
constexpr int SUPER_UNROLL = KMC_SUPER_UNROLL;
constexpr int SUPER_BATCH = SUPER_THREADS * SUPER_UNROLL;
constexpr int SUPER_LIMIT = SUPER_SLOTS - 1 - SUPER_BATCH;
constexpr uint32_t SUPER_MAX_PASSES = 1u << 16;

struct SuperHashSmem {
  unsigned long long tk[SUPER_SLOTS];  // slot keys (kHashEmpty when free)
  uint32_t tc[SUPER_SLOTS];            // slot counts
  uint32_t n_used;                     // slots claimed in this pass
  uint32_t sb;                         // super bucket being counted
};

struct SuperArgs {
  const uint64_t *keys;                   // the upper sweep's output
  const unsigned long long *super_base;   // first key of each super bucket [n_super + 1]
  const uint32_t *list;                   // the super buckets to count
  uint32_t n_list;
  uint32_t *work;                         // claim counter (zero at launch)
};

// Pass of a key when a bucket is counted in 2^lg passes: the top lg bits of
// a multiplicative hash.  Doubling the passes splits pass q into 2q and
// 2q + 1, so the passes already counted stay a prefix [0, 2p).
__device__ __forceinline__ uint32_t super_pass_of(uint64_t key, int lg) {
  return lg ? (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> (64 - lg)) : 0u;
}

template <int THREADS>
__global__ void __launch_bounds__(THREADS, KMC_SUPER_MINB)
super_hash_kernel(SuperArgs a, CountOut<uint64_t> out, uint32_t *err) {
  constexpr int SPT = SUPER_SLOTS / THREADS;
  static_assert(THREADS == SUPER_THREADS && SUPER_SLOTS % THREADS == 0 && SPT <= 32, "layout");
  static_assert(SUPER_LIMIT > 0 && SUPER_LIMIT + SUPER_BATCH < SUPER_SLOTS, "probes must end");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SuperHashSmem &s = *reinterpret_cast<SuperHashSmem *>(smem_raw);
  const int tid = threadIdx.x;
  const unsigned lane = lane_id();
#pragma unroll
  for (int q = 0; q < SPT; ++q) {
    s.tk[q * THREADS + tid] = kHashEmpty;
    s.tc[q * THREADS + tid] = 0;
  }
  unsigned long long n_distinct = 0;
  for (;;) {
    if (tid == 0) {
      const uint32_t i = atomicAdd(a.work, 1u);
      s.sb = i < a.n_list ? a.list[i] : 0xFFFFFFFFu;
      s.n_used = 0;
    }
    __syncthreads();
    const uint32_t sb = s.sb;
    if (sb == 0xFFFFFFFFu) break;
    const uint64_t st = a.super_base[sb], n = a.super_base[sb + 1] - st;
    const uint64_t *src = a.keys + st;
    int lg = 0;  // the bucket is counted in P = 2^lg passes
    uint32_t P = 1;
    for (uint32_t p = 0; p < P;) {
      bool over = false;
      uint64_t nxt[SUPER_UNROLL];
#pragma unroll
      for (int u = 0; u < SUPER_UNROLL; ++u) {
        const uint64_t e = (uint64_t)u * THREADS + tid;
        nxt[u] = e < n ? src[e] : kHashEmpty;
      }
      for (uint64_t e0 = 0; e0 < n; e0 += SUPER_BATCH) {
        uint64_t key[SUPER_UNROLL];
#pragma unroll
        for (int u = 0; u < SUPER_UNROLL; ++u) {
          key[u] = nxt[u];
          const uint64_t e = e0 + SUPER_BATCH + (uint64_t)u * THREADS + tid;  // next batch, in flight
          nxt[u] = e < n ? src[e] : kHashEmpty;
        }
        uint32_t fresh = 0;   // slots this thread claimed
        bool lost = false;    // a probe gave up (cannot happen: SUPER_LIMIT + SUPER_BATCH < SUPER_SLOTS)
#pragma unroll
        for (int u = 0; u < SUPER_UNROLL; ++u) {
          if (key[u] == kHashEmpty || (lg && super_pass_of(key[u], lg) != p)) continue;
          uint32_t h = (uint32_t)(((uint64_t)(uint32_t)key[u] * SUPER_SLOTS) >> 32);
          bool placed = false;
          for (int probe = 0; probe < SUPER_SLOTS; ++probe) {
            const unsigned long long old = atomicCAS(&s.tk[h], kHashEmpty, key[u]);
            if (old == kHashEmpty || old == key[u]) {
              fresh += old == kHashEmpty;
              placed = true;
              break;
            }
            h = h + 1 == (uint32_t)SUPER_SLOTS ? 0u : h + 1;
          }
          if (placed) atomicAdd(&s.tc[h], 1u);
          else lost = true;
        }
        // slots taken after this batch: the warp that adds last sees the total
        const uint32_t wf = __reduce_add_sync(FULL, fresh);
        bool full = false;
        if (lane == 0 && wf) full = atomicAdd(&s.n_used, wf) + wf > (uint32_t)SUPER_LIMIT;
        over = __syncthreads_or(full || lost);
        if (over) break;
      }
      if (over) {
        // too many distinct keys for this pass: clear it and split it (and
        // every later pass) in two; passes 0..p-1, already emitted, become
        // passes 0..2p-1
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
          s.tk[q * THREADS + tid] = kHashEmpty;
          s.tc[q * THREADS + tid] = 0;
        }
        if (tid == 0) s.n_used = 0;
        ++lg;
        P *= 2;
        p *= 2;
        __syncthreads();
        if (P > SUPER_MAX_PASSES) {  // cannot happen for a bucket below 2^32 keys
          if (tid == 0) atomicOr(err, ERR_CAPACITY);
          break;
        }
        continue;
      }
      // occupied slots are the distinct keys of pass p: emit and clear them
      uint32_t keep = 0;
      uint32_t cc[SPT];
#pragma unroll
      for (int q = 0; q < SPT; ++q) {
        cc[q] = s.tc[q * THREADS + tid];
        n_distinct += cc[q] != 0;
        if (cc[q] >= out.ci && cc[q] <= out.cx) keep |= 1u << q;  // ci >= 1
      }
      const uint32_t nk = (uint32_t)__popc(keep);
      const uint32_t incl = warp_incl_scan(nk);
      const uint32_t wtot = __shfl_sync(FULL, incl, 31);
      unsigned long long wbase = 0;
      if (lane == 31 && wtot) wbase = atomicAdd(out.n, (unsigned long long)wtot);
      wbase = __shfl_sync(FULL, wbase, 31);
      const bool fits = wbase + wtot <= out.cap;
      if (!fits && lane == 0) atomicOr(err, ERR_CAPACITY);
      uint64_t q0 = wbase + incl - nk;
#pragma unroll
      for (int q = 0; q < SPT; ++q) {
        if (cc[q]) {
          const int e = q * THREADS + tid;
          if (fits && ((keep >> q) & 1u)) {
            out.keys[q0] = out.mixer.unmix(s.tk[e]);
            out.counts[q0] = cc[q];
            ++q0;
          }
          s.tk[e] = kHashEmpty;
          s.tc[e] = 0;
        }
      }
      if (tid == 0) s.n_used = 0;
      ++p;
      __syncthreads();  // the table is clear for the next pass or bucket
    }
  }
  const unsigned long long nd = __reduce_add_sync(FULL, (unsigned)n_distinct);
  if (lane == 0 && nd) atomicAdd(out.n_distinct, nd);
}

// Pairs mode: sort every tile of (key, value) pairs in place (keys/vals are
// read and written at the same positions).  Used to put the survivors in
// global order and to order signatures by weight.
template <typename K, typename V, int THREADS, int IPT>
struct TilePairsSmem {
  typename BlockSort<K, V, THREADS, IPT>::Smem bs;
  uint32_t tile;
};

template <typename K, typename V, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS, 3)
tile_pairs_kernel(K *keys, V *vals, TilePlan plan, uint32_t *work, uint32_t *big_list,
                  uint32_t *n_big, unsigned long long *big_keys, uint32_t big_cap,
                  uint32_t *err) {
  using BS = BlockSort<K, V, THREADS, IPT>;
  using SM = TilePairsSmem<K, V, THREADS, IPT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &sm = *reinterpret_cast<SM *>(smem_raw);
  const uint32_t nt = *plan.n_tiles;
  const unsigned lane = lane_id();
  for (;;) {
    const uint32_t t = next_tile(work, &sm.tile);
    if (t >= nt) break;
    uint64_t st, en;
    int nbits;
    tile_range(plan, t, nt, &st, &en, &nbits);
    const uint64_t n64 = en - st;
    if (n64 <= 1) continue;
    if (n64 > (uint64_t)BS::TILE) {
      if (threadIdx.x == 0) push_big(t, n64, big_list, n_big, big_keys, big_cap, err);
      continue;
    }
    const int n = (int)n64;
    K k[IPT];
    V v[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      if (BS::valid(n, i)) {
        k[i] = keys[st + BS::elem(n, i)];
        v[i] = vals[st + BS::elem(n, i)];
      }
    }
    BS::sort(k, v, nbits, n, sm.bs);
    for (int e = threadIdx.x; e < n; e += THREADS) {
      keys[st + e] = sm.bs.keys[e];
      vals[st + e] = sm.bs.vals[e];
    }
    __syncthreads();
  }
}

// Weighted count mode: tiles of (key, weight) pairs; equal keys are
// grouped as in count mode and a key's count is the sum of its weights.
// Used after expanding distinct (k,x)-mers into their k-mers, each weighted
// by the (k,x)-mer's multiplicity.
template <typename K, int THREADS, int IPT>
struct TileWCountSmem {
  typename BlockSort<K, uint32_t, THREADS, IPT>::Smem bs;
  uint16_t heads[THREADS * IPT + 1];
  unsigned long long wsum[THREADS * IPT + 1];  // wsum[e+1] = weights of elements 0..e
  unsigned long long ws64[THREADS / 32 + 1];
  uint32_t tile;
  unsigned long long base;
};

template <typename K, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS)
tile_wcount_kernel(const K *__restrict__ keys, const uint32_t *__restrict__ wts, TilePlan plan,
                   uint32_t *work, CountOut<K> out, uint32_t *big_list, uint32_t *n_big,
                   unsigned long long *big_keys, uint32_t big_cap, uint32_t *err) {
  using BS = BlockSort<K, uint32_t, THREADS, IPT>;
  using SM = TileWCountSmem<K, THREADS, IPT>;
  static_assert(BS::TILE < 65536, "heads are 16-bit");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &sm = *reinterpret_cast<SM *>(smem_raw);
  const uint32_t nt = *plan.n_tiles;
  for (;;) {
    const uint32_t t = next_tile(work, &sm.tile);
    if (t >= nt) break;
    uint64_t st, en;
    int nbits;
    tile_range(plan, t, nt, &st, &en, &nbits);
    const uint64_t n64 = en - st;
    if (n64 == 0) continue;
    if (n64 > (uint64_t)BS::TILE) {
      if (threadIdx.x == 0) push_big(t, n64, big_list, n_big, big_keys, big_cap, err);
      continue;
    }
    const int n = (int)n64;
    K k[IPT];
    uint32_t v[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
      if (BS::valid(n, i)) {
        k[i] = keys[st + BS::elem(n, i)];
        v[i] = wts[st + BS::elem(n, i)];
      }
    }
    BS::sort(k, v, nbits < out.sort_bits ? nbits : out.sort_bits, n, sm.bs);
    if (nbits > out.sort_bits) group_equal_runs_kv<K, uint32_t, THREADS>(sm.bs.keys, sm.bs.vals, n, out.sort_bits);
    // inclusive prefix sums of the weights (thread-contiguous chunks)
    const int e0 = threadIdx.x * IPT;
    unsigned long long loc = 0;
    for (int j = 0; j < IPT; ++j)
      if (e0 + j < n) loc += sm.bs.vals[e0 + j];
    unsigned long long tot64;
    unsigned long long pre = block_excl_scan<unsigned long long, THREADS>(loc, sm.ws64, &tot64);
    for (int j = 0; j < IPT; ++j)
      if (e0 + j < n) { pre += sm.bs.vals[e0 + j]; sm.wsum[e0 + j + 1] = pre; }
    if (threadIdx.x == 0) sm.wsum[0] = 0;
    __syncthreads();
    // heads of runs of equal keys
    uint32_t nh = 0;
    for (int j = 0; j < IPT; ++j) {
      const int e = e0 + j;
      if (e < n && (e == 0 || sm.bs.keys[e] != sm.bs.keys[e - 1])) ++nh;
    }
    uint32_t U;
    uint32_t hb = block_excl_scan<uint32_t, THREADS>(nh, sm.bs.ws, &U);
    for (int j = 0; j < IPT; ++j) {
      const int e = e0 + j;
      if (e < n && (e == 0 || sm.bs.keys[e] != sm.bs.keys[e - 1])) sm.heads[hb++] = (uint16_t)e;
    }
    if (threadIdx.x == 0) sm.heads[U] = (uint16_t)n;
    __syncthreads();
    const uint32_t Q = (U + THREADS - 1) / THREADS;
    const uint32_t u0 = threadIdx.x * Q;
    uint32_t keep = 0;
    for (uint32_t j = 0; j < Q; ++j) {
      const uint32_t u = u0 + j;
      if (u < U) {
        const unsigned long long c = sm.wsum[sm.heads[u + 1]] - sm.wsum[sm.heads[u]];
        const bool kp = c >= out.ci && c <= out.cx;
        if (kp && c > 0xFFFFFFFFull) atomicOr(err, ERR_OVERFLOW);
        keep += kp && c <= 0xFFFFFFFFull;
      }
    }
    uint32_t ktot;
    uint32_t kb = block_excl_scan<uint32_t, THREADS>(keep, sm.bs.ws, &ktot);
    if (threadIdx.x == 0) {
      sm.base = ktot ? atomicAdd(out.n, (unsigned long long)ktot) : 0ull;
      atomicAdd(out.n_distinct, (unsigned long long)U);
    }
    __syncthreads();
    const uint64_t base = sm.base;
    if (base + ktot > out.cap) {
      if (threadIdx.x == 0) atomicOr(err, ERR_CAPACITY);
    } else {
      for (uint32_t j = 0; j < Q; ++j) {
        const uint32_t u = u0 + j;
        if (u < U) {
          const uint32_t h = sm.heads[u];
          const unsigned long long c = sm.wsum[sm.heads[u + 1]] - sm.wsum[h];
          if (c >= out.ci && c <= out.cx && c <= 0xFFFFFFFFull) {
            out.keys[base + kb] = out.mixer.unmix(sm.bs.keys[h]);
            out.counts[base + kb] = (uint32_t)c;
            ++kb;
          }
        }
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- big tiles
// One CTA per bucket larger than a tile: LSD passes (8-bit digits) through
// global memory with a scratch buffer; each pass is a digit histogram, a
// scan, and a stable chunked scatter.  A pass whose digit is the same for
// every key is skipped (all-identical buckets cost one histogram per pass).

template <typename K, typename V, int THREADS, int IPT>
struct BigSmem {
  static constexpr int NW = THREADS / 32;
  static constexpr int CH = THREADS * IPT;
  uint32_t cnt[NW][257];
  unsigned long long offs[257];
  uint32_t ws[NW + 1];
  uint32_t pos[CH];
  uint32_t flag;
  unsigned long long base;
};

// Sorts src[0..n) (+ payload) on bits [0, nbits); returns the buffer that
// holds the result (src or dst).
template <typename K, typename V, int THREADS, int IPT>
__device__ bool big_sort(K *src_k, V *src_v, K *dst_k, V *dst_v, uint64_t n, int nbits,
                         BigSmem<K, V, THREADS, IPT> &sm) {
  constexpr bool HAS_V = !std::is_same<V, NoVal>::value;
  constexpr int NW = THREADS / 32, CH = THREADS * IPT;
  const unsigned lane = lane_id(), w = threadIdx.x >> 5;
  bool in_dst = false;
  for (int bit = 0; bit < nbits; bit += 8) {
    const int nb = nbits - bit < 8 ? nbits - bit : 8;
    K *sk = in_dst ? dst_k : src_k;
    V *sv = in_dst ? dst_v : src_v;
    K *dk = in_dst ? src_k : dst_k;
    V *dv = in_dst ? src_v : dst_v;
    // histogram (warp-aggregated)
    for (int i = threadIdx.x; i < 257; i += THREADS) sm.offs[i] = 0;
    __syncthreads();
    for (uint64_t e = threadIdx.x; e < n + (THREADS - 1) - ((n + THREADS - 1) % THREADS) ; e += THREADS) {
      unsigned d = e < n ? KeyTraits<K>::digit(sk[e], bit, nb) : 256u;
      unsigned peers = __match_any_sync(FULL, d);
      if (d < 256u && (int)lane == __ffs(peers) - 1) atomicAdd(&sm.offs[d], (unsigned long long)__popc(peers));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long acc = 0;
      uint32_t single = 0;
      for (int d = 0; d < 256; ++d) {
        unsigned long long c = sm.offs[d];
        if (c == n) single = 1;
        sm.offs[d] = acc;
        acc += c;
      }
      sm.flag = single;
    }
    __syncthreads();
    if (sm.flag) continue;  // every key has this digit: the pass is the identity
    for (uint64_t c0 = 0; c0 < n; c0 += CH) {
      for (int i = lane; i < 257; i += 32) sm.cnt[w][i] = 0;
      __syncwarp();
      K k[IPT];
      V v[IPT];
      unsigned dg[IPT];
      uint32_t rank[IPT];
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        uint64_t e = c0 + w * 32 * IPT + i * 32 + lane;
        bool ok = e < n;
        k[i] = ok ? sk[e] : KeyTraits<K>::max_key();
        if constexpr (HAS_V) v[i] = ok ? sv[e] : V();
        dg[i] = ok ? KeyTraits<K>::digit(k[i], bit, nb) : 256u;
        unsigned peers = __match_any_sync(FULL, dg[i]);
        int leader = __ffs(peers) - 1;
        uint32_t b = 0;
        if ((int)lane == leader) {
          b = sm.cnt[w][dg[i]];
          sm.cnt[w][dg[i]] = b + __popc(peers);
        }
        b = __shfl_sync(FULL, b, leader);
        rank[i] = b + __popc(peers & lanemask_lt());
        __syncwarp();
      }
      __syncthreads();
      // per digit: exclusive prefix over warps, then add the running offset
      for (int d = threadIdx.x; d < 256; d += THREADS) {
        uint32_t acc = 0;
        for (int ww = 0; ww < NW; ++ww) {
          uint32_t c = sm.cnt[ww][d];
          sm.cnt[ww][d] = acc;
          acc += c;
        }
        sm.pos[d] = acc;  // chunk total of digit d (pos[] reused as scratch)
      }
      __syncthreads();
#pragma unroll
      for (int i = 0; i < IPT; ++i) {
        if (dg[i] < 256u) {
          unsigned long long p = sm.offs[dg[i]] + sm.cnt[w][dg[i]] + rank[i];
          dk[p] = k[i];
          if constexpr (HAS_V) dv[p] = v[i];
        }
      }
      __syncthreads();
      for (int d = threadIdx.x; d < 256; d += THREADS) sm.offs[d] += sm.pos[d];
      __syncthreads();
    }
    in_dst = !in_dst;
  }
  return in_dst;
}

template <typename K, int THREADS, int IPT>
__device__ void big_count_range(K *src, K *dst, uint64_t n, int nbits, uint32_t group, const CountOut<K> &out,
                                uint32_t *err, K *sorted_out, BigSmem<K, NoVal, THREADS, IPT> &sm) {
  constexpr int CH = THREADS * IPT;
  const bool in_dst = big_sort<K, NoVal, THREADS, IPT>(src, (NoVal *)nullptr, dst, (NoVal *)nullptr, n, nbits, sm);
  const K *a = in_dst ? dst : src;
  if (sorted_out)
    for (uint64_t e = threadIdx.x; e < n; e += THREADS) sorted_out[e] = a[e];
  // heads: run starts; the run open at the end of a chunk continues in the next
  uint64_t open = 0;  // start of the open run (element 0 always starts one)
  uint32_t *ws = sm.ws;
  unsigned long long n_runs = 0;
  for (uint64_t c0 = 0; c0 < n; c0 += CH) {
    // compact head positions of this chunk (excluding element 0, the first open run)
    uint32_t nh = 0;
    const uint64_t e0 = c0 + (uint64_t)threadIdx.x * IPT;
    for (int j = 0; j < IPT; ++j) {
      uint64_t e = e0 + j;
      if (e < n && e > 0 && a[e] != a[e - 1]) ++nh;
    }
    uint32_t tot;
    uint32_t hb = block_excl_scan<uint32_t, THREADS>(nh, ws, &tot);
    for (int j = 0; j < IPT; ++j) {
      uint64_t e = e0 + j;
      if (e < n && e > 0 && a[e] != a[e - 1]) sm.pos[hb++] = (uint32_t)(e - c0);
    }
    __syncthreads();
    // runs closed in this chunk: [prev, pos[0]), [pos[0], pos[1]), ...; plus the
    // final run when this is the last chunk.
    const bool last = c0 + CH >= n;
    const uint32_t nclosed = tot + (last ? 1u : 0u);
    uint32_t keep = 0;
    const uint32_t Q = (nclosed + THREADS - 1) / THREADS;
    const uint32_t r0 = threadIdx.x * Q;
    for (uint32_t j = 0; j < Q; ++j) {
      uint32_t r = r0 + j;
      if (r < nclosed) {
        uint64_t rs = r == 0 ? open : c0 + sm.pos[r - 1];
        uint64_t re = r < tot ? c0 + sm.pos[r] : n;
        uint64_t c = re - rs;
        if (c > 0xFFFFFFFFull && c >= out.ci && c <= out.cx) atomicOr(err, ERR_OVERFLOW);
        keep += (c >= out.ci && c <= out.cx && c <= 0xFFFFFFFFull);
      }
    }
    uint32_t ktot;
    uint32_t kb = block_excl_scan<uint32_t, THREADS>(keep, ws, &ktot);
    if (threadIdx.x == 0) sm.base = ktot ? atomicAdd(out.n, (unsigned long long)ktot) : 0ull;
    __syncthreads();
    const uint64_t base = sm.base;
    if (base + ktot > out.cap) {
      if (threadIdx.x == 0) atomicOr(err, ERR_CAPACITY);
    } else {
      for (uint32_t j = 0; j < Q; ++j) {
        uint32_t r = r0 + j;
        if (r < nclosed) {
          uint64_t rs = r == 0 ? open : c0 + sm.pos[r - 1];
          uint64_t re = r < tot ? c0 + sm.pos[r] : n;
          uint64_t c = re - rs;
          if (c >= out.ci && c <= out.cx && c <= 0xFFFFFFFFull) {
            out.keys[base + kb] = out.mixer.unmix(a[rs]);
            out.counts[base + kb] = (uint32_t)c;
            if (out.slots) out.slots[base + kb] = group / out.bins_per_slot;
            ++kb;
          }
        }
      }
    }
    n_runs += nclosed;
    if (tot) open = c0 + sm.pos[tot - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out.n_distinct, n_runs);
  __syncthreads();
}

// Count mode big tiles: sort (in place + scratch), then run-length count
// chunk by chunk, carrying the open run across chunks.
template <typename K, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS)
big_count_kernel(K *keys, TilePlan plan, const uint32_t *big_list, const uint32_t *n_big,
                 K *scratch, unsigned long long *scratch_cursor, CountOut<K> out, uint32_t *err,
                 K *sorted_out) {
  using SM = BigSmem<K, NoVal, THREADS, IPT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &sm = *reinterpret_cast<SM *>(smem_raw);
  const uint32_t nt = *plan.n_tiles;
  const uint32_t nbig = *n_big;
  for (uint32_t bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
    const uint32_t t = big_list[bi];
    uint64_t st, en;
    int nbits;
    uint32_t group;
    tile_range(plan, t, nt, &st, &en, &nbits, &group);
    const uint64_t n = en - st;
    if (threadIdx.x == 0) sm.base = atomicAdd(scratch_cursor, (unsigned long long)n);
    __syncthreads();
    big_count_range<K, THREADS, IPT>(keys + st, scratch + sm.base, n, nbits, group, out, err,
                                     sorted_out ? sorted_out + st : nullptr, sm);
  }
}

// Count mode big tiles without a full sort: a big tile's keys are split by
// bits kGroupBits .. kGroupBits+S (one more radix partition step, into global
// scratch at the tile's own positions) into sub-buckets of about half a
// tile, and each sub-bucket is counted like a tile.  A sub-bucket still
// above a tile (copies of a few keys) is sorted through global memory.
template <typename K, int THREADS, int IPT, int BIPT>
struct BigGroupSmem {
  union U {
    TileGroupSmem<K, THREADS, IPT> g;
    BigSmem<K, NoVal, THREADS, BIPT> b;
  } u;
  uint64_t lo[kGroupDigits + 1];  // sub-bucket starts (tile-relative)
};

template <typename K, int THREADS, int IPT, int BIPT>
__global__ void __launch_bounds__(THREADS, 1)
big_group_kernel(K *keys, TilePlan plan, const uint32_t *big_list, const uint32_t *n_big, K *scratch,
                 CountOut<K> out, int key_bits, uint32_t *err) {
  using SM = BigGroupSmem<K, THREADS, IPT, BIPT>;
  constexpr int TILE = THREADS * IPT;
  constexpr int DPT = kGroupDigits / THREADS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &s = *reinterpret_cast<SM *>(smem_raw);
  auto &g = s.u.g;
  const uint32_t nt = *plan.n_tiles;
  const uint32_t nbig = *n_big;
  const int tid = threadIdx.x;
  for (uint32_t bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
    const uint32_t t = big_list[bi];
    uint64_t st, en;
    int nbits;
    uint32_t group;
    tile_range(plan, t, nt, &st, &en, &nbits, &group);
    const uint64_t n = en - st;
    if (n >= (1ull << 32)) {  // positions below are 32-bit
      if (tid == 0) atomicOr(err, ERR_CAPACITY);
      continue;
    }
    int S = 0;
    while (S < kGroupBits && (n >> S) > (uint64_t)TILE / 2) ++S;
    const uint32_t smask = (1u << S) - 1u;
    __syncthreads();  // the previous big tile is done with shared memory
    for (int i = tid; i < kGroupDigits + 4; i += THREADS) g.off[i] = 0;
    __syncthreads();
    for (uint64_t e = tid; e < n; e += THREADS)
      atomicAdd(&g.off[(uint32_t)((uint64_t)keys[st + e] >> kGroupBits) & smask], 1u);
    __syncthreads();
    {  // exclusive scan of the sub-digit counts
      uint32_t c[DPT];
#pragma unroll
      for (int q = 0; q < DPT; q += 4) {
        const uint4 v = *reinterpret_cast<const uint4 *>(&g.off[DPT * tid + q]);
        c[q] = v.x; c[q + 1] = v.y; c[q + 2] = v.z; c[q + 3] = v.w;
      }
      uint32_t sum = 0;
#pragma unroll
      for (int q = 0; q < DPT; ++q) sum += c[q];
      uint32_t tot;
      uint32_t run = block_excl_scan<uint32_t, THREADS>(sum, g.ws, &tot);
#pragma unroll
      for (int q = 0; q < DPT; ++q) {
        const uint32_t x = c[q];
        g.off[DPT * tid + q] = run;
        s.lo[DPT * tid + q] = run;
        run += x;
      }
      if (tid == 0) s.lo[kGroupDigits] = n;
    }
    __syncthreads();
    for (uint64_t e = tid; e < n; e += THREADS) {
      const K key = keys[st + e];
      const uint32_t p = atomicAdd(&g.off[(uint32_t)((uint64_t)key >> kGroupBits) & smask], 1u);
      scratch[st + p] = key;
    }
    __syncthreads();
    for (uint32_t sb = 0; sb <= smask; ++sb) {
      const uint64_t lo = s.lo[sb], hi = s.lo[sb + 1];
      const uint64_t m = hi - lo;
      if (m == 0) continue;
      if (m <= (uint64_t)TILE) {
        for (int e = tid; e < (int)m; e += THREADS) g.a[e] = scratch[st + lo + e];
        __syncthreads();
        group_core<K, THREADS, IPT>(g, (int)m, 0, group, out, err, []() {});
      } else {
        // the tile's own range in keys is free now: the sort's second buffer
        big_count_range<K, THREADS, BIPT>(scratch + st + lo, keys + st + lo, m, key_bits, group, out, err,
                                          nullptr, s.u.b);
      }
      __syncthreads();
    }
  }
}

// Pairs mode big tiles: sort; copy back if the result ended in scratch.
template <typename K, typename V, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS)
big_pairs_kernel(K *keys, V *vals, TilePlan plan, const uint32_t *big_list, const uint32_t *n_big,
                 K *scratch_k, V *scratch_v, unsigned long long *scratch_cursor) {
  using SM = BigSmem<K, V, THREADS, IPT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &sm = *reinterpret_cast<SM *>(smem_raw);
  const uint32_t nt = *plan.n_tiles;
  const uint32_t nbig = *n_big;
  for (uint32_t bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
  const uint32_t t = big_list[bi];
  uint64_t st, en;
  int nbits;
  tile_range(plan, t, nt, &st, &en, &nbits);
  const uint64_t n = en - st;
  if (threadIdx.x == 0) sm.base = atomicAdd(scratch_cursor, (unsigned long long)n);
  __syncthreads();
  K *sk = scratch_k + sm.base;
  V *sv = scratch_v + sm.base;
  if (big_sort<K, V, THREADS, IPT>(keys + st, vals + st, sk, sv, n, nbits, sm)) {
    for (uint64_t e = threadIdx.x; e < n; e += THREADS) {
      keys[st + e] = sk[e];
      vals[st + e] = sv[e];
    }
  }
  __syncthreads();
  }
}

// Weighted count of big tiles: sorted through global scratch, then one
// thread walks the runs (big tiles of weighted keys are rare).
template <typename K, int THREADS, int IPT>
__global__ void __launch_bounds__(THREADS)
big_wcount_kernel(K *keys, uint32_t *wts, TilePlan plan, const uint32_t *big_list, K *scratch_k,
                  uint32_t *scratch_v, unsigned long long *scratch_cursor, CountOut<K> out,
                  uint32_t *err) {
  using SM = BigSmem<K, uint32_t, THREADS, IPT>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SM &sm = *reinterpret_cast<SM *>(smem_raw);
  const uint32_t t = big_list[blockIdx.x];
  const uint32_t nt = *plan.n_tiles;
  uint64_t st, en;
  int nbits;
  tile_range(plan, t, nt, &st, &en, &nbits);
  const uint64_t n = en - st;
  if (threadIdx.x == 0) sm.base = atomicAdd(scratch_cursor, (unsigned long long)n);
  __syncthreads();
  K *sk = scratch_k + sm.base;
  uint32_t *sv = scratch_v + sm.base;
  const bool in_scratch = big_sort<K, uint32_t, THREADS, IPT>(keys + st, wts + st, sk, sv, n, nbits, sm);
  __syncthreads();
  if (threadIdx.x != 0) return;
  const K *a = in_scratch ? sk : keys + st;
  const uint32_t *w = in_scratch ? sv : wts + st;
  unsigned long long runs = 0;
  uint64_t i = 0;
  while (i < n) {
    uint64_t j = i;
    unsigned long long c = 0;
    while (j < n && a[j] == a[i]) c += w[j++];
    ++runs;
    if (c >= out.ci && c <= out.cx) {
      if (c > 0xFFFFFFFFull) {
        atomicOr(err, ERR_OVERFLOW);
      } else {
        const unsigned long long p = atomicAdd(out.n, 1ull);
        if (p < out.cap) {
          out.keys[p] = out.mixer.unmix(a[i]);
          out.counts[p] = (uint32_t)c;
        } else {
          atomicOr(err, ERR_CAPACITY);
        }
      }
    }
    i = j;
  }
  atomicAdd(out.n_distinct, runs);
}

// ---------------------------------------------------------------- plan kernels

// flag[i] = 1 where a tile starts (see plan_tiles in sortlib.cu for the rule).
__global__ void plan_flags_kernel(const uint32_t *cnt, const uint64_t *base, uint64_t nbk,
                                  const uint32_t *group_base, uint32_t n_groups,
                                  uint32_t tile_cap, uint32_t *flag);
constexpr uint32_t kGreedySegment = 1024;
__global__ void plan_greedy_flags_kernel(const uint32_t *cnt, const uint32_t *group_base,
                                         uint32_t n_groups, uint64_t nbk, uint32_t tile_cap,
                                         uint32_t *flag);
__global__ void plan_emit_kernel(const uint32_t *flag, const uint64_t *flag_scan, uint64_t nbk,
                                 uint32_t *tile_first, uint32_t *n_tiles);

// ---------------------------------------------------------------- host API
struct DeviceArena;  // defined in api

// Exclusive scan of n values (uint32 or uint64 input) into uint64 out[n+1]
// (out[n] = total).  `tmp` must hold scan_tmp_words(n) uint64 words.
size_t scan_tmp_words(uint64_t n);
cudaError_t device_excl_scan_u32(const uint32_t *in, uint64_t *out, uint64_t n, uint64_t *tmp,
                                 cudaStream_t st);
cudaError_t device_excl_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, uint64_t *tmp,
                                 cudaStream_t st);

}  // namespace kmc
