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

// ------------------------------------------------------------ (k,x)-mers
// Sect. 2.3: a super k-mer is split into as few (k,x)-mers as possible:
// runs of k-mers of one orientation (direct when the k-mer is not larger
// than its reverse complement), cut greedily into groups of at most x+1
// k-mers; a group of x'+1 k-mers is stored as the (k+x')-mer in the
// orientation in which its k-mers are canonical.  Key layout (key_bits =
// 2 + 2(k+x)): [x' : 2 bits][k+x' symbols, first symbol most significant]
// [zeros : 2(x-x') bits].

__device__ __forceinline__ uint64_t rc_any(uint64_t v, int len) { return revcomp64(v, len); }
__device__ __forceinline__ u128 rc_any(u128 v, int len) { return revcomp128(v, len); }

template <typename K1>
__device__ __forceinline__ K1 kx_key(const uint64_t *wds, uint32_t g0, uint32_t gl, bool rev,
                                     int k, int x) {
  const int xp = (int)gl - 1;
  const int len = k + xp;
  K1 v = get_kmer<K1>(wds, g0, len);
  if (rev) v = rc_any(v, len);
  return ((K1)(uint32_t)xp << (2 * (k + x))) | (v << (2 * (x - xp)));
}

// Calls f(key) for every (k,x)-mer of one super k-mer record (n k-mers).
template <typename K1, typename K0, typename F>
__device__ __forceinline__ void for_record_kxmers(const uint64_t *wds, uint32_t n, int k, int x,
                                                  F f) {
  const K0 kmask = (2 * k >= (int)(8 * sizeof(K0))) ? ~K0(0) : ((K0(1) << (2 * k)) - 1);
  K0 fw = get_kmer<K0>(wds, 0, k);
  K0 rc = rc_any(fw, k);
  uint32_t g0 = 0, gl = 0;
  bool go = false;
  for (uint32_t j = 0; j < n; ++j) {
    if (j > 0) {
      const uint32_t c = (uint32_t)get_bits(wds, 2ull * (j + k - 1), 2);
      fw = ((fw << 2) | (K0)c) & kmask;
      rc = (rc >> 2) | ((K0)(3u - c) << (2 * k - 2));
    }
    const bool o = rc < fw;  // reverse orientation; a palindrome counts as direct
    if (gl > 0 && o == go && gl < (uint32_t)x + 1) {
      ++gl;
    } else {
      if (gl > 0) f(kx_key<K1>(wds, g0, gl, go, k, x));
      g0 = j;
      gl = 1;
      go = o;
    }
  }
  if (gl > 0) f(kx_key<K1>(wds, g0, gl, go, k, x));
}

template <typename K1>
struct KxxArgs {
  const Chunk *chunks;
  const PieceDesc *pieces;
  int k, x, key_bits;
  const uint32_t *group_base;
  const uint8_t *group_D;
  Mixer<K1> mixer;
};

// a4 for x > 0, count pass: one thread per super k-mer record; per-bin
// histogram of the top D bits of the mixed (k,x)-mer keys.
template <typename K1, typename K0>
__global__ void __launch_bounds__(KX_THREADS)
kxx_count_kernel(KxxArgs<K1> a, uint32_t *__restrict__ hist) {
  __shared__ uint32_t h[1 << KX_SMEM_D];
  const Chunk c = a.chunks[blockIdx.x];
  const PieceDesc pd = a.pieces[c.piece];
  const int D = a.group_D[c.bin];
  const uint32_t ND = 1u << D;
  uint32_t *hb = hist + a.group_base[c.bin];
  const bool in_smem = D <= KX_SMEM_D;
  if (in_smem) {
    for (uint32_t i = threadIdx.x; i < ND; i += KX_THREADS) h[i] = 0;
    __syncthreads();
  }
  for (uint32_t r = threadIdx.x; r < c.n_rec; r += KX_THREADS) {
    const uint64_t e = pd.index[c.r0 + r];
    const uint32_t n = (uint32_t)((e >> 25) & 127u) + 1u;
    for_record_kxmers<K1, K0>(pd.words + (e >> 32), n, a.k, a.x, [&](K1 key) {
      const uint32_t d = top_digit<K1>(a.mixer.mix(key), a.key_bits, D);
      atomicAdd(in_smem ? &h[d] : &hb[d], 1u);
    });
  }
  if (in_smem) {
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < ND; i += KX_THREADS)
      if (h[i]) atomicAdd(&hb[i], h[i]);
  }
}

// a4 for x > 0, scatter pass: the same keys written into their buckets
// (count the chunk, reserve per digit, write).
template <typename K1, typename K0>
__global__ void __launch_bounds__(KX_THREADS)
kxx_scatter_kernel(KxxArgs<K1> a, const uint64_t *__restrict__ bucket_base,
                   uint32_t *__restrict__ cursor, K1 *__restrict__ keys, uint64_t n_keys,
                   uint32_t *err) {
  __shared__ uint32_t h[1 << KX_SMEM_D];
  __shared__ unsigned long long gb[1 << KX_SMEM_D];
  const Chunk c = a.chunks[blockIdx.x];
  const PieceDesc pd = a.pieces[c.piece];
  const int D = a.group_D[c.bin];
  const uint32_t ND = 1u << D;
  const uint32_t g0 = a.group_base[c.bin];
  const bool in_smem = D <= KX_SMEM_D;
  if (in_smem) {
    for (uint32_t i = threadIdx.x; i < ND; i += KX_THREADS) h[i] = 0;
    __syncthreads();
    for (uint32_t r = threadIdx.x; r < c.n_rec; r += KX_THREADS) {
      const uint64_t e = pd.index[c.r0 + r];
      const uint32_t n = (uint32_t)((e >> 25) & 127u) + 1u;
      for_record_kxmers<K1, K0>(pd.words + (e >> 32), n, a.k, a.x, [&](K1 key) {
        atomicAdd(&h[top_digit<K1>(a.mixer.mix(key), a.key_bits, D)], 1u);
      });
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < ND; i += KX_THREADS) {
      if (h[i]) gb[i] = bucket_base[g0 + i] + atomicAdd(&cursor[g0 + i], h[i]);
      h[i] = 0;
    }
    __syncthreads();
  }
  for (uint32_t r = threadIdx.x; r < c.n_rec; r += KX_THREADS) {
    const uint64_t e = pd.index[c.r0 + r];
    const uint32_t n = (uint32_t)((e >> 25) & 127u) + 1u;
    for_record_kxmers<K1, K0>(pd.words + (e >> 32), n, a.k, a.x, [&](K1 key) {
      const K1 mk = a.mixer.mix(key);
      const uint32_t d = top_digit<K1>(mk, a.key_bits, D);
      const uint64_t p = in_smem ? gb[d] + atomicAdd(&h[d], 1u)
                                 : bucket_base[g0 + d] + atomicAdd(&cursor[g0 + d], 1u);
      if (p < n_keys) keys[p] = mk; else atomicOr(err, ERR_CAPACITY);
    });
  }
}

// Expansion (Sect. 2.4: the k-mers of the sorted (k,x)-mers are collected):
// every distinct (k,x)-mer, with its multiplicity m, yields its x'+1
// k-mers, each canonical by construction, with weight m.  Pass 0 counts
// the mixed k-mers' top D bits, pass 1 scatters (mixed k-mer, weight).
template <typename K1, typename K0>
__global__ void expand_kernel(const K1 *__restrict__ kx, const uint32_t *__restrict__ mult,
                              uint64_t n1, int k, int x, Mixer<K0> mix0, int D, int pass,
                              uint32_t *__restrict__ hist_or_cursor,
                              const uint64_t *__restrict__ base, K0 *__restrict__ out_k,
                              uint32_t *__restrict__ out_w, uint64_t cap, uint32_t *err) {
  const K0 kmask = (2 * k >= (int)(8 * sizeof(K0))) ? ~K0(0) : ((K0(1) << (2 * k)) - 1);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n1;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const K1 key = kx[i];
    const int xp = (int)(uint32_t)(key >> (2 * (k + x)));
    const K1 v = key >> (2 * (x - xp));  // the k+x' symbols (x' bits shifted out below)
    for (int j = 0; j <= xp; ++j) {
      const K0 kmer = (K0)(v >> (2 * (xp - j))) & kmask;
      const K0 mk = mix0.mix(kmer);
      const uint32_t d = top_digit<K0>(mk, 2 * k, D);
      if (pass == 0) {
        atomicAdd(&hist_or_cursor[d], 1u);
      } else {
        const uint64_t p = base[d] + atomicAdd(&hist_or_cursor[d], 1u);
        if (p < cap) {
          out_k[p] = mk;
          out_w[p] = mult[i];
        } else {
          atomicOr(err, ERR_CAPACITY);
        }
      }
    }
  }
}

// Unmixes keys into most-significant-word-first 64-bit words (inspection).
template <typename K>
__global__ void unmix_words_kernel(const K *in, uint64_t n, Mixer<K> mix, uint64_t *out) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const K v = mix.unmix(in[i]);
    if (sizeof(K) == 8) {
      out[i] = (uint64_t)v;
    } else {
      out[2 * i] = (uint64_t)((u128)v >> 64);
      out[2 * i + 1] = (uint64_t)v;
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
int count_tiles(Handle &h, const TilePlan &plan, uint64_t n_keys, K *keys, const Mixer<K> &mixer,
                uint64_t ci, uint64_t cx, DevBuf &out_k, DevBuf &out_c, uint64_t *n_sv_out,
                K *sorted_out) {
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
        as<uint32_t>(h.err), sorted_out); KMC_COUNT_LAUNCH();
  }
  KMC_CUDA_TRY(cudaGetLastError());
  uint32_t nbig = 0;
  unsigned long long bigk = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&nbig, c32 + 1, 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(&bigk, c64 + 2, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  h.stats.n_big_tiles += nbig;
  if (nbig) {
    if (dev_ensure(ss.big_scratch, (bigk + 1) * sizeof(K), h.st)) return KMC_ENOMEM;
    StageScope sc(h, KMC_STAGE_BIG_SORT);
    big_count_kernel<K, CNT_THREADS, BIG_IPT><<<nbig, CNT_THREADS, sizeof(BSM), h.st>>>(
        keys, plan, as<uint32_t>(ss.big_list), as<K>(ss.big_scratch), c64 + 3, out,
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
};

int build_meta(Handle &h, int key_bits, int tile, double keys_per_kmer, SortMeta *m) {
  SortScratch &ss = h.ss;
  const uint32_t B = h.p.n_bins;
  std::vector<uint32_t> gbase(B + 1);
  std::vector<uint8_t> gD(B);
  uint64_t NB = 0;
  for (uint32_t b = 0; b < B; ++b) {
    gD[b] = (uint8_t)digits_for((uint64_t)(h.bin_kmers[b] * keys_per_kmer), key_bits, tile);
    gbase[b] = (uint32_t)NB;
    NB += 1ull << gD[b];
  }
  gbase[B] = (uint32_t)NB;
  if (NB >= 0xFFFFFFF0ull) return KMC_EINVAL;
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
  const size_t o_pd = (chunks.size() + 1) * sizeof(Chunk);
  const size_t o_gb = o_pd + (pds.size() + 1) * sizeof(PieceDesc);
  const size_t o_gd = o_gb + (B + 1) * 4;
  memcpy(meta.data(), chunks.data(), chunks.size() * sizeof(Chunk));
  memcpy(meta.data() + o_pd, pds.data(), pds.size() * sizeof(PieceDesc));
  memcpy(meta.data() + o_gb, gbase.data(), (B + 1) * 4);
  memcpy(meta.data() + o_gd, gD.data(), B);
  KMC_CUDA_TRY(cudaMemcpyAsync(ss.cursor.p, meta.data(), meta_bytes, cudaMemcpyHostToDevice, h.st));
  char *base = static_cast<char *>(ss.cursor.p);
  m->n_chunks = chunks.size();
  m->NB = NB;
  m->chunks = reinterpret_cast<const Chunk *>(base);
  m->pieces = reinterpret_cast<const PieceDesc *>(base + o_pd);
  m->group_base = reinterpret_cast<const uint32_t *>(base + o_gb);
  m->group_D = reinterpret_cast<const uint8_t *>(base + o_gd);
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
    KMC_CUDA_TRY(cudaMemcpyAsync(h.out_kmers.p, sv_k.p, n_sv * sizeof(K0), cudaMemcpyDeviceToDevice, h.st));
    KMC_CUDA_TRY(cudaMemcpyAsync(h.out_counts.p, sv_c.p, n_sv * 4, cudaMemcpyDeviceToDevice, h.st));
    if constexpr (sizeof(K0) == 8) {
      rc = sort_pairs_u64(h, as<uint64_t>(h.out_kmers), as<uint32_t>(h.out_counts), n_sv, 2 * k);
    } else {
      rc = sort_pairs_u128(h, as<u128>(h.out_kmers), as<uint32_t>(h.out_counts), n_sv, 2 * k);
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

template <typename K, int IPT>
int sort_phase_x0(Handle &h) {
  SortScratch &ss = h.ss;
  constexpr int TILE = CNT_THREADS * IPT;
  const int k = (int)h.p.k;
  const int key_bits = 2 * k;
  const uint64_t n_keys = h.stats.n_kmer_positions;
  h.stats.n_sorted_keys = n_keys;
  SortMeta meta;
  int rc = build_meta(h, key_bits, TILE, 1.0, &meta);
  if (rc) return rc;
  KxArgs<K> a;
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
  KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, NB * 4, h.st));
  if (meta.n_chunks) {
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
  KMC_CUDA_TRY(cudaMemsetAsync(hist, 0, NB * 4, h.st));  // hist becomes the per-bucket cursor
  if (dev_ensure(ss.keys, (n_keys + 1) * sizeof(K), h.st)) return KMC_ENOMEM;
  K *keys = as<K>(ss.keys);
  if (meta.n_chunks) {
    static bool attr = false;
    if (!attr) {
      KMC_CUDA_TRY(cudaFuncSetAttribute(kx0_scatter_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(KxScatterSmem<K>)));
      attr = true;
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
  K *sorted_out = nullptr;
  if (h.p.debug_flags & KMC_DEBUG_KEEP_KEYS) {
    if (dev_ensure(ss.sorted_keys, (n_keys + 1) * sizeof(K), h.st)) return KMC_ENOMEM;
    sorted_out = as<K>(ss.sorted_keys);
  }
  uint64_t n_sv = 0;
  h.stats.n_big_tiles = 0;
  rc = count_tiles<K, IPT>(h, plan, n_keys, keys, a.mixer, h.p.cutoff_min, h.p.cutoff_max,
                           ss.sv_keys, ss.sv_counts, &n_sv, sorted_out);
  if (rc) return rc;
  uint32_t nt = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&nt, n_tiles_dev, 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  h.stats.n_tiles = nt;
  h.stats.x_used = 0;
  return order_result<K>(h, ss.sv_keys, ss.sv_counts, n_sv, k);
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
  if (dev_ensure(ss.keys, (n_keys1 + 1) * sizeof(K1), h.st)) return KMC_ENOMEM;
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
  static bool attr = false;
  if (!attr) {
    KMC_CUDA_TRY(cudaFuncSetAttribute(tile_wcount_kernel<K0, CNT_THREADS, IPT2>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(WSM)));
    KMC_CUDA_TRY(cudaFuncSetAttribute(big_wcount_kernel<K0, CNT_THREADS, BIG_IPT>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BWSM)));
    attr = true;
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

int sort_phase(Handle &h) {
  const uint32_t k = h.p.k;
  const int x = (int)resolve_x(k, h.p.x);
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
