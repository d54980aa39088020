// Kernels of the sorting phase that build keys from the bins' super k-mer
// records (paper Sect. 2.3, 2.4): canonical k-mers (x = 0) or (k,x)-mers
// and their expansion.  Kept in a header so that the single-set path
// (count.cu) and the batched path (batch.cu) compile the same kernels.
#pragma once
#include "common.cuh"
#include "sortlib.cuh"

namespace kmc {
namespace {

constexpr int KX_THREADS = 256;
constexpr int KX_RECORDS_PER_CHUNK = 512;
constexpr int CNT_THREADS = 256;
constexpr int CNT_IPT64 = 16;   // tile = 4096 64-bit keys
constexpr int CNT_IPT128 = 8;   // tile = 2048 128-bit keys
constexpr int BIG_IPT = 16;
constexpr int GRP_THREADS = 512;  // tile_group_kernel (same tile sizes as the sort kernels)

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
  const unsigned long long *n_chunks_dyn;  // batches: chunk count on the device (else NULL)
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
  if (a.n_chunks_dyn && blockIdx.x >= *a.n_chunks_dyn) return;
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
  if (a.n_chunks_dyn && blockIdx.x >= *a.n_chunks_dyn) return;
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

}  // namespace
}  // namespace kmc
