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
constexpr int KX_RECORDS_PER_CHUNK = 2048;
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
  int noncanonical = 0;                    // 1: keys are the k-mers as read (Suppl. S1 -b)
};

// The key of k-mer j of a record: canonical (Sect. 2.1), or as read (-b).
template <typename K>
__device__ __forceinline__ K kmer_key(const KxArgs<K> &a, const uint64_t *wds, uint32_t j) {
  return a.noncanonical ? get_kmer<K>(wds, j, a.k) : canonical_kmer<K>(wds, j, a.k);
}

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
      if (ok) key = a.mixer.mix(kmer_key<K>(a, pd.words + woff, j));
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
        key = ok ? a.mixer.mix(kmer_key<K>(a, pd.words + woff, j)) : K(0);
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

// ------------------------------------------------- x = 0, generate + partition
// The same result as kx0_count + kx0_scatter with each key built once and
// moved by two coalesced radix partition sweeps.  A bin's D digit bits
// (D <= SWEEP_BITS_MAX) split into an upper digit of S = min(D, 8) bits
// ("super buckets") and a lower one of E = D - S bits.
//  * kx0_gen_kernel writes every chunk's mixed canonical k-mers contiguously
//    into its bin's range of an unpartitioned array (one atomic per chunk
//    reserves the range; writes are coalesced) and counts upper digits.
//  * kx0_sweep_kernel<0> moves a bin's keys into its super buckets, in
//    tiles of SWEEP_TILE keys: the tile is sorted by digit in shared memory
//    (one atomic per key gives the rank), one global atomic per digit
//    reserves the tile's share of each super bucket, and the keys go out in
//    digit order, so consecutive threads write consecutive addresses.
//  * kx0_sweep_kernel<1> does the same inside each super bucket (one CTA
//    owns it: a histogram pass, then the sweep with cursors in shared
//    memory) for the lower digit, which puts every key in its final bucket,
//    and stores the final bucket sizes.

constexpr int SWEEP_THREADS = 512;
constexpr int SWEEP_UPPER = 8;                  // bits of the upper digit
constexpr int SWEEP_BITS_MAX = 2 * SWEEP_UPPER; // digit bits per bin this path supports

template <typename K>
struct SweepTraits {
  static constexpr int IPT = 128 / (int)sizeof(K);        // 16 u64 / 8 u128 keys per thread
  static constexpr int TILE = SWEEP_THREADS * IPT;        // keys per tile (64 KB)
};

struct PartUnit {
  uint64_t start;  // first key (index into the unpartitioned array)
  uint32_t n;      // keys
  uint32_t bin;
};

struct KxGenSmem {
  uint32_t h[1 << SWEEP_UPPER];
  uint32_t bt[KX_RECORDS_PER_CHUNK / 32 + 1];  // k-mers per 32-record batch, then offsets
  unsigned long long base;
};

// Upper digit of a key of a bin with D digit bits (S = min(D, 8) top bits).
template <typename K>
__device__ __forceinline__ uint32_t upper_digit(K key, int key_bits, int D) {
  const int S = D < SWEEP_UPPER ? D : SWEEP_UPPER;
  return S ? (uint32_t)(uint64_t)(key >> (key_bits - S)) : 0u;
}
// Lower digit (the E = D - S bits below the upper digit).
template <typename K>
__device__ __forceinline__ uint32_t lower_digit(K key, int key_bits, int D) {
  const int S = D < SWEEP_UPPER ? D : SWEEP_UPPER;
  const int E = D - S;
  return E ? (uint32_t)(uint64_t)(key >> (key_bits - D)) & ((1u << E) - 1u) : 0u;
}

// sgroup_base[bin]: index of the bin's first super bucket (2^S per bin).
template <typename K, bool NONCANON = false>
__global__ void __launch_bounds__(KX_THREADS)
kx0_gen_kernel(KxArgs<K> a, const uint32_t *__restrict__ sgroup_base, uint32_t *__restrict__ super_hist,
               const uint64_t *__restrict__ bin_key_base, unsigned long long *__restrict__ bin_fill,
               K *__restrict__ keys, uint64_t n_keys, uint32_t *err) {
  __shared__ KxGenSmem s;
  if (a.n_chunks_dyn && blockIdx.x >= *a.n_chunks_dyn) return;
  const Chunk c = a.chunks[blockIdx.x];
  const int D = a.group_D[c.bin];
  const uint32_t NS = 1u << (D < SWEEP_UPPER ? D : SWEEP_UPPER);
  const PieceDesc pd = a.pieces[c.piece];
  const unsigned w = threadIdx.x >> 5, lane = lane_id();
  const uint64_t r_end = c.r0 + c.n_rec;
  for (uint32_t i = threadIdx.x; i < NS; i += KX_THREADS) s.h[i] = 0;
  // k-mers per batch of 32 records, then the chunk's range in its bin
  for (uint64_t r = c.r0 + 32ull * w; r < r_end; r += 32ull * (KX_THREADS / 32)) {
    const RecBatch b = load_batch(pd.index, r, r_end);
    if (lane == 0) s.bt[(r - c.r0) / 32] = b.total;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t nb = (c.n_rec + 31) / 32;
    uint32_t run = 0;
    for (uint32_t i = 0; i < nb; ++i) {
      const uint32_t t = s.bt[i];
      s.bt[i] = run;
      run += t;
    }
    s.base = bin_key_base[c.bin] + atomicAdd(&bin_fill[c.bin], (unsigned long long)run);
  }
  __syncthreads();
  const uint64_t base = s.base;
  for (uint64_t r = c.r0 + 32ull * w; r < r_end; r += 32ull * (KX_THREADS / 32)) {
    const RecBatch b = load_batch(pd.index, r, r_end);
    const uint64_t kb = base + s.bt[(r - c.r0) / 32];
    for (uint32_t it = 0; 32 * it < b.total; ++it) {
      uint32_t rec, j;
      locate(b, it, &rec, &j);
      const uint64_t woff = __shfl_sync(FULL, b.woff, rec);
      if (32 * it + lane >= b.total) continue;
      const K key = a.mixer.mix(NONCANON ? get_kmer<K>(pd.words + woff, j, a.k)
                                         : canonical_kmer<K>(pd.words + woff, j, a.k));
      const uint64_t p = kb + 32 * it + lane;
      if (p < n_keys) keys[p] = key; else atomicOr(err, ERR_CAPACITY);
      atomicAdd(&s.h[upper_digit<K>(key, a.key_bits, D)], 1u);
    }
  }
  __syncthreads();
  uint32_t *hb = super_hist + sgroup_base[c.bin];
  for (uint32_t i = threadIdx.x; i < NS; i += KX_THREADS)
    if (s.h[i]) atomicAdd(&hb[i], s.h[i]);
}

template <typename K>
struct SweepSmem {
  K sorted[SweepTraits<K>::TILE];         // the tile in digit order
  uint32_t h[1 << SWEEP_UPPER];           // tile digit counts
  uint32_t lstart[(1 << SWEEP_UPPER) + 1];  // tile digit starts
  unsigned long long gpos[1 << SWEEP_UPPER];  // global position of each digit's run
  unsigned long long cur[1 << SWEEP_UPPER];   // MODE 1: the super bucket's cursors
  uint32_t ws[SWEEP_THREADS / 32 + 1];
  uint32_t bin;
};

// Arguments of both sweeps.
template <typename K>
struct SweepArgs {
  const K *in;
  K *out;
  uint64_t n_keys;
  int key_bits;
  const uint8_t *group_D;        // digit bits per bin
  const uint32_t *group_base;    // first final bucket of each bin
  const uint32_t *sgroup_base;   // first super bucket of each bin [bins + 1]
  uint32_t n_bins;
  const unsigned long long *super_base;  // first key of each super bucket [n_super + 1]
  unsigned long long *super_cursor;      // MODE 0: keys placed per super bucket
  uint32_t *fine_hist;                   // MODE 1: final bucket sizes (written)
  const PartUnit *units;                 // MODE 0: the bins' tiles
  uint32_t n_units;
  uint32_t n_super;
  uint32_t *err;
  const uint8_t *fused = nullptr;        // MODE 1: bins counted straight from their super buckets
};

// One tile of n keys at in[st ..]: digits (MODE 0 upper, MODE 1 lower),
// the tile sorted by digit in shared memory, each digit's run written at
// gpos[digit] (filled by reserve(), called by thread 0..255 once the tile
// histogram is in s.h; reserve(t) returns the run's global start).
template <typename K, int MODE, typename R>
__device__ __forceinline__ void sweep_tile(const SweepArgs<K> &a, SweepSmem<K> &s, uint64_t st, uint32_t n,
                                           int D, R reserve) {
  constexpr int IPT = SweepTraits<K>::IPT;
  const int tid = threadIdx.x;
  const int nd = 1 << (MODE == 0 ? (D < SWEEP_UPPER ? D : SWEEP_UPPER) : (D - (D < SWEEP_UPPER ? D : SWEEP_UPPER)));
  for (int i = tid; i < nd; i += SWEEP_THREADS) s.h[i] = 0;
  K key[IPT];
  uint32_t rank[IPT / 2];  // two 16-bit ranks per word
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t e = tid + i * SWEEP_THREADS;
    if (e < n) key[i] = a.in[st + e];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t e = tid + i * SWEEP_THREADS;
    uint32_t r = 0;
    if (e < n) {
      const uint32_t d = MODE == 0 ? upper_digit<K>(key[i], a.key_bits, D) : lower_digit<K>(key[i], a.key_bits, D);
      r = atomicAdd(&s.h[d], 1u);
    }
    if (i & 1) rank[i / 2] |= r << 16; else rank[i / 2] = r;
  }
  __syncthreads();
  // digit starts inside the tile (warp scans over the <= 256 counters) and
  // the runs' global places
  if (tid < (1 << SWEEP_UPPER)) {
    const uint32_t c = tid < nd ? s.h[tid] : 0u;
    uint32_t inc = warp_incl_scan(c);
    if ((tid & 31) == 31) s.ws[tid >> 5] = inc;
    __syncwarp();
    s.lstart[tid] = inc - c;  // warp-local for now
    if (tid < nd) s.gpos[tid] = c ? reserve(tid, c) : 0ull;
  }
  __syncthreads();
  if (tid < (1 << SWEEP_UPPER)) {
    uint32_t add = 0;
    for (int w = 0; w < (tid >> 5); ++w) add += s.ws[w];
    s.lstart[tid] += add;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const uint32_t e = tid + i * SWEEP_THREADS;
    if (e < n) {
      const uint32_t d = MODE == 0 ? upper_digit<K>(key[i], a.key_bits, D) : lower_digit<K>(key[i], a.key_bits, D);
      s.sorted[s.lstart[d] + ((rank[i / 2] >> (16 * (i & 1))) & 0xFFFFu)] = key[i];
    }
  }
  __syncthreads();
  for (uint32_t i = tid; i < n; i += SWEEP_THREADS) {
    const K k = s.sorted[i];
    const uint32_t d = MODE == 0 ? upper_digit<K>(k, a.key_bits, D) : lower_digit<K>(k, a.key_bits, D);
    const uint64_t p = s.gpos[d] + (i - s.lstart[d]);
    if (p < a.n_keys) a.out[p] = k; else atomicOr(a.err, ERR_CAPACITY);
  }
  __syncthreads();
}

// MODE 0: persistent CTAs over the bins' tiles (units).  MODE 1: one CTA per
// super bucket.
template <typename K, int MODE>
__global__ void __launch_bounds__(SWEEP_THREADS, 2) kx0_sweep_kernel(SweepArgs<K> a) {
  constexpr int TILE = SweepTraits<K>::TILE;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SweepSmem<K> &s = *reinterpret_cast<SweepSmem<K> *>(smem_raw);
  const int tid = threadIdx.x;
  if (MODE == 0) {
    for (uint32_t u = blockIdx.x; u < a.n_units; u += gridDim.x) {
      const PartUnit un = a.units[u];
      const int D = (int)a.group_D[un.bin];
      const uint32_t sb0 = a.sgroup_base[un.bin];
      sweep_tile<K, 0>(a, s, un.start, un.n, D, [&](uint32_t d, uint32_t c) -> unsigned long long {
        return a.super_base[sb0 + d] + atomicAdd(&a.super_cursor[sb0 + d], (unsigned long long)c);
      });
    }
  } else {
    const uint32_t sb = blockIdx.x;
    if (sb >= a.n_super) return;
    if (tid == 0) {
      uint32_t lo = 0, hi = a.n_bins;  // bin holding super bucket sb
      while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) / 2;
        if (a.sgroup_base[mid] <= sb) lo = mid; else hi = mid;
      }
      s.bin = lo;
    }
    __syncthreads();
    const uint32_t bin = s.bin;
    const int D = (int)a.group_D[bin];
    const int S = D < SWEEP_UPPER ? D : SWEEP_UPPER;
    const int E = D - S;
    const uint64_t st = a.super_base[sb], en = a.super_base[sb + 1];
    if (a.fused && a.fused[bin]) {
      // the bin has no lower digit (E = 0) and its super buckets are counted
      // in place by super_hash_kernel: only the bucket size is recorded
      if (tid == 0) a.fine_hist[a.group_base[bin] + (sb - a.sgroup_base[bin])] = (uint32_t)(en - st);
      return;
    }
    // histogram of the lower digits over the whole super bucket
    for (int i = tid; i < (1 << E); i += SWEEP_THREADS) s.h[i] = 0;
    __syncthreads();
    for (uint64_t e = st + tid; e < en; e += SWEEP_THREADS)
      atomicAdd(&s.h[lower_digit<K>(a.in[e], a.key_bits, D)], 1u);
    __syncthreads();
    // final bucket sizes, and the cursors (exclusive prefix from st)
    const uint32_t fb = a.group_base[bin] + ((sb - a.sgroup_base[bin]) << E);
    if (tid == 0) {
      unsigned long long run = st;
      for (int i = 0; i < (1 << E); ++i) {
        a.fine_hist[fb + i] = s.h[i];
        s.cur[i] = run;
        run += s.h[i];
      }
    }
    __syncthreads();
    for (uint64_t t0 = st; t0 < en; t0 += TILE) {
      const uint32_t n = (uint32_t)((en - t0) < (uint64_t)TILE ? (en - t0) : (uint64_t)TILE);
      sweep_tile<K, 1>(a, s, t0, n, D, [&](uint32_t d, uint32_t c) -> unsigned long long {
        const unsigned long long g = s.cur[d];
        s.cur[d] = g + c;  // only thread d touches cursor d
        return g;
      });
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
