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

namespace kmc {

namespace {

constexpr int PACK_THREADS = 256;
constexpr int SIG_THREADS = 256;
constexpr int SIG_TPOS = 2048;                       // k-mer start positions owned by a CTA
constexpr int SIG_NSIG = SIG_TPOS + kSuperkmerCap;   // positions whose signature is computed
constexpr int SIG_NMM = SIG_NSIG + 64;               // m-mer values (window w <= 62)
constexpr int SIG_NPK = (SIG_NMM + 64 + 64) / 32 + 4;  // packed words staged
constexpr int SIG_NMK = (SIG_NMM + 64 + 64) / 64 + 4;  // mask words staged
constexpr int SIG_SMEM_BINS = 2048;                  // per-bin histograms kept in smem up to this
constexpr int SCAT_THREADS = 256;
constexpr int SCAT_PER_CTA = 2048;
constexpr int STREAM_PAD_WORDS = 8;                  // zero / invalid words after a stream

// ------------------------------------------------------------------ a1

// 2-bit code of an ASCII base (A0 C1 G2 T3) and whether it is one.
__device__ __forceinline__ unsigned base_code(unsigned c, bool *ok) {
  unsigned code = ((c >> 1) ^ (c >> 2)) & 3u;   // A 0x41->0, C 0x43->1, G 0x47->2, T 0x54->3
  const unsigned ref = 0x54474341u >> (8 * code);  // "ACGT" little-endian
  *ok = (ref & 0xFFu) == c;
  return code;
}

// Thread t packs stream positions [64t, 64t+64): two 2-bit words and one
// invalid-mask word (bit set = not a base, or outside [mis, n_stream)).
__global__ void __launch_bounds__(PACK_THREADS)
pack_kernel(const uint8_t *__restrict__ aligned, uint64_t n_stream, uint32_t mis,
            uint64_t *__restrict__ packed, uint64_t *__restrict__ inval, uint64_t n_mwords) {
  const uint64_t t = (uint64_t)blockIdx.x * PACK_THREADS + threadIdx.x;
  if (t >= n_mwords) return;
  const uint64_t q0 = t * 64;
  uint64_t pw[2] = {0, 0}, iv = ~0ull;
  if (q0 < n_stream) {
    iv = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint64_t cq = q0 + 16 * c;
      uint8_t by[16];
      if (cq >= mis && cq + 16 <= n_stream) {
        uint4 v = *reinterpret_cast<const uint4 *>(aligned + cq);
        memcpy(by, &v, 16);
      } else {
        for (int j = 0; j < 16; ++j) {
          uint64_t q = cq + j;
          by[j] = (q >= mis && q < n_stream) ? aligned[q] : (uint8_t)'N';
        }
      }
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const int i = 16 * c + j;  // 0..63
        bool ok;
        unsigned code = base_code(by[j], &ok);
        const uint64_t q = q0 + i;
        if (q < mis || q >= n_stream) ok = false;
        if (!ok) code = 0;
        pw[i >> 5] |= (uint64_t)code << (62 - 2 * (i & 31));
        if (!ok) iv |= 1ull << (63 - i);
      }
    }
  }
  packed[2 * t] = pw[0];
  packed[2 * t + 1] = pw[1];
  inval[t] = iv;
}

// Marks read starts (bit set at the stream position of each read's first
// byte) and checks that offsets do not decrease.
__global__ void starts_kernel(const uint64_t *__restrict__ offsets, uint64_t r0, uint64_t r1,
                              uint64_t byte_start, uint32_t mis, uint64_t n_stream,
                              unsigned long long *smask, uint32_t *err) {
  for (uint64_t i = r0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < r1;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t a = offsets[i], b = offsets[i + 1];
    if (b < a || a < byte_start) atomicOr(err, ERR_INPUT);
    const uint64_t q = a - byte_start + mis;
    if (a >= byte_start && q < n_stream) atomicOr(&smask[q >> 6], 1ull << (63 - (q & 63)));
  }
}

// ------------------------------------------------------------------ a2

struct SigArgs {
  const uint64_t *packed, *inval, *smask;
  uint64_t n_pwords, n_mwords, n_stream;
  const uint64_t *offsets;
  uint64_t r0, r1, byte_start;
  uint32_t mis;
  int k, m;
  const uint32_t *map;
  uint32_t n_bins;
  uint64_t *list;                 // super k-mer list (NULL in sample mode)
  unsigned long long *n_list;
  uint64_t list_cap;
  unsigned long long *bin_rec, *bin_words, *bin_kmers;  // [n_bins]
  unsigned long long *sig_weight;  // sample mode: k-mers per signature
  uint32_t *err;
};

struct SigSmem {
  uint64_t pk[SIG_NPK];
  uint64_t iv[SIG_NMK];
  uint64_t sm[SIG_NMK];
  int64_t lastw[SIG_NMK];          // last read start before each staged mask word
  uint32_t mm[2][SIG_NMM];         // m-mer values, then window minima
  uint8_t valid[SIG_NSIG];
  uint8_t brk[SIG_NSIG];
  uint16_t blist[SIG_NSIG + 1];
  uint16_t bidx[SIG_NSIG];
  uint32_t ws[SIG_THREADS / 32 + 1];
  uint32_t h_rec[SIG_SMEM_BINS], h_words[SIG_SMEM_BINS], h_kmers[SIG_SMEM_BINS];
  int64_t rs0;
  unsigned long long out_base;
};

// One CTA owns the k-mer start positions [t0, t0+SIG_TPOS) of the stream.
// It computes, for positions t0-1 .. t0+SIG_NSIG-2, the Sect. 2.2 signature
// of the k-mer starting there (sliding minimum over the k-m+1 m-mers of the
// canonical, rule-filtered m-mer values), the k-mer's validity, and super
// k-mer starts: a valid k-mer starts a super k-mer when the previous one is
// invalid, has another signature, or when its position in its read is a
// multiple of kSuperkmerCap.  It then emits the super k-mers that start in
// its range (each ends within kSuperkmerCap positions, inside the window).
__global__ void __launch_bounds__(SIG_THREADS) sig_kernel(SigArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SigSmem &s = *reinterpret_cast<SigSmem *>(smem_raw);
  const int tid = threadIdx.x;
  const int64_t t0 = (int64_t)blockIdx.x * SIG_TPOS;
  const int k = a.k, m = a.m, w = k - m + 1;
  const uint32_t SENT = 1u << (2 * m);
  const bool small_bins = a.n_bins <= (uint32_t)SIG_SMEM_BINS;
  // staged ranges
  const int64_t pw0 = t0 >= 32 ? t0 / 32 - 1 : 0;   // first packed word
  const int64_t LB = pw0 * 32;                     // its first position
  const int64_t mw0 = t0 >= 64 ? t0 / 64 - 1 : 0;   // first mask word
  const int64_t LBm = mw0 * 64;
  for (int i = tid; i < SIG_NPK; i += SIG_THREADS) {
    uint64_t gi = (uint64_t)(pw0 + i);
    s.pk[i] = gi < a.n_pwords ? a.packed[gi] : 0ull;
  }
  for (int i = tid; i < SIG_NMK; i += SIG_THREADS) {
    uint64_t gi = (uint64_t)(mw0 + i);
    s.iv[i] = gi < a.n_mwords ? a.inval[gi] : ~0ull;
    s.sm[i] = gi < a.n_mwords ? a.smask[gi] : 0ull;
  }
  if (small_bins && a.list)
    for (int i = tid; i < (int)a.n_bins; i += SIG_THREADS) s.h_rec[i] = s.h_words[i] = s.h_kmers[i] = 0;
  if (tid == 0) {
    // read containing stream position LBm: largest i with start(i) <= LBm
    uint64_t lo = a.r0, hi = a.r1;  // search in [r0, r1)
    int64_t rs = 0;
    while (lo < hi) {
      uint64_t mid = (lo + hi) / 2;
      int64_t sp = (int64_t)(a.offsets[mid] - a.byte_start) + a.mis;
      if (sp <= LBm) { rs = sp; lo = mid + 1; } else hi = mid;
    }
    s.rs0 = rs;
  }
  __syncthreads();
  if (tid < 32) {
    // last read start strictly before each staged mask word (prefix max)
    int64_t carry = s.rs0;
    for (int base = 0; base < SIG_NMK; base += 32) {
      int i = base + tid;
      int64_t here = -1;
      if (i < SIG_NMK && s.sm[i]) here = LBm + (int64_t)i * 64 + 64 - __ffsll((long long)s.sm[i]);
      // inclusive prefix max over lanes
      int64_t v = here;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        int64_t o = __shfl_up_sync(FULL, v, d);
        if (tid >= d && o > v) v = o;
      }
      int64_t excl = __shfl_up_sync(FULL, v, 1);
      if (tid == 0) excl = -1;
      int64_t before = excl > carry ? excl : carry;
      if (i < SIG_NMK) s.lastw[i] = before;
      int64_t tot = __shfl_sync(FULL, v, 31);
      if (tot > carry) carry = tot;
    }
  }
  // m-mer values at positions t0-1+j, j in [0, SIG_NMM)
  for (int j = tid; j < SIG_NMM; j += SIG_THREADS) {
    const int64_t pos = t0 - 1 + j;
    uint32_t v = SENT;
    if (pos >= 0) {
      uint32_t f = (uint32_t)get_bits(s.pk, (uint64_t)(2 * (pos - LB)), 2 * m);
      uint32_t r = revcomp32(f, m);
      uint32_t c = f < r ? f : r;            // canonical m-mer (Sect. 2.1)
      v = mmer_allowed(c, m) ? c : SENT;     // Sect. 2.2 filter
    }
    s.mm[0][j] = v;
  }
  __syncthreads();
  // sliding-window minimum: doubling to the largest power of two P <= w
  int src = 0, P = 1;
  while (2 * P <= w) {
    const int lim = SIG_NMM - 2 * P + 1;
    for (int j = tid; j < lim; j += SIG_THREADS) {
      uint32_t x = s.mm[src][j], y = s.mm[src][j + P];
      s.mm[src ^ 1][j] = x < y ? x : y;
    }
    __syncthreads();
    src ^= 1;
    P *= 2;
  }
  // signature, validity and cut flag per window position j in [0, SIG_NSIG)
  uint32_t *sig = s.mm[src ^ 1];
  for (int j = tid; j < SIG_NSIG; j += SIG_THREADS) {
    uint32_t x = s.mm[src][j], y = s.mm[src][j + w - P];
    sig[j] = x < y ? x : y;
    const int64_t pos = t0 - 1 + j;
    bool ok = pos >= 0;
    if (ok) {
      const uint64_t lp = (uint64_t)(pos - LBm);
      ok = get_bits(s.iv, lp, k) == 0ull;
      if (ok && k > 1) ok = get_bits(s.sm, lp + 1, k - 1) == 0ull;
    }
    uint8_t cut = 0;
    if (ok) {
      // start of the read holding pos: last read start at or before pos
      const uint64_t lp = (uint64_t)(pos - LBm);
      const int wi = (int)(lp >> 6);
      const uint64_t x2 = s.sm[wi] & (~0ull << (63 - (lp & 63)));
      int64_t rs = x2 ? LBm + (int64_t)wi * 64 + 64 - __ffsll((long long)x2) : s.lastw[wi];
      cut = ((pos - rs) % kSuperkmerCap) == 0;
    }
    s.valid[j] = ok ? (uint8_t)(1 + cut) : (uint8_t)0;  // 0 invalid, 1 valid, 2 valid + cut
  }
  __syncthreads();
  // break flags (j >= 1): invalid, or a super k-mer starts here
  for (int j = tid; j < SIG_NSIG; j += SIG_THREADS) {
    uint8_t b = 1;
    if (j >= 1 && s.valid[j]) b = (s.valid[j - 1] == 0) || (sig[j] != sig[j - 1]) || (s.valid[j] == 2);
    s.brk[j] = b;
  }
  __syncthreads();
  // compact break positions (j in [1, SIG_NSIG)); contiguous chunks per thread
  constexpr int PER = (SIG_NSIG + SIG_THREADS - 1) / SIG_THREADS;
  const int j0 = 1 + tid * PER;
  uint32_t nb = 0;
  for (int q = 0; q < PER; ++q) {
    int j = j0 + q;
    if (j < SIG_NSIG && s.brk[j]) ++nb;
  }
  uint32_t nbt;
  uint32_t bi = block_excl_scan<uint32_t, SIG_THREADS>(nb, s.ws, &nbt);
  for (int q = 0; q < PER; ++q) {
    int j = j0 + q;
    if (j < SIG_NSIG && s.brk[j]) { s.blist[bi] = (uint16_t)j; s.bidx[j] = (uint16_t)bi; ++bi; }
  }
  if (tid == 0) s.blist[nbt] = (uint16_t)SIG_NSIG;
  __syncthreads();
  // owned super k-mer starts: j in [1, SIG_TPOS], valid and break
  uint32_t ns = 0;
  for (int q = 0; q < PER; ++q) {
    int j = j0 + q;
    if (j <= SIG_TPOS && s.valid[j] && s.brk[j]) ++ns;
  }
  uint32_t nst;
  uint32_t si = block_excl_scan<uint32_t, SIG_THREADS>(ns, s.ws, &nst);
  if (a.list) {
    if (tid == 0) s.out_base = nst ? atomicAdd(a.n_list, (unsigned long long)nst) : 0ull;
    __syncthreads();
    if (s.out_base + nst > a.list_cap) {
      if (tid == 0) atomicOr(a.err, ERR_CAPACITY);
      return;
    }
  }
  for (int q = 0; q < PER; ++q) {
    int j = j0 + q;
    if (!(j <= SIG_TPOS && s.valid[j] && s.brk[j])) continue;
    const uint32_t n = (uint32_t)s.blist[s.bidx[j] + 1] - (uint32_t)j;  // k-mers in the super k-mer
    const uint32_t g = sig[j];
    if (!a.list) {  // sample mode: signature weights
      atomicAdd(&a.sig_weight[g], (unsigned long long)n);
      continue;
    }
    const uint64_t pos = (uint64_t)(t0 - 1 + j);
    a.list[s.out_base + si] = (pos << 32) | ((uint64_t)(n - 1) << 25) | g;
    ++si;
    const uint32_t bin = a.map[g];
    const uint32_t nw = (2 * (n + k - 1) + 63) / 64;
    if (small_bins) {
      atomicAdd(&s.h_rec[bin], 1u);
      atomicAdd(&s.h_words[bin], nw);
      atomicAdd(&s.h_kmers[bin], n);
    } else {
      atomicAdd(&a.bin_rec[bin], 1ull);
      atomicAdd(&a.bin_words[bin], (unsigned long long)nw);
      atomicAdd(&a.bin_kmers[bin], (unsigned long long)n);
    }
  }
  if (small_bins && a.list) {
    __syncthreads();
    for (int i = tid; i < (int)a.n_bins; i += SIG_THREADS) {
      if (s.h_rec[i]) {
        atomicAdd(&a.bin_rec[i], (unsigned long long)s.h_rec[i]);
        atomicAdd(&a.bin_words[i], (unsigned long long)s.h_words[i]);
        atomicAdd(&a.bin_kmers[i], (unsigned long long)s.h_kmers[i]);
      }
    }
  }
}

// ------------------------------------------------------------------ a3

struct ScatSmem {
  uint32_t c_rec[SIG_SMEM_BINS], c_words[SIG_SMEM_BINS];
  unsigned long long b_rec[SIG_SMEM_BINS], b_words[SIG_SMEM_BINS];
};

// Scatters super k-mer records into their bins: an index entry (word
// offset | n_kmers-1 | signature) and the packed bases (Sect. 2.4: super
// k-mers are sent to bins).  Space is reserved per CTA and bin with one
// global atomic per non-empty bin (per record when there are many bins).
__global__ void __launch_bounds__(SCAT_THREADS)
scatter_kernel(const uint64_t *__restrict__ list, uint64_t n_list, const uint32_t *__restrict__ map,
               uint32_t n_bins, int k, const uint64_t *__restrict__ packed,
               unsigned long long *rec_cursor, unsigned long long *word_cursor,
               uint64_t *__restrict__ index, uint64_t *__restrict__ words) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatSmem &s = *reinterpret_cast<ScatSmem *>(smem_raw);
  const bool small_bins = n_bins <= (uint32_t)SIG_SMEM_BINS;
  const uint64_t c0 = (uint64_t)blockIdx.x * SCAT_PER_CTA;
  constexpr int PER = SCAT_PER_CTA / SCAT_THREADS;
  uint64_t rec[PER];
  uint32_t bin[PER], nw[PER];
  if (small_bins) {
    for (int i = threadIdx.x; i < (int)n_bins; i += SCAT_THREADS) s.c_rec[i] = s.c_words[i] = 0;
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const uint64_t i = c0 + (uint64_t)q * SCAT_THREADS + threadIdx.x;
    rec[q] = i < n_list ? list[i] : ~0ull;
    if (i < n_list) {
      const uint32_t n = (uint32_t)((rec[q] >> 25) & 127u) + 1;
      bin[q] = map[rec[q] & 0x1FFFFFFu];
      nw[q] = (2 * (n + k - 1) + 63) / 64;
      if (small_bins) {
        atomicAdd(&s.c_rec[bin[q]], 1u);
        atomicAdd(&s.c_words[bin[q]], nw[q]);
      }
    }
  }
  if (small_bins) {
    __syncthreads();
    for (int i = threadIdx.x; i < (int)n_bins; i += SCAT_THREADS) {
      if (s.c_rec[i]) {
        s.b_rec[i] = atomicAdd(&rec_cursor[i], (unsigned long long)s.c_rec[i]);
        s.b_words[i] = atomicAdd(&word_cursor[i], (unsigned long long)s.c_words[i]);
      }
      s.c_rec[i] = 0;
      s.c_words[i] = 0;
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const uint64_t i = c0 + (uint64_t)q * SCAT_THREADS + threadIdx.x;
    if (i >= n_list) continue;
    uint64_t ri, wi;
    if (small_bins) {
      ri = s.b_rec[bin[q]] + atomicAdd(&s.c_rec[bin[q]], 1u);
      wi = s.b_words[bin[q]] + atomicAdd(&s.c_words[bin[q]], nw[q]);
    } else {
      ri = atomicAdd(&rec_cursor[bin[q]], 1ull);
      wi = atomicAdd(&word_cursor[bin[q]], (unsigned long long)nw[q]);
    }
    const uint64_t pos = rec[q] >> 32;
    const uint32_t n = (uint32_t)((rec[q] >> 25) & 127u) + 1;
    const uint32_t nbits = 2 * (n + k - 1);
    for (uint32_t j = 0; j < nw[q]; ++j) {
      uint64_t v = get_bits(packed, 2 * pos + 64ull * j, 64);
      const uint32_t used = nbits - 64 * j;
      if (used < 64) v &= ~0ull << (64 - used);
      words[wi + j] = v;
    }
    index[ri] = (wi << 32) | (rec[q] & 0xFFFFFFFFull);
  }
}

// ------------------------------------------------------------------ bin map

// Sort key for the map: heaviest signature first, ties by smaller signature.
__global__ void map_keys_kernel(const unsigned long long *w, uint32_t n_sig, uint64_t *keys,
                                uint32_t *vals) {
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sig; s += gridDim.x * blockDim.x) {
    const uint64_t wt = w[s] > 0xFFFFFFFFull ? 0xFFFFFFFFull : w[s];
    keys[s] = ((0xFFFFFFFFull - wt) << 24) | s;
    vals[s] = s;
  }
}
__global__ void map_weights_kernel(const uint64_t *keys, uint32_t n_sig, uint64_t *wts) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_sig; i += gridDim.x * blockDim.x)
    wts[i] = 0xFFFFFFFFull - (keys[i] >> 24);
}
// Sect. 2.4 merge of signatures into bins: the signature whose sorted-order
// preceding weight is W goes to bin floor(W*B/total); unseen: s mod B.
__global__ void map_assign_kernel(const uint64_t *keys, const uint64_t *prefix, uint32_t n_sig,
                                  uint32_t n_bins, uint32_t *map) {
  const uint64_t total = prefix[n_sig];
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_sig; i += gridDim.x * blockDim.x) {
    const uint32_t sg = (uint32_t)(keys[i] & 0xFFFFFFu);
    const uint64_t wt = 0xFFFFFFFFull - (keys[i] >> 24);
    map[sg] = (wt == 0 || total == 0) ? sg % n_bins : (uint32_t)((prefix[i] * n_bins) / total);
  }
}

// Converts the raw super k-mer list of a piece into (read index, position in
// read) for inspection.
__global__ void dbg_locate_kernel(const uint64_t *list, uint64_t n, const uint64_t *offsets,
                                  uint64_t r0, uint64_t r1, uint64_t byte_start, uint32_t mis,
                                  uint64_t read_base, uint64_t *read_idx, uint32_t *rel) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t q = list[i] >> 32;
    const uint64_t b = q - mis + byte_start;  // byte offset in the caller's buffer
    uint64_t lo = r0, hi = r1, r = r0;
    while (lo < hi) {
      uint64_t mid = (lo + hi) / 2;
      if (offsets[mid] <= b) { r = mid; lo = mid + 1; } else hi = mid;
    }
    // skip empty reads that share the start
    while (r + 1 < r1 && offsets[r + 1] <= b) ++r;
    read_idx[i] = read_base + r;
    rel[i] = (uint32_t)(b - offsets[r]);
  }
}

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
  return a;
}

int launch_sig(Handle &h, const SigArgs &a, uint64_t n_stream, int stage) {
  const uint64_t n_tiles = (n_stream + SIG_TPOS - 1) / SIG_TPOS;
  static bool attr_set = false;
  if (!attr_set) {
    KMC_CUDA_TRY(cudaFuncSetAttribute(sig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sizeof(SigSmem)));
    attr_set = true;
  }
  if (n_tiles == 0) return KMC_OK;
  StageScope sc(h, stage);
  sig_kernel<<<(unsigned)n_tiles, SIG_THREADS, sizeof(SigSmem), h.st>>>(a); KMC_COUNT_LAUNCH();
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
    static bool attr_set = false;
    if (!attr_set) {
      KMC_CUDA_TRY(cudaFuncSetAttribute(scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)sizeof(ScatSmem)));
      attr_set = true;
    }
    StageScope sc(h, KMC_STAGE_BIN_SCATTER);
    scatter_kernel<<<(unsigned)((n_rec + SCAT_PER_CTA - 1) / SCAT_PER_CTA), SCAT_THREADS,
                     sizeof(ScatSmem), h.st>>>(as<uint64_t>(ds.list), n_rec, as<uint32_t>(h.map), B,
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
