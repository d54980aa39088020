// Kernels of the distribution phase (paper Sect. 2.4, Fig. 1): 2-bit
// packing, read-start marks, the signature scan and the bin scatter.  Kept
// in a header so that the single-set path (distribute.cu) and the batched
// path (batch.cu) compile the same kernels.
//
// A "stream" is the bytes of a run of whole reads, starting at the 16-byte
// aligned address at or before the first read; stream position q is byte
// (aligned + q); the `mis` bytes before the first read are invalid.
//
// Batches: several read sets share one stream; set s owns bins
// [s*bins_per_slot, (s+1)*bins_per_slot), so the sets never mix.  Sizes that
// only the device knows (stream length, number of super k-mers) can be read
// from device memory (`dyn`), so a batch runs without host synchronisation.
#pragma once
#include <atomic>

#include "common.cuh"
#include "sortlib.cuh"

namespace kmc {

// Sizes of one batch, in device memory (all zero-initialised by the host).
struct BatchDyn {
  unsigned long long n_stream;   // stream length (bases)
  unsigned long long n_reads;    // reads
  unsigned long long n_list;     // super k-mers found (written by the scan)
  unsigned long long n_chunks;   // record chunks (written by the chunk planner)
  unsigned long long n_sv;       // k-mers kept (written by the counting)
  unsigned long long n_sets;     // sets in the batch
  unsigned long long pad[2];
};

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
constexpr int SCAT_PER_CTA = 1024;
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
            uint64_t *__restrict__ packed, uint64_t *__restrict__ inval, uint64_t n_mwords,
            const unsigned long long *n_stream_dyn = nullptr) {
  const uint64_t t = (uint64_t)blockIdx.x * PACK_THREADS + threadIdx.x;
  if (t >= n_mwords) return;
  if (n_stream_dyn && *n_stream_dyn < n_stream) n_stream = *n_stream_dyn;
  const uint64_t q0 = t * 64;
  uint64_t pw[2] = {0, 0}, iv = ~0ull;
  if (q0 < n_stream) {
    iv = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const uint64_t cq = q0 + 16 * c;
      uint32_t wd[4];
      if (cq >= mis && cq + 16 <= n_stream) {
        const uint4 v = *reinterpret_cast<const uint4 *>(aligned + cq);
        wd[0] = v.x; wd[1] = v.y; wd[2] = v.z; wd[3] = v.w;
      } else {  // a stream edge: bytes outside [mis, n_stream) read as 'N'
        uint8_t by[16];
        for (int j = 0; j < 16; ++j) {
          const uint64_t q = cq + j;
          by[j] = (q >= mis && q < n_stream) ? aligned[q] : (uint8_t)'N';
        }
        memcpy(wd, by, 16);
      }
      // four bases per 32-bit word (byte j = base j): codes from bits 1-2
      // and 2-3 of each byte; a byte is a base when it equals "ACGT"[code]
#pragma unroll
      for (int qw = 0; qw < 4; ++qw) {
        const uint32_t w = wd[qw];
        uint32_t cd = ((w >> 1) ^ (w >> 2)) & 0x03030303u;
        const uint32_t sel = (cd & 0x3u) | ((cd >> 4) & 0x30u) | ((cd >> 8) & 0x300u) | ((cd >> 12) & 0x3000u);
        const uint32_t ok = __vcmpeq4(w, __byte_perm(0x54474341u, 0u, sel));  // 0xFF per base
        cd &= ok;
        const uint32_t g8 = ((cd & 3u) << 6) | (((cd >> 8) & 3u) << 4) | (((cd >> 16) & 3u) << 2) | (cd >> 24);
        const uint32_t nb = ~ok;
        const uint32_t i4 = ((nb >> 4) & 8u) | ((nb >> 13) & 4u) | ((nb >> 22) & 2u) | (nb >> 31);
        const int kq = 4 * c + qw;  // bases 4 kq .. 4 kq + 3 of the thread's 64
        pw[kq >> 3] |= (uint64_t)g8 << (56 - 8 * (kq & 7));
        iv |= (uint64_t)i4 << (60 - 4 * kq);
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
                              unsigned long long *smask, uint32_t *err,
                              const unsigned long long *n_reads_dyn = nullptr) {
  if (n_reads_dyn && *n_reads_dyn < r1) r1 = *n_reads_dyn;
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
  // batches (all optional): stream length on the device, set boundaries
  const unsigned long long *n_stream_dyn;
  const unsigned long long *n_reads_dyn;  // reads on the device (caps r1)
  const uint64_t *set_starts;      // stream position where set s begins, [n_slots + 1]
  uint32_t n_slots;                // 0 or 1: a single set
  uint32_t bins_per_slot;
  uint32_t no_filter;              // 1: canonical minimizers (no Sect. 2.2 filter)
  const uint32_t *abm;             // allowed m-mers of length m, one bit each (lane-block scan)
};

// Set holding stream position pos (largest s with set_starts[s] <= pos).
__device__ __forceinline__ uint32_t slot_of(const uint64_t *set_starts, uint32_t n_slots,
                                            uint64_t pos) {
  if (n_slots <= 1) return 0;
  uint32_t lo = 0, hi = n_slots;
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) / 2;
    if (set_starts[mid] <= pos) lo = mid; else hi = mid;
  }
  return lo;
}

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
  if (a.n_stream_dyn && (unsigned long long)t0 >= *a.n_stream_dyn) return;
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
    if (a.n_reads_dyn && *a.n_reads_dyn < hi) hi = *a.n_reads_dyn;
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
      v = (a.no_filter || mmer_allowed(c, m)) ? c : SENT;  // Sect. 2.2 filter
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
    const uint32_t bin = slot_of(a.set_starts, a.n_slots, pos) * a.bins_per_slot + a.map[g];
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

// The Sect. 2.2 rule as one bit per m-mer (4^m / 32 words), built on the
// device once per handle or batch engine: the lane-block scan looks a
// canonical m-mer up instead of testing its AAA / ACA / AA patterns.
inline uint32_t mmer_bm_words(int m) { return ((1u << (2 * m)) + 31u) / 32u; }
__global__ void mmer_bm_kernel(uint32_t *bm, int m, uint32_t n_words) {
  for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < n_words; w += gridDim.x * blockDim.x) {
    uint32_t bits = 0;
    for (int b = 0; b < 32; ++b) {
      const uint32_t v = w * 32u + (uint32_t)b;
      if (v < (1u << (2 * m)) && mmer_allowed(v, m)) bits |= 1u << b;
    }
    bm[w] = bits;
  }
}
// Launches the build on `st` (bm holds mmer_bm_words(m) words); 1 launch.
inline cudaError_t build_mmer_bm(uint32_t *bm, int m, cudaStream_t st) {
  const uint32_t n = mmer_bm_words(m);
  mmer_bm_kernel<<<(n + 255) / 256, 256, 0, st>>>(bm, m, n);
  return cudaGetLastError();
}
__device__ __forceinline__ bool mmer_bit(const uint32_t *bm, uint32_t v) {
  return (__ldg(bm + (v >> 5)) >> (v & 31u)) & 1u;
}

// ----------------------------------------------- a2, lane-block version
// Same result as sig_kernel, organised for fewer instructions per position.
// Each of the 256 lanes of a CTA owns a block of w = k-m+1 consecutive
// positions.  A lane rolls its m-mer values (canonical, rule-filtered) over
// its block and stores them with their running prefix minima in its own
// shared-memory row; the minimum over the window [p, p+w-1] is then the
// smaller of the suffix minimum of p's block (from p) and the prefix minimum
// of the next block (to p+w-1): van Herk / Gil-Werman with block size w.
// The last lane only lends its prefix minima, so a CTA covers (lanes-1)*w positions,
// starting one position before the k-mer starts it owns and extending
// kSuperkmerCap past them (a super k-mer never spans more).

constexpr int SIG2_LANES = 256;
constexpr int SIG2_MAXW = 64;
// Mask words staged per CTA (the lanes' blocks, the k-1 positions after
// them, alignment); twice as many packed words (32 bases each) are staged.
__host__ __device__ inline int sig2_mwords(int k, int m) {
  return (SIG2_LANES * (k - m + 1) + 2 * k + 256) / 64 + 4;
}
static_assert((kSuperkmerCap & (kSuperkmerCap - 1)) == 0, "cut test uses a mask");
// a CTA's per-bin counters are packed in 21-bit fields
static_assert((SIG2_LANES - 1) * SIG2_MAXW * 8 < (1 << 21), "per-CTA counts fit 21 bits");

__host__ __device__ inline int sig2_own(int k, int m) {
  const int w = k - m + 1;
  return (SIG2_LANES - 1) * w - 1 - kSuperkmerCap;  // owned k-mer start positions per CTA
}
__host__ __device__ inline int sig2_stride(int k, int m) {
  return (k - m + 1) | 1;  // odd row stride: lanes touching the same column hit distinct banks
}
__host__ __device__ inline int sig2_hist_bins(uint32_t n_bins) {
  return n_bins <= (uint32_t)SIG_SMEM_BINS ? (int)n_bins : 0;
}
// m-mer values and signatures are kept as 16-bit words when m <= 7 (the
// sentinel 4^m fits), which halves the largest shared array and lets more
// CTAs share an SM.
inline size_t sig2_value_bytes(int m) { return m <= 7 ? 2 : 4; }
inline size_t sig2_smem_bytes(int k, int m, uint32_t n_bins) {
  const size_t vb = 2 * (size_t)SIG2_LANES * sig2_stride(k, m) * sig2_value_bytes(m);
  const size_t mw = (size_t)sig2_mwords(k, m);
  return 2 * mw * 8 + 4 * mw * 8 + (size_t)SIG2_LANES * 8 +
         ((vb + 7) & ~(size_t)7) + (size_t)sig2_hist_bins(n_bins) * 8;
}
// The lane-block form pays off once a block holds several positions.
inline bool sig2_applies(int k, int m) { return k - m + 1 >= 8 && k - m + 1 <= SIG2_MAXW; }

// VT: 16- or 32-bit m-mer values; NOFILTER: canonical minimizers instead of
// signatures (a compile-time switch, so that the signature scan pays
// nothing for it).
template <typename VT, bool NOFILTER>
__global__ void __launch_bounds__(SIG2_LANES) sig2_kernel(SigArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = threadIdx.x;
  const int k = a.k, m = a.m, w = k - m + 1;
  const int own = sig2_own(k, m), stride = sig2_stride(k, m);
  const int64_t T0 = (int64_t)blockIdx.x * own;        // first owned start
  if (a.n_stream_dyn && (unsigned long long)T0 >= *a.n_stream_dyn) return;
  const int64_t B0 = T0 - 1;                           // first position of lane 0's block
  const uint32_t SENT = 1u << (2 * m);
  const int hb = sig2_hist_bins(a.n_bins);
  const bool small_bins = hb > 0;
  // shared memory carve-up
  uint64_t *pk = reinterpret_cast<uint64_t *>(smem_raw);
  const int MW = sig2_mwords(k, m), PW = 2 * MW;
  uint64_t *iv = pk + PW;                               // invalid bases
  uint64_t *sm = iv + MW;                               // read starts
  uint64_t *cm = sm + MW;                               // invalid base or read start
  int64_t *lastw = reinterpret_cast<int64_t *>(cm + MW);
  int64_t *fbrk = lastw + MW;                           // first break of each lane's block
  VT *V = reinterpret_cast<VT *>(fbrk + SIG2_LANES);   // values, then signatures
  VT *P = V + SIG2_LANES * stride;                     // prefix minima
  // per-bin records | words << 21 | k-mers << 42 of this CTA (fields < 2^21)
  unsigned long long *hpk = reinterpret_cast<unsigned long long *>(
      (reinterpret_cast<uintptr_t>(P + SIG2_LANES * stride) + 7) & ~(uintptr_t)7);
  __shared__ uint32_t ws[SIG2_LANES / 32 + 1];
  __shared__ int64_t rs0;
  __shared__ unsigned long long out_base;
  // stage packed codes and masks from position B0 (rounded down to a word)
  const int64_t pw0 = B0 >= 0 ? B0 / 32 : -1;
  const int64_t LB = pw0 * 32;
  const int64_t mw0 = B0 >= 0 ? B0 / 64 : -1;
  const int64_t LBm = mw0 * 64;
  for (int i = L; i < PW; i += SIG2_LANES) {
    const int64_t gi = pw0 + i;
    pk[i] = (gi >= 0 && (uint64_t)gi < a.n_pwords) ? a.packed[gi] : 0ull;
  }
  for (int i = L; i < MW; i += SIG2_LANES) {
    const int64_t gi = mw0 + i;
    const bool in = gi >= 0 && (uint64_t)gi < a.n_mwords;
    const uint64_t x = in ? a.inval[gi] : ~0ull, y = in ? a.smask[gi] : 0ull;
    iv[i] = x;
    sm[i] = y;
    cm[i] = x | y;
  }
  if (small_bins && a.list)
    for (int i = L; i < hb; i += SIG2_LANES) hpk[i] = 0;
  if (L < 32) {
    // last read start before position LBm: the read-start mask read
    // backwards, 32 words (2,048 positions) per step
    int64_t rs = 0;
    for (int64_t wb = mw0 - 1; wb >= 0; wb -= 32) {
      const int64_t wq = wb - L;
      const uint64_t x = (wq >= 0 && (uint64_t)wq < a.n_mwords) ? a.smask[wq] : 0ull;
      const unsigned hit = __ballot_sync(FULL, x != 0);
      if (hit) {
        const int src = __ffs(hit) - 1;  // the highest word with a start
        const uint64_t xs = __shfl_sync(FULL, x, src);
        rs = (wb - src) * 64 + 63 - (__ffsll((long long)xs) - 1);
        break;
      }
    }
    if (L == 0) rs0 = rs;
  }
  __syncthreads();
  if (L < 32) {
    // last read start strictly before each staged mask word (prefix max)
    int64_t carry = rs0;
    for (int base = 0; base < MW; base += 32) {
      const int i = base + L;
      int64_t here = -1;
      if (i < MW && sm[i]) here = LBm + (int64_t)i * 64 + 64 - __ffsll((long long)sm[i]);
      int64_t v = here;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int64_t o = __shfl_up_sync(FULL, v, d);
        if (L >= d && o > v) v = o;
      }
      int64_t excl = __shfl_up_sync(FULL, v, 1);
      if (L == 0) excl = -1;
      if (i < MW) lastw[i] = excl > carry ? excl : carry;
      const int64_t tot = __shfl_sync(FULL, v, 31);
      if (tot > carry) carry = tot;
    }
  }
  // phase 1: m-mer values of the lane's block and their prefix minima; the
  // 2-bit codes stream out of a register word, refilled every 32 bases
  const int64_t p0 = B0 + (int64_t)L * w;               // >= B0 >= LB, LBm
  {
    const uint32_t *abm = a.abm;  // allowed m-mers (Sect. 2.2)
    const uint32_t mmask = SENT - 1u;
    const uint32_t bit0 = (uint32_t)(2 * (p0 - LB));
    int wi = (int)(bit0 >> 6);
    uint64_t cur = pk[wi] << (bit0 & 63);
    int rem = 32 - (int)((bit0 & 63) >> 1);
    uint32_t fw = 0, rc = 0;
    const int rsh = 2 * m - 2;
    for (int q = 0; q < m - 1; ++q) {
      if (rem == 0) { cur = pk[++wi]; rem = 32; }
      const uint32_t c = (uint32_t)(cur >> 62);
      cur <<= 2;
      --rem;
      fw = ((fw << 2) | c) & mmask;
      rc = (rc >> 2) | ((3u - c) << rsh);
    }
    uint32_t pm = 0xFFFFFFFFu;
    for (int j = 0; j < w; ++j) {
      if (rem == 0) { cur = pk[++wi]; rem = 32; }
      const uint32_t c = (uint32_t)(cur >> 62);
      cur <<= 2;
      --rem;
      fw = ((fw << 2) | c) & mmask;
      rc = (rc >> 2) | ((3u - c) << rsh);
      const uint32_t cn = fw < rc ? fw : rc;                 // canonical m-mer (Sect. 2.1)
      const uint32_t v = (NOFILTER || mmer_bit(abm, cn)) ? cn : SENT;  // Sect. 2.2 filter
      V[L * stride + j] = (VT)v;
      pm = v < pm ? v : pm;
      P[L * stride + j] = (VT)pm;
    }
  }
  __syncthreads();
  // phase 2: window minima = signatures (lane 255 only lends prefix minima)
  if (L < SIG2_LANES - 1) {
    uint32_t sfx = 0xFFFFFFFFu;
    for (int j = w - 1; j >= 0; --j) {
      const uint32_t v = V[L * stride + j];
      sfx = v < sfx ? v : sfx;
      const uint32_t nx = j > 0 ? (uint32_t)P[(L + 1) * stride + j - 1] : 0xFFFFFFFFu;
      V[L * stride + j] = (VT)(sfx < nx ? sfx : nx);
    }
  }
  __syncthreads();
  // phase 3: validity, cut rule, breaks and owned starts of the lane's block.
  // Positions are local (lp = position - LBm).  A k-mer at lp is valid when
  // base lp is a base and the next "bad" position (invalid base or read
  // start) after lp is at least lp + k away; both masks stream out of
  // register words, and the next bad position is searched only once passed.
  uint64_t brk_mask = 0, start_mask = 0;
  if (L < SIG2_LANES - 1) {
    auto valid_at = [&](uint64_t lp) -> bool {  // direct test (one position)
      if ((iv[lp >> 6] >> (63 - (lp & 63))) & 1ull) return false;
      return k == 1 || get_bits(cm, lp + 1, k - 1) == 0ull;
    };
    const uint32_t lp0 = (uint32_t)(p0 - LBm);
    // lane 0's first position precedes the owned range: no start flag needed
    bool pv = false;
    uint32_t psig = 0;
    if (L > 0) {
      pv = valid_at(lp0 - 1);
      psig = V[(L - 1) * stride + (w - 1)];
    }
    // last read start strictly before lp0 (local; may be negative)
    int32_t rs;
    {
      const int wi = (int)(lp0 >> 6);
      const unsigned o = lp0 & 63;
      const uint64_t x = o ? (sm[wi] & (~0ull << (64 - o))) : 0ull;
      rs = x ? wi * 64 + 64 - __ffsll((long long)x) : (int32_t)(lastw[wi] - LBm);
    }
    // Bit-parallel over the lane's w positions, MSB first (bit 63 - j is
    // position lp0 + j).  valid: base j is a base and no bad position (an
    // invalid base or a read start) lies in (j, j + k): a sliding OR of
    // width k-1 over the 128-bit window of bad bits from lp0 + 1, built by
    // doubling.
    const uint64_t wmask = w >= 64 ? ~0ull : ~(~0ull >> w);  // the top w bits
    const uint64_t inv_b = get_bits(iv, lp0, 64);
    uint64_t valid = ~inv_b;
    if (k > 1) {
      uint64_t H = get_bits(cm, (uint64_t)lp0 + 1, 64), Lo = get_bits(cm, (uint64_t)lp0 + 65, 64);
      int width = 1;
      while (2 * width <= k - 1) {  // R[i] = OR of the window [i, i + 2 width)
        H |= (H << width) | (Lo >> (64 - width));
        Lo |= Lo << width;
        width *= 2;
      }
      const int rest = k - 1 - width;  // then [i, i + k - 1) = R[i] | R[i + rest]
      if (rest > 0) H |= (H << rest) | (Lo >> (64 - rest));
      valid &= ~H;
    }
    valid &= wmask;
    // cuts: every read start, and the multiples of kSuperkmerCap from the
    // read start before the window up to the first start in it
    const uint64_t starts = get_bits(sm, lp0, 64) & wmask;
    uint64_t cut = starts;
    {
      const uint32_t d = (uint32_t)((int32_t)lp0 - rs);
      const uint32_t c = (kSuperkmerCap - (d & (kSuperkmerCap - 1))) & (kSuperkmerCap - 1);
      const uint32_t f = starts ? (uint32_t)__clzll((long long)starts) : 64u;
      if (c < f && c < (uint32_t)w) cut |= 1ull << (63 - c);
    }
    // signature changes
    uint64_t chg = 0;
    {
      uint32_t prev = psig;
      for (int j = 0; j < w; ++j) {
        const uint32_t sg = V[L * stride + j];
        chg |= (uint64_t)(sg != prev) << (63 - j);
        prev = sg;
      }
    }
    const uint64_t prev_valid = (valid >> 1) | (pv ? 1ull << 63 : 0ull);
    const uint64_t st = valid & (~prev_valid | chg | cut);
    const uint64_t brk = (~valid | st) & wmask;
    // owned starts: local positions [own_lo, own_hi)
    const int32_t olo = (int32_t)(T0 - LBm) - (int32_t)lp0, ohi = olo + own;
    const int j0 = olo < 0 ? 0 : (olo > 64 ? 64 : olo), j1 = ohi < 0 ? 0 : (ohi > 64 ? 64 : ohi);
    const uint64_t own_m = (j1 > j0) ? ((j1 - j0 >= 64 ? ~0ull : ((1ull << (j1 - j0)) - 1)) << (64 - j1)) : 0ull;
    brk_mask = __brevll(brk);
    start_mask = __brevll(st & own_m);
  }
  fbrk[L] = brk_mask ? p0 + (__ffsll((long long)brk_mask) - 1) : INT64_MAX;
  __syncthreads();
  // phase 4: emit the owned super k-mers (each ends at the next break)
  const uint32_t ns = (uint32_t)__popcll(start_mask);
  uint32_t nst;
  uint32_t si = block_excl_scan<uint32_t, SIG2_LANES>(ns, ws, &nst);
  if (a.list) {
    if (L == 0) out_base = nst ? atomicAdd(a.n_list, (unsigned long long)nst) : 0ull;
    __syncthreads();
    if (out_base + nst > a.list_cap) {
      if (L == 0) atomicOr(a.err, ERR_CAPACITY);
      return;
    }
  }
  uint64_t bits = start_mask;
  while (bits) {
    const int j = __ffsll((long long)bits) - 1;
    bits &= bits - 1;
    const int64_t pos = p0 + j;
    // next break after j: in this block, else the first break of a later block
    const uint64_t after = j < 63 ? (brk_mask >> (j + 1)) << (j + 1) : 0ull;
    int64_t end;
    if (after) {
      end = p0 + (__ffsll((long long)after) - 1);
    } else {
      end = B0 + (int64_t)(SIG2_LANES - 1) * w;  // end of the covered positions
      for (int l2 = L + 1; l2 < SIG2_LANES - 1; ++l2) {
        const int64_t f = fbrk[l2];
        if (f != INT64_MAX) { end = f; break; }
      }
    }
    const uint32_t n = (uint32_t)(end - pos);
    const uint32_t g = V[L * stride + j];
    if (!a.list) {  // sample mode: signature weights
      atomicAdd(&a.sig_weight[g], (unsigned long long)n);
      continue;
    }
    a.list[out_base + si] = ((uint64_t)pos << 32) | ((uint64_t)(n - 1) << 25) | g;
    ++si;
    const uint32_t bin = slot_of(a.set_starts, a.n_slots, (uint64_t)pos) * a.bins_per_slot + a.map[g];
    const uint32_t nw = (2 * (n + k - 1) + 63) / 64;
    if (small_bins) {
      atomicAdd(&hpk[bin], 1ull | ((unsigned long long)nw << 21) | ((unsigned long long)n << 42));
    } else {
      atomicAdd(&a.bin_rec[bin], 1ull);
      atomicAdd(&a.bin_words[bin], (unsigned long long)nw);
      atomicAdd(&a.bin_kmers[bin], (unsigned long long)n);
    }
  }
  if (small_bins && a.list) {
    __syncthreads();
    for (int i = L; i < hb; i += SIG2_LANES) {
      const unsigned long long v = hpk[i];
      if (v) {
        atomicAdd(&a.bin_rec[i], v & 0x1FFFFFull);
        atomicAdd(&a.bin_words[i], (v >> 21) & 0x1FFFFFull);
        atomicAdd(&a.bin_kmers[i], v >> 42);
      }
    }
  }
}

// Raises the shared-memory limits of both signature kernels (once per
// device; must not run inside a graph capture).
inline cudaError_t sig_prepare() {
  static std::atomic<uint8_t> done[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && done[dev].load()) return cudaSuccess;
  e = cudaFuncSetAttribute(sig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(SigSmem));
  if (e != cudaSuccess) return e;
  const int s32 = (int)sig2_smem_bytes(SIG2_MAXW, 8, SIG_SMEM_BINS);
  const int s16 = (int)sig2_smem_bytes(SIG2_MAXW, 1, SIG_SMEM_BINS);
  if ((e = cudaFuncSetAttribute(sig2_kernel<uint32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32)) ||
      (e = cudaFuncSetAttribute(sig2_kernel<uint32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s32)) ||
      (e = cudaFuncSetAttribute(sig2_kernel<uint16_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, s16)) ||
      (e = cudaFuncSetAttribute(sig2_kernel<uint16_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, s16)))
    return e;
  if (dev < 64) done[dev].store(1);
  return cudaSuccess;
}

// Launches the signature scan over stream positions [0, n_stream) (the
// lane-block kernel unless `tile` asks for the tile-doubling one or the
// window is outside its range).  Returns the launches made (0 or 1).
inline int sig_launch(const SigArgs &a, uint64_t n_stream, bool tile, cudaStream_t st) {
  if (!tile && sig2_applies(a.k, a.m)) {
    const uint64_t own = (uint64_t)sig2_own(a.k, a.m);
    const uint64_t g = (n_stream + own - 1) / own;
    if (g == 0) return 0;
    const size_t sm = sig2_smem_bytes(a.k, a.m, a.n_bins);
    if (a.m <= 7) {
      if (a.no_filter) sig2_kernel<uint16_t, true><<<(unsigned)g, SIG2_LANES, sm, st>>>(a);
      else sig2_kernel<uint16_t, false><<<(unsigned)g, SIG2_LANES, sm, st>>>(a);
    } else {
      if (a.no_filter) sig2_kernel<uint32_t, true><<<(unsigned)g, SIG2_LANES, sm, st>>>(a);
      else sig2_kernel<uint32_t, false><<<(unsigned)g, SIG2_LANES, sm, st>>>(a);
    }
    return 1;
  }
  const uint64_t g = (n_stream + SIG_TPOS - 1) / SIG_TPOS;
  if (g == 0) return 0;
  sig_kernel<<<(unsigned)g, SIG_THREADS, sizeof(SigSmem), st>>>(a);
  return 1;
}

// ------------------------------------------------------------------ a3

// Per-CTA scratch of the bin scatter: the record table, the word slots and,
// after it, the per-bin counters and bases for hb bins (hb = n_bins when
// n_bins <= SIG_SMEM_BINS, else 0).
constexpr int SCAT_WCAP = SCAT_PER_CTA * 5;  // word slots (records of up to 5 words on average)
struct ScatSmem {
  unsigned long long wi[SCAT_PER_CTA];   // first destination word of each record
  uint32_t pos[SCAT_PER_CTA];            // stream position of each record
  uint32_t wofs[SCAT_PER_CTA];           // first word slot of each record (nw before the scan)
  uint16_t nbits[SCAT_PER_CTA];          // bits of each record
  uint16_t wrec[SCAT_WCAP];              // record of each word slot
  uint32_t ws[SCAT_THREADS / 32 + 1];
};
inline size_t scat_smem_bytes(uint32_t n_bins) {
  const size_t hb = n_bins <= (uint32_t)SIG_SMEM_BINS ? n_bins : 0;
  return ((sizeof(ScatSmem) + 15) & ~(size_t)15) + hb * 24;
}

// Scatters super k-mer records into their bins: an index entry (word
// offset | n_kmers-1 | signature) and the packed bases (Sect. 2.4: super
// k-mers are sent to bins).  Space is reserved per CTA and bin with one
// global atomic per non-empty bin (per record when there are many bins).
// The bases are copied one word per thread over the CTA's word slots in
// record order, so that neighbouring threads read neighbouring words and
// all loads of a thread are independent.
__global__ void __launch_bounds__(SCAT_THREADS)
scatter_kernel(const uint64_t *__restrict__ list, uint64_t n_list, const uint32_t *__restrict__ map,
               uint32_t n_bins, int k, const uint64_t *__restrict__ packed,
               unsigned long long *rec_cursor, unsigned long long *word_cursor,
               uint64_t *__restrict__ index, uint64_t *__restrict__ words,
               const unsigned long long *n_list_dyn = nullptr, const uint64_t *set_starts = nullptr,
               uint32_t n_slots = 0, uint32_t bins_per_slot = 0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatSmem &s = *reinterpret_cast<ScatSmem *>(smem_raw);
  const bool small_bins = n_bins <= (uint32_t)SIG_SMEM_BINS;
  const uint32_t hb = small_bins ? n_bins : 0u;
  uint32_t *c_rec = reinterpret_cast<uint32_t *>(smem_raw + ((sizeof(ScatSmem) + 15) & ~(size_t)15));
  uint32_t *c_words = c_rec + hb;
  unsigned long long *b_rec = reinterpret_cast<unsigned long long *>(c_words + hb);  // 8-byte aligned
  unsigned long long *b_words = b_rec + hb;
  const uint64_t c0 = (uint64_t)blockIdx.x * SCAT_PER_CTA;
  if (n_list_dyn) {
    n_list = *n_list_dyn;
    if (c0 >= n_list) return;
  }
  const uint32_t n_here = (uint32_t)(n_list - c0 < (uint64_t)SCAT_PER_CTA ? n_list - c0 : (uint64_t)SCAT_PER_CTA);
  constexpr int PER = SCAT_PER_CTA / SCAT_THREADS;
  const int tid = threadIdx.x;
  uint64_t rec[PER];
  uint32_t bin[PER], nw[PER];
  for (uint32_t i = tid; i < hb; i += SCAT_THREADS) c_rec[i] = c_words[i] = 0;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const uint32_t e = (uint32_t)q * SCAT_THREADS + tid;
    rec[q] = e < n_here ? list[c0 + e] : ~0ull;
    nw[q] = 0;
    if (e < n_here) {
      const uint32_t n = (uint32_t)((rec[q] >> 25) & 127u) + 1;
      bin[q] = slot_of(set_starts, n_slots, rec[q] >> 32) * bins_per_slot + map[rec[q] & 0x1FFFFFFu];
      nw[q] = (2 * (n + k - 1) + 63) / 64;
      if (small_bins) {
        atomicAdd(&c_rec[bin[q]], 1u);
        atomicAdd(&c_words[bin[q]], nw[q]);
      }
    }
  }
  if (small_bins) {
    __syncthreads();
    for (uint32_t i = tid; i < hb; i += SCAT_THREADS) {
      if (c_rec[i]) {
        b_rec[i] = atomicAdd(&rec_cursor[i], (unsigned long long)c_rec[i]);
        b_words[i] = atomicAdd(&word_cursor[i], (unsigned long long)c_words[i]);
      }
      c_rec[i] = 0;
      c_words[i] = 0;
    }
    __syncthreads();
  }
  // index entries, and the record table for the word copy
#pragma unroll
  for (int q = 0; q < PER; ++q) {
    const uint32_t e = (uint32_t)q * SCAT_THREADS + tid;
    if (e >= n_here) continue;
    uint64_t ri, wi;
    if (small_bins) {
      ri = b_rec[bin[q]] + atomicAdd(&c_rec[bin[q]], 1u);
      wi = b_words[bin[q]] + atomicAdd(&c_words[bin[q]], nw[q]);
    } else {
      ri = atomicAdd(&rec_cursor[bin[q]], 1ull);
      wi = atomicAdd(&word_cursor[bin[q]], (unsigned long long)nw[q]);
    }
    const uint32_t n = (uint32_t)((rec[q] >> 25) & 127u) + 1;
    index[ri] = (wi << 32) | (rec[q] & 0xFFFFFFFFull);
    s.wi[e] = wi;
    s.pos[e] = (uint32_t)(rec[q] >> 32);
    s.nbits[e] = (uint16_t)(2 * (n + k - 1));
    s.wofs[e] = nw[q];
  }
  __syncthreads();
  // word slots: exclusive scan of the records' word counts in record order
  // (thread t scans records PER t .. PER t + PER - 1)
  uint32_t W;
  {
    uint32_t c[PER], sum = 0;
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const uint32_t e = (uint32_t)PER * tid + j;
      c[j] = e < n_here ? s.wofs[e] : 0u;
      sum += c[j];
    }
    uint32_t run = block_excl_scan<uint32_t, SCAT_THREADS>(sum, s.ws, &W);
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const uint32_t e = (uint32_t)PER * tid + j;
      if (e < n_here) s.wofs[e] = run;
      run += c[j];
    }
  }
  __syncthreads();
  if (W <= (uint32_t)SCAT_WCAP) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const uint32_t e = (uint32_t)q * SCAT_THREADS + tid;
      if (e < n_here)
        for (uint32_t j = 0; j < nw[q]; ++j) s.wrec[s.wofs[e] + j] = (uint16_t)e;
    }
    __syncthreads();
#pragma unroll 4
    for (uint32_t i = tid; i < W; i += SCAT_THREADS) {
      const uint32_t e = s.wrec[i];
      const uint32_t j = i - s.wofs[e];
      uint64_t v = get_bits(packed, 2ull * s.pos[e] + 64ull * j, 64);
      const uint32_t used = (uint32_t)s.nbits[e] - 64 * j;
      if (used < 64) v &= ~0ull << (64 - used);
      words[s.wi[e] + j] = v;
    }
  } else {
    // more words than slots: each thread copies its own records
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const uint32_t e = (uint32_t)q * SCAT_THREADS + tid;
      if (e >= n_here) continue;
      const uint64_t wi = s.wi[e];
      const uint32_t nbits = s.nbits[e];
      for (uint32_t j = 0; j < nw[q]; ++j) {
        uint64_t v = get_bits(packed, 2ull * s.pos[e] + 64ull * j, 64);
        const uint32_t used = nbits - 64 * j;
        if (used < 64) v &= ~0ull << (64 - used);
        words[wi + j] = v;
      }
    }
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

// The same map without a sort, for up to MAP_DIRECT_MAX signatures (m <= 7:
// 4^m m-mers and the sentinel): the
// weight preceding signature s in the order above is summed directly,
// W(s) = sum of w(t) over the t with w(t) > w(s), or w(t) = w(s) and t < s
// (weights clamped to 32 bits as in the sort key).  CTA (x, y) takes
// signatures [256x, 256x + 256) against the y-th slice of all signatures.
constexpr uint32_t MAP_DIRECT_MAX = (1u << 14) + 1u;
constexpr int MAP_DIRECT_SLICES = 16;
__global__ void __launch_bounds__(256) map_prefix_kernel(const unsigned long long *__restrict__ w, uint32_t n_sig,
                                                         unsigned long long *__restrict__ before,
                                                         unsigned long long *__restrict__ total) {
  __shared__ uint32_t ws[1024];
  const uint32_t sg = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t my = sg < n_sig ? (uint32_t)min(w[sg], 0xFFFFFFFFull) : 0u;
  const uint32_t per = (n_sig + gridDim.y - 1) / gridDim.y;
  const uint32_t t0 = blockIdx.y * per, t1 = min(t0 + per, n_sig);
  unsigned long long acc = 0;
  for (uint32_t c = t0; c < t1; c += 1024) {
    const uint32_t m = min(1024u, t1 - c);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) ws[i] = (uint32_t)min(w[c + i], 0xFFFFFFFFull);
    __syncthreads();
    for (uint32_t j = 0; j < m; ++j) {
      const uint32_t x = ws[j];
      if (x > my || (x == my && c + j < sg)) acc += x;
    }
  }
  if (sg < n_sig && my) {
    if (acc) atomicAdd(&before[sg], acc);
    if (blockIdx.y == 0) atomicAdd(total, (unsigned long long)my);
  }
}
__global__ void map_direct_assign_kernel(const unsigned long long *w, const unsigned long long *before,
                                         const unsigned long long *total, uint32_t n_sig, uint32_t n_bins,
                                         uint32_t *map) {
  const uint64_t tot = *total;
  for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_sig; s += gridDim.x * blockDim.x)
    map[s] = (w[s] == 0 || tot == 0) ? s % n_bins : (uint32_t)((before[s] * n_bins) / tot);
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

}  // namespace
}  // namespace kmc
