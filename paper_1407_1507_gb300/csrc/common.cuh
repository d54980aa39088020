// Device helpers shared by the kernels of the GB300 k-mer counter.
//
// Bit streams.  Bases are 2-bit codes A=0 C=1 G=2 T=3 (paper Suppl. S4
// [map]); a sequence is packed MSB-first into 64-bit words: base i sits in
// bits [63-2(i%32), 62-2(i%32)] of word i/32, so a number read out of the
// stream has its first symbol most significant, as in the paper's coding.
// One-bit masks (invalid base, read start) use the same MSB-first layout.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kmc {

typedef unsigned __int128 u128;

// Device-side error word bits (set with atomicOr, read by the host).
enum : uint32_t {
  ERR_OVERFLOW = 1u << 0,   // a count above UINT32_MAX inside the cutoffs
  ERR_INPUT = 1u << 1,      // malformed offsets
  ERR_CAPACITY = 1u << 2,   // an internal buffer bound was exceeded
  ERR_TIMEOUT = 1u << 3,    // a bounded device-side wait gave up
};

constexpr int kSuperkmerCap = 128;  // max k-mers per super k-mer record
constexpr unsigned FULL = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned r;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
  return r;
}

// nbits (1..64) bits of an MSB-first bit stream starting at bit `pos`,
// right-aligned.  Reads words pos/64 and pos/64+1.
__device__ __forceinline__ uint64_t get_bits(const uint64_t *w, uint64_t pos, int nbits) {
  uint64_t i = pos >> 6;
  unsigned s = (unsigned)(pos & 63);
  uint64_t hi = w[i];
  uint64_t v = hi << s;
  if (s) v |= w[i + 1] >> (64 - s);
  return nbits == 64 ? v : (v >> (64 - nbits));
}

// Reverse complement of an m-mer held in the low 2m bits (m <= 16):
// complement every 2-bit code (3 - c, i.e. bitwise not) and reverse the
// order of the codes.
__device__ __forceinline__ uint32_t revcomp32(uint32_t v, int m) {
  uint32_t x = __brev(~v);                                       // codes reversed, bits swapped
  x = ((x >> 1) & 0x55555555u) | ((x & 0x55555555u) << 1);      // swap bits back inside codes
  return x >> (32 - 2 * m);
}

// Reverse complement of a k-mer in the low 2k bits (k <= 32).
__device__ __forceinline__ uint64_t revcomp64(uint64_t v, int k) {
  uint64_t x = __brevll(~v);
  x = ((x >> 1) & 0x5555555555555555ull) | ((x & 0x5555555555555555ull) << 1);
  return x >> (64 - 2 * k);
}

// 2k-bit value (k <= 64) of the k symbols starting at symbol index `sym`
// of a packed 2-bit stream.
template <typename K>
__device__ __forceinline__ K get_kmer(const uint64_t *w, uint64_t sym, int k);
template <>
__device__ __forceinline__ uint64_t get_kmer<uint64_t>(const uint64_t *w, uint64_t sym, int k) {
  return get_bits(w, 2 * sym, 2 * k);
}
template <>
__device__ __forceinline__ unsigned __int128 get_kmer<unsigned __int128>(const uint64_t *w,
                                                                         uint64_t sym, int k) {
  if (k <= 32) return get_bits(w, 2 * sym, 2 * k);
  uint64_t hi = get_bits(w, 2 * sym, 64);
  uint64_t lo = get_bits(w, 2 * sym + 64, 2 * k - 64);
  return ((unsigned __int128)hi << (2 * k - 64)) | lo;
}

// Reverse complement of a k-mer in the low 2k bits (k <= 64).
__device__ __forceinline__ u128 revcomp128(u128 v, int k) {
  uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
  // reverse the full 128-bit value: new_hi = rev(lo), new_lo = rev(hi)
  uint64_t nh = __brevll(~lo), nl = __brevll(~hi);
  nh = ((nh >> 1) & 0x5555555555555555ull) | ((nh & 0x5555555555555555ull) << 1);
  nl = ((nl >> 1) & 0x5555555555555555ull) | ((nl & 0x5555555555555555ull) << 1);
  u128 x = ((u128)nh << 64) | nl;
  return x >> (128 - 2 * k);
}

// Sect. 2.2 signature rule on a canonical m-mer c (low 2m bits): allowed
// unless it starts with AAA, starts with ACA, or has AA at a position >= 1.
__device__ __forceinline__ bool mmer_allowed(uint32_t c, int m) {
  if (m >= 3) {
    uint32_t top3 = (c >> (2 * m - 6)) & 63u;
    if (top3 == 0u || top3 == 4u) return false;  // AAA.., ACA..
    // isA: bit 2j set when the code in slot j (from the low end) is A (00).
    uint32_t a = ~(c | (c >> 1)) & 0x55555555u & ((1u << (2 * m)) - 1u);
    uint32_t aa = a & (a >> 2);                  // slots j and j+1 both A
    // slot pair (j, j+1) is the symbol pair starting at index m-2-j; index >= 1
    // means j <= m-3, i.e. bits below 2(m-2).
    if (aa & ((1u << (2 * (m - 2))) - 1u)) return false;
  }
  return true;
}

// Key traits: W-bit keys (64 or 128).
template <typename K> struct KeyTraits;
template <> struct KeyTraits<uint64_t> {
  static constexpr int BITS = 64;
  __device__ __forceinline__ static uint64_t max_key() { return ~0ull; }
  __device__ __forceinline__ static unsigned digit(uint64_t k, int bit, int nbits) {
    return (unsigned)(k >> bit) & ((1u << nbits) - 1u);
  }
};
template <> struct KeyTraits<u128> {
  static constexpr int BITS = 128;
  __device__ __forceinline__ static u128 max_key() { return ~(u128)0; }
  __device__ __forceinline__ static unsigned digit(u128 k, int bit, int nbits) {
    return (unsigned)(uint64_t)(k >> bit) & ((1u << nbits) - 1u);
  }
};

// Top `nbits` bits of a key with `sig_bits` significant low bits.
template <typename K>
__device__ __forceinline__ uint32_t top_digit(K key, int sig_bits, int nbits) {
  if (nbits == 0) return 0;
  return (uint32_t)(uint64_t)(key >> (sig_bits - nbits));
}

// ------------------------------------------------ bulk copies (TMA engine)
// One-dimensional global -> shared copies by the tensor memory accelerator,
// completed on an mbarrier (transaction count in bytes).  Addresses and the
// size must be multiples of 16 bytes.

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Orders this thread's earlier shared-memory accesses before later
// async-proxy (bulk copy) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Arrives on the barrier and announces `bytes` of copies completing on it,
// then starts the copy of `bytes` from global `src` to shared `dst`.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Waits until the barrier's phase with the given parity has completed;
// gives up after about `limit_ns` nanoseconds and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          uint64_t limit_ns = 1000000000ull) {
  const uint32_t a = smem_addr(bar);
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (it == 0) t0 = global_ns();
    else if (global_ns() - t0 > limit_ns) return false;
  }
}

}  // namespace kmc

namespace kmc {
// Kernels launched by this thread (host side); every launch site bumps it.
extern thread_local uint64_t g_launches;
}
#define KMC_COUNT_LAUNCH() (++::kmc::g_launches)

#define KMC_CUDA_TRY(expr)                                      \
  do {                                                          \
    cudaError_t _e = (expr);                                    \
    if (_e != cudaSuccess) return ::kmc::cuda_fail(_e, #expr);  \
  } while (0)
