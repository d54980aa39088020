// Allocation-free counting of a small read set (kmc_count_small_noalloc).
//
// This is a variant of the oversized-bucket kernel (big_count_kernel): one
// CTA sorts keys through global-memory scratch with LSD passes and
// run-length counts them.  Here the scratch is not allocated per call but is
// a fixed array in the library's device image, so a call allocates nothing.
// The same CTA also extracts the canonical k-mers of the reads first.
#include <mutex>

#include "internal.h"
#include "sortlib.cuh"

namespace kmc {

namespace {

constexpr uint64_t kNoAllocMaxBases = KMC_NOALLOC_MAX_BASES;
constexpr int NA_THREADS = 1024;
constexpr int NA_IPT = 4;

// Two key buffers (sort ping-pong) of kNoAllocMaxBases keys each.  Every
// GPU that loads the library holds this array (16 MiB) until the process
// exits.  All calls share it; it keeps the last call's contents.
static __device__ __align__(256) unsigned long long g_noalloc_scratch[2 * kNoAllocMaxBases];

struct NaSmem {
  BigSmem<uint64_t, NoVal, NA_THREADS, NA_IPT> big;
  unsigned long long n_keys;
  unsigned long long out_base;
  uint32_t bad;
};

// One CTA: (1) every thread walks whole reads and appends the canonical
// k-mer of every valid window to scratch A; (2) LSD radix sort of the keys
// on their 2k bits (scratch A <-> B); (3) run-length count with the
// inclusive cutoffs, written in ascending k-mer order.  *n_out receives the
// number of k-mers in the result (entries beyond `capacity` are not
// written), or UINT64_MAX if the offsets are malformed.
__global__ void __launch_bounds__(NA_THREADS)
count_small_kernel(const uint8_t *__restrict__ bases, const uint64_t *__restrict__ offsets,
                   uint64_t n_reads, uint64_t n_bases, int k, uint64_t ci, uint64_t cx,
                   unsigned long long *scratch, uint64_t *out_kmers, uint32_t *out_counts,
                   uint64_t capacity, uint64_t *n_out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  NaSmem &sm = *reinterpret_cast<NaSmem *>(smem_raw);
  constexpr int CH = NA_THREADS * NA_IPT;
  uint64_t *A = reinterpret_cast<uint64_t *>(scratch);
  uint64_t *B = A + kNoAllocMaxBases;
  if (threadIdx.x == 0) {
    sm.n_keys = 0;  // the scratch keeps old contents: only this counter must restart
    sm.out_base = 0;
    sm.bad = (offsets[0] != 0 || offsets[n_reads] != n_bases) ? 1u : 0u;
  }
  __syncthreads();
  // (1) canonical k-mers (rolling forward and reverse-complement values)
  const uint64_t kmask = k == 32 ? ~0ull : ((1ull << (2 * k)) - 1);
  const volatile uint32_t &bad = sm.bad;  // other threads may set it: read it afresh
  for (uint64_t r = threadIdx.x; r < n_reads && !bad; r += NA_THREADS) {
    const uint64_t a = offsets[r], e = offsets[r + 1];
    if (e < a || e > n_bases) { sm.bad = 1; break; }
    uint64_t fw = 0, rc = 0;
    int run = 0;
    for (uint64_t i = a; i < e; ++i) {
      const unsigned c = bases[i];
      unsigned code;
      if (c == 'A') code = 0; else if (c == 'C') code = 1; else if (c == 'G') code = 2;
      else if (c == 'T') code = 3; else { run = 0; continue; }
      fw = ((fw << 2) | code) & kmask;
      rc = (rc >> 2) | ((uint64_t)(3u - code) << (2 * k - 2));
      if (++run >= k) {
        const unsigned long long slot = atomicAdd(&sm.n_keys, 1ull);
        if (slot < n_bases) A[slot] = fw < rc ? fw : rc;  // n_bases <= kNoAllocMaxBases
        else sm.bad = 1;  // only malformed (overlapping) offsets get here
      }
    }
  }
  __syncthreads();
  if (sm.bad) {
    if (threadIdx.x == 0) *n_out = ~0ull;
    return;
  }
  const uint64_t n = sm.n_keys;
  // (2) sort: LSD over the 2k value bits, so the result is in value order
  const bool in_b = big_sort<uint64_t, NoVal, NA_THREADS, NA_IPT>(A, (NoVal *)nullptr, B,
                                                                 (NoVal *)nullptr, n, 2 * k, sm.big);
  const uint64_t *s = in_b ? B : A;
  // (3) run-length count, chunk by chunk, carrying the run open at a chunk end
  uint64_t open = 0;
  for (uint64_t c0 = 0; c0 < n; c0 += CH) {
    uint32_t nh = 0;
    const uint64_t e0 = c0 + (uint64_t)threadIdx.x * NA_IPT;
    for (int j = 0; j < NA_IPT; ++j) {
      const uint64_t e = e0 + j;
      if (e < n && e > 0 && s[e] != s[e - 1]) ++nh;
    }
    uint32_t tot;
    uint32_t hb = block_excl_scan<uint32_t, NA_THREADS>(nh, sm.big.ws, &tot);
    for (int j = 0; j < NA_IPT; ++j) {
      const uint64_t e = e0 + j;
      if (e < n && e > 0 && s[e] != s[e - 1]) sm.big.pos[hb++] = (uint32_t)(e - c0);
    }
    __syncthreads();
    const bool last = c0 + CH >= n;
    const uint32_t nclosed = tot + (last ? 1u : 0u);
    const uint32_t Q = (nclosed + NA_THREADS - 1) / NA_THREADS;
    const uint32_t r0 = threadIdx.x * Q;
    uint32_t keep = 0;
    for (uint32_t j = 0; j < Q; ++j) {
      const uint32_t r = r0 + j;
      if (r < nclosed) {
        const uint64_t rs = r == 0 ? open : c0 + sm.big.pos[r - 1];
        const uint64_t re = r < tot ? c0 + sm.big.pos[r] : n;
        keep += (re - rs >= ci && re - rs <= cx);
      }
    }
    uint32_t ktot;
    uint32_t kb = block_excl_scan<uint32_t, NA_THREADS>(keep, sm.big.ws, &ktot);
    const uint64_t base = sm.out_base;
    for (uint32_t j = 0; j < Q; ++j) {
      const uint32_t r = r0 + j;
      if (r < nclosed) {
        const uint64_t rs = r == 0 ? open : c0 + sm.big.pos[r - 1];
        const uint64_t re = r < tot ? c0 + sm.big.pos[r] : n;
        if (re - rs >= ci && re - rs <= cx) {
          if (base + kb < capacity) {
            out_kmers[base + kb] = s[rs];
            out_counts[base + kb] = (uint32_t)(re - rs);
          }
          ++kb;
        }
      }
    }
    if (tot) open = c0 + sm.big.pos[tot - 1];
    __syncthreads();
    if (threadIdx.x == 0) sm.out_base = base + ktot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *n_out = sm.out_base;
}

// Device address of the scratch array, looked up once per device.
std::mutex g_na_mu;
void *g_na_ptr[256];
bool g_na_attr[256];

}  // namespace

}  // namespace kmc

extern "C" int kmc_count_small_noalloc(const char *d_bases, const uint64_t *d_offsets,
                                       uint64_t n_reads, uint64_t n_bases, uint32_t k,
                                       uint64_t cutoff_min, uint64_t cutoff_max,
                                       uint64_t *d_kmers, uint32_t *d_counts, uint64_t capacity,
                                       uint64_t *d_n_out, void *cuda_stream) {
  using namespace kmc;
  if (k < 1 || k > 32 || cutoff_min > cutoff_max || !d_offsets || !d_n_out ||
      (n_bases && !d_bases) || (capacity && (!d_kmers || !d_counts)))
    return KMC_EINVAL;
  if (n_bases > kNoAllocMaxBases) return KMC_EINVAL;  // beyond the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return KMC_ECUDA;
  void *ptr = nullptr;
  {
    std::lock_guard<std::mutex> g(g_na_mu);
    if (!g_na_ptr[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_na_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_na_ptr[dev] = nullptr;
        return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
      }
    }
    if (!g_na_attr[dev]) {
      cudaError_t e = cudaFuncSetAttribute(count_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)sizeof(NaSmem));
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(count_small_kernel)");
      g_na_attr[dev] = true;
    }
    ptr = g_na_ptr[dev];
  }
  // A k-mer in the result has count >= 1, so cutoff_min 0 keeps the same
  // k-mers as cutoff_min 1.
  const uint64_t ci = cutoff_min ? cutoff_min : 1;
  // An error left pending by earlier, unrelated work of this thread would
  // otherwise be read back below as this launch's failure: report it as
  // such, leave it pending for its owner, and launch nothing.
  cudaError_t pending = cudaPeekAtLastError();
  if (pending != cudaSuccess) return cuda_fail(pending, "error pending before count_small_kernel");
  count_small_kernel<<<1, NA_THREADS, sizeof(NaSmem), static_cast<cudaStream_t>(cuda_stream)>>>(
      reinterpret_cast<const uint8_t *>(d_bases), d_offsets, n_reads, n_bases, (int)k, ci,
      cutoff_max, static_cast<unsigned long long *>(ptr), d_kmers, d_counts, capacity, d_n_out);
  KMC_COUNT_LAUNCH();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "count_small_kernel launch");
  return KMC_OK;
}
