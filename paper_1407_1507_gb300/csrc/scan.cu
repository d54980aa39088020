// Device-wide exclusive scan (three phases: block sums, scan of the sums,
// block rescan; no inter-block waiting) and the tile planner of the sort.
#include "sortlib.cuh"

namespace kmc {

namespace {
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_IPT = 16;
constexpr uint64_t SCAN_BLOCK = (uint64_t)SCAN_THREADS * SCAN_IPT;

template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS)
scan_reduce_kernel(const T *in, uint64_t n, uint64_t *block_sums) {
  __shared__ uint64_t ws[SCAN_THREADS / 32 + 1];
  const uint64_t b0 = (uint64_t)blockIdx.x * SCAN_BLOCK;
  uint64_t s = 0;
  for (int j = 0; j < SCAN_IPT; ++j) {
    uint64_t i = b0 + (uint64_t)j * SCAN_THREADS + threadIdx.x;
    if (i < n) s += (uint64_t)in[i];
  }
  uint64_t tot;
  (void)block_excl_scan<uint64_t, SCAN_THREADS>(s, ws, &tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// out[i] = base[block] + exclusive prefix inside the block; out[n] = total
// (written by the block holding element n-1, or block 0 when n == 0).
template <typename T>
__global__ void __launch_bounds__(SCAN_THREADS)
scan_apply_kernel(const T *in, uint64_t n, const uint64_t *block_base, uint64_t *out) {
  __shared__ uint64_t ws[SCAN_THREADS / 32 + 1];
  const uint64_t b0 = (uint64_t)blockIdx.x * SCAN_BLOCK;
  const uint64_t t0 = b0 + (uint64_t)threadIdx.x * SCAN_IPT;  // blocked: thread owns IPT items
  uint64_t v[SCAN_IPT];
  uint64_t s = 0;
#pragma unroll
  for (int j = 0; j < SCAN_IPT; ++j) {
    uint64_t i = t0 + j;
    v[j] = i < n ? (uint64_t)in[i] : 0;
    s += v[j];
  }
  uint64_t tot;
  uint64_t pre = block_excl_scan<uint64_t, SCAN_THREADS>(s, ws, &tot) +
                 (block_base ? block_base[blockIdx.x] : 0);
#pragma unroll
  for (int j = 0; j < SCAN_IPT; ++j) {
    uint64_t i = t0 + j;
    if (i < n) out[i] = pre;
    pre += v[j];
  }
  const uint64_t last_block = n ? (n - 1) / SCAN_BLOCK : 0;
  if (blockIdx.x == last_block && threadIdx.x == SCAN_THREADS - 1) out[n] = pre;
}

template <typename T>
cudaError_t excl_scan(const T *in, uint64_t *out, uint64_t n, uint64_t *tmp, cudaStream_t st) {
  const uint64_t nb = n ? (n + SCAN_BLOCK - 1) / SCAN_BLOCK : 1;
  if (nb == 1) {
    scan_apply_kernel<T><<<1, SCAN_THREADS, 0, st>>>(in, n, nullptr, out); KMC_COUNT_LAUNCH();
    return cudaGetLastError();
  }
  uint64_t *sums = tmp;             // nb
  uint64_t *sums_scan = tmp + nb;   // nb + 1
  uint64_t *rest = tmp + 2 * nb + 1;
  scan_reduce_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, sums); KMC_COUNT_LAUNCH();
  cudaError_t e = excl_scan<uint64_t>(sums, sums_scan, nb, rest, st);
  if (e != cudaSuccess) return e;
  scan_apply_kernel<T><<<(unsigned)nb, SCAN_THREADS, 0, st>>>(in, n, sums_scan, out); KMC_COUNT_LAUNCH();
  return cudaGetLastError();
}
}  // namespace

size_t scan_tmp_words(uint64_t n) {
  size_t w = 0;
  uint64_t nb = n ? (n + SCAN_BLOCK - 1) / SCAN_BLOCK : 1;
  while (nb > 1) {
    w += 2 * nb + 1;
    nb = (nb + SCAN_BLOCK - 1) / SCAN_BLOCK;
  }
  return w + 2;
}

cudaError_t device_excl_scan_u32(const uint32_t *in, uint64_t *out, uint64_t n, uint64_t *tmp,
                                 cudaStream_t st) {
  return excl_scan<uint32_t>(in, out, n, tmp, st);
}
cudaError_t device_excl_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, uint64_t *tmp,
                                 cudaStream_t st) {
  return excl_scan<uint64_t>(in, out, n, tmp, st);
}

// Tile rule over the buckets of one group (digit d, count c[d], in-group
// exclusive prefix P[d], half = tile_cap/2): a tile starts at d when d == 0,
// when c[d] > half or c[d-1] > half, or when floor(P[d]/half) differs from
// floor(P[d-1]/half).  Between two starts every bucket has the same
// floor(P/half) and holds at most `half` keys, so a tile of several buckets
// holds fewer than tile_cap keys; a bucket above `half` is a tile alone.
__global__ void plan_flags_kernel(const uint32_t *cnt, const uint64_t *base, uint64_t nbk,
                                  const uint32_t *group_base, uint32_t n_groups,
                                  uint32_t tile_cap, uint32_t *flag) {
  const uint64_t half = tile_cap / 2;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nbk;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t d = (uint32_t)i - group_base[group_of(group_base, n_groups, (uint32_t)i)];
    uint32_t f = 1;
    if (d != 0) {
      const uint64_t g0 = base[i - d];
      const uint64_t P = base[i] - g0, Pp = base[i - 1] - g0;
      f = (cnt[i] > half) || (cnt[i - 1] > half) || (P / half != Pp / half);
    }
    flag[i] = f;
  }
}

// Greedy variant: consecutive buckets join the current tile while it stays
// within tile_cap keys; a bucket that does not fit starts a new tile (a
// bucket above tile_cap is a tile alone).  Tiles come out nearly full,
// which the parallel rule above cannot promise.  The flattened buckets are
// cut into segments of kGreedySegment; a tile also starts at every segment
// start and every group start, so each segment is planned by one warp on
// its own (a huge bin does not serialise the plan).  The warp loads 32
// counts at a time and every lane replays the same sequential decision over
// them (shuffles), so the loop stays coalesced and uniform.
__global__ void plan_greedy_flags_kernel(const uint32_t *__restrict__ cnt,
                                         const uint32_t *__restrict__ group_base,
                                         uint32_t n_groups, uint64_t nbk, uint32_t tile_cap,
                                         uint32_t *__restrict__ flag) {
  const uint64_t seg = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t i0 = seg * kGreedySegment;
  if (i0 >= nbk) return;  // whole warps leave together
  const uint64_t i1 = i0 + kGreedySegment < nbk ? i0 + kGreedySegment : nbk;
  uint64_t acc = 0;
  for (uint64_t base = i0; base < i1; base += 32) {
    const uint64_t i = base + lane;
    uint32_t c = 0;
    bool gstart = false;
    if (i < i1) {
      c = cnt[i];
      gstart = group_base[group_of(group_base, n_groups, (uint32_t)i)] == (uint32_t)i;
    }
    const unsigned gmask = __ballot_sync(0xFFFFFFFFu, gstart);
    uint32_t mask = 0;
    const uint32_t lim = i1 - base < 32 ? (uint32_t)(i1 - base) : 32u;
    for (uint32_t j = 0; j < 32; ++j) {
      const uint32_t cj = __shfl_sync(0xFFFFFFFFu, c, j);
      if (j < lim) {
        const bool start = (base + j == i0) || ((gmask >> j) & 1u) || acc + cj > tile_cap;
        if (start) { mask |= 1u << j; acc = cj; } else { acc += cj; }
      }
    }
    if (i < i1) flag[i] = (mask >> lane) & 1u;
  }
}

__global__ void plan_emit_kernel(const uint32_t *flag, const uint64_t *flag_scan, uint64_t nbk,
                                 uint32_t *tile_first, uint32_t *n_tiles) {
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nbk;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (flag[i]) tile_first[flag_scan[i]] = (uint32_t)i;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) *n_tiles = (uint32_t)flag_scan[nbk];
}

}  // namespace kmc
