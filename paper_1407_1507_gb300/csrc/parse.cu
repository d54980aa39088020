// FASTQ / FASTA input read on the device (Sect. 2.4: the reads come from
// FASTQ or FASTA files; Suppl. S1 -fq / -fa / -fm).  The raw file bytes are
// in device memory; the kernels find its lines and write the reads' bases,
// contiguous, with their offsets, which then go through the device-input
// distribution path unchanged.
//
// Line structure needs global positions: the line index of a byte is the
// number of newlines before it.  Every pass works on chunks of
// PARSE_THREADS x PARSE_SEG bytes (a thread takes PARSE_SEG consecutive
// bytes); per-chunk counts are scanned on the device between passes.
//   A: newlines (and FASTA header-line starts) per chunk.
//   B (FASTA): for every line start, whether the line is a header ('>'),
//      stored per line index, so that any byte can tell its line's kind.
//   C: bytes kept per chunk, and the format checks.
//   D: the kept bytes written at their scanned places; each read's offset
//      written where its sequence starts.
// Kept bytes: FASTQ, the bytes of line 4r+1 (read r); FASTA, the bytes of
// non-header lines (record r = the r-th header); never '\n', nor a '\r'
// that ends a line.
#include "internal.h"
#include "sortlib.cuh"

namespace kmc {
namespace {

constexpr int PARSE_THREADS = 256;
constexpr int PARSE_SEG = 64;
constexpr uint64_t PARSE_CHUNK = (uint64_t)PARSE_THREADS * PARSE_SEG;

struct ParseArgs {
  const uint8_t *raw;
  uint64_t n;
  uint32_t fastq;                  // 1: FASTQ, 0: FASTA
  uint32_t *nl_cnt, *hs_cnt, *kept_cnt;           // per chunk
  const uint64_t *nl_base, *hs_base, *kept_base;  // their exclusive scans
  uint8_t *hdr;                    // FASTA: per line, 1 when it is a header
  uint8_t *out;                    // kept bytes
  uint64_t *offsets;               // read starts in `out`
  uint32_t *err;
};

// Bytes [s, s + PARSE_SEG) of the raw file (zero past the end).
__device__ __forceinline__ void load_seg(const ParseArgs &a, uint64_t s, uint8_t (&b)[PARSE_SEG]) {
  if (s + PARSE_SEG <= a.n && ((uintptr_t)(a.raw + s) & 15u) == 0) {
#pragma unroll
    for (int q = 0; q < PARSE_SEG / 16; ++q) {
      const uint4 v = *reinterpret_cast<const uint4 *>(a.raw + s + 16 * q);
      memcpy(b + 16 * q, &v, 16);
    }
  } else {
#pragma unroll
    for (int j = 0; j < PARSE_SEG; ++j) b[j] = s + j < a.n ? a.raw[s + j] : 0;
  }
}

template <int PASS>
__global__ void __launch_bounds__(PARSE_THREADS) parse_kernel(ParseArgs a) {
  __shared__ uint64_t ws64[PARSE_THREADS / 32 + 1];
  const uint64_t c = blockIdx.x;
  const uint64_t s = c * PARSE_CHUNK + (uint64_t)threadIdx.x * PARSE_SEG;
  uint8_t b[PARSE_SEG];
  load_seg(a, s, b);
  const bool live = s < a.n;
  const uint32_t len = live ? (uint32_t)(a.n - s < (uint64_t)PARSE_SEG ? a.n - s : (uint64_t)PARSE_SEG) : 0u;
  const uint8_t before = (s > 0 && live) ? a.raw[s - 1] : (uint8_t)'\n';  // position 0 starts a line
  const uint8_t after = s + len < a.n ? a.raw[s + len] : (uint8_t)0;      // the byte after the segment
  // newlines and header starts of this thread's bytes
  uint32_t nl = 0, hs = 0;
  {
    uint8_t prev = before;
    for (uint32_t j = 0; j < len; ++j) {
      nl += b[j] == '\n';
      hs += prev == '\n' && b[j] == '>';
      prev = b[j];
    }
  }
  if (PASS == 0) {  // A
    uint64_t tot;
    block_excl_scan<uint64_t, PARSE_THREADS>(((uint64_t)hs << 32) | nl, ws64, &tot);
    if (threadIdx.x == 0) {
      a.nl_cnt[c] = (uint32_t)tot;
      a.hs_cnt[c] = (uint32_t)(tot >> 32);
    }
    return;
  }
  uint64_t tot;
  const uint64_t pre = block_excl_scan<uint64_t, PARSE_THREADS>(((uint64_t)hs << 32) | nl, ws64, &tot);
  uint64_t li = a.nl_base[c] + (uint32_t)pre;          // line index of byte s
  uint64_t hi = a.hs_base[c] + (pre >> 32);            // headers before byte s
  if (PASS == 1) {  // B (FASTA): header flags per line
    uint8_t prev = before;
    for (uint32_t j = 0; j < len; ++j) {
      if (prev == '\n') a.hdr[li] = b[j] == '>';
      if (b[j] == '\n') ++li;
      prev = b[j];
    }
    return;
  }
  // C and D: which bytes are kept
  uint32_t kept = 0;
  uint64_t kb = 0;
  if (PASS == 3) {
    uint64_t ktot;
    // the kept count of this thread is recomputed below; scan it first
    uint32_t k0 = 0;
    {
      uint64_t l2 = li;
      uint8_t prev = before;
      bool h = !a.fastq && live && a.hdr[l2];
      for (uint32_t j = 0; j < len; ++j) {
        if (prev == '\n') h = !a.fastq && a.hdr[l2];
        const uint8_t x = b[j];
        const bool eol = j + 1 < len ? b[j + 1] == '\n' : (s + len == a.n || after == '\n');
        const bool seq = a.fastq ? (l2 & 3u) == 1u : !h;
        k0 += seq && x != '\n' && !(x == '\r' && eol);
        if (x == '\n') ++l2;
        prev = x;
      }
    }
    kb = a.kept_base[c] + (uint32_t)block_excl_scan<uint64_t, PARSE_THREADS>(k0, ws64, &ktot);
  }
  uint8_t prev = before;
  bool h = !a.fastq && live && a.hdr[li];
  for (uint32_t j = 0; j < len; ++j) {
    const uint8_t x = b[j];
    if (prev == '\n') {  // a line starts here
      if (a.fastq) {
        const uint32_t kind = (uint32_t)(li & 3u);
        if ((kind == 0 && x != '@') || (kind == 2 && x != '+')) atomicOr(a.err, ERR_INPUT);
        if (PASS == 3 && kind == 1) a.offsets[li >> 2] = kb;
      } else {
        h = a.hdr[li];
        if (PASS == 3 && h) a.offsets[hi] = kb;
        hi += h;
      }
    }
    // a '\r' that ends a line (before '\n' or the end of the file) is dropped
    const bool eol = j + 1 < len ? b[j + 1] == '\n' : (s + len == a.n || after == '\n');
    const bool seq = a.fastq ? (li & 3u) == 1u : !h;
    if (seq && x != '\n' && !(x == '\r' && eol)) {
      if (PASS == 3) a.out[kb++] = x;
      ++kept;
    }
    if (x == '\n') ++li;
    prev = x;
  }
  if (PASS == 2) {
    uint64_t ktot;
    block_excl_scan<uint64_t, PARSE_THREADS>(kept, ws64, &ktot);
    if (threadIdx.x == 0) a.kept_cnt[c] = (uint32_t)ktot;
  }
}

}  // namespace

// Reads the FASTQ (fastq = true) or FASTA file of n bytes at d_raw (device
// memory) into contiguous bases (*d_bases) and offsets (*d_offsets, n_reads
// + 1 entries) in scratch owned by the handle.  KMC_EINPUT for a malformed
// file.
int parse_reads(Handle &h, const uint8_t *d_raw, uint64_t n, bool fastq, const char **d_bases,
                const uint64_t **d_offsets, uint64_t *n_reads, uint64_t *n_bases) {
  DistScratch &ds = h.ds;
  *n_reads = 0;
  *n_bases = 0;
  if (n == 0) return KMC_OK;
  const uint64_t nc = (n + PARSE_CHUNK - 1) / PARSE_CHUNK;
  if (dev_ensure(ds.fq_cnt, nc * 12 + 16, h.st) || dev_ensure(ds.fq_base, (nc + 1) * 24 + 16, h.st) ||
      dev_ensure(ds.fq_tmp, scan_tmp_words(nc) * 8, h.st) || dev_ensure(ds.fq_small, 64, h.st))
    return KMC_ENOMEM;
  ParseArgs a;
  a.raw = d_raw;
  a.n = n;
  a.fastq = fastq ? 1u : 0u;
  a.nl_cnt = as<uint32_t>(ds.fq_cnt);
  a.hs_cnt = a.nl_cnt + nc;
  a.kept_cnt = a.hs_cnt + nc;
  uint64_t *bases_u64 = as<uint64_t>(ds.fq_base);
  a.nl_base = bases_u64;
  a.hs_base = bases_u64 + (nc + 1);
  a.kept_base = bases_u64 + 2 * (nc + 1);
  a.hdr = nullptr;
  a.out = nullptr;
  a.offsets = nullptr;
  a.err = as<uint32_t>(h.err);
  // the first and last bytes decide two format checks and the line count
  uint8_t ends[2] = {0, 0};
  KMC_CUDA_TRY(cudaMemcpyAsync(&ends[0], d_raw, 1, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(&ends[1], d_raw + n - 1, 1, cudaMemcpyDeviceToHost, h.st));
  parse_kernel<0><<<(unsigned)nc, PARSE_THREADS, 0, h.st>>>(a);
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  KMC_CUDA_TRY(device_excl_scan_u32(a.nl_cnt, bases_u64, nc, as<uint64_t>(ds.fq_tmp), h.st));
  KMC_CUDA_TRY(device_excl_scan_u32(a.hs_cnt, bases_u64 + (nc + 1), nc, as<uint64_t>(ds.fq_tmp), h.st));
  uint64_t tot[2] = {0, 0};
  KMC_CUDA_TRY(cudaMemcpyAsync(&tot[0], bases_u64 + nc, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaMemcpyAsync(&tot[1], bases_u64 + (nc + 1) + nc, 8, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  const uint64_t n_nl = tot[0], n_hdr = tot[1];
  const uint64_t n_lines = n_nl + (ends[1] != '\n' ? 1 : 0);
  uint64_t nr;
  if (fastq) {
    if (n_lines % 4) return KMC_EINPUT;  // the last record is incomplete
    nr = n_lines / 4;
  } else {
    if (ends[0] != '>') return KMC_EINPUT;  // a FASTA file starts with a header
    nr = n_hdr;
    if (dev_ensure(ds.fq_hdr, n_lines + 16, h.st)) return KMC_ENOMEM;
    a.hdr = as<uint8_t>(ds.fq_hdr);
    parse_kernel<1><<<(unsigned)nc, PARSE_THREADS, 0, h.st>>>(a);
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  parse_kernel<2><<<(unsigned)nc, PARSE_THREADS, 0, h.st>>>(a);
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  KMC_CUDA_TRY(device_excl_scan_u32(a.kept_cnt, bases_u64 + 2 * (nc + 1), nc, as<uint64_t>(ds.fq_tmp), h.st));
  uint64_t kept = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&kept, bases_u64 + 2 * (nc + 1) + nc, 8, cudaMemcpyDeviceToHost, h.st));
  int rc = check_device_error(h);  // synchronises; format errors found by pass C
  if (rc) return rc;
  if (dev_ensure(ds.fq_bases, kept + 64, h.st) || dev_ensure(ds.fq_offsets, (nr + 1) * 8, h.st))
    return KMC_ENOMEM;
  a.out = as<uint8_t>(ds.fq_bases);
  a.offsets = as<uint64_t>(ds.fq_offsets);
  parse_kernel<3><<<(unsigned)nc, PARSE_THREADS, 0, h.st>>>(a);
  KMC_COUNT_LAUNCH();
  KMC_CUDA_TRY(cudaGetLastError());
  KMC_CUDA_TRY(cudaMemcpyAsync(a.offsets + nr, &kept, 8, cudaMemcpyHostToDevice, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));  // `kept` lives on this stack frame
  *d_bases = reinterpret_cast<const char *>(a.out);
  *d_offsets = a.offsets;
  *n_reads = nr;
  *n_bases = kept;
  return KMC_OK;
}

}  // namespace kmc
