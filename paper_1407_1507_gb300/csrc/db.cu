// KMC 2 output database (Suppl. "Database format"): .kmc_pre / .kmc_suf.
//
// Writer: after kmc_count the sorted result (canonical k-mers, counts) is in
// device memory.  Each k-mer's signature (Sect. 2.2) picks its bin through
// the map; the records must be grouped by bin and ordered by k-mer value
// inside a bin, which is a stable partition of the value-ordered result by
// bin: sorting the unique keys (bin << 32 | index) gives it.  Prefix arrays
// are the exclusive scan of the per-(bin, prefix) counts.  The host writes
// the two files.
//
// Reader: the files are checked and loaded with the format section's
// procedure, then a kernel answers batches of queries the way the section's
// worked example looks one k-mer up (signature -> map -> prefix array range
// -> binary search over the suffixes).
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"
#include "sortlib.cuh"

namespace kmc {
namespace {

constexpr uint32_t kDbVersion = 0x200;
constexpr size_t kDbHeaderBytes = 68;
constexpr int DB_THREADS = 256;

int db_lut(int k, uint32_t n_bins) {
  const int base = k % 4, wide = base + 4;
  if (wide <= k && (uint64_t)n_bins << (2 * wide) <= (1ull << 24)) return wide;
  return base;
}

int db_counter_size(uint32_t max_count) {
  if (max_count < (1u << 8)) return 1;
  if (max_count < (1u << 16)) return 2;
  if (max_count < (1u << 24)) return 3;
  return 4;
}

// k-mer i of an array of ceil(k/32)-word k-mers (most significant word first).
template <typename K>
__device__ __forceinline__ K load_kmer(const uint64_t *w, uint64_t i, int words);
template <>
__device__ __forceinline__ uint64_t load_kmer<uint64_t>(const uint64_t *w, uint64_t i, int) {
  return w[i];
}
template <>
__device__ __forceinline__ u128 load_kmer<u128>(const uint64_t *w, uint64_t i, int words) {
  return words == 1 ? (u128)w[i] : (((u128)w[2 * i]) << 64) | w[2 * i + 1];
}

__device__ __forceinline__ uint64_t rc_of(uint64_t v, int k) { return revcomp64(v, k); }
__device__ __forceinline__ u128 rc_of(u128 v, int k) { return revcomp128(v, k); }

// Sect. 2.2: the signature of a canonical k-mer value is its smallest
// canonical m-mer that the rule allows, 4^m when none is allowed.
template <typename K>
__device__ uint32_t kmer_signature(K v, int k, int m) {
  const uint32_t mmask = (1u << (2 * m)) - 1u;
  uint32_t best = 1u << (2 * m);
  for (int i = 0; i + m <= k; ++i) {
    const uint32_t fw = (uint32_t)(v >> (2 * (k - m - i))) & mmask;
    const uint32_t rc = revcomp32(fw, m);
    const uint32_t c = fw < rc ? fw : rc;
    if (c < best && mmer_allowed(c, m)) best = c;
  }
  return best;
}

// Top lut symbols of a k-mer value (0 when lut = 0).
template <typename K>
__device__ __forceinline__ uint32_t kmer_prefix(K v, int k, int lut) {
  return lut ? (uint32_t)(v >> (2 * (k - lut))) : 0u;
}

template <typename K>
__device__ __forceinline__ K low_bits(K v, int bits) {
  return bits >= (int)(8 * sizeof(K)) ? v : (v & ((K(1) << bits) - 1));
}

// Per k-mer: bin (from the signature and the map), the sort key
// (bin << 32 | index), and the (bin, prefix) count; the largest count.
template <typename K>
__global__ void db_scan_kernel(const uint64_t *__restrict__ kmers, const uint32_t *__restrict__ counts, uint64_t n,
                               int words, int k, int m, int lut, const uint32_t *__restrict__ map, uint32_t n_bins,
                               uint64_t *__restrict__ keys, uint32_t *__restrict__ idx, uint32_t *__restrict__ cnt_bp,
                               uint32_t *max_count, uint32_t *err) {
  const uint32_t P = 1u << (2 * lut);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const K v = load_kmer<K>(kmers, i, words);
    const uint32_t b = map[kmer_signature<K>(v, k, m)];
    if (b >= n_bins) {
      atomicOr(err, ERR_INPUT);
      continue;
    }
    keys[i] = ((uint64_t)b << 32) | i;
    idx[i] = (uint32_t)i;
    atomicAdd(&cnt_bp[(uint64_t)b * P + kmer_prefix<K>(v, k, lut)], 1u);
    atomicMax(max_count, counts[i]);
  }
}

// Record p of the .kmc_suf data: the suffix of k-mer idx[p], then its count.
template <typename K>
__global__ void db_record_kernel(const uint64_t *__restrict__ kmers, const uint32_t *__restrict__ counts,
                                 const uint32_t *__restrict__ idx, uint64_t n, int words, int k, int lut, int csize,
                                 uint8_t *__restrict__ rec) {
  const int sb = (k - lut) / 4, rb = sb + csize;
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = idx[p];
    const K s = low_bits<K>(load_kmer<K>(kmers, i, words), 2 * (k - lut));
    uint8_t *r = rec + p * rb;
    for (int j = 0; j < sb; ++j) r[j] = (uint8_t)(uint64_t)(s >> (8 * (sb - 1 - j)));
    const uint32_t c = counts[i];
    for (int j = 0; j < csize; ++j) r[sb + j] = (uint8_t)(c >> (8 * j));
  }
}

struct DbView {
  const uint32_t *map;
  const uint64_t *firsts;  // n_arrays * 4^lut + 1
  const uint8_t *rec;
  uint32_t n_map, n_arrays;
  int k, m, lut, csize;
};

template <typename K>
__global__ void db_lookup_kernel(DbView db, const uint64_t *__restrict__ q, uint64_t n, int words,
                                 uint32_t *__restrict__ out) {
  const int sb = (db.k - db.lut) / 4, rb = sb + db.csize;
  const uint32_t P = 1u << (2 * db.lut);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
    const K v = low_bits<K>(load_kmer<K>(q, i, words), 2 * db.k);
    const K r = rc_of(v, db.k);
    const K c = v < r ? v : r;  // Sect. 2.1 canonical form
    const uint32_t sig = kmer_signature<K>(c, db.k, db.m);
    uint32_t found = 0;
    const uint32_t a = sig < db.n_map ? db.map[sig] : db.n_arrays;
    if (a < db.n_arrays) {
      const uint64_t e = (uint64_t)a * P + kmer_prefix<K>(c, db.k, db.lut);
      uint64_t lo = db.firsts[e], hi = db.firsts[e + 1];
      const K key = low_bits<K>(c, 2 * (db.k - db.lut));
      while (lo < hi) {  // binary search over the range's suffixes
        const uint64_t mid = (lo + hi) / 2;
        const uint8_t *rr = db.rec + mid * rb;
        K s = 0;
        for (int j = 0; j < sb; ++j) s = (s << 8) | K(rr[j]);
        if (s == key) {
          for (int j = db.csize - 1; j >= 0; --j) found = (found << 8) | rr[sb + j];
          break;
        }
        if (s < key) lo = mid + 1; else hi = mid;
      }
    }
    out[i] = found;
  }
}

inline unsigned db_grid(uint64_t n) {
  const uint64_t g = (n + DB_THREADS - 1) / DB_THREADS;
  return (unsigned)(g < 1 ? 1 : (g > 65535 * 4 ? 65535 * 4 : g));
}

void put_u32(std::vector<uint8_t> &b, uint32_t v) {
  for (int i = 0; i < 4; ++i) b.push_back((uint8_t)(v >> (8 * i)));
}
void put_u64(std::vector<uint8_t> &b, uint64_t v) {
  for (int i = 0; i < 8; ++i) b.push_back((uint8_t)(v >> (8 * i)));
}
uint32_t get_u32(const uint8_t *p) {
  uint32_t v = 0;
  for (int i = 3; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}
uint64_t get_u64(const uint8_t *p) {
  uint64_t v = 0;
  for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
  return v;
}

int io_fail(const std::string &what) {
  set_error_text(what.c_str());
  return KMC_EIO;
}

bool write_file(const std::string &path, const std::vector<uint8_t> &head, const uint8_t *body, size_t nbody,
                const std::vector<uint8_t> &tail) {
  FILE *f = fopen(path.c_str(), "wb");
  if (!f) return false;
  bool ok = fwrite(head.data(), 1, head.size(), f) == head.size();
  if (ok && nbody) ok = fwrite(body, 1, nbody, f) == nbody;
  if (ok && !tail.empty()) ok = fwrite(tail.data(), 1, tail.size(), f) == tail.size();
  ok = (fclose(f) == 0) && ok;
  return ok;
}

bool read_file(const std::string &path, std::vector<uint8_t> &out) {
  FILE *f = fopen(path.c_str(), "rb");
  if (!f) return false;
  bool ok = fseek(f, 0, SEEK_END) == 0;
  const long sz = ok ? ftell(f) : -1;
  ok = ok && sz >= 0 && fseek(f, 0, SEEK_SET) == 0;
  if (ok) {
    out.resize((size_t)sz);
    ok = sz == 0 || fread(out.data(), 1, (size_t)sz, f) == (size_t)sz;
  }
  fclose(f);
  return ok;
}

template <typename K>
int db_build(Handle &h, int lut, std::vector<uint64_t> &firsts, std::vector<uint8_t> &records, int *csize_out) {
  const uint64_t n = h.n_out;
  const int k = (int)h.p.k, m = (int)h.m_used, words = h.key_words;
  const uint32_t B = h.p.n_bins;
  const uint64_t NP = (uint64_t)B << (2 * lut);
  // scratch of this call, released (stream-ordered) on every return path
  struct Scratch {
    DevBuf keys, idx, cnt, fst, tmp, mx, rec;
    cudaStream_t st;
    ~Scratch() {
      for (DevBuf *b : {&keys, &idx, &cnt, &fst, &tmp, &mx, &rec}) dev_release(*b, st);
    }
  } sc;
  sc.st = h.st;
  DevBuf &keys = sc.keys, &idx = sc.idx, &cnt = sc.cnt, &fst = sc.fst, &tmp = sc.tmp, &mx = sc.mx, &rec = sc.rec;
  if (dev_ensure(keys, (n + 1) * 8, h.st) || dev_ensure(idx, (n + 1) * 4, h.st) ||
      dev_ensure(cnt, NP * 4 + 4, h.st) || dev_ensure(fst, (NP + 1) * 8, h.st) ||
      dev_ensure(tmp, scan_tmp_words(NP) * 8, h.st) || dev_ensure(mx, 8, h.st))
    return KMC_ENOMEM;
  KMC_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, NP * 4, h.st));
  KMC_CUDA_TRY(cudaMemsetAsync(mx.p, 0, 4, h.st));
  if (n) {
    db_scan_kernel<K><<<db_grid(n), DB_THREADS, 0, h.st>>>(
        as<uint64_t>(h.out_kmers), as<uint32_t>(h.out_counts), n, words, k, m, lut, as<uint32_t>(h.map), B,
        as<uint64_t>(keys), as<uint32_t>(idx), as<uint32_t>(cnt), as<uint32_t>(mx), as<uint32_t>(h.err));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  KMC_CUDA_TRY(device_excl_scan_u32(as<uint32_t>(cnt), as<uint64_t>(fst), NP, as<uint64_t>(tmp), h.st));
  uint32_t maxc = 0;
  KMC_CUDA_TRY(cudaMemcpyAsync(&maxc, mx.p, 4, cudaMemcpyDeviceToHost, h.st));
  int rc = check_device_error(h);  // synchronises
  if (rc) return rc;
  const int csize = db_counter_size(maxc);
  const int rb = (k - lut) / 4 + csize;
  if (n > 1) {
    int bb = 1;
    while (bb < 32 && (1ull << bb) < B) ++bb;
    rc = sort_pairs_u64(h, as<uint64_t>(keys), as<uint32_t>(idx), n, 32 + bb);
    if (rc) return rc;
  }
  if (dev_ensure(rec, n * rb + 16, h.st)) return KMC_ENOMEM;
  if (n) {
    db_record_kernel<K><<<db_grid(n), DB_THREADS, 0, h.st>>>(as<uint64_t>(h.out_kmers), as<uint32_t>(h.out_counts),
                                                             as<uint32_t>(idx), n, words, k, lut, csize,
                                                             as<uint8_t>(rec));
    KMC_COUNT_LAUNCH();
    KMC_CUDA_TRY(cudaGetLastError());
  }
  firsts.resize(NP + 1);
  records.resize(n * rb);
  KMC_CUDA_TRY(cudaMemcpyAsync(firsts.data(), fst.p, (NP + 1) * 8, cudaMemcpyDeviceToHost, h.st));
  if (n) KMC_CUDA_TRY(cudaMemcpyAsync(records.data(), rec.p, n * rb, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  *csize_out = csize;
  return KMC_OK;
}

}  // namespace
}  // namespace kmc

using namespace kmc;

struct kmc_db {
  int device = 0;
  kmc_db_info info{};
  DevBuf map, firsts, rec;
  cudaStream_t st = nullptr;  // for allocation and upload
};

extern "C" {

int kmc_db_write(kmc_handle *kh, const char *path) {
  if (!kh || !path) return KMC_EINVAL;
  Handle &h = kh->h;
  if (!h.counted || !h.map_ready) return KMC_ESTATE;
  if (h.p.debug_flags & KMC_DEBUG_MINIMIZER) return KMC_EINVAL;  // the format's map is by signature
  if (!h.p.canonical) return KMC_EINVAL;  // lookups take the canonical form
  DeviceGuard g(h.p.device);
  const int k = (int)h.p.k, m = (int)h.m_used;
  const uint32_t B = h.p.n_bins;
  const int lut = db_lut(k, B);
  std::vector<uint64_t> firsts;
  std::vector<uint8_t> records;
  int csize = 1;
  int rc = k <= 32 ? db_build<uint64_t>(h, lut, firsts, records, &csize)
                   : db_build<u128>(h, lut, firsts, records, &csize);
  if (rc) return rc;
  std::vector<uint32_t> map(h.n_sig);
  KMC_CUDA_TRY(cudaMemcpyAsync(map.data(), h.map.p, (size_t)h.n_sig * 4, cudaMemcpyDeviceToHost, h.st));
  KMC_CUDA_TRY(cudaStreamSynchronize(h.st));
  // .kmc_pre: marker, prefix arrays + guard, map, header, header size, marker
  std::vector<uint8_t> pre;
  pre.reserve(4 + firsts.size() * 8 + map.size() * 4 + kDbHeaderBytes + 8);
  for (char c : std::string("KMCP")) pre.push_back((uint8_t)c);
  for (uint64_t v : firsts) put_u64(pre, v);
  for (uint32_t v : map) put_u32(pre, v);
  const size_t h0 = pre.size();
  put_u32(pre, (uint32_t)k);
  put_u32(pre, 0);  // mode: occurrence counters
  put_u32(pre, (uint32_t)csize);
  put_u32(pre, (uint32_t)lut);
  put_u32(pre, (uint32_t)m);
  put_u32(pre, (uint32_t)std::max<uint64_t>(h.p.cutoff_min, 1));
  put_u32(pre, (uint32_t)std::min<uint64_t>(h.p.cutoff_max, 0xFFFFFFFFull));
  put_u64(pre, h.n_out);
  for (int i = 0; i < 7; ++i) put_u32(pre, 0);
  put_u32(pre, kDbVersion);
  put_u32(pre, (uint32_t)(pre.size() - h0));
  for (char c : std::string("KMCP")) pre.push_back((uint8_t)c);
  const std::string base(path);
  if (!write_file(base + ".kmc_pre", pre, nullptr, 0, {})) return io_fail("cannot write " + base + ".kmc_pre");
  const std::vector<uint8_t> ms{'K', 'M', 'C', 'S'};
  if (!write_file(base + ".kmc_suf", ms, records.data(), records.size(), ms))
    return io_fail("cannot write " + base + ".kmc_suf");
  return KMC_OK;
}

int kmc_db_open(kmc_db **out, const char *path, int device) {
  if (!out || !path) return KMC_EINVAL;
  *out = nullptr;
  const std::string base(path);
  std::vector<uint8_t> pre, suf;
  if (!read_file(base + ".kmc_pre", pre)) return io_fail("cannot read " + base + ".kmc_pre");
  if (!read_file(base + ".kmc_suf", suf)) return io_fail("cannot read " + base + ".kmc_suf");
  // the format section's procedure: both markers, then the header from its
  // position in the last 8 bytes
  if (pre.size() < 12 + kDbHeaderBytes || memcmp(pre.data(), "KMCP", 4) || memcmp(pre.data() + pre.size() - 4, "KMCP", 4))
    return io_fail(base + ".kmc_pre: no KMCP markers");
  if (suf.size() < 8 || memcmp(suf.data(), "KMCS", 4) || memcmp(suf.data() + suf.size() - 4, "KMCS", 4))
    return io_fail(base + ".kmc_suf: no KMCS markers");
  const uint64_t x = get_u32(pre.data() + pre.size() - 8);
  if (x != kDbHeaderBytes || x + 8 > pre.size() - 4) return io_fail(base + ".kmc_pre: bad header position");
  const uint8_t *hp = pre.data() + pre.size() - 8 - x;
  kmc_db_info in{};
  in.kmer_length = get_u32(hp);
  in.mode = get_u32(hp + 4);
  in.counter_size = get_u32(hp + 8);
  in.lut_prefix_length = get_u32(hp + 12);
  in.signature_length = get_u32(hp + 16);
  in.min_count = get_u32(hp + 20);
  in.max_count = get_u32(hp + 24);
  in.total_kmers = get_u64(hp + 28);
  in.kmc_ver = get_u32(hp + 64);
  const uint32_t k = in.kmer_length, lut = in.lut_prefix_length, m = in.signature_length;
  if (in.mode != 0 || k < 1 || k > 64 || in.counter_size < 1 || in.counter_size > 4 || lut > k || (k - lut) % 4 ||
      m < 1 || m > KMC_MAX_M || lut > 12)
    return io_fail(base + ".kmc_pre: unsupported header");
  const uint64_t n_map = (1ull << (2 * m)) + 1;
  const uint64_t h0 = pre.size() - 8 - x;
  if (h0 < 4 + 4 * n_map + 8) return io_fail(base + ".kmc_pre: too short for its map");
  const uint64_t map_off = h0 - 4 * n_map;
  if ((map_off - 4) % 8) return io_fail(base + ".kmc_pre: prefix region not whole words");
  const uint64_t n_pref = (map_off - 4) / 8, P = 1ull << (2 * lut);
  if (n_pref < 1 || (n_pref - 1) % P) return io_fail(base + ".kmc_pre: prefix arrays do not divide");
  in.n_arrays = (uint32_t)((n_pref - 1) / P);
  const uint64_t rb = (k - lut) / 4 + in.counter_size;
  if (suf.size() - 8 != in.total_kmers * rb) return io_fail(base + ".kmc_suf: size does not match the header");
  if (get_u64(pre.data() + 4 + 8 * (n_pref - 1)) != in.total_kmers)
    return io_fail(base + ".kmc_pre: guard does not match the header");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return KMC_EINVAL;
  }
  DeviceGuard g(device);
  kmc_db *db = new (std::nothrow) kmc_db();
  if (!db) return KMC_ENOMEM;
  db->device = device;
  db->info = in;
  if (cudaStreamCreateWithFlags(&db->st, cudaStreamNonBlocking) != cudaSuccess) {
    delete db;
    return cuda_fail(cudaGetLastError(), "cudaStreamCreate");
  }
  auto fail = [&](int rc) {
    for (DevBuf *b : {&db->map, &db->firsts, &db->rec}) dev_release(*b, db->st);
    cudaStreamSynchronize(db->st);
    cudaStreamDestroy(db->st);
    delete db;
    return rc;
  };
  if (dev_ensure(db->map, n_map * 4, db->st) || dev_ensure(db->firsts, n_pref * 8, db->st) ||
      dev_ensure(db->rec, suf.size() - 8 + 16, db->st))
    return fail(KMC_ENOMEM);
  if (cudaMemcpyAsync(db->map.p, pre.data() + map_off, n_map * 4, cudaMemcpyHostToDevice, db->st) != cudaSuccess ||
      cudaMemcpyAsync(db->firsts.p, pre.data() + 4, n_pref * 8, cudaMemcpyHostToDevice, db->st) != cudaSuccess ||
      (suf.size() > 8 &&
       cudaMemcpyAsync(db->rec.p, suf.data() + 4, suf.size() - 8, cudaMemcpyHostToDevice, db->st) != cudaSuccess) ||
      cudaStreamSynchronize(db->st) != cudaSuccess)
    return fail(cuda_fail(cudaGetLastError(), "database upload"));
  *out = db;
  return KMC_OK;
}

int kmc_db_info_get(const kmc_db *db, kmc_db_info *info) {
  if (!db || !info) return KMC_EINVAL;
  *info = db->info;
  return KMC_OK;
}

int kmc_db_lookup(kmc_db *db, const uint64_t *d_kmers, uint64_t n, uint32_t *d_counts, void *cuda_stream) {
  if (!db || (n && (!d_kmers || !d_counts))) return KMC_EINVAL;
  if (!n) return KMC_OK;
  DeviceGuard g(db->device);
  DbView v;
  v.map = as<uint32_t>(db->map);
  v.firsts = as<uint64_t>(db->firsts);
  v.rec = as<uint8_t>(db->rec);
  v.n_map = (1u << (2 * db->info.signature_length)) + 1u;
  v.n_arrays = db->info.n_arrays;
  v.k = (int)db->info.kmer_length;
  v.m = (int)db->info.signature_length;
  v.lut = (int)db->info.lut_prefix_length;
  v.csize = (int)db->info.counter_size;
  const int words = (v.k + 31) / 32;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  if (v.k <= 32)
    db_lookup_kernel<uint64_t><<<db_grid(n), DB_THREADS, 0, st>>>(v, d_kmers, n, words, d_counts);
  else
    db_lookup_kernel<u128><<<db_grid(n), DB_THREADS, 0, st>>>(v, d_kmers, n, words, d_counts);
  KMC_COUNT_LAUNCH();
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? KMC_OK : cuda_fail(e, "kmc_db_lookup");
}

void kmc_db_close(kmc_db *db) {
  if (!db) return;
  {
    DeviceGuard g(db->device);
    for (DevBuf *b : {&db->map, &db->firsts, &db->rec}) dev_release(*b, db->st);
    cudaStreamSynchronize(db->st);
    cudaStreamDestroy(db->st);
  }
  delete db;
}

}  // extern "C"
