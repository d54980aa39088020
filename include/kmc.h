/*
 * kmc.h -- C ABI of a GB300 (sm_103a) k-mer counter built on the method of
 * KMC 2 (Deorowicz, Kokot, Grabowski, Debudaj-Grabysz, "KMC 2: Fast and
 * resource-frugal k-mer counting", arXiv 1407.1507).
 *
 * The problem (paper Sect. 1): given a collection of reads, report every
 * canonical k-mer (Sect. 2.1: the smaller of a k-mer and its reverse
 * complement under A < C < G < T) with its number of occurrences, keeping
 * only the k-mers whose count n satisfies cutoff_min <= n <= cutoff_max
 * (Sect. 2.5; Suppl. S1 options -ci, -cx).  Every step runs in CUDA kernels
 * of this library: 2-bit packing, the signature scan (Sect. 2.2), super
 * k-mer binning (Sect. 2.4, Fig. 1), (k,x)-mer construction (Sect. 2.3),
 * radix sorting, expansion and run-length counting (Sect. 2.4, Fig. 2).
 * Options of Suppl. S1 beyond these: k-mers as read instead of canonical
 * (-b, kmc_params.canonical = 0) and a counter maximum (-cs,
 * kmc_params.counter_max).  Around the counting path: FASTQ / FASTA input
 * read on the device (kmc_add_file_bytes), KMC 2's database files with
 * batched lookups (kmc_db_*), batched read sets (kmc_batch_*) and a
 * request server (kmc_server_*).
 *
 * Conventions (all calls):
 *   - Return KMC_OK (0) on success, a negative KMC_E* code otherwise;
 *     kmc_strerror() names it.  A handle whose call failed with
 *     KMC_ECUDA, KMC_ETIMEOUT or KMC_ENOMEM must be closed.
 *   - Bases: ASCII.  'A','C','G','T' are bases; ANY other byte (including
 *     lower case and 'N') breaks the read there: no k-mer spans it, and no
 *     k-mer spans two reads.  Reads shorter than k add nothing.
 *   - A k-mer is returned as W = ceil(k/32) uint64 words, most significant
 *     word first, its value right-aligned in the low 2k bits, the first
 *     symbol most significant, A=0 C=1 G=2 T=3 (Suppl. S4 [map] coding).
 *     The result is sorted ascending by that value, one count per k-mer.
 *   - A handle is not thread safe; distinct handles may be used from
 *     different threads.  All work of a handle is ordered on its stream.
 *   - The library allocates its own device and pinned host memory
 *     (cudaMallocAsync on the handle's stream) and frees it in kmc_close.
 */
#ifndef KMC_GB300_KMC_H
#define KMC_GB300_KMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------- error codes */
#define KMC_OK 0
#define KMC_EINVAL (-1)    /* bad argument or parameter                     */
#define KMC_ESTATE (-2)    /* call out of order (e.g. result before count)  */
#define KMC_ENOMEM (-3)    /* device or pinned host allocation failed       */
#define KMC_ECUDA (-4)     /* a CUDA call or kernel launch failed           */
#define KMC_EOVERFLOW (-5) /* a count exceeds UINT32_MAX                    */
#define KMC_ETRUNC (-6)    /* caller capacity too small; *n_out still set    */
#define KMC_ETIMEOUT (-7)  /* a device-side bounded wait gave up            */
#define KMC_EAGAIN (-8)    /* not ready yet (server poll)                   */
#define KMC_EINPUT (-9)    /* malformed read offsets or FASTQ / FASTA file    */
#define KMC_EIO (-10)      /* a database file cannot be read or written, or
                              is not in the KMC 2 format                    */
#define KMC_ECANCELED (-11) /* the job was cancelled (kmc_server_cancel)    */

#define KMC_AUTO 0xFFFFFFFFu
#define KMC_MAX_K 64u
#define KMC_MIN_M 3u
#define KMC_MAX_M 11u

/* ---------------------------------------------------------- parameters */
typedef struct {
  uint32_t k;          /* k-mer length, 1..64 (Suppl. S1 -k; default 25)           */
  uint32_t m;          /* signature length, 3..11 and m < k (Sect. 2.2; Suppl.
                          S1 -p gives 5..7, default 7).  Values m >= k are
                          clamped to k-1 for k >= 4; k <= 3 uses no signature
                          (one bin).                                          */
  uint32_t n_bins;     /* number of bins, 1..65536 (Sect. 2.4 uses <= 512)        */
  uint32_t x;          /* (k,x)-mer extension, 0..3, or KMC_AUTO (Sect. 2.3)      */
  uint64_t cutoff_min; /* keep count >= cutoff_min (Suppl. S1 -ci; default 2)     */
  uint64_t cutoff_max; /* keep count <= cutoff_max (Suppl. S1 -cx; default 1e9)   */
  uint32_t canonical;  /* 1: canonical k-mers (Sect. 2.1, default); 0: k-mers as
                          read, no transformation into canonical form (Suppl.
                          S1 -b), with x = 0 or KMC_AUTO only                 */
  int32_t device;      /* CUDA device ordinal                                     */
  void *cuda_stream;   /* cudaStream_t to run on, or NULL for a stream of the
                          handle's own                                        */
  uint32_t debug_flags;/* KMC_DEBUG_* bits: keep intermediates for inspection     */
  uint32_t reserved0;  /* must be zero                                            */
  uint64_t piece_bytes;/* reads are distributed in pieces of about this many
                          bytes (0 = 256 MiB: a piece's bins then stay close
                          to L2-sized while they are filled); bounds the
                          distribution scratch, never changes the result      */
  uint64_t device_budget; /* device bytes for the bins and the sort buffers
                          (0 = no limit).  With a limit, a piece whose bins
                          would take the bins past half of it is moved to
                          pinned host memory (async copy) and read from there
                          over NVLink-C2C by the sort, and (x = 0) the bins
                          are sorted in waves whose two key buffers take at
                          most a quarter each; a single bin larger than a
                          wave is still sorted whole.  Never changes the
                          result.  Not applied to x > 0.                      */
  uint64_t counter_max;/* 0: exact counts (default); else a count above it is
                          reported as counter_max (Suppl. S1 -cs, "maximal
                          value of a counter"); the cutoffs apply to the true
                          count.  kmc_count only (batched / served: 0)         */
} kmc_params;

/* Fills *p with the paper's defaults: k=25, m=7, 512 bins, x=KMC_AUTO,
 * cutoffs [2, 1e9], canonical, device 0, own stream. */
void kmc_default_params(kmc_params *p);

/* ---------------------------------------------------------- statistics */
typedef struct {
  uint64_t n_reads;          /* reads added                                    */
  uint64_t n_bases;          /* bytes added                                    */
  uint64_t n_kmer_positions; /* valid k-mer positions (sum of all counts)      */
  uint64_t n_superkmers;     /* super k-mers (Sect. 2.4)                       */
  uint64_t n_sorted_keys;    /* (k,x)-mers sorted (Sect. 2.3)                  */
  uint64_t n_distinct;       /* distinct canonical k-mers before cutoffs       */
  uint64_t n_out;            /* k-mers in the result                           */
  uint64_t max_bin_kmers;    /* k-mer positions in the largest bin             */
  uint64_t bin_bytes;        /* bytes of super k-mer records in the bins       */
  uint32_t x_used;           /* x chosen (resolves KMC_AUTO)                   */
  uint32_t m_used;           /* signature length used                          */
  uint32_t n_tiles;          /* sort tiles processed                           */
  uint32_t n_big_tiles;      /* tiles too large for one CTA's shared memory    */
  float ms_distribute;       /* device time: pack, signatures, binning         */
  float ms_sort;             /* device time: (k,x)-mers, sort, count           */
  float ms_order;            /* device time: global ordering of the result     */
  float ms_total;            /* device time of the last kmc_count              */
  /* device time per kernel stage (CUDA events on the handle's stream),
   * summed since kmc_open / kmc_reset, in the KMC_STAGE_* order below */
  float ms_stage[12];
  uint64_t n_launches;       /* kernels launched since kmc_open / kmc_reset    */
  uint64_t spilled_bytes;    /* bin bytes moved to pinned host memory          */
  uint32_t n_waves;          /* bin waves of the last kmc_count (1 without a
                                device_budget)                                 */
  uint32_t reserved_s;
  uint64_t n_fused_keys;     /* keys counted straight from their super buckets
                                (one shared-memory pass, no lower sweep)        */
} kmc_stats;

/* Stage indices of kmc_stats.ms_stage. */
enum {
  KMC_STAGE_PACK = 0,      /* 2-bit packing and read-start marks             */
  KMC_STAGE_SIGNATURE,     /* signature scan, super k-mer list               */
  KMC_STAGE_BIN_SCATTER,   /* super k-mer records into bins                  */
  KMC_STAGE_BIN_MAP,       /* sample histogram and bin map                   */
  KMC_STAGE_KX_COUNT,      /* (k,x)-mer digit histogram                      */
  KMC_STAGE_PLAN,          /* scans and tile plan                            */
  KMC_STAGE_KX_SCATTER,    /* (k,x)-mer keys into digit buckets              */
  KMC_STAGE_TILE_SORT,     /* shared-memory radix sort + run-length count    */
  KMC_STAGE_BIG_SORT,      /* buckets larger than a tile                     */
  KMC_STAGE_ORDER,         /* global order of the counted k-mers             */
  KMC_STAGE_OTHER,
  KMC_N_STAGES
};

/* ---------------------------------------------------------- handle */
typedef struct kmc_handle kmc_handle;

/* Validates *p and creates a handle (device memory is allocated lazily).
 * *h is set to NULL on failure.  Errors: KMC_EINVAL, KMC_ECUDA, KMC_ENOMEM. */
int kmc_open(kmc_handle **h, const kmc_params *p);

/* Adds reads held in HOST memory: read i is bases[offsets[i] .. offsets[i+1]),
 * offsets has n_reads+1 non-decreasing entries and offsets[0] == 0.  The
 * bytes are copied before the call returns, so the caller may free them at
 * once.  Pinned (page-locked) input is copied in pieces of up to 256 MiB on
 * a second stream, the copy of one piece overlapping the distribution of the
 * one before; pageable input goes through pinned staging buffers.  May be
 * called repeatedly before kmc_count; each call appends.
 * Errors: KMC_EINVAL (NULL pointer with n_reads > 0), KMC_EINPUT (offsets
 * not non-decreasing or not starting at 0; decreasing offsets are found by
 * the device, after the reads were staged), KMC_ESTATE (after kmc_count
 * without kmc_reset), KMC_ENOMEM, KMC_ECUDA. */
int kmc_add_reads(kmc_handle *h, const char *bases, const uint64_t *offsets, uint64_t n_reads);

/* As kmc_add_reads, for reads already in DEVICE memory of the handle's
 * device: d_bases has n_bases bytes, d_offsets n_reads+1 entries with
 * d_offsets[0] == 0 and d_offsets[n_reads] == n_bases.  The buffers are
 * only read, by kernels ordered on the handle's stream; they must stay valid
 * until kmc_add_reads_device returns (it synchronises with its own work).
 * Malformed offsets are detected on the device: KMC_EINPUT. */
int kmc_add_reads_device(kmc_handle *h, const char *d_bases, const uint64_t *d_offsets,
                         uint64_t n_reads, uint64_t n_bases);

/* FASTQ or FASTA file contents (Sect. 2.4: reads come from FASTQ/FASTA
 * files; Suppl. S1 -fq, -fa, -fm), read on the device; the host only copies
 * the bytes.  format KMC_FORMAT_FASTQ: records of four lines ("@" header,
 * sequence, "+" line, quality); each sequence line is a read.
 * KMC_FORMAT_FASTA (also multi-FASTA): records of a ">" header line and any
 * number of sequence lines; a record's read is its sequence lines joined
 * without line breaks (a genome may be one read).  In both, a "\r" that ends
 * a line is dropped, a final newline may be missing, and the read's bytes
 * follow the conventions of kmc_add_reads (any byte other than A/C/G/T breaks
 * it).  n_reads and n_bases of kmc_stats count the reads and their bases.
 * kmc_add_file_bytes takes host memory (copied before it returns),
 * kmc_add_file_bytes_device device memory (read during the call).  Errors:
 * KMC_EINVAL (unknown format), KMC_EINPUT (a FASTQ record that does not
 * start with "@", has no "+" line or is incomplete; a FASTA file that does
 * not start with ">"), KMC_ESTATE, KMC_ENOMEM, KMC_ECUDA. */
#define KMC_FORMAT_FASTQ 1u
#define KMC_FORMAT_FASTA 2u
int kmc_add_file_bytes(kmc_handle *h, const char *bytes, uint64_t n_bytes, uint32_t format);
int kmc_add_file_bytes_device(kmc_handle *h, const char *d_bytes, uint64_t n_bytes, uint32_t format);

/* Runs the sorting phase over all reads added and keeps the result on the
 * device.  Blocks until done.  May be called again (it recounts the same
 * reads).  Errors: KMC_ESTATE (no kmc_add_reads since open/reset is fine:
 * the result is empty), KMC_EOVERFLOW, KMC_ENOMEM, KMC_ECUDA, KMC_ETIMEOUT. */
int kmc_count(kmc_handle *h);

/* Number of k-mers in the result.  Errors: KMC_ESTATE before kmc_count. */
int kmc_result_size(const kmc_handle *h, uint64_t *n);

/* Copies the result to HOST buffers: kmers gets n*ceil(k/32) uint64 words,
 * counts n uint32.  If capacity < n nothing is copied and KMC_ETRUNC is
 * returned; *n_out is set to n in both cases.  Either buffer may be NULL to
 * skip it.  Errors: KMC_ESTATE, KMC_ETRUNC, KMC_ECUDA. */
int kmc_result(kmc_handle *h, uint64_t *kmers, uint32_t *counts, uint64_t capacity,
               uint64_t *n_out);

/* Device pointers to the result (owned by the handle, valid until the next
 * kmc_count, kmc_reset or kmc_close): *d_kmers holds n*ceil(k/32) words
 * laid out as in kmc_result, *d_counts n counts.  Errors: KMC_ESTATE. */
int kmc_result_device(kmc_handle *h, const uint64_t **d_kmers, const uint32_t **d_counts,
                      uint64_t *n);

/* Statistics of the reads added and the last kmc_count. */
int kmc_stats_get(const kmc_handle *h, kmc_stats *s);

/* Forgets the reads and the result; keeps device allocations for reuse. */
int kmc_reset(kmc_handle *h);

/* Releases everything the handle owns.  NULL is a no-op. */
void kmc_close(kmc_handle *h);

/* Static string naming an error code. */
const char *kmc_strerror(int code);

/* ---------------------------------------------------------- bin map
 * Sect. 2.4: the 4^m signatures (plus the sentinel 4^m of k-mers with no
 * allowed m-mer) are merged into n_bins bins from a signature histogram of
 * a sample of the input.  By default the map is built on the device from
 * the first kmc_add_reads call's reads (at most 2^20 of them): signatures
 * sorted by sample weight, heaviest first (ties: smaller signature first),
 * cut into consecutive groups of about total/n_bins weight; unseen
 * signatures go to bin (signature mod n_bins).  The result never depends
 * on the map.  kmc_set_bin_map replaces it (before the first
 * kmc_add_reads): map has 4^m+1 entries, each < n_bins, in host memory,
 * copied.  kmc_get_bin_map copies the map in use (after the first
 * kmc_add_reads) to a host buffer of 4^m+1 entries.  Errors: KMC_EINVAL,
 * KMC_ESTATE. */
int kmc_set_bin_map(kmc_handle *h, const uint32_t *map, uint64_t n_entries);
int kmc_get_bin_map(const kmc_handle *h, uint32_t *map, uint64_t n_entries);

/* ---------------------------------------------------------- database
 * KMC 2's output database (Suppl. "Database format"): two files, <path>.kmc_pre
 * and <path>.kmc_suf, integers least significant byte first.
 *
 * .kmc_pre: "KMCP"; the prefix arrays, one per bin in bin order, each of
 * 4^lut uint64 (element x = index of the bin's first record whose first lut
 * symbols have value x), then one uint64 guard (the number of records); the
 * map, 4^m + 1 uint32 (signature -> bin, the map kmc_count used); the header
 * (kmer_length, mode = 0, counter_size, lut_prefix_length, signature_length,
 * min_count, max_count as uint32, total_kmers as uint64, seven unused uint32
 * written as 0, KMC_VER = 0x200 as uint32: 68 bytes); the header's size
 * (uint32, so that the header starts that many + 8 bytes before the end);
 * "KMCP".  .kmc_suf: "KMCS"; one record per k-mer, grouped by bin and ordered
 * by k-mer value inside a bin: the last k - lut symbols of the canonical
 * k-mer, four per byte, first symbol in the top bits, then the count on
 * counter_size bytes; "KMCS".  Where the format leaves a choice:
 * lut = (k mod 4) + 4 when that is at most k and n_bins * 4^lut <= 2^24, else
 * k mod 4; counter_size = the fewest bytes holding the largest count;
 * min_count = max(cutoff_min, 1), max_count = min(cutoff_max, 2^32 - 1).
 *
 * kmc_db_write: after kmc_count, writes the result of the handle; the
 * records and prefix arrays are built on the device (each k-mer's
 * signature, Sect. 2.2, picks its bin through the map).  path is the common
 * prefix of the two file names.  Errors: KMC_ESTATE (before kmc_count),
 * KMC_EINVAL (a handle counting k-mers as read, canonical = 0, or binning
 * by minimizers), KMC_EIO (a file cannot be written), KMC_ENOMEM, KMC_ECUDA.
 *
 * kmc_db_open: reads a database with the format section's procedure (both
 * markers, the header position, the header, the map and prefix arrays, the
 * records) and loads it into the memory of CUDA device `device`.  Errors:
 * KMC_EIO (missing, truncated or malformed file; nothing is allocated),
 * KMC_EINVAL, KMC_ENOMEM, KMC_ECUDA.
 *
 * kmc_db_lookup: counts of n query k-mers, as the format section looks one
 * up: the canonical form (Sect. 2.1), its signature, the map, the prefix
 * array range, a binary search over the suffixes; 0 for a k-mer that is not
 * in the database.  d_kmers (device memory) holds n * ceil(k/32) words, laid
 * out as in kmc_result (bits above 2k are ignored; either strand); d_counts
 * (device memory) receives n uint32.  Runs on cuda_stream (NULL: the legacy
 * default stream) and returns without waiting.  Errors: KMC_EINVAL.
 *
 * kmc_db_info_get fills the header fields; kmc_db_close releases the
 * database (NULL is a no-op). */
typedef struct kmc_db kmc_db;
typedef struct {
  uint32_t kmer_length, mode, counter_size, lut_prefix_length, signature_length;
  uint32_t min_count, max_count;
  uint64_t total_kmers;
  uint32_t kmc_ver;
  uint32_t n_arrays; /* prefix arrays (bins) */
} kmc_db_info;
int kmc_db_write(kmc_handle *h, const char *path);
int kmc_db_open(kmc_db **db, const char *path, int device);
int kmc_db_info_get(const kmc_db *db, kmc_db_info *info);
int kmc_db_lookup(kmc_db *db, const uint64_t *d_kmers, uint64_t n, uint32_t *d_counts, void *cuda_stream);
void kmc_db_close(kmc_db *db);

/* ---------------------------------------------------------- introspection
 * Intermediate results, for checking each step against a CPU restatement.
 *
 * kmc_debug_superkmers: the super k-mers found by the signature scan
 * (Sect. 2.4, Fig. 1) of all reads added, in no particular order: read
 * index, position of the first k-mer in the read, number of k-mers and
 * signature (4^m for none).  Super k-mers are maximal runs of consecutive
 * valid k-mers with one signature, additionally cut before every k-mer whose
 * position in its read is a multiple of 128 (a bound on record size; it does
 * not change the result).  Needs KMC_DEBUG_KEEP_SUPERKMERS in
 * params.debug_flags at open (keeps the list).  capacity < n: KMC_ETRUNC with *n_out = n.
 *
 * kmc_debug_bin_keys: after kmc_count, the sorted (k,x)-mer keys of one bin
 * (Sect. 2.3): each key is ceil((2(k+x)+2)/64) words, most significant
 * first; for x = 0 a key is the canonical k-mer value, for x > 0 it is
 * [x' in the top 2 bits][the k+x' symbols of the stored (k,x)-mer,
 * first symbol most significant, zero padded].  Needs KMC_DEBUG_KEEP_KEYS
 * in params.debug_flags at open (keeps the sorted keys). */
int kmc_debug_superkmers(kmc_handle *h, uint64_t *read_index, uint32_t *pos, uint32_t *n_kmers,
                         uint32_t *sig, uint64_t capacity, uint64_t *n_out);
int kmc_debug_bin_keys(kmc_handle *h, uint32_t bin, uint64_t *keys, uint64_t capacity,
                       uint64_t *n_out, uint32_t *words_per_key);

/* ---------------------------------------------------------- batches
 * Many independent read sets counted together.  A sub-batch packs whole sets
 * into one input stream; set s owns its own range of bins, so the sets never
 * mix (the counts of each set are exactly what kmc_count gives for it alone).
 * All buffers are sized from the capacity given at open, and the launch
 * sequence of a sub-batch reads every data-dependent size from device memory,
 * so it runs without host synchronisation: it is captured once as a CUDA
 * graph and replayed for every sub-batch of the same k.  A set larger than
 * the capacity, or of 4 MiB of bases or more, is counted by the single-set
 * path instead, two such sets at a time on streams of their own (the batch
 * pays for itself while per-set launches and host steps dominate).  With KMC_BATCH_AUTOTUNE
 * the first sub-batch of each k times a few settings (bins per set, bucket
 * width, tile size) and the fastest is kept for the handle's lifetime.
 *
 * kmc_batch_open: base parameters (k is given per set; m, n_bins (ignored:
 *   tuned), cutoffs, device, stream as in kmc_params; x must be 0 or
 *   KMC_AUTO), capacity of one sub-batch: max_bases (1 KiB .. 2 GiB) bytes,
 *   max_reads reads, max_sets sets (<= 65536).  Device memory of about
 *   60 bytes per byte of capacity is allocated per k in use.
 * kmc_batch_run: counts n_sets host read sets (each as in kmc_add_reads;
 *   k[s] in 1..32).  Blocks.  Results replace those of the previous run.
 * kmc_batch_result: host arrays of set `set` (page-locked memory owned by
 *   the handle and reused by the next run; valid
 *   until the next run or close): n k-mers (one uint64 each, layout as in
 *   kmc_result) ascending, and their counts. */
#define KMC_BATCH_AUTOTUNE 1u
#define KMC_BATCH_NO_GRAPH 2u
typedef struct kmc_batch kmc_batch;
typedef struct {
  float ms_device;          /* device time of the sub-batches (CUDA events)   */
  float ms_wall;            /* wall time of the last kmc_batch_run            */
  uint32_t n_sub_batches;   /* sub-batches run (graph replays)                */
  uint32_t n_single;        /* sets counted by the single-set path            */
  uint32_t tuning_runs;     /* sub-batch runs spent by the autotuner          */
  uint32_t bins_per_set;    /* tuning in use (last k)                         */
  uint32_t tile_keys;
  uint32_t bucket_keys;
  uint64_t n_kmers_out;     /* k-mers in all results                          */
} kmc_batch_stats;
int kmc_batch_open(kmc_batch **b, const kmc_params *p, uint64_t max_bases, uint64_t max_reads,
                   uint32_t max_sets, uint32_t flags);
int kmc_batch_run(kmc_batch *b, uint32_t n_sets, const char *const *bases,
                  const uint64_t *const *offsets, const uint64_t *n_reads, const uint32_t *k);
int kmc_batch_result(kmc_batch *b, uint32_t set, const uint64_t **kmers, const uint32_t **counts,
                     uint64_t *n);
int kmc_batch_stats_get(const kmc_batch *b, kmc_batch_stats *s);
void kmc_batch_close(kmc_batch *b);

/* ---------------------------------------------------------- serving
 * A request loop with continuous batching.  kmc_server_submit copies a
 * job's host reads and queues it (it never blocks on the GPU).  n_workers
 * worker threads, each with its own CUDA stream and resident batch engines
 * (kmc_batch_*), repeatedly admit queued jobs in arrival order while they
 * fit one batch (batch_bases bytes, batch_reads reads, batch_sets jobs; a job
 * of 4 MiB of bases or more runs alone, on the worker's own single-set handle
 * for its k, its result written into a recycled page-locked buffer) and
 * the device-memory budget: the predicted footprint of a job is 32 bytes
 * per input byte, and the jobs in flight never exceed mem_budget (a job is
 * always admitted when nothing is in flight).  Jobs that arrive while
 * batches run join the next batch that has room.  A job's result is exactly
 * what kmc_count gives for its reads alone.
 * kmc_server_wait: KMC_OK when done, KMC_EAGAIN on timeout (timeout_s < 0
 *   waits without limit), or the job's error code.
 * kmc_server_result: host arrays owned by the server until
 *   kmc_server_release; latency = completion - submission (wall clock).
 * kmc_server_stats_get: completed jobs, p50 / p99 / mean latency, batches,
 *   the largest batch, the most jobs in flight, wall time from the first
 *   submission to the last completion. */
typedef struct kmc_server kmc_server;
typedef struct {
  kmc_params base;       /* m, cutoffs, device (k is given per job; x = 0)  */
  uint64_t batch_bases;  /* capacity of one batch, bytes (0 = 128 MiB)      */
  uint64_t batch_reads;  /* reads per batch (0 = batch_bases / 64)          */
  uint32_t batch_sets;   /* jobs per batch (0 = 256)                        */
  uint32_t n_workers;    /* batches in flight, 1..8 (0 = 2)                 */
  uint64_t mem_budget;   /* predicted device bytes in flight (0 = workers x
                            32 x batch_bases)                               */
  uint32_t batch_flags;  /* KMC_BATCH_* for the workers' batch handles      */
  uint32_t reserved0;
  uint64_t warm_k_mask;  /* bit k set (1..32): every worker builds and
                            captures its engine for k at open, on synthetic
                            reads, so that first requests do not pay for it */
} kmc_server_cfg;
typedef struct {
  uint64_t jobs_done;
  uint64_t jobs_queued;
  uint64_t batches;
  uint64_t max_batch_jobs;
  uint64_t max_inflight_jobs;
  double p50_ms, p99_ms, mean_ms;
  double wall_s;
  int32_t error;          /* last job error (0 = none)                      */
  int32_t reserved0;
} kmc_server_stats;
int kmc_server_open(kmc_server **s, const kmc_server_cfg *cfg);
int kmc_server_submit(kmc_server *s, uint32_t k, const char *bases, const uint64_t *offsets,
                      uint64_t n_reads, uint64_t *job_id);
/* kmc_server_submit_ref: as kmc_server_submit without the copy: the server
 *   reads the caller's host buffers in place, so they must stay valid and
 *   unchanged until kmc_server_wait reports the job finished (or it is
 *   cancelled).  Submission then costs no host copy, whatever the job size. */
int kmc_server_submit_ref(kmc_server *s, uint32_t k, const char *bases, const uint64_t *offsets,
                          uint64_t n_reads, uint64_t *job_id);
int kmc_server_wait(kmc_server *s, uint64_t job_id, double timeout_s);
int kmc_server_result(kmc_server *s, uint64_t job_id, const uint64_t **kmers,
                      const uint32_t **counts, uint64_t *n, double *latency_ms);
int kmc_server_release(kmc_server *s, uint64_t job_id);
/* kmc_server_cancel: a job still waiting in the queue is removed from it and
 *   ends with KMC_ECANCELED (kmc_server_wait and kmc_server_result return
 *   it; release it as any other finished job).  A job already admitted to a
 *   batch runs to the end: KMC_ESTATE, and so for a finished job.
 *   Errors: KMC_EINVAL (unknown job). */
int kmc_server_cancel(kmc_server *s, uint64_t job_id);
int kmc_server_stats_get(kmc_server *s, kmc_server_stats *st);
void kmc_server_close(kmc_server *s);

/* ---------------------------------------------------------- no allocation
 * The paper has no counterpart to this entry point; it serves callers that
 * must not allocate GPU memory.  Examples: code that runs while a CUDA graph
 * is being captured (cudaMalloc is not allowed there), a service that owns
 * a fixed memory budget or hands all device memory to its own allocator,
 * and latency-sensitive code that cannot afford the device-wide
 * synchronisation that cudaMalloc / cudaFree may cause.
 *
 * kmc_count_small_noalloc counts the canonical k-mers of a small read set
 * already in device memory and writes the result, sorted ascending by value
 * and filtered by the inclusive cutoffs, to caller-provided device arrays.
 * It allocates nothing: its only scratch is a fixed array of
 * 2 * KMC_NOALLOC_MAX_BASES 64-bit words (16 MiB) compiled into the
 * library, which every GPU that loads the library holds until the process
 * exits.
 *   d_bases / d_offsets: as in kmc_add_reads_device (device memory;
 *     d_offsets[0] == 0, non-decreasing, d_offsets[n_reads] == n_bases).
 *   n_bases: at most KMC_NOALLOC_MAX_BASES, else KMC_EINVAL and nothing runs.
 *   k: 1..32 (one 64-bit word per k-mer), else KMC_EINVAL.
 *   d_kmers / d_counts: device arrays of `capacity` entries (k-mer value
 *     right-aligned, count); entries beyond capacity are not written.
 *   d_n_out: device uint64; receives the number of k-mers in the result
 *     (possibly above capacity), or UINT64_MAX if the offsets are malformed.
 * The work is one kernel launched on cuda_stream (NULL = legacy default
 * stream) of the calling thread's current device; the call returns without
 * waiting for it.  The first call on a device looks up the scratch array's
 * device address (cudaGetSymbolAddress) with that device current; make that
 * first call before any stream capture.  All calls share the scratch array
 * and it keeps the last call's contents: calls whose kernels may overlap on
 * the GPU (different streams without ordering) race on it and give wrong
 * results; order them on one stream. */
#define KMC_NOALLOC_MAX_BASES (1u << 20)
int kmc_count_small_noalloc(const char *d_bases, const uint64_t *d_offsets, uint64_t n_reads,
                            uint64_t n_bases, uint32_t k, uint64_t cutoff_min,
                            uint64_t cutoff_max, uint64_t *d_kmers, uint32_t *d_counts,
                            uint64_t capacity, uint64_t *d_n_out, void *cuda_stream);

#define KMC_DEBUG_KEEP_SUPERKMERS 1u
#define KMC_DEBUG_KEEP_KEYS 2u
/* Sorts count tiles on 8 key bits instead of 24, so that distinct keys
 * sharing their sorted bits become common and the regrouping of such runs
 * is exercised (tests); the result is the same, only slower. */
#define KMC_DEBUG_NARROW_SORT 4u
/* Computes signatures with the tile-doubling scan kernel instead of the
 * lane-block one (both give the same super k-mers; for cross-checks). */
#define KMC_DEBUG_SIG_TILE 8u
/* Bins by canonical minimizers (the smallest canonical m-mer, no Sect. 2.2
 * filter) instead of signatures: the comparison of Sect. 2.2 and of the
 * paper's signatures-versus-minimizers table (super k-mers per read, k-mers
 * in the largest bin).  The counts are the same; kmc_db_write refuses such a
 * handle (KMC_EINVAL), the format's map being one of signatures. */
#define KMC_DEBUG_MINIMIZER 16u
/* Failure-path check of the device-side bounded waits: the tile kernel of
 * wide keys (k >= 32, x = 0) first waits, with a limit of 200 us, on an
 * mbarrier that nothing arrives on; the wait gives up, the kernel waits
 * (bounded) for its own bulk copy still in flight, reports the timeout and
 * returns, and kmc_count returns KMC_ETIMEOUT.  The handle must then be
 * closed; the CUDA context stays usable. */
#define KMC_DEBUG_WAIT_TIMEOUT 32u

/* Failure-path check of the host side: after `after` more successful device
 * or pinned host allocations of this library (any handle, any thread), the
 * next one fails as if the memory were exhausted, once; the call that made
 * it returns KMC_ENOMEM and the handle can still be closed.  after < 0
 * cancels a pending injection.  For tests only. */
int kmc_debug_fail_alloc(int64_t after);

#ifdef __cplusplus
}
#endif
#endif
