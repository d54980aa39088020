/*
 * CPU ORACLE for KMC 2's k-mer counting (Deorowicz, Kokot, Grabowski,
 * Debudaj-Grabysz: "KMC 2: Fast and resource-frugal k-mer counting").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, __graft_entry__.smoke() and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and it never imports it.
 *
 * Everything here is written from the paper's definitions, plainly and
 * slowly, so that it can be checked against the paper by eye:
 *
 *   oracle_count          the plain definition of the result (Sect. 1 and
 *                         2.1: every k-long substring of every read,
 *                         canonicalised as the smaller of itself and its
 *                         reverse complement; Sect. 2.5 and Suppl. S1: the
 *                         count cutoffs -ci / -cx), using a hash table.
 *   oracle_signature      Sect. 2.2: canonical minimiser restricted to
 *                         m-mers that do not start with AAA or ACA and have
 *                         no AA except at their start.
 *   oracle_position_sigs  the signature of every k-mer position of a read
 *                         set (invalid positions get ORACLE_NO_KMER).
 *   oracle_superkmers     Sect. 2.1/2.4, Fig. 1: maximal runs of consecutive
 *                         k-mers sharing a signature.
 *   oracle_kxmers         Sect. 2.3, Fig. 2: split of a super k-mer into as
 *                         few (k,x)-mers as possible.
 *   oracle_bin_map        Sect. 2.4: signatures merged into bins from a
 *                         histogram of a sample (our reading of the merge
 *                         heuristic, see oracle_bin_map).
 *
 * Readings of points the paper leaves open (all listed with the design notes):
 *   - any byte other than upper-case A, C, G, T breaks a read; no k-mer
 *     spans it or a read boundary;
 *   - both count cutoffs are inclusive for kept k-mers (ci <= n <= cx);
 *   - a palindromic k-mer (equal to its reverse complement) is one k-mer;
 *   - signature rule "reading A": canonicalise each m-mer, then drop it if
 *     it breaks the rule; a k-mer with no allowed m-mer gets the sentinel
 *     signature 4^m.
 *
 * Coding (Suppl. S4, [map]): A->0, C->1, G->2, T->3; a string is a number
 * whose FIRST symbol is the MOST significant 2-bit digit ("ACGAC" = 97).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef unsigned __int128 u128;

#define ORACLE_NO_KMER 0xFFFFFFFFu

/* ------------------------------------------------------------ 2-bit code */

/* Suppl. S4 [map]: A->0, C->1, G->2, T->3; anything else is not a base. */
int oracle_code(uint8_t c) {
  switch (c) {
    case 'A': return 0;
    case 'C': return 1;
    case 'G': return 2;
    case 'T': return 3;
    default: return -1;
  }
}

/* Value of codes[0..len) with codes[0] most significant. */
static u128 value_of(const int *codes, int len) {
  u128 v = 0;
  for (int i = 0; i < len; ++i) v = (v << 2) | (u128)codes[i];
  return v;
}

/* Reverse complement of codes[0..len): read backwards, complement each
 * symbol (A<->T, C<->G, i.e. 3 - code). */
static u128 revcomp_value_of(const int *codes, int len) {
  u128 v = 0;
  for (int i = len - 1; i >= 0; --i) v = (v << 2) | (u128)(3 - codes[i]);
  return v;
}

/* ------------------------------------------------------------ signatures */

/* Sect. 2.2: an m-mer may be a signature unless it starts with AAA, starts
 * with ACA, or contains AA anywhere except at its beginning (positions 0,1).
 * `v` holds the m-mer, first symbol most significant. */
int oracle_mmer_allowed(uint32_t v, int m) {
  int s[32];
  for (int i = m - 1; i >= 0; --i) { s[i] = (int)(v & 3u); v >>= 2; }
  if (m >= 3 && s[0] == 0 && s[1] == 0 && s[2] == 0) return 0;      /* AAA... */
  if (m >= 3 && s[0] == 0 && s[1] == 1 && s[2] == 0) return 0;      /* ACA... */
  for (int i = 1; i + 1 < m; ++i)
    if (s[i] == 0 && s[i + 1] == 0) return 0;                         /* ..AA.. */
  return 1;
}

/* Sect. 2.2 (reading A): the smallest canonical m-mer of the k-mer that is
 * allowed; 4^m when no m-mer of the k-mer is allowed. */
uint32_t oracle_signature(const int *kmer, int k, int m) {
  uint32_t best = 1u << (2 * m); /* sentinel 4^m */
  for (int i = 0; i + m <= k; ++i) {
    uint32_t f = (uint32_t)value_of(kmer + i, m);
    uint32_t r = (uint32_t)revcomp_value_of(kmer + i, m);
    uint32_t c = f < r ? f : r; /* canonical m-mer (Sect. 2.1) */
    if (oracle_mmer_allowed(c, m) && c < best) best = c;
  }
  return best;
}

/* Plain (non-canonical, unfiltered) minimiser of a k-mer, Sect. 2.1. */
uint32_t oracle_plain_minimizer(const int *kmer, int k, int m) {
  uint32_t best = 0xFFFFFFFFu;
  for (int i = 0; i + m <= k; ++i) {
    uint32_t f = (uint32_t)value_of(kmer + i, m);
    if (f < best) best = f;
  }
  return best;
}

/* Codes of a read; returns the number of bases. Non-bases become -1. */
static void codes_of(const uint8_t *s, uint64_t n, int *out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = oracle_code(s[i]);
}

/* 1 if the k bases starting at codes[p] are all A/C/G/T. */
static int window_valid(const int *codes, uint64_t p, int k) {
  for (int j = 0; j < k; ++j)
    if (codes[p + j] < 0) return 0;
  return 1;
}

/*
 * Signature of every k-mer start position of the read set, in input order:
 * out[offsets[r] + p] for read r, position p.  Positions whose window is not
 * a valid k-mer (runs off the read, or holds a non-ACGT byte) get
 * ORACLE_NO_KMER.  `out` has offsets[n_reads] entries.
 */
void oracle_position_sigs(const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads,
                          int k, int m, uint32_t *out) {
  for (uint64_t r = 0; r < n_reads; ++r) {
    uint64_t a = offsets[r], L = offsets[r + 1] - a;
    int *codes = (int *)malloc((L ? L : 1) * sizeof(int));
    codes_of(bases + a, L, codes);
    for (uint64_t p = 0; p < L; ++p) {
      if (p + (uint64_t)k <= L && window_valid(codes, p, k))
        out[a + p] = oracle_signature(codes + p, k, m);
      else
        out[a + p] = ORACLE_NO_KMER;
    }
    free(codes);
  }
}

/*
 * Sect. 2.1/2.4 and Fig. 1: split one read into super k-mers, i.e. maximal
 * runs of consecutive valid k-mers that share one signature.  For each super
 * k-mer writes its first k-mer's position in the read, its number of k-mers
 * and its signature.  Returns the number of super k-mers (at most `cap` are
 * written).  `use_minimizer` = 1 uses the canonical minimiser without the
 * Sect. 2.2 filter (Fig. 1, top), for comparison.  `cut_every` > 0 also
 * starts a new super k-mer at every read position that is a multiple of it.
 */
uint64_t oracle_superkmers(const uint8_t *read, uint64_t L, int k, int m, int use_minimizer,
                           uint32_t cut_every, uint64_t *start, uint32_t *n_kmers, uint32_t *sig,
                           uint64_t cap) {
  int *codes = (int *)malloc((L ? L : 1) * sizeof(int));
  codes_of(read, L, codes);
  uint64_t n = 0;
  int open = 0;
  uint32_t cur = 0;
  for (uint64_t p = 0; p + (uint64_t)k <= L; ++p) {
    if (!window_valid(codes, p, k)) { open = 0; continue; }
    uint32_t s;
    if (use_minimizer) {
      s = 0xFFFFFFFFu;
      for (int i = 0; i + m <= k; ++i) {
        uint32_t f = (uint32_t)value_of(codes + p + i, m);
        uint32_t r = (uint32_t)revcomp_value_of(codes + p + i, m);
        uint32_t c = f < r ? f : r;
        if (c < s) s = c;
      }
    } else {
      s = oracle_signature(codes + p, k, m);
    }
    /* reading: a super k-mer may also be cut before every k-mer whose
     * position in the read is a multiple of cut_every (0 = never); this bounds
     * record sizes and leaves the counts unchanged. */
    int cut = cut_every && (p % cut_every) == 0;
    if (open && s == cur && !cut) {
      if (n - 1 < cap) n_kmers[n - 1] += 1;
    } else {
      if (n < cap) { start[n] = p; n_kmers[n] = 1; sig[n] = s; }
      ++n;
      open = 1;
      cur = s;
    }
  }
  free(codes);
  return n;
}

/* ------------------------------------------------------------ (k,x)-mers */

/*
 * Sect. 2.3 and Fig. 2: split a super k-mer (codes of n_kmers + k - 1
 * bases) into as few (k,x)-mers as possible.  A (k,x)-mer is a (k+x')-mer,
 * 0 <= x' <= x, stored in the orientation in which all of its k-mers are
 * canonical, and neighbouring (k,x)-mers share no k-mer.  k-mer i is
 * "direct" when it is not larger than its reverse complement (a palindrome
 * counts as direct).  Reading: a group is a run of consecutive k-mers of one
 * orientation, cut greedily from the left into pieces of at most x+1
 * k-mers; a run of r k-mers needs ceil(r/(x+1)) groups, the minimum, and
 * this reproduces Fig. 2.
 *
 * For group g writes: first k-mer index gstart[g], x' = xp[g], orientation
 * rev[g] (1 = stored as reverse complement) and the (k+x')-mer value
 * (first stored symbol most significant) as val_hi[g]:val_lo[g].  Returns
 * the number of groups.
 */
uint64_t oracle_kxmers(const int *codes, uint64_t n_kmers, int k, int x, uint64_t *gstart,
                       uint32_t *xp, uint32_t *rev, uint64_t *val_hi, uint64_t *val_lo,
                       uint64_t cap) {
  uint64_t g = 0;
  uint64_t i = 0;
  while (i < n_kmers) {
    int o = revcomp_value_of(codes + i, k) < value_of(codes + i, k); /* 1 = reverse */
    uint64_t len = 1;
    while (len < (uint64_t)x + 1 && i + len < n_kmers) {
      int o2 = revcomp_value_of(codes + i + len, k) < value_of(codes + i + len, k);
      if (o2 != o) break;
      ++len;
    }
    if (g < cap) {
      int span = k + (int)len - 1;
      gstart[g] = i;
      xp[g] = (uint32_t)(len - 1);
      rev[g] = (uint32_t)o;
      u128 v = o ? revcomp_value_of(codes + i, span) : value_of(codes + i, span);
      val_hi[g] = (uint64_t)(v >> 64);
      val_lo[g] = (uint64_t)v;
    }
    ++g;
    i += len;
  }
  return g;
}

/* ------------------------------------------------------------ bin map */

/*
 * Sect. 2.4: the 4^m signatures (plus the sentinel 4^m) are merged into at
 * most B bins from a histogram of signatures found in a sample of the input,
 * merging the least frequent ones.  Our reading: sort the seen signatures by
 * sample weight, heaviest first (ties: smaller signature first), and cut the
 * sorted list into consecutive groups of about total/B weight each: the
 * signature whose preceding weight sum is W goes to bin floor(W*B/total).
 * Heavy signatures thus get bins of their own and light ones share bins.
 * Unseen signatures go to bin (signature mod B).  The counting result does
 * not depend on the map.
 */
typedef struct { uint64_t w; uint32_t s; } sigw_t;
static int cmp_sigw(const void *a, const void *b) {
  const sigw_t *x = (const sigw_t *)a, *y = (const sigw_t *)b;
  if (x->w != y->w) return x->w > y->w ? -1 : 1;
  return x->s < y->s ? -1 : (x->s > y->s ? 1 : 0);
}

void oracle_bin_map(const uint64_t *weight, uint32_t n_sig, uint32_t B, uint32_t *map) {
  sigw_t *v = (sigw_t *)malloc((size_t)n_sig * sizeof(sigw_t));
  uint32_t nv = 0;
  u128 total = 0;
  for (uint32_t s = 0; s < n_sig; ++s) {
    if (weight[s]) { v[nv].w = weight[s]; v[nv].s = s; ++nv; total += weight[s]; }
    else map[s] = s % B;
  }
  qsort(v, nv, sizeof(sigw_t), cmp_sigw);
  u128 before = 0;
  for (uint32_t i = 0; i < nv; ++i) {
    map[v[i].s] = (uint32_t)((before * B) / total);
    before += v[i].w;
  }
  free(v);
}

/* ------------------------------------------------------------ counting */

/*
 * The plain definition (Sect. 1, 2.1): for every read, every k-long window
 * of A/C/G/T bases is a k-mer; its canonical form is the smaller of the
 * k-mer and its reverse complement; count each occurrence; keep the
 * canonical k-mers whose count n satisfies ci <= n <= cx (Sect. 2.5, Suppl.
 * S1 options -ci and -cx); report them sorted ascending by value.
 *
 * Memory is bounded by hash partitioning: worker t of T in pass q of P only
 * counts the k-mers whose hash h satisfies h mod (P*T) == q*T + t, so every
 * k-mer is counted by exactly one worker in exactly one pass.
 */
typedef struct {
  u128 *key;
  uint64_t *cnt;
  uint8_t *used;
  uint64_t cap, n;
} table_t;

static uint64_t hash128(u128 x) {
  uint64_t a = (uint64_t)x, b = (uint64_t)(x >> 64);
  uint64_t h = a * 0x9E3779B97F4A7C15ull ^ (b + 0x632BE59BD9B4E019ull) * 0xC2B2AE3D27D4EB4Full;
  h ^= h >> 29;
  h *= 0xBF58476D1CE4E5B9ull;
  h ^= h >> 32;
  return h;
}

static int table_init(table_t *t, uint64_t cap) {
  t->cap = cap;
  t->n = 0;
  t->key = (u128 *)malloc(cap * sizeof(u128));
  t->cnt = (uint64_t *)malloc(cap * sizeof(uint64_t));
  t->used = (uint8_t *)calloc(cap, 1);
  return (t->key && t->cnt && t->used) ? 0 : -1;
}

static void table_free(table_t *t) {
  free(t->key);
  free(t->cnt);
  free(t->used);
  memset(t, 0, sizeof(*t));
}

static int table_add(table_t *t, u128 key);

static int table_grow(table_t *t) {
  table_t nt;
  if (table_init(&nt, t->cap * 2)) return -1;
  for (uint64_t i = 0; i < t->cap; ++i) {
    if (!t->used[i]) continue;
    uint64_t h = hash128(t->key[i]) & (nt.cap - 1);
    while (nt.used[h]) h = (h + 1) & (nt.cap - 1);
    nt.used[h] = 1;
    nt.key[h] = t->key[i];
    nt.cnt[h] = t->cnt[i];
    nt.n++;
  }
  table_free(t);
  *t = nt;
  return 0;
}

static int table_add(table_t *t, u128 key) {
  if ((t->n + 1) * 2 > t->cap && table_grow(t)) return -1;
  uint64_t h = hash128(key) & (t->cap - 1);
  while (t->used[h]) {
    if (t->key[h] == key) { t->cnt[h] += 1; return 0; }
    h = (h + 1) & (t->cap - 1);
  }
  t->used[h] = 1;
  t->key[h] = key;
  t->cnt[h] = 1;
  t->n++;
  return 0;
}

typedef struct { u128 key; uint64_t cnt; } kc_t;

typedef struct {
  const uint8_t *bases;
  const uint64_t *offsets;
  uint64_t n_reads;
  int k;
  uint64_t ci, cx;
  uint64_t part, n_parts;
  kc_t *out;
  uint64_t n_out, out_cap;
  uint64_t n_pos; /* valid k-mer positions seen (all partitions) */
  int err;
  int canonical;  /* 1: canonical k-mers (Sect. 2.1); 0: as read (Suppl. S1 -b) */
} work_t;

static void *count_worker(void *arg) {
  work_t *w = (work_t *)arg;
  table_t t;
  if (table_init(&t, 1u << 16)) { w->err = -1; return NULL; }
  int codes_cap = 0;
  int *codes = NULL;
  const int k = w->k;
  for (uint64_t r = 0; r < w->n_reads; ++r) {
    uint64_t a = w->offsets[r], L = w->offsets[r + 1] - a;
    if (L < (uint64_t)k) continue;
    if ((uint64_t)codes_cap < L) {
      free(codes);
      codes_cap = (int)L;
      codes = (int *)malloc(L * sizeof(int));
    }
    codes_of(w->bases + a, L, codes);
    for (uint64_t p = 0; p + (uint64_t)k <= L; ++p) {
      if (!window_valid(codes, p, k)) continue;
      u128 f = value_of(codes + p, k);
      u128 rc = revcomp_value_of(codes + p, k);
      u128 c = (w->canonical && rc < f) ? rc : f; /* canonical k-mer, or as read */
      w->n_pos++;
      if (hash128(c) % w->n_parts != w->part) continue;
      if (table_add(&t, c)) { w->err = -1; goto done; }
    }
  }
  for (uint64_t i = 0; i < t.cap; ++i) {
    if (!t.used[i]) continue;
    if (t.cnt[i] < w->ci || t.cnt[i] > w->cx) continue; /* cutoffs, inclusive */
    if (w->n_out == w->out_cap) {
      uint64_t nc = w->out_cap ? w->out_cap * 2 : 1024;
      kc_t *no = (kc_t *)realloc(w->out, nc * sizeof(kc_t));
      if (!no) { w->err = -1; goto done; }
      w->out = no;
      w->out_cap = nc;
    }
    w->out[w->n_out].key = t.key[i];
    w->out[w->n_out].cnt = t.cnt[i];
    w->n_out++;
  }
done:
  free(codes);
  table_free(&t);
  return NULL;
}

static int cmp_kc(const void *a, const void *b) {
  const kc_t *x = (const kc_t *)a, *y = (const kc_t *)b;
  return x->key < y->key ? -1 : (x->key > y->key ? 1 : 0);
}

/*
 * Count canonical k-mers (1 <= k <= 64).  Output: n_out k-mers, each as
 * ceil(k/32) uint64 words, most significant word first, value right-aligned
 * (low 2k bits), sorted ascending; counts as uint32.  Returns 0; -1 on bad
 * arguments or allocation failure; -2 if a count exceeds UINT32_MAX; -3 if
 * `cap` is too small (n_out is still set).  n_pos_out (if not NULL) receives
 * the number of valid k-mer positions.
 */
int oracle_count_mode(const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads, int k,
                      uint64_t ci, uint64_t cx, int canonical, int n_threads, int n_passes,
                      uint64_t *out_words, uint32_t *out_counts, uint64_t cap, uint64_t *n_out,
                      uint64_t *n_pos_out);

int oracle_count(const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads, int k,
                 uint64_t ci, uint64_t cx, int n_threads, int n_passes, uint64_t *out_words,
                 uint32_t *out_counts, uint64_t cap, uint64_t *n_out, uint64_t *n_pos_out) {
  return oracle_count_mode(bases, offsets, n_reads, k, ci, cx, 1, n_threads, n_passes, out_words,
                           out_counts, cap, n_out, n_pos_out);
}

static int count_passes(const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads, int k,
                        uint64_t ci, uint64_t cx, int canonical, int n_threads, int n_passes,
                        int q_first, int q_last, uint64_t *out_words, uint32_t *out_counts,
                        uint64_t cap, uint64_t *n_out, uint64_t *n_pos_out);

/* As oracle_count; canonical = 0 counts the k-mers as they are read
 * (Suppl. S1 option -b: no transformation into canonical form). */
int oracle_count_mode(const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads, int k,
                      uint64_t ci, uint64_t cx, int canonical, int n_threads, int n_passes,
                      uint64_t *out_words, uint32_t *out_counts, uint64_t cap, uint64_t *n_out,
                      uint64_t *n_pos_out) {
  return count_passes(bases, offsets, n_reads, k, ci, cx, canonical, n_threads, n_passes, 0, n_passes,
                      out_words, out_counts, cap, n_out, n_pos_out);
}

/* One pass of oracle_count_mode with n_passes passes: the exact counts of the
 * k-mers c with (hash(c) mod (n_passes * n_threads)) div n_threads == which,
 * about 1/n_passes of them (a sample of a result too large to hold). */
int oracle_count_sample(const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads, int k,
                        uint64_t ci, uint64_t cx, int canonical, int n_threads, int n_passes, int which,
                        uint64_t *out_words, uint32_t *out_counts, uint64_t cap, uint64_t *n_out,
                        uint64_t *n_pos_out) {
  if (which < 0 || which >= n_passes) return -1;
  return count_passes(bases, offsets, n_reads, k, ci, cx, canonical, n_threads, n_passes, which, which + 1,
                      out_words, out_counts, cap, n_out, n_pos_out);
}

/* hash(c) mod n_parts of n k-mer values (ceil(k/32) words each, most
 * significant first), the class oracle_count_sample selects by. */
void oracle_hash_parts(const uint64_t *words, uint64_t n, int k, uint64_t n_parts, uint64_t *out) {
  const int w = (k + 31) / 32;
  for (uint64_t i = 0; i < n; ++i) {
    u128 v = 0;
    for (int j = 0; j < w; ++j) v = (v << 64) | words[i * w + j];
    out[i] = hash128(v) % n_parts;
  }
}

static int count_passes(const uint8_t *bases, const uint64_t *offsets, uint64_t n_reads, int k,
                        uint64_t ci, uint64_t cx, int canonical, int n_threads, int n_passes,
                        int q_first, int q_last, uint64_t *out_words, uint32_t *out_counts,
                        uint64_t cap, uint64_t *n_out, uint64_t *n_pos_out) {
  if (k < 1 || k > 64 || n_threads < 1 || n_passes < 1) return -1;
  uint64_t total = 0, npos = 0;
  int rc = 0;
  const int words = (k + 31) / 32;
  for (int q = q_first; q < q_last && rc == 0; ++q) {
    work_t *w = (work_t *)calloc((size_t)n_threads, sizeof(work_t));
    pthread_t *th = (pthread_t *)malloc((size_t)n_threads * sizeof(pthread_t));
    for (int t = 0; t < n_threads; ++t) {
      w[t].bases = bases;
      w[t].offsets = offsets;
      w[t].n_reads = n_reads;
      w[t].k = k;
      w[t].ci = ci;
      w[t].cx = cx;
      w[t].canonical = canonical;
      w[t].part = (uint64_t)q * (uint64_t)n_threads + (uint64_t)t;
      w[t].n_parts = (uint64_t)n_passes * (uint64_t)n_threads;
      if (n_threads > 1) pthread_create(&th[t], NULL, count_worker, &w[t]);
      else count_worker(&w[t]);
    }
    if (n_threads > 1)
      for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
    uint64_t pass_n = 0;
    for (int t = 0; t < n_threads; ++t) {
      if (w[t].err) rc = -1;
      pass_n += w[t].n_out;
    }
    if (q == q_first) npos = w[0].n_pos;
    kc_t *all = (kc_t *)malloc((pass_n ? pass_n : 1) * sizeof(kc_t));
    uint64_t j = 0;
    for (int t = 0; t < n_threads; ++t) {
      memcpy(all + j, w[t].out, w[t].n_out * sizeof(kc_t));
      j += w[t].n_out;
      free(w[t].out);
    }
    /* Passes hold disjoint hash classes: sort each pass, merge at the end. */
    qsort(all, pass_n, sizeof(kc_t), cmp_kc);
    for (uint64_t i = 0; i < pass_n && rc == 0; ++i) {
      if (all[i].cnt > 0xFFFFFFFFull) rc = -2;
      if (total + i < cap) {
        for (int wd = 0; wd < words; ++wd)
          out_words[(total + i) * words + wd] = (uint64_t)(all[i].key >> (64 * (words - 1 - wd)));
        out_counts[total + i] = (uint32_t)all[i].cnt;
      }
    }
    total += pass_n;
    free(all);
    free(w);
    free(th);
  }
  *n_out = total;
  if (n_pos_out) *n_pos_out = npos;
  if (rc) return rc;
  if (q_last - q_first > 1 && total <= cap) {
    /* merge the per-pass sorted runs: one more plain sort over the words */
    kc_t *all = (kc_t *)malloc((total ? total : 1) * sizeof(kc_t));
    for (uint64_t i = 0; i < total; ++i) {
      u128 v = 0;
      for (int wd = 0; wd < words; ++wd) v = (v << 64) | (u128)out_words[i * words + wd];
      all[i].key = v;
      all[i].cnt = out_counts[i];
    }
    qsort(all, total, sizeof(kc_t), cmp_kc);
    for (uint64_t i = 0; i < total; ++i) {
      for (int wd = 0; wd < words; ++wd)
        out_words[i * words + wd] = (uint64_t)(all[i].key >> (64 * (words - 1 - wd)));
      out_counts[i] = (uint32_t)all[i].cnt;
    }
    free(all);
  }
  return total > cap ? -3 : 0;
}
