/*
 * Seeded synthetic genomes and sequencing reads.
 *
 * This file is shared by the CUDA path's benchmarks and by the CPU oracle's
 * tests as their common INPUT generator.  It holds none of the counting
 * method's arithmetic: no 2-bit coding, no k-mers, no signatures.  It only
 * writes ASCII bases ('A','C','G','T','N') and read offsets.
 *
 * Determinism: every random draw comes from splitmix64 streams keyed by
 * (seed, index), all probabilities are compared as integer thresholds, and
 * the only floating point (building the order-3 Markov table) uses + - * /
 * and sqrt, which IEEE-754 rounds identically on x86-64 and AArch64 as long
 * as FMA contraction is off (the build passes -ffp-contract=off).  So the
 * same seed gives the same bytes on both machines.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static const char kBase[4] = {'A', 'C', 'G', 'T'};

static inline uint64_t sm64_next(uint64_t *s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Independent stream number `idx` of generator `seed`. */
static inline uint64_t sm64_stream(uint64_t seed, uint64_t idx) {
  uint64_t s = seed ^ (0xD1B54A32D192ED03ull * (idx + 1));
  (void)sm64_next(&s);
  return s;
}

/* Uniform integer in [0, n) (Lemire's multiply-shift; n >= 1). */
static inline uint64_t uniform_below(uint64_t *s, uint64_t n) {
  return (uint64_t)(((unsigned __int128)sm64_next(s) * n) >> 64);
}

/* Probability -> 32-bit threshold for comparing against 32 random bits. */
static uint32_t p_to_u32(double p) {
  if (p <= 0.0) return 0;
  if (p >= 1.0) return 0xFFFFFFFFu;
  return (uint32_t)(p * 4294967296.0);
}

/* ---------------------------------------------------------------- genome */

/* iid uniform ACGT; blocks of 2^20 bases use their own stream (parallel). */
void synth_genome_iid(uint8_t *out, uint64_t n, uint64_t seed) {
  const uint64_t BLK = 1ull << 20;
  int64_t nblk = (int64_t)((n + BLK - 1) / BLK);
#pragma omp parallel for schedule(static)
  for (int64_t b = 0; b < nblk; ++b) {
    uint64_t s = sm64_stream(seed, (uint64_t)b);
    uint64_t lo = (uint64_t)b * BLK, hi = lo + BLK < n ? lo + BLK : n;
    uint64_t r = 0;
    for (uint64_t i = lo; i < hi; ++i) {
      if (((i - lo) & 31) == 0) r = sm64_next(&s);
      out[i] = (uint8_t)kBase[r & 3];
      r >>= 2;
    }
  }
}

/*
 * Order-3 Markov table: for each of the 64 contexts (last three bases, the
 * oldest in the high bits) a next-base distribution drawn from Dirichlet(1)
 * (sorted-uniform spacings), then C and G are weighted by a common factor
 * lambda found by bisection so that the chain's stationary GC fraction is
 * gc_target (within tol).  Outputs cumulative 32-bit thresholds
 * thr[ctx*3 + j] = P(next <= j) * 2^32 for j = 0,1,2.
 * Returns the achieved stationary GC fraction.
 */
static void tilt(const double *base, double lam, double *p) {
  for (int c = 0; c < 64; ++c) {
    double w[4], z = 0.0;
    for (int j = 0; j < 4; ++j) {
      w[j] = base[c * 4 + j] * ((j == 1 || j == 2) ? lam : 1.0);
      z += w[j];
    }
    for (int j = 0; j < 4; ++j) p[c * 4 + j] = w[j] / z;
  }
}

static double stationary_gc(const double *p) {
  double pi[64], nx[64];
  for (int c = 0; c < 64; ++c) pi[c] = 1.0 / 64.0;
  for (int it = 0; it < 4000; ++it) {
    for (int c = 0; c < 64; ++c) nx[c] = 0.0;
    for (int c = 0; c < 64; ++c)
      for (int j = 0; j < 4; ++j) nx[((c << 2) | j) & 63] += pi[c] * p[c * 4 + j];
    for (int c = 0; c < 64; ++c) pi[c] = nx[c];
  }
  double gc = 0.0;
  for (int c = 0; c < 64; ++c) gc += pi[c] * (p[c * 4 + 1] + p[c * 4 + 2]);
  return gc;
}

double synth_markov3_table(uint64_t seed, double gc_target, double tol, uint32_t *thr) {
  double base[256], p[256];
  uint64_t s = sm64_stream(seed, 0x4D41524Bull);
  for (int c = 0; c < 64; ++c) {
    /* Dirichlet(1,1,1,1): spacings of 3 sorted uniforms on [0,1]. */
    double u[3];
    for (int j = 0; j < 3; ++j) u[j] = (double)(sm64_next(&s) >> 11) * (1.0 / 9007199254740992.0);
    for (int a = 0; a < 3; ++a)
      for (int b = a + 1; b < 3; ++b)
        if (u[b] < u[a]) { double t = u[a]; u[a] = u[b]; u[b] = t; }
    base[c * 4 + 0] = u[0];
    base[c * 4 + 1] = u[1] - u[0];
    base[c * 4 + 2] = u[2] - u[1];
    base[c * 4 + 3] = 1.0 - u[2];
    for (int j = 0; j < 4; ++j)
      if (base[c * 4 + j] < 1e-6) base[c * 4 + j] = 1e-6; /* keep every transition possible */
  }
  double lo = 1e-4, hi = 1e4, gc = 0.0;
  for (int it = 0; it < 200; ++it) {
    double mid = __builtin_sqrt(lo * hi);
    tilt(base, mid, p);
    gc = stationary_gc(p);
    if (gc > gc_target + tol) hi = mid;
    else if (gc < gc_target - tol) lo = mid;
    else break;
  }
  for (int c = 0; c < 64; ++c) {
    double acc = 0.0;
    for (int j = 0; j < 3; ++j) {
      acc += p[c * 4 + j];
      double t = acc * 4294967296.0;
      thr[c * 3 + j] = t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
    }
  }
  return gc;
}

void synth_genome_markov3(uint8_t *out, uint64_t n, const uint32_t *thr, uint64_t seed) {
  uint64_t s = sm64_stream(seed, 0x47454E4Full);
  unsigned ctx = (unsigned)(sm64_next(&s) & 63);
  for (uint64_t i = 0; i < n; ++i) {
    uint32_t r = (uint32_t)(sm64_next(&s) >> 32);
    const uint32_t *t = thr + ctx * 3;
    unsigned b = r < t[0] ? 0u : r < t[1] ? 1u : r < t[2] ? 2u : 3u;
    out[i] = (uint8_t)kBase[b];
    ctx = ((ctx << 2) | b) & 63u;
  }
}

/*
 * Interspersed repeats: `families` consensus elements of `elem_len` iid
 * bases; `copies` copies of each, every base of a copy substituted with
 * probability `divergence` (uniformly to one of the other three bases).
 * Copies overwrite the genome in disjoint slots (genome cut into
 * families*copies equal slots, slots shuffled, random offset inside the
 * slot), so the genome length is unchanged.  Returns 0, or -1 if a slot is
 * shorter than an element.
 */
int synth_insert_repeats(uint8_t *g, uint64_t n, uint32_t families, uint32_t copies,
                         uint32_t elem_len, double divergence, uint64_t seed) {
  uint64_t total = (uint64_t)families * copies;
  if (total == 0) return 0;
  uint64_t slot = n / total;
  if (slot < elem_len) return -1;
  uint64_t *perm = (uint64_t *)malloc(total * sizeof(uint64_t));
  uint8_t *cons = (uint8_t *)malloc((size_t)elem_len);
  if (!perm || !cons) { free(perm); free(cons); return -2; }
  uint64_t s = sm64_stream(seed, 0x5245504Full);
  for (uint64_t i = 0; i < total; ++i) perm[i] = i;
  for (uint64_t i = total - 1; i > 0; --i) {
    uint64_t j = uniform_below(&s, i + 1);
    uint64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
  }
  uint32_t thr = p_to_u32(divergence);
  for (uint32_t f = 0; f < families; ++f) {
    uint64_t fs = sm64_stream(seed, 0x46414D00ull + f);
    for (uint32_t i = 0; i < elem_len; ++i) cons[i] = (uint8_t)(sm64_next(&fs) & 3);
    for (uint32_t c = 0; c < copies; ++c) {
      uint64_t idx = (uint64_t)f * copies + c;
      uint64_t cs = sm64_stream(seed, 0x434F5059000000ull + idx);
      uint64_t off = perm[idx] * slot + uniform_below(&cs, slot - elem_len + 1);
      for (uint32_t i = 0; i < elem_len; ++i) {
        unsigned b = cons[i];
        if ((uint32_t)(sm64_next(&cs) >> 32) < thr) b = (b + 1 + (unsigned)uniform_below(&cs, 3)) & 3u;
        g[off + i] = (uint8_t)kBase[b];
      }
    }
  }
  free(perm);
  free(cons);
  return 0;
}

/* ----------------------------------------------------------------- reads */

static inline uint8_t comp_ascii(uint8_t c) {
  switch (c) {
    case 'A': return 'T';
    case 'C': return 'G';
    case 'G': return 'C';
    case 'T': return 'A';
    default: return 'N';
  }
}
static inline unsigned idx_ascii(uint8_t c) {
  return c == 'A' ? 0u : c == 'C' ? 1u : c == 'G' ? 2u : 3u;
}

/*
 * Reads sampled from a genome: read i has length offsets[i+1]-offsets[i]
 * (the caller fills offsets), starts uniformly in [0, G-len], comes from
 * either strand with probability 1/2, then each base is substituted with
 * probability sub_rate (uniformly to one of the other three bases) and,
 * independently, replaced by 'N' with probability n_rate.  Read i draws
 * from stream i of `seed`, so reads are generated in parallel and the
 * result does not depend on the thread count.  Returns 0, or -1 if a read
 * is longer than the genome.
 */
int synth_reads(const uint8_t *g, uint64_t G, const uint64_t *offsets, uint64_t n_reads,
                double sub_rate, double n_rate, uint64_t seed, uint8_t *out) {
  uint32_t t_sub = p_to_u32(sub_rate), t_n = p_to_u32(n_rate);
  int bad = 0;
#pragma omp parallel for schedule(static, 4096) reduction(| : bad)
  for (int64_t ii = 0; ii < (int64_t)n_reads; ++ii) {
    uint64_t i = (uint64_t)ii;
    uint64_t L = offsets[i + 1] - offsets[i];
    if (L > G) { bad |= 1; continue; }
    uint64_t s = sm64_stream(seed, i);
    uint64_t start = uniform_below(&s, G - L + 1);
    int rev = (int)(sm64_next(&s) & 1);
    uint8_t *o = out + offsets[i];
    if (!rev) {
      memcpy(o, g + start, (size_t)L);
    } else {
      for (uint64_t j = 0; j < L; ++j) o[j] = comp_ascii(g[start + L - 1 - j]);
    }
    for (uint64_t j = 0; j < L; ++j) {
      uint64_t r = sm64_next(&s);
      if ((uint32_t)(r >> 32) < t_sub) {
        unsigned b = idx_ascii(o[j]);
        o[j] = (uint8_t)kBase[(b + 1 + (unsigned)uniform_below(&s, 3)) & 3u];
      }
      if ((uint32_t)r < t_n) o[j] = 'N';
    }
  }
  return bad ? -1 : 0;
}
