/*
 * pqgen.c -- seeded synthetic column generator for the three-table plan
 * (dimension D, middle table M, fact table F).
 *
 * This module only draws random inputs.  It holds none of the relational
 * arithmetic (no filter, hash, join, aggregate or ranking); both the CUDA
 * path and the CPU oracle consume the arrays it writes.
 *
 * Schema (all integers, strings dictionary-encoded as in the paper, Sec. 6.1):
 *   D: key int32 dense 1..N_D, seg int8 uniform 0..4
 *   M: key int64 = 4*i + U{0..3}, dref int32 uniform over D keys,
 *      date int32 uniform 0..2405
 *   F: mkey int64 (each M key repeated U{1..7} times, in M order -- or Zipf
 *      distributed foreign keys for the skewed variant), price int64 cents
 *      uniform 90,000..10,500,000, disc int8 uniform 0..10,
 *      date2 int32 = M.date + U{1..121}
 *
 * Random numbers: a counter-based SplitMix64 stream (Steele, Lea & Flood,
 * "Fast splittable pseudorandom number generators", OOPSLA 2014): the i-th
 * value of stream s is mix64(state_s + (i+1)*GAMMA).  Because every value is
 * a pure function of (seed, stream, index), the output does not depend on the
 * number of OpenMP threads.  Bounded integers use Lemire's multiply-shift
 * (bias below range/2^64, irrelevant for synthetic data).
 * Zipf variates use rejection-inversion (Hoermann & Derflinger, ACM TOMACS
 * 1996), restated here from the method's description.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GAMMA 0xDA942042E4DD58B5ULL

static inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static inline uint64_t stream_state(uint64_t seed, uint64_t tag) {
  return mix64(mix64(seed + 0x632BE59BD9B4E019ULL) ^ (tag * 0xD1B54A32D192ED03ULL));
}

static inline uint64_t draw(uint64_t state, uint64_t i) {
  return mix64(state + (i + 1) * GAMMA);
}

static inline uint64_t bounded(uint64_t u, uint64_t range) {
  return (uint64_t)(((unsigned __int128)u * (unsigned __int128)range) >> 64);
}

static inline double unit_double(uint64_t u) {
  return (double)(u >> 11) * (1.0 / 9007199254740992.0);
}

enum {
  TAG_D_SEG = 1,
  TAG_M_KEY = 2,
  TAG_M_DREF = 3,
  TAG_M_DATE = 4,
  TAG_F_PRICE = 6,
  TAG_F_DISC = 7,
  TAG_F_DATE = 8,
  TAG_F_ZIPF = 9,
  TAG_PERM = 10,
  TAG_F_REP = 64 /* + lap */
};

int pqgen_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* D: key = i + 1, seg = U{0..4}. */
void pqgen_d(uint64_t seed, int64_t n_d, int32_t* key, int8_t* seg) {
  const uint64_t s_seg = stream_state(seed, TAG_D_SEG);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_d; ++i) {
    key[i] = (int32_t)(i + 1);
    seg[i] = (int8_t)bounded(draw(s_seg, (uint64_t)i), 5);
  }
}

/* M: key = 4 i + U{0..3}; dref = U{1..n_d}; date = U{0..2405}. */
void pqgen_m(uint64_t seed, int64_t n_m, int64_t n_d, int64_t* key, int32_t* dref,
             int32_t* date) {
  const uint64_t s_key = stream_state(seed, TAG_M_KEY);
  const uint64_t s_dref = stream_state(seed, TAG_M_DREF);
  const uint64_t s_date = stream_state(seed, TAG_M_DATE);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_m; ++i) {
    key[i] = 4 * i + (int64_t)bounded(draw(s_key, (uint64_t)i), 4);
    dref[i] = (int32_t)(1 + bounded(draw(s_dref, (uint64_t)i), (uint64_t)n_d));
    date[i] = (int32_t)bounded(draw(s_date, (uint64_t)i), 2406);
  }
}

static inline void fill_f_row(uint64_t s_price, uint64_t s_disc, uint64_t s_date, int64_t row,
                              int64_t mk, int32_t md, int64_t* mkey, int64_t* price,
                              int8_t* disc, int32_t* date2) {
  mkey[row] = mk;
  price[row] = 90000 + (int64_t)bounded(draw(s_price, (uint64_t)row), 10500000 - 90000 + 1);
  disc[row] = (int8_t)bounded(draw(s_disc, (uint64_t)row), 11);
  date2[row] = md + 1 + (int32_t)bounded(draw(s_date, (uint64_t)row), 121);
}

static inline int64_t rep_of(uint64_t s_rep, int64_t i) {
  return 1 + (int64_t)bounded(draw(s_rep, (uint64_t)i), 7);
}

/*
 * F clustered by M key: walk M rows in order, emitting r_i = U{1..7} copies of
 * each.  If all M rows are used up before n_f rows exist, a new lap over M
 * starts with fresh repeat draws; the last run is truncated at n_f.
 */
void pqgen_f_clustered(uint64_t seed, int64_t n_f, int64_t n_m, const int64_t* m_key,
                       const int32_t* m_date, int64_t* mkey, int64_t* price, int8_t* disc,
                       int32_t* date2) {
  if (n_f <= 0 || n_m <= 0) return;
  const uint64_t s_price = stream_state(seed, TAG_F_PRICE);
  const uint64_t s_disc = stream_state(seed, TAG_F_DISC);
  const uint64_t s_date = stream_state(seed, TAG_F_DATE);
  enum { MAXT = 1024 };
  int64_t part_sum[MAXT + 1];
  int64_t done = 0;
  for (int lap = 0; done < n_f; ++lap) {
    const uint64_t s_rep = stream_state(seed, (uint64_t)TAG_F_REP + (uint64_t)lap);
    int nt = pqgen_threads();
    if (nt > MAXT) nt = MAXT;
    const int64_t per = (n_m + nt - 1) / nt;
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int t = 0; t < nt; ++t) {
      int64_t lo = (int64_t)t * per, hi = lo + per;
      if (hi > n_m) hi = n_m;
      int64_t s = 0;
      for (int64_t i = lo; i < hi; ++i) s += rep_of(s_rep, i);
      part_sum[t + 1] = s;
    }
    part_sum[0] = 0;
    for (int t = 0; t < nt; ++t) part_sum[t + 1] += part_sum[t];
    const int64_t base = done;
#pragma omp parallel for schedule(static) num_threads(nt)
    for (int t = 0; t < nt; ++t) {
      int64_t lo = (int64_t)t * per, hi = lo + per;
      if (hi > n_m) hi = n_m;
      int64_t row = base + part_sum[t];
      for (int64_t i = lo; i < hi && row < n_f; ++i) {
        const int64_t r = rep_of(s_rep, i);
        for (int64_t c = 0; c < r && row < n_f; ++c, ++row)
          fill_f_row(s_price, s_disc, s_date, row, m_key[i], m_date[i], mkey, price, disc, date2);
      }
    }
    int64_t lap_rows = part_sum[nt];
    done = (base + lap_rows < n_f) ? base + lap_rows : n_f;
  }
}

/* First F row of every M row in the first lap (start[n_m] = end of lap 0,
 * clipped to n_f).  Used to cut self-consistent (M slice, F slice) pairs. */
void pqgen_f_starts(uint64_t seed, int64_t n_m, int64_t n_f, int64_t* start) {
  const uint64_t s_rep = stream_state(seed, (uint64_t)TAG_F_REP);
  int64_t row = 0;
  for (int64_t i = 0; i < n_m; ++i) {
    start[i] = row < n_f ? row : n_f;
    row += rep_of(s_rep, i);
  }
  start[n_m] = row < n_f ? row : n_f;
}

/* ---- Zipf(s) over ranks 1..n by rejection-inversion ---- */
typedef struct {
  double s, n, h_x1, h_n, sq;
} zipf_t;

static double zh(const zipf_t* z, double x) { return exp(-z->s * log(x)); }
/* H(x) = integral of x^-s, normalised so that it is continuous at s = 1. */
static double zH(const zipf_t* z, double x) {
  double lx = log(x);
  double t = (1.0 - z->s) * lx;
  if (fabs(t) < 1e-8) return lx * (1.0 + 0.5 * t);
  return expm1(t) / (1.0 - z->s);
}
static double zHinv(const zipf_t* z, double y) {
  double t = y * (1.0 - z->s);
  if (fabs(t) < 1e-8) return exp(y * (1.0 - 0.5 * t));
  return exp(log1p(t) / (1.0 - z->s));
}
static void zipf_init(zipf_t* z, double s, int64_t n) {
  z->s = s;
  z->n = (double)n;
  z->h_x1 = zH(z, 1.5) - 1.0;
  z->h_n = zH(z, z->n + 0.5);
  z->sq = 2.0 - zHinv(z, zH(z, 2.5) - zh(z, 2.0));
}
static int64_t zipf_draw(const zipf_t* z, uint64_t st, uint64_t j) {
  for (uint64_t a = 0; a < 64; ++a) {
    double u01 = unit_double(draw(st, j * 64 + a));
    double u = z->h_n + u01 * (z->h_x1 - z->h_n);
    double x = zHinv(z, u);
    double kf = floor(x + 0.5);
    if (kf < 1.0) kf = 1.0;
    if (kf > z->n) kf = z->n;
    if (kf - x <= z->sq || u >= zH(z, kf + 0.5) - zh(z, kf)) return (int64_t)kf;
  }
  return 1;
}

static int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

/*
 * F with Zipf(s) foreign keys into M (not co-partitioned): each F row draws a
 * rank k (1 = most frequent); rank k maps to M row perm(k-1) under the seeded
 * affine permutation r -> (a r + b) mod n_m.  date2 = M.date + U{1..121}.
 */
void pqgen_f_zipf(uint64_t seed, int64_t n_f, int64_t n_m, double s, const int64_t* m_key,
                  const int32_t* m_date, int64_t* mkey, int64_t* price, int8_t* disc,
                  int32_t* date2) {
  if (n_f <= 0 || n_m <= 0) return;
  const uint64_t s_price = stream_state(seed, TAG_F_PRICE);
  const uint64_t s_disc = stream_state(seed, TAG_F_DISC);
  const uint64_t s_date = stream_state(seed, TAG_F_DATE);
  const uint64_t s_z = stream_state(seed, TAG_F_ZIPF);
  const uint64_t s_p = stream_state(seed, TAG_PERM);
  int64_t a = 1 + (int64_t)bounded(draw(s_p, 0), (uint64_t)n_m);
  while (gcd64(a, n_m) != 1) ++a;
  const int64_t b = (int64_t)bounded(draw(s_p, 1), (uint64_t)n_m);
  zipf_t z;
  zipf_init(&z, s, n_m);
#pragma omp parallel for schedule(static)
  for (int64_t j = 0; j < n_f; ++j) {
    int64_t k = zipf_draw(&z, s_z, (uint64_t)j);
    int64_t m = (int64_t)(((__int128)a * (k - 1) + b) % n_m);
    fill_f_row(s_price, s_disc, s_date, j, m_key[m], m_date[m], mkey, price, disc, date2);
  }
}

/* Uniform integers and lognormal sizes for query streams (serving workload). */
void pqgen_uniform_i64(uint64_t seed, uint64_t tag, int64_t n, int64_t lo, int64_t hi,
                       int64_t* out) {
  const uint64_t st = stream_state(seed, 1000 + tag);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    out[i] = lo + (int64_t)bounded(draw(st, (uint64_t)i), (uint64_t)(hi - lo + 1));
}

void pqgen_uniform_f64(uint64_t seed, uint64_t tag, int64_t n, double* out) {
  const uint64_t st = stream_state(seed, 2000 + tag);
  for (int64_t i = 0; i < n; ++i) {
    double u = unit_double(draw(st, (uint64_t)i));
    out[i] = u > 0.0 ? u : 1.0 / 9007199254740992.0;
  }
}
