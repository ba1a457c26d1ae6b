/*
 * Plain C FP64 oracle of the Chebyshev moment loop (TEST INFRASTRUCTURE).
 *
 * Only the tests and the CPU-baseline leg of the benchmark load this file's
 * shared object; the library never does.  It repeats the method directly,
 * without any of the CUDA path's tables or layouts, for problem sizes where
 * the dense numpy oracle is too slow:
 *
 *   - states of a sector (k up spins out of N, Sec. 2) are listed in
 *     increasing order by stepping to the next integer with the same number
 *     of set bits; the full space is 0..2^N-1;
 *   - the rank of a state is the textbook combinadic sum_j C(p_j, j+1) over
 *     its set-bit positions p_0 < p_1 < ... (its position in that order);
 *   - H = sum_b J_b S_i.S_j (Eq. E-3-1-1) is applied state by state: +J/4
 *     when bits i and j agree, -J/4 and a J/2 hop to s^(1<<i|1<<j) when not;
 *   - v_0 has components sign(splitmix64(splitmix64(splitmix64(seed)^r)^s))
 *     / sqrt(D) (top bit 0 -> +1), v_1 = H'v_0, v_{n+1} = 2H'v_n - v_{n-1}
 *     with H' = (H - c)/m (Eq. E-2-3), and the moments (Eq. E-2-6, E-2-7,
 *     normalised to mu_0 = 1) follow from mu_{2n} = 2<v_n,v_n> - mu_0 and
 *     mu_{2n+1} = 2<v_{n+1},v_n> - mu_1.
 *
 * Threads: OpenMP over states (each state's row is written by one thread and
 * the dot products are summed per thread and then in thread order).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static uint64_t oracle_splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

static uint64_t binom_table[65][65];

static void init_binom(void) {
  static int done = 0;
  if (done) return;
  for (int n = 0; n <= 64; ++n) {
    for (int k = 0; k <= 64; ++k) binom_table[n][k] = 0;
    binom_table[n][0] = 1;
    for (int k = 1; k <= n; ++k)
      binom_table[n][k] = binom_table[n - 1][k - 1] + (k <= n - 1 ? binom_table[n - 1][k] : 0);
  }
  done = 1;
}

static uint64_t textbook_rank(uint64_t s) {
  uint64_t r = 0;
  int j = 0;
  /* visit the set bits from the lowest up: position p of the (j+1)-th one adds C(p, j+1) */
  while (s) {
    const int p = __builtin_ctzll(s);
    r += binom_table[p][++j];
    s &= s - 1;
  }
  return r;
}

static int popcount64(uint64_t x) {
  int c = 0;
  while (x) {
    c += (int)(x & 1ULL);
    x >>= 1;
  }
  return c;
}

int oracle_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

int64_t oracle_sector_dim(int n_sites, int n_up) {
  init_binom();
  if (n_sites < 1 || n_sites > 40) return -1;
  if (n_up < 0) return (int64_t)1 << n_sites;
  if (n_up > n_sites) return -1;
  return (int64_t)binom_table[n_sites][n_up];
}

/* Fills states[0..D) with the sector's bitstrings in increasing order. */
int oracle_sector_states(int n_sites, int n_up, uint64_t *states) {
  int64_t D = oracle_sector_dim(n_sites, n_up);
  if (D < 0) return 1;
  if (n_up < 0) {
    for (int64_t i = 0; i < D; ++i) states[i] = (uint64_t)i;
    return 0;
  }
  uint64_t s = (n_up == 0) ? 0 : ((n_up == 64) ? ~0ULL : ((1ULL << n_up) - 1));
  for (int64_t i = 0; i < D; ++i) {
    states[i] = s;
    if (s == 0) break;
    /* next integer with the same number of set bits */
    uint64_t low = s & (~s + 1);
    uint64_t ripple = s + low;
    uint64_t ones = ((s ^ ripple) >> 2) / low;
    s = ripple | ones;
  }
  return 0;
}

uint64_t oracle_rank(uint64_t s) {
  init_binom();
  return textbook_rank(s);
}

/*
 * Moments of one sector.  mu[K] always; mu_M / mu_M2 (may be NULL) receive
 * the moments weighted by M(s) = popcount(s) - N/2 and M(s)^2 when n_up < 0.
 * max_steps > 0 stops after that many matrix-vector products (a bounded
 * timing sample: later moments are left at zero).  Returns 0 on success.
 */
int oracle_kpm_moments(int n_sites, int n_bonds, const int32_t *bi, const int32_t *bj,
                       const double *J, int n_up, double m, double c, int K, int R,
                       uint64_t seed, uint64_t r0, int max_steps, double *mu, double *mu_M,
                       double *mu_M2) {
  init_binom();
  int64_t D = oracle_sector_dim(n_sites, n_up);
  if (D <= 0 || K < 2 || (K & 1) || R < 1) return 1;
  uint64_t *states = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)D);
  double *va = (double *)malloc(sizeof(double) * (size_t)D * (size_t)R);
  double *vb = (double *)malloc(sizeof(double) * (size_t)D * (size_t)R);
  double *v0 = (double *)malloc(sizeof(double) * (size_t)D * (size_t)R);
  if (!states || !va || !vb || !v0) {
    free(states); free(va); free(vb); free(v0);
    return 2;
  }
  oracle_sector_states(n_sites, n_up, states);
  const int full = n_up < 0;
  const double norm = 1.0 / sqrt((double)D);
  const uint64_t hs = oracle_splitmix64(seed);
  memset(mu, 0, sizeof(double) * (size_t)K);
  if (full && mu_M) memset(mu_M, 0, sizeof(double) * (size_t)K);
  if (full && mu_M2) memset(mu_M2, 0, sizeof(double) * (size_t)K);

#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < D; ++i)
    for (int r = 0; r < R; ++r) {
      uint64_t hr = oracle_splitmix64(hs ^ (r0 + (uint64_t)r));
      uint64_t h = oracle_splitmix64(hr ^ states[i]);
      v0[i * R + r] = ((h >> 63) ? -1.0 : 1.0) * norm;
    }

  /* step 0: v_1 = H'v_0; step n >= 1: v_{n+1} = 2H'v_n - v_{n-1} */
  const int steps = K / 2;
  const int last = (max_steps > 0 && max_steps < steps) ? max_steps : steps;
  const int nthr = oracle_num_threads();
  double *part = (double *)calloc((size_t)nthr * 6, sizeof(double));
  double *prev = v0, *cur = va, *next = vb;
  for (int step = 0; step < last; ++step) {
    const double twoa = (step == 0) ? 1.0 : 2.0;
    const double *x = (step == 0) ? v0 : cur;
    double *y = (step == 0) ? cur : next;
    const double *z = (step == 0) ? NULL : prev;
    memset(part, 0, sizeof(double) * (size_t)nthr * 6);
#pragma omp parallel num_threads(nthr)
    {
      /* <x|W|x> and <y|W|x> for W = 1, M, M^2 */
      double l_xx[3] = {0, 0, 0}, l_yx[3] = {0, 0, 0};
#pragma omp for schedule(static)
      for (int64_t i = 0; i < D; ++i) {
        uint64_t s = states[i];
        double diag = 0.0;
        double *yi = y + i * R;
        for (int r = 0; r < R; ++r) yi[r] = 0.0;
        for (int b = 0; b < n_bonds; ++b) {
          uint64_t bit_i = (s >> bi[b]) & 1ULL, bit_j = (s >> bj[b]) & 1ULL;
          if (bit_i == bit_j) {
            diag += 0.25 * J[b];
          } else {
            diag -= 0.25 * J[b];
            uint64_t t = s ^ ((1ULL << bi[b]) | (1ULL << bj[b]));
            int64_t jr = full ? (int64_t)t : (int64_t)textbook_rank(t);
            for (int r = 0; r < R; ++r) yi[r] += 0.5 * J[b] * x[jr * R + r];
          }
        }
        double Ms = (double)popcount64(s) - 0.5 * n_sites;
        double wt[3] = {1.0, Ms, Ms * Ms};
        for (int r = 0; r < R; ++r) {
          double xi = x[i * R + r];
          double hx = yi[r] + diag * xi;
          double val = twoa * (hx - c * xi) / m;
          if (z) val -= z[i * R + r];
          yi[r] = val;
          for (int q = 0; q < 3; ++q) {
            l_xx[q] += wt[q] * xi * xi;
            l_yx[q] += wt[q] * val * xi;
          }
        }
      }
#ifdef _OPENMP
      int tid = omp_get_thread_num();
#else
      int tid = 0;
#endif
      for (int q = 0; q < 3; ++q) {
        part[tid * 6 + q] = l_xx[q];
        part[tid * 6 + 3 + q] = l_yx[q];
      }
    }
    double s_xx[3] = {0, 0, 0}, s_yx[3] = {0, 0, 0};
    for (int t = 0; t < nthr; ++t)
      for (int q = 0; q < 3; ++q) {
        s_xx[q] += part[t * 6 + q];
        s_yx[q] += part[t * 6 + 3 + q];
      }
    double *outs[3] = {mu, mu_M, mu_M2};
    for (int q = 0; q < (full ? 3 : 1); ++q) {
      double *o = outs[q];
      if (!o) continue;
      if (step == 0) {
        o[0] = s_xx[q] / R;
        o[1] = s_yx[q] / R;
      } else {
        o[2 * step] = 2.0 * s_xx[q] / R - o[0];
        o[2 * step + 1] = 2.0 * s_yx[q] / R - o[1];
      }
    }
    if (step > 0) {
      double *old = prev;
      prev = cur;
      cur = next;
      next = old;
    } else {
      prev = v0;
    }
  }
  free(part);
  free(states);
  free(va);
  free(vb);
  free(v0);
  return 0;
}

/*
 * Streaming evaluation of the first moments for sectors too large to store
 * (TEST INFRASTRUCTURE).
 *
 * The recursion above keeps three vectors of the sector in memory.  For the
 * largest sectors (N = 34, D = C(34,17) = 2 333 606 220: 18.7 GB per FP64
 * vector and R = 1) that is too much for a test, yet the first moments have
 * a plain local form: the random vector v_0 is a function of the bitstring
 * alone, so
 *     v_1(s) = [ (d(s) - c) v_0(s) + sum_{b anti-aligned at s} (J_b/2) v_0(s ^ mask_b) ] / m
 *     v_2(s) = 2 [ (d(s) - c) v_1(s) + sum_{b anti-aligned at s} (J_b/2) v_1(s ^ mask_b) ] / m - v_0(s)
 * (Eq. E-2-3 for H', the three-term recursion, d(s) the diagonal of
 * Eq. E-3-1-1) can be evaluated at any single state by recomputing v_0 and
 * v_1 at its neighbours.  The moments then follow from sums over the states:
 *     mu_0 = <v0,v0>, mu_1 = <v1,v0>, mu_2 = 2<v1,v1> - mu_0,
 *     mu_3 = 2<v2,v1> - mu_1, mu_4 = 2<v2,v2> - mu_0
 * averaged over the R vectors.  The states are visited in rank order in
 * chunks of 2^16 (the first state of a chunk by the textbook inverse of the
 * colex rank); each chunk's sums are formed in FP64 and the chunk sums are
 * added in chunk order, so the result does not depend on the thread count.
 * n_mom = 3 stops after mu_2 (only v_1 is needed), n_mom = 5 gives mu_0..mu_4.
 */

/* Bitstring of colex rank r among the n-bit strings with k set bits: the
   highest set bit is the largest p with C(p, k) <= r, then the next one with
   k - 1 bits for the remainder, and so on. */
static uint64_t textbook_unrank(uint64_t r, int n_sites, int k) {
  uint64_t s = 0;
  for (int p = n_sites - 1; p >= 0 && k > 0; --p) {
    if (binom_table[p][k] <= r) {
      s |= 1ULL << p;
      r -= binom_table[p][k];
      --k;
    }
  }
  return s;
}

typedef struct {
  int n_bonds;
  const int32_t *bi, *bj;
  const double *J;
  double m, c, norm;
  uint64_t hr;
} local_model;

static double local_v0(const local_model *L, uint64_t s) {
  uint64_t h = oracle_splitmix64(L->hr ^ s);
  return ((h >> 63) ? -1.0 : 1.0) * L->norm;
}

/* (H x)(s) for x given as a function of the bitstring */
static double local_apply(const local_model *L, uint64_t s, double (*x)(const local_model *, uint64_t)) {
  double diag = 0.0, hop = 0.0;
  for (int b = 0; b < L->n_bonds; ++b) {
    uint64_t bit_i = (s >> L->bi[b]) & 1ULL, bit_j = (s >> L->bj[b]) & 1ULL;
    if (bit_i == bit_j) {
      diag += 0.25 * L->J[b];
    } else {
      diag -= 0.25 * L->J[b];
      hop += 0.5 * L->J[b] * x(L, s ^ ((1ULL << L->bi[b]) | (1ULL << L->bj[b])));
    }
  }
  return diag * x(L, s) + hop;
}

static double local_v1(const local_model *L, uint64_t s) {
  return (local_apply(L, s, local_v0) - L->c * local_v0(L, s)) / L->m;
}

static double local_v2(const local_model *L, uint64_t s) {
  return 2.0 * (local_apply(L, s, local_v1) - L->c * local_v1(L, s)) / L->m - local_v0(L, s);
}

int oracle_local_moments(int n_sites, int n_bonds, const int32_t *bi, const int32_t *bj,
                         const double *J, int n_up, double m, double c, int R, uint64_t seed,
                         uint64_t r0, int n_mom, int64_t max_states, double *mu) {
  init_binom();
  int64_t D = oracle_sector_dim(n_sites, n_up);
  if (D <= 0 || R < 1 || (n_mom != 3 && n_mom != 5) || n_sites > 40) return 1;
  const int64_t chunk = (int64_t)1 << 16;
  /* max_states > 0: only the first max_states ranks (a timing sample; the sums are
     then partial), with the normalisation of the whole sector */
  const int64_t n_states = (max_states > 0 && max_states < D) ? max_states : D;
  const int64_t n_chunks = (n_states + chunk - 1) / chunk;
  double *part = (double *)calloc((size_t)n_chunks * 5, sizeof(double));
  if (!part) return 2;
  const uint64_t hs = oracle_splitmix64(seed);
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ch = 0; ch < n_chunks; ++ch) {
    const int64_t i0 = ch * chunk;
    const int64_t i1 = (i0 + chunk < n_states) ? i0 + chunk : n_states;
    uint64_t s = (n_up < 0) ? (uint64_t)i0 : textbook_unrank((uint64_t)i0, n_sites, n_up);
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t i = i0; i < i1; ++i) {
      for (int r = 0; r < R; ++r) {
        local_model L = {n_bonds, bi, bj, J, m, c, 1.0 / sqrt((double)D),
                         oracle_splitmix64(hs ^ (r0 + (uint64_t)r))};
        const double x0 = local_v0(&L, s);
        const double x1 = local_v1(&L, s);
        acc[0] += x0 * x0;
        acc[1] += x1 * x0;
        acc[2] += x1 * x1;
        if (n_mom == 5) {
          const double x2 = local_v2(&L, s);
          acc[3] += x2 * x1;
          acc[4] += x2 * x2;
        }
      }
      if (n_up < 0) {
        ++s;
      } else if (i + 1 < i1) {
        uint64_t low = s & (~s + 1);
        uint64_t ripple = s + low;
        uint64_t ones = ((s ^ ripple) >> 2) / low;
        s = ripple | ones;
      }
    }
    for (int q = 0; q < 5; ++q) part[ch * 5 + q] = acc[q];
  }
  double tot[5] = {0, 0, 0, 0, 0};
  for (int64_t ch = 0; ch < n_chunks; ++ch)
    for (int q = 0; q < 5; ++q) tot[q] += part[ch * 5 + q];
  free(part);
  for (int q = 0; q < 5; ++q) tot[q] /= R;
  mu[0] = tot[0];
  mu[1] = tot[1];
  mu[2] = 2.0 * tot[2] - mu[0];
  if (n_mom == 5) {
    mu[3] = 2.0 * tot[3] - mu[1];
    mu[4] = 2.0 * tot[4] - mu[0];
  }
  return 0;
}

/*
 * The recursion of oracle_kpm_moments for one sector with two stored vectors
 * only (TEST INFRASTRUCTURE), for sectors whose four arrays of D entries
 * would not fit in host memory.  Same arithmetic, same steps: v_0 is
 * regenerated from the hash where it is needed (the first step), the states
 * are visited in rank order in chunks of 2^16 starting from the textbook
 * inverse of the colex rank, neighbours are found by the textbook rank, and
 * v_{n+1}(s) = 2 H' v_n(s) - v_{n-1}(s) overwrites v_{n-1}(s) in place (it
 * reads v_{n-1} at s only).  Dot products are summed per chunk in FP64 and
 * the chunk sums in chunk order.  R = 1 vector (index r0); mu[K] is filled up
 * to max_steps matrix-vector products (0 = all K/2).
 */
int oracle_kpm_moments_lean(int n_sites, int n_bonds, const int32_t *bi, const int32_t *bj,
                            const double *J, int n_up, double m, double c, int K, uint64_t seed,
                            uint64_t r0, int max_steps, double *mu) {
  init_binom();
  int64_t D = oracle_sector_dim(n_sites, n_up);
  if (D <= 0 || K < 2 || (K & 1) || n_sites > 40) return 1;
  const int full = n_up < 0;
  const double norm = 1.0 / sqrt((double)D);
  const uint64_t hr = oracle_splitmix64(oracle_splitmix64(seed) ^ r0);
  const int64_t chunk = (int64_t)1 << 16;
  const int64_t n_chunks = (D + chunk - 1) / chunk;
  double *va = (double *)malloc(sizeof(double) * (size_t)D);
  double *vb = (double *)malloc(sizeof(double) * (size_t)D);
  double *part = (double *)calloc((size_t)n_chunks * 2, sizeof(double));
  if (!va || !vb || !part) {
    free(va); free(vb); free(part);
    return 2;
  }
  memset(mu, 0, sizeof(double) * (size_t)K);
  const int steps = K / 2;
  const int last = (max_steps > 0 && max_steps < steps) ? max_steps : steps;
  /* step 0 reads v_0 from the hash and writes v_1 into va; step n >= 1 reads
     x = v_n and overwrites z = v_{n-1} with v_{n+1} */
  double *x = NULL, *z = va;
  for (int step = 0; step < last; ++step) {
    const double twoa = (step == 0) ? 1.0 : 2.0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < n_chunks; ++ch) {
      const int64_t i0 = ch * chunk;
      const int64_t i1 = (i0 + chunk < D) ? i0 + chunk : D;
      uint64_t s = full ? (uint64_t)i0 : textbook_unrank((uint64_t)i0, n_sites, n_up);
      double l_xx = 0.0, l_yx = 0.0;
      for (int64_t i = i0; i < i1; ++i) {
        double diag = 0.0, hop = 0.0;
        for (int b = 0; b < n_bonds; ++b) {
          uint64_t bit_i = (s >> bi[b]) & 1ULL, bit_j = (s >> bj[b]) & 1ULL;
          if (bit_i == bit_j) {
            diag += 0.25 * J[b];
          } else {
            diag -= 0.25 * J[b];
            uint64_t t = s ^ ((1ULL << bi[b]) | (1ULL << bj[b]));
            double xt;
            if (step == 0)
              xt = ((oracle_splitmix64(hr ^ t) >> 63) ? -1.0 : 1.0) * norm;
            else
              xt = x[full ? (int64_t)t : (int64_t)textbook_rank(t)];
            hop += 0.5 * J[b] * xt;
          }
        }
        const double xi = (step == 0) ? ((oracle_splitmix64(hr ^ s) >> 63) ? -1.0 : 1.0) * norm : x[i];
        double val = twoa * (hop + diag * xi - c * xi) / m;
        if (step > 0) val -= z[i];
        z[i] = val;
        l_xx += xi * xi;
        l_yx += val * xi;
        if (full) {
          ++s;
        } else if (i + 1 < i1) {
          uint64_t low = s & (~s + 1);
          uint64_t ripple = s + low;
          uint64_t ones = ((s ^ ripple) >> 2) / low;
          s = ripple | ones;
        }
      }
      part[2 * ch] = l_xx;
      part[2 * ch + 1] = l_yx;
    }
    double s_xx = 0.0, s_yx = 0.0;
    for (int64_t ch = 0; ch < n_chunks; ++ch) {
      s_xx += part[2 * ch];
      s_yx += part[2 * ch + 1];
    }
    if (step == 0) {
      mu[0] = s_xx;
      mu[1] = s_yx;
      x = va;   /* v_1 */
      z = vb;   /* v_0 is not stored: the next step writes v_2 = 2 H' v_1 - v_0 */
      /* fill vb with v_0 so that the next step can subtract it in place */
#pragma omp parallel for schedule(dynamic, 1)
      for (int64_t ch = 0; ch < n_chunks; ++ch) {
        const int64_t i0 = ch * chunk;
        const int64_t i1 = (i0 + chunk < D) ? i0 + chunk : D;
        uint64_t s = full ? (uint64_t)i0 : textbook_unrank((uint64_t)i0, n_sites, n_up);
        for (int64_t i = i0; i < i1; ++i) {
          vb[i] = ((oracle_splitmix64(hr ^ s) >> 63) ? -1.0 : 1.0) * norm;
          if (full) {
            ++s;
          } else if (i + 1 < i1) {
            uint64_t low = s & (~s + 1);
            uint64_t ripple = s + low;
            uint64_t ones = ((s ^ ripple) >> 2) / low;
            s = ripple | ones;
          }
        }
      }
    } else {
      mu[2 * step] = 2.0 * s_xx - mu[0];
      mu[2 * step + 1] = 2.0 * s_yx - mu[1];
      double *t = x;  /* z now holds v_{n+1}: it becomes x, x becomes z */
      x = z;
      z = t;
    }
  }
  free(va);
  free(vb);
  free(part);
  return 0;
}

/*
 * Spin-s Heisenberg models (TEST INFRASTRUCTURE): the same recursion for
 * local spin s = two_s/2 (Sec. 3.4 treats s = 5/2).  A state stores the
 * digit q_i = m_i + s of site i in bits 3i .. 3i+2 of its code; a sector is
 * the set of states with digit sum Q (total S^z = Q - N s), listed by
 * increasing code (an odometer over the digits, site 0 fastest), and the rank
 * of a state is its position in that list, found by binary search.  H =
 * sum_b J_b [S^z_i S^z_j + (S^+_i S^-_j + S^-_i S^+_j)/2] with the textbook
 * ladder elements S^+|m> = sqrt(s(s+1) - m(m+1))|m+1>,
 * S^-|m> = sqrt(s(s+1) - m(m-1))|m-1>.  Random vectors use the code in place
 * of the bitstring.  Q = -1 selects all (2s+1)^N states (then mu_M, mu_M2
 * are the M- and M^2-weighted moments).
 */
static int64_t spin_list_states(int n_sites, int two_s, int Q, uint64_t *out) {
  int q[24];
  for (int i = 0; i < n_sites; ++i) q[i] = 0;
  int64_t n = 0;
  for (;;) {
    int sum = 0;
    uint64_t code = 0;
    for (int i = 0; i < n_sites; ++i) {
      sum += q[i];
      code |= (uint64_t)q[i] << (3 * i);
    }
    if (Q < 0 || sum == Q) {
      if (out) out[n] = code;
      ++n;
    }
    int i = 0;
    while (i < n_sites && q[i] == two_s) q[i++] = 0;
    if (i == n_sites) break;
    ++q[i];
  }
  return n;
}

int64_t oracle_spin_sector_dim(int n_sites, int two_s, int Q) {
  if (n_sites < 1 || n_sites > 20 || two_s < 1 || two_s > 7) return -1;
  return spin_list_states(n_sites, two_s, Q, NULL);
}

static int64_t spin_rank(const uint64_t *states, int64_t D, uint64_t code) {
  int64_t lo = 0, hi = D - 1;
  while (lo < hi) {
    int64_t mid = (lo + hi) / 2;
    if (states[mid] < code)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

int oracle_spin_moments(int n_sites, int two_s, int n_bonds, const int32_t *bi, const int32_t *bj,
                        const double *J, int Q, double m, double c, int K, int R, uint64_t seed,
                        uint64_t r0, double *mu, double *mu_M, double *mu_M2) {
  int64_t D = oracle_spin_sector_dim(n_sites, two_s, Q);
  if (D <= 0 || K < 2 || (K & 1) || R < 1) return 1;
  uint64_t *states = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)D);
  double *v0 = (double *)malloc(sizeof(double) * (size_t)D * (size_t)R);
  double *va = (double *)malloc(sizeof(double) * (size_t)D * (size_t)R);
  double *vb = (double *)malloc(sizeof(double) * (size_t)D * (size_t)R);
  if (!states || !v0 || !va || !vb) {
    free(states); free(v0); free(va); free(vb);
    return 2;
  }
  spin_list_states(n_sites, two_s, Q, states);
  const double s = 0.5 * two_s;
  const double norm = 1.0 / sqrt((double)D);
  const uint64_t hs = oracle_splitmix64(seed);
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < D; ++i)
    for (int r = 0; r < R; ++r) {
      uint64_t h = oracle_splitmix64(oracle_splitmix64(hs ^ (r0 + (uint64_t)r)) ^ states[i]);
      v0[i * R + r] = ((h >> 63) ? -1.0 : 1.0) * norm;
    }
  const int steps = K / 2;
  const int nthr = oracle_num_threads();
  double *part = (double *)calloc((size_t)nthr * 6, sizeof(double));
  double *prev = v0, *cur = va, *next = vb;
  const int full = Q < 0;
  for (int step = 0; step < steps; ++step) {
    const double twoa = (step == 0) ? 1.0 : 2.0;
    const double *x = (step == 0) ? v0 : cur;
    double *y = (step == 0) ? cur : next;
    const double *z = (step == 0) ? NULL : prev;
    memset(part, 0, sizeof(double) * (size_t)nthr * 6);
#pragma omp parallel num_threads(nthr)
    {
      double l_xx[3] = {0, 0, 0}, l_yx[3] = {0, 0, 0};
#pragma omp for schedule(static)
      for (int64_t i = 0; i < D; ++i) {
        const uint64_t code = states[i];
        double *yi = y + i * R;
        for (int r = 0; r < R; ++r) yi[r] = 0.0;
        double diag = 0.0;
        int qsum = 0;
        for (int t = 0; t < n_sites; ++t) qsum += (int)((code >> (3 * t)) & 7);
        for (int b = 0; b < n_bonds; ++b) {
          const int qi = (int)((code >> (3 * bi[b])) & 7), qj = (int)((code >> (3 * bj[b])) & 7);
          const double mi = qi - s, mj = qj - s;
          diag += J[b] * mi * mj;
          for (int dir = 0; dir < 2; ++dir) {
            const int di = dir == 0 ? 1 : -1, dj = -di;
            const int ni = qi + di, nj = qj + dj;
            if (ni < 0 || ni > two_s || nj < 0 || nj > two_s) continue;
            const double amp = 0.5 * J[b] * sqrt(s * (s + 1) - mi * (mi + di)) *
                               sqrt(s * (s + 1) - mj * (mj + dj));
            const uint64_t nc = (code & ~((7ULL << (3 * bi[b])) | (7ULL << (3 * bj[b])))) |
                                ((uint64_t)ni << (3 * bi[b])) | ((uint64_t)nj << (3 * bj[b]));
            const int64_t jr = spin_rank(states, D, nc);
            for (int r = 0; r < R; ++r) yi[r] += amp * x[jr * R + r];
          }
        }
        const double Ms = qsum - 0.5 * n_sites * two_s;
        const double wt[3] = {1.0, Ms, Ms * Ms};
        for (int r = 0; r < R; ++r) {
          const double xi = x[i * R + r];
          double val = twoa * (yi[r] + diag * xi - c * xi) / m;
          if (z) val -= z[i * R + r];
          yi[r] = val;
          for (int qq = 0; qq < 3; ++qq) {
            l_xx[qq] += wt[qq] * xi * xi;
            l_yx[qq] += wt[qq] * val * xi;
          }
        }
      }
#ifdef _OPENMP
      int tid = omp_get_thread_num();
#else
      int tid = 0;
#endif
      for (int qq = 0; qq < 3; ++qq) {
        part[tid * 6 + qq] = l_xx[qq];
        part[tid * 6 + 3 + qq] = l_yx[qq];
      }
    }
    double s_xx[3] = {0, 0, 0}, s_yx[3] = {0, 0, 0};
    for (int t = 0; t < nthr; ++t)
      for (int qq = 0; qq < 3; ++qq) {
        s_xx[qq] += part[t * 6 + qq];
        s_yx[qq] += part[t * 6 + 3 + qq];
      }
    double *outs[3] = {mu, mu_M, mu_M2};
    for (int qq = 0; qq < (full ? 3 : 1); ++qq) {
      double *o = outs[qq];
      if (!o) continue;
      if (step == 0) {
        o[0] = s_xx[qq] / R;
        o[1] = s_yx[qq] / R;
      } else {
        o[2 * step] = 2.0 * s_xx[qq] / R - o[0];
        o[2 * step + 1] = 2.0 * s_yx[qq] / R - o[1];
      }
    }
    if (step > 0) {
      double *old = prev;
      prev = cur;
      cur = next;
      next = old;
    } else {
      prev = v0;
    }
  }
  free(part);
  free(states);
  free(v0);
  free(va);
  free(vb);
  return 0;
}
