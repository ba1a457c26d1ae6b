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
  for (int p = 0; p < 64 && (s >> p); ++p)
    if ((s >> p) & 1ULL) r += binom_table[p][++j];
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
