// Spin-s Heisenberg models: the moment loop of Eq. E-2-6 / E-2-7 and the
// Lanczos bounds of Eq. E-2-3 / E-2-4 for local spin s > 1/2, as in the
// paper's ring of N = 10 spins s = 5/2 (Sec. 3.4).
//
// Basis.  A state stores the digit q_i = m_i + s in {0 .. 2s} of site i in
// bits 3i .. 3i+2 of its code (2s + 1 <= 8).  The total S^z = sum_i m_i
// commutes with H; sector Q holds the states of digit sum Q (M = Q - N s),
// ordered by increasing code.  With the low L = N/2 sites ("lo") and the
// high H = N - L sites ("hi") of a code,
//     rank(code) = lo_rank[lo] + hi_rank[c][hi],  c = digit sum of lo,
// where lo_rank is the position of lo among the low strings of digit sum c
// and hi_rank[c][hi] counts the states of the sector (digit sum of hi plus c)
// whose high part is smaller than hi.  The whole (2s+1)^N space is ranked by
// the base-(2s+1) value of the digits.  A hi-block is the run of ranks that
// share one hi; its lo parts are lo_list[lo_start[c] ..] in increasing order.
//
// Hamiltonian (Eq. E-3-1-1): H = sum_b J_b [S^z_i S^z_j + (S^+_i S^-_j +
// S^-_i S^+_j)/2] with S^+|m> = sqrt(s(s+1) - m(m+1))|m+1> and
// S^-|m> = sqrt(s(s+1) - m(m-1))|m-1>: per bond a diagonal J m_i m_j and up
// to two neighbours, found by changing two digits.
//
// Layout and reduction follow the spin-1/2 loop: the R random vectors are
// interleaved per state (rows of 16-byte chunks, G lanes per state), tiles of
// consecutive ranks are handed out by a per-step atomic queue, each tile's
// dot products go to its own slot and are summed per sector in tile order by
// a second kernel.  This path is matrix-free (no neighbour lists) and has no
// adjoint.  In the FP32 form every coefficient of H' is an unevaluated pair
// of floats (hi + lo), as in the spin-1/2 loop.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kpm_device.cuh"
#include "kpm_run.h"

namespace kpm {

namespace {

constexpr int kSpinMaxSites = 16;
constexpr int kSpinMaxBonds = 256;
constexpr int kSpinBits = 3;
constexpr int64_t kSpinMaxTable = int64_t(1) << 26;  // entries of the hi_rank table

struct SpinSectorDev {
  int64_t row0, dim;
  int32_t Q;          // digit sum; -1 = whole space
  int32_t out_index;
  double inv_a, b, Mval;
};

struct SpinTablesDev {
  const uint32_t *lo_rank, *hi_rank, *lo_list, *lo_start, *hb_code, *hb_off;
  const Tile *tiles;
  const SpinSectorDev *sectors;
  const int32_t *tile_begin, *tile_end;
  int32_t n_tiles, n_sectors, N, L, H, two_s, d, cmax;  // cmax = 2s L
};

struct SpinBondsDev {
  int32_t n_bonds;
  int16_t bi[kSpinMaxBonds], bj[kSpinMaxBonds];
  double J[kSpinMaxBonds];
  double cp[8], cm[8];   // S^+ and S^- matrix elements for digit q (0 outside the range)
  double s;              // spin
  int64_t dpow[kSpinMaxSites];  // d^i (whole-space ranks)
};

// Digit q of site i.
__host__ __device__ __forceinline__ int digit(uint64_t code, int i) {
  return (int)((code >> (kSpinBits * i)) & 7u);
}

// Host plan of one call.
struct SpinPlan {
  int N = 0, two_s = 0, d = 0, L = 0, H = 0, cmax = 0;
  int n_sectors = 0;
  std::vector<int> Q;
  std::vector<int64_t> dim, row0;
  int64_t total_rows = 0;
  std::vector<uint32_t> lo_rank, hi_rank, lo_list, lo_start, hb_code, hb_off;
  std::vector<int32_t> hb_begin;
  std::vector<Tile> tiles;
  std::vector<int32_t> tile_begin, tile_end;
};

int64_t pow_int(int64_t b, int e) {
  int64_t r = 1;
  for (int i = 0; i < e; ++i) r *= b;
  return r;
}

// Digit strings of n sites (codes, increasing) whose digits are all <= two_s.
std::vector<uint32_t> valid_codes(int n, int two_s) {
  std::vector<uint32_t> out;
  std::vector<int> q(n, 0);
  for (;;) {
    uint32_t code = 0;
    for (int i = 0; i < n; ++i) code |= (uint32_t)q[i] << (kSpinBits * i);
    out.push_back(code);
    int i = 0;
    while (i < n && q[i] == two_s) q[i++] = 0;
    if (i == n) break;
    ++q[i];
  }
  std::sort(out.begin(), out.end());
  return out;
}

int digit_sum(uint64_t code, int n) {
  int s = 0;
  for (int i = 0; i < n; ++i) s += digit(code, i);
  return s;
}

int validate_spin_model(const kpm_spin_model *m) {
  KPM_REQUIRE(m != nullptr, KPM_EINVAL, "model is NULL");
  KPM_REQUIRE(m->two_s >= 1 && m->two_s <= 7, KPM_EINVAL, "two_s = %d outside 1..7", m->two_s);
  KPM_REQUIRE(m->n_sites >= 1 && m->n_sites <= kSpinMaxSites, KPM_EINVAL,
              "n_sites = %d outside 1..%d", m->n_sites, kSpinMaxSites);
  KPM_REQUIRE(m->n_bonds >= 0 && m->n_bonds <= kSpinMaxBonds, KPM_EINVAL, "n_bonds = %d",
              m->n_bonds);
  KPM_REQUIRE(m->n_bonds == 0 || (m->bi && m->bj && m->J), KPM_EINVAL, "NULL bond arrays");
  for (int b = 0; b < m->n_bonds; ++b) {
    KPM_REQUIRE(m->bi[b] >= 0 && m->bi[b] < m->n_sites && m->bj[b] >= 0 &&
                    m->bj[b] < m->n_sites && m->bi[b] != m->bj[b],
                KPM_EINVAL, "bond %d = (%d, %d)", b, m->bi[b], m->bj[b]);
    KPM_REQUIRE(std::isfinite(m->J[b]), KPM_EINVAL, "J[%d] not finite", b);
  }
  return KPM_OK;
}

int build_spin_plan(const kpm_spin_model *m, int n_sectors, const int32_t *Q, int64_t tile_states,
                    SpinPlan *p) {
  KPM_TRY(validate_spin_model(m));
  KPM_REQUIRE(n_sectors >= 1 && Q != nullptr, KPM_EINVAL, "need at least one sector");
  p->N = m->n_sites;
  p->two_s = m->two_s;
  p->d = m->two_s + 1;
  p->L = p->N / 2;
  p->H = p->N - p->L;
  p->cmax = p->two_s * p->L;
  const int qmax = p->two_s * p->N;
  KPM_REQUIRE((int64_t)(p->cmax + 1) << (kSpinBits * p->H) <= kSpinMaxTable, KPM_EINVAL,
              "N = %d, 2s = %d: rank tables too large", p->N, p->two_s);
  for (int i = 0; i < n_sectors; ++i)
    KPM_REQUIRE(Q[i] >= -1 && Q[i] <= qmax, KPM_EINVAL, "sector %d: Q = %d outside -1..%d", i,
                Q[i], qmax);
  p->n_sectors = n_sectors;
  p->Q.assign(Q, Q + n_sectors);
  // low strings by digit sum
  const std::vector<uint32_t> lo_codes = valid_codes(p->L, p->two_s);
  const std::vector<uint32_t> hi_codes = valid_codes(p->H, p->two_s);
  std::vector<int64_t> n_lo(p->cmax + 1, 0);
  p->lo_rank.assign((size_t)1 << (kSpinBits * p->L), 0u);
  for (uint32_t c : lo_codes) p->lo_rank[c] = (uint32_t)n_lo[digit_sum(c, p->L)]++;
  p->lo_start.assign(p->cmax + 2, 0u);
  for (int c = 0; c <= p->cmax; ++c) p->lo_start[c + 1] = p->lo_start[c] + (uint32_t)n_lo[c];
  p->lo_list.assign(lo_codes.size(), 0u);
  {
    std::vector<uint32_t> fill(p->lo_start.begin(), p->lo_start.end() - 1);
    for (uint32_t c : lo_codes) p->lo_list[fill[digit_sum(c, p->L)]++] = c;
  }
  // hi_rank[c][hi]: states of sector (sum(hi) + c) with a smaller high part
  const size_t nhi = (size_t)1 << (kSpinBits * p->H);
  p->hi_rank.assign((size_t)(p->cmax + 1) * nhi, 0u);
  std::vector<int64_t> run(qmax + 1, 0);
  for (uint32_t h : hi_codes) {
    const int sh = digit_sum(h, p->H);
    for (int c = 0; c <= p->cmax; ++c) {
      const int q = sh + c;
      KPM_REQUIRE(run[q] < (int64_t)UINT32_MAX, KPM_EINVAL, "sector too large for 32-bit ranks");
      p->hi_rank[(size_t)c * nhi + h] = (uint32_t)run[q];
    }
    for (int q = 0; q <= qmax; ++q) {
      const int c = q - sh;
      if (c >= 0 && c <= p->cmax) run[q] += n_lo[c];
    }
  }
  // sectors, hi-blocks and tiles
  p->dim.resize(n_sectors);
  p->row0.resize(n_sectors);
  p->hb_begin.resize(n_sectors + 1);
  p->hb_code.clear();
  p->hb_off.clear();
  p->tiles.clear();
  p->tile_begin.resize(n_sectors);
  p->tile_end.resize(n_sectors);
  int64_t rows = 0;
  for (int i = 0; i < n_sectors; ++i) {
    const int q = Q[i];
    p->hb_begin[i] = (int32_t)p->hb_code.size();
    int64_t D = 0;
    if (q < 0) {
      D = pow_int(p->d, p->N);
    } else {
      for (uint32_t h : hi_codes) {
        const int c = q - digit_sum(h, p->H);
        if (c < 0 || c > p->cmax || n_lo[c] == 0) continue;
        p->hb_code.push_back(h);
        p->hb_off.push_back((uint32_t)D);
        D += n_lo[c];
      }
    }
    KPM_REQUIRE(D > 0, KPM_EINVAL, "sector %d (Q = %d) is empty", i, q);
    KPM_REQUIRE(D < (int64_t)UINT32_MAX, KPM_EINVAL, "sector %d: dimension %lld too large", i,
                (long long)D);
    p->dim[i] = D;
    p->row0[i] = rows;
    rows += D;
    p->tile_begin[i] = (int32_t)p->tiles.size();
    uint32_t b = (uint32_t)p->hb_begin[i];
    const uint32_t b_end = (uint32_t)p->hb_code.size();
    for (int64_t r0 = 0; r0 < D; r0 += tile_states) {
      Tile t{};
      t.row0 = p->row0[i] + r0;
      t.rank0 = (uint32_t)r0;
      t.count = (uint32_t)std::min<int64_t>(tile_states, D - r0);
      t.sector = i;
      if (q >= 0) {
        while (b + 1 < b_end && p->hb_off[b + 1] <= (uint32_t)r0) ++b;
        t.b_first = b;
        uint32_t bl = b;
        const uint32_t r_last = (uint32_t)(r0 + t.count - 1);
        while (bl + 1 < b_end && p->hb_off[bl + 1] <= r_last) ++bl;
        t.b_last = bl;
      }
      p->tiles.push_back(t);
    }
    p->tile_end[i] = (int32_t)p->tiles.size();
  }
  p->hb_begin[n_sectors] = (int32_t)p->hb_code.size();
  p->total_rows = rows;
  KPM_REQUIRE(p->tiles.size() < (size_t)INT32_MAX, KPM_EINVAL, "too many tiles");
  return KPM_OK;
}

void fill_spin_bonds(const kpm_spin_model *m, SpinBondsDev *b) {
  std::memset(b, 0, sizeof(*b));
  b->n_bonds = m->n_bonds;
  for (int k = 0; k < m->n_bonds; ++k) {
    b->bi[k] = (int16_t)m->bi[k];
    b->bj[k] = (int16_t)m->bj[k];
    b->J[k] = m->J[k];
  }
  const double s = 0.5 * m->two_s;
  b->s = s;
  for (int q = 0; q < 8; ++q) {
    const double mm = q - s;
    b->cp[q] = q < m->two_s ? std::sqrt(s * (s + 1) - mm * (mm + 1)) : 0.0;
    b->cm[q] = (q > 0 && q <= m->two_s) ? std::sqrt(s * (s + 1) - mm * (mm - 1)) : 0.0;
  }
  int64_t p = 1;
  for (int i = 0; i < kSpinMaxSites; ++i) {
    b->dpow[i] = p;
    p *= (m->two_s + 1);
  }
}

// Code of rank r in sector Q (hi-block walk forward from b, as in the spin-1/2 loop).
__device__ __forceinline__ uint64_t spin_unrank(uint32_t r, int Q, uint32_t b_last, uint32_t &b,
                                                const SpinTablesDev &tb) {
  while (b < b_last && __ldg(tb.hb_off + b + 1) <= r) ++b;
  const uint32_t hi = __ldg(tb.hb_code + b);
  int sh = 0;
  for (int i = 0; i < tb.H; ++i) sh += digit(hi, i);
  const int c = Q - sh;
  const uint32_t lo = __ldg(tb.lo_list + __ldg(tb.lo_start + c) + (r - __ldg(tb.hb_off + b)));
  return ((uint64_t)hi << (kSpinBits * tb.L)) | lo;
}

// Code of whole-space rank r (base-d digits).
__device__ __forceinline__ uint64_t spin_full_code(int64_t r, const SpinTablesDev &tb) {
  uint64_t code = 0;
  for (int i = 0; i < tb.N; ++i) {
    code |= (uint64_t)(r % tb.d) << (kSpinBits * i);
    r /= tb.d;
  }
  return code;
}

__device__ __forceinline__ int64_t spin_rank(uint64_t code, int c, const SpinTablesDev &tb) {
  const uint32_t lo = (uint32_t)(code & ((1ull << (kSpinBits * tb.L)) - 1));
  const uint32_t hi = (uint32_t)(code >> (kSpinBits * tb.L));
  return (int64_t)__ldg(tb.lo_rank + lo) +
         (int64_t)__ldg(tb.hi_rank + ((size_t)c << (kSpinBits * tb.H)) + hi);
}

// Calls f(neighbour row, amplitude) for every off-diagonal element of H in
// the column of state `code` (row `row`, rank `rank` in its sector) and
// returns the diagonal element.
template <typename F>
__device__ __forceinline__ double spin_apply(uint64_t code, int64_t rank, const SpinSectorDev &sd,
                                             const SpinTablesDev &tb, const SpinBondsDev &bd,
                                             F &&f) {
  const bool full = sd.Q < 0;
  int clo = 0;
  if (!full)
    for (int i = 0; i < tb.L; ++i) clo += digit(code, i);
  double diag = 0.0;
  for (int b = 0; b < bd.n_bonds; ++b) {
    const int i = bd.bi[b], j = bd.bj[b];
    const int qi = digit(code, i), qj = digit(code, j);
    const double J = bd.J[b];
    diag += J * (qi - bd.s) * (qj - bd.s);
    // S^+_i S^-_j (dir 0) and S^-_i S^+_j (dir 1)
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const int di = dir == 0 ? 1 : -1;
      const double amp = 0.5 * J * (dir == 0 ? bd.cp[qi] * bd.cm[qj] : bd.cm[qi] * bd.cp[qj]);
      if (amp == 0.0) continue;
      const uint64_t nc = (uint64_t)((int64_t)code + (int64_t)di * ((int64_t)1 << (kSpinBits * i)) -
                                     (int64_t)di * ((int64_t)1 << (kSpinBits * j)));
      int64_t nr;
      if (full) {
        nr = rank + di * (bd.dpow[i] - bd.dpow[j]);
      } else {
        const int c2 = clo + (i < tb.L ? di : 0) - (j < tb.L ? di : 0);
        nr = spin_rank(nc, c2, tb);
      }
      f(sd.row0 + nr, amp);
    }
  }
  return diag;
}

struct SpinStepArgs {
  const void *x;
  void *zy;
  SpinTablesDev tb;
  double *partials;  // [n_tiles][NQ]
  int *queue;
  int Rp, G, gpw, first, NQ;
  double half_q;     // N s (M = digit sum - N s)
};

template <typename T, int CPL>
__global__ void __launch_bounds__(kThreads)
    spin_step_kernel(const __grid_constant__ SpinStepArgs a, const __grid_constant__ SpinBondsDev bd) {
  using C = Chunk<T>;
  using V = typename C::type;
  constexpr bool PAIR = sizeof(T) == 4;
  __shared__ double s_red[kWarps * 6];
  __shared__ int s_tile;
  const V *__restrict__ x = reinterpret_cast<const V *>(a.x);
  V *__restrict__ zy = reinterpret_cast<V *>(a.zy);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / a.G, sub = lane - grp * a.G;
  const bool active = grp < a.gpw;
  const int64_t crow = a.Rp / C::W;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.queue, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= a.tb.n_tiles) break;
    const Tile tile = a.tb.tiles[t];
    const SpinSectorDev sd = a.tb.sectors[tile.sector];
    const double A = (a.first ? 1.0 : 2.0) * sd.inv_a;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    uint32_t hb = tile.b_first;
    if (active) {
      for (uint32_t u = warp * a.gpw + grp; u < tile.count; u += kWarps * a.gpw) {
        const int64_t row = tile.row0 + u;
        const int64_t rank = (int64_t)tile.rank0 + u;
        const uint64_t code =
            sd.Q < 0 ? spin_full_code(rank, a.tb) : spin_unrank((uint32_t)rank, sd.Q, tile.b_last, hb, a.tb);
        V h[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) h[c] = V{};
        const double diag = spin_apply(code, rank, sd, a.tb, bd, [&](int64_t nrow, double amp) {
          const double coef = A * amp;
          const T hi = (T)coef;
          const T lo = PAIR ? (T)(coef - (double)hi) : (T)0;
          const V *src = x + nrow * crow + sub;
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const V v = __ldg(src + c * a.G);
            h[c] = C::fma(hi, v, h[c]);
            if (PAIR) h[c] = C::fma(lo, v, h[c]);
          }
        });
        const double ad = A * (diag - sd.b);
        const T ad_hi = (T)ad;
        const T ad_lo = PAIR ? (T)(ad - (double)ad_hi) : (T)0;
        const double M = sd.Q < 0 ? 0.0 : sd.Mval;
        double Ms = M;
        if (sd.Q < 0) {
          int q = 0;
          for (int i = 0; i < a.tb.N; ++i) q += digit(code, i);
          Ms = q - a.half_q;
        }
        double pxx = 0.0, pyx = 0.0;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int64_t idx = row * crow + sub + c * a.G;
          const V xv = x[idx];
          const V zv = a.first ? V{} : zy[idx];
          V hh = h[c];
          if (PAIR) hh = C::fma(ad_lo, xv, hh);
          const V y = C::fma_sub(ad_hi, xv, hh, zv);
          zy[idx] = y;
#pragma unroll
          for (int e = 0; e < C::W; ++e) {
            const double xe = (double)C::get(xv, e), ye = (double)C::get(y, e);
            pxx = fma(xe, xe, pxx);
            pyx = fma(ye, xe, pyx);
          }
        }
        acc[0] += pxx;
        acc[1] += pyx;
        acc[2] += Ms * pxx;
        acc[3] += Ms * pyx;
        acc[4] += Ms * Ms * pxx;
        acc[5] += Ms * Ms * pyx;
      }
    }
    block_sum<6>(acc, s_red);
    if (threadIdx.x == 0)
      for (int q = 0; q < a.NQ; ++q) a.partials[(int64_t)t * a.NQ + q] = acc[q];
  }
}

// sums[sec][q] = sum over the sector's tiles in tile order; one block per sector.
__global__ void __launch_bounds__(kThreads)
    spin_reduce_kernel(const double *partials, SpinTablesDev tb, int NQ, double *sums) {
  __shared__ double s_red[kWarps * 6];
  const int sec = blockIdx.x;
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int t = tb.tile_begin[sec] + threadIdx.x; t < tb.tile_end[sec]; t += kThreads)
    for (int q = 0; q < NQ; ++q) v[q] += partials[(int64_t)t * NQ + q];
  block_sum<6>(v, s_red);
  if (threadIdx.x == 0)
    for (int q = 0; q < NQ; ++q) sums[(int64_t)sec * NQ + q] = v[q];
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
    spin_init_kernel(void *v0, SpinTablesDev tb, uint64_t seed, uint64_t r0, int R, int Rp, int G,
                     int gpw, int uniform) {
  using C = Chunk<T>;
  using V = typename C::type;
  __shared__ uint64_t s_hr[512];
  const uint64_t hs = splitmix64(seed);
  for (int col = threadIdx.x; col < R; col += kThreads) s_hr[col] = splitmix64(hs ^ (r0 + (uint64_t)col));
  __syncthreads();
  V *v = reinterpret_cast<V *>(v0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / G, sub = lane - grp * G;
  if (grp >= gpw) return;
  const int crow = Rp / C::W;
  for (int t = blockIdx.x; t < tb.n_tiles; t += gridDim.x) {
    const Tile tile = tb.tiles[t];
    const SpinSectorDev sd = tb.sectors[tile.sector];
    const T norm = (T)(1.0 / sqrt((double)sd.dim));
    uint32_t hb = tile.b_first;
    for (uint32_t u = warp * gpw + grp; u < tile.count; u += kWarps * gpw) {
      const int64_t row = tile.row0 + u;
      const int64_t rank = (int64_t)tile.rank0 + u;
      const uint64_t code =
          sd.Q < 0 ? spin_full_code(rank, tb) : spin_unrank((uint32_t)rank, sd.Q, tile.b_last, hb, tb);
      for (int ch = sub; ch < crow; ch += G) {
        V val;
#pragma unroll
        for (int e = 0; e < C::W; ++e) {
          const int col = ch * C::W + e;
          T xv = 0;
          if (col < R) {
            const uint64_t h = splitmix64(s_hr[col] ^ code);
            xv = uniform ? (T)(2.0 * (((double)(h >> 11) + 0.5) * 0x1.0p-53) - 1.0)
                         : ((h >> 63) ? -norm : norm);
          }
          C::set(val, e, xv);
        }
        v[row * crow + ch] = val;
      }
    }
  }
}

// mu[out][n] (and mu_M, mu_M2) from the per-step sums, as in the spin-1/2 loop.
__global__ void spin_assemble_kernel(const double *sums, const SpinSectorDev *sectors, double *mu,
                                     double *mu_M, double *mu_M2, int *flag, int n_sectors, int K,
                                     int NQ, double inv_R) {
  const int total = n_sectors * K;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int sec = i / K, n = i - sec * K;
    const int step = n / 2, odd = n & 1;
    const bool full = sectors[sec].Q < 0;
    for (int q = 0; q < 3; ++q) {
      double *out = q == 0 ? mu : (q == 1 ? mu_M : mu_M2);
      if (!out) continue;
      const int qq = (full ? 2 * q : 0) + odd;
      const double raw = sums[((int64_t)step * n_sectors + sec) * NQ + qq] * inv_R;
      const double base = sums[(int64_t)sec * NQ + qq] * inv_R;
      double val = step == 0 ? raw : 2.0 * raw - base;
      if (!full && q > 0) val *= q == 1 ? sectors[sec].Mval : sectors[sec].Mval * sectors[sec].Mval;
      out[(int64_t)sectors[sec].out_index * K + n] = val;
      if (q == 0 && !(fabs(val) <= 1.0 + 1e-6)) atomicOr(flag, 1);
    }
  }
}

// Lanczos kernels of the spin-s bounds, one thread per state on rows of 2 doubles:
// mode 1: P = H Q - coef P, out = <P, Q>; mode 2: P -= coef Q, out = |P|^2;
// mode 3: P /= coef.  Per-tile sums go to partials.
struct SpinLanczosArgs {
  double2 *P;
  const double2 *Q;
  SpinTablesDev tb;
  double *partials;
  const double *coef;  // [n_sectors]
  int *queue;
  int mode;
};

__global__ void __launch_bounds__(kThreads)
    spin_lanczos_kernel(const __grid_constant__ SpinLanczosArgs a, const __grid_constant__ SpinBondsDev bd) {
  __shared__ double s_red[kWarps];
  __shared__ int s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.queue, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= a.tb.n_tiles) break;
    const Tile tile = a.tb.tiles[t];
    const SpinSectorDev sd = a.tb.sectors[tile.sector];
    const double c0 = a.coef[tile.sector];
    double acc[1] = {0.0};
    uint32_t hb = tile.b_first;
    for (uint32_t u = threadIdx.x; u < tile.count; u += kThreads) {
      const int64_t row = tile.row0 + u;
      if (a.mode == 1) {
        const int64_t rank = (int64_t)tile.rank0 + u;
        const uint64_t code = sd.Q < 0 ? spin_full_code(rank, a.tb)
                                       : spin_unrank((uint32_t)rank, sd.Q, tile.b_last, hb, a.tb);
        double h = 0.0;
        const double diag = spin_apply(code, rank, sd, a.tb, bd, [&](int64_t nrow, double amp) {
          h = fma(amp, __ldg(&a.Q[nrow].x), h);
        });
        const double q = a.Q[row].x;
        const double w = fma(diag, q, h) - c0 * a.P[row].x;
        a.P[row].x = w;
        acc[0] = fma(w, q, acc[0]);
      } else if (a.mode == 2) {
        const double w = a.P[row].x - c0 * a.Q[row].x;
        a.P[row].x = w;
        acc[0] = fma(w, w, acc[0]);
      } else {
        a.P[row].x = c0 > 0.0 ? a.P[row].x / c0 : 0.0;
      }
    }
    block_sum<1>(acc, s_red);
    if (threadIdx.x == 0) a.partials[t] = acc[0];
  }
}

// out[sec] = sum of the sector's tile partials (mode sqrt: square root).
__global__ void spin_lanczos_reduce_kernel(const double *partials, SpinTablesDev tb, double *out,
                                           int take_sqrt) {
  __shared__ double s_red[kWarps];
  const int sec = blockIdx.x;
  double v[1] = {0.0};
  for (int t = tb.tile_begin[sec] + threadIdx.x; t < tb.tile_end[sec]; t += kThreads) v[0] += partials[t];
  block_sum<1>(v, s_red);
  if (threadIdx.x == 0) out[sec] = take_sqrt ? sqrt(v[0]) : v[0];
}

// Device state of one spin-s call.
struct SpinRun {
  SpinPlan plan;
  RowLayout lay;
  SpinBondsDev bonds;
  SpinTablesDev tb{};
  int NQ = 2;
  int grid = 1;
  size_t vec_bytes = 0;
};

int64_t spin_tile_states(const RowLayout &lay, int64_t rows) {
  const int64_t big = (int64_t)16 * kWarps * lay.gpw;
  const int64_t small = std::max<int64_t>((int64_t)kWarps * lay.gpw, rows / (4 * 152));
  return std::max<int64_t>(1, std::min(big, small));
}

int prepare_spin(const kpm_spin_model *m, int n_sectors, const int32_t *Q, int R, int precision,
                 SpinRun *run) {
  KPM_TRY(validate_spin_model(m));
  KPM_TRY(make_layout(R, precision, &run->lay));
  int64_t rows = 0;
  SpinPlan probe;
  KPM_TRY(build_spin_plan(m, n_sectors, Q, int64_t(1) << 40, &probe));
  rows = probe.total_rows;
  KPM_TRY(build_spin_plan(m, n_sectors, Q, spin_tile_states(run->lay, rows), &run->plan));
  fill_spin_bonds(m, &run->bonds);
  bool full = false;
  for (int i = 0; i < n_sectors; ++i) full |= Q[i] < 0;
  run->NQ = full ? 6 : 2;
  run->vec_bytes = align256((size_t)run->plan.total_rows * run->lay.Rp * run->lay.elem);
  return KPM_OK;
}

size_t spin_tables_bytes(const SpinPlan &p) {
  return align256(p.lo_rank.size() * 4) + align256(p.hi_rank.size() * 4) +
         align256(p.lo_list.size() * 4) + align256(p.lo_start.size() * 4) +
         align256(std::max<size_t>(1, p.hb_code.size()) * 4) +
         align256(std::max<size_t>(1, p.hb_off.size()) * 4) + align256(p.tiles.size() * sizeof(Tile)) +
         align256(p.n_sectors * sizeof(SpinSectorDev)) + 2 * align256(p.n_sectors * 4);
}

template <typename U>
int put(Arena &ar, const std::vector<U> &v, const U **out, cudaStream_t s) {
  U *d = ar.take<U>(std::max<size_t>(1, v.size()));
  KPM_REQUIRE(d != nullptr, KPM_ENOMEM, "scratch too small for the spin tables");
  if (!v.empty()) KPM_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(U), cudaMemcpyHostToDevice, s));
  *out = d;
  return KPM_OK;
}

int upload_spin(SpinRun &r, const double *a, const double *b, Arena &ar, cudaStream_t s) {
  const SpinPlan &p = r.plan;
  std::vector<SpinSectorDev> sec(p.n_sectors);
  for (int i = 0; i < p.n_sectors; ++i) {
    KPM_REQUIRE(a[i] > 0.0 && std::isfinite(a[i]) && std::isfinite(b[i]), KPM_EINVAL,
                "sector %d: a = %g, b = %g", i, a[i], b[i]);
    sec[i].row0 = p.row0[i];
    sec[i].dim = p.dim[i];
    sec[i].Q = p.Q[i];
    sec[i].out_index = i;
    sec[i].inv_a = 1.0 / a[i];
    sec[i].b = b[i];
    sec[i].Mval = p.Q[i] < 0 ? 0.0 : p.Q[i] - 0.5 * p.N * p.two_s;
  }
  SpinTablesDev &tb = r.tb;
  KPM_TRY(put(ar, p.lo_rank, &tb.lo_rank, s));
  KPM_TRY(put(ar, p.hi_rank, &tb.hi_rank, s));
  KPM_TRY(put(ar, p.lo_list, &tb.lo_list, s));
  KPM_TRY(put(ar, p.lo_start, &tb.lo_start, s));
  KPM_TRY(put(ar, p.hb_code, &tb.hb_code, s));
  KPM_TRY(put(ar, p.hb_off, &tb.hb_off, s));
  KPM_TRY(put(ar, p.tiles, &tb.tiles, s));
  KPM_TRY(put(ar, sec, &tb.sectors, s));
  KPM_TRY(put(ar, p.tile_begin, &tb.tile_begin, s));
  KPM_TRY(put(ar, p.tile_end, &tb.tile_end, s));
  tb.n_tiles = (int32_t)p.tiles.size();
  tb.n_sectors = p.n_sectors;
  tb.N = p.N;
  tb.L = p.L;
  tb.H = p.H;
  tb.two_s = p.two_s;
  tb.d = p.d;
  tb.cmax = p.cmax;
  return KPM_OK;
}

template <typename T, int CPL>
void *spin_step_ptr() {
  return reinterpret_cast<void *>(&spin_step_kernel<T, CPL>);
}

void *pick_spin_step(int precision, int cpl) {
  if (precision == KPM_FP32) {
    switch (cpl) {
      case 1: return spin_step_ptr<float, 1>();
      case 2: return spin_step_ptr<float, 2>();
      case 3: return spin_step_ptr<float, 3>();
      case 4: return spin_step_ptr<float, 4>();
      default: return spin_step_ptr<float, 8>();
    }
  }
  switch (cpl) {
    case 1: return spin_step_ptr<double, 1>();
    case 2: return spin_step_ptr<double, 2>();
    case 3: return spin_step_ptr<double, 3>();
    case 4: return spin_step_ptr<double, 4>();
    default: return spin_step_ptr<double, 8>();
  }
}

int spin_grid(void *fn, int64_t n_tiles) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0) != cudaSuccess) per_sm = 1;
  return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * sm_count(), n_tiles));
}

// Releases a stream-ordered allocation when the call returns, also on errors.
struct StreamAlloc {
  void *p = nullptr;
  cudaStream_t s = nullptr;
  ~StreamAlloc() {
    if (p) {
      cudaFreeAsync(p, s);
      cudaStreamSynchronize(s);
    }
  }
};

}  // namespace

}  // namespace kpm

using namespace kpm;

extern "C" int64_t kpm_spin_sector_dim(int32_t n_sites, int32_t two_s, int32_t Q) {
  if (two_s < 1 || two_s > 7 || n_sites < 1 || n_sites > kSpinMaxSites) return -1;
  const int qmax = two_s * n_sites;
  if (Q < -1 || Q > qmax) return -1;
  // coefficient of x^Q in (1 + x + .. + x^{2s})^N by repeated convolution
  std::vector<int64_t> poly(1, 1);
  for (int i = 0; i < n_sites; ++i) {
    std::vector<int64_t> nxt(poly.size() + two_s, 0);
    for (size_t k = 0; k < poly.size(); ++k)
      for (int q = 0; q <= two_s; ++q) nxt[k + q] += poly[k];
    poly.swap(nxt);
  }
  if (Q < 0) {
    int64_t t = 0;
    for (int64_t v : poly) t += v;
    return t;
  }
  return poly[Q];
}

extern "C" int kpm_spin_moments(const kpm_spin_model *model, int32_t n_sectors, const int32_t *Q,
                                const double *a, const double *b, int32_t n_moments, int32_t R,
                                uint64_t seed, uint64_t r0, int32_t precision, double *mu,
                                double *mu_M, double *mu_M2, int32_t on_device, void *stream_ptr) {
  clear_error();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_ptr);
  KPM_REQUIRE(mu && a && b, KPM_EINVAL, "NULL argument");
  KPM_REQUIRE(n_moments >= 2 && n_moments % 2 == 0, KPM_EINVAL, "n_moments = %d", n_moments);
  SpinRun r;
  KPM_TRY(prepare_spin(model, n_sectors, Q, R, precision, &r));
  const int S = n_moments / 2;
  const size_t SK = (size_t)n_sectors * n_moments;
  const size_t bytes = 2 * r.vec_bytes + spin_tables_bytes(r.plan) +
                       align256(r.plan.tiles.size() * r.NQ * 8) +
                       align256((size_t)S * n_sectors * r.NQ * 8) + align256((size_t)S * 4) + 256 +
                       (on_device ? 0 : 3 * align256(SK * 8)) + 4096;
  StreamAlloc mem;
  mem.s = s;
  KPM_CUDA(cudaMallocAsync(&mem.p, bytes, s));
  Arena ar{reinterpret_cast<char *>(mem.p), bytes, 0};
  void *vA = ar.take<char>(r.vec_bytes), *vB = ar.take<char>(r.vec_bytes);
  double *partials = ar.take<double>(r.plan.tiles.size() * r.NQ);
  double *sums = ar.take<double>((size_t)S * n_sectors * r.NQ);
  int *queues = ar.take<int>(S);
  int *flag = ar.take<int>(1);
  KPM_REQUIRE(vA && vB && partials && sums && queues && flag, KPM_ENOMEM, "scratch too small");
  KPM_TRY(upload_spin(r, a, b, ar, s));
  double *dmu = mu, *dmuM = mu_M, *dmuM2 = mu_M2;
  if (!on_device) {
    dmu = ar.take<double>(SK);
    dmuM = mu_M ? ar.take<double>(SK) : nullptr;
    dmuM2 = mu_M2 ? ar.take<double>(SK) : nullptr;
  }
  KPM_CUDA(cudaMemsetAsync(queues, 0, (size_t)S * 4, s));
  KPM_CUDA(cudaMemsetAsync(flag, 0, 4, s));
  const int igrid = (int)std::min<int64_t>((int64_t)r.plan.tiles.size(), (int64_t)8 * sm_count());
  if (precision == KPM_FP32)
    spin_init_kernel<float><<<igrid, kThreads, 0, s>>>(vA, r.tb, seed, r0, R, r.lay.Rp, r.lay.G, r.lay.gpw, 0);
  else
    spin_init_kernel<double><<<igrid, kThreads, 0, s>>>(vA, r.tb, seed, r0, R, r.lay.Rp, r.lay.G, r.lay.gpw, 0);
  KPM_CUDA(cudaGetLastError());
  void *fn = pick_spin_step(precision, r.lay.cpl);
  const int grid = spin_grid(fn, (int64_t)r.plan.tiles.size());
  SpinStepArgs sa;
  sa.tb = r.tb;
  sa.partials = partials;
  sa.Rp = r.lay.Rp;
  sa.G = r.lay.G;
  sa.gpw = r.lay.gpw;
  sa.NQ = r.NQ;
  sa.half_q = 0.5 * r.plan.N * r.plan.two_s;
  void *x = vA, *zy = vB;
  for (int step = 0; step < S; ++step) {
    sa.x = x;
    sa.zy = zy;
    sa.first = step == 0 ? 1 : 0;
    sa.queue = queues + step;
    void *args[] = {(void *)&sa, (void *)&r.bonds};
    KPM_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, 0, s));
    spin_reduce_kernel<<<n_sectors, kThreads, 0, s>>>(partials, r.tb, r.NQ,
                                                      sums + (size_t)step * n_sectors * r.NQ);
    KPM_CUDA(cudaGetLastError());
    count_launches(2);
    if (step == 0) {
      // x = v_0, zy = v_1: the next step reads v_1 and overwrites v_0 with v_2
      std::swap(x, zy);
    } else {
      std::swap(x, zy);
    }
  }
  spin_assemble_kernel<<<(int)std::min<size_t>(4096, (SK + 255) / 256), 256, 0, s>>>(
      sums, r.tb.sectors, dmu, dmuM, dmuM2, flag, n_sectors, n_moments, r.NQ, 1.0 / R);
  KPM_CUDA(cudaGetLastError());
  count_launches(2);
  int hflag = 0;
  if (!on_device) {
    KPM_CUDA(cudaMemcpyAsync(mu, dmu, SK * 8, cudaMemcpyDeviceToHost, s));
    if (mu_M) KPM_CUDA(cudaMemcpyAsync(mu_M, dmuM, SK * 8, cudaMemcpyDeviceToHost, s));
    if (mu_M2) KPM_CUDA(cudaMemcpyAsync(mu_M2, dmuM2, SK * 8, cudaMemcpyDeviceToHost, s));
  }
  KPM_CUDA(cudaMemcpyAsync(&hflag, flag, 4, cudaMemcpyDeviceToHost, s));
  KPM_CUDA(cudaStreamSynchronize(s));
  if (hflag) {
    set_error("some |mu_n| > 1 + 1e-6: the rescaled spectrum leaves [-1, 1]");
    return KPM_EBOUNDS;
  }
  return KPM_OK;
}

extern "C" int kpm_spin_bounds(const kpm_spin_model *model, int32_t n_sectors, const int32_t *Q,
                               double eps, int32_t max_iter, double tol, uint64_t seed,
                               double *a_out, double *b_out, double *e_min, double *e_max,
                               void *stream_ptr) {
  clear_error();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_ptr);
  KPM_REQUIRE(a_out && b_out, KPM_EINVAL, "a and b outputs are required");
  KPM_REQUIRE(max_iter >= 1 && max_iter <= 1000, KPM_EINVAL, "max_iter = %d", max_iter);
  KPM_REQUIRE(eps >= 0.0 && eps < 2.0, KPM_EINVAL, "eps = %g", eps);
  SpinRun r;
  KPM_TRY(prepare_spin(model, n_sectors, Q, 2, KPM_FP64, &r));
  const size_t nt = r.plan.tiles.size();
  const size_t bytes = 2 * r.vec_bytes + spin_tables_bytes(r.plan) + align256(nt * 8) +
                       4 * align256((size_t)n_sectors * 8) + align256((size_t)4 * (max_iter + 2) * 4) + 4096;
  StreamAlloc mem;
  mem.s = s;
  KPM_CUDA(cudaMallocAsync(&mem.p, bytes, s));
  Arena ar{reinterpret_cast<char *>(mem.p), bytes, 0};
  double2 *P = ar.take<double2>(r.vec_bytes / 16), *Qv = ar.take<double2>(r.vec_bytes / 16);
  double *partials = ar.take<double>(nt);
  double *d_coef = ar.take<double>(n_sectors), *d_out = ar.take<double>(n_sectors);
  double *d_zero = ar.take<double>(n_sectors), *d_norm = ar.take<double>(n_sectors);
  int *queues = ar.take<int>((size_t)4 * (max_iter + 2));
  KPM_REQUIRE(P && Qv && partials && d_coef && d_out && d_zero && d_norm && queues, KPM_ENOMEM,
              "scratch too small");
  std::vector<double> ones(n_sectors, 1.0);
  KPM_TRY(upload_spin(r, ones.data(), std::vector<double>(n_sectors, 0.0).data(), ar, s));
  KPM_CUDA(cudaMemsetAsync(queues, 0, (size_t)4 * (max_iter + 2) * 4, s));
  KPM_CUDA(cudaMemsetAsync(d_zero, 0, n_sectors * 8, s));
  const int igrid = (int)std::min<int64_t>((int64_t)nt, (int64_t)8 * sm_count());
  spin_init_kernel<double><<<igrid, kThreads, 0, s>>>(P, r.tb, seed, 0, 1, r.lay.Rp, r.lay.G, r.lay.gpw, 1);
  KPM_CUDA(cudaGetLastError());
  const int grid = spin_grid((void *)spin_lanczos_kernel, (int64_t)nt);
  int qslot = 0;
  auto lanczos = [&](int mode, double2 *Pp, const double2 *Qq, const double *coef, double *out,
                     int take_sqrt) -> int {
    SpinLanczosArgs la;
    la.P = Pp;
    la.Q = Qq;
    la.tb = r.tb;
    la.partials = partials;
    la.coef = coef;
    la.queue = queues + qslot++;
    la.mode = mode;
    void *args[] = {(void *)&la, (void *)&r.bonds};
    KPM_CUDA(cudaLaunchKernel((void *)spin_lanczos_kernel, dim3(grid), dim3(kThreads), args, 0, s));
    count_launches(1);
    if (out) {
      spin_lanczos_reduce_kernel<<<n_sectors, kThreads, 0, s>>>(partials, r.tb, out, take_sqrt);
      KPM_CUDA(cudaGetLastError());
      count_launches(1);
    }
    return KPM_OK;
  };
  // normalise the start vector (P): |P| with alpha = 0, then P /= |P|
  KPM_TRY(lanczos(2, P, Qv, d_zero, d_norm, 1));
  KPM_TRY(lanczos(3, P, Qv, d_norm, nullptr, 0));
  std::swap(P, Qv);  // Qv = q_0
  KPM_CUDA(cudaMemsetAsync(P, 0, r.vec_bytes, s));
  std::vector<std::vector<double>> al(n_sectors), be(n_sectors);
  for (int i = 0; i < n_sectors; ++i) be[i].push_back(0.0);
  std::vector<double> h_alpha(n_sectors), h_beta(n_sectors, 0.0);
  std::vector<int> active(n_sectors, 1);
  double jabs = 0.0;
  for (int k = 0; k < model->n_bonds; ++k) jabs += std::fabs(model->J[k]);
  const double spin = 0.5 * model->two_s;
  const double breakdown = 1e-12 * std::max(1.0, jabs * spin * (spin + 1));
  std::vector<double> lo_s(n_sectors), hi_s(n_sectors), worst_s(n_sectors);
  int it = 0;
  for (; it < max_iter; ++it) {
    if (qslot + 4 > 4 * (max_iter + 2)) break;
    // w = H q_j - beta_j q_{j-1}; alpha_j = <w, q_j>
    KPM_CUDA(cudaMemcpyAsync(d_coef, h_beta.data(), n_sectors * 8, cudaMemcpyHostToDevice, s));
    KPM_TRY(lanczos(1, P, Qv, d_coef, d_out, 0));
    KPM_CUDA(cudaMemcpyAsync(h_alpha.data(), d_out, n_sectors * 8, cudaMemcpyDeviceToHost, s));
    KPM_CUDA(cudaStreamSynchronize(s));
    // w -= alpha_j q_j; beta_{j+1} = |w|
    KPM_CUDA(cudaMemcpyAsync(d_coef, h_alpha.data(), n_sectors * 8, cudaMemcpyHostToDevice, s));
    KPM_TRY(lanczos(2, P, Qv, d_coef, d_out, 1));
    std::vector<double> bnext(n_sectors);
    KPM_CUDA(cudaMemcpyAsync(bnext.data(), d_out, n_sectors * 8, cudaMemcpyDeviceToHost, s));
    KPM_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < n_sectors; ++i) {
      if (!active[i]) {
        bnext[i] = 0.0;
        continue;
      }
      al[i].push_back(h_alpha[i]);
      if (bnext[i] <= breakdown || (int64_t)al[i].size() >= r.plan.dim[i]) {
        be[i].push_back(0.0);
        active[i] = 0;
        bnext[i] = 0.0;
      } else {
        be[i].push_back(bnext[i]);
      }
    }
    // q_{j+1} = w / beta_{j+1} (sectors that stopped get zero rows)
    KPM_CUDA(cudaMemcpyAsync(d_coef, bnext.data(), n_sectors * 8, cudaMemcpyHostToDevice, s));
    KPM_TRY(lanczos(3, P, Qv, d_coef, nullptr, 0));
    std::swap(P, Qv);  // Qv = q_{j+1}, P = q_j
    h_beta = bnext;
    bool any = false;
    for (int i = 0; i < n_sectors; ++i) any |= active[i] != 0;
    // convergence check every 8 steps
    if (!any || (it + 1) % 8 == 0 || it + 1 == max_iter) {
      double worst_all = 0.0;
      for (int i = 0; i < n_sectors; ++i) {
        const int m = (int)al[i].size();
        const double bres = std::fabs(be[i].back());
        const double tmin = tridiag_eig(al[i], be[i], m, 0);
        const double tmax = tridiag_eig(al[i], be[i], m, m - 1);
        const double rmin = bres * ritz_last_component(al[i], be[i], m, tmin);
        const double rmax = bres * ritz_last_component(al[i], be[i], m, tmax);
        lo_s[i] = tmin - rmin;
        hi_s[i] = tmax + rmax;
        worst_s[i] = std::max(rmin / std::max(1.0, std::fabs(tmin)), rmax / std::max(1.0, std::fabs(tmax)));
        worst_all = std::max(worst_all, worst_s[i]);
      }
      if (!any || worst_all <= tol) {
        ++it;
        break;
      }
    }
  }
  int status = KPM_OK;
  for (int i = 0; i < n_sectors; ++i) {
    if (worst_s[i] > tol) status = KPM_ENOTCONV;
    double m_ = (hi_s[i] - lo_s[i]) / (2.0 - eps);
    const double c_ = 0.5 * (hi_s[i] + lo_s[i]);
    m_ = std::max(m_, 1e-12 * std::max(1.0, std::fabs(c_)));
    a_out[i] = m_;
    b_out[i] = c_;
    if (e_min) e_min[i] = lo_s[i];
    if (e_max) e_max[i] = hi_s[i];
  }
  if (status == KPM_ENOTCONV) set_error("spin Lanczos residual bound above tol after %d steps", it);
  return status;
}
