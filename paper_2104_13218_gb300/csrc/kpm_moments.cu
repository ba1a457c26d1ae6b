// The hot loop of the method: stochastic Chebyshev moments (Eq. E-2-6, E-2-7)
// by the three-term recursion v_{n+1} = 2 H' v_n - v_{n-1} with
// H' = (H - b)/a (Eq. E-2-3), H the Heisenberg Hamiltonian of Eq. E-3-1-1
// applied matrix-free on S^z bitstrings.
//
// Layout: the R random vectors of a sector are interleaved per basis state
// (row = state, Rp >= R values per row, 16-byte chunks), all sectors stacked
// in one array, so one pass over the rows serves every vector and every
// sector.  One fused kernel per recursion step reads v_n (own row and the
// rows of the bit-flipped neighbours) and v_{n-1}, writes v_{n+1} over
// v_{n-1} and produces the two dot products <v_n|v_n> and <v_{n+1}|v_n>
// (and their M- and M^2-weighted forms for a full-space run) from which
// mu_{2n} = 2<v_n|v_n> - mu_0 and mu_{2n+1} = 2<v_{n+1}|v_n> - mu_1.
// Tiles of consecutive states are handed out by a per-step atomic queue to a
// persistent grid (to blocks in the matrix-free kernel, to single warps in
// the neighbour-list kernel); each tile's partial sums are written to its own
// slot and reduced in tile order (by the last block to finish, or at the
// start of the next step), so results do not depend on the schedule.
#include <cmath>
#include <cstdio>
#include <mutex>
#include <type_traits>
#include <vector>

#include "kpm_device.cuh"
#include "kpm_run.h"

namespace kpm {

struct StepArgs {
  const void *x;
  void *zy;
  TablesDev tb;
  double *partials;
  double *sums;     // this step's [n_sectors][NQ]
  int *queue;
  int *done;
  int Rp, G, gpw, first;
  double half_n;    // N/2
  // list kernel only: the previous step's tile slot and its sums ([n_sectors][NQ]),
  // reduced at the start of this step (NULL on the first step)
  const double *prev_partials;
  double *prev_sums;
};

constexpr int kGB = 4;  // neighbour rows gathered per batch in the cooperative path

// Minimum resident blocks per SM requested from the compiler for the step kernel.
#ifndef KPM_STEP_MIN_BLOCKS
#define KPM_STEP_MIN_BLOCKS 3
#endif

template <typename T, int CPL, bool FULL>
__global__ void __launch_bounds__(kThreads, KPM_STEP_MIN_BLOCKS)
    cheb_step_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ BondsDev bd) {
  using C = Chunk<T>;
  using V = typename C::type;
  constexpr int W = C::W;
  constexpr int NQ = FULL ? 6 : 2;
  // The FP32 form carries every coefficient of H' as an unevaluated sum hi + lo
  // of two floats: rounding the operator itself to FP32 would perturb it the
  // same way at every step and shift its spectrum; with the pair, the
  // remaining FP32 rounding (of the vectors and the sums) changes from step
  // to step.
  constexpr bool PAIR = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  T *s_dh = reinterpret_cast<T *>(s_dyn);  // diagonal A (d - b), hi part, [table_size]
  T *s_dl = s_dh + bd.table_size;          // lo part (FP32 only)
  __shared__ T s_aj[kMaxBonds];            // per-bond path: A J_b / 2
  __shared__ T s_jh[kMaxBonds];            // per-bond path: J_b / 2
  __shared__ T s_gh[kMaxGroups], s_gl[kMaxGroups];  // grouped path: A J_g / 2 = hi + lo
  __shared__ double s_red[kWarps * NQ];
  __shared__ int s_tile;
  __shared__ int s_last;
  __shared__ int s_sec;

  const V *__restrict__ x = reinterpret_cast<const V *>(a.x);
  V *__restrict__ zy = reinterpret_cast<V *>(a.zy);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / a.G, sub = lane - grp * a.G;
  const bool active = grp < a.gpw;
  const int64_t crow = a.Rp / W;  // chunks per row
  const int nb = bd.n_bonds;
  const bool grouped = bd.n_groups > 0;
  for (int b = threadIdx.x; b < nb; b += kThreads) s_jh[b] = (T)(0.5 * bd.J[b]);
  if (threadIdx.x == 0) s_sec = -1;

  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.queue, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= a.tb.n_tiles) break;
    const Tile tile = a.tb.tiles[t];
    const SectorDev sd = a.tb.sectors[tile.sector];
    const double A = (a.first ? 1.0 : 2.0) * sd.inv_a;
    if (s_sec != tile.sector) {
      // coefficients of this sector's H' (rebuilt only when the sector changes)
      __syncthreads();
      if (grouped) {
        if (threadIdx.x < bd.n_groups) {
          const double c = A * 0.5 * bd.gJ[threadIdx.x];
          const T hi = (T)c;
          s_gh[threadIdx.x] = hi;
          s_gl[threadIdx.x] = PAIR ? (T)(c - (double)hi) : (T)0;
        }
        for (int idx = threadIdx.x; idx < bd.table_size; idx += kThreads) {
          double d = bd.J_quarter_sum;
          for (int g = 0; g < bd.n_groups; ++g) {
            const int size = bd.gstart[g + 1] - bd.gstart[g];
            const int ng = (idx / bd.tstride[g]) % (size + 1);
            d -= ng * (0.5 * bd.gJ[g]);
          }
          const double ad = A * (d - sd.b);
          const T hi = (T)ad;
          s_dh[idx] = hi;
          if (PAIR) s_dl[idx] = (T)(ad - (double)hi);
        }
      } else {
        for (int b = threadIdx.x; b < nb; b += kThreads) s_aj[b] = (T)(A * 0.5 * bd.J[b]);
      }
      __syncthreads();
      if (threadIdx.x == 0) s_sec = tile.sector;
    }
    __syncthreads();

    double acc64[NQ];
    KahanF accf[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc64[q] = 0.0;
    const T A_t = (T)A, b_t = (T)sd.b;
    // FULL only adds the M-weighted dot products; each tile decides its own basis
    const bool full_tile = sd.n_up < 0;
    uint32_t hb = tile.b_first;
    const int G = a.G;
    const bool coop = G >= 2;
    const int gbase = grp * G;  // first lane of this lane's group (idle lanes: past the groups)
    const uint32_t gmaskG = G >= 32 ? 0xffffffffu : ((1u << G) - 1u);
    // Which states this warp visits.  Cooperative layouts: a contiguous run of
    // the tile per warp (groups of the warp take consecutive states), so that a
    // group steps to its next state arithmetically when gpw <= 4; one-lane
    // layouts: the warp's 32 lanes take 32 consecutive states per iteration.
    uint32_t u_begin, u_end, u_step;
    if (coop) {
      const uint32_t per = ((tile.count + kWarps - 1) / kWarps + a.gpw - 1) / a.gpw * a.gpw;
      u_begin = min(tile.count, warp * per);
      u_end = min(tile.count, u_begin + per);
      u_step = a.gpw;
    } else {
      u_begin = warp * a.gpw;
      u_end = tile.count;
      u_step = kWarps * a.gpw;
    }
    const bool stepping = coop && a.gpw <= 4 && !full_tile;
    uint64_t s_next = 0;
    if (stepping && active && u_begin + grp < u_end)
      s_next = sector_unrank_search(tile.rank0 + u_begin + grp, sd.n_up, tile.b_first, tile.b_last,
                                    a.tb);
    // Warp-uniform loop over the warp's states, so that ballots and shuffles see all lanes.
    for (uint32_t ub = u_begin; ub < u_end; ub += u_step) {
      const uint32_t u = ub + grp;
      const bool valid = active && u < u_end;
      uint64_t s = 0;
      int64_t row = 0;
      V xv[CPL], zv[CPL];
      if (valid) {
        row = tile.row0 + u;
        if (full_tile) {
          s = (uint64_t)(row - sd.row0);
        } else if (stepping) {
          s = s_next;
          uint64_t t = s;
          for (int i = 0; i < a.gpw; ++i) t = next_same_popcount(t);
          s_next = t;
        } else {
          s = sector_unrank(tile.rank0 + u, sd.n_up, tile.b_last, hb, a.tb);
        }
        // own rows early: their latency overlaps the bond pass and the gathers
        const V *xo = x + row * crow + sub;
        const V *zo = zy + row * crow + sub;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          xv[c] = xo[c * G];
          zv[c] = a.first ? V{} : __ldcs(zo + c * G);
        }
      }
      V acc[CPL];
#pragma unroll
      for (int c = 0; c < CPL; ++c) acc[c] = V{};
      T ad_hi = 0, ad_lo = 0;
      if (coop) {
        // The G lanes of a group share the state: in pass p lane `sub` tests bond
        // p*G + sub; the ranks of the anti-aligned bonds' neighbours are then
        // shuffled to every lane of the group, each of which gathers its chunks.
        int tidx = 0;
        T dsum = 0;
        for (int p = 0; p < bd.n_pass; ++p) {
          const int b = p * G + sub;
          bool fl = false;
          uint32_t nc = 0;  // first 16-byte chunk of the neighbour's row (< 2^32, checked on the host)
          if (valid && b < nb) {
            const uint64_t m = bd.mask[b];
            const uint64_t tt = s & m;
            if (tt != 0 && tt != m) {
              fl = true;
              const uint64_t f = s ^ m;
              const uint32_t rk = full_tile ? (uint32_t)f : sector_rank(f, a.tb);
              nc = ((uint32_t)sd.row0 + rk) * (uint32_t)crow;
            }
          }
          const uint32_t F =
              (uint32_t)(((uint64_t)__ballot_sync(0xffffffffu, fl) >> gbase) & gmaskG);
          if (grouped) {
#pragma unroll
            for (int g = 0; g < kMaxGroups; ++g) {
              if (g < bd.n_groups) {
                uint32_t Fg = F & bd.pmask[p][g];
                tidx += __popc(Fg) * bd.tstride[g];
                const int nmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)__popc(Fg));
                V gs[CPL];
#pragma unroll
                for (int c = 0; c < CPL; ++c) gs[c] = V{};
                // batches of kGB neighbours: all shuffles, then all loads, then the sums
                for (int i = 0; i < nmax; i += kGB) {
                  uint32_t ci[kGB];
                  bool ok[kGB];
#pragma unroll
                  for (int q = 0; q < kGB; ++q) {
                    ok[q] = Fg != 0;
                    const int j = ok[q] ? __ffs(Fg) - 1 : 0;
                    ci[q] = __shfl_sync(0xffffffffu, nc, (gbase + j) & 31);
                    if (ok[q]) Fg &= Fg - 1;
                  }
                  V v[kGB][CPL];
#pragma unroll
                  for (int q = 0; q < kGB; ++q) {
#pragma unroll
                    for (int c = 0; c < CPL; ++c) v[q][c] = ok[q] ? __ldg(x + ci[q] + sub + c * G) : V{};
                  }
#pragma unroll
                  for (int q = 0; q < kGB; ++q) {
#pragma unroll
                    for (int c = 0; c < CPL; ++c) gs[c] = C::add(gs[c], v[q][c]);
                  }
                }
                const T gh = s_gh[g], gl = s_gl[g];
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                  acc[c] = C::fma(gh, gs[c], acc[c]);
                  if (PAIR) acc[c] = C::fma(gl, gs[c], acc[c]);
                }
              }
            }
          } else {
            uint32_t Fb = F;
            const int nmax = (int)__reduce_max_sync(0xffffffffu, (unsigned)__popc(Fb));
            for (int i = 0; i < nmax; ++i) {
              const int j = Fb ? __ffs(Fb) - 1 : 0;
              const uint32_t cidx = __shfl_sync(0xffffffffu, nc, (gbase + j) & 31);
              if (Fb) {
                Fb &= Fb - 1;
                const int bb = p * G + j;
                const T aj = s_aj[bb];
                dsum += s_jh[bb];
                const V *src = x + cidx + sub;
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[c] = C::fma(aj, __ldg(src + c * G), acc[c]);
              }
            }
          }
        }
        if (grouped) {
          ad_hi = s_dh[tidx];
          if (PAIR) ad_lo = s_dl[tidx];
        } else {
          ad_hi = A_t * (((T)bd.J_quarter_sum - dsum) - b_t);
        }
      } else if (valid) {
        // one lane per state: the lane walks all bonds itself
        if (grouped) {
          int tidx = 0;
#pragma unroll
          for (int g = 0; g < kMaxGroups; ++g) {
            if (g < bd.n_groups) {
              V gs[CPL];
#pragma unroll
              for (int c = 0; c < CPL; ++c) gs[c] = V{};
              int cnt = 0;
              const int k1 = bd.gstart[g + 1];
              for (int k0 = bd.gstart[g]; k0 < k1; k0 += 8) {
                int64_t nrow[8];
                bool fl[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  fl[j] = false;
                  nrow[j] = 0;
                  if (k0 + j < k1) {
                    const uint64_t m = bd.mask[bd.order[k0 + j]];
                    const uint64_t tt = s & m;
                    if (tt != 0 && tt != m) {
                      fl[j] = true;
                      const uint64_t f = s ^ m;
                      nrow[j] = sd.row0 + (full_tile ? (int64_t)f : (int64_t)sector_rank(f, a.tb));
                    }
                  }
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                  if (fl[j]) {
                    ++cnt;
                    const V *src = x + nrow[j] * crow + sub;
#pragma unroll
                    for (int c = 0; c < CPL; ++c) gs[c] = C::add(gs[c], __ldg(src + c * G));
                  }
                }
              }
              tidx += cnt * bd.tstride[g];
              const T gh = s_gh[g], gl = s_gl[g];
#pragma unroll
              for (int c = 0; c < CPL; ++c) {
                acc[c] = C::fma(gh, gs[c], acc[c]);
                if (PAIR) acc[c] = C::fma(gl, gs[c], acc[c]);
              }
            }
          }
          ad_hi = s_dh[tidx];
          if (PAIR) ad_lo = s_dl[tidx];
        } else {
          T d = (T)bd.J_quarter_sum;
          for (int b0 = 0; b0 < nb; b0 += 8) {
            int64_t nrow[8];
            bool fl[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int b = b0 + j;
              fl[j] = false;
              nrow[j] = 0;
              if (b < nb) {
                const uint64_t m = bd.mask[b];
                const uint64_t tt = s & m;
                if (tt != 0 && tt != m) {
                  fl[j] = true;
                  d -= s_jh[b];
                  const uint64_t f = s ^ m;
                  nrow[j] = sd.row0 + (full_tile ? (int64_t)f : (int64_t)sector_rank(f, a.tb));
                }
              }
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              if (fl[j]) {
                const T aj = s_aj[b0 + j];
                const V *src = x + nrow[j] * crow + sub;
#pragma unroll
                for (int c = 0; c < CPL; ++c) acc[c] = C::fma(aj, __ldg(src + c * G), acc[c]);
              }
            }
          }
          ad_hi = A_t * (d - b_t);
        }
      }
      if (valid) {
        V *zo = zy + row * crow + sub;
        using P2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
        P2 paa{}, pba{};
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          V h = acc[c];
          if (PAIR) h = C::fma(ad_lo, xv[c], h);
          const V y = C::fma_sub(ad_hi, xv[c], h, zv[c]);
          C::dots(xv[c], y, paa, pba);
          __stcs(zo + c * G, y);
        }
        const T pxx = paa.x + paa.y, pyx = pba.x + pba.y;
        if constexpr (sizeof(T) == 8) {
          acc64[0] += pxx;
          acc64[1] += pyx;
          if (FULL) {
            const double M = (double)__popcll(s) - a.half_n;
            acc64[2] += M * pxx;
            acc64[3] += M * pyx;
            acc64[4] += M * M * pxx;
            acc64[5] += M * M * pyx;
          }
        } else {
          accf[0].add(pxx);
          accf[1].add(pyx);
          if (FULL) {
            const float M = (float)__popcll(s) - (float)a.half_n;
            accf[2].add(M * pxx);
            accf[3].add(M * pyx);
            accf[4].add(M * M * pxx);
            accf[5].add(M * M * pyx);
          }
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc64[q] = accf[q].value();
    }
    block_sum<NQ>(acc64, s_red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) a.partials[(int64_t)t * NQ + q] = acc64[q];
    }
  }

  // The last block to finish sums the tile partials of every sector in tile order.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(a.done, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (int sec = warp; sec < a.tb.n_sectors; sec += kWarps) {
      const int t0 = a.tb.tile_begin[sec], t1 = a.tb.tile_end[sec];
      double v[NQ];
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] = 0.0;
      for (int t = t0 + lane; t < t1; t += 32) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) v[q] += __ldcg(a.partials + (int64_t)t * NQ + q);
      }
#pragma unroll
      for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
      if (lane == 0) {
#pragma unroll
        for (int q = 0; q < NQ; ++q) a.sums[sec * NQ + q] = v[q];
      }
    }
  }
}

// ---------------------------------------------------------------- neighbour lists
// The structure of H' does not change during a run: for every basis state the
// anti-aligned bonds and the ranks of the bit-flipped neighbours are found
// once, here, and stored as the state's neighbour list; the list step kernel
// then reads them instead of recomputing bitstrings and ranks at every step.
// Neighbour rows gathered per batch in the list kernel, by row type and
// chunks per lane.  Measured on the ring (R=100: FP32 CPL 2, FP64 CPL 2) and
// J1-J2 workloads (R=64 FP32 and R=32 FP64: CPL 1).
#ifndef KPM_LIST_BATCH_F32_CPL1
#define KPM_LIST_BATCH_F32_CPL1 16
#endif
#ifndef KPM_LIST_BATCH_F32_CPL2
#define KPM_LIST_BATCH_F32_CPL2 2
#endif
#ifndef KPM_LIST_BATCH_F32_ONE
#define KPM_LIST_BATCH_F32_ONE 8  // FP32 rows of one state per warp (unpadded lists)
#endif
#ifndef KPM_LIST_BATCH_F64
#define KPM_LIST_BATCH_F64 4  // chunks per lane and batch (4 rows at CPL 1, 2 at CPL 2)
#endif

// Neighbour rows per gather batch of the list kernel.
__host__ __device__ constexpr int list_batch(bool fp32, int cpl) {
  return fp32 ? (cpl == 1 ? KPM_LIST_BATCH_F32_CPL1 : KPM_LIST_BATCH_F32_CPL2)
              : (KPM_LIST_BATCH_F64 / cpl > 0 ? KPM_LIST_BATCH_F64 / cpl : 1);
}

// Minimum resident blocks per SM requested for the list kernel: 4 (64
// registers) for FP32 rows at 2 chunks per lane, 3 (80 registers) otherwise,
// as measured on the ring and J1-J2 workloads.
#ifndef KPM_LIST_MIN_BLOCKS_F32_CPL2
#define KPM_LIST_MIN_BLOCKS_F32_CPL2 4
#endif
#ifndef KPM_LIST_MIN_BLOCKS
#define KPM_LIST_MIN_BLOCKS 3
#endif

// Shared memory budget (KB) of the hi-block kernel's staged block and rank table.
#ifndef KPM_BLOCK_SMEM_KB
#define KPM_BLOCK_SMEM_KB 48
#endif
// FP32 rows of 17..32 chunks run as two states per warp (1) or one (0) unless
// the schedule says otherwise.
#ifndef KPM_TWO_STATE_DEFAULT
#define KPM_TWO_STATE_DEFAULT 1
#endif

// Padding unit of each group's list entries: the FP32 gather batch, except for
// FP32 rows of one chunk per lane and one state per warp; 1 in FP64.
inline int list_pad(int precision, int cpl, int gpw) {
  return precision == KPM_FP32 && (cpl != 1 || gpw > 1) ? list_batch(true, cpl) : 1;
}

struct ListArgs {
  uint32_t *lists;
  TablesDev tb;
  int stride;           // entries per state
  uint64_t rstride;     // word offset between states (stride: state-major lists)
  uint64_t estride;     // word offset between a state's entries (1: state-major)
  uint32_t crow;        // 16-byte chunks per row
  int batch;            // each group's entries are padded to a multiple of this
  uint32_t zero_chunk;  // first chunk of the all-zero row after the last state
};

__global__ void __launch_bounds__(kThreads)
    build_lists_kernel(const __grid_constant__ ListArgs a, const __grid_constant__ BondsDev bd) {
  for (int t = blockIdx.x; t < a.tb.n_tiles; t += gridDim.x) {
    const Tile tile = a.tb.tiles[t];
    const SectorDev sd = a.tb.sectors[tile.sector];
    const bool full_tile = sd.n_up < 0;
    uint32_t hb = tile.b_first;
    for (uint32_t u = threadIdx.x; u < tile.count; u += kThreads) {
      const int64_t row = tile.row0 + u;
      const uint64_t s = full_tile ? (uint64_t)(row - sd.row0)
                                   : sector_unrank(tile.rank0 + u, sd.n_up, tile.b_last, hb, a.tb);
      uint32_t *L = a.lists + (size_t)row * a.rstride;
      const uint64_t es = a.estride;
      uint32_t hdr = 0;
      int e = 1;
      for (int g = 0; g < bd.n_groups; ++g) {
        uint32_t cnt = 0;
        for (int k = bd.gstart[g]; k < bd.gstart[g + 1]; ++k) {
          const uint64_t m = bd.mask[bd.order[k]];
          const uint64_t tt = s & m;
          if (tt != 0 && tt != m) {
            const uint64_t f = s ^ m;
            const uint32_t rk = full_tile ? (uint32_t)f : sector_rank(f, a.tb);
            L[(e++) * es] = ((uint32_t)sd.row0 + rk) * a.crow;
            ++cnt;
          }
        }
        hdr |= cnt << (8 * g);
        // pad the group to whole gather batches with the zero row
        for (uint32_t k = cnt; k % a.batch != 0; ++k) L[(e++) * es] = a.zero_chunk;
      }
      L[0] = hdr;
    }
  }
}


// out[sec][q] = sum over the sector's tiles, in tile order per thread and then
// over the block, of the per-tile sums ts[t][q].  Called by a whole block.
template <int NQ>
__device__ void reduce_sector_tiles(const double *ts, const TablesDev &tb, int sec, double *out,
                                    double *s_red) {
  double v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = 0.0;
  for (int t = tb.tile_begin[sec] + threadIdx.x; t < tb.tile_end[sec]; t += kThreads) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) v[q] += __ldcg(ts + (int64_t)t * NQ + q);
  }
  block_sum<NQ>(v, s_red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) out[(size_t)sec * NQ + q] = v[q];
  }
}

// Bytes after the zero row that the list kernel's gathers may read (and
// ignore) when a lane's last chunk slot lies past the end of a row.
constexpr size_t kRowSlack = 32 * 16;

// Shared memory of the list kernel: per warp two buffers of gpw lists.
constexpr size_t kMaxListSmem = 48 * 1024;
inline size_t list_smem_bytes(int gpw, int stride) {
  return (size_t)kWarps * 2 * gpw * stride * sizeof(uint32_t);
}


// One Chebyshev step driven by the neighbour lists (cooperative layouts with
// grouped couplings).  Warps work independently: each takes small tiles from
// the step's queue and writes the tile's dot products to the tile's own slot
// of this step, so the loop has no block-wide barriers.  The slots of the
// previous step are summed per sector, in tile order, at the start of the
// next step (and for the last step by reduce_tile_sums_kernel).  A warp
// copies the lists of its next gpw states into its own shared-memory buffer
// (cp.async, double-buffered) while it works on the current ones, so the
// neighbour indices are on chip when the gathers start; the G lanes of a
// state gather their own chunks of the listed rows.
template <typename T, int CPL, bool FULL>
__global__ void __launch_bounds__(kThreads, (sizeof(T) == 4 && CPL == 2) ? KPM_LIST_MIN_BLOCKS_F32_CPL2
                                                                          : KPM_LIST_MIN_BLOCKS)
    cheb_step_list_kernel(const __grid_constant__ StepArgs a, const __grid_constant__ BondsDev bd,
                          const uint32_t *__restrict__ lists, int stride, CoefDev cf) {
  using C = Chunk<T>;
  using V = typename C::type;
  constexpr int NQ = FULL ? 6 : 2;
  constexpr bool PAIR = sizeof(T) == 4;
  const V *__restrict__ x = reinterpret_cast<const V *>(a.x);
  V *__restrict__ zy = reinterpret_cast<V *>(a.zy);
  const int lane = threadIdx.x & 31;
  const int G = a.G, gpw = a.gpw;
  const int grp = lane / G, sub = lane - grp * G;
  const bool active = grp < gpw;
  const uint32_t crow = (uint32_t)(a.Rp / C::W);
  // chunk c of a lane is sub + c * G; with the two-state FP32 mapping
  // (G = 16, CPL = 2) the last slots of a row may lie past its chunks
  bool valid[CPL];
  // chunk offsets of the gathers: a slot past the row reads the row's last
  // chunk (ignored), so that a gather touches only the row's own cache lines
  uint32_t coff[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    valid[c] = (uint32_t)(sub + c * G) < crow;
    coff[c] = valid[c] ? (uint32_t)(sub + c * G) : crow - 1;
  }
  const int ng = bd.n_groups;
  // per-slot base pointers of the gathers: row chunk ci of slot c is xs[c][ci]
  const V *xs[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) xs[c] = x + coff[c];
  const int kind = a.first ? 0 : 1;
  const T *dh_all = reinterpret_cast<const T *>(cf.diag_hi);
  const T *dl_all = reinterpret_cast<const T *>(cf.diag_lo);
  const T *gh_all = reinterpret_cast<const T *>(cf.grp_hi);
  const T *gl_all = reinterpret_cast<const T *>(cf.grp_lo);
  extern __shared__ __align__(16) uint32_t s_lists[];  // [kWarps][2][gpw * stride]
  const int span = gpw * stride;
  uint32_t *wbuf = s_lists + (threadIdx.x >> 5) * 2 * span;
  if (a.prev_sums != nullptr) {
    __shared__ double s_red[kWarps * NQ];
    for (int sec = blockIdx.x; sec < a.tb.n_sectors; sec += gridDim.x)
      reduce_sector_tiles<NQ>(a.prev_partials, a.tb, sec, a.prev_sums, s_red);
  }
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(a.queue, 1);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= a.tb.n_tiles) break;
    const Tile tile = a.tb.tiles[t];
    const SectorDev sd = a.tb.sectors[tile.sector];
    if (lane == 0) {
      // the tile's lists and own rows are read in order: start them towards L2 now
      prefetch_range_l2(lists + (size_t)tile.row0 * stride,
                        lists + ((size_t)tile.row0 + tile.count) * stride);
      const size_t rb = (size_t)a.Rp * sizeof(T);
      const char *xb = reinterpret_cast<const char *>(a.x) + (size_t)tile.row0 * rb;
      prefetch_range_l2(xb, xb + tile.count * rb);
      if (!a.first) {
        const char *zb = reinterpret_cast<const char *>(a.zy) + (size_t)tile.row0 * rb;
        prefetch_range_l2(zb, zb + tile.count * rb);
      }
    }
    const size_t cbase = (size_t)tile.sector * 2 + kind;
    const T *dh = dh_all + cbase * bd.table_size;
    const T *dl = dl_all + cbase * bd.table_size;
    T gh[kMaxGroups], gl[kMaxGroups];
#pragma unroll
    for (int g = 0; g < kMaxGroups; ++g) {
      gh[g] = g < ng ? __ldg(gh_all + cbase * kMaxGroups + g) : (T)0;
      gl[g] = (PAIR && g < ng) ? __ldg(gl_all + cbase * kMaxGroups + g) : (T)0;
    }

    double acc64[NQ];
    KahanF accf[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc64[q] = 0.0;
    {
      // lists of iteration `it` (states it*gpw ..) into wbuf[it & 1]
      const uint32_t n_iter = (tile.count + gpw - 1) / gpw;
      auto copy_lists = [&](uint32_t it) {
        const uint32_t s0 = it * gpw;
        const int nw = (int)min((uint32_t)gpw, tile.count - s0) * stride;
        const uint32_t *src = lists + (size_t)(tile.row0 + s0) * stride;
        uint32_t *dst = wbuf + (it & 1) * span;
        for (int w = lane; w < nw; w += 32) cp_async4(dst + w, src + w);
      };
      copy_lists(0);
      cp_async_commit();
      for (uint32_t it = 0; it < n_iter; ++it) {
        if (it + 1 < n_iter) copy_lists(it + 1);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
        const uint32_t u = it * gpw + grp;
        const uint32_t *L = wbuf + (it & 1) * span + grp * stride;
        if (active && u < tile.count) {
          const int64_t row = tile.row0 + u;
          const uint32_t own = (uint32_t)row * crow + sub;
          V xv[CPL], zv[CPL], acc[CPL];
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            xv[c] = valid[c] ? x[own + c * G] : V{};
            zv[c] = (a.first || !valid[c]) ? V{} : __ldcs(zy + own + c * G);
            acc[c] = V{};
          }
          const uint32_t hdr = L[0];
          // diagonal of this state: the table entry for its flip counts, loaded
          // before the gathers so that its latency is hidden behind them
          int tidx = 0;
#pragma unroll
          for (int g = 0; g < kMaxGroups; ++g)
            if (g < ng) tidx += (int)((hdr >> (8 * g)) & 255u) * bd.tstride[g];
          const T ad_hi = __ldg(dh + tidx);
          const T ad_lo = PAIR ? __ldg(dl + tidx) : (T)0;
          int e = 1;
#pragma unroll
          for (int g = 0; g < kMaxGroups; ++g) {
            if (g < ng) {
              const int cnt = (hdr >> (8 * g)) & 255u;
              V gs[CPL];
#pragma unroll
              for (int c = 0; c < CPL; ++c) gs[c] = V{};
              if (sizeof(T) == 4 && (CPL != 1 || gpw > 1)) {
                // FP32 lists (except rows of one chunk per lane and one state per
                // warp) pad each group to whole batches with the index of an
                // all-zero row, so every batch is gathered without predicates
                constexpr int B = list_batch(true, CPL);
                const int padded = (cnt + B - 1) / B * B;
                for (int i = 0; i < padded; i += B) {
                  V v[B][CPL];
#pragma unroll
                  for (int q = 0; q < B; ++q) {
                    const uint32_t ci = L[e + i + q];
#pragma unroll
                    for (int c = 0; c < CPL; ++c) v[q][c] = __ldg(xs[c] + ci);
                  }
#pragma unroll
                  for (int q = 0; q < B; ++q) {
#pragma unroll
                    for (int c = 0; c < CPL; ++c) gs[c] = C::add(gs[c], v[q][c]);
                  }
                }
                e += padded;
              } else {
                // Unpadded lists (FP64; FP32 rows of one chunk per lane and one state
                // per warp): the last batch is predicated.  With one state per warp
                // the predicates are uniform over the warp and the skipped loads
                // move no data.
                constexpr int B = sizeof(T) == 4 ? KPM_LIST_BATCH_F32_ONE : list_batch(false, CPL);
                for (int i = 0; i < cnt; i += B) {
                  uint32_t ci[B];
#pragma unroll
                  for (int q = 0; q < B; ++q) ci[q] = (i + q < cnt) ? L[e + i + q] : 0u;
                  V v[B][CPL];
#pragma unroll
                  for (int q = 0; q < B; ++q) {
#pragma unroll
                    for (int c = 0; c < CPL; ++c)
                      v[q][c] = (i + q < cnt) ? __ldg(xs[c] + ci[q]) : V{};
                  }
#pragma unroll
                  for (int q = 0; q < B; ++q) {
#pragma unroll
                    for (int c = 0; c < CPL; ++c) gs[c] = C::add(gs[c], v[q][c]);
                  }
                }
                e += cnt;
              }
#pragma unroll
              for (int c = 0; c < CPL; ++c) {
                acc[c] = C::fma(gh[g], gs[c], acc[c]);
                if (PAIR) acc[c] = C::fma(gl[g], gs[c], acc[c]);
              }
            }
          }
          using P2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
          P2 paa{}, pba{};
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            V h = acc[c];
            if (PAIR) h = C::fma(ad_lo, xv[c], h);
            const V y = C::fma_sub(ad_hi, xv[c], h, zv[c]);
            if (valid[c]) {
              C::dots(xv[c], y, paa, pba);
              __stcs(zy + own + c * G, y);
            }
          }
          const T pxx = paa.x + paa.y, pyx = pba.x + pba.y;
          if constexpr (sizeof(T) == 8) {
            acc64[0] += pxx;
            acc64[1] += pyx;
            if (FULL) {
              const double M = sd.n_up < 0 ? (double)__popcll((uint64_t)(row - sd.row0)) - a.half_n : sd.Mval;
              acc64[2] += M * pxx;
              acc64[3] += M * pyx;
              acc64[4] += M * M * pxx;
              acc64[5] += M * M * pyx;
            }
          } else {
            accf[0].add(pxx);
            accf[1].add(pyx);
            if (FULL) {
              const float M = sd.n_up < 0 ? (float)__popcll((uint64_t)(row - sd.row0)) - (float)a.half_n
                                          : (float)sd.Mval;
              accf[2].add(M * pxx);
              accf[3].add(M * pyx);
              accf[4].add(M * M * pxx);
              accf[5].add(M * M * pyx);
            }
          }
        }
        __syncwarp();  // the buffer read here is refilled by the next iteration's copy
      }
      cp_async_wait<0>();
    }
    if constexpr (sizeof(T) == 4) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) acc64[q] = accf[q].value();
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc64[q] = warp_sum(acc64[q]);
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) a.partials[(int64_t)t * NQ + q] = acc64[q];
    }
  }
}

// Sums of the list kernel's last step: one block per sector.
template <int NQ>
__global__ void __launch_bounds__(kThreads) reduce_tile_sums_kernel(const double *ts, TablesDev tb,
                                                                    double *sums) {
  __shared__ double s_red[kWarps * NQ];
  reduce_sector_tiles<NQ>(ts, tb, blockIdx.x, sums, s_red);
}

// ---------------------------------------------------------------- per-vector moments
// The moments of each random vector separately, mu^(r)_n = <r|T_n(H')|r>
// (the terms of the average in Eq. E-2-7), for realisation statistics and
// sampled checks.  After a step the column kernel reads v_n and v_{n+1} once
// more and forms, per chunk of rows of one sector, <v_n^r|v_n^r> and
// <v_{n+1}^r|v_n^r> for every vector r in FP64; the chunk sums are then added
// per sector in chunk order.  This costs one extra read of both vectors per
// step and is only done when per-vector moments are asked for.
struct ColArgs {
  const void *x, *y;
  const int64_t *chunks;  // (row_begin, row_end, sector) per chunk
  double *part;           // [n_chunks][R][2]
  int R, Rp;
};

template <typename T>
__global__ void __launch_bounds__(kThreads) column_dots_kernel(const __grid_constant__ ColArgs a) {
  __shared__ double s_xx[kThreads], s_yx[kThreads];
  const int64_t ch = blockIdx.x;
  const int64_t r_begin = a.chunks[3 * ch], r_end = a.chunks[3 * ch + 1];
  const T *x = reinterpret_cast<const T *>(a.x);
  const T *y = reinterpret_cast<const T *>(a.y);
  const int cols = min(a.R, kThreads);
  const int nl = kThreads / cols;
  const int cl = threadIdx.x % cols, rl = threadIdx.x / cols;
  for (int c0 = 0; c0 < a.R; c0 += cols) {
    const int col = c0 + cl;
    double xx = 0.0, yx = 0.0;
    if (rl < nl && col < a.R) {
      for (int64_t row = r_begin + rl; row < r_end; row += nl) {
        const double xv = (double)x[row * a.Rp + col];
        const double yv = (double)y[row * a.Rp + col];
        xx = fma(xv, xv, xx);
        yx = fma(yv, xv, yx);
      }
    }
    s_xx[threadIdx.x] = xx;
    s_yx[threadIdx.x] = yx;
    __syncthreads();
    if ((int)threadIdx.x < cols && c0 + (int)threadIdx.x < a.R) {
      double sx = 0.0, sy = 0.0;
      for (int l = 0; l < nl; ++l) {
        sx += s_xx[l * cols + threadIdx.x];
        sy += s_yx[l * cols + threadIdx.x];
      }
      double *o = a.part + (ch * a.R + c0 + threadIdx.x) * 2;
      o[0] = sx;
      o[1] = sy;
    }
    __syncthreads();
  }
}

// out[sec][r][q] = sum over the sector's chunks (in order) of part[chunk][r][q].
__global__ void __launch_bounds__(kThreads)
    column_reduce_kernel(const double *part, const int64_t *sec_ranges, double *out, int R) {
  const int sec = blockIdx.x;
  const int64_t c0 = sec_ranges[2 * sec], c1 = sec_ranges[2 * sec + 1];
  for (int i = threadIdx.x; i < 2 * R; i += kThreads) {
    double v = 0.0;
    for (int64_t c = c0; c < c1; ++c) v += part[c * 2 * R + i];
    out[(int64_t)sec * 2 * R + i] = v;
  }
}

// mu_r[out_index][r][n] from the per-vector sums (no average over r).
struct AssembleRArgs {
  const double *sums_r;  // [S][n_sectors][R][2]
  const SectorDev *sectors;
  double *mu_r;
  int n_sectors, K, R;
};

__global__ void assemble_r_kernel(const __grid_constant__ AssembleRArgs a) {
  const int64_t total = (int64_t)a.n_sectors * a.R * a.K;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int n = (int)(i % a.K);
    const int r = (int)((i / a.K) % a.R);
    const int sec = (int)(i / ((int64_t)a.K * a.R));
    const int step = n / 2, q = n & 1;
    const double raw = a.sums_r[(((int64_t)step * a.n_sectors + sec) * a.R + r) * 2 + q];
    const double base = a.sums_r[((int64_t)sec * a.R + r) * 2 + q];  // mu_0 or mu_1 of vector r
    const double val = step == 0 ? raw : 2.0 * raw - base;
    a.mu_r[((int64_t)a.sectors[sec].out_index * a.R + r) * a.K + n] = val;
  }
}

// ---------------------------------------------------------------- random vectors

struct InitArgs {
  void *v0;
  TablesDev tb;
  uint64_t seed, r0;
  int R, Rp, G, gpw;
  int uniform;  // 0: +-1/sqrt(D) signs; 1: uniform values in (-1, 1), not normalised
  int basis;    // 1: vector r is the unit vector of the state of rank r0 + r (zero if none)
};

template <typename T>
__global__ void __launch_bounds__(kThreads) init_vectors_kernel(const __grid_constant__ InitArgs a) {
  using C = Chunk<T>;
  using V = typename C::type;
  constexpr int W = C::W;
  __shared__ uint64_t s_hr[512];
  const uint64_t hs = splitmix64(a.seed);
  for (int col = threadIdx.x; col < a.R; col += kThreads) s_hr[col] = splitmix64(hs ^ (a.r0 + (uint64_t)col));
  __syncthreads();
  V *v = reinterpret_cast<V *>(a.v0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int grp = lane / a.G, sub = lane - grp * a.G;
  if (grp >= a.gpw) return;
  const int crow = a.Rp / W;
  for (int t = blockIdx.x; t < a.tb.n_tiles; t += gridDim.x) {
    const Tile tile = a.tb.tiles[t];
    const SectorDev sd = a.tb.sectors[tile.sector];
    const T norm = (T)(1.0 / sqrt((double)sd.dim));
    uint32_t hb = tile.b_first;
    for (uint32_t u = warp * a.gpw + grp; u < tile.count; u += kWarps * a.gpw) {
      const int64_t row = tile.row0 + u;
      uint64_t s;
      if (sd.n_up < 0)
        s = (uint64_t)(row - sd.row0);
      else
        s = sector_unrank(tile.rank0 + u, sd.n_up, tile.b_last, hb, a.tb);
      for (int ch = sub; ch < crow; ch += a.G) {
        V val;
#pragma unroll
        for (int e = 0; e < W; ++e) {
          const int col = ch * W + e;
          T x = 0;
          if (col < a.R && a.basis) {
            x = (uint64_t)(row - sd.row0) == a.r0 + (uint64_t)col ? (T)1 : (T)0;
          } else if (col < a.R) {
            const uint64_t h = splitmix64(s_hr[col] ^ s);
            if (a.uniform)
              x = (T)(2.0 * (((double)(h >> 11) + 0.5) * 0x1.0p-53) - 1.0);
            else
              x = (h >> 63) ? -norm : norm;
          }
          C::set(val, e, x);
        }
        v[row * crow + ch] = val;
      }
    }
  }
}

// ---------------------------------------------------------------- moments

struct AssembleArgs {
  const double *sums;  // [S][n_sectors][NQ]
  const SectorDev *sectors;
  double *mu, *mu_M, *mu_M2;
  int *flag;
  int n_sectors, K, NQ;
  double inv_R;
};

__global__ void assemble_kernel(const __grid_constant__ AssembleArgs a) {
  const int total = a.n_sectors * a.K;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    const int sec = i / a.K, n = i - sec * a.K;
    const int step = n / 2;
    const bool odd = n & 1;
    const int nq_out = a.mu_M ? 3 : 1;
    const bool full = a.sectors[sec].n_up < 0;
    for (int q = 0; q < 3; ++q) {
      double *out = q == 0 ? a.mu : (q == 1 ? a.mu_M : a.mu_M2);
      if (!out) continue;
      double val;
      if (full || q == 0) {
        const int qq = 2 * q + (odd ? 1 : 0);
        const double raw = a.sums[((int64_t)step * a.n_sectors + sec) * a.NQ + qq] * a.inv_R;
        if (step == 0) {
          val = raw;
        } else {
          const double base = a.sums[(int64_t)sec * a.NQ + qq] * a.inv_R;  // mu_0 or mu_1
          val = 2.0 * raw - base;
        }
      } else {
        // a sector: M and M^2 are constants, mu_M = M mu, mu_M2 = M^2 mu
        const int qq = odd ? 1 : 0;
        const double raw = a.sums[((int64_t)step * a.n_sectors + sec) * a.NQ + qq] * a.inv_R;
        const double base = a.sums[(int64_t)sec * a.NQ + qq] * a.inv_R;
        const double m0 = step == 0 ? raw : 2.0 * raw - base;
        const double M = a.sectors[sec].Mval;
        val = (q == 1 ? M : M * M) * m0;
      }
      out[(int64_t)a.sectors[sec].out_index * a.K + n] = val;
      if (q == 0 && !(fabs(val) <= 1.0 + 1e-6)) atomicOr(a.flag, 1);
    }
    (void)nq_out;
  }
}

// ---------------------------------------------------------------- host driver

namespace {

using StepFn = void (*)(const StepArgs, const BondsDev);

template <typename T, int CPL, bool FULL>
void *step_ptr() {
  return reinterpret_cast<void *>(&cheb_step_kernel<T, CPL, FULL>);
}

void *pick_step(int precision, int cpl, bool full);

template <typename T, int CPL, bool FULL>
void *list_ptr() {
  return reinterpret_cast<void *>(&cheb_step_list_kernel<T, CPL, FULL>);
}

void *pick_list(int precision, int cpl, bool full) {
  if (precision == KPM_FP32) {
    if (cpl == 1) return full ? list_ptr<float, 1, true>() : list_ptr<float, 1, false>();
    return full ? list_ptr<float, 2, true>() : list_ptr<float, 2, false>();
  }
  if (cpl == 1) return full ? list_ptr<double, 1, true>() : list_ptr<double, 1, false>();
  return full ? list_ptr<double, 2, true>() : list_ptr<double, 2, false>();
}

void *pick_kernel(const MomentsRun &r) {
  if (r.block_L > 0) return block_kernel_ptr(r.precision);
  if (r.list_stride > 0) return pick_list(r.precision, r.lay.cpl, r.plan.any_full);
  return pick_step(r.precision, r.lay.cpl, r.plan.any_full);
}

void *pick_step(int precision, int cpl, bool full) {
  if (precision == KPM_FP32) {
    switch (cpl) {
      case 1: return full ? step_ptr<float, 1, true>() : step_ptr<float, 1, false>();
      case 2: return full ? step_ptr<float, 2, true>() : step_ptr<float, 2, false>();
      case 3: return full ? step_ptr<float, 3, true>() : step_ptr<float, 3, false>();
      case 4: return full ? step_ptr<float, 4, true>() : step_ptr<float, 4, false>();
      default: return full ? step_ptr<float, 8, true>() : step_ptr<float, 8, false>();
    }
  }
  switch (cpl) {
    case 1: return full ? step_ptr<double, 1, true>() : step_ptr<double, 1, false>();
    case 2: return full ? step_ptr<double, 2, true>() : step_ptr<double, 2, false>();
    case 3: return full ? step_ptr<double, 3, true>() : step_ptr<double, 3, false>();
    case 4: return full ? step_ptr<double, 4, true>() : step_ptr<double, 4, false>();
    default: return full ? step_ptr<double, 8, true>() : step_ptr<double, 8, false>();
  }
}

size_t step_smem(const MomentsRun &r) {
  // matrix-free kernel: diagonal table, hi + lo floats (FP32) or one double
  // (FP64) per entry; list kernel: two list buffers of gpw states per warp
  if (r.block_L > 0) return block_smem_bytes(r);
  if (r.list_stride > 0) return list_smem_bytes(r.lay.gpw, r.list_stride);
  return (size_t)r.bonds.table_size * 8;
}

}  // namespace

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

int prepare_run(const kpm_model *m, int n_sectors, const int32_t *n_up, int K, int R,
                int precision, MomentsRun *run, const Knobs &knobs, int vectors,
                bool per_vector) {
  KPM_TRY(validate_model(m));
  KPM_REQUIRE(vectors == kVecRademacher || vectors == kVecBasis, KPM_EINVAL,
              "vectors = %d (KPM_VECTORS_RADEMACHER or KPM_VECTORS_BASIS)", vectors);
  run->knobs = knobs;
  run->vectors = vectors;
  run->per_vector = per_vector;
  KPM_TRY(validate_sectors(m, n_sectors, n_up));
  KPM_REQUIRE(K >= 2 && (K % 2) == 0, KPM_EINVAL, "n_moments = %d must be even and >= 2", K);
  KPM_TRY(make_layout(R, precision, &run->lay));
  run->precision = precision;
  run->K = K;
  run->S = K / 2;
  int64_t rows = 0;
  bool full = false;
  for (int s = 0; s < n_sectors; ++s) {
    rows += kpm_sector_dim(m->n_sites, n_up[s]);
    full |= n_up[s] < 0;
  }
  fill_bonds(m, &run->bonds);
  fill_pass_masks(&run->bonds, run->lay.G);
  // neighbour lists for cooperative layouts with grouped couplings (CPL 1 or 2)
  run->list_stride = 0;
  if (knobs.lists != 0 && run->lay.G >= 2 && (run->lay.cpl == 1 || run->lay.cpl == 2) &&
      run->bonds.n_groups > 0 && m->n_bonds <= 255) {
    // FP32 rows of 17..32 chunks: two states per warp, 16 lanes x 2 chunks
    // each (the row layout in memory is unchanged; lanes whose second slot
    // lies past the row's chunks skip it), which halves the per-state work
    // of the warp.
    const int two_state = knobs.two_state >= 0 ? knobs.two_state : KPM_TWO_STATE_DEFAULT;
    if (precision == KPM_FP32 && run->lay.cpl == 1 && run->lay.G > 16 && two_state != 0) {
      run->lay.G = 16;
      run->lay.cpl = 2;
      run->lay.gpw = 2;
    }
    // header word, then each group's entries (FP32: padded to whole gather batches)
    const int B = list_pad(precision, run->lay.cpl, run->lay.gpw);
    int stride = 1;
    for (int g = 0; g < run->bonds.n_groups; ++g) {
      const int size = run->bonds.gstart[g + 1] - run->bonds.gstart[g];
      stride += (size + B - 1) / B * B;
    }
    if (list_smem_bytes(run->lay.gpw, stride) <= kMaxListSmem) run->list_stride = stride;
  }
  // hi-block kernel: one lane per state (one 16-byte chunk per row), sectors
  // only, grouped couplings; the low split L is the largest at which the
  // largest block (C(L, L/2) rows) and the 16-bit lo_rank table fit 48 KB of
  // shared memory
  run->block_L = 0;
  if (knobs.block != 0 && run->lay.G == 1 && run->lay.cpl == 1 && run->list_stride == 0 &&
      run->bonds.n_groups > 0 && m->n_bonds <= kBlockMaxBonds) {
    bool sectors_only = true;
    for (int s2 = 0; s2 < n_sectors; ++s2) sectors_only &= n_up[s2] >= 0;
    int Lb = 0;
    for (int Lc = std::min(m->n_sites / 2, 16); Lc >= 1; --Lc) {
      const size_t bytes = (((size_t)2 << Lc) + 15) / 16 * 16 + (size_t)binom(Lc, Lc / 2) * 16;
      if (bytes <= KPM_BLOCK_SMEM_KB * 1024 && m->n_sites - Lc <= 22) {
        Lb = Lc;
        break;
      }
    }
    if (sectors_only && Lb > 0) run->block_L = Lb;
  }
  int64_t ts = run->list_stride > 0 ? list_tile_states(run->lay.gpw, rows)
                                    : choose_tile_states(run->lay.gpw, rows);
  if (knobs.tile_states > 0) {
    // a tuned tile size, in whole warp groups, within the list kernel's tile limit
    const int64_t g = run->lay.gpw;
    ts = std::max<int64_t>(knobs.tile_states, g);
    ts = (ts + g - 1) / g * g;
    if (run->list_stride > 0)
      ts = std::max<int64_t>(ts, (rows + KPM_LIST_MAX_TILES - 1) / KPM_LIST_MAX_TILES);
  }
  KPM_TRY(build_plan(m, n_sectors, n_up, ts, &run->plan, run->block_L));
  if (run->block_L > 0) {
    // split the bonds by where their sites lie, each kind sorted by coupling group
    BlockBondsDev &bb = run->bb;
    bb = BlockBondsDev{};
    const int L = run->block_L;
    bb.L = L;
    bb.n_groups = run->bonds.n_groups;
    for (int g = 0; g < kMaxGroups; ++g) bb.tstride[g] = run->bonds.tstride[g];
    int nl = 0, nh = 0, nx = 0;
    for (int g = 0; g < run->bonds.n_groups; ++g) {
      bb.low_gs[g] = nl;
      bb.high_gs[g] = nh;
      bb.cross_gs[g] = nx;
      for (int k = run->bonds.gstart[g]; k < run->bonds.gstart[g + 1]; ++k) {
        const int b = run->bonds.order[k];
        const int i = std::min(m->bi[b], m->bj[b]), j = std::max(m->bi[b], m->bj[b]);
        if (j < L) {
          bb.low_mask[nl++] = (1u << i) | (1u << j);
        } else if (i >= L) {
          bb.high_mask[nh++] = (1u << (i - L)) | (1u << (j - L));
        } else {
          bb.cross_lo[nx] = (uint8_t)i;
          bb.cross_hi[nx] = (uint8_t)(j - L);
          ++nx;
        }
      }
    }
    for (int g = run->bonds.n_groups; g <= kMaxGroups; ++g) {
      bb.low_gs[g] = nl;
      bb.high_gs[g] = nh;
      bb.cross_gs[g] = nx;
    }
    run->max_block = 0;
    for (int s2 = 0; s2 < n_sectors; ++s2) {
      const int k = n_up[s2];
      for (int c = std::max(0, k - (m->n_sites - L)); c <= std::min(L, k); ++c)
        run->max_block = std::max<int64_t>(run->max_block, binom(L, c));
    }
  }
  if (per_vector) {
    // chunks of rows, each inside one sector, for the per-vector column sums
    const int64_t ch = std::min<int64_t>(65536, std::max<int64_t>(256, run->plan.total_rows / 2048));
    run->cd_chunks.clear();
    std::vector<int64_t> ranges;
    for (int sidx = 0; sidx < run->plan.n_sectors; ++sidx) {
      const int64_t r0s = run->plan.row0[sidx], r1s = r0s + run->plan.dim[sidx];
      ranges.push_back((int64_t)run->cd_chunks.size() / 3);
      for (int64_t r = r0s; r < r1s; r += ch) {
        run->cd_chunks.push_back(r);
        run->cd_chunks.push_back(std::min(r + ch, r1s));
        run->cd_chunks.push_back(sidx);
      }
      ranges.push_back((int64_t)run->cd_chunks.size() / 3);
    }
    run->n_cd = (int)(run->cd_chunks.size() / 3);
    run->cd_chunks.insert(run->cd_chunks.end(), ranges.begin(), ranges.end());
  }
  run->NQ = run->plan.any_full ? 6 : 2;
  KPM_REQUIRE((uint64_t)(run->plan.total_rows + 1) * (run->lay.Rp / run->lay.vec_width) < (1ull << 32),
              KPM_EINVAL, "%lld rows x %d chunks exceed 32-bit chunk indices",
              (long long)run->plan.total_rows, run->lay.Rp / run->lay.vec_width);
  // one all-zero row after the last state: the padding entries of the lists point to it
  run->vec_bytes = align256((size_t)(run->plan.total_rows + 1) * run->lay.Rp * run->lay.elem + kRowSlack);
  (void)full;
  return KPM_OK;
}

size_t coef_bytes(const MomentsRun &r, int which) {
  // which: 0/1 diagonal hi/lo, 2/3 group hi/lo
  const size_t per = which < 2 ? (size_t)r.bonds.table_size : (size_t)kMaxGroups;
  return align256((size_t)r.plan.n_sectors * 2 * per * r.lay.elem);
}

size_t run_bytes(const MomentsRun &r) {
  const bool lists = r.list_stride > 0;
  size_t coef = 0;
  if (lists)
    for (int w = 0; w < 4; ++w) coef += coef_bytes(r, w);
  if (r.block_L > 0)
    for (int w = 0; w < 4; ++w) coef += coef_bytes(r, w);
  const size_t nblk = r.plan.hb_hi.size();
  const size_t slots = std::max(r.plan.tiles.size(), r.block_L > 0 ? nblk : 0);
  return 2 * r.vec_bytes + tables_bytes(r.plan) + coef +
         (r.block_L > 0 ? align256(nblk * sizeof(int32_t)) +
                              align256((size_t)2 * r.plan.n_sectors * sizeof(int32_t))
                        : 0) +
         align256((size_t)r.plan.total_rows * r.list_stride * sizeof(uint32_t)) +
         align256((lists ? 2 : 1) * slots * r.NQ * sizeof(double)) +
         align256((size_t)r.S * r.plan.n_sectors * r.NQ * sizeof(double)) +
         align256((size_t)2 * r.S * sizeof(int)) + 256 +
         (r.per_vector ? align256(r.cd_chunks.size() * sizeof(int64_t)) +
                             align256((size_t)r.n_cd * r.lay.R * 2 * sizeof(double)) +
                             align256((size_t)r.S * r.plan.n_sectors * r.lay.R * 2 * sizeof(double))
                       : 0);
}

namespace {

// Coefficients of H' for the list kernel: per sector and kind of step (A = 1/a
// on the first step, 2/a later), the diagonal A (d - b) for each combination
// of anti-aligned bond counts per group, d = sum_bonds J/4 - sum_g n_g J_g / 2,
// and the flip amplitude A J_g / 2 of each group; each split into the nearest
// value of the vector type plus (FP32) the rounding remainder.
template <typename T>
int upload_coefficients_t(MomentsRun &r, const std::vector<SectorDev> &sec, Arena &arena,
                          cudaStream_t s) {
  const BondsDev &bd = r.bonds;
  const int ns = r.plan.n_sectors, ng = bd.n_groups, tsz = bd.table_size;
  const bool pair = sizeof(T) == 4;
  std::vector<T> dh((size_t)ns * 2 * tsz), dl(dh.size(), (T)0);
  std::vector<T> gh((size_t)ns * 2 * kMaxGroups, (T)0), gl(gh.size(), (T)0);
  std::vector<double> d(tsz);
  for (int idx = 0; idx < tsz; ++idx) {
    double v = bd.J_quarter_sum;
    for (int g = 0; g < ng; ++g) {
      const int size = bd.gstart[g + 1] - bd.gstart[g];
      v -= ((idx / bd.tstride[g]) % (size + 1)) * (0.5 * bd.gJ[g]);
    }
    d[idx] = v;
  }
  for (int i = 0; i < ns; ++i)
    for (int kind = 0; kind < 2; ++kind) {
      const double A = (kind == 0 ? 1.0 : 2.0) * sec[i].inv_a;
      const size_t base = (size_t)i * 2 + kind;
      for (int idx = 0; idx < tsz; ++idx) {
        const double ad = A * (d[idx] - sec[i].b);
        const T hi = (T)ad;
        dh[base * tsz + idx] = hi;
        if (pair) dl[base * tsz + idx] = (T)(ad - (double)hi);
      }
      for (int g = 0; g < ng; ++g) {
        const double c = A * 0.5 * bd.gJ[g];
        const T hi = (T)c;
        gh[base * kMaxGroups + g] = hi;
        if (pair) gl[base * kMaxGroups + g] = (T)(c - (double)hi);
      }
    }
  const std::vector<T> *src[4] = {&dh, &dl, &gh, &gl};
  for (int w = 0; w < 4; ++w) {
    r.coef[w] = arena.take<char>(coef_bytes(r, w));
    KPM_REQUIRE(r.coef[w] != nullptr, KPM_ENOMEM, "workspace too small for the step coefficients");
    KPM_CUDA(cudaMemcpyAsync(r.coef[w], src[w]->data(), src[w]->size() * sizeof(T),
                             cudaMemcpyHostToDevice, s));
  }
  return KPM_OK;
}

int upload_coefficients(MomentsRun &r, const std::vector<SectorDev> &sec, Arena &arena,
                        cudaStream_t s) {
  return r.precision == KPM_FP32 ? upload_coefficients_t<float>(r, sec, arena, s)
                                 : upload_coefficients_t<double>(r, sec, arena, s);
}

}  // namespace

int setup_run(MomentsRun &r, const double *a, const double *b, Arena &arena, cudaStream_t s,
              const int *out_index) {
  r.vA = arena.take<char>(r.vec_bytes);
  r.vB = arena.take<char>(r.vec_bytes);
  const size_t slots = std::max(r.plan.tiles.size(), r.block_L > 0 ? r.plan.hb_hi.size() : 0);
  const size_t n_partials = (r.list_stride > 0 ? 2 : 1) * slots * r.NQ;
  r.partials = arena.take<double>(std::max<size_t>(1, n_partials));
  r.sums = arena.take<double>((size_t)r.S * r.plan.n_sectors * r.NQ);
  r.counters = arena.take<int>((size_t)2 * r.S);
  r.flag = arena.take<int>(1);
  KPM_REQUIRE(r.vA && r.vB && r.partials && r.sums && r.counters && r.flag, KPM_ENOMEM,
              "workspace too small for the moment run");
  std::vector<SectorDev> sec(r.plan.n_sectors);
  for (int i = 0; i < r.plan.n_sectors; ++i) {
    KPM_REQUIRE(a[i] > 0.0 && std::isfinite(a[i]) && std::isfinite(b[i]), KPM_EINVAL,
                "sector %d: rescaling a = %g, b = %g (need a > 0, finite)", i, a[i], b[i]);
    sec[i].row0 = r.plan.row0[i];
    sec[i].dim = r.plan.dim[i];
    sec[i].n_up = r.plan.n_up[i];
    sec[i].hb_begin = r.plan.hb_begin[i];
    sec[i].inv_a = 1.0 / a[i];
    sec[i].b = b[i];
    sec[i].Mval = r.plan.n_up[i] < 0 ? 0.0 : r.plan.n_up[i] - 0.5 * r.plan.N;
    sec[i].out_index = out_index ? out_index[i] : i;
    sec[i].pad2 = 0;
  }
  KPM_TRY(upload_tables(r.plan, sec, arena, s, &r.tb));
  if (r.list_stride > 0) {
    r.lists = arena.take<uint32_t>((size_t)r.plan.total_rows * r.list_stride);
    KPM_REQUIRE(r.lists != nullptr, KPM_ENOMEM, "workspace too small for the neighbour lists");
    ListArgs la;
    la.lists = r.lists;
    la.tb = r.tb;
    la.stride = r.list_stride;
    la.rstride = (uint64_t)r.list_stride;
    la.estride = 1;
    la.crow = (uint32_t)(r.lay.Rp / r.lay.vec_width);
    la.batch = list_pad(r.precision, r.lay.cpl, r.lay.gpw);
    la.zero_chunk = (uint32_t)r.plan.total_rows * la.crow;
    const size_t row_bytes = (size_t)r.lay.Rp * r.lay.elem;
    const size_t zero_off = (size_t)r.plan.total_rows * row_bytes;  // the zero row of both vectors
    KPM_CUDA(cudaMemsetAsync(static_cast<char *>(r.vA) + zero_off, 0, row_bytes, s));
    KPM_CUDA(cudaMemsetAsync(static_cast<char *>(r.vB) + zero_off, 0, row_bytes, s));
    const int grid = (int)std::min<int64_t>((int64_t)r.plan.tiles.size(), (int64_t)8 * sm_count());
    build_lists_kernel<<<grid, kThreads, 0, s>>>(la, r.bonds);
    KPM_CUDA(cudaGetLastError());
    count_launches(1);
    KPM_TRY(upload_coefficients(r, sec, arena, s));
  }
  if (r.block_L > 0) {
    // sector of every hi-block, and each sector's block range (for the sums)
    const size_t nblk = r.plan.hb_hi.size();
    std::vector<int32_t> bsec(nblk), ranges(2 * (size_t)r.plan.n_sectors);
    for (int i = 0; i < r.plan.n_sectors; ++i) {
      const int32_t b0 = r.plan.hb_begin[i];
      const int32_t b1 = i + 1 < r.plan.n_sectors ? r.plan.hb_begin[i + 1] : (int32_t)nblk;
      for (int32_t b = b0; b < b1; ++b) bsec[b] = i;
      ranges[i] = b0;
      ranges[r.plan.n_sectors + i] = b1;
    }
    int32_t *dsec = arena.take<int32_t>(nblk);
    r.blk_ranges = arena.take<int32_t>(ranges.size());
    KPM_REQUIRE(dsec && r.blk_ranges, KPM_ENOMEM, "workspace too small for the hi-block tables");
    KPM_CUDA(cudaMemcpyAsync(dsec, bsec.data(), nblk * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    KPM_CUDA(cudaMemcpyAsync(r.blk_ranges, ranges.data(), ranges.size() * sizeof(int32_t),
                             cudaMemcpyHostToDevice, s));
    r.blk_sector = dsec;
    r.tbb = r.tb;
    r.tbb.tile_begin = r.blk_ranges;
    r.tbb.tile_end = r.blk_ranges + r.plan.n_sectors;
    r.tbb.n_tiles = (int32_t)nblk;
    KPM_TRY(upload_coefficients(r, sec, arena, s));
  }
  if (r.per_vector) {
    int64_t *cd = arena.take<int64_t>(r.cd_chunks.size());
    r.cd_part = arena.take<double>((size_t)r.n_cd * r.lay.R * 2);
    r.sums_r = arena.take<double>((size_t)r.S * r.plan.n_sectors * r.lay.R * 2);
    KPM_REQUIRE(cd && r.cd_part && r.sums_r, KPM_ENOMEM,
                "workspace too small for the per-vector moments");
    KPM_CUDA(cudaMemcpyAsync(cd, r.cd_chunks.data(), r.cd_chunks.size() * sizeof(int64_t),
                             cudaMemcpyHostToDevice, s));
    r.cd_dev = cd;
  }
  KPM_CUDA(cudaMemsetAsync(r.counters, 0, sizeof(int) * 2 * r.S, s));
  KPM_CUDA(cudaMemsetAsync(r.flag, 0, sizeof(int), s));
  void *fn = pick_kernel(r);
  int per_sm = 0;
  if (r.block_L > 0 && step_smem(r) > 48 * 1024)
    KPM_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)step_smem(r)));
  KPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, step_smem(r)));
  per_sm = std::max(per_sm, 1);
  if (r.knobs.blocks_per_sm > 0) per_sm = std::min(per_sm, r.knobs.blocks_per_sm);
  const int64_t items = r.block_L > 0 ? (int64_t)r.plan.hb_hi.size() : (int64_t)r.plan.tiles.size();
  r.grid = (int)std::min<int64_t>((int64_t)per_sm * sm_count(), items);
  r.grid = std::max(r.grid, 1);
  return KPM_OK;
}

int launch_build_lists(const TablesDev &tb, const BondsDev &bd, int64_t n_tiles, uint32_t *lists,
                       int stride, uint32_t crow, int batch, uint32_t zero_chunk, cudaStream_t s,
                       uint64_t entry_stride) {
  ListArgs la;
  la.lists = lists;
  la.tb = tb;
  la.stride = stride;
  la.rstride = entry_stride == 1 ? (uint64_t)stride : 1;
  la.estride = entry_stride;
  la.crow = crow;
  la.batch = batch;
  la.zero_chunk = zero_chunk;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(n_tiles, (int64_t)8 * sm_count()));
  void *args[] = {(void *)&la, (void *)&bd};
  KPM_CUDA(cudaLaunchKernel((void *)build_lists_kernel, dim3(grid), dim3(kThreads), args, 0, s));
  count_launches(1);
  return KPM_OK;
}

int launch_init(const MomentsRun &r, void *v0, uint64_t seed, uint64_t r0, cudaStream_t s,
                bool uniform) {
  InitArgs a;
  a.uniform = uniform ? 1 : 0;
  a.basis = (!uniform && r.vectors == kVecBasis) ? 1 : 0;
  a.v0 = v0;
  a.tb = r.tb;
  a.seed = seed;
  a.r0 = r0;
  a.R = r.lay.R;
  a.Rp = r.lay.Rp;
  a.G = r.lay.G;
  a.gpw = r.lay.gpw;
  const int grid = (int)std::min<int64_t>((int64_t)r.plan.tiles.size(), (int64_t)8 * sm_count());
  if (r.precision == KPM_FP32)
    init_vectors_kernel<float><<<grid, kThreads, 0, s>>>(a);
  else
    init_vectors_kernel<double><<<grid, kThreads, 0, s>>>(a);
  KPM_CUDA(cudaGetLastError());
  count_launches(1);
  return KPM_OK;
}

int launch_step(const MomentsRun &r, const void *x, void *zy, int first, int step, cudaStream_t s) {
  StepArgs a;
  a.x = x;
  a.zy = zy;
  a.tb = r.tb;
  a.partials = r.partials;
  a.sums = r.sums + (size_t)step * r.plan.n_sectors * r.NQ;
  a.queue = r.counters + 2 * step;
  a.done = r.counters + 2 * step + 1;
  a.Rp = r.lay.Rp;
  a.G = r.lay.G;
  a.gpw = r.lay.gpw;
  a.first = first;
  a.half_n = 0.5 * r.plan.N;
  a.prev_partials = nullptr;
  a.prev_sums = nullptr;
  CoefDev cf{r.coef[0], r.coef[1], r.coef[2], r.coef[3]};
  if (r.list_stride > 0) {
    // alternate tile slots; the previous step's slot is reduced by this launch
    const size_t slot = r.plan.tiles.size() * r.NQ;
    a.partials = r.partials + (step & 1) * slot;
    if (step > 0) {
      a.prev_partials = r.partials + ((step - 1) & 1) * slot;
      a.prev_sums = r.sums + (size_t)(step - 1) * r.plan.n_sectors * r.NQ;
    }
  }
  if (r.block_L > 0) {
    // the hi-block kernel writes one slot per block; the sums follow in block order
    cudaEvent_t b0 = nullptr, b1 = nullptr;
    const bool bprof = r.profile && profiling();
    if (bprof) {
      KPM_CUDA(cudaEventCreate(&b0));
      KPM_CUDA(cudaEventCreate(&b1));
      KPM_CUDA(cudaEventRecord(b0, s));
    }
    KPM_TRY(launch_block_step(r, x, zy, first, r.partials, a.queue, cf, s));
    count_launches(1);
    if (bprof) {
      KPM_CUDA(cudaEventRecord(b1, s));
      profile_push(b0, b1);
    }
    reduce_tile_sums_kernel<2><<<r.plan.n_sectors, kThreads, 0, s>>>(r.partials, r.tbb, a.sums);
    KPM_CUDA(cudaGetLastError());
    count_launches(1);
    return KPM_OK;
  }
  void *fn = pick_kernel(r);
  const uint32_t *lists = r.lists;
  int stride = r.list_stride;
  void *args_q[] = {(void *)&a, (void *)&r.bonds};
  void *args_l[] = {(void *)&a, (void *)&r.bonds, (void *)&lists, (void *)&stride, (void *)&cf};
  void **args = r.list_stride > 0 ? args_l : args_q;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  const bool prof = r.profile && profiling();
  if (prof) {
    KPM_CUDA(cudaEventCreate(&e0));
    KPM_CUDA(cudaEventCreate(&e1));
    KPM_CUDA(cudaEventRecord(e0, s));
  }
  KPM_CUDA(cudaLaunchKernel(fn, dim3(r.grid), dim3(kThreads), args, step_smem(r), s));
  count_launches(1);
  if (prof) {
    KPM_CUDA(cudaEventRecord(e1, s));
    profile_push(e0, e1);
  }
  return KPM_OK;
}

int launch_finish(const MomentsRun &r, cudaStream_t s) {
  if (r.list_stride == 0) return KPM_OK;
  const int last = r.S - 1;
  const double *ts = r.partials + (last & 1) * r.plan.tiles.size() * r.NQ;
  double *out = r.sums + (size_t)last * r.plan.n_sectors * r.NQ;
  if (r.NQ == 6)
    reduce_tile_sums_kernel<6><<<r.plan.n_sectors, kThreads, 0, s>>>(ts, r.tb, out);
  else
    reduce_tile_sums_kernel<2><<<r.plan.n_sectors, kThreads, 0, s>>>(ts, r.tb, out);
  KPM_CUDA(cudaGetLastError());
  count_launches(1);
  return KPM_OK;
}

int launch_column_dots(const MomentsRun &r, const void *x, const void *y, int step,
                       cudaStream_t s) {
  if (!r.per_vector) return KPM_OK;
  ColArgs a;
  a.x = x;
  a.y = y;
  a.chunks = r.cd_dev;
  a.part = r.cd_part;
  a.R = r.lay.R;
  a.Rp = r.lay.Rp;
  if (r.precision == KPM_FP32)
    column_dots_kernel<float><<<r.n_cd, kThreads, 0, s>>>(a);
  else
    column_dots_kernel<double><<<r.n_cd, kThreads, 0, s>>>(a);
  KPM_CUDA(cudaGetLastError());
  double *out = r.sums_r + (size_t)step * r.plan.n_sectors * r.lay.R * 2;
  column_reduce_kernel<<<r.plan.n_sectors, kThreads, 0, s>>>(r.cd_part, r.cd_dev + 3 * (size_t)r.n_cd,
                                                             out, r.lay.R);
  KPM_CUDA(cudaGetLastError());
  count_launches(2);
  return KPM_OK;
}

int launch_assemble(const MomentsRun &r, double *mu, double *mu_M, double *mu_M2, cudaStream_t s,
                    double *mu_r) {
  KPM_TRY(launch_finish(r, s));
  if (r.per_vector && mu_r != nullptr) {
    AssembleRArgs ar;
    ar.sums_r = r.sums_r;
    ar.sectors = r.tb.sectors;
    ar.mu_r = mu_r;
    ar.n_sectors = r.plan.n_sectors;
    ar.K = r.K;
    ar.R = r.lay.R;
    const int64_t tot = (int64_t)r.plan.n_sectors * r.lay.R * r.K;
    assemble_r_kernel<<<(int)std::min<int64_t>(4096, (tot + 255) / 256), 256, 0, s>>>(ar);
    KPM_CUDA(cudaGetLastError());
    count_launches(1);
  }
  AssembleArgs a;
  a.sums = r.sums;
  a.sectors = r.tb.sectors;
  a.mu = mu;
  a.mu_M = mu_M;
  a.mu_M2 = mu_M2;
  a.flag = r.flag;
  a.n_sectors = r.plan.n_sectors;
  a.K = r.K;
  a.NQ = r.NQ;
  a.inv_R = 1.0 / r.lay.R;
  const int total = r.plan.n_sectors * r.K;
  assemble_kernel<<<(total + 255) / 256, 256, 0, s>>>(a);
  KPM_CUDA(cudaGetLastError());
  count_launches(1);
  return KPM_OK;
}

int prepare_job(const kpm_model *m, int n_sectors, const int32_t *n_up, int K, int R,
                int precision, MomentsJob *job, const Knobs &knobs, int vectors,
                bool per_vector) {
  KPM_TRY(validate_model(m));
  KPM_TRY(validate_sectors(m, n_sectors, n_up));
  job->n_sectors = n_sectors;
  job->K = K;
  job->nup_main.clear();
  job->nup_side.clear();
  job->map_main.clear();
  job->map_side.clear();
  for (int i = 0; i < n_sectors; ++i) {
    const int64_t min_dim = knobs.side_min_dim >= 0 ? knobs.side_min_dim : kFP32MinSectorDim;
    const bool small = precision == KPM_FP32 && kpm_sector_dim(m->n_sites, n_up[i]) < min_dim;
    (small ? job->nup_side : job->nup_main).push_back(n_up[i]);
    (small ? job->map_side : job->map_main).push_back(i);
  }
  job->has_main = !job->nup_main.empty();
  job->has_side = !job->nup_side.empty();
  if (job->has_main)
    KPM_TRY(prepare_run(m, (int)job->nup_main.size(), job->nup_main.data(), K, R, precision,
                        &job->main, knobs, vectors, per_vector));
  if (job->has_side) {
    KPM_TRY(prepare_run(m, (int)job->nup_side.size(), job->nup_side.data(), K, R, KPM_FP64,
                        &job->side, knobs, vectors, per_vector));
    job->side.profile = false;
  }
  return KPM_OK;
}

size_t job_bytes(const MomentsJob &job) {
  return (job.has_main ? run_bytes(job.main) : 0) + (job.has_side ? run_bytes(job.side) : 0);
}

int setup_job(MomentsJob &job, const double *a, const double *b, Arena &arena, cudaStream_t s) {
  for (int part = 0; part < 2; ++part) {
    const bool has = part == 0 ? job.has_main : job.has_side;
    if (!has) continue;
    MomentsRun &r = part == 0 ? job.main : job.side;
    const std::vector<int> &map = part == 0 ? job.map_main : job.map_side;
    std::vector<double> as(map.size()), bs(map.size());
    for (size_t i = 0; i < map.size(); ++i) {
      as[i] = a[map[i]];
      bs[i] = b[map[i]];
    }
    KPM_TRY(setup_run(r, as.data(), bs.data(), arena, s, map.data()));
  }
  return KPM_OK;
}

namespace {

// Forks `side` from `s` and joins it back when it goes out of scope, also on
// an early error return, so that work queued on `s` afterwards (such as the
// release of the workspace) is ordered after everything queued on `side`.
struct ForkJoin {
  cudaStream_t s = nullptr, side = nullptr;
  cudaEvent_t ev = nullptr;
  int fork(cudaStream_t main, cudaStream_t other) {
    KPM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    KPM_CUDA(cudaEventRecord(ev, main));
    KPM_CUDA(cudaStreamWaitEvent(other, ev, 0));
    s = main;
    side = other;
    return KPM_OK;
  }
  ~ForkJoin() {
    if (ev == nullptr) return;
    if (side != nullptr && cudaEventRecord(ev, side) == cudaSuccess) cudaStreamWaitEvent(s, ev, 0);
    cudaEventDestroy(ev);
  }
};

}  // namespace

int run_job(MomentsJob &job, uint64_t seed, uint64_t r0, double *mu, double *mu_M, double *mu_M2,
            cudaStream_t s, cudaStream_t side, double *mu_r) {
  const bool fork = side != nullptr && job.has_main && job.has_side;
  cudaStream_t ss = fork ? side : s;
  ForkJoin fj;
  if (fork) KPM_TRY(fj.fork(s, ss));
  // The two runs are independent; with a side stream their launches are
  // interleaved so that the small FP64 run fills the main run's idle SMs.
  MomentsRun *runs[2] = {job.has_main ? &job.main : nullptr, job.has_side ? &job.side : nullptr};
  cudaStream_t st[2] = {s, ss};
  void *xs[2] = {nullptr, nullptr}, *zs[2] = {nullptr, nullptr};
  const int S = job.K / 2;
  for (int k = 0; k < 2; ++k) {
    if (!runs[k]) continue;
    KPM_TRY(launch_init(*runs[k], runs[k]->vA, seed, r0, st[k]));
    KPM_TRY(launch_step(*runs[k], runs[k]->vA, runs[k]->vB, 1, 0, st[k]));
    KPM_TRY(launch_column_dots(*runs[k], runs[k]->vA, runs[k]->vB, 0, st[k]));
    xs[k] = runs[k]->vB;
    zs[k] = runs[k]->vA;
    if (!fork) {
      // serial: all steps of this run, then the next run
      for (int step = 1; step < S; ++step) {
        KPM_TRY(launch_step(*runs[k], xs[k], zs[k], 0, step, st[k]));
        KPM_TRY(launch_column_dots(*runs[k], xs[k], zs[k], step, st[k]));
        std::swap(xs[k], zs[k]);
      }
      KPM_TRY(launch_assemble(*runs[k], mu, mu_M, mu_M2, st[k], mu_r));
    }
  }
  if (fork) {
    for (int step = 1; step < S; ++step)
      for (int k = 0; k < 2; ++k) {
        KPM_TRY(launch_step(*runs[k], xs[k], zs[k], 0, step, st[k]));
        KPM_TRY(launch_column_dots(*runs[k], xs[k], zs[k], step, st[k]));
        std::swap(xs[k], zs[k]);
      }
    for (int k = 0; k < 2; ++k) KPM_TRY(launch_assemble(*runs[k], mu, mu_M, mu_M2, st[k], mu_r));
  }
  return KPM_OK;  // fj joins the side stream into s here
}

// A non-blocking, lowest-priority stream per device for the FP64 side run,
// created on first use and kept until the process exits.
int side_stream(cudaStream_t *out) {
  static std::mutex mtx;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  KPM_CUDA(cudaGetDevice(&dev));
  KPM_REQUIRE(dev >= 0 && dev < 64, KPM_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(mtx);
  if (streams[dev] == nullptr) {
    int lo = 0, hi = 0;
    KPM_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    KPM_CUDA(cudaStreamCreateWithPriority(&streams[dev], cudaStreamNonBlocking, lo));
  }
  *out = streams[dev];
  return KPM_OK;
}

}  // namespace kpm

using namespace kpm;

namespace kpm {

// Options of a kpm_moments_ex call, checked; NULL means the defaults.
int read_opts(const kpm_opts *o, kpm_opts *out) {
  kpm_opts d{};
  d.precision = KPM_FP64;
  d.vectors = KPM_VECTORS_RADEMACHER;
  if (o != nullptr) d = *o;
  KPM_REQUIRE(d.precision == KPM_FP64 || d.precision == KPM_FP32, KPM_EINVAL, "precision %d",
              d.precision);
  KPM_REQUIRE(d.vectors == KPM_VECTORS_RADEMACHER || d.vectors == KPM_VECTORS_BASIS, KPM_EINVAL,
              "vectors %d", d.vectors);
  KPM_REQUIRE(d.ckpt_interval >= 0, KPM_EINVAL, "ckpt_interval %d", d.ckpt_interval);
  *out = d;
  return KPM_OK;
}

// The knobs for this problem: the autotuner's choice when asked for and
// available, the defaults otherwise.
Knobs knobs_for(const kpm_model *m, int n_sectors, const int32_t *n_up, int K, int R,
                const kpm_opts &o);

int moments_impl(const kpm_model *model, int32_t n_sectors, const int32_t *n_up, const double *a,
                 const double *b, double eps, int32_t n_moments, int32_t R, uint64_t seed,
                 uint64_t r0, const kpm_opts &o, double *mu, double *mu_M, double *mu_M2,
                 double *mu_r, int32_t on_device, void *workspace, size_t ws_bytes,
                 void *stream_ptr) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
  KPM_REQUIRE(mu != nullptr, KPM_EINVAL, "mu is NULL");
  KPM_REQUIRE((mu_r != nullptr) == (o.per_vector != 0), KPM_EINVAL,
              "mu_r must be given exactly when opts.per_vector is set");
  MomentsJob job;
  KPM_TRY(prepare_job(model, n_sectors, n_up, n_moments, R, o.precision, &job,
                      knobs_for(model, n_sectors, n_up, n_moments, R, o), o.vectors,
                      o.per_vector != 0));
  std::vector<double> av, bv;
  if (a == nullptr || b == nullptr) {
    av.resize(n_sectors);
    bv.resize(n_sectors);
    int rc = kpm_bounds(model, n_sectors, n_up, eps, 100, 1e-8, splitmix64(seed ^ 0x5EEDB0D5ull),
                        av.data(), bv.data(), nullptr, nullptr, nullptr, 0, stream_ptr);
    if (rc != KPM_OK && rc != KPM_ENOTCONV) return rc;
    a = av.data();
    b = bv.data();
  }
  const size_t SK = (size_t)n_sectors * n_moments;
  const size_t out_bytes = align256(SK * sizeof(double));
  const size_t r_bytes = mu_r ? align256(SK * R * sizeof(double)) : 0;
  const size_t need = job_bytes(job) + (on_device ? 0 : 3 * out_bytes + r_bytes);
  Workspace ws;
  KPM_TRY(ws.acquire(workspace, ws_bytes, need, stream));
  Arena arena{reinterpret_cast<char *>(ws.ptr), ws.size, 0};
  KPM_TRY(setup_job(job, a, b, arena, stream));
  double *dmu = mu, *dmuM = mu_M, *dmuM2 = mu_M2, *dmur = mu_r;
  if (!on_device) {
    dmu = arena.take<double>(SK);
    dmuM = mu_M ? arena.take<double>(SK) : nullptr;
    dmuM2 = mu_M2 ? arena.take<double>(SK) : nullptr;
    dmur = mu_r ? arena.take<double>(SK * R) : nullptr;
    KPM_REQUIRE(dmu && (!mu_M || dmuM) && (!mu_M2 || dmuM2) && (!mu_r || dmur), KPM_ENOMEM,
                "workspace too small");
  }
  cudaStream_t side = nullptr;
  if (job.has_main && job.has_side) KPM_TRY(side_stream(&side));
  KPM_TRY(run_job(job, seed, r0, dmu, dmuM, dmuM2, stream, side, dmur));
  const size_t nbytes = SK * sizeof(double);
  if (!on_device) {
    KPM_CUDA(cudaMemcpyAsync(mu, dmu, nbytes, cudaMemcpyDeviceToHost, stream));
    if (mu_M) KPM_CUDA(cudaMemcpyAsync(mu_M, dmuM, nbytes, cudaMemcpyDeviceToHost, stream));
    if (mu_M2) KPM_CUDA(cudaMemcpyAsync(mu_M2, dmuM2, nbytes, cudaMemcpyDeviceToHost, stream));
    if (mu_r) KPM_CUDA(cudaMemcpyAsync(mu_r, dmur, nbytes * R, cudaMemcpyDeviceToHost, stream));
  }
  int flags[2] = {0, 0};
  if (job.has_main)
    KPM_CUDA(cudaMemcpyAsync(&flags[0], job.main.flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
  if (job.has_side)
    KPM_CUDA(cudaMemcpyAsync(&flags[1], job.side.flag, sizeof(int), cudaMemcpyDeviceToHost, stream));
  KPM_CUDA(cudaStreamSynchronize(stream));
  if (flags[0] || flags[1]) {
    set_error("some |mu_n| > 1 + 1e-6: the rescaled spectrum leaves [-1, 1]");
    return KPM_EBOUNDS;
  }
  return KPM_OK;
}

}  // namespace kpm

extern "C" size_t kpm_moments_workspace_size(const kpm_model *model, int32_t n_sectors,
                                             const int32_t *n_up, int32_t n_moments, int32_t R,
                                             int32_t precision) {
  kpm_opts o{};
  o.precision = precision;
  return kpm_moments_ex_workspace_size(model, n_sectors, n_up, n_moments, R, &o);
}

extern "C" size_t kpm_moments_ex_workspace_size(const kpm_model *model, int32_t n_sectors,
                                                const int32_t *n_up, int32_t n_moments,
                                                int32_t R, const kpm_opts *opts) {
  kpm_opts o;
  if (read_opts(opts, &o) != KPM_OK) return 0;
  MomentsJob job;
  if (prepare_job(model, n_sectors, n_up, n_moments, R, o.precision, &job,
                  knobs_for(model, n_sectors, n_up, n_moments, R, o), o.vectors,
                  o.per_vector != 0) != KPM_OK)
    return 0;
  return job_bytes(job);
}

extern "C" int kpm_moments(const kpm_model *model, int32_t n_sectors, const int32_t *n_up,
                           const double *a, const double *b, double eps, int32_t n_moments,
                           int32_t R, uint64_t seed, uint64_t r0, int32_t precision, double *mu,
                           double *mu_M, double *mu_M2, int32_t on_device, void *workspace,
                           size_t ws_bytes, void *stream_ptr) {
  clear_error();
  kpm_opts o{};
  o.precision = precision;
  KPM_TRY(read_opts(&o, &o));
  return moments_impl(model, n_sectors, n_up, a, b, eps, n_moments, R, seed, r0, o, mu, mu_M,
                      mu_M2, nullptr, on_device, workspace, ws_bytes, stream_ptr);
}

extern "C" int kpm_moments_ex(const kpm_model *model, int32_t n_sectors, const int32_t *n_up,
                              const double *a, const double *b, double eps, int32_t n_moments,
                              int32_t R, uint64_t seed, uint64_t r0, const kpm_opts *opts,
                              double *mu, double *mu_M, double *mu_M2, double *mu_r,
                              int32_t on_device, void *workspace, size_t ws_bytes,
                              void *stream_ptr) {
  clear_error();
  kpm_opts o;
  KPM_TRY(read_opts(opts, &o));
  return moments_impl(model, n_sectors, n_up, a, b, eps, n_moments, R, seed, r0, o, mu, mu_M,
                      mu_M2, mu_r, on_device, workspace, ws_bytes, stream_ptr);
}
