// Reverse-mode derivative of the Chebyshev moments with respect to the
// couplings J_b (the paper has no derivative; this differentiates the
// recursion that implements Eq. E-2-6 / E-2-7).
//
// Forward: v_1 = H' v_0, v_{n+1} = 2 H' v_n - v_{n-1} (n = 1 .. S-1),
// mu^W_0 = <v_0|W|v_0>, mu^W_1 = <v_1|W|v_0>, mu^W_{2n} = 2<v_n|W|v_n> - mu^W_0,
// mu^W_{2n+1} = 2<v_{n+1}|W|v_n> - mu^W_1 for W = 1, M, M^2 (diagonal, commuting
// with H).  With cotangents gbar^W_i = dL/dmu^W_i and the per-state weight
// w_i(s) = gbar_i + gbar^M_i M(s) + gbar^{M2}_i M(s)^2, the adjoint vectors
// lambda_n = dL/dv_n obey
//   lambda_n = d_n + 2 H' lambda_{n+1} - lambda_{n+2},   lambda_{S+1} = lambda_{S+2} = 0,
//   d_n = 4 w_{2n} v_n + 2 w_{2n+1} v_{n+1} + c_n v_{n-1},
//   c_n = 2 w_{2n-1} for n >= 2,  c_1 = w_1 - sum_{j>=1} w_{2j+1}
// (w_i = 0 for i >= K), and with a, b fixed and H_b = S_i . S_j,
//   dL/dJ_b = (1/R) [sum_{n=1}^{S-1} (2/a) <lambda_{n+1}, H_b v_n> + (1/a) <lambda_1, H_b v_0>]
// (the dot products run over all R vectors; 1/R is the average in mu_n).
// The reverse sweep regenerates v_{n-1} = 2 H' v_n - v_{n+1} in the same pass
// that builds lambda_n (both gather the same bit-flipped neighbours) and
// resets the pair (v_{n-1}, v_n) from the copies stored every ckpt_interval
// steps of the forward pass, which bounds the round-off of the regeneration.
// <lambda_{n+1}, H_b v_n> = sum_s v_n(s) [H_b lambda_{n+1}](s) is accumulated
// from the gathers of lambda_{n+1}: per parameter class in registers when
// there are at most kMaxClasses classes, and otherwise per bond (up to 256),
// in per-warp shared-memory slots fed by a warp-wide butterfly sum of each
// bond's term; the tile's bond sums are then added per class.  With
// own(s) = <v_n(s), lambda_{n+1}(s)>, the term of bond b at state s is
// own(s)/4 if its bits agree and <v_n(s), lambda_{n+1}(s ^ mask_b)>/2 -
// own(s)/4 if they differ.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "kpm_device.cuh"
#include "kpm_run.h"

namespace kpm {

struct AdjArgs {
  const double2 *Vg;   // v_n (gathered)
  double2 *Vo;         // v_{n+1} in, v_{n-1} out
  const double2 *Lg;   // lambda_{n+1} (gathered)
  double2 *Lo;         // lambda_{n+2} in, lambda_n out
  TablesDev tb;
  const double *G[3];  // cotangents [sector][K] (NULL = 0)
  const double *hbar;  // [sector][3]
  double *gpart;       // [n_tiles][pstride]: per class (few classes) or per bond (many)
  int *queue;
  int n, S, K, mode;   // mode 0: lambda_S = d_S; 1: general step; 2: gradient of n = 0
  int lz_zero;         // lambda_{n+2} = 0
  int Rp, G_lanes, gpw, n_classes;
  int pstride;         // entries per tile in gpart
  int cstart[kMaxClasses + 1];
  double half_n;
  // neighbour lists of the forward run (list path): per state a header with
  // the anti-aligned bond count of each coupling group, then the first chunk
  // of every flipped neighbour's row, group by group; every group lies in one
  // parameter class gclass[g], which has nbclass[p] bonds in all
  const uint32_t *lists;
  int list_stride;
  int gclass[kMaxGroups];
  int nbclass[kMaxClasses];
};

__device__ __forceinline__ double cot_at(const double *g, int sec, int K, int i) {
  return (g != nullptr && i >= 0 && i < K) ? g[(int64_t)sec * K + i] : 0.0;
}

template <int CPL, bool FULL>
__global__ void __launch_bounds__(kThreads)
    adjoint_step_kernel(const __grid_constant__ AdjArgs a, const __grid_constant__ BondsDev bd) {
  using V = double2;
  __shared__ double s_red[kWarps * kMaxClasses];
  __shared__ int s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = a.G_lanes;
  const int grp = lane / G, sub = lane - grp * G;
  const bool active = grp < a.gpw;
  const int64_t crow = a.Rp / 2;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.queue, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= a.tb.n_tiles) break;
    const Tile tile = a.tb.tiles[t];
    const SectorDev sd = a.tb.sectors[tile.sector];
    const int sec = tile.sector;
    const int n = a.n;
    // weight triples (gbar, gbar^M, gbar^M2) of the direct terms
    double w4[3], w2p[3], wc[3];
    for (int q = 0; q < 3; ++q) {
      w4[q] = 4.0 * cot_at(a.G[q], sec, a.K, 2 * n);
      w2p[q] = 2.0 * cot_at(a.G[q], sec, a.K, 2 * n + 1);
      wc[q] = (n >= 2) ? 2.0 * cot_at(a.G[q], sec, a.K, 2 * n - 1) : a.hbar[sec * 3 + q];
    }
    const double A = 2.0 * sd.inv_a;
    const bool full_tile = sd.n_up < 0;
    double acc[kMaxClasses];
#pragma unroll
    for (int p = 0; p < kMaxClasses; ++p) acc[p] = 0.0;
    uint32_t hb = tile.b_first;
    if (active) {
      for (uint32_t u = warp * a.gpw + grp; u < tile.count; u += kWarps * a.gpw) {
        const int64_t row = tile.row0 + u;
        uint64_t s;
        if (full_tile)
          s = (uint64_t)(row - sd.row0);
        else
          s = sector_unrank(tile.rank0 + u, sd.n_up, tile.b_last, hb, a.tb);
        const double M = full_tile ? (double)__popcll(s) - a.half_n : sd.Mval;
        const double c4 = w4[0] + M * (w4[1] + M * w4[2]);
        const double c2p = w2p[0] + M * (w2p[1] + M * w2p[2]);
        const double cm = wc[0] + M * (wc[1] + M * wc[2]);
        if (a.mode == 0) {
          // lambda_S = c_S v_{S-1}; here Vg = v_{S-1}
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const V v = a.Vg[row * crow + sub + c * G];
            a.Lo[row * crow + sub + c * G] = make_double2(cm * v.x, cm * v.y);
          }
          continue;
        }
        double d = bd.J_quarter_sum;
        V hv[CPL], hl[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          hv[c] = make_double2(0.0, 0.0);
          hl[c] = make_double2(0.0, 0.0);
        }
        V vn[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) vn[c] = a.Vg[row * crow + sub + c * G];
        double dsig[kMaxClasses];
        double tnb[kMaxClasses];
#pragma unroll
        for (int p = 0; p < kMaxClasses; ++p) {
          dsig[p] = 0.0;
          tnb[p] = 0.0;
          if (p < a.n_classes) {
            for (int b = a.cstart[p]; b < a.cstart[p + 1]; ++b) {
              const uint64_t m = bd.mask[b];
              const uint64_t tt = s & m;
              if (tt != 0 && tt != m) {
                d -= 0.5 * bd.J[b];
                dsig[p] -= 0.25;
                const uint64_t f = s ^ m;
                const int64_t nr =
                    sd.row0 + (full_tile ? (int64_t)f : (int64_t)sector_rank(f, a.tb));
                const double jh = 0.5 * bd.J[b];
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                  const V l = __ldg(a.Lg + nr * crow + sub + c * G);
                  hl[c].x = fma(jh, l.x, hl[c].x);
                  hl[c].y = fma(jh, l.y, hl[c].y);
                  tnb[p] = fma(vn[c].x, l.x, fma(vn[c].y, l.y, tnb[p]));
                  if (a.mode == 1) {
                    const V v = __ldg(a.Vg + nr * crow + sub + c * G);
                    hv[c].x = fma(jh, v.x, hv[c].x);
                    hv[c].y = fma(jh, v.y, hv[c].y);
                  }
                }
              } else {
                dsig[p] += 0.25;
              }
            }
          }
        }
        double own = 0.0;  // <v_n(s), lambda_{n+1}(s)> over this lane's values
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int64_t idx = row * crow + sub + c * G;
          const V lg = a.Lg[idx];
          own = fma(vn[c].x, lg.x, fma(vn[c].y, lg.y, own));
          if (a.mode == 1) {
            const V vp = a.Vo[idx];  // v_{n+1}
            V vm;                    // v_{n-1} = A (H - b) v_n - v_{n+1}
            vm.x = A * (fma(d, vn[c].x, hv[c].x) - sd.b * vn[c].x) - vp.x;
            vm.y = A * (fma(d, vn[c].y, hv[c].y) - sd.b * vn[c].y) - vp.y;
            a.Vo[idx] = vm;
            V lz = make_double2(0.0, 0.0);
            if (!a.lz_zero) lz = a.Lo[idx];
            V ln;
            ln.x = c4 * vn[c].x + c2p * vp.x + cm * vm.x +
                   A * (fma(d, lg.x, hl[c].x) - sd.b * lg.x) - lz.x;
            ln.y = c4 * vn[c].y + c2p * vp.y + cm * vm.y +
                   A * (fma(d, lg.y, hl[c].y) - sd.b * lg.y) - lz.y;
            a.Lo[idx] = ln;
          }
        }
#pragma unroll
        for (int p = 0; p < kMaxClasses; ++p) acc[p] += 0.5 * tnb[p] + dsig[p] * own;
      }
    }
    if (a.mode != 0) {
      block_sum<kMaxClasses>(acc, s_red);
      if (threadIdx.x == 0) {
        const double f = (a.mode == 2 ? 1.0 : 2.0) * sd.inv_a;
        for (int p = 0; p < a.n_classes; ++p) a.gpart[(int64_t)t * a.pstride + p] += f * acc[p];
      }
    } else {
      __syncthreads();
    }
  }
}

// The same step with per-bond sums (more than kMaxClasses parameter classes).
// The loop over a warp's states is warp-uniform so that every lane takes
// part in the per-bond butterfly sums.
template <int CPL>
__global__ void __launch_bounds__(kThreads)
    adjoint_step_bonds_kernel(const __grid_constant__ AdjArgs a, const __grid_constant__ BondsDev bd) {
  using V = double2;
  extern __shared__ double s_acc[];  // [kWarps][n_bonds]
  __shared__ int s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = a.G_lanes;
  const int grp = lane / G, sub = lane - grp * G;
  const bool active = grp < a.gpw;
  const int64_t crow = a.Rp / 2;
  const int nb = bd.n_bonds;
  double *wacc = s_acc + warp * nb;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.queue, 1);
    for (int b = lane; b < nb; b += 32) wacc[b] = 0.0;
    __syncthreads();
    const int t = s_tile;
    if (t >= a.tb.n_tiles) break;
    const Tile tile = a.tb.tiles[t];
    const SectorDev sd = a.tb.sectors[tile.sector];
    const int sec = tile.sector;
    const int n = a.n;
    double w4[3], w2p[3], wc[3];
    for (int q = 0; q < 3; ++q) {
      w4[q] = 4.0 * cot_at(a.G[q], sec, a.K, 2 * n);
      w2p[q] = 2.0 * cot_at(a.G[q], sec, a.K, 2 * n + 1);
      wc[q] = (n >= 2) ? 2.0 * cot_at(a.G[q], sec, a.K, 2 * n - 1) : a.hbar[sec * 3 + q];
    }
    const double A = 2.0 * sd.inv_a;
    const bool full_tile = sd.n_up < 0;
    uint32_t hb = tile.b_first;
    for (uint32_t ub = warp * a.gpw; ub < tile.count; ub += kWarps * a.gpw) {
      const uint32_t u = ub + grp;
      const bool valid = active && u < tile.count;
      const int64_t row = tile.row0 + u;
      uint64_t s = 0;
      if (valid)
        s = full_tile ? (uint64_t)(row - sd.row0)
                      : sector_unrank(tile.rank0 + u, sd.n_up, tile.b_last, hb, a.tb);
      const double M = full_tile ? (double)__popcll(s) - a.half_n : sd.Mval;
      const double c4 = w4[0] + M * (w4[1] + M * w4[2]);
      const double c2p = w2p[0] + M * (w2p[1] + M * w2p[2]);
      const double cm = wc[0] + M * (wc[1] + M * wc[2]);
      if (a.mode == 0) {
        if (valid) {
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const V v = a.Vg[row * crow + sub + c * G];
            a.Lo[row * crow + sub + c * G] = make_double2(cm * v.x, cm * v.y);
          }
        }
        continue;
      }
      V vn[CPL], lo[CPL], hv[CPL], hl[CPL];
      double own = 0.0;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        vn[c] = make_double2(0.0, 0.0);
        lo[c] = make_double2(0.0, 0.0);
        hv[c] = make_double2(0.0, 0.0);
        hl[c] = make_double2(0.0, 0.0);
        if (valid) {
          vn[c] = a.Vg[row * crow + sub + c * G];
          lo[c] = a.Lg[row * crow + sub + c * G];
          own = fma(vn[c].x, lo[c].x, fma(vn[c].y, lo[c].y, own));
        }
      }
      double d = bd.J_quarter_sum;
      for (int b = 0; b < nb; ++b) {
        double term = 0.0;
        if (valid) {
          const uint64_t m = bd.mask[b];
          const uint64_t tt = s & m;
          if (tt != 0 && tt != m) {
            d -= 0.5 * bd.J[b];
            const uint64_t f = s ^ m;
            const int64_t nr = sd.row0 + (full_tile ? (int64_t)f : (int64_t)sector_rank(f, a.tb));
            const double jh = 0.5 * bd.J[b];
            double tnb = 0.0;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
              const V l = __ldg(a.Lg + nr * crow + sub + c * G);
              hl[c].x = fma(jh, l.x, hl[c].x);
              hl[c].y = fma(jh, l.y, hl[c].y);
              tnb = fma(vn[c].x, l.x, fma(vn[c].y, l.y, tnb));
              if (a.mode == 1) {
                const V v = __ldg(a.Vg + nr * crow + sub + c * G);
                hv[c].x = fma(jh, v.x, hv[c].x);
                hv[c].y = fma(jh, v.y, hv[c].y);
              }
            }
            term = 0.5 * tnb - 0.25 * own;
          } else {
            term = 0.25 * own;
          }
        }
        term = warp_sum(term);  // lane 0 holds the warp's sum for bond b
        if (lane == 0) wacc[b] += term;
      }
      if (valid && a.mode == 1) {
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int64_t idx = row * crow + sub + c * G;
          const V vp = a.Vo[idx];
          V vm;
          vm.x = A * (fma(d, vn[c].x, hv[c].x) - sd.b * vn[c].x) - vp.x;
          vm.y = A * (fma(d, vn[c].y, hv[c].y) - sd.b * vn[c].y) - vp.y;
          a.Vo[idx] = vm;
          V lz = make_double2(0.0, 0.0);
          if (!a.lz_zero) lz = a.Lo[idx];
          V ln;
          ln.x = c4 * vn[c].x + c2p * vp.x + cm * vm.x + A * (fma(d, lo[c].x, hl[c].x) - sd.b * lo[c].x) - lz.x;
          ln.y = c4 * vn[c].y + c2p * vp.y + cm * vm.y + A * (fma(d, lo[c].y, hl[c].y) - sd.b * lo[c].y) - lz.y;
          a.Lo[idx] = ln;
        }
      }
    }
    __syncthreads();
    if (a.mode != 0) {
      const double f = (a.mode == 2 ? 1.0 : 2.0) * sd.inv_a;
      for (int b = threadIdx.x; b < nb; b += kThreads) {
        double v = 0.0;
        for (int w = 0; w < kWarps; ++w) v += s_acc[w * nb + b];
        a.gpart[(int64_t)t * a.pstride + b] += f * v;
      }
    }
    __syncthreads();
  }
}

// The same step driven by the forward run's neighbour lists (coupling groups
// that each lie in one parameter class): the flipped neighbours' rows come from
// the list instead of bond tests and ranks, which every lane of a state would
// otherwise repeat.
// Neighbours whose rows the list-driven adjoint loads together.
#ifndef KPM_ADJ_BATCH
#define KPM_ADJ_BATCH 4
#endif
constexpr int kAdjBatch = KPM_ADJ_BATCH;

#ifndef KPM_ADJ_MIN_BLOCKS
#define KPM_ADJ_MIN_BLOCKS 3
#endif

template <int CPL, bool FULL>
__global__ void __launch_bounds__(kThreads, KPM_ADJ_MIN_BLOCKS)
    adjoint_list_kernel(const __grid_constant__ AdjArgs a, const __grid_constant__ BondsDev bd) {
  using V = double2;
  __shared__ double s_red[kWarps * kMaxClasses];
  __shared__ int s_tile;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int G = a.G_lanes;
  const int grp = lane / G, sub = lane - grp * G;
  const bool active = grp < a.gpw;
  const int64_t crow = a.Rp / 2;
  const int ng = bd.n_groups;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.queue, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= a.tb.n_tiles) break;
    const Tile tile = a.tb.tiles[t];
    const SectorDev sd = a.tb.sectors[tile.sector];
    const int sec = tile.sector;
    const int n = a.n;
    double w4[3], w2p[3], wc[3];
    for (int q = 0; q < 3; ++q) {
      w4[q] = 4.0 * cot_at(a.G[q], sec, a.K, 2 * n);
      w2p[q] = 2.0 * cot_at(a.G[q], sec, a.K, 2 * n + 1);
      wc[q] = (n >= 2) ? 2.0 * cot_at(a.G[q], sec, a.K, 2 * n - 1) : a.hbar[sec * 3 + q];
    }
    const double A = 2.0 * sd.inv_a;
    const bool full_tile = sd.n_up < 0;
    // per coupling group: sums over the tile's states of <v_n(s), lambda(s ^ mask)>
    // over the group's anti-aligned bonds, and of cnt_g * <v_n(s), lambda(s)>;
    // and the sum of <v_n(s), lambda(s)>.  They are turned into per-class sums
    // once per tile.
    double acc_tg[kMaxGroups], acc_ao[kMaxGroups], acc_own = 0.0;
#pragma unroll
    for (int g = 0; g < kMaxGroups; ++g) {
      acc_tg[g] = 0.0;
      acc_ao[g] = 0.0;
    }
    if (active) {
      for (uint32_t u = warp * a.gpw + grp; u < tile.count; u += kWarps * a.gpw) {
        const int64_t row = tile.row0 + u;
        const double M = full_tile ? (double)__popcll((uint64_t)(row - sd.row0)) - a.half_n : sd.Mval;
        const double c4 = w4[0] + M * (w4[1] + M * w4[2]);
        const double c2p = w2p[0] + M * (w2p[1] + M * w2p[2]);
        const double cm = wc[0] + M * (wc[1] + M * wc[2]);
        if (a.mode == 0) {
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const V v = a.Vg[row * crow + sub + c * G];
            a.Lo[row * crow + sub + c * G] = make_double2(cm * v.x, cm * v.y);
          }
          continue;
        }
        const uint32_t *Ls = a.lists + (size_t)row * a.list_stride;
        const uint32_t hdr = __ldg(Ls);
        V vn[CPL], lg[CPL], hv[CPL], hl[CPL];
        double own = 0.0;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int64_t idx = row * crow + sub + c * G;
          vn[c] = a.Vg[idx];
          lg[c] = a.Lg[idx];
          own = fma(vn[c].x, lg[c].x, fma(vn[c].y, lg[c].y, own));
          hv[c] = make_double2(0.0, 0.0);
          hl[c] = make_double2(0.0, 0.0);
        }
        double d = bd.J_quarter_sum;
        acc_own += own;
        int e = 1;
#pragma unroll
        for (int g = 0; g < kMaxGroups; ++g) {
          if (g < ng) {
            const int cnt = (int)((hdr >> (8 * g)) & 255u);
            const double jh = 0.5 * bd.gJ[g];
            d -= cnt * jh;
            // the group's neighbour rows are summed first; the coupling and the
            // dot product with v_n(s) are applied once per group
            V sl[CPL], sv[CPL];
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
              sl[c] = make_double2(0.0, 0.0);
              sv[c] = make_double2(0.0, 0.0);
            }
            // kAdjBatch neighbours at a time: their indices, then their rows, so
            // that the loads of a batch are in flight together
            for (int i0 = 0; i0 < cnt; i0 += kAdjBatch) {
              uint32_t ci[kAdjBatch];
#pragma unroll
              for (int q = 0; q < kAdjBatch; ++q) ci[q] = i0 + q < cnt ? __ldg(Ls + e + i0 + q) : 0u;
              V l[kAdjBatch][CPL], v[kAdjBatch][CPL];
#pragma unroll
              for (int q = 0; q < kAdjBatch; ++q) {
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                  const bool ok = i0 + q < cnt;
                  l[q][c] = ok ? __ldg(a.Lg + ci[q] + sub + c * G) : make_double2(0.0, 0.0);
                  v[q][c] = (ok && a.mode == 1) ? __ldg(a.Vg + ci[q] + sub + c * G) : make_double2(0.0, 0.0);
                }
              }
#pragma unroll
              for (int q = 0; q < kAdjBatch; ++q) {
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                  sl[c].x += l[q][c].x;
                  sl[c].y += l[q][c].y;
                  sv[c].x += v[q][c].x;
                  sv[c].y += v[q][c].y;
                }
              }
            }
            e += cnt;
            double tg = 0.0;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
              hl[c].x = fma(jh, sl[c].x, hl[c].x);
              hl[c].y = fma(jh, sl[c].y, hl[c].y);
              hv[c].x = fma(jh, sv[c].x, hv[c].x);
              hv[c].y = fma(jh, sv[c].y, hv[c].y);
              tg = fma(vn[c].x, sl[c].x, fma(vn[c].y, sl[c].y, tg));
            }
            acc_tg[g] += tg;
            acc_ao[g] += cnt * own;
          }
        }
        if (a.mode == 1) {
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int64_t idx = row * crow + sub + c * G;
            const V vp = a.Vo[idx];  // v_{n+1}
            V vm;                    // v_{n-1} = A (H - b) v_n - v_{n+1}
            vm.x = A * (fma(d, vn[c].x, hv[c].x) - sd.b * vn[c].x) - vp.x;
            vm.y = A * (fma(d, vn[c].y, hv[c].y) - sd.b * vn[c].y) - vp.y;
            a.Vo[idx] = vm;
            V lz = make_double2(0.0, 0.0);
            if (!a.lz_zero) lz = a.Lo[idx];
            V ln;
            ln.x = c4 * vn[c].x + c2p * vp.x + cm * vm.x + A * (fma(d, lg[c].x, hl[c].x) - sd.b * lg[c].x) - lz.x;
            ln.y = c4 * vn[c].y + c2p * vp.y + cm * vm.y + A * (fma(d, lg[c].y, hl[c].y) - sd.b * lg[c].y) - lz.y;
            a.Lo[idx] = ln;
          }
        }
      }
    }
    // per class: sum over its bonds of <v_n(s), lambda(s ^ mask)>/2 (anti-aligned)
    // and +-own/4 (aligned / anti-aligned)
    double acc[kMaxClasses];
#pragma unroll
    for (int p = 0; p < kMaxClasses; ++p) acc[p] = 0.25 * a.nbclass[p] * acc_own;
#pragma unroll
    for (int g = 0; g < kMaxGroups; ++g) {
      if (g < ng) {
        const int pg = a.gclass[g];
#pragma unroll
        for (int p = 0; p < kMaxClasses; ++p)
          if (p == pg) acc[p] += 0.5 * acc_tg[g] - 0.5 * acc_ao[g];
      }
    }
    if (a.mode != 0) {
      block_sum<kMaxClasses>(acc, s_red);
      if (threadIdx.x == 0) {
        const double f = (a.mode == 2 ? 1.0 : 2.0) * sd.inv_a;
        for (int p = 0; p < a.n_classes; ++p) a.gpart[(int64_t)t * a.pstride + p] += f * acc[p];
      }
    } else {
      __syncthreads();
    }
  }
}

// hbar[s][q] = gbar^q_1 - sum_{j>=1} gbar^q_{2j+1}
__global__ void adjoint_hbar_kernel(const double *g0, const double *g1, const double *g2,
                                    double *hbar, int S, int K) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= S * 3) return;
  const int s = i / 3, q = i % 3;
  const double *g = q == 0 ? g0 : (q == 1 ? g1 : g2);
  double h = 0.0;
  if (g) {
    h = K > 1 ? g[(int64_t)s * K + 1] : 0.0;
    for (int j = 3; j < K; j += 2) h -= g[(int64_t)s * K + j];
  }
  hbar[i] = h;
}

// dL/dtheta_p = (1/R) sum over tiles (tile order) of the entries e in
// [estart[p], estart[p+1]) of gpart[t][e] (the class itself, or the class's
// bonds); the 1/R is the average over the random vectors in
// mu_n = (1/R) sum_r <r|T_n|r>, left out of the per-vector recursion above.
__global__ void adjoint_final_kernel(const double *gpart, int n_tiles, int pstride,
                                     const int *estart, double inv_R, double *out) {
  const int p = blockIdx.x;
  double v = 0.0;
  for (int e = estart[p]; e < estart[p + 1]; ++e)
    for (int t = threadIdx.x; t < n_tiles; t += 32) v += gpart[(int64_t)t * pstride + e];
  v = warp_sum(v);
  if (threadIdx.x == 0) out[p] = v * inv_R;
}

namespace {

template <int CPL, bool FULL>
void *adj_ptr() {
  return reinterpret_cast<void *>(&adjoint_step_kernel<CPL, FULL>);
}

template <int CPL>
void *adjb_ptr() {
  return reinterpret_cast<void *>(&adjoint_step_bonds_kernel<CPL>);
}

void *pick_adj_bonds(int cpl) {
  switch (cpl) {
    case 1: return adjb_ptr<1>();
    case 2: return adjb_ptr<2>();
    case 3: return adjb_ptr<3>();
    case 4: return adjb_ptr<4>();
    default: return adjb_ptr<8>();
  }
}

template <int CPL, bool FULL>
void *adjl_ptr() {
  return reinterpret_cast<void *>(&adjoint_list_kernel<CPL, FULL>);
}

void *pick_adj_list(int cpl, bool full) {
  if (cpl == 1) return full ? adjl_ptr<1, true>() : adjl_ptr<1, false>();
  return full ? adjl_ptr<2, true>() : adjl_ptr<2, false>();
}

void *pick_adj(int cpl, bool full) {
  switch (cpl) {
    case 1: return full ? adj_ptr<1, true>() : adj_ptr<1, false>();
    case 2: return full ? adj_ptr<2, true>() : adj_ptr<2, false>();
    case 3: return full ? adj_ptr<3, true>() : adj_ptr<3, false>();
    case 4: return full ? adj_ptr<4, true>() : adj_ptr<4, false>();
    default: return full ? adj_ptr<8, true>() : adj_ptr<8, false>();
  }
}

struct AdjPlan {
  MomentsRun run;
  kpm_model sorted;              // bonds sorted by class
  std::vector<int32_t> bi, bj;
  std::vector<double> J;
  int cstart[kMaxClasses + 1];
  std::vector<int> estart;       // per class: first entry of gpart (class or bond index)
  int n_classes = 0;
  bool by_bond = false;          // more than kMaxClasses classes: per-bond sums
  int pstride = kMaxClasses;
  int k = 32, n_ckpt = 0;
  size_t bytes = 0;
};

int prepare_adjoint(const kpm_model *m, const int32_t *bond_class, int n_classes, int n_sectors,
                    const int32_t *n_up, int K, int R, int ckpt, AdjPlan *ap,
                    int vectors = kVecRademacher) {
  KPM_TRY(validate_model(m));
  int P = n_classes;
  if (bond_class == nullptr) P = m->n_bonds;
  KPM_REQUIRE(P >= 1 && P <= kMaxBonds, KPM_EINVAL, "n_classes = %d outside 1..%d", P, kMaxBonds);
  std::vector<int> cls(m->n_bonds);
  for (int b = 0; b < m->n_bonds; ++b) {
    cls[b] = bond_class ? bond_class[b] : b;
    KPM_REQUIRE(cls[b] >= 0 && cls[b] < P, KPM_EINVAL, "bond_class[%d] = %d", b, cls[b]);
  }
  ap->n_classes = P;
  ap->bi.clear();
  ap->bj.clear();
  ap->J.clear();
  for (int p = 0; p < P; ++p) {
    if (p < kMaxClasses) ap->cstart[p] = (int)ap->bi.size();
    for (int b = 0; b < m->n_bonds; ++b)
      if (cls[b] == p) {
        ap->bi.push_back(m->bi[b]);
        ap->bj.push_back(m->bj[b]);
        ap->J.push_back(m->J[b]);
      }
  }
  std::vector<int> cs(P + 1);
  {
    // class boundaries in the class-sorted bond list, for any number of classes
    int pos = 0;
    for (int p = 0; p < P; ++p) {
      cs[p] = pos;
      for (int b = 0; b < m->n_bonds; ++b) pos += cls[b] == p ? 1 : 0;
    }
    cs[P] = pos;
  }
  for (int p = P; p <= kMaxClasses; ++p) ap->cstart[p] = (int)ap->bi.size();
  ap->by_bond = P > kMaxClasses;
  if (ap->by_bond) {
    ap->estart = cs;  // gpart holds per-bond sums in class-sorted bond order
    ap->pstride = std::max(1, m->n_bonds);
  } else {
    ap->estart.resize(P + 1);
    for (int p = 0; p <= P; ++p) ap->estart[p] = p;
    ap->pstride = kMaxClasses;
  }
  ap->sorted.n_sites = m->n_sites;
  ap->sorted.n_bonds = m->n_bonds;
  ap->sorted.bi = ap->bi.data();
  ap->sorted.bj = ap->bj.data();
  ap->sorted.J = ap->J.data();
  KPM_TRY(prepare_run(&ap->sorted, n_sectors, n_up, K, R, KPM_FP64, &ap->run, Knobs(), vectors));
  ap->k = ckpt > 0 ? ckpt : 32;
  ap->n_ckpt = (ap->run.S + ap->k - 1) / ap->k;
  const MomentsRun &r = ap->run;
  const size_t SK = (size_t)n_sectors * K;
  ap->bytes = run_bytes(r) + 2 * r.vec_bytes + (size_t)ap->n_ckpt * 2 * r.vec_bytes +
              align256(std::max<size_t>(1, r.plan.tiles.size()) *
                       std::max(kMaxClasses, m->n_bonds) * 8) +
              align256((size_t)n_sectors * 3 * 8) + align256((size_t)(r.S + 2) * 4) +
              3 * align256(SK * 8) + align256((size_t)kMaxBonds * 8) +
              align256((size_t)(kMaxBonds + 1) * 4) + 1024;
  return KPM_OK;
}

}  // namespace

}  // namespace kpm

using namespace kpm;

extern "C" size_t kpm_moments_backward_workspace_size(const kpm_model *model, int32_t n_sectors,
                                                      const int32_t *n_up, int32_t n_moments,
                                                      int32_t R, int32_t ckpt_interval) {
  AdjPlan ap;
  if (model == nullptr) return 0;
  std::vector<int32_t> cls(model->n_bonds, 0);
  if (prepare_adjoint(model, cls.data(), 1, n_sectors, n_up, n_moments, R, ckpt_interval, &ap) !=
      KPM_OK)
    return 0;
  return ap.bytes;
}

namespace {

int backward_impl(const kpm_model *model, const int32_t *bond_class, int32_t n_classes,
                  int32_t n_sectors, const int32_t *n_up, const double *a, const double *b,
                  int32_t n_moments, int32_t R, uint64_t seed, uint64_t r0, int32_t precision,
                  int32_t vectors, int32_t ckpt_interval, const double *dL_dmu,
                  const double *dL_dmu_M, const double *dL_dmu_M2, double *dL_dtheta,
                  int32_t on_device, void *workspace, size_t ws_bytes, void *stream_ptr) {
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
  KPM_REQUIRE(precision == KPM_FP64, KPM_EINVAL, "the adjoint runs in FP64 only");
  KPM_REQUIRE(a && b && dL_dmu && dL_dtheta, KPM_EINVAL, "NULL argument");
  AdjPlan ap;
  KPM_TRY(prepare_adjoint(model, bond_class, n_classes, n_sectors, n_up, n_moments, R,
                          ckpt_interval, &ap, vectors));
  MomentsRun &run = ap.run;
  Workspace ws;
  KPM_TRY(ws.acquire(workspace, ws_bytes, ap.bytes, stream));
  Arena arena{reinterpret_cast<char *>(ws.ptr), ws.size, 0};
  KPM_TRY(setup_run(run, a, b, arena, stream));
  double2 *LA = arena.take<double2>(run.vec_bytes / 16);
  double2 *LB = arena.take<double2>(run.vec_bytes / 16);
  std::vector<char *> ck(2 * ap.n_ckpt);
  for (auto &p : ck) p = arena.take<char>(run.vec_bytes);
  const size_t n_gpart = std::max<size_t>(1, run.plan.tiles.size()) * ap.pstride;
  double *gpart = arena.take<double>(n_gpart);
  int *estart = arena.take<int>(ap.estart.size());
  double *hbar = arena.take<double>((size_t)n_sectors * 3);
  int *queues = arena.take<int>((size_t)run.S + 2);
  const size_t SK = (size_t)n_sectors * n_moments;
  double *dg[3] = {nullptr, nullptr, nullptr};
  double *dtheta = arena.take<double>(std::max(kMaxClasses, ap.n_classes));
  bool ok = LA && LB && gpart && estart && hbar && queues && dtheta;
  for (auto p : ck) ok = ok && p;
  const double *gin[3] = {dL_dmu, dL_dmu_M, dL_dmu_M2};
  for (int q = 0; q < 3; ++q) {
    if (!gin[q]) continue;
    if (on_device) {
      dg[q] = const_cast<double *>(gin[q]);
    } else {
      dg[q] = arena.take<double>(SK);
      ok = ok && dg[q];
      if (dg[q]) KPM_CUDA(cudaMemcpyAsync(dg[q], gin[q], SK * 8, cudaMemcpyHostToDevice, stream));
    }
  }
  KPM_REQUIRE(ok, KPM_ENOMEM, "workspace too small for the adjoint");
  KPM_CUDA(cudaMemsetAsync(gpart, 0, n_gpart * 8, stream));
  KPM_CUDA(cudaMemcpyAsync(estart, ap.estart.data(), ap.estart.size() * sizeof(int),
                           cudaMemcpyHostToDevice, stream));
  KPM_CUDA(cudaMemsetAsync(queues, 0, ((size_t)run.S + 2) * 4, stream));
  adjoint_hbar_kernel<<<(n_sectors * 3 + 127) / 128, 128, 0, stream>>>(dg[0], dg[1], dg[2], hbar,
                                                                       n_sectors, n_moments);
  KPM_CUDA(cudaGetLastError());
  count_launches(1);

  // forward pass with checkpoints of (v_j, v_{j+1}), j = 0, k, 2k, ...
  const int S = run.S;
  KPM_TRY(launch_init(run, run.vA, seed, r0, stream));
  KPM_TRY(launch_step(run, run.vA, run.vB, 1, 0, stream));
  KPM_CUDA(cudaMemcpyAsync(ck[0], run.vA, run.vec_bytes, cudaMemcpyDeviceToDevice, stream));
  KPM_CUDA(cudaMemcpyAsync(ck[1], run.vB, run.vec_bytes, cudaMemcpyDeviceToDevice, stream));
  void *x = run.vB, *zy = run.vA;  // x = v_n, zy = v_{n-1}
  for (int n = 1; n < S; ++n) {
    KPM_TRY(launch_step(run, x, zy, 0, n, stream));
    std::swap(x, zy);  // x = v_{n+1}, zy = v_n
    if (n % ap.k == 0) {
      const int c = n / ap.k;
      KPM_CUDA(cudaMemcpyAsync(ck[2 * c], zy, run.vec_bytes, cudaMemcpyDeviceToDevice, stream));
      KPM_CUDA(cudaMemcpyAsync(ck[2 * c + 1], x, run.vec_bytes, cudaMemcpyDeviceToDevice, stream));
    }
  }
  // reverse sweep: x = v_S, zy = v_{S-1}
  AdjArgs ar;
  std::memset(&ar, 0, sizeof(ar));
  ar.tb = run.tb;
  for (int q = 0; q < 3; ++q) ar.G[q] = dg[q];
  ar.hbar = hbar;
  ar.gpart = gpart;
  ar.S = S;
  ar.K = n_moments;
  ar.Rp = run.lay.Rp;
  ar.G_lanes = run.lay.G;
  ar.gpw = run.lay.gpw;
  ar.n_classes = ap.n_classes;
  ar.pstride = ap.pstride;
  for (int p = 0; p <= kMaxClasses; ++p) ar.cstart[p] = ap.cstart[p];
  ar.half_n = 0.5 * run.plan.N;
  // list path: the forward run has neighbour lists (at most 2 chunks per lane)
  // and every coupling group lies in one parameter class
  bool use_lists = !ap.by_bond && run.list_stride > 0 && run.lists != nullptr &&
                   (run.lay.cpl == 1 || run.lay.cpl == 2) && run.bonds.n_groups > 0;
  if (use_lists) {
    for (int p = 0; p < kMaxClasses; ++p)
      ar.nbclass[p] = p < ap.n_classes ? ap.cstart[p + 1] - ap.cstart[p] : 0;
    for (int g = 0; g < run.bonds.n_groups && use_lists; ++g) {
      int pg = -1;
      for (int k = run.bonds.gstart[g]; k < run.bonds.gstart[g + 1]; ++k) {
        const int b = run.bonds.order[k];  // index into the class-sorted bond list
        int p = 0;
        while (p + 1 <= ap.n_classes && ap.cstart[p + 1] <= b) ++p;
        if (pg < 0) pg = p;
        if (p != pg) use_lists = false;
      }
      ar.gclass[g] = pg;
    }
    ar.lists = run.lists;
    ar.list_stride = run.list_stride;
  }
  void *fn = ap.by_bond ? pick_adj_bonds(run.lay.cpl)
                        : (use_lists ? pick_adj_list(run.lay.cpl, run.plan.any_full)
                                     : pick_adj(run.lay.cpl, run.plan.any_full));
  const size_t smem = ap.by_bond ? (size_t)kWarps * std::max(1, model->n_bonds) * sizeof(double) : 0;
  int per_sm = 0;
  KPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
  int dev = 0, nsm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * nsm, (int64_t)run.plan.tiles.size()));
  auto launch = [&](int mode, int n, const void *Vg, void *Vo, const void *Lg, void *Lo, int lz_zero,
                    int qslot) -> int {
    ar.mode = mode;
    ar.n = n;
    ar.Vg = (const double2 *)Vg;
    ar.Vo = (double2 *)Vo;
    ar.Lg = (const double2 *)Lg;
    ar.Lo = (double2 *)Lo;
    ar.lz_zero = lz_zero;
    ar.queue = queues + qslot;
    void *args[] = {(void *)&ar, (void *)&run.bonds};
    KPM_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, smem, stream));
    count_launches(1);
    return KPM_OK;
  };
  void *Vg = zy, *Vo = x;  // top: lambda_S = c_S v_{S-1}
  void *Lg = LB, *Lo = LA;
  KPM_TRY(launch(0, S, Vg, Vo, Lg, Lo, 1, S + 1));  // LA = lambda_S
  // step n: Vg = v_n, Vo = v_{n+1}, Lg = lambda_{n+1}, Lo = lambda_{n+2}
  Lg = LA;
  Lo = LB;
  for (int n = S - 1; n >= 1; --n) {
    KPM_TRY(launch(1, n, Vg, Vo, Lg, Lo, n == S - 1 ? 1 : 0, n));
    // now Vo = v_{n-1}, Lo = lambda_n
    std::swap(Vg, Vo);  // Vg = v_{n-1}, Vo = v_n
    std::swap(Lg, Lo);  // Lg = lambda_n, Lo = lambda_{n+1}
    const int j = n - 1;
    if (j % ap.k == 0) {
      const int c = j / ap.k;
      KPM_CUDA(cudaMemcpyAsync(Vg, ck[2 * c], run.vec_bytes, cudaMemcpyDeviceToDevice, stream));
      KPM_CUDA(cudaMemcpyAsync(Vo, ck[2 * c + 1], run.vec_bytes, cudaMemcpyDeviceToDevice, stream));
    }
  }
  // n = 0: (1/a) <lambda_1, H_b v_0> with Vg = v_0, Lg = lambda_1
  KPM_TRY(launch(2, 0, Vg, Vo, Lg, Lo, 1, 0));
  adjoint_final_kernel<<<ap.n_classes, 32, 0, stream>>>(gpart, (int)run.plan.tiles.size(),
                                                        ap.pstride, estart, 1.0 / R, dtheta);
  KPM_CUDA(cudaGetLastError());
  count_launches(1);
  if (on_device)
    KPM_CUDA(cudaMemcpyAsync(dL_dtheta, dtheta, ap.n_classes * 8, cudaMemcpyDeviceToDevice, stream));
  else
    KPM_CUDA(cudaMemcpyAsync(dL_dtheta, dtheta, ap.n_classes * 8, cudaMemcpyDeviceToHost, stream));
  KPM_CUDA(cudaStreamSynchronize(stream));
  return KPM_OK;
}

}  // namespace

extern "C" int kpm_moments_backward(const kpm_model *model, const int32_t *bond_class,
                                    int32_t n_classes, int32_t n_sectors, const int32_t *n_up,
                                    const double *a, const double *b, int32_t n_moments, int32_t R,
                                    uint64_t seed, uint64_t r0, int32_t precision,
                                    int32_t ckpt_interval, const double *dL_dmu,
                                    const double *dL_dmu_M, const double *dL_dmu_M2,
                                    double *dL_dtheta, int32_t on_device, void *workspace,
                                    size_t ws_bytes, void *stream_ptr) {
  clear_error();
  return backward_impl(model, bond_class, n_classes, n_sectors, n_up, a, b, n_moments, R, seed, r0,
                       precision, KPM_VECTORS_RADEMACHER, ckpt_interval, dL_dmu, dL_dmu_M,
                       dL_dmu_M2, dL_dtheta, on_device, workspace, ws_bytes, stream_ptr);
}

extern "C" int kpm_moments_backward_ex(const kpm_model *model, const int32_t *bond_class,
                                       int32_t n_classes, int32_t n_sectors, const int32_t *n_up,
                                       const double *a, const double *b, int32_t n_moments,
                                       int32_t R, uint64_t seed, uint64_t r0,
                                       const kpm_opts *opts, const double *dL_dmu,
                                       const double *dL_dmu_M, const double *dL_dmu_M2,
                                       double *dL_dtheta, int32_t on_device, void *workspace,
                                       size_t ws_bytes, void *stream_ptr) {
  clear_error();
  kpm_opts o{};
  if (opts) o = *opts;
  KPM_REQUIRE(o.vectors == KPM_VECTORS_RADEMACHER || o.vectors == KPM_VECTORS_BASIS, KPM_EINVAL,
              "vectors %d", o.vectors);
  KPM_REQUIRE(o.per_vector == 0, KPM_EINVAL, "the adjoint has no per-vector form");
  return backward_impl(model, bond_class, n_classes, n_sectors, n_up, a, b, n_moments, R, seed, r0,
                       o.precision, o.vectors, o.ckpt_interval, dL_dmu, dL_dmu_M, dL_dmu_M2,
                       dL_dtheta, on_device, workspace, ws_bytes, stream_ptr);
}
