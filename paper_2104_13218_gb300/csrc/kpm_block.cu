// The Chebyshev step (Eq. E-2-6 / E-2-7 with H' of Eq. E-2-3) by hi-blocks,
// for S^z-sector runs whose rows fit one 16-byte chunk (one lane per state:
// R <= 4 in FP32, R <= 2 in FP64), such as the N = 34 ring.
//
// A sector's states are ordered by their value, so the states that share the
// bits at and above L (the "high" pattern h) form one contiguous hi-block,
// whose low parts are the L-bit patterns with c = n_up - popcount(h) set bits
// in increasing order (index j = colex rank of the low part).  The bonds of
// the Hamiltonian (Eq. E-3-1-1) then fall into three kinds:
//   - low bonds (both sites below L): the flipped state lies in the same
//     block, at index lo_rank[lo ^ mask]; the block's rows are staged in
//     shared memory, and so is lo_rank (16-bit), so these gathers never leave
//     the SM;
//   - high bonds (both sites at or above L): whether they are anti-aligned is
//     a property of the block, and the flipped state is the state with the
//     SAME index j in block h ^ mask.  Each such partner block is read as a
//     contiguous, coalesced stream, row j for state j;
//   - cross bonds (one site on each side): per block, which low bit value
//     makes the bond anti-aligned and the partner block (whose class is
//     c +- 1) are fixed; the partner row is lo_rank[lo ^ bit] in that block.
// One CTA processes one hi-block at a time, taken in order from an atomic
// queue, so the grid sweeps the vectors in memory order and the partner
// blocks of nearby high patterns are still in L2.  The block's dot products
// (FP32 form: compensated FP32 sums per thread over at most a few dozen
// states, then FP64) go to the block's own slot and are summed per sector in
// block order afterwards.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kpm_device.cuh"
#include "kpm_run.h"

namespace kpm {

namespace {

struct BlockArgs {
  const void *x;
  void *zy;
  TablesDev tb;
  const int32_t *blk_sector;
  double *partials;   // [n_blocks][2]
  int *queue;
  int n_blocks;
  int first;
  int table_size;
  CoefDev cf;
};

// 16-byte asynchronous copy global -> shared (L2 only).
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

// States per thread and iteration, and resident blocks per SM asked of the compiler.
#ifndef KPM_BLOCK_NS
#define KPM_BLOCK_NS 1
#endif
#ifndef KPM_BLOCK_HB
#define KPM_BLOCK_HB 8  // high-bond partner rows loaded together
#endif
#ifndef KPM_BLOCK_MIN_BLOCKS
#define KPM_BLOCK_MIN_BLOCKS 4
#endif
constexpr int NS = KPM_BLOCK_NS;

template <typename T>
__global__ void __launch_bounds__(kThreads, KPM_BLOCK_MIN_BLOCKS)
    cheb_block_kernel(const __grid_constant__ BlockArgs a, const __grid_constant__ BlockBondsDev bb) {
  using C = Chunk<T>;
  using V = typename C::type;
  constexpr bool PAIR = sizeof(T) == 4;
  extern __shared__ __align__(16) unsigned char s_dyn[];
  const int L = bb.L;
  const uint32_t nlo = 1u << L;
  uint16_t *s_lorank = reinterpret_cast<uint16_t *>(s_dyn);
  V *s_x = reinterpret_cast<V *>(s_dyn + ((nlo * 2 + 15) & ~15u));
  __shared__ int64_t s_hoff[kBlockMaxBonds];   // partner block rows of the anti-aligned high bonds
  __shared__ int32_t s_hgs[kMaxGroups + 1];    // ... grouped: entries s_hgs[g] .. s_hgs[g+1]
  __shared__ int64_t s_coff[kBlockMaxBonds];   // cross bonds: partner block row
  __shared__ uint8_t s_cneed[kBlockMaxBonds];  // cross bonds: low bit value that makes them anti-aligned
  __shared__ double s_red[kWarps * 2];
  __shared__ int s_blk;
  const V *__restrict__ x = reinterpret_cast<const V *>(a.x);
  V *__restrict__ zy = reinterpret_cast<V *>(a.zy);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kind = a.first ? 0 : 1;
  const T *dh_all = reinterpret_cast<const T *>(a.cf.diag_hi);
  const T *dl_all = reinterpret_cast<const T *>(a.cf.diag_lo);
  const T *gh_all = reinterpret_cast<const T *>(a.cf.grp_hi);
  const T *gl_all = reinterpret_cast<const T *>(a.cf.grp_lo);
  // colex ranks of all low patterns, once per CTA (every rank < 2^16)
  for (uint32_t i = tid; i < nlo; i += kThreads) s_lorank[i] = (uint16_t)__ldg(a.tb.lo_rank + i);
  const uint32_t nhi = 1u << a.tb.H;
  for (;;) {
    __syncthreads();  // the previous block's shared data is no longer read
    if (tid == 0) s_blk = atomicAdd(a.queue, 1);
    __syncthreads();
    const int b = s_blk;
    if (b >= a.n_blocks) break;
    const int sec = a.blk_sector[b];
    const SectorDev sd = a.tb.sectors[sec];
    const uint32_t h = __ldg(a.tb.hb_hi + b);
    const int c = sd.n_up - __popc(h);
    const uint32_t ls0 = __ldg(a.tb.lo_start + c);
    const uint32_t nc = __ldg(a.tb.lo_start + c + 1) - ls0;
    const int64_t rowb = sd.row0 + __ldg(a.tb.hb_off + b);
    // stage the block's own rows
    for (uint32_t j = tid; j < nc; j += kThreads) cp_async16(s_x + j, x + rowb + j);
    cp_async_commit();
    // block constants: partner blocks of the anti-aligned high bonds, grouped
    // (warp 0, one bond per lane), and the cross bonds' partner blocks (warp 1)
    if (warp == 0) {
      int base = 0;
      for (int g = 0; g < bb.n_groups; ++g) {
        if (lane == 0) s_hgs[g] = base;
        for (int k0 = bb.high_gs[g]; k0 < bb.high_gs[g + 1]; k0 += 32) {
          const int k = k0 + lane;
          bool anti = false;
          int64_t off = 0;
          if (k < bb.high_gs[g + 1]) {
            const uint32_t m = bb.high_mask[k];
            anti = __popc(h & m) == 1;
            if (anti) off = sd.row0 + __ldg(a.tb.hi_rank + (size_t)c * nhi + (h ^ m));
          }
          const uint32_t bal = __ballot_sync(0xffffffffu, anti);
          if (anti) s_hoff[base + __popc(bal & ((1u << lane) - 1u))] = off;
          base += __popc(bal);
        }
      }
      if (lane == 0) s_hgs[bb.n_groups] = base;
    } else if (warp == 1) {
      const int nx = bb.cross_gs[bb.n_groups];
      for (int k = lane; k < nx; k += 32) {
        const int jh = bb.cross_hi[k];
        const uint32_t hbit = (h >> jh) & 1u;
        // anti-aligned when the low bit differs from the high bit; the partner's
        // low part then has one set bit more (hbit = 1) or fewer (hbit = 0)
        const int c2 = c + (hbit ? 1 : -1);
        int64_t off = -1;
        if (c2 >= 0 && c2 <= L) off = sd.row0 + __ldg(a.tb.hi_rank + (size_t)c2 * nhi + (h ^ (1u << jh)));
        s_coff[k] = off;
        s_cneed[k] = (uint8_t)(hbit ^ 1u);
      }
    }
    cp_async_wait<0>();
    __syncthreads();
    const size_t cbase = (size_t)sec * 2 + kind;
    const T *dh = dh_all + cbase * a.table_size;
    const T *dl = dl_all + cbase * a.table_size;
    // the high bonds' flip counts per group are the same for the whole block
    int tbase = 0;
#pragma unroll
    for (int g = 0; g < kMaxGroups; ++g)
      if (g < bb.n_groups) tbase += (s_hgs[g + 1] - s_hgs[g]) * bb.tstride[g];
    KahanF kxx, kyx;
    double acc64[2] = {0.0, 0.0};
    const T *ghg = gh_all + cbase * kMaxGroups;
    const T *glg = gl_all + cbase * kMaxGroups;
    // NS states per thread and iteration, so that their loads are in flight together
    for (uint32_t j0 = tid; j0 < nc; j0 += kThreads * NS) {
      uint32_t jj[NS], lo[NS];
      bool ok[NS];
      V xv[NS], zv[NS], acc[NS];
      int tidx[NS];
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        jj[q] = j0 + q * kThreads;
        ok[q] = jj[q] < nc;
        const uint32_t jc = ok[q] ? jj[q] : j0;  // an idle slot repeats a valid state, unused
        jj[q] = jc;
        lo[q] = __ldg(a.tb.lo_list + ls0 + jc);
        xv[q] = s_x[jc];
        zv[q] = a.first ? V{} : __ldcs(zy + rowb + jc);
        acc[q] = V{};
        tidx[q] = tbase;
      }
#pragma unroll
      for (int g = 0; g < kMaxGroups; ++g) {
        if (g < bb.n_groups) {
          V gs[NS];
#pragma unroll
          for (int q = 0; q < NS; ++q) gs[q] = V{};
          // high bonds: coalesced rows of the partner blocks, KPM_BLOCK_HB at a
          // time (the count is the same for the whole block: no divergence)
          const int e0 = s_hgs[g], e1 = s_hgs[g + 1];
          for (int e = e0; e < e1; e += KPM_BLOCK_HB) {
            V v[KPM_BLOCK_HB][NS];
#pragma unroll
            for (int i = 0; i < KPM_BLOCK_HB; ++i) {
              if (e + i < e1) {
                const int64_t o = s_hoff[e + i];
#pragma unroll
                for (int q = 0; q < NS; ++q) v[i][q] = __ldg(x + o + jj[q]);
              } else {
#pragma unroll
                for (int q = 0; q < NS; ++q) v[i][q] = V{};
              }
            }
#pragma unroll
            for (int i = 0; i < KPM_BLOCK_HB; ++i) {
#pragma unroll
              for (int q = 0; q < NS; ++q) gs[q] = C::add(gs[q], v[i][q]);
            }
          }
          // cross bonds: a row of the partner block
          for (int k = bb.cross_gs[g]; k < bb.cross_gs[g + 1]; ++k) {
            const uint32_t bit = 1u << bb.cross_lo[k];
            const bool need = s_cneed[k] != 0;
            const int64_t co = s_coff[k];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
              if (((lo[q] & bit) != 0) == need) {
                tidx[q] += bb.tstride[g];
                gs[q] = C::add(gs[q], __ldg(x + co + s_lorank[lo[q] ^ bit]));
              }
            }
          }
          // low bonds: rows of this block, from shared memory
          for (int k = bb.low_gs[g]; k < bb.low_gs[g + 1]; ++k) {
            const uint32_t m = bb.low_mask[k];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
              const uint32_t t = lo[q] & m;
              if (t != 0 && t != m) {
                tidx[q] += bb.tstride[g];
                gs[q] = C::add(gs[q], s_x[s_lorank[lo[q] ^ m]]);
              }
            }
          }
          const T ghi = __ldg(ghg + g);
          const T glo = PAIR ? __ldg(glg + g) : (T)0;
#pragma unroll
          for (int q = 0; q < NS; ++q) {
            acc[q] = C::fma(ghi, gs[q], acc[q]);
            if (PAIR) acc[q] = C::fma(glo, gs[q], acc[q]);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < NS; ++q) {
        if (!ok[q]) continue;
        const T ad_hi = __ldg(dh + tidx[q]);
        V h = acc[q];
        if (PAIR) h = C::fma(__ldg(dl + tidx[q]), xv[q], h);
        const V y = C::fma_sub(ad_hi, xv[q], h, zv[q]);
        __stcs(zy + rowb + jj[q], y);
        using P2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
        P2 paa{}, pba{};
        C::dots(xv[q], y, paa, pba);
        if constexpr (sizeof(T) == 8) {
          acc64[0] += paa.x + paa.y;
          acc64[1] += pba.x + pba.y;
        } else {
          kxx.add(paa.x + paa.y);
          kyx.add(pba.x + pba.y);
        }
      }
    }
    if constexpr (sizeof(T) == 4) {
      acc64[0] = kxx.value();
      acc64[1] = kyx.value();
    }
    block_sum<2>(acc64, s_red);
    if (tid == 0) {
      a.partials[(int64_t)b * 2] = acc64[0];
      a.partials[(int64_t)b * 2 + 1] = acc64[1];
    }
  }
}

}  // namespace

size_t block_smem_bytes(const MomentsRun &r) {
  const size_t nlo = (size_t)1 << r.block_L;
  return ((nlo * 2 + 15) & ~size_t(15)) + (size_t)r.max_block * 16;
}

void *block_kernel_ptr(int precision) {
  return precision == KPM_FP32 ? reinterpret_cast<void *>(&cheb_block_kernel<float>)
                               : reinterpret_cast<void *>(&cheb_block_kernel<double>);
}

int launch_block_step(const MomentsRun &r, const void *x, void *zy, int first, double *partials,
                      int *queue, CoefDev cf, cudaStream_t s) {
  BlockArgs a;
  a.x = x;
  a.zy = zy;
  a.tb = r.tb;
  a.blk_sector = r.blk_sector;
  a.partials = partials;
  a.queue = queue;
  a.n_blocks = (int)r.plan.hb_hi.size();
  a.first = first;
  a.table_size = r.bonds.table_size;
  a.cf = cf;
  void *args[] = {(void *)&a, (void *)&r.bb};
  KPM_CUDA(cudaLaunchKernel(block_kernel_ptr(r.precision), dim3(r.grid), dim3(kThreads), args,
                            block_smem_bytes(r), s));
  return KPM_OK;
}

}  // namespace kpm
