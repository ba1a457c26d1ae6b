// Device helpers shared by the kernels of libkpm: the counter-based random
// signs, rank/unrank of S^z sector states, 16-byte vector chunks and warp
// reductions.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "kpm_internal.h"

namespace kpm {

// splitmix64 output for generator state x (Steele, Lea and Flood; the
// published mixing constants of the splitmix64 reference generator).
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Rank of bitstring t inside its popcount sector, from the split tables.
__device__ __forceinline__ uint32_t sector_rank(uint64_t t, const TablesDev &tb) {
  const uint32_t lomask = (1u << tb.L) - 1u;
  const uint32_t lo = (uint32_t)t & lomask;
  const uint32_t hi = (uint32_t)(t >> tb.L);
  const uint32_t c = __popc(lo);
  return __ldg(tb.lo_rank + lo) + __ldg(tb.hi_rank + ((size_t)c << tb.H) + hi);
}

// Walks hi-block index b forward to the block holding rank r (ranks of one
// caller only increase), then returns the bitstring of rank r in sector k.
__device__ __forceinline__ uint64_t sector_unrank(uint32_t r, int k, uint32_t b_last, uint32_t &b,
                                                  const TablesDev &tb) {
  while (b < b_last && __ldg(tb.hb_off + b + 1) <= r) ++b;
  const uint32_t hi = __ldg(tb.hb_hi + b);
  const int c = k - __popc(hi);
  const uint32_t lo = __ldg(tb.lo_list + __ldg(tb.lo_start + c) + (r - __ldg(tb.hb_off + b)));
  return ((uint64_t)hi << tb.L) | lo;
}

// Bitstring of rank r in sector k by binary search over the hi-blocks
// [b_lo, b_hi] (the block holding r is among them).
__device__ __forceinline__ uint64_t sector_unrank_search(uint32_t r, int k, uint32_t b_lo,
                                                         uint32_t b_hi, const TablesDev &tb) {
  while (b_lo < b_hi) {
    const uint32_t mid = (b_lo + b_hi + 1) >> 1;
    if (__ldg(tb.hb_off + mid) <= r)
      b_lo = mid;
    else
      b_hi = mid - 1;
  }
  const uint32_t hi = __ldg(tb.hb_hi + b_lo);
  const int c = k - __popc(hi);
  const uint32_t lo = __ldg(tb.lo_list + __ldg(tb.lo_start + c) + (r - __ldg(tb.hb_off + b_lo)));
  return ((uint64_t)hi << tb.L) | lo;
}

// Next larger integer with the same number of set bits (s != 0): the state of
// rank r + 1 in a sector, from the state of rank r.
__device__ __forceinline__ uint64_t next_same_popcount(uint64_t s) {
  const uint64_t t = s | (s - 1);
  const uint64_t nt = ~t;
  return (t + 1) | (((nt & (0 - nt)) - 1) >> (__ffsll((long long)s)));
}

// Packed two-wide FP32 arithmetic (PTX f32x2, sm_100 and later): one
// instruction updates two floats held in a 64-bit register pair.
__device__ __forceinline__ unsigned long long f2_bits(float2 v) {
  return *reinterpret_cast<unsigned long long *>(&v);
}
__device__ __forceinline__ float2 f2_from(unsigned long long r) {
  return *reinterpret_cast<float2 *>(&r);
}
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)));
  return f2_from(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(f2_bits(a)), "l"(f2_bits(b)), "l"(f2_bits(c)));
  return f2_from(d);
}

// 4-byte asynchronous copy global -> shared (through L1), and its group fences.
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Bulk prefetch of [src, src + bytes) into L2 (16-byte aligned start and size).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
// The same for an arbitrary byte range, widened to 16-byte boundaries.
__device__ __forceinline__ void prefetch_range_l2(const void *begin, const void *end) {
  const uintptr_t b0 = reinterpret_cast<uintptr_t>(begin) & ~uintptr_t(15);
  const uintptr_t b1 = (reinterpret_cast<uintptr_t>(end) + 15) & ~uintptr_t(15);
  if (b1 > b0) bulk_prefetch_l2(reinterpret_cast<const void *>(b0), (unsigned)(b1 - b0));
}

// A 16-byte chunk of a row with the element-wise operations of the step.
template <typename T>
struct Chunk;
template <>
struct Chunk<float> {
  using type = float4;
  static constexpr int W = 4;
  __device__ static __forceinline__ float2 lo(const float4 &v) { return make_float2(v.x, v.y); }
  __device__ static __forceinline__ float2 hi(const float4 &v) { return make_float2(v.z, v.w); }
  __device__ static __forceinline__ float4 join(float2 l, float2 h) { return make_float4(l.x, l.y, h.x, h.y); }
  // acc + v
  __device__ static __forceinline__ float4 add(const float4 &acc, const float4 &v) {
    return join(add2(lo(acc), lo(v)), add2(hi(acc), hi(v)));
  }
  // s * v + acc
  __device__ static __forceinline__ float4 fma(float s, const float4 &v, const float4 &acc) {
    const float2 ss = make_float2(s, s);
    return join(fma2(ss, lo(v), lo(acc)), fma2(ss, hi(v), hi(acc)));
  }
  // s * v + acc - z
  __device__ static __forceinline__ float4 fma_sub(float s, const float4 &v, const float4 &acc,
                                                   const float4 &z) {
    const float2 ss = make_float2(s, s);
    return join(sub2(fma2(ss, lo(v), lo(acc)), lo(z)), sub2(fma2(ss, hi(v), hi(acc)), hi(z)));
  }
  // running dot products: p_aa += a.a, p_ba += b.a (two lanes of partial sums each)
  __device__ static __forceinline__ void dots(const float4 &a, const float4 &b, float2 &paa,
                                              float2 &pba) {
    paa = fma2(lo(a), lo(a), paa);
    paa = fma2(hi(a), hi(a), paa);
    pba = fma2(lo(b), lo(a), pba);
    pba = fma2(hi(b), hi(a), pba);
  }
  __device__ static __forceinline__ float get(const float4 &v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
  }
  __device__ static __forceinline__ void set(float4 &v, int i, float x) {
    if (i == 0) v.x = x; else if (i == 1) v.y = x; else if (i == 2) v.z = x; else v.w = x;
  }
};
template <>
struct Chunk<double> {
  using type = double2;
  static constexpr int W = 2;
  __device__ static __forceinline__ double2 add(const double2 &acc, const double2 &v) {
    return make_double2(acc.x + v.x, acc.y + v.y);
  }
  __device__ static __forceinline__ double2 fma(double s, const double2 &v, const double2 &acc) {
    return make_double2(::fma(s, v.x, acc.x), ::fma(s, v.y, acc.y));
  }
  __device__ static __forceinline__ double2 fma_sub(double s, const double2 &v, const double2 &acc,
                                                    const double2 &z) {
    return make_double2(::fma(s, v.x, acc.x) - z.x, ::fma(s, v.y, acc.y) - z.y);
  }
  __device__ static __forceinline__ void dots(const double2 &a, const double2 &b, double2 &paa,
                                              double2 &pba) {
    paa.x = ::fma(a.x, a.x, paa.x);
    paa.y = ::fma(a.y, a.y, paa.y);
    pba.x = ::fma(b.x, a.x, pba.x);
    pba.y = ::fma(b.y, a.y, pba.y);
  }
  __device__ static __forceinline__ double get(const double2 &v, int i) { return i == 0 ? v.x : v.y; }
  __device__ static __forceinline__ void set(double2 &v, int i, double x) {
    if (i == 0) v.x = x; else v.y = x;
  }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block reduction of NQ values per thread; result valid in thread 0.
// `scratch` holds kWarps * NQ doubles.  All threads of the block must call it.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ], double *scratch) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) scratch[warp * NQ + q] = v[q];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = lane < kWarps ? scratch[lane * NQ + q] : 0.0;
      v[q] = warp_sum(x);
    }
  }
  __syncthreads();
}

// Compensated (Kahan) FP32 accumulator: the FP32 form keeps its running dot
// products in FP32 pairs and hands them to FP64 at the end of a tile.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    float y = x - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

}  // namespace kpm
