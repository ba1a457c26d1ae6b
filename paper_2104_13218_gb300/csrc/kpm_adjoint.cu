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
// per parameter class from the gathers of lambda_{n+1}.
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
  double *gpart;       // [n_tiles][kMaxClasses]
  int *queue;
  int n, S, K, mode;   // mode 0: lambda_S = d_S; 1: general step; 2: gradient of n = 0
  int lz_zero;         // lambda_{n+2} = 0
  int Rp, G_lanes, gpw, n_classes;
  int cstart[kMaxClasses + 1];
  double half_n;
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
  const int nb = bd.n_bonds;
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
        for (int p = 0; p < a.n_classes; ++p) a.gpart[(int64_t)t * kMaxClasses + p] += f * acc[p];
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

// dL/dtheta_p = (1/R) sum over tiles (tile order) of gpart[t][p]; the 1/R is the
// average over the random vectors in mu_n = (1/R) sum_r <r|T_n|r>, left out of
// the per-vector recursion above.
__global__ void adjoint_final_kernel(const double *gpart, int n_tiles, int P, double inv_R,
                                     double *out) {
  const int p = blockIdx.x;
  double v = 0.0;
  for (int t = threadIdx.x; t < n_tiles; t += 32) v += gpart[(int64_t)t * kMaxClasses + p];
  v = warp_sum(v);
  if (threadIdx.x == 0) out[p] = v * inv_R;
}

namespace {

template <int CPL, bool FULL>
void *adj_ptr() {
  return reinterpret_cast<void *>(&adjoint_step_kernel<CPL, FULL>);
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
  int n_classes = 0;
  int k = 32, n_ckpt = 0;
  size_t bytes = 0;
};

int prepare_adjoint(const kpm_model *m, const int32_t *bond_class, int n_classes, int n_sectors,
                    const int32_t *n_up, int K, int R, int ckpt, AdjPlan *ap) {
  KPM_TRY(validate_model(m));
  int P = n_classes;
  if (bond_class == nullptr) P = m->n_bonds;
  KPM_REQUIRE(P >= 1 && P <= kMaxClasses, KPM_EINVAL, "n_classes = %d outside 1..%d", P,
              kMaxClasses);
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
    ap->cstart[p] = (int)ap->bi.size();
    for (int b = 0; b < m->n_bonds; ++b)
      if (cls[b] == p) {
        ap->bi.push_back(m->bi[b]);
        ap->bj.push_back(m->bj[b]);
        ap->J.push_back(m->J[b]);
      }
  }
  for (int p = P; p <= kMaxClasses; ++p) ap->cstart[p] = (int)ap->bi.size();
  ap->sorted.n_sites = m->n_sites;
  ap->sorted.n_bonds = m->n_bonds;
  ap->sorted.bi = ap->bi.data();
  ap->sorted.bj = ap->bj.data();
  ap->sorted.J = ap->J.data();
  KPM_TRY(prepare_run(&ap->sorted, n_sectors, n_up, K, R, KPM_FP64, &ap->run));
  ap->k = ckpt > 0 ? ckpt : 32;
  ap->n_ckpt = (ap->run.S + ap->k - 1) / ap->k;
  const MomentsRun &r = ap->run;
  const size_t SK = (size_t)n_sectors * K;
  ap->bytes = run_bytes(r) + 2 * r.vec_bytes + (size_t)ap->n_ckpt * 2 * r.vec_bytes +
              align256(std::max<size_t>(1, r.plan.tiles.size()) * kMaxClasses * 8) +
              align256((size_t)n_sectors * 3 * 8) + align256((size_t)(r.S + 2) * 4) +
              3 * align256(SK * 8) + align256(kMaxClasses * 8) + 1024;
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

extern "C" int kpm_moments_backward(const kpm_model *model, const int32_t *bond_class,
                                    int32_t n_classes, int32_t n_sectors, const int32_t *n_up,
                                    const double *a, const double *b, int32_t n_moments, int32_t R,
                                    uint64_t seed, uint64_t r0, int32_t precision,
                                    int32_t ckpt_interval, const double *dL_dmu,
                                    const double *dL_dmu_M, const double *dL_dmu_M2,
                                    double *dL_dtheta, int32_t on_device, void *workspace,
                                    size_t ws_bytes, void *stream_ptr) {
  clear_error();
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
  KPM_REQUIRE(precision == KPM_FP64, KPM_EINVAL, "the adjoint runs in FP64 only");
  KPM_REQUIRE(a && b && dL_dmu && dL_dtheta, KPM_EINVAL, "NULL argument");
  AdjPlan ap;
  KPM_TRY(prepare_adjoint(model, bond_class, n_classes, n_sectors, n_up, n_moments, R,
                          ckpt_interval, &ap));
  MomentsRun &run = ap.run;
  Workspace ws;
  KPM_TRY(ws.acquire(workspace, ws_bytes, ap.bytes, stream));
  Arena arena{reinterpret_cast<char *>(ws.ptr), ws.size, 0};
  KPM_TRY(setup_run(run, a, b, arena, stream));
  double2 *LA = arena.take<double2>(run.vec_bytes / 16);
  double2 *LB = arena.take<double2>(run.vec_bytes / 16);
  std::vector<char *> ck(2 * ap.n_ckpt);
  for (auto &p : ck) p = arena.take<char>(run.vec_bytes);
  double *gpart = arena.take<double>(std::max<size_t>(1, run.plan.tiles.size()) * kMaxClasses);
  double *hbar = arena.take<double>((size_t)n_sectors * 3);
  int *queues = arena.take<int>((size_t)run.S + 2);
  const size_t SK = (size_t)n_sectors * n_moments;
  double *dg[3] = {nullptr, nullptr, nullptr};
  double *dtheta = arena.take<double>(kMaxClasses);
  bool ok = LA && LB && gpart && hbar && queues && dtheta;
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
  KPM_CUDA(cudaMemsetAsync(gpart, 0, std::max<size_t>(1, run.plan.tiles.size()) * kMaxClasses * 8, stream));
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
  for (int p = 0; p <= kMaxClasses; ++p) ar.cstart[p] = ap.cstart[p];
  ar.half_n = 0.5 * run.plan.N;
  void *fn = pick_adj(run.lay.cpl, run.plan.any_full);
  int per_sm = 0;
  KPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, 0));
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
    KPM_CUDA(cudaLaunchKernel(fn, dim3(grid), dim3(kThreads), args, 0, stream));
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
                                                        ap.n_classes, 1.0 / R, dtheta);
  KPM_CUDA(cudaGetLastError());
  count_launches(1);
  if (on_device)
    KPM_CUDA(cudaMemcpyAsync(dL_dtheta, dtheta, ap.n_classes * 8, cudaMemcpyDeviceToDevice, stream));
  else
    KPM_CUDA(cudaMemcpyAsync(dL_dtheta, dtheta, ap.n_classes * 8, cudaMemcpyDeviceToHost, stream));
  KPM_CUDA(cudaStreamSynchronize(stream));
  return KPM_OK;
}
