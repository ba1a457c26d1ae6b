// Spectral bounds of every sector for the rescaling of Eq. E-2-3 / E-2-4,
// from the Lanczos method the paper uses for extremal energies (Sec. 3.1.2).
//
// All sectors run together: one Lanczos sequence per sector, its vectors
// stored as 2-value rows (16 bytes per state, the second value unused) in the
// same stacked layout as the moment loop.  Each iteration is two kernels:
//   q_j = x_j / |x_j|,  w = H q_j - beta_j q_{j-1}  (written over q_{j-1}),
//   alpha_j = <w, q_j>;
//   x_{j+1} = w - alpha_j q_j,  beta_{j+1} = |x_{j+1}|,
// with per-tile partial sums reduced in tile order by the last block of each
// kernel.  With grouped couplings (and lists of at most 2 GiB) the product
// reads per-state neighbour lists built once; otherwise it ranks the flipped
// states on the fly.  The host then finds the extreme eigenvalues of each tridiagonal
// matrix by Sturm-sequence bisection and widens them by the residual bound
// |beta_{m+1} y_m| of the Ritz pair (y the Ritz vector of the tridiagonal
// matrix), which brackets an eigenvalue of H.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kpm_device.cuh"
#include "kpm_run.h"

namespace kpm {

constexpr int kMaxLanczos = 1000;
// Lanczos sequences per sector: one, from a start vector with components
// uniform in (-1, 1) (such a vector is orthogonal to no eigenvector with
// probability one).  Rows keep two values so that they are 16 bytes wide.
constexpr int kLanczosColumns = 1;
// Neighbour rows loaded together by the Lanczos product.
constexpr int kLanczosBatch = 8;

struct LanczosArgs {
  double2 *X;        // x_j = beta_j q_j, unnormalised (mode 1: read; mode 2: x_{j+1} written)
  double2 *P;        // mode 1: q_{j-1} in, w out; mode 2: w in
  double2 *Q;        // mode 1: q_j out; mode 2: q_j in
  TablesDev tb;
  const uint32_t *lists;  // entry-major neighbour lists (row indices), or null: ranks on the fly
  uint64_t list_estride;  // word offset between a state's entries
  double *partials;  // [n_tiles][2]
  const double *nrm; // |x_j| per [sector][2] (mode 1)
  const double *sub; // coefficient of q_{j-1} per [sector][2] (mode 1; 0 for j = 0)
  const double *alp; // alpha_j per [sector][2] (mode 2)
  double *out;       // mode 0: |x_0|; mode 1: alpha_j; mode 2: beta_{j+1}
  int *queue, *done;
  int mode;          // 0 = |x_0|, 1 = matrix-vector product, 2 = orthogonalise
  double breakdown;  // beta below this ends a sequence
};

// One Lanczos half-iteration over all sectors, one state per thread:
//   mode 1: q_j = x_j / |x_j| (written), w = H q_j - beta_j q_{j-1} (written over
//           q_{j-1}), alpha_j = <w, q_j>;
//   mode 2: x_{j+1} = w - alpha_j q_j (written), beta_{j+1} = |x_{j+1}|;
//   mode 0: |x_0|.
// The normalisation of x_j is folded into the next product, so that an
// iteration takes two passes.  Per-tile partial sums are reduced in tile order
// by the last block.
__global__ void __launch_bounds__(kThreads)
    lanczos_kernel(const __grid_constant__ LanczosArgs a, const __grid_constant__ BondsDev bd) {
  __shared__ double s_red[kWarps * 2];
  __shared__ int s_tile, s_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(a.queue, 1);
    __syncthreads();
    const int t = s_tile;
    if (t >= a.tb.n_tiles) break;
    const Tile tile = a.tb.tiles[t];
    const SectorDev sd = a.tb.sectors[tile.sector];
    double acc[2] = {0.0, 0.0};
    uint32_t hb = tile.b_first;
    if (a.mode == 1) {
      const double n = a.nrm[tile.sector * 2];
      const double sc = n > 0.0 ? 1.0 / n : 0.0;
      const double c = a.sub[tile.sector * 2];
      for (uint32_t u = threadIdx.x; u < tile.count; u += kThreads) {
        const int64_t row = tile.row0 + u;
        double d = bd.J_quarter_sum;
        double h0 = 0.0;
        if (a.lists != nullptr) {
          const uint32_t *L = a.lists + row;
          const uint64_t es = a.list_estride;
          const uint32_t hdr = __ldg(L);
          int e = 1;
          for (int g = 0; g < bd.n_groups; ++g) {
            const int cnt = (int)((hdr >> (8 * g)) & 255u);
            double gs = 0.0;
            // batches of independent loads: the indices, then the rows
            for (int k = 0; k < cnt; k += kLanczosBatch) {
              uint32_t nb[kLanczosBatch];
#pragma unroll
              for (int q = 0; q < kLanczosBatch; ++q)
                nb[q] = k + q < cnt ? __ldg(L + (uint64_t)(e + k + q) * es) : 0u;
              double v[kLanczosBatch];
#pragma unroll
              for (int q = 0; q < kLanczosBatch; ++q) v[q] = k + q < cnt ? __ldg(&a.X[nb[q]].x) : 0.0;
#pragma unroll
              for (int q = 0; q < kLanczosBatch; ++q) gs += v[q];
            }
            e += cnt;
            d -= cnt * (0.5 * bd.gJ[g]);
            h0 = fma(0.5 * bd.gJ[g], gs, h0);
          }
        } else {
          uint64_t s;
          if (sd.n_up < 0)
            s = (uint64_t)(row - sd.row0);
          else
            s = sector_unrank(tile.rank0 + u, sd.n_up, tile.b_last, hb, a.tb);
          for (int b0 = 0; b0 < bd.n_bonds; b0 += kLanczosBatch) {
            int64_t nr[kLanczosBatch];
#pragma unroll
            for (int q = 0; q < kLanczosBatch; ++q) {
              nr[q] = -1;
              const int b = b0 + q;
              if (b < bd.n_bonds) {
                const uint64_t m = bd.mask[b];
                const uint64_t tt = s & m;
                if (tt != 0 && tt != m) {
                  d -= 0.5 * bd.J[b];
                  const uint64_t f = s ^ m;
                  nr[q] = sd.row0 + (sd.n_up < 0 ? (int64_t)f : (int64_t)sector_rank(f, a.tb));
                }
              }
            }
            double v[kLanczosBatch];
#pragma unroll
            for (int q = 0; q < kLanczosBatch; ++q) v[q] = nr[q] >= 0 ? __ldg(&a.X[nr[q]].x) : 0.0;
#pragma unroll
            for (int q = 0; q < kLanczosBatch; ++q)
              if (nr[q] >= 0) h0 = fma(0.5 * bd.J[b0 + q], v[q], h0);
          }
        }
        const double q = a.X[row].x * sc;
        const double w = fma(d, q, h0 * sc) - c * a.P[row].x;
        a.Q[row].x = q;
        a.P[row].x = w;
        acc[0] = fma(w, q, acc[0]);
      }
    } else if (a.mode == 2) {
      const double al = a.alp[tile.sector * 2];
      for (uint32_t u = threadIdx.x; u < tile.count; u += kThreads) {
        const int64_t row = tile.row0 + u;
        const double w = a.P[row].x - al * a.Q[row].x;
        a.X[row].x = w;
        acc[0] = fma(w, w, acc[0]);
      }
    } else {
      for (uint32_t u = threadIdx.x; u < tile.count; u += kThreads) {
        const double x = a.X[tile.row0 + u].x;
        acc[0] = fma(x, x, acc[0]);
      }
    }
    block_sum<2>(acc, s_red);
    if (threadIdx.x == 0) {
      a.partials[(int64_t)t * 2] = acc[0];
      a.partials[(int64_t)t * 2 + 1] = acc[1];
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(a.done, 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  for (int sec = warp; sec < a.tb.n_sectors; sec += kWarps) {
    double v0 = 0.0, v1 = 0.0;
    for (int t = a.tb.tile_begin[sec] + lane; t < a.tb.tile_end[sec]; t += 32) {
      v0 += __ldcg(a.partials + (int64_t)t * 2);
      v1 += __ldcg(a.partials + (int64_t)t * 2 + 1);
    }
    v0 = warp_sum(v0);
    v1 = warp_sum(v1);
    if (lane == 0) {
      if (a.mode == 1) {
        a.out[sec * 2] = v0;
        a.out[sec * 2 + 1] = v1;
      } else {
        const double b0 = sqrt(v0), b1 = sqrt(v1);
        a.out[sec * 2] = b0 > a.breakdown ? b0 : 0.0;
        a.out[sec * 2 + 1] = b1 > a.breakdown ? b1 : 0.0;
      }
    }
  }
}

// Number of eigenvalues of the m x m tridiagonal (alpha, beta) below x.
int sturm_count(const std::vector<double> &al, const std::vector<double> &be, int m, double x) {
  int count = 0;
  double d = 1.0;
  for (int i = 0; i < m; ++i) {
    const double b2 = i > 0 ? be[i] * be[i] : 0.0;
    d = al[i] - x - (i > 0 ? b2 / d : 0.0);
    if (d == 0.0) d = -1e-300;
    if (d < 0.0) ++count;
  }
  return count;
}

// k-th smallest eigenvalue (0-based) by bisection.
double tridiag_eig(const std::vector<double> &al, const std::vector<double> &be, int m, int k) {
  double lo = al[0], hi = al[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(be[i]) : 0.0) + (i + 1 < m ? std::fabs(be[i + 1]) : 0.0);
    lo = std::min(lo, al[i] - r);
    hi = std::max(hi, al[i] + r);
  }
  const double scale = std::max({1.0, std::fabs(lo), std::fabs(hi)});
  for (int it = 0; it < 200 && hi - lo > 4e-16 * scale; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_count(al, be, m, mid) > k)
      hi = mid;
    else
      lo = mid;
  }
  return 0.5 * (lo + hi);
}

// |last component| of the unit eigenvector of T for eigenvalue theta, by
// three steps of inverse iteration, each a tridiagonal solve of
// (T - sigma) z = y by forward elimination and back substitution.
double ritz_last_component(const std::vector<double> &al, const std::vector<double> &be, int m,
                           double theta) {
  if (m == 1) return 1.0;
  const double sigma = theta + 1e-13 * std::max(1.0, std::fabs(theta));
  std::vector<double> y(m, 1.0), cp(m, 0.0), dp(m, 0.0);
  for (int it = 0; it < 3; ++it) {
    for (int i = 0; i < m; ++i) {
      double denom = al[i] - sigma - (i > 0 ? be[i] * cp[i - 1] : 0.0);
      if (std::fabs(denom) < 1e-300) denom = 1e-300;
      cp[i] = (i + 1 < m) ? be[i + 1] / denom : 0.0;
      dp[i] = (y[i] - (i > 0 ? be[i] * dp[i - 1] : 0.0)) / denom;
    }
    y[m - 1] = dp[m - 1];
    for (int i = m - 2; i >= 0; --i) y[i] = dp[i] - cp[i] * y[i + 1];
    double nrm = 0.0;
    for (int i = 0; i < m; ++i) nrm += y[i] * y[i];
    nrm = std::sqrt(nrm);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) return 1.0;
    for (int i = 0; i < m; ++i) y[i] /= nrm;
  }
  return std::fabs(y[m - 1]);
}

namespace {

int sm_count_b() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return std::max(n, 1);
}

struct BoundsLayout {
  MomentsRun run;    // plan with R = 2 FP64 rows
  int list_stride = 0;  // > 0: the product reads neighbour lists of this many entries
  uint64_t list_estride = 0;  // entry-major lists: word offset between entries
  size_t list_bytes = 0;
  size_t bytes = 0;
};

// Neighbour lists of the Lanczos product (grouped couplings; at most this many
// bytes, beyond which the ranks are computed on the fly).
constexpr size_t kBoundsListMaxBytes = (size_t)2 << 30;

int prepare_bounds(const kpm_model *m, int n_sectors, const int32_t *n_up, BoundsLayout *bl) {
  KPM_TRY(prepare_run(m, n_sectors, n_up, 2, 2, KPM_FP64, &bl->run));
  const MomentsRun &r = bl->run;
  bl->list_stride = 0;
  bl->list_estride = 0;
  bl->list_bytes = 0;
  if (r.bonds.n_groups > 0 && m->n_bonds <= 255 && r.plan.total_rows < ((int64_t)1 << 32)) {
    const uint64_t es = (uint64_t)(r.plan.total_rows + 63) / 64 * 64;
    const size_t lb = align256((size_t)es * (1 + m->n_bonds) * sizeof(uint32_t));
    if (lb <= kBoundsListMaxBytes) {
      bl->list_stride = 1 + m->n_bonds;
      bl->list_estride = es;
      bl->list_bytes = lb;
    }
  }
  bl->bytes = 3 * r.vec_bytes + bl->list_bytes + tables_bytes(r.plan) +
              align256(std::max<size_t>(1, r.plan.tiles.size()) * 2 * sizeof(double)) +
              2 * align256((size_t)(kMaxLanczos + 1) * n_sectors * 2 * sizeof(double)) +
              align256((size_t)4 * (kMaxLanczos + 2) * sizeof(int)) +
              align256((size_t)n_sectors * 2 * sizeof(double)) + 1024;
  return KPM_OK;
}

}  // namespace

}  // namespace kpm

using namespace kpm;

extern "C" size_t kpm_bounds_workspace_size(const kpm_model *model, int32_t n_sectors,
                                            const int32_t *n_up) {
  BoundsLayout bl;
  if (prepare_bounds(model, n_sectors, n_up, &bl) != KPM_OK) return 0;
  return bl.bytes;
}

extern "C" int kpm_bounds(const kpm_model *model, int32_t n_sectors, const int32_t *n_up,
                          double eps, int32_t max_iter, double tol, uint64_t seed, double *a_out,
                          double *b_out, double *e_min, double *e_max, void *workspace,
                          size_t ws_bytes, void *stream_ptr) {
  clear_error();
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
  KPM_REQUIRE(a_out && b_out, KPM_EINVAL, "a and b outputs are required");
  KPM_REQUIRE(max_iter >= 1 && max_iter <= kMaxLanczos, KPM_EINVAL, "max_iter = %d outside 1..%d",
              max_iter, kMaxLanczos);
  KPM_REQUIRE(eps >= 0.0 && eps < 2.0, KPM_EINVAL, "eps = %g outside [0, 2)", eps);
  BoundsLayout bl;
  KPM_TRY(prepare_bounds(model, n_sectors, n_up, &bl));
  MomentsRun &r = bl.run;
  Workspace ws;
  KPM_TRY(ws.acquire(workspace, ws_bytes, bl.bytes, stream));
  Arena arena{reinterpret_cast<char *>(ws.ptr), ws.size, 0};
  double2 *X = arena.take<double2>(r.vec_bytes / sizeof(double2));
  double2 *P = arena.take<double2>(r.vec_bytes / sizeof(double2));
  double2 *Q = arena.take<double2>(r.vec_bytes / sizeof(double2));
  uint32_t *lists = bl.list_stride > 0 ? arena.take<uint32_t>(bl.list_bytes / sizeof(uint32_t)) : nullptr;
  double *partials = arena.take<double>(std::max<size_t>(1, r.plan.tiles.size()) * 2);
  const size_t nab = (size_t)(kMaxLanczos + 1) * n_sectors * 2;
  double *alpha = arena.take<double>(nab);
  double *beta = arena.take<double>(nab);
  int *counters = arena.take<int>((size_t)4 * (kMaxLanczos + 2));
  double *norm0 = arena.take<double>((size_t)n_sectors * 2);
  KPM_REQUIRE(X && P && Q && partials && alpha && beta && counters && norm0 &&
                  (bl.list_stride == 0 || lists), KPM_ENOMEM,
              "workspace too small for kpm_bounds");
  std::vector<SectorDev> sec(n_sectors);
  for (int i = 0; i < n_sectors; ++i) {
    sec[i].row0 = r.plan.row0[i];
    sec[i].dim = r.plan.dim[i];
    sec[i].n_up = r.plan.n_up[i];
    sec[i].hb_begin = r.plan.hb_begin[i];
    sec[i].inv_a = 1.0;
    sec[i].b = 0.0;
    sec[i].Mval = 0.0;
  }
  KPM_TRY(upload_tables(r.plan, sec, arena, stream, &r.tb));
  KPM_CUDA(cudaMemsetAsync(counters, 0, sizeof(int) * 4 * (kMaxLanczos + 2), stream));
  KPM_CUDA(cudaMemsetAsync(beta, 0, sizeof(double) * nab, stream));
  KPM_CUDA(cudaMemsetAsync(alpha, 0, sizeof(double) * nab, stream));
  // x_0: uniform random values (a vector of +-1 signs can be exactly orthogonal
  // to an eigenvector in a small sector); q_{-1} = 0
  KPM_TRY(launch_init(r, X, seed, 0, stream, true));
  KPM_CUDA(cudaMemsetAsync(P, 0, r.vec_bytes, stream));
  if (lists)
    KPM_TRY(launch_build_lists(r.tb, r.bonds, (int64_t)r.plan.tiles.size(), lists, bl.list_stride,
                               1, 1, 0, stream, bl.list_estride));

  double jabs = 0.0;
  for (int b = 0; b < model->n_bonds; ++b) jabs += std::fabs(model->J[b]);
  int per_sm = 0;
  KPM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lanczos_kernel, kThreads, 0));
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)std::max(per_sm, 1) * sm_count_b(), (int64_t)r.plan.tiles.size()));
  LanczosArgs la{};
  la.tb = r.tb;
  la.lists = lists;
  la.list_estride = bl.list_estride;
  la.partials = partials;
  la.breakdown = 0.0;
  auto launch = [&](int mode, int *queue) -> int {
    la.mode = mode;
    la.queue = queue;
    la.done = queue + 1;
    void *args[] = {(void *)&la, (void *)&r.bonds};
    KPM_CUDA(cudaLaunchKernel((void *)lanczos_kernel, dim3(grid), dim3(kThreads), args, 0, stream));
    count_launches(1);
    return KPM_OK;
  };
  // |x_0|
  la.X = X;
  la.out = norm0;
  KPM_TRY(launch(0, counters + 4 * (kMaxLanczos + 1)));
  la.breakdown = 1e-12 * std::max(1.0, jabs);
  // Iterations run in chunks; after each chunk the host reads alpha and beta
  // and stops once every sector's extreme Ritz values meet tol.  beta_0 = 0
  // (the memset above): the first product subtracts nothing.  The next chunk
  // is queued before the host checks the last one, so that the check overlaps
  // it; a chunk queued after convergence only writes alpha, beta entries that
  // are not read, and the result is the same as without the overlap.
  constexpr int kChunk = 16;
  std::vector<double> h_alpha(nab), h_beta(nab);
  std::vector<double> lo_s(n_sectors), hi_s(n_sectors), worst_s(n_sectors);
  int queued = 0;  // iterations queued on the stream
  auto enqueue_chunk = [&]() -> int {
    const int end = std::min(queued + kChunk, (int)max_iter);
    for (int j = queued; j < end; ++j) {
      // mode 1: q_j = x_j / |x_j| into Q, w = H q_j - beta_j q_{j-1} over P, alpha_j
      la.X = X;
      la.P = P;
      la.Q = Q;
      la.nrm = j == 0 ? norm0 : beta + (size_t)j * n_sectors * 2;
      la.sub = beta + (size_t)j * n_sectors * 2;
      la.out = alpha + (size_t)j * n_sectors * 2;
      KPM_TRY(launch(1, counters + 4 * j));
      // mode 2: x_{j+1} = w - alpha_j q_j into X, beta_{j+1} = |x_{j+1}|
      la.alp = alpha + (size_t)j * n_sectors * 2;
      la.out = beta + (size_t)(j + 1) * n_sectors * 2;
      KPM_TRY(launch(2, counters + 4 * j + 2));
      std::swap(P, Q);  // P = q_j (the next q_{j-1}); Q is free for q_{j+1}
    }
    queued = end;
    return KPM_OK;
  };
  cudaEvent_t copied;
  KPM_CUDA(cudaEventCreateWithFlags(&copied, cudaEventDisableTiming));
  struct EventGuard {
    cudaEvent_t e;
    ~EventGuard() { cudaEventDestroy(e); }
  } copied_guard{copied};
  KPM_TRY(enqueue_chunk());
  int done_iters = 0;
  for (;;) {
    done_iters = queued;
    const size_t used = (size_t)(done_iters + 1) * n_sectors * 2;
    KPM_CUDA(cudaMemcpyAsync(h_alpha.data(), alpha, sizeof(double) * used, cudaMemcpyDeviceToHost, stream));
    KPM_CUDA(cudaMemcpyAsync(h_beta.data(), beta, sizeof(double) * used, cudaMemcpyDeviceToHost, stream));
    KPM_CUDA(cudaEventRecord(copied, stream));
    if (queued < max_iter) KPM_TRY(enqueue_chunk());
    KPM_CUDA(cudaEventSynchronize(copied));
    double worst_all = 0.0;
    for (int s = 0; s < n_sectors; ++s) {
      double lo = INFINITY, hi = -INFINITY, worst = 0.0;
      for (int col = 0; col < kLanczosColumns; ++col) {
        std::vector<double> al, be;
        be.push_back(0.0);
        int m = 0;
        for (int j = 0; j < done_iters; ++j) {
          al.push_back(h_alpha[((size_t)j * n_sectors + s) * 2 + col]);
          ++m;
          const double bnext = h_beta[((size_t)(j + 1) * n_sectors + s) * 2 + col];
          if (bnext == 0.0 || m >= r.plan.dim[s]) {
            be.push_back(0.0);
            break;
          }
          be.push_back(bnext);
        }
        // be[i] couples i-1 and i (i >= 1); be[m] is the residual coupling
        const double bres = be.size() > (size_t)m ? std::fabs(be[m]) : 0.0;
        const double tmin = tridiag_eig(al, be, m, 0);
        const double tmax = tridiag_eig(al, be, m, m - 1);
        const double rmin = bres * ritz_last_component(al, be, m, tmin);
        const double rmax = bres * ritz_last_component(al, be, m, tmax);
        lo = std::min(lo, tmin - rmin);
        hi = std::max(hi, tmax + rmax);
        worst = std::max({worst, rmin / std::max(1.0, std::fabs(tmin)),
                          rmax / std::max(1.0, std::fabs(tmax))});
      }
      lo_s[s] = lo;
      hi_s[s] = hi;
      worst_s[s] = worst;
      worst_all = std::max(worst_all, worst);
    }
    if (worst_all <= tol || done_iters >= max_iter) break;
  }
  // the call returns with its stream idle (a chunk queued after convergence)
  KPM_CUDA(cudaStreamSynchronize(stream));

  int status = KPM_OK;
  for (int s = 0; s < n_sectors; ++s) {
    if (worst_s[s] > tol) status = KPM_ENOTCONV;
    double m_ = (hi_s[s] - lo_s[s]) / (2.0 - eps);
    const double c_ = 0.5 * (hi_s[s] + lo_s[s]);
    m_ = std::max(m_, 1e-12 * std::max(1.0, std::fabs(c_)));
    a_out[s] = m_;
    b_out[s] = c_;
    if (e_min) e_min[s] = lo_s[s];
    if (e_max) e_max[s] = hi_s[s];
  }
  if (status == KPM_ENOTCONV)
    set_error("Lanczos residual bound above tol after %d iterations", done_iters);
  return status;
}
