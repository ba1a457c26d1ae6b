// Autotuner of the moment loop (the paper has no counterpart): a search over
// the choices that change only the schedule of the Chebyshev step, not its
// arithmetic beyond the order of the sums:
//   - neighbour-list, hi-block or matrix-free kernel (where they apply),
//   - states per tile,
//   - resident blocks per SM of the persistent grid,
//   - FP32 rows of 17..32 chunks as two states per warp or one,
//   - the dimension below which sectors of the FP32 form run in FP64 (only
//     upwards from the default: a larger threshold runs more sectors in FP64,
//     never fewer).
// Each candidate is timed on a short run of the real problem (random
// vectors, the first step and trial_steps further steps, assembly) with CUDA
// events on the caller's stream; the search is one pass of coordinate
// descent from the defaults.  The best choice is kept per problem (model,
// sectors, R, precision) for the life of the process, and calls with
// opts.tuned = 1 use it.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kpm_run.h"

namespace kpm {

namespace {

std::mutex g_tune_mutex;
std::map<std::string, Knobs> g_tuned;

std::string problem_key(const kpm_model *m, int n_sectors, const int32_t *n_up, int R,
                        int precision) {
  std::string k;
  char buf[64];
  snprintf(buf, sizeof(buf), "N%d|B%d|R%d|P%d|", m->n_sites, m->n_bonds, R, precision);
  k += buf;
  for (int b = 0; b < m->n_bonds; ++b) {
    snprintf(buf, sizeof(buf), "%d,%d,%.17g;", m->bi[b], m->bj[b], m->J[b]);
    k += buf;
  }
  k += "|S";
  for (int i = 0; i < n_sectors; ++i) {
    snprintf(buf, sizeof(buf), "%d,", n_up[i]);
    k += buf;
  }
  return k;
}

void describe(const Knobs &kn, bool lists, bool block, char *out, size_t len) {
  snprintf(out, len, "kernel=%s tile_states=%lld blocks_per_sm=%d two_state=%d side_min_dim=%lld",
           block ? "hi-block" : (lists ? "list" : "matrix-free"), (long long)kn.tile_states,
           kn.blocks_per_sm, kn.two_state, (long long)kn.side_min_dim);
}

// Times one candidate: init, 1 + steps matrix-vector products and assembly.
int time_candidate(const kpm_model *m, int n_sectors, const int32_t *n_up, const double *a,
                   const double *b, int R, int precision, int steps, const Knobs &kn,
                   cudaStream_t s, double *ms, bool *uses_lists, Knobs *resolved,
                   bool *uses_block = nullptr) {
  MomentsJob job;
  const int K = 2 * (steps + 1);
  KPM_TRY(prepare_job(m, n_sectors, n_up, K, R, precision, &job, kn));
  Workspace ws;
  const size_t out_bytes = align256((size_t)n_sectors * K * sizeof(double));
  KPM_TRY(ws.acquire(nullptr, 0, job_bytes(job) + out_bytes, s));
  Arena arena{reinterpret_cast<char *>(ws.ptr), ws.size, 0};
  KPM_TRY(setup_job(job, a, b, arena, s));
  double *mu = arena.take<double>((size_t)n_sectors * K);
  KPM_REQUIRE(mu != nullptr, KPM_ENOMEM, "workspace too small");
  cudaEvent_t e0, e1;
  KPM_CUDA(cudaEventCreate(&e0));
  KPM_CUDA(cudaEventCreate(&e1));
  double best = 1e300;
  for (int rep = 0; rep < 2; ++rep) {
    // the counters of the tile queues start at zero for every run
    for (int part = 0; part < 2; ++part) {
      MomentsRun *r = part == 0 ? (job.has_main ? &job.main : nullptr)
                                : (job.has_side ? &job.side : nullptr);
      if (r) KPM_CUDA(cudaMemsetAsync(r->counters, 0, sizeof(int) * 2 * r->S, s));
    }
    KPM_CUDA(cudaEventRecord(e0, s));
    KPM_TRY(run_job(job, 1, 0, mu, nullptr, nullptr, s));
    KPM_CUDA(cudaEventRecord(e1, s));
    KPM_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    KPM_CUDA(cudaEventElapsedTime(&t, e0, e1));
    best = std::min(best, (double)t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = best;
  if (uses_lists) *uses_lists = job.has_main && job.main.list_stride > 0;
  if (uses_block) *uses_block = job.has_main && job.main.block_L > 0;
  if (resolved) {
    *resolved = kn;
    if (job.has_main) resolved->tile_states = job.main.plan.tile_states;
  }
  return KPM_OK;
}

}  // namespace

Knobs knobs_for(const kpm_model *m, int n_sectors, const int32_t *n_up, int K, int R,
                const kpm_opts &o) {
  (void)K;
  if (!o.tuned || m == nullptr || n_up == nullptr || validate_model(m) != KPM_OK) return Knobs();
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tuned.find(problem_key(m, n_sectors, n_up, R, o.precision));
  return it == g_tuned.end() ? Knobs() : it->second;
}

}  // namespace kpm

using namespace kpm;

extern "C" int kpm_autotune(const kpm_model *model, int32_t n_sectors, const int32_t *n_up,
                            const double *a, const double *b, int32_t R, int32_t precision,
                            int32_t trial_steps, double *default_ms, double *best_ms,
                            char *report, size_t report_len, void *stream_ptr) {
  clear_error();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_ptr);
  KPM_REQUIRE(a != nullptr && b != nullptr, KPM_EINVAL, "kpm_autotune needs a and b");
  KPM_REQUIRE(trial_steps >= 1 && trial_steps <= 10000, KPM_EINVAL, "trial_steps = %d",
              trial_steps);
  KPM_TRY(validate_model(model));
  KPM_TRY(validate_sectors(model, n_sectors, n_up));
  Knobs best;
  double t_def = 0.0;
  bool lists = false;
  Knobs resolved;
  KPM_TRY(time_candidate(model, n_sectors, n_up, a, b, R, precision, trial_steps, best, s, &t_def,
                         &lists, &resolved));
  const int64_t ts0 = resolved.tile_states;
  bool uses_block = false;
  {
    MomentsJob probe;
    if (prepare_job(model, n_sectors, n_up, 2, R, precision, &probe) == KPM_OK)
      uses_block = probe.has_main && probe.main.block_L > 0;
  }
  double t_best = t_def;
  std::string log;
  char line[256];
  auto consider = [&](const Knobs &cand) -> int {
    double t = 0.0;
    bool l = false, bk = false;
    int rc = time_candidate(model, n_sectors, n_up, a, b, R, precision, trial_steps, cand, s, &t,
                            &l, nullptr, &bk);
    if (rc == KPM_ENOMEM) return KPM_OK;  // a candidate that does not fit is skipped
    KPM_TRY(rc);
    describe(cand, l, bk, line, sizeof(line));
    log += line;
    snprintf(line, sizeof(line), ": %.4f ms\n", t);
    log += line;
    if (t < t_best) {
      t_best = t;
      best = cand;
    }
    return KPM_OK;
  };
  // 1. kernel
  if (lists) {
    Knobs c = best;
    c.lists = 0;
    KPM_TRY(consider(c));
  }
  if (uses_block) {
    Knobs c = best;
    c.block = 0;
    KPM_TRY(consider(c));
  }
  // 2. states per tile
  {
    const Knobs base = best;
    for (int64_t f : {ts0 / 4, ts0 / 2, ts0 * 2, ts0 * 4}) {
      if (f < 1) continue;
      Knobs c = base;
      c.tile_states = f;
      KPM_TRY(consider(c));
    }
  }
  // 3. resident blocks per SM
  {
    const Knobs base = best;
    for (int bps : {1, 2, 3}) {
      Knobs c = base;
      c.blocks_per_sm = bps;
      KPM_TRY(consider(c));
    }
  }
  // 4. two states per warp (FP32 rows of 17..32 chunks)
  if (precision == KPM_FP32) {
    Knobs c = best;
    c.two_state = 0;
    KPM_TRY(consider(c));
  }
  // 5. FP64 side run of small sectors (only more sectors in FP64, never fewer)
  if (precision == KPM_FP32) {
    const Knobs base = best;
    for (int64_t d : {(int64_t)8192, (int64_t)65536}) {
      Knobs c = base;
      c.side_min_dim = d;
      KPM_TRY(consider(c));
    }
  }
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tuned[problem_key(model, n_sectors, n_up, R, precision)] = best;
  }
  if (default_ms) *default_ms = t_def / (trial_steps + 1);
  if (best_ms) *best_ms = t_best / (trial_steps + 1);
  if (report && report_len > 0) {
    bool l_best = false, b_best = false;
    // the kernel the best choice resolves to
    MomentsJob job;
    if (prepare_job(model, n_sectors, n_up, 2, R, precision, &job, best) == KPM_OK) {
      l_best = job.has_main && job.main.list_stride > 0;
      b_best = job.has_main && job.main.block_L > 0;
    }
    describe(best, l_best, b_best, line, sizeof(line));
    std::string out = std::string("best: ") + line + "\n" + log;
    snprintf(report, report_len, "%s", out.c_str());
  }
  return KPM_OK;
}

// ---------------------------------------------------------------- FP64 rate
// Instrumentation (no counterpart in the paper): the FP64 fused multiply-add
// rate of the device, for the roofline of the FP64 form of the step.  Every
// thread runs 8 independent chains x <- x * c + d (c slightly below 1, so the
// values stay bounded) and writes their sum, which keeps the chains live.
namespace kpm {
__global__ void __launch_bounds__(256) fp64_fma_kernel(double *out, int iters, double c, double d) {
  double x[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = fma(x[k], c, d);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += x[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}
}  // namespace kpm

extern "C" int kpm_fp64_peak(double *tflops, double *ms, void *stream_ptr) {
  clear_error();
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_ptr);
  KPM_REQUIRE(tflops != nullptr, KPM_EINVAL, "tflops is NULL");
  const int blocks = 8 * sm_count(), threads = 256;
  double *out = nullptr;
  KPM_CUDA(cudaMallocAsync(&out, (size_t)blocks * threads * sizeof(double), s));
  struct Release {
    double *p;
    cudaStream_t s;
    ~Release() {
      cudaFreeAsync(p, s);
      cudaStreamSynchronize(s);
    }
  } release{out, s};
  cudaEvent_t e0, e1;
  KPM_CUDA(cudaEventCreate(&e0));
  KPM_CUDA(cudaEventCreate(&e1));
  int iters = 4096;
  float t = 0.f;
  // grow the run until it lasts at least 50 ms
  for (int tries = 0; tries < 12; ++tries) {
    fp64_fma_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.9999999, 1e-7);
    KPM_CUDA(cudaEventRecord(e0, s));
    fp64_fma_kernel<<<blocks, threads, 0, s>>>(out, iters, 0.9999999, 1e-7);
    KPM_CUDA(cudaEventRecord(e1, s));
    KPM_CUDA(cudaEventSynchronize(e1));
    KPM_CUDA(cudaGetLastError());
    KPM_CUDA(cudaEventElapsedTime(&t, e0, e1));
    count_launches(2);
    if (t >= 50.f) break;
    iters *= 2;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * 8.0 * (double)iters * blocks * threads;
  *tflops = flops / (t * 1e-3) / 1e12;
  if (ms) *ms = t;
  return KPM_OK;
}
