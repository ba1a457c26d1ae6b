// kpm_moments_static: the moment loop with its scratch in a fixed device
// array compiled into the library, for callers that cannot allocate device
// memory themselves.
//
// Such callers are, for example, applications whose framework reserves the
// device memory up front in its own pool (a further cudaMalloc then fails or
// fragments that pool), and latency-critical loops that must not enter the
// CUDA allocator (cudaFree waits for the whole device).  They still pass their
// own input and output buffers; only the scratch (two interleaved vectors,
// the basis tables, the per-tile partial sums and the work-queue counters)
// comes from the array below.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds kStaticScratchBytes for it until the process exits.  Its name
// is only a host-side stand-in in host code, so the device address is looked
// up with cudaGetSymbolAddress while the device is current and then handed to
// the kernels.  The lookup is made once per device and CUDA context: the first
// call on a device does it, and so does the first call after the context was
// replaced (cudaDeviceReset destroys the primary context, and the array's
// address in the new one need not be the old one).  The context is identified
// by its unique id (cuCtxGetId, reached through the runtime's driver entry
// points, so no driver library is linked).  All calls share the array: the
// counters and flags that must start at zero are cleared at the start of every
// call, and two calls whose work overlaps on the GPU (for instance on two
// streams) race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "kpm_run.h"

namespace kpm {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;  // 64 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
void *g_static_ptr[kMaxDevices] = {};
unsigned long long g_static_ctx[kMaxDevices] = {};

using CtxGetCurrentFn = int (*)(void **);
using CtxGetIdFn = int (*)(void *, unsigned long long *);

// Unique id of the calling thread's current CUDA context (0 if there is none
// or the driver cannot tell).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool looked_up = false;
  if (!looked_up) {
    looked_up = true;
    void *f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  }
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (get_current == nullptr || get_id == nullptr || get_current(&ctx) != 0 || ctx == nullptr ||
      get_id(ctx, &id) != 0)
    return 0;
  return id;
}

// Device address of the scratch array in the current device's context, looked
// up on the first call in each device context.
int static_scratch(void **out) {
  int dev = 0;
  KPM_CUDA(cudaGetDevice(&dev));
  KPM_REQUIRE(dev >= 0 && dev < kMaxDevices, KPM_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_static_mutex);
  unsigned long long ctx = current_context_id();
  if (g_static_ptr[dev] == nullptr || ctx == 0 || ctx != g_static_ctx[dev]) {
    void *p = nullptr;
    KPM_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_ptr[dev] = p;
    // the lookup creates the context if there was none yet
    g_static_ctx[dev] = ctx != 0 ? ctx : current_context_id();
  }
  *out = g_static_ptr[dev];
  return KPM_OK;
}

}  // namespace

}  // namespace kpm

using namespace kpm;

extern "C" size_t kpm_static_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" int kpm_moments_static(const kpm_model *model, int32_t n_sectors, const int32_t *n_up,
                                  const double *a, const double *b, int32_t n_moments, int32_t R,
                                  uint64_t seed, uint64_t r0, int32_t precision, double *mu,
                                  double *mu_M, double *mu_M2, void *stream_ptr) {
  clear_error();
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_ptr);
  KPM_REQUIRE(mu != nullptr, KPM_EINVAL, "mu is NULL");
  KPM_REQUIRE(a != nullptr && b != nullptr, KPM_EINVAL,
              "kpm_moments_static needs the rescaling a and b (it runs no bound estimate)");
  MomentsJob job;
  KPM_TRY(prepare_job(model, n_sectors, n_up, n_moments, R, precision, &job));
  const size_t need = job_bytes(job);
  KPM_REQUIRE(need <= kStaticScratchBytes, KPM_ENOMEM,
              "kpm_moments_static: this problem needs %zu bytes of scratch, the static array "
              "holds %zu; use kpm_moments with a workspace instead",
              need, kStaticScratchBytes);
  void *scratch = nullptr;
  KPM_TRY(static_scratch(&scratch));
  Arena arena{reinterpret_cast<char *>(scratch), kStaticScratchBytes, 0};
  KPM_TRY(setup_job(job, a, b, arena, stream));
  KPM_TRY(run_job(job, seed, r0, mu, mu_M, mu_M2, stream));
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
