/*
 * kpm.h -- C ABI of the GB300 Chebyshev typicality library (libkpm.so).
 *
 * The library computes, on one NVIDIA GB300 (sm_103a), the stochastic
 * Chebyshev moments of a spin-1/2 Heisenberg Hamiltonian
 *
 *     H = sum_b J_b S_{i_b} . S_{j_b}                         (Sec. 3.1, Eq. E-3-1-1)
 *
 * rescaled as H' = (H - b) / a (the paper's c and m, Eq. E-2-3 and E-2-4), the
 * moments mu_n = (1/R) sum_r <r| T_n(H') |r> with unit-norm random vectors
 * (Eq. E-2-6 and E-2-7), and from them the thermodynamics Z, E, C and chi
 * by the Jackson kernel (Eq. E-2-8) and Gauss-Chebyshev quadrature (Eq. quad
 * and the sector sum that follows it), together with the derivatives with
 * respect to the couplings.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Basis: site i is bit i of the S^z bitstring s (bit set = spin up).  A
 *   sector is selected by its number of up spins n_up = N/2 + M; its states
 *   are ordered by their value as integers and indexed by that rank
 *   (0 .. C(N, n_up) - 1).  n_up = -1 selects the whole 2^N space, indexed
 *   by s itself.  N <= 34 (every sector rank then fits in 32 bits).
 * - Random vectors: component s of vector r is +-1/sqrt(D), the sign being
 *   the top bit of splitmix64(splitmix64(splitmix64(seed) ^ r) ^ s) (clear ->
 *   +1), where splitmix64(x) is the published splitmix64 output for state x.
 *   r runs over r0 .. r0+R-1, so disjoint r0 ranges give independent vectors.
 * - Moments of a run with K moments are stored as mu[sector * K + n],
 *   n = 0 .. K-1.  mu_M and mu_M2 hold the same traces weighted by the
 *   magnetisation M(s) = popcount(s) - N/2 and by M(s)^2 (for a sector these
 *   are M mu and M^2 mu; for the full space they are measured).  K must be
 *   even: the run performs K/2 matrix-vector products and obtains two
 *   moments from each (mu_{2n} = 2<v_n|v_n> - mu_0, mu_{2n+1} =
 *   2<v_{n+1}|v_n> - mu_1).
 * - Pointers: the model arrays, n_up, a and b are HOST memory.  The moment,
 *   thermodynamic and gradient arrays are host memory when the call's
 *   `on_device` argument is 0 and device memory of the current device when
 *   it is 1.  The caller owns every buffer.
 * - Workspace: calls that need device scratch take (workspace, ws_bytes).
 *   With workspace == NULL the library allocates the scratch itself with
 *   cudaMallocAsync on `stream` and frees it before returning; otherwise the
 *   region must be device memory of at least the size the matching
 *   *_workspace_size query returns, aligned to 256 bytes.
 * - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *   Every call enqueues its work on that stream, then waits for it, and
 *   returns a status; results are complete when the call returns.
 * - Status: 0 (KPM_OK) or one of the KPM_E* codes below; the call never
 *   aborts the process.  kpm_last_error() returns a message for the last
 *   failure on the calling thread.
 */
#ifndef KPM_H
#define KPM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KPM_VERSION 1

/* status codes */
#define KPM_OK 0
#define KPM_EINVAL 1    /* invalid argument (sizes, pointers, K odd, N > 34, ...) */
#define KPM_ENOMEM 2    /* device memory or workspace too small */
#define KPM_ECUDA 3     /* a CUDA runtime call failed (message in kpm_last_error) */
#define KPM_ENOTCONV 5  /* Lanczos bound estimate did not reach the requested tolerance */
#define KPM_EBOUNDS 6   /* |mu_n| > 1 + 1e-6: the spectrum of H' left [-1, 1]; results are written */

/* vector storage precision of the moment loop */
#define KPM_FP64 0      /* vectors and arithmetic in FP64 */
#define KPM_FP32 1      /* vectors and arithmetic in FP32, dot products reduced in FP64;
                           sectors below 1024 states are stored in FP64 (in such tiny
                           sectors FP32 rounding stays coherent and grows with the order) */

/* damping kernel g_n (Eq. E-2-8) */
#define KPM_KERNEL_NONE 0     /* g_n = 1 */
#define KPM_KERNEL_JACKSON 1  /* Jackson kernel with N_deg = K */

/* Heisenberg model H = sum_b J[b] S_{bi[b]} . S_{bj[b]}; all arrays host memory. */
typedef struct {
  int32_t n_sites;        /* N, 1 .. 34 */
  int32_t n_bonds;        /* 0 .. 256 */
  const int32_t *bi;      /* [n_bonds] first site of each bond, 0 .. N-1 */
  const int32_t *bj;      /* [n_bonds] second site, != bi[b] */
  const double *J;        /* [n_bonds] coupling J_b */
} kpm_model;

/* Library version (KPM_VERSION). */
int kpm_version(void);

/* Message of the last failing call on this thread ("" if none). */
const char *kpm_last_error(void);

/* Dimension of a sector: C(n_sites, n_up), or 2^n_sites for n_up = -1; -1 if invalid. */
int64_t kpm_sector_dim(int32_t n_sites, int32_t n_up);

/*
 * kpm_bounds -- spectral bounds and rescaling of each sector.
 *
 * The paper rescales H into [-1 + eps/2, 1 - eps/2] with
 * a = (Emax - Emin)/(2 - eps) and b = (Emax + Emin)/2 (Eq. E-2-3, E-2-4)
 * and obtains extremal energies with the Lanczos method (Sec. 3.1.2).  This
 * call runs up to max_iter Lanczos steps in FP64 on the GPU for every sector
 * at once (one start vector per sector with components uniform in (-1, 1)
 * from `seed`), in chunks of 16 steps, stopping after the first
 * chunk at which every extreme Ritz value's residual bound is within tol
 * (relative to max(1, |E|)); it widens the extreme Ritz values by their
 * residual bounds and returns per sector (host arrays of n_sectors entries):
 *   e_min, e_max  -- the widened extremal eigenvalue estimates (may be NULL);
 *   a, b          -- the rescaling of Eq. E-2-4 from them.  A sector whose
 *                    spectrum is one point gets a = 1e-12 * max(1, |b|).
 * Returns KPM_ENOTCONV (outputs still written) when some sector's residual
 * bound exceeds tol * max(1, |E|).  Workspace: kpm_bounds_workspace_size.
 */
int kpm_bounds(const kpm_model *model, int32_t n_sectors, const int32_t *n_up, double eps,
               int32_t max_iter, double tol, uint64_t seed, double *a, double *b,
               double *e_min, double *e_max, void *workspace, size_t ws_bytes, void *stream);

size_t kpm_bounds_workspace_size(const kpm_model *model, int32_t n_sectors, const int32_t *n_up);

/*
 * kpm_moments -- stochastic Chebyshev moments of every sector in one pass.
 *
 * Computes mu_n = (1/R) sum_r <r|T_n(H')|r>, n = 0..K-1 (Eq. E-2-6, E-2-7,
 * normalised so that mu_0 = 1), for all sectors in the same kernel launches,
 * with R random vectors per sector interleaved per basis state.
 *   a, b          -- host [n_sectors] rescaling of each sector (H' = (H - b)/a);
 *                    if either is NULL, kpm_bounds is run first with eps,
 *                    100 Lanczos steps and tol 1e-8.
 *   n_moments     -- K, even, >= 2.
 *   R             -- random vectors per sector, 1 .. 512.
 *   seed, r0      -- random-vector stream (see the conventions above).
 *   precision     -- KPM_FP64 or KPM_FP32.
 *   mu            -- [n_sectors][K] output (required).
 *   mu_M, mu_M2   -- [n_sectors][K] magnetisation-weighted outputs (may be NULL).
 *   on_device     -- 1 if mu, mu_M, mu_M2 are device pointers.
 * Returns KPM_EBOUNDS (moments still written) when some |mu_n| > 1 + 1e-6.
 * Workspace: kpm_moments_workspace_size.
 * Streams: with KPM_FP32, sectors of fewer than 1024 states are computed in
 * FP64 (FP32 rounding would stay coherent there); when such sectors come
 * with larger ones, their launches go to an internal non-blocking,
 * lowest-priority stream of the current device (created on the first such
 * call and kept until exit), forked from `stream` and joined back into it
 * with events.  Like every call here, kpm_moments synchronises `stream`
 * before it returns, so all of its work has finished by then.
 */
int kpm_moments(const kpm_model *model, int32_t n_sectors, const int32_t *n_up,
                const double *a, const double *b, double eps, int32_t n_moments, int32_t R,
                uint64_t seed, uint64_t r0, int32_t precision, double *mu, double *mu_M,
                double *mu_M2, int32_t on_device, void *workspace, size_t ws_bytes,
                void *stream);

size_t kpm_moments_workspace_size(const kpm_model *model, int32_t n_sectors,
                                  const int32_t *n_up, int32_t n_moments, int32_t R,
                                  int32_t precision);

/*
 * kpm_thermo -- Z, E, C and chi on a temperature grid from the moments.
 *
 * For sector G with dimension dim[G], rescaling (a[G], b[G]) and moments
 * mu^G (mu_0 = 1):
 *   gamma_k = g_0 mu_0 + 2 sum_{n>=1} g_n mu_n cos(n pi (k - 1/2)/Nq)   (Eq. quad ff.)
 *   E_k     = a cos(pi (k - 1/2)/Nq) + b
 *   w_k     = mult (dim/Nq) gamma_k exp(-(E_k - E_ref)/T),  E_ref = min E_k
 *   Z = exp(-E_ref/T) sum w,  E = sum w E_k / sum w,
 *   C = sum w (E_k - E)^2 / (T^2 sum w)                               (Eq. E-2-2-B)
 *   chi = (<M^2> - <M>^2) / T, <M^p> = sum w^(p) / sum w                (Eq. E-2-2-C)
 * where w^(1), w^(2) are built in the same way from mu_M and mu_M2,
 * mult = 2 for a sector flagged in `mirror` (it stands for +M and -M, whose
 * <M> contributions cancel: its mu_M is not used) and 1 otherwise.
 * k_B = 1 and chi is in units of (g mu_B)^2.  Outputs per temperature:
 *   lnZ = ln|Z|, signZ = sign of Z (the truncated density may be negative),
 *   E, C, chi.
 * n_quad = Nq (0 -> K).  mirror may be NULL (no mirrored sectors).  dim, a,
 * b, mirror and T are host arrays; mu, mu_M, mu_M2 and the outputs follow
 * on_device.  No workspace (a few KB of scratch are allocated on `stream`).
 */
int kpm_thermo(int32_t n_sectors, int32_t n_moments, const double *mu, const double *mu_M,
               const double *mu_M2, const double *dim, const int32_t *mirror, const double *a,
               const double *b, int32_t kernel, int32_t n_quad, int32_t n_T, const double *T,
               double *lnZ, double *signZ, double *E, double *C, double *chi,
               int32_t on_device, void *stream);

/*
 * kpm_thermo_backward -- dL/dmu, dL/dmu_M, dL/dmu_M2 from dL/d{lnZ, E, C, chi}.
 *
 * Same inputs as kpm_thermo plus the cotangents of its outputs ([n_T] each,
 * NULL = zero), all following on_device.  Writes the [n_sectors][K]
 * gradients (dL_dmu_M / dL_dmu_M2 may be NULL when not wanted).  The
 * rescaling, the dimensions and the temperatures are constants.
 */
int kpm_thermo_backward(int32_t n_sectors, int32_t n_moments, const double *mu,
                        const double *mu_M, const double *mu_M2, const double *dim,
                        const int32_t *mirror, const double *a, const double *b,
                        int32_t kernel, int32_t n_quad, int32_t n_T, const double *T,
                        const double *dL_dlnZ, const double *dL_dE, const double *dL_dC,
                        const double *dL_dchi, double *dL_dmu, double *dL_dmu_M,
                        double *dL_dmu_M2, int32_t on_device, void *stream);

/*
 * kpm_moments_backward -- dL/dtheta for couplings J_b = theta[bond_class[b]].
 *
 * Given the cotangents dL/dmu, dL/dmu_M, dL/dmu_M2 ([n_sectors][K], the
 * latter two may be NULL) of a kpm_moments run with the same model,
 * sectors, a, b, K, R, seed and r0, returns in dL_dtheta[n_classes] the
 * derivative with respect to the coupling parameters, with a and b held
 * fixed.  bond_class (host, [n_bonds], values 0 .. n_classes-1, n_classes
 * <= 8) may be NULL, then every bond is its own class (n_bonds <= 8).
 * The paper has no derivative; this is the reverse-mode (adjoint) form of
 * the recursion of kpm_moments: it reruns the forward recursion storing
 * (v_n, v_{n+1}) every ckpt_interval steps (0 -> 32), then sweeps back with
 * lambda_n = d_n + 2 H' lambda_{n+1} - lambda_{n+2}, regenerating v_{n-1} =
 * 2 H' v_n - v_{n+1} on the way and resetting it to the stored pair at each
 * checkpoint, and accumulates dL/dJ_b = (1/R) [sum_n (2/a) <lambda_{n+1}, H_b v_n>
 * + (1/a) <lambda_1, H_b v_0>] (dot products over all R vectors).  FP64 only (precision must be KPM_FP64).
 * Workspace: kpm_moments_backward_workspace_size.
 */
int kpm_moments_backward(const kpm_model *model, const int32_t *bond_class, int32_t n_classes,
                         int32_t n_sectors, const int32_t *n_up, const double *a,
                         const double *b, int32_t n_moments, int32_t R, uint64_t seed,
                         uint64_t r0, int32_t precision, int32_t ckpt_interval,
                         const double *dL_dmu, const double *dL_dmu_M,
                         const double *dL_dmu_M2, double *dL_dtheta, int32_t on_device,
                         void *workspace, size_t ws_bytes, void *stream);

size_t kpm_moments_backward_workspace_size(const kpm_model *model, int32_t n_sectors,
                                           const int32_t *n_up, int32_t n_moments,
                                           int32_t R, int32_t ckpt_interval);

/*
 * kpm_moments_static -- kpm_moments without any device allocation.
 *
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc: applications whose framework reserves the device
 * memory up front in its own pool (where a further cudaMalloc fails or
 * fragments the pool), and latency-critical loops that must stay out of the
 * CUDA allocator (cudaFree waits for the whole device).  It computes exactly
 * what kpm_moments computes, with the same kernels, but takes its scratch
 * from a fixed array of kpm_static_scratch_bytes() bytes (64 MiB) compiled
 * into the library, which every GPU that loads the library holds until the
 * process exits.
 *   a, b         -- host [n_sectors] rescaling (required: no bound estimate is run).
 *   mu, mu_M, mu_M2 -- DEVICE arrays [n_sectors][K] (mu_M, mu_M2 may be NULL).
 *   other arguments as in kpm_moments.
 * Returns KPM_ENOMEM, with the needed size in kpm_last_error(), when the
 * problem's scratch (kpm_moments_workspace_size) exceeds the array.  The
 * first call on a device looks up the array's device address with
 * cudaGetSymbolAddress while that device is current; make that first call
 * before any stream capture.  All calls share the array and every call
 * clears the parts that must start at zero; calls whose work overlaps on the
 * GPU (different streams or threads) race on it and must be serialised by
 * the caller.
 */
int kpm_moments_static(const kpm_model *model, int32_t n_sectors, const int32_t *n_up,
                       const double *a, const double *b, int32_t n_moments, int32_t R,
                       uint64_t seed, uint64_t r0, int32_t precision, double *mu, double *mu_M,
                       double *mu_M2, void *stream);

/* Size in bytes of the fixed scratch array behind kpm_moments_static. */
size_t kpm_static_scratch_bytes(void);

/*
 * Instrumentation (no counterpart in the paper; used by the benchmark).
 * kpm_profile_enable(1) starts recording a CUDA event pair around every
 * launch of the fused Chebyshev step kernel, on the stream it is launched
 * on, and clears earlier records; kpm_profile_enable(0) stops recording.
 * kpm_profile_read waits for the recorded events, returns the summed
 * device time of the recorded step launches (ms) and their count, and
 * clears the records.  kernel_launches returns the number of kernels the
 * library launched since it was loaded (any pointer may be NULL).
 */
int kpm_profile_enable(int32_t on);
int kpm_profile_read(double *step_ms_total, int64_t *step_launches, int64_t *kernel_launches);

#ifdef __cplusplus
}
#endif

#endif /* KPM_H */
