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

#define KPM_VERSION 2

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

/* random vectors of the trace estimator */
#define KPM_VECTORS_RADEMACHER 0  /* +-1/sqrt(D) signs from the counter-based hash (default) */
#define KPM_VECTORS_BASIS 1       /* unit vectors: vector r is the basis state of rank r0 + r
                                     (the zero vector when r0 + r >= D); summing R * mu over
                                     r0 = 0, R, 2R, ... < D gives the complete-basis trace
                                     D * (1/D) Tr T_n(H') exactly (Sec. 2, after Eq. E-2-7) */

/* Heisenberg model H = sum_b J[b] S_{bi[b]} . S_{bj[b]}; all arrays host memory. */
typedef struct {
  int32_t n_sites;        /* N, 1 .. 34 */
  int32_t n_bonds;        /* 0 .. 256 */
  const int32_t *bi;      /* [n_bonds] first site of each bond, 0 .. N-1 */
  const int32_t *bj;      /* [n_bonds] second site, != bi[b] */
  const double *J;        /* [n_bonds] coupling J_b */
} kpm_model;

/* Options of the *_ex entry points (zero-initialised = the defaults of kpm_moments
   with KPM_FP64).  A NULL pointer means the defaults. */
typedef struct {
  int32_t precision;      /* KPM_FP64 (default 0) or KPM_FP32 */
  int32_t vectors;        /* KPM_VECTORS_RADEMACHER (0) or KPM_VECTORS_BASIS */
  int32_t per_vector;     /* 1: also return the moments of every vector separately (mu_r) */
  int32_t tuned;          /* 1: run with the schedule kpm_autotune chose for this problem
                             (model, sectors, R, precision), if it has been tuned */
  int32_t ckpt_interval;  /* adjoint: steps between stored vector pairs (0 -> 32) */
  int32_t reserved[3];    /* must be 0 */
} kpm_opts;

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
 * kpm_moments_ex -- kpm_moments with options and per-vector moments.
 *
 * Same as kpm_moments (same arguments, layouts and status codes) with the
 * precision and the kind of random vectors taken from *opts, and, when
 * opts->per_vector is 1, the moments of each vector r = r0 .. r0+R-1
 * separately:
 *   mu_r[(sector * R + r) * K + n] = <r|T_n(H')|r>       (required iff per_vector)
 * (the terms of the average in Eq. E-2-7: mu = (1/R) sum_r mu_r up to rounding),
 * following on_device like mu.  With per-vector moments every step is
 * followed by a column pass that reads v_n and v_{n+1} once more (FP64 dot
 * products per vector), so the run moves about 1.7x the bytes.  With
 * KPM_VECTORS_BASIS, vector r is the unit vector of the state of rank r0 + r
 * of every sector (zero where r0 + r >= D), so R * mu summed over disjoint r0
 * ranges covering 0 .. D-1 is the exact trace Tr T_n(H') (Sec. 2, the complete
 * basis after Eq. E-2-7).  opts->tuned = 1 uses the schedule kpm_autotune
 * found for this problem (results agree to rounding order).
 * Workspace: kpm_moments_ex_workspace_size with the same opts.
 */
int kpm_moments_ex(const kpm_model *model, int32_t n_sectors, const int32_t *n_up,
                   const double *a, const double *b, double eps, int32_t n_moments, int32_t R,
                   uint64_t seed, uint64_t r0, const kpm_opts *opts, double *mu, double *mu_M,
                   double *mu_M2, double *mu_r, int32_t on_device, void *workspace,
                   size_t ws_bytes, void *stream);

size_t kpm_moments_ex_workspace_size(const kpm_model *model, int32_t n_sectors,
                                     const int32_t *n_up, int32_t n_moments, int32_t R,
                                     const kpm_opts *opts);

/*
 * kpm_autotune -- choose the schedule of the moment loop for one problem.
 *
 * The paper has no counterpart.  Times short runs of the problem (the random
 * vectors, 1 + trial_steps matrix-vector products and the assembly, best of
 * two, CUDA events on `stream`) for a one-pass coordinate search over: the
 * neighbour-list or the matrix-free step kernel, the states per tile, the
 * resident blocks per SM, one or two states per warp for FP32 rows of 17..32
 * chunks, and (FP32) the sector dimension below which sectors run in FP64
 * (searched upwards from 1024 only).  None of these changes the arithmetic
 * beyond the order of the sums.  The best choice is kept for the life of the
 * process, keyed by (model, sectors, R, precision), and used by calls whose
 * kpm_opts.tuned is 1.  a, b: host [n_sectors] rescaling.  Outputs (host, may
 * be NULL): default_ms and best_ms, the measured time per matrix-vector
 * product of the default and of the chosen schedule; report, a text listing
 * the chosen schedule and every candidate's time (truncated to report_len).
 * The trial runs allocate their scratch with cudaMallocAsync on `stream`.
 */
int kpm_autotune(const kpm_model *model, int32_t n_sectors, const int32_t *n_up,
                 const double *a, const double *b, int32_t R, int32_t precision,
                 int32_t trial_steps, double *default_ms, double *best_ms, char *report,
                 size_t report_len, void *stream);

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
 * kpm_thermo_ex -- kpm_thermo in a magnetic field.
 *
 * The Zeeman term g mu_B B sum_i s^z_i of Eq. E-3-1-1 commutes with H and
 * adds h M to every energy of the sector with magnetisation M (h = g mu_B B,
 * `field`), so the same moments serve every field: E_k = a x_k + b + h M.
 * M: host [n_sectors] magnetisation of each sector (NAN for a full-space
 * run, where M varies from state to state: field must then be 0; M may be
 * NULL when field is 0).  A sector flagged in `mirror` stands for +M and -M
 * (their moments agree in expectation): in a field its two members enter
 * with energies shifted by +h M and -h M and <M> contributions +M and -M.
 * Other arguments and outputs as for kpm_thermo.
 */
int kpm_thermo_ex(int32_t n_sectors, int32_t n_moments, const double *mu, const double *mu_M,
                  const double *mu_M2, const double *dim, const int32_t *mirror, const double *M,
                  const double *a, const double *b, double field, int32_t kernel, int32_t n_quad,
                  int32_t n_T, const double *T, double *lnZ, double *signZ, double *E, double *C,
                  double *chi, int32_t on_device, void *stream);

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

/* kpm_thermo_backward in a magnetic field (M and field as in kpm_thermo_ex). */
int kpm_thermo_backward_ex(int32_t n_sectors, int32_t n_moments, const double *mu,
                           const double *mu_M, const double *mu_M2, const double *dim,
                           const int32_t *mirror, const double *M, const double *a,
                           const double *b, double field, int32_t kernel, int32_t n_quad,
                           int32_t n_T, const double *T, const double *dL_dlnZ,
                           const double *dL_dE, const double *dL_dC, const double *dL_dchi,
                           double *dL_dmu, double *dL_dmu_M, double *dL_dmu_M2,
                           int32_t on_device, void *stream);

/*
 * kpm_realisations -- statistics over P realisations of the trace estimator.
 *
 * Sec. 3 treats each realisation O_i(beta) of an observable as a random
 * measurement: mean O-bar = (1/P) sum_i O_i (Eq. E-3-1), variance
 * dO^2 = mean(O^2) - O-bar^2 (Eq. E-3-2) and, against an exact curve O_E,
 * the systematic deviation |O-bar - O_E| (Eq. E-3-3).  Here realisation p
 * uses the vectors p*R_per .. p*R_per + R_per - 1 of one per-vector moment
 * run (kpm_moments_ex with per_vector = 1): its moments are their average,
 * its observables lnZ, E, C, chi follow from the quadrature of kpm_thermo_ex
 * (same dim, mirror, M, a, b, field, kernel, n_quad, T).  P = R / R_per (R a
 * multiple of R_per; R_per = 1 gives P = R realisations of one vector each).
 * Sector runs only (M finite; mu_M = M mu and mu_M2 = M^2 mu are formed here).
 *   mu_r   -- [n_sectors][R][K] per-vector moments (follows on_device).
 *   exact  -- [4][n_T] exact lnZ, E, C, chi (may be NULL; follows on_device).
 *   mean, var -- [4][n_T] outputs; dev -- [4][n_T] (NULL, or requires exact);
 *   all    -- [P][4][n_T] every realisation's curves (may be NULL).
 * Rows of the [4][n_T] arrays are lnZ, E, C, chi.  Scratch is allocated with
 * cudaMallocAsync on `stream`.
 */
int kpm_realisations(int32_t n_sectors, int32_t n_moments, int32_t R, int32_t R_per,
                     const double *mu_r, const double *dim, const int32_t *mirror,
                     const double *M, const double *a, const double *b, double field,
                     int32_t kernel, int32_t n_quad, int32_t n_T, const double *T,
                     const double *exact, double *mean, double *var, double *dev, double *all,
                     int32_t on_device, void *stream);

/*
 * kpm_moments_backward -- dL/dtheta for couplings J_b = theta[bond_class[b]].
 *
 * Given the cotangents dL/dmu, dL/dmu_M, dL/dmu_M2 ([n_sectors][K], the
 * latter two may be NULL) of a kpm_moments run with the same model,
 * sectors, a, b, K, R, seed and r0, returns in dL_dtheta[n_classes] the
 * derivative with respect to the coupling parameters, with a and b held
 * fixed.  bond_class (host, [n_bonds], values 0 .. n_classes-1, n_classes
 * <= 256) may be NULL, then every bond is its own class (dL/dJ_b per bond).
 * Up to 8 classes are summed in registers; more classes are summed per bond
 * in shared memory and then per class.
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
 * kpm_moments_backward_ex -- kpm_moments_backward with options: opts->precision
 * (must be KPM_FP64), opts->vectors (the random vectors of the forward run
 * being differentiated, e.g. KPM_VECTORS_BASIS for complete-basis traces) and
 * opts->ckpt_interval; opts->per_vector must be 0.  Workspace as for
 * kpm_moments_backward.
 */
int kpm_moments_backward_ex(const kpm_model *model, const int32_t *bond_class, int32_t n_classes,
                            int32_t n_sectors, const int32_t *n_up, const double *a,
                            const double *b, int32_t n_moments, int32_t R, uint64_t seed,
                            uint64_t r0, const kpm_opts *opts, const double *dL_dmu,
                            const double *dL_dmu_M, const double *dL_dmu_M2, double *dL_dtheta,
                            int32_t on_device, void *workspace, size_t ws_bytes, void *stream);

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
 * cudaGetSymbolAddress while that device is current (and so does the first
 * call after the device's context was replaced, e.g. by cudaDeviceReset).
 * Like kpm_moments, every
 * call waits for `stream` before it returns (it reads the EBOUNDS flag back to
 * the host).  All calls share the array and every call clears the parts that
 * must start at zero; calls whose work overlaps on the GPU (different streams
 * or threads) race on it and must be serialised by the caller.
 */
int kpm_moments_static(const kpm_model *model, int32_t n_sectors, const int32_t *n_up,
                       const double *a, const double *b, int32_t n_moments, int32_t R,
                       uint64_t seed, uint64_t r0, int32_t precision, double *mu, double *mu_M,
                       double *mu_M2, void *stream);

/* Size in bytes of the fixed scratch array behind kpm_moments_static. */
size_t kpm_static_scratch_bytes(void);

/*
 * Spin-s Heisenberg models (Sec. 3.4: the ring of N = 10 spins s = 5/2)
 * ---------------------------------------------------------------------
 * H = sum_b J_b S_i . S_j for local spin s = two_s/2 (Eq. E-3-1-1), in the
 * S^z product basis.  A state stores the digit q_i = m_i + s of site i in bits
 * 3i .. 3i+2 of its code; sector Q holds the states of digit sum Q (total
 * S^z = M = Q - N s) ordered by increasing code, and Q = -1 the whole
 * (2s+1)^N space ordered by the base-(2s+1) value of the digits.  Random
 * vectors follow the spin-1/2 convention with the code in place of the
 * bitstring.  Limits: two_s 1 .. 7, N <= 16, sector dimensions below 2^32,
 * and rank tables of at most 2^26 entries ((2s N/2 + 1) * 8^(N - N/2)).
 * These calls allocate their device scratch with cudaMallocAsync on
 * `stream` and free it before returning; there is no adjoint for s > 1/2.
 */
typedef struct {
  int32_t n_sites;   /* N, 1 .. 16 */
  int32_t n_bonds;   /* 0 .. 256 */
  int32_t two_s;     /* 2s, 1 .. 7 */
  int32_t pad;
  const int32_t *bi; /* [n_bonds] host */
  const int32_t *bj;
  const double *J;
} kpm_spin_model;

/* Dimension of sector Q (coefficient of x^Q in (1 + x + .. + x^{2s})^N; Q = -1:
   (2s+1)^N); -1 if invalid. */
int64_t kpm_spin_sector_dim(int32_t n_sites, int32_t two_s, int32_t Q);

/*
 * kpm_spin_bounds -- Lanczos bounds and rescaling (Eq. E-2-3, E-2-4) of spin-s
 * sectors: one FP64 Lanczos sequence per sector (start vector uniform in
 * (-1, 1) from `seed`), checked every 8 steps, stopping when the extreme Ritz
 * values' residual bounds are within tol relative to max(1, |E|); outputs and
 * status as kpm_bounds (a, b, e_min, e_max host arrays; KPM_ENOTCONV when
 * max_iter steps do not reach tol).
 */
int kpm_spin_bounds(const kpm_spin_model *model, int32_t n_sectors, const int32_t *Q, double eps,
                    int32_t max_iter, double tol, uint64_t seed, double *a, double *b,
                    double *e_min, double *e_max, void *stream);

/*
 * kpm_spin_moments -- the stochastic Chebyshev moments of kpm_moments (Eq. E-2-6,
 * E-2-7, mu_0 = 1) for spin-s sectors: a, b host [n_sectors] (required); K
 * even >= 2; R 1 .. 512; precision KPM_FP64 or KPM_FP32 (FP32 vectors, FP64
 * dot products, coefficients as float pairs); mu [n_sectors][K] and, if not
 * NULL, mu_M, mu_M2 (M- and M^2-weighted, M = digit sum - N s; for a sector M mu
 * and M^2 mu); on_device as for kpm_moments.  KPM_EBOUNDS when |mu_n| > 1 + 1e-6.
 * The thermodynamics follow from kpm_thermo_ex with dim = kpm_spin_sector_dim
 * and M = Q - N s.
 */
int kpm_spin_moments(const kpm_spin_model *model, int32_t n_sectors, const int32_t *Q,
                     const double *a, const double *b, int32_t n_moments, int32_t R,
                     uint64_t seed, uint64_t r0, int32_t precision, double *mu, double *mu_M,
                     double *mu_M2, int32_t on_device, void *stream);

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

/*
 * kpm_fp64_peak -- measured FP64 fused multiply-add rate of the current device
 * (instrumentation for the roofline of the FP64 form; no counterpart in the
 * paper).  Runs 8 independent FMA chains per thread on 8 blocks of 256
 * threads per SM, growing the run until one timed launch lasts >= 50 ms
 * (CUDA events on `stream`), and returns *tflops = 2 x FMAs / time in
 * TFLOP/s and *ms the timed launch (ms may be NULL).  Changes no device
 * setting; allocates its output buffer with cudaMallocAsync.
 */
int kpm_fp64_peak(double *tflops, double *ms, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* KPM_H */
