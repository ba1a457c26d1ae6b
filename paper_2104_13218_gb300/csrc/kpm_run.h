// Driver of the Chebyshev moment loop shared by kpm_moments and the adjoint.
#pragma once

#include "kpm_internal.h"

namespace kpm {

// Choices of the moment loop that do not change its results beyond rounding
// order: which step kernel, the tile size, the persistent grid, the row
// mapping and which sectors of the FP32 form run in FP64.  Zero / negative
// values select the library's defaults; kpm_autotune searches them.
struct Knobs {
  int lists = -1;            // neighbour-list kernel: -1 default, 0 off, 1 on (where it applies)
  int64_t tile_states = 0;   // states per tile (0: default for the kernel)
  int blocks_per_sm = 0;     // persistent grid: resident blocks per SM used (0: all that fit)
  int two_state = -1;        // FP32 rows of 17..32 chunks as two states per warp: -1 default
  int64_t side_min_dim = -1; // FP32 form: sectors below this dimension run in FP64 (-1: 1024)
  int block = -1;            // hi-block kernel for one-lane sector layouts: -1 default, 0 off
};

// Coefficients of H' per sector and kind of step (first: A = 1/a, later:
// A = 2/a), computed on the host once per run: the diagonal A (d - b) for every
// combination of anti-aligned bond counts per coupling group, and A J_g / 2 for
// every group, each as hi (+ lo in FP32).
struct CoefDev {
  const void *diag_hi, *diag_lo;  // [n_sectors][2][table_size] of T
  const void *grp_hi, *grp_lo;    // [n_sectors][2][kMaxGroups] of T
};

// Bonds of the hi-block kernel, split by where their sites lie relative to the
// low bits (L): low bonds (both sites below L, masks on the low bits), high
// bonds (both at or above L, masks on the high bits) and cross bonds (one of
// each: low bit position, high bit position).  Each list is sorted by
// coupling group; *_gs[g] .. *_gs[g+1] are the bonds of group g.
constexpr int kBlockMaxBonds = 64;
struct BlockBondsDev {
  int32_t L;
  int32_t n_groups;
  int32_t tstride[kMaxGroups];
  int32_t low_gs[kMaxGroups + 1], high_gs[kMaxGroups + 1], cross_gs[kMaxGroups + 1];
  uint32_t low_mask[kBlockMaxBonds];
  uint32_t high_mask[kBlockMaxBonds];
  uint8_t cross_lo[kBlockMaxBonds], cross_hi[kBlockMaxBonds];
};

// Random vectors of a run: Rademacher signs (Eq. E-2-7 with the sign
// convention of the library) or, for complete-basis traces, unit vectors.
constexpr int kVecRademacher = 0;
constexpr int kVecBasis = 1;

// Everything one forward run needs on the device.
struct MomentsRun {
  Plan plan;
  RowLayout lay;
  BondsDev bonds;
  TablesDev tb;
  int precision = KPM_FP64;
  int K = 0, S = 0;        // moments, matrix-vector products (S = K/2)
  int NQ = 2;              // dot products per step: 2, or 6 with a full-space sector
  int grid = 0;            // persistent grid of the step kernel
  size_t vec_bytes = 0;    // one interleaved vector (all sectors)
  void *vA = nullptr, *vB = nullptr;
  double *partials = nullptr;  // [n_tiles][NQ] ([2][n_tiles][NQ] with lists)
  double *sums = nullptr;      // [S][n_sectors][NQ]
  int *counters = nullptr;     // [2*S]: tile queue and finished-block count per step
  int *flag = nullptr;         // EBOUNDS flag
  bool profile = true;         // bracket step launches with events when profiling
  // Neighbour lists (cooperative layouts with grouped couplings): per state,
  // list_stride words: a header with the number of anti-aligned bonds of each
  // coupling group (8 bits per group), then the first 16-byte chunk index of
  // each bit-flipped neighbour's row, group by group.  Built once per run.
  int list_stride = 0;         // 0: no lists (the step works matrix-free)
  uint32_t *lists = nullptr;
  // With lists: coefficients of H' per sector and kind of step (first, later),
  // diagonal table hi / lo and group couplings hi / lo (lo only in FP32), and
  // two slots of per-tile sums (partials) used by alternate steps.
  void *coef[4] = {nullptr, nullptr, nullptr, nullptr};
  Knobs knobs;
  // Hi-block kernel (one lane per state, sector runs): one work item per
  // hi-block, whose rows are staged in shared memory; block_L > 0 selects it
  // and is the low split of the rank tables.
  int block_L = 0;
  int64_t max_block = 0;           // states of the largest hi-block
  BlockBondsDev bb{};
  const int32_t *blk_sector = nullptr;  // [n_blocks] sector of each hi-block
  TablesDev tbb{};                 // tables whose "tiles" are the hi-blocks (for the sums)
  int32_t *blk_ranges = nullptr;   // [2][n_sectors]: first / end hi-block of each sector
  int vectors = kVecRademacher;
  // Per-vector moments (optional): the rows are cut into chunks of one
  // sector each; after every step a column kernel writes each chunk's
  // per-vector dot products (cd_part) and a second kernel sums them per
  // sector in chunk order into sums_r [S][n_sectors][R][2].
  bool per_vector = false;
  std::vector<int64_t> cd_chunks;  // host: (row_begin, row_end, sector) per chunk
  const int64_t *cd_dev = nullptr; // device copy
  int n_cd = 0;
  double *cd_part = nullptr;       // [n_cd][R][2]
  double *sums_r = nullptr;        // [S][n_sectors][R][2]
};

// The FP32 form stores sectors smaller than this in FP64: in a tiny sector the
// +-1/sqrt(D) vectors keep few distinct magnitudes, FP32 rounding errors stay
// coherent instead of averaging out, and they grow linearly with the order.
constexpr int64_t kFP32MinSectorDim = 1024;

// A kpm_moments call: the main run, plus (FP32 form only) an FP64 run of the
// sectors below kFP32MinSectorDim.
struct MomentsJob {
  MomentsRun main, side;
  bool has_main = false, has_side = false;
  std::vector<int32_t> nup_main, nup_side;
  std::vector<int> map_main, map_side;  // job sector -> caller sector
  int n_sectors = 0, K = 0;
};
int prepare_job(const kpm_model *m, int n_sectors, const int32_t *n_up, int K, int R,
                int precision, MomentsJob *job, const Knobs &knobs = Knobs(),
                int vectors = kVecRademacher, bool per_vector = false);
size_t job_bytes(const MomentsJob &job);
int setup_job(MomentsJob &job, const double *a, const double *b, Arena &arena, cudaStream_t s);
// init + K/2 steps + assembly of both runs, all on stream s, or with a side
// stream the FP64 side run on `side` (forked from and joined back into s).
int run_job(MomentsJob &job, uint64_t seed, uint64_t r0, double *mu, double *mu_M, double *mu_M2,
            cudaStream_t s, cudaStream_t side = nullptr, double *mu_r = nullptr);
// The side stream of the current device (created on first use).
int side_stream(cudaStream_t *out);

// Builds the plan and the layout; no device work.
int prepare_run(const kpm_model *m, int n_sectors, const int32_t *n_up, int K, int R,
                int precision, MomentsRun *run, const Knobs &knobs = Knobs(),
                int vectors = kVecRademacher, bool per_vector = false);
// Device bytes of the run's vectors (2), tables, partials, sums and counters.
size_t run_bytes(const MomentsRun &run);
// Carves the run's buffers from the arena and uploads tables (a, b per sector).
int setup_run(MomentsRun &run, const double *a, const double *b, Arena &arena,
              cudaStream_t stream, const int *out_index = nullptr);
// Neighbour lists of every state of the tables' tiles (header word of
// per-group counts, then each group's neighbour chunks = row * crow, each
// group padded with zero_chunk to a multiple of batch).  entry_stride 1:
// state-major (state row's entries at row * stride + e); otherwise
// entry-major (at e * entry_stride + row).
int launch_build_lists(const TablesDev &tb, const BondsDev &bd, int64_t n_tiles, uint32_t *lists,
                       int stride, uint32_t crow, int batch, uint32_t zero_chunk, cudaStream_t s,
                       uint64_t entry_stride = 1);
// v0 <- random vectors r0 .. r0+R-1 (padding columns zero): signs +-1/sqrt(D), or
// with `uniform` values uniform in (-1, 1) from the same hash (Lanczos start vectors).
int launch_init(const MomentsRun &run, void *v0, uint64_t seed, uint64_t r0, cudaStream_t s,
                bool uniform = false);
// One fused step.  first = 1: y = H' x (y written to zy, z not read).
// first = 0: zy <- 2 H' x - zy.  Dot products of this step go to sums[step].
int launch_step(const MomentsRun &run, const void *x, void *zy, int first, int step,
                cudaStream_t s);
// mu, mu_M, mu_M2 (device, may be NULL except mu) from sums; sets *flag on |mu| > 1+1e-6.
// With per-vector moments also mu_r [caller sectors][R][K] (device).
int launch_assemble(const MomentsRun &run, double *mu, double *mu_M, double *mu_M2,
                    cudaStream_t s, double *mu_r = nullptr);
// Per-vector dot products of step `step` (x = v_n, y = v_{n+1}) into sums_r.
int launch_column_dots(const MomentsRun &run, const void *x, const void *y, int step,
                       cudaStream_t s);
// Number of streaming multiprocessors of the current device.
int sm_count();
// The hi-block kernel (kpm_block.cu): shared memory, launch of one step.
size_t block_smem_bytes(const MomentsRun &run);
int launch_block_step(const MomentsRun &run, const void *x, void *zy, int first, double *partials,
                      int *queue, CoefDev cf, cudaStream_t s);
void *block_kernel_ptr(int precision);

}  // namespace kpm
