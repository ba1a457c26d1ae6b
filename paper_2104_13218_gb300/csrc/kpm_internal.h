// Internal declarations of libkpm: host-side plan of the S^z basis, the tile
// list of one launch, error helpers and the argument structs of the kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "kpm.h"

namespace kpm {

constexpr int kMaxSites = 34;
constexpr int kMaxBonds = 256;
constexpr int kMaxClasses = 8;
constexpr int kThreads = 256;     // threads per block of the streaming kernels
constexpr int kWarps = kThreads / 32;

// ---------------------------------------------------------------- errors
void set_error(const char *fmt, ...);
void clear_error();

#define KPM_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess) {                                                             \
      ::kpm::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                       __LINE__);                                                        \
      return KPM_ECUDA;                                                                  \
    }                                                                                    \
  } while (0)

#define KPM_REQUIRE(cond, code, ...) \
  do {                               \
    if (!(cond)) {                   \
      ::kpm::set_error(__VA_ARGS__); \
      return (code);                 \
    }                                \
  } while (0)

#define KPM_TRY(expr)       \
  do {                      \
    int rc_ = (expr);       \
    if (rc_ != KPM_OK) {    \
      return rc_;           \
    }                       \
  } while (0)

// ---------------------------------------------------------------- plan
// A tile is a run of consecutive ranks of one sector, processed by one block
// (by one warp in the neighbour-list step kernel).
struct Tile {
  int64_t row0;      // global row (over all sectors) of the first state
  uint32_t rank0;    // rank of the first state inside its sector
  uint32_t count;    // number of states
  uint32_t b_first;  // hi-block (global index into hb_*) holding rank0 (sector mode)
  uint32_t b_last;   // hi-block holding rank0 + count - 1
  int32_t sector;
  int32_t pad;
};
static_assert(sizeof(Tile) == 32, "Tile layout");

// Per-sector constants read by the kernels.
struct SectorDev {
  int64_t row0;      // first global row
  int64_t dim;
  int32_t n_up;      // -1 = full space
  int32_t hb_begin;  // first hi-block of this sector
  double inv_a;      // 1/a
  double b;          // shift
  double Mval;       // magnetisation of the sector (full space: 0)
  int32_t out_index; // row of this sector in the caller's moment arrays
  int32_t pad2;
};

// The S^z basis of one call: split rank tables shared by all sectors.
// rank(s) = lo_rank[s & (2^L - 1)] + hi_rank[c][s >> L], c = popcount(s & (2^L - 1)):
// the colex rank sum_j C(p_j, j+1) split into the contribution of the low L
// bits and of the high H = N - L bits (which depends on how many of the
// state's set bits lie below).  Hi-block b of a sector is the run of ranks
// sharing the high pattern hb_hi[b]; it starts at rank hb_off[b] and its low
// parts are lo_list[lo_start[c] ..] in increasing order.
struct Plan {
  int N = 0, L = 0, H = 0;
  int n_sectors = 0;
  bool any_full = false, any_sector = false;
  std::vector<int> n_up;
  std::vector<int64_t> dim, row0;
  int64_t total_rows = 0;
  std::vector<uint32_t> lo_rank, hi_rank, lo_list, lo_start, hb_hi, hb_off;
  std::vector<int32_t> hb_begin;
  std::vector<Tile> tiles;
  std::vector<int32_t> tile_begin, tile_end;
  int64_t tile_states = 0;
};

int64_t binom(int n, int k);
int validate_model(const kpm_model *m);
int validate_sectors(const kpm_model *m, int n_sectors, const int32_t *n_up);
// Builds tables and tiles; tile_states = states per tile (a power of two).
// L_split > 0 sets the low/high split of the rank tables (default N/2).
int build_plan(const kpm_model *m, int n_sectors, const int32_t *n_up, int64_t tile_states,
               Plan *plan, int L_split = 0);
// States per tile for a layout with gpw states per warp and total_rows rows.
int64_t choose_tile_states(int gpw, int64_t total_rows);
// States per tile of the list kernel, whose tiles are taken by single warps.
#ifndef KPM_LIST_TILE_STATES
#define KPM_LIST_TILE_STATES 16
#endif
#ifndef KPM_LIST_MAX_TILES
#define KPM_LIST_MAX_TILES (1 << 22)
#endif
int64_t list_tile_states(int gpw, int64_t total_rows);

// Device copies of the plan's tables (pointers into a workspace).
struct TablesDev {
  const uint32_t *lo_rank;
  const uint32_t *hi_rank;
  const uint32_t *lo_list;
  const uint32_t *lo_start;
  const uint32_t *hb_hi;
  const uint32_t *hb_off;
  const Tile *tiles;
  const SectorDev *sectors;
  const int32_t *tile_begin;
  const int32_t *tile_end;
  int32_t n_tiles;
  int32_t n_sectors;
  int32_t N, L, H;
  int32_t pad;
};

constexpr int kMaxGroups = 4;       // distinct coupling values handled by the grouped step
constexpr int kMaxDiagTable = 4096; // entries of the per-sector diagonal table

// Bond list as kernel parameter (constant bank, broadcast to the warp).
// Bonds with equal J form a group; `order` lists the bonds group by group.
// The step kernel sums the gathered neighbours of each group and applies the
// group's coupling once, and reads the diagonal from a table indexed by the
// number of anti-aligned bonds per group, index = sum_g n_g * tstride[g].
struct BondsDev {
  int32_t n_bonds;
  int32_t n_sites;
  double J_quarter_sum;            // sum_b J_b / 4
  uint64_t mask[kMaxBonds];        // (1 << i_b) | (1 << j_b)
  double J[kMaxBonds];
  int32_t n_groups;                // 0: more than kMaxGroups values (per-bond path)
  int32_t table_size;              // prod_g (group size + 1)
  int32_t gstart[kMaxGroups + 1];  // group g = order[gstart[g] .. gstart[g+1])
  int32_t tstride[kMaxGroups];
  double gJ[kMaxGroups];
  uint8_t order[kMaxBonds];
  // Cooperative layouts (G >= 2 lanes per state): in pass p lane j of a group
  // tests bond p*G + j; pmask[p][g] has bit j set when that bond is in group g.
  int32_t G;                       // lanes per state this table was built for
  int32_t n_pass;                  // ceil(n_bonds / G)
  uint32_t pmask[kMaxBonds / 2][kMaxGroups];
};
// Fills pmask / n_pass for a layout with G lanes per state.
void fill_pass_masks(BondsDev *b, int G);
void fill_bonds(const kpm_model *m, BondsDev *out);

// Simple bump allocator over a workspace region (256-byte aligned pieces).
struct Arena {
  char *base = nullptr;
  size_t size = 0, used = 0;
  template <typename T>
  T *take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    if (used + bytes > size) return nullptr;
    T *p = reinterpret_cast<T *>(base + used);
    used += bytes;
    return p;
  }
};
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of the device copies of the plan tables.
size_t tables_bytes(const Plan &p);
// Uploads the plan's tables into the arena (async on stream).
int upload_tables(const Plan &p, const std::vector<SectorDev> &sectors, Arena &arena,
                  cudaStream_t stream, TablesDev *out);

// Scoped workspace: either the caller's region or a stream-ordered allocation.
struct Workspace {
  void *ptr = nullptr;
  size_t size = 0;
  bool owned = false;
  cudaStream_t stream = nullptr;
  int acquire(void *user, size_t user_bytes, size_t need, cudaStream_t s);
  ~Workspace();
};

// Row layout of the interleaved vectors: each state's row holds Rp values
// (R rounded up so that the row is G lanes x CPL chunks of 16 bytes).
struct RowLayout {
  int R = 0, Rp = 0;
  int vec_width = 0;   // values per 16-byte chunk: 4 (FP32) or 2 (FP64)
  int chunks = 0;      // 16-byte chunks per row
  int cpl = 0;         // chunks per lane
  int G = 0;           // lanes per state
  int gpw = 0;         // states per warp
  int elem = 0;        // bytes per value
};
int make_layout(int R, int precision, RowLayout *out);

// Tridiagonal eigenvalue tools of the Lanczos bounds (diagonal al[0..m),
// couplings be[1..m), be[i] between i-1 and i): the k-th smallest eigenvalue
// by Sturm bisection, and |last component| of the unit eigenvector of theta.
double tridiag_eig(const std::vector<double> &al, const std::vector<double> &be, int m, int k);
double ritz_last_component(const std::vector<double> &al, const std::vector<double> &be, int m,
                           double theta);

// Instrumentation: count kernel launches; bracket step launches with events.
void count_launches(int n);
bool profiling();
void profile_push(cudaEvent_t start, cudaEvent_t stop);

}  // namespace kpm
