// Host side of libkpm: argument checks, the split combinadic rank tables of
// the S^z sectors (Sec. 2: the basis is decomposed by total magnetisation M,
// sector = states with N/2 + M up spins), the tile list of a launch, the
// workspace and the row layout of the interleaved random vectors.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>

#include "kpm_internal.h"

namespace kpm {

namespace {
thread_local char g_error[1024] = "";
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_error, sizeof(g_error), fmt, ap);
  va_end(ap);
}

void clear_error() { g_error[0] = '\0'; }

const char *last_error() { return g_error; }

namespace {
// Pascal's triangle up to n = 64 (C(64, 32) < 2^63), built once.
struct PascalTable {
  int64_t c[65][65];
  PascalTable() {
    for (int n = 0; n <= 64; ++n) {
      c[n][0] = 1;
      for (int k = 1; k <= 64; ++k) c[n][k] = n == 0 ? 0 : c[n - 1][k - 1] + c[n - 1][k];
    }
  }
};
const PascalTable &pascal() {
  static const PascalTable t;
  return t;
}
}  // namespace

int64_t binom(int n, int k) {
  if (k < 0 || n < 0 || k > n || n > 64) return 0;
  return pascal().c[n][k];
}

int validate_model(const kpm_model *m) {
  KPM_REQUIRE(m != nullptr, KPM_EINVAL, "model is NULL");
  KPM_REQUIRE(m->n_sites >= 1 && m->n_sites <= kMaxSites, KPM_EINVAL,
              "n_sites = %d outside 1..%d", m->n_sites, kMaxSites);
  KPM_REQUIRE(m->n_bonds >= 0 && m->n_bonds <= kMaxBonds, KPM_EINVAL,
              "n_bonds = %d outside 0..%d", m->n_bonds, kMaxBonds);
  if (m->n_bonds > 0)
    KPM_REQUIRE(m->bi && m->bj && m->J, KPM_EINVAL, "bond arrays are NULL");
  for (int b = 0; b < m->n_bonds; ++b) {
    KPM_REQUIRE(m->bi[b] >= 0 && m->bi[b] < m->n_sites && m->bj[b] >= 0 &&
                    m->bj[b] < m->n_sites && m->bi[b] != m->bj[b],
                KPM_EINVAL, "bond %d = (%d, %d) is not a pair of distinct sites", b, m->bi[b],
                m->bj[b]);
  }
  return KPM_OK;
}

int validate_sectors(const kpm_model *m, int n_sectors, const int32_t *n_up) {
  KPM_REQUIRE(n_sectors >= 1 && n_up != nullptr, KPM_EINVAL, "need at least one sector");
  for (int s = 0; s < n_sectors; ++s)
    KPM_REQUIRE(n_up[s] >= -1 && n_up[s] <= m->n_sites, KPM_EINVAL,
                "n_up[%d] = %d outside -1..%d", s, n_up[s], m->n_sites);
  return KPM_OK;
}

int64_t choose_tile_states(int gpw, int64_t total_rows) {
  // 32 block iterations of kWarps * gpw states, but at least ~4 tiles per SM
  // for small problems (152 SMs).
  int64_t big = (int64_t)32 * kWarps * gpw;
  int64_t small = std::max<int64_t>((int64_t)kWarps * gpw, total_rows / (4 * 152));
  return std::max<int64_t>(1, std::min(big, small));
}

int64_t list_tile_states(int gpw, int64_t total_rows) {
  // Small warp tiles keep the states being worked on at any moment (about one
  // tile per resident warp) close together, so that their neighbours' rows
  // are shared in L2; tiles are enlarged only to stay within the tile limit.
  int64_t t = std::max<int64_t>(KPM_LIST_TILE_STATES, gpw);
  t = std::max<int64_t>(t, (total_rows + KPM_LIST_MAX_TILES - 1) / KPM_LIST_MAX_TILES);
  return (t + gpw - 1) / gpw * gpw;
}

int build_plan(const kpm_model *m, int n_sectors, const int32_t *n_up, int64_t tile_states,
               Plan *p, int L_split) {
  KPM_TRY(validate_model(m));
  KPM_TRY(validate_sectors(m, n_sectors, n_up));
  KPM_REQUIRE(tile_states >= 1, KPM_EINVAL, "tile_states < 1");
  const int N = m->n_sites;
  for (int s = 0; s < n_sectors; ++s)
    KPM_REQUIRE(n_up[s] >= 0 || N <= 32, KPM_EINVAL,
                "the full 2^N space is limited to N <= 32 (ranks are 32-bit); use sectors");
  p->N = N;
  p->L = (L_split > 0 && L_split <= N) ? L_split : N / 2;
  p->H = N - p->L;
  KPM_REQUIRE(p->H <= 24, KPM_EINVAL, "high part of %d bits: rank tables too large", p->H);
  p->n_sectors = n_sectors;
  p->n_up.assign(n_up, n_up + n_sectors);
  p->dim.resize(n_sectors);
  p->row0.resize(n_sectors);
  p->any_full = p->any_sector = false;
  int64_t rows = 0;
  for (int s = 0; s < n_sectors; ++s) {
    p->dim[s] = n_up[s] < 0 ? ((int64_t)1 << N) : binom(N, n_up[s]);
    p->row0[s] = rows;
    rows += p->dim[s];
    if (n_up[s] < 0)
      p->any_full = true;
    else
      p->any_sector = true;
  }
  p->total_rows = rows;
  p->tile_states = tile_states;

  const int L = p->L, H = p->H;
  const uint32_t nlo = 1u << L, nhi = 1u << H;
  const auto &C = pascal().c;  // C[n][k], n <= 64
  p->lo_rank.clear();
  p->hi_rank.clear();
  p->lo_list.clear();
  p->lo_start.clear();
  p->hb_hi.clear();
  p->hb_off.clear();
  p->hb_begin.assign(n_sectors, 0);
  if (p->any_sector) {
    // low part: colex rank of the low bits among patterns of equal popcount
    p->lo_rank.resize(nlo);
    std::vector<uint32_t> count(L + 2, 0);
    for (uint32_t lo = 0; lo < nlo; ++lo) {
      uint64_t r = 0;
      int j = 0;
      for (int q = 0; q < L; ++q)
        if ((lo >> q) & 1u) r += (uint64_t)C[q][++j];
      p->lo_rank[lo] = (uint32_t)r;
      count[__builtin_popcount(lo)]++;
    }
    p->lo_start.assign(L + 2, 0);
    for (int c = 0; c <= L; ++c) p->lo_start[c + 1] = p->lo_start[c] + count[c];
    p->lo_list.resize(nlo);
    std::vector<uint32_t> fill(p->lo_start.begin(), p->lo_start.end());
    for (uint32_t lo = 0; lo < nlo; ++lo) p->lo_list[fill[__builtin_popcount(lo)]++] = lo;
    // high part given c set bits below it: the terms C(L + q, j) of its set
    // bits q, the j-th set bit overall; built from the entry without the top
    // bit, so each entry costs one addition
    p->hi_rank.resize((size_t)(L + 1) * nhi);
    for (int c = 0; c <= L; ++c) {
      uint32_t *row = p->hi_rank.data() + (size_t)c * nhi;
      row[0] = 0;
      for (uint32_t hi = 1; hi < nhi; ++hi) {
        const int top = 31 - __builtin_clz(hi);
        const uint32_t rest = hi & ~(1u << top);
        row[hi] = row[rest] + (uint32_t)C[L + top][c + __builtin_popcount(hi)];
      }
    }
    // hi-blocks of every sector in increasing order of the high pattern
    for (int s = 0; s < n_sectors; ++s) {
      p->hb_begin[s] = (int32_t)p->hb_hi.size();
      if (n_up[s] < 0) continue;
      int64_t covered = 0;
      for (uint32_t hi = 0; hi < nhi; ++hi) {
        int c = n_up[s] - __builtin_popcount(hi);
        if (c < 0 || c > L) continue;
        p->hb_hi.push_back(hi);
        p->hb_off.push_back(p->hi_rank[(size_t)c * nhi + hi]);
        covered += binom(L, c);
      }
      KPM_REQUIRE(covered == p->dim[s], KPM_EINVAL, "internal: sector %d blocks cover %lld of %lld",
                  s, (long long)covered, (long long)p->dim[s]);
    }
  }
  // tiles
  p->tiles.clear();
  p->tile_begin.assign(n_sectors, 0);
  p->tile_end.assign(n_sectors, 0);
  size_t n_tiles = 0;
  for (int s = 0; s < n_sectors; ++s) n_tiles += (size_t)((p->dim[s] + tile_states - 1) / tile_states);
  p->tiles.reserve(n_tiles);
  for (int s = 0; s < n_sectors; ++s) {
    p->tile_begin[s] = (int32_t)p->tiles.size();
    const int32_t hb0 = p->hb_begin[s];
    const int32_t hb1 = (n_up[s] < 0) ? hb0
                                      : ((s + 1 < n_sectors) ? p->hb_begin[s + 1] : (int32_t)p->hb_hi.size());
    // hi-block holding a rank: tiles are in increasing rank order, so the
    // block index only moves forward (hb_off increases within a sector)
    int32_t blk = hb0;
    auto block_of = [&](uint32_t rank) {
      while (blk + 1 < hb1 && p->hb_off[blk + 1] <= rank) ++blk;
      return (uint32_t)blk;
    };
    for (int64_t r0 = 0; r0 < p->dim[s]; r0 += tile_states) {
      Tile t;
      t.row0 = p->row0[s] + r0;
      t.rank0 = (uint32_t)r0;
      t.count = (uint32_t)std::min<int64_t>(tile_states, p->dim[s] - r0);
      t.sector = s;
      t.pad = 0;
      t.b_first = t.b_last = 0;
      if (n_up[s] >= 0) {
        t.b_first = block_of((uint32_t)r0);
        t.b_last = block_of((uint32_t)(r0 + t.count - 1));
      }
      p->tiles.push_back(t);
    }
    p->tile_end[s] = (int32_t)p->tiles.size();
  }
  KPM_REQUIRE(p->tiles.size() < (size_t)INT32_MAX, KPM_EINVAL, "too many tiles");
  return KPM_OK;
}

void fill_bonds(const kpm_model *m, BondsDev *out) {
  std::memset(out, 0, sizeof(*out));
  out->n_bonds = m->n_bonds;
  out->n_sites = m->n_sites;
  double q = 0.0;
  for (int b = 0; b < m->n_bonds; ++b) {
    out->mask[b] = (1ull << m->bi[b]) | (1ull << m->bj[b]);
    out->J[b] = m->J[b];
    q += 0.25 * m->J[b];
  }
  out->J_quarter_sum = q;
  // groups of equal couplings, in order of first appearance
  std::vector<double> vals;
  std::vector<int> gid(m->n_bonds);
  for (int b = 0; b < m->n_bonds; ++b) {
    int g = -1;
    for (size_t v = 0; v < vals.size(); ++v)
      if (vals[v] == m->J[b]) g = (int)v;
    if (g < 0) {
      g = (int)vals.size();
      vals.push_back(m->J[b]);
    }
    gid[b] = g;
  }
  int64_t tsize = 1;
  for (size_t g = 0; g < vals.size(); ++g) {
    int cnt = 0;
    for (int b = 0; b < m->n_bonds; ++b) cnt += gid[b] == (int)g;
    tsize *= (cnt + 1);
  }
  for (int b = 0; b < m->n_bonds; ++b) out->order[b] = (uint8_t)b;
  if (vals.size() > (size_t)kMaxGroups || tsize > kMaxDiagTable || m->n_bonds == 0) {
    out->n_groups = 0;
    out->table_size = 0;
    return;
  }
  out->n_groups = (int32_t)vals.size();
  int k = 0, stride = 1;
  for (int g = 0; g < out->n_groups; ++g) {
    out->gstart[g] = k;
    out->tstride[g] = stride;
    out->gJ[g] = vals[g];
    for (int b = 0; b < m->n_bonds; ++b)
      if (gid[b] == g) out->order[k++] = (uint8_t)b;
    stride *= (k - out->gstart[g]) + 1;
  }
  out->gstart[out->n_groups] = k;
  out->table_size = stride;
}

void fill_pass_masks(BondsDev *b, int G) {
  b->G = G;
  b->n_pass = G >= 2 ? (b->n_bonds + G - 1) / G : 0;
  std::memset(b->pmask, 0, sizeof(b->pmask));
  if (G < 2 || b->n_groups == 0) return;
  for (int g = 0; g < b->n_groups; ++g)
    for (int k = b->gstart[g]; k < b->gstart[g + 1]; ++k) {
      const int bond = b->order[k];
      b->pmask[bond / G][g] |= 1u << (bond % G);
    }
}

size_t tables_bytes(const Plan &p) {
  return align256(p.lo_rank.size() * 4) + align256(p.hi_rank.size() * 4) +
         align256(p.lo_list.size() * 4) + align256(p.lo_start.size() * 4) +
         align256(p.hb_hi.size() * 4) + align256(p.hb_off.size() * 4) +
         align256(p.tiles.size() * sizeof(Tile)) +
         align256((size_t)p.n_sectors * sizeof(SectorDev)) +
         2 * align256((size_t)p.n_sectors * 4) + 256 * 8;
}

namespace {
template <typename T>
int put(Arena &a, const std::vector<T> &v, cudaStream_t s, const T **out) {
  size_t n = std::max<size_t>(v.size(), 1);
  T *d = a.take<T>(n);
  KPM_REQUIRE(d != nullptr, KPM_ENOMEM, "workspace too small for the basis tables");
  if (!v.empty()) KPM_CUDA(cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  *out = d;
  return KPM_OK;
}
}  // namespace

int upload_tables(const Plan &p, const std::vector<SectorDev> &sectors, Arena &arena,
                  cudaStream_t s, TablesDev *t) {
  KPM_TRY(put(arena, p.lo_rank, s, &t->lo_rank));
  KPM_TRY(put(arena, p.hi_rank, s, &t->hi_rank));
  KPM_TRY(put(arena, p.lo_list, s, &t->lo_list));
  KPM_TRY(put(arena, p.lo_start, s, &t->lo_start));
  KPM_TRY(put(arena, p.hb_hi, s, &t->hb_hi));
  KPM_TRY(put(arena, p.hb_off, s, &t->hb_off));
  KPM_TRY(put(arena, p.tiles, s, &t->tiles));
  KPM_TRY(put(arena, sectors, s, &t->sectors));
  KPM_TRY(put(arena, p.tile_begin, s, &t->tile_begin));
  KPM_TRY(put(arena, p.tile_end, s, &t->tile_end));
  t->n_tiles = (int32_t)p.tiles.size();
  t->n_sectors = p.n_sectors;
  t->N = p.N;
  t->L = p.L;
  t->H = p.H;
  t->pad = 0;
  return KPM_OK;
}

int Workspace::acquire(void *user, size_t user_bytes, size_t need, cudaStream_t s) {
  stream = s;
  if (user != nullptr) {
    KPM_REQUIRE(user_bytes >= need, KPM_ENOMEM, "workspace of %zu bytes, need %zu", user_bytes,
                need);
    KPM_REQUIRE(((uintptr_t)user & 255) == 0, KPM_EINVAL, "workspace not 256-byte aligned");
    ptr = user;
    size = user_bytes;
    owned = false;
    return KPM_OK;
  }
  size_t free_b = 0, total_b = 0;
  KPM_CUDA(cudaMemGetInfo(&free_b, &total_b));
  KPM_REQUIRE(need <= free_b, KPM_ENOMEM, "need %zu bytes of device memory, %zu free", need,
              free_b);
  KPM_CUDA(cudaMallocAsync(&ptr, need, s));
  size = need;
  owned = true;
  return KPM_OK;
}

Workspace::~Workspace() {
  if (owned && ptr) {
    cudaFreeAsync(ptr, stream);
    cudaStreamSynchronize(stream);
  }
}

int make_layout(int R, int precision, RowLayout *o) {
  KPM_REQUIRE(precision == KPM_FP64 || precision == KPM_FP32, KPM_EINVAL, "precision %d",
              precision);
  KPM_REQUIRE(R >= 1, KPM_EINVAL, "R = %d < 1", R);
  o->R = R;
  o->vec_width = precision == KPM_FP32 ? 4 : 2;
  o->elem = precision == KPM_FP32 ? 4 : 8;
  o->chunks = (R + o->vec_width - 1) / o->vec_width;
  KPM_REQUIRE(R <= 512, KPM_EINVAL, "R = %d too large (max 512)", R);
  o->cpl = (o->chunks + 31) / 32;
#ifdef KPM_MIN_CPL
  if (o->chunks >= 2 * KPM_MIN_CPL && o->cpl < KPM_MIN_CPL) o->cpl = KPM_MIN_CPL;
#endif
  if (o->cpl > 4) o->cpl = 8;  // chunks-per-lane layouts: 1, 2, 3, 4, 8
  o->G = (o->chunks + o->cpl - 1) / o->cpl;
  o->gpw = 32 / o->G;
  o->Rp = o->G * o->cpl * o->vec_width;
  return KPM_OK;
}

namespace {
std::atomic<long long> g_launches{0};
std::atomic<bool> g_profiling{false};
std::mutex g_prof_mutex;
std::vector<std::pair<cudaEvent_t, cudaEvent_t>> g_events;
}  // namespace

void count_launches(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool profiling() { return g_profiling.load(std::memory_order_relaxed); }

void profile_push(cudaEvent_t start, cudaEvent_t stop) {
  std::lock_guard<std::mutex> lock(g_prof_mutex);
  g_events.emplace_back(start, stop);
}

}  // namespace kpm

extern "C" {

int kpm_profile_enable(int32_t on) {
  std::lock_guard<std::mutex> lock(kpm::g_prof_mutex);
  if (on) {
    for (auto &e : kpm::g_events) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    kpm::g_events.clear();
  }
  kpm::g_profiling.store(on != 0);
  return KPM_OK;
}

int kpm_profile_read(double *step_ms_total, int64_t *step_launches, int64_t *kernel_launches) {
  std::lock_guard<std::mutex> lock(kpm::g_prof_mutex);
  double total = 0.0;
  int rc = KPM_OK;
  for (auto &e : kpm::g_events) {
    float ms = 0.f;
    if (cudaEventSynchronize(e.second) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e.first, e.second) != cudaSuccess)
      rc = KPM_ECUDA;
    total += ms;
    cudaEventDestroy(e.first);
    cudaEventDestroy(e.second);
  }
  if (step_ms_total) *step_ms_total = total;
  if (step_launches) *step_launches = (int64_t)kpm::g_events.size();
  if (kernel_launches) *kernel_launches = kpm::g_launches.load();
  kpm::g_events.clear();
  if (rc != KPM_OK) kpm::set_error("kpm_profile_read: event query failed");
  return rc;
}

int kpm_version(void) { return KPM_VERSION; }

const char *kpm_last_error(void) { return kpm::last_error(); }

int64_t kpm_sector_dim(int32_t n_sites, int32_t n_up) {
  if (n_sites < 1 || n_sites > kpm::kMaxSites || n_up < -1 || n_up > n_sites) return -1;
  return n_up < 0 ? ((int64_t)1 << n_sites) : kpm::binom(n_sites, n_up);
}

}  // extern "C"
