// Prints the host-side basis plan (hi-blocks and tiles) and the binomial table
// of libkpm for a few chains and tile sizes, one record per line, so that
// tests/test_plan_host.py can check them against plain combinatorics.
#include <cstdio>
#include <vector>

#include "kpm_internal.h"

int main() {
  for (int n = 0; n <= 64; ++n)
    for (int k = 0; k <= n; ++k) std::printf("binom %d %d %lld\n", n, k, (long long)kpm::binom(n, k));
  for (int N : {1, 2, 5, 8, 11, 14}) {
    std::vector<int32_t> bi, bj;
    std::vector<double> J;
    for (int i = 0; i + 1 < N; ++i) {
      bi.push_back(i);
      bj.push_back(i + 1);
      J.push_back(1.0);
    }
    kpm_model m{N, (int32_t)bi.size(), bi.data(), bj.data(), J.data()};
    std::vector<int32_t> nup;
    for (int k = 0; k <= N; ++k) nup.push_back(k);
    nup.push_back(-1);
    for (long ts : {1L, 3L, 16L, 100L}) {
      kpm::Plan p;
      if (kpm::build_plan(&m, (int)nup.size(), nup.data(), ts, &p) != KPM_OK) {
        std::printf("error %d %ld\n", N, ts);
        continue;
      }
      std::printf("plan %d %ld %d %d\n", N, ts, p.L, p.n_sectors);
      for (int s = 0; s < p.n_sectors; ++s)
        std::printf("sector %d %d %lld %lld %d %d %d\n", s, p.n_up[s], (long long)p.dim[s],
                    (long long)p.row0[s], p.hb_begin[s], p.tile_begin[s], p.tile_end[s]);
      for (size_t b = 0; b < p.hb_hi.size(); ++b) std::printf("block %zu %u %u\n", b, p.hb_hi[b], p.hb_off[b]);
      for (size_t t = 0; t < p.tiles.size(); ++t) {
        const kpm::Tile &x = p.tiles[t];
        std::printf("tile %zu %lld %u %u %u %u %d\n", t, (long long)x.row0, x.rank0, x.count, x.b_first,
                    x.b_last, x.sector);
      }
    }
  }
  for (int gpw : {1, 2, 4, 16})
    for (long rows : {1L, 1000L, 1L << 20, 1L << 26, 3000000000L})
      std::printf("lts %d %ld %lld\n", gpw, rows, (long long)kpm::list_tile_states(gpw, rows));
  return 0;
}
