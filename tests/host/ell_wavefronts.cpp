// Shared-memory wavefronts of the down-spin gathers of the apply (T_dn
// through the warp-tiled ELL of tables.cpp), replayed on the host for one
// spin table: every (slot, h, quarter warp) of every 64-column tile is one
// 16-byte load per lane of 8 lanes, which costs as many wavefronts as the
// most distinct sources it reads in one 16-byte bank group (rank mod 8), at
// least one (the rule the hardware follows: the shared-load pattern probe of
// libed_probes, ed_probe_shared_loads, measured one wavefront per quarter
// warp without conflicts and one more per extra distinct address in a bank
// group of that quarter).  Reads "Ns n_bonds n" and the bonds from stdin
// (p q t dx dy dz per line), prints the ratio of the replayed wavefronts to
// one per quarter warp for the ascending-order and the hop-ordered table:
//   ascending <ratio> hop <ratio> slots_asc <per tile> slots_hop <per tile>
#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include "tables.h"

static void replay(const ed::SpinTable& T, double* ratio, double* slots_per_tile) {
  const int ntile = (T.dim + 63) / 64;
  long wf = 0, quarters = 0, slots = 0;
  for (int c = 0; c < ntile; ++c)
    for (int s = T.tslot_off[c]; s < T.tslot_off[c + 1]; ++s) {
      ++slots;
      for (int h = 0; h < 2; ++h)
        for (int ph = 0; ph < 4; ++ph) {
          std::vector<uint32_t> u;
          for (int i = 0; i < 8; ++i)
            u.push_back((T.ell[(size_t)s * 64 + 2 * (8 * ph + i) + h] & 0x7FFFFFFFu) >> 5);
          std::sort(u.begin(), u.end());
          u.erase(std::unique(u.begin(), u.end()), u.end());
          int cnt[8] = {0};
          for (uint32_t r : u) cnt[r & 7u]++;
          wf += std::max(1, *std::max_element(cnt, cnt + 8));
          ++quarters;
        }
    }
  *ratio = quarters ? (double)wf / (double)quarters : 1.0;
  *slots_per_tile = ntile ? (double)slots / ntile : 0.0;
}

int main() {
  int Ns, nb, n;
  if (std::scanf("%d %d %d", &Ns, &nb, &n) != 3) return 2;
  std::vector<int32_t> p(nb), q(nb);
  std::vector<double> t(nb), d(3 * nb);
  for (int b = 0; b < nb; ++b)
    if (std::scanf("%d %d %lf %lf %lf %lf", &p[b], &q[b], &t[b], &d[3 * b], &d[3 * b + 1],
                   &d[3 * b + 2]) != 6)
      return 2;
  ed::LatticeHost L;
  const std::string err = ed::make_lattice(L, Ns, nb, p.data(), q.data(), t.data(), d.data(),
                                           8.0, nullptr);
  if (!err.empty()) {
    std::printf("fail: %s\n", err.c_str());
    return 1;
  }
  double ra, rh, sa, sh;
  replay(ed::build_spin_table(L, n, false), &ra, &sa);
  replay(ed::build_spin_table(L, n, true), &rh, &sh);
  std::printf("ascending %.4f hop %.4f slots_asc %.3f slots_hop %.3f\n", ra, rh, sa, sh);
  return 0;
}
