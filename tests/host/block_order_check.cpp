// Host check of the apply's CTA order: builds the up-spin table of a
// lattice given on stdin, takes the rows in ed::block_order(T, 1) order and
// groups nr consecutive ones per CTA (as the engine does), and prints per nr
// whether every row appears once and, for windows of a quarter of the CTAs
// taken consecutively (the CTAs resident together), the mean fraction of
// all rows their rows gather from, in natural and in this order.
//   stdin: Ns n n_bonds, then n_bonds lines "p q t dx dy dz", then the nr list
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "tables.h"

int main() {
  int Ns, n, nb;
  if (std::scanf("%d %d %d", &Ns, &n, &nb) != 3) return 2;
  std::vector<int32_t> p(nb), q(nb);
  std::vector<double> t(nb), d(3 * nb);
  for (int b = 0; b < nb; ++b)
    if (std::scanf("%d %d %lf %lf %lf %lf", &p[b], &q[b], &t[b], &d[3 * b], &d[3 * b + 1],
                   &d[3 * b + 2]) != 6)
      return 2;
  ed::LatticeHost L;
  if (!ed::make_lattice(L, Ns, nb, p.data(), q.data(), t.data(), d.data(), 1.0, nullptr).empty())
    return 3;
  const ed::SpinTable T = ed::build_spin_table(L, n);
  int nr;
  while (std::scanf("%d", &nr) == 1) {
    const int nblk = (T.dim + nr - 1) / nr;
    const std::vector<int> rows = ed::block_order(T, 1);
    std::vector<int> seen(T.dim, 0);
    bool perm = (int)rows.size() == T.dim;
    for (int i = 0; perm && i < (int)rows.size(); ++i) {
      if (rows[i] < 0 || rows[i] >= T.dim || seen[rows[i]]) perm = false;
      else seen[rows[i]] = 1;
    }
    // mean over windows (start step W/4) of |sources of the window| / dim,
    // CTA b holding rows order[b*nr .. b*nr + nr)
    auto window_union = [&](const std::vector<int>& order) {
      const int W = std::max(1, nblk / 4);
      const int step = std::max(1, W / 4);
      double sum = 0.0;
      int cnt = 0;
      std::vector<int> mark(T.dim, -1);
      for (int s0 = 0; s0 + W <= nblk; s0 += step, ++cnt) {
        int u = 0;
        for (int i = s0 * nr; i < std::min(T.dim, (s0 + W) * nr); ++i) {
          const int r = order[i];
          for (int e = T.off[r]; e < T.off[r + 1]; ++e) {
            const int src = (int)(T.ent[e] & 0xFFFFu);
            if (mark[src] != s0) { mark[src] = s0; ++u; }
          }
        }
        sum += (double)u / T.dim;
      }
      return cnt ? sum / cnt : 0.0;
    };
    double u_nat = 0.0, u_ord = 0.0;
    if (perm) {
      std::vector<int> nat(T.dim);
      for (int r = 0; r < T.dim; ++r) nat[r] = r;
      u_nat = window_union(nat);
      u_ord = window_union(rows);
    }
    std::printf("%d %d %d %.6f %.6f\n", nr, nblk, perm ? 1 : 0, u_nat, u_ord);
  }
  return 0;
}
