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

#include "kernels.cuh"
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
    // the engine's block maps on this order: the apply blocks (nr rows) and
    // the row-gather T_up blocks (kTupRows rows, chunks of 256 pairs of a
    // row of dim_dn = dim columns) cover every row, and every (row, chunk),
    // exactly once
    bool maps_ok = perm;
    if (perm) {
      std::vector<ed::ApplyBlock> map;
      ed::append_apply_blocks(map, 0, T.dim, nr, &rows);
      std::vector<int> cnt(T.dim, 0);
      for (const ed::ApplyBlock& b : map) {
        if (b.nrows < 1 || b.nrows > nr || b.nrows > 4 || b.row0 != b.row[0]) maps_ok = false;
        for (int r = 0; r < b.nrows && maps_ok; ++r) ++cnt[b.row[r]];
      }
      const int npairs = (T.dim + 1) / 2, chunk = 256;
      std::vector<ed::ApplyBlock> tmap;
      for (int pc = 0; pc < npairs; pc += chunk) ed::append_tup_chunk(tmap, 0, T.dim, ed::kTupRows, pc, &rows);
      std::vector<int> tcnt((size_t)T.dim * ((npairs + chunk - 1) / chunk), 0);
      for (const ed::ApplyBlock& b : tmap) {
        if (b.nrows < 1 || b.nrows > ed::kTupRows || b.pc % chunk != 0) { maps_ok = false; break; }
        for (int r = 0; r < b.nrows; ++r) ++tcnt[(size_t)b.row[r] * ((npairs + chunk - 1) / chunk) + b.pc / chunk];
      }
      for (int c : cnt) maps_ok = maps_ok && c == 1;
      for (int c : tcnt) maps_ok = maps_ok && c == 1;
    }
    std::printf("%d %d %d %.6f %.6f %d\n", nr, nblk, perm ? 1 : 0, u_nat, u_ord, maps_ok ? 1 : 0);
  }
  return 0;
}
