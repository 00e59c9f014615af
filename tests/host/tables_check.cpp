// Host check of the table builder (tables.cpp), built with AddressSanitizer
// and UndefinedBehaviorSanitizer: for a lattice given on stdin and every
// particle number, the spin basis, the combinadic ranks, the connection
// table with its padded rows and warp-tiled ELL, the apply's CTA order and
// the c / c+ maps are built and checked against their definitions.  Prints
// "ok <checks>" or the first violated invariant.
//   stdin: Ns n_bonds, then n_bonds lines "p q t dx dy dz"
#include <algorithm>
#include <cstdio>
#include <map>
#include <vector>

#include "tables.h"

static int g_checks = 0;
#define REQUIRE(c, ...)                          \
  do {                                           \
    ++g_checks;                                  \
    if (!(c)) {                                  \
      std::printf("fail: " __VA_ARGS__);         \
      std::printf("\n");                         \
      return 1;                                  \
    }                                            \
  } while (0)

static int popc(uint32_t x) { return __builtin_popcount(x); }

int main() {
  int Ns, nb;
  if (std::scanf("%d %d", &Ns, &nb) != 2) return 2;
  std::vector<int32_t> p(nb), q(nb);
  std::vector<double> t(nb), d(3 * nb);
  for (int b = 0; b < nb; ++b)
    if (std::scanf("%d %d %lf %lf %lf %lf", &p[b], &q[b], &t[b], &d[3 * b], &d[3 * b + 1],
                   &d[3 * b + 2]) != 6)
      return 2;
  ed::LatticeHost L;
  const std::string err = ed::make_lattice(L, Ns, nb, p.data(), q.data(), t.data(), d.data(),
                                           2.0, nullptr);
  REQUIRE(err.empty(), "make_lattice: %s", err.c_str());
  const int ng = 2 * L.n_classes;
  for (int n = 0; n <= Ns; ++n) {
    const std::vector<uint32_t> words = ed::spin_basis(Ns, n);
    REQUIRE(words.size() == ed::binomial(Ns, n), "basis size n=%d", n);
    for (size_t i = 0; i < words.size(); ++i) {
      REQUIRE(popc(words[i]) == n && (words[i] >> Ns) == 0, "basis word n=%d i=%zu", n, i);
      REQUIRE(i == 0 || words[i - 1] < words[i], "basis order n=%d i=%zu", n, i);
      REQUIRE(ed::combinadic_rank(words[i]) == i, "rank n=%d i=%zu", n, i);
    }
    const ed::SpinTable T = ed::build_spin_table(L, n);
    const int dim = T.dim;
    REQUIRE(dim == (int)words.size() && (int)T.off.size() == dim + 1, "table size n=%d", n);
    // every entry is a hop along a bond into the target row, with the
    // Jordan-Wigner sign of the sites strictly between p and q
    std::map<std::pair<int, int>, int> hops;   // (target, source) -> count
    for (int r = 0; r < dim; ++r) {
      REQUIRE(T.off[r] <= T.off[r + 1], "off monotone n=%d r=%d", n, r);
      for (int e = T.off[r]; e < T.off[r + 1]; ++e) {
        const uint32_t en = T.ent[e];
        const int src = (int)(en & 0xFFFFu), g = (int)((en >> 16) & 0xFFu);
        REQUIRE(src < dim && g < ng, "entry range n=%d r=%d", n, r);
        const uint32_t diff = words[r] ^ words[src];
        REQUIRE(popc(diff) == 2, "entry is one hop n=%d r=%d", n, r);
        bool found = false;
        for (int b = 0; b < nb && !found; ++b) {
          if (L.bond_class[b] != g / 2) continue;
          const int from = (g & 1) ? q[b] : p[b], to = (g & 1) ? p[b] : q[b];
          if (diff != ((1u << from) | (1u << to))) continue;
          if (!((words[src] >> from) & 1u) || ((words[src] >> to) & 1u)) continue;
          const int lo = std::min(from, to), hi = std::max(from, to);
          const uint32_t between = ((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u);
          const uint32_t neg = (uint32_t)(popc(words[src] & between) & 1);
          found = (en >> 31) == neg;
        }
        REQUIRE(found, "entry matches a bond hop with its sign n=%d r=%d e=%d", n, r, e);
        hops[{r, src}] += 1;
      }
    }
    // and every hop of every bond is present
    int nhops = 0;
    for (int b = 0; b < nb; ++b)
      for (int x = 0; x < dim; ++x)
        for (int dir = 0; dir < 2; ++dir) {
          const int from = dir ? q[b] : p[b], to = dir ? p[b] : q[b];
          if (!((words[x] >> from) & 1u) || ((words[x] >> to) & 1u)) continue;
          ++nhops;
        }
    REQUIRE(nhops == T.off[dim], "hop count n=%d: %d vs %d", n, nhops, T.off[dim]);
    // padded rows: multiples of 4, real entries first in order, padding null
    REQUIRE((int)T.pad_off.size() == dim + 1, "pad_off size n=%d", n);
    for (int r = 0; r < dim; ++r) {
      const int e0 = T.pad_off[r], e1 = T.pad_off[r + 1], len = T.off[r + 1] - T.off[r];
      REQUIRE((e1 - e0) % 4 == 0 && e1 - e0 >= len && e1 - e0 < len + 4, "pad length n=%d r=%d", n, r);
      for (int k = 0; k < e1 - e0; ++k) {
        const uint32_t en = T.pad_ent[e0 + k];
        if (k < len) REQUIRE(en == T.ent[T.off[r] + k], "pad copy n=%d r=%d", n, r);
        else REQUIRE((en & ed::kNullEntry) && (int)(en & 0xFFFFu) == r, "pad null n=%d r=%d", n, r);
      }
    }
    // warp-tiled ELL: every column's slot entries are its CSR entries (same
    // rank and sign), the rest point at the zero columns dim .. dim + 7
    auto check_ell = [&](const ed::SpinTable& T) -> int {
    const int ntile = (dim + 63) / 64;
    REQUIRE((int)T.tslot_off.size() == ntile + 1, "tslot_off size n=%d", n);
    for (int c = 0; c < ntile; ++c) {
      const int s0 = T.tslot_off[c], s1 = T.tslot_off[c + 1];
      REQUIRE((s1 - s0) % 2 == 0 && s0 <= s1, "tile slots even n=%d c=%d", n, c);
      for (int l = 0; l < 32; ++l)
        for (int h = 0; h < 2; ++h) {
          const int col = 64 * c + 2 * l + h;
          std::vector<std::pair<uint32_t, uint32_t>> got, want;
          for (int s = s0; s < s1; ++s) {
            REQUIRE((size_t)(2 * (s * 32 + l) + h) < T.ell.size(), "ell index n=%d", n);
            const uint32_t en = T.ell[2 * (s * 32 + l) + h];
            const uint32_t rank = (en & 0x7FFFFFFFu) >> 5;
            REQUIRE((en & 0x7FFFFFFFu) == ed::tile_offset(rank), "ell offset form n=%d", n);
            REQUIRE(rank < (uint32_t)dim + ed::kZeroCols, "ell rank range n=%d", n);
            if (rank < (uint32_t)dim) got.push_back({rank, en >> 31});
          }
          if (col < dim)
            for (int e = T.off[col]; e < T.off[col + 1]; ++e)
              want.push_back({T.ent[e] & 0xFFFFu, T.ent[e] >> 31});
          std::sort(got.begin(), got.end());
          std::sort(want.begin(), want.end());
          REQUIRE(got == want, "ell column n=%d col=%d", n, col);
        }
    }
    return 0;
    };
    if (check_ell(T)) return 1;
    // hop order: a permutation of the basis whose table is the ascending
    // one relabelled (same hops, groups and signs), with its own ELL; the
    // tile search takes seconds under the sanitizers past a few thousand
    // columns, so the largest bases (Ns=16 near half filling) skip it here
    if (dim <= 4000) {
    const ed::SpinTable H = ed::build_spin_table(L, n, true);
    REQUIRE(H.dim == dim && (int)H.order.size() == dim, "hop table size n=%d", n);
    {
      std::vector<int> seen(dim, 0);
      for (int i = 0; i < dim; ++i) {
        const int o = H.order[i];
        REQUIRE(o >= 0 && o < dim && !seen[o], "hop order permutation n=%d", n);
        seen[o] = 1;
        REQUIRE(H.words[i] == words[o], "hop order words n=%d i=%d", n, i);
      }
      for (int i = 0; i < dim; ++i) {
        std::vector<uint32_t> a, b;
        for (int e = H.off[i]; e < H.off[i + 1]; ++e)
          a.push_back(((uint32_t)H.order[H.ent[e] & 0xFFFFu]) | (H.ent[e] & 0xFFFF0000u));
        const int o = H.order[i];
        for (int e = T.off[o]; e < T.off[o + 1]; ++e) b.push_back(T.ent[e]);
        std::sort(a.begin(), a.end());
        std::sort(b.begin(), b.end());
        REQUIRE(a == b, "hop order row n=%d i=%d", n, i);
      }
      // the 64-column tiles hold the columns of the order sorted by
      // decreasing per-group hop counts (the columns of a tile may come in
      // any order): sorted within each tile, the keys do not increase
      std::vector<std::vector<int>> keys(dim, std::vector<int>(ng, 0));
      for (int i = 0; i < dim; ++i)
        for (int e = H.off[i]; e < H.off[i + 1]; ++e) keys[i][(H.ent[e] >> 16) & 0xFFu]++;
      for (int t0 = 0; t0 < dim; t0 += 64)
        std::sort(keys.begin() + t0, keys.begin() + std::min(dim, t0 + 64),
                  [](const std::vector<int>& x, const std::vector<int>& y) { return y < x; });
      for (int i = 1; i < dim; ++i)
        REQUIRE(!(keys[i - 1] < keys[i]), "hop order keys n=%d i=%d", n, i);
    }
    if (check_ell(H)) return 1;
    }
    // CTA order: a permutation of the rows
    const std::vector<int> order = ed::block_order(T, 1);
    std::vector<int> seen(dim, 0);
    REQUIRE((int)order.size() == dim, "order size n=%d", n);
    for (int r : order) {
      REQUIRE(r >= 0 && r < dim && !seen[r], "order permutation n=%d", n);
      seen[r] = 1;
    }
    // c / c+ maps into n - 1 and n + 1 (spin 0 and 1, every site)
    for (int site = 0; site < Ns; ++site)
      for (int spin = 0; spin < 2; ++spin)
        for (int create = 0; create < 2; ++create) {
          const int nd = create ? n + 1 : n - 1;
          if (nd < 0 || nd > Ns) continue;
          const int n_up = spin == 0 ? n : 1, n_dn = spin == 0 ? 1 : n;
          if (n_up > Ns || n_dn > Ns) continue;
          const std::vector<int32_t> m = ed::fermion_map(Ns, n_up, n_dn, site, spin, create != 0);
          const std::vector<uint32_t> dst = ed::spin_basis(Ns, nd);
          REQUIRE(m.size() == dst.size(), "map size n=%d", n);
          for (size_t k = 0; k < m.size(); ++k) {
            if (m[k] == 0x7FFFFFFF) {
              REQUIRE(((dst[k] >> site) & 1u) == (create ? 0u : 1u), "map hole n=%d", n);
              continue;
            }
            const uint32_t src = (uint32_t)m[k] & 0x7FFFFFFFu;
            REQUIRE(src < words.size(), "map source range n=%d", n);
            REQUIRE((words[src] ^ dst[k]) == (1u << site), "map source word n=%d", n);
          }
        }
  }
  // coefficients: conjugate pairs of modulus t
  std::vector<double> cf(2 * ng);
  const double A[3] = {0.37, -0.21, 0.11};
  ed::group_coefficients(L, A, cf.data());
  for (int c = 0; c < L.n_classes; ++c) {
    REQUIRE(cf[4 * c] == cf[4 * c + 2] && cf[4 * c + 1] == -cf[4 * c + 3], "conjugate pair %d", c);
  }
  std::printf("ok %d\n", g_checks);
  return 0;
}
