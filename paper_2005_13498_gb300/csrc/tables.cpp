// Basis enumeration, combinadic ranks, connection tables, sector maps.
#include "tables.h"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace ed {

uint64_t binomial(int n, int k) {
  if (k < 0 || k > n) return 0;
  uint64_t r = 1;
  for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;
  return r;
}

static int popc(uint32_t x) { return __builtin_popcount(x); }

std::vector<uint32_t> spin_basis(int Ns, int n) {
  std::vector<uint32_t> out;
  out.reserve((size_t)binomial(Ns, n));
  if (n == 0) {
    out.push_back(0u);
    return out;
  }
  // next word with the same popcount (lowest-set-bit carry), ascending
  uint32_t w = (n >= 32) ? 0xFFFFFFFFu : ((1u << n) - 1u);
  const uint64_t limit = 1ull << Ns;
  while ((uint64_t)w < limit) {
    out.push_back(w);
    const uint32_t low = w & (0u - w);
    const uint32_t ripple = w + low;
    if (ripple == 0u) break;
    const uint32_t ones = ((ripple ^ w) >> 2) / low;
    w = ripple | ones;
  }
  return out;
}

uint32_t combinadic_rank(uint32_t word) {
  uint32_t r = 0;
  int k = 1;
  while (word) {
    const int pos = __builtin_ctz(word);
    r += (uint32_t)binomial(pos, k);
    ++k;
    word &= word - 1;
  }
  return r;
}

std::string make_lattice(LatticeHost& L, int Ns, int n_bonds, const int32_t* p,
                         const int32_t* q, const double* t, const double* d,
                         double U, const double* eps) {
  if (n_bonds < 0) return "n_bonds < 0";
  if (n_bonds > 0 && (!p || !q || !t || !d)) return "bond arrays must not be NULL";
  if (!std::isfinite(U)) return "U is not finite";
  L = LatticeHost();
  L.Ns = Ns;
  L.n_bonds = n_bonds;
  L.U = U;
  for (int b = 0; b < n_bonds; ++b) {
    if (p[b] < 0 || p[b] >= Ns || q[b] < 0 || q[b] >= Ns)
      return "bond " + std::to_string(b) + ": site index out of range";
    if (p[b] == q[b]) return "bond " + std::to_string(b) + ": p == q";
    if (!std::isfinite(t[b]) || !std::isfinite(d[3 * b]) ||
        !std::isfinite(d[3 * b + 1]) || !std::isfinite(d[3 * b + 2]))
      return "bond " + std::to_string(b) + ": non-finite value";
    L.p.push_back(p[b]);
    L.q.push_back(q[b]);
    L.t.push_back(t[b]);
    for (int k = 0; k < 3; ++k) L.d.push_back(d[3 * b + k]);
  }
  if (eps) {
    L.has_eps = true;
    for (int i = 0; i < Ns; ++i) {
      if (!std::isfinite(eps[i])) return "eps is not finite";
      L.eps.push_back(eps[i]);
    }
  }
  // bond classes: identical (t, d) <=> identical coefficient at every A
  for (int b = 0; b < n_bonds; ++b) {
    int c = -1;
    for (int k = 0; k < L.n_classes; ++k) {
      if (L.class_t[k] == L.t[b] && L.class_d[3 * k] == L.d[3 * b] &&
          L.class_d[3 * k + 1] == L.d[3 * b + 1] && L.class_d[3 * k + 2] == L.d[3 * b + 2]) {
        c = k;
        break;
      }
    }
    if (c < 0) {
      c = L.n_classes++;
      L.class_t.push_back(L.t[b]);
      for (int k = 0; k < 3; ++k) L.class_d.push_back(L.d[3 * b + k]);
    }
    L.bond_class.push_back(c);
  }
  if (2 * L.n_classes > 256) return "more than 128 distinct bond classes";
  return "";
}

// Distributes the entries of 64 column lists (column l = 2 * lane + h) over
// K slots, each list in its own column of the slots, so that the loads one
// gather instruction makes (one slot, one h, 32 lanes) are spread over the
// shared-memory banks.  The hardware serves a 16-byte-per-lane load a quarter
// warp (8 lanes) at a time; sources of distinct rank mod 8 fall in distinct
// 16-byte bank groups (16-byte columns: rank mod 8; 32-byte swizzled
// columns: 2 (rank mod 4) + bit 2 of rank, also a bijection of rank mod 8),
// and equal ranks are a broadcast.  Greedy, slot by slot: within each quarter
// warp the lanes with the longest remaining lists choose first, each taking
// the entry that adds the fewest conflicts; a lane with slack (fewer entries
// left than slots) leaves the slot empty rather than add a conflict.  An
// empty lane reads one of the eight zero columns dim .. dim + 7, the same one
// for every empty lane of the quarter warp (a broadcast), picked in a bank
// group the quarter warp's real entries leave free, so empty slots need no
// test in the kernel.  Returns [K][64] entries (rank | sign << 31).
static std::vector<uint32_t> assign_slots(std::vector<std::vector<uint32_t>> lists, int K,
                                          uint32_t dim) {
  std::vector<uint32_t> out((size_t)K * 64, kEllNull);
  for (int k = 0; k < K; ++k) {
    const int slack = K - k;
    for (int h = 0; h < 2; ++h) {
      for (int ph = 0; ph < 4; ++ph) {
        int cols[8];
        for (int i = 0; i < 8; ++i) cols[i] = 2 * (8 * ph + i) + h;
        std::stable_sort(cols, cols + 8, [&](int a, int b) {
          return lists[a].size() > lists[b].size();
        });
        std::vector<uint32_t> used;   // ranks already read in this quarter warp
        auto cost = [&](uint32_t rank) {
          int n = 0;
          for (uint32_t r : used)
            if (r != rank && (r & 7u) == (rank & 7u)) ++n;
          return n;
        };
        for (int i = 0; i < 8; ++i) {
          std::vector<uint32_t>& L = lists[cols[i]];
          if (L.empty()) continue;
          size_t best = 0;
          int bc = cost(L[0] & 0xFFFFu);
          for (size_t j = 1; j < L.size() && bc > 0; ++j) {
            const int cj = cost(L[j] & 0xFFFFu);
            if (cj < bc) { bc = cj; best = j; }
          }
          if (bc > 0 && (int)L.size() < slack) continue;   // wait for a later slot
          out[(size_t)k * 64 + cols[i]] = L[best];
          used.push_back(L[best] & 0xFFFFu);
          L.erase(L.begin() + best);
        }
        // the zero column for this quarter warp's empty lanes
        uint32_t zero = dim;
        for (uint32_t z = 0; z < 8; ++z) {
          bool free_bank = true;
          for (uint32_t r : used)
            if ((r & 7u) == ((dim + z) & 7u)) free_bank = false;
          if (free_bank) { zero = dim + z; break; }
        }
        for (int i = 0; i < 8; ++i)
          if (out[(size_t)k * 64 + cols[i]] == kEllNull) out[(size_t)k * 64 + cols[i]] = zero;
      }
    }
  }
  return out;
}

SpinTable build_spin_table(const LatticeHost& L, int n, bool hop_order) {
  SpinTable T;
  T.n = n;
  T.words = spin_basis(L.Ns, n);
  T.dim = (int)T.words.size();
  T.order.resize(T.dim);
  for (int i = 0; i < T.dim; ++i) T.order[i] = i;
  // pos[rank]: position of the state of that ascending-word rank
  std::vector<uint32_t> pos(T.dim);
  for (int i = 0; i < T.dim; ++i) pos[i] = (uint32_t)i;
  if (hop_order) {
    const int ngrp = 2 * L.n_classes;
    std::vector<int32_t> key((size_t)T.dim * ngrp, 0);   // hops into each state, per group
    for (int r = 0; r < T.dim; ++r) {
      const uint32_t y = T.words[r];
      for (int b = 0; b < L.n_bonds; ++b) {
        const uint32_t bp = 1u << L.p[b], bq = 1u << L.q[b];
        if ((y & bq) && !(y & bp)) key[(size_t)r * ngrp + 2 * L.bond_class[b]]++;
        if ((y & bp) && !(y & bq)) key[(size_t)r * ngrp + 2 * L.bond_class[b] + 1]++;
      }
    }
    std::stable_sort(T.order.begin(), T.order.end(), [&](int a, int b) {
      return std::lexicographical_compare(key.begin() + (size_t)b * ngrp,
                                          key.begin() + (size_t)(b + 1) * ngrp,
                                          key.begin() + (size_t)a * ngrp,
                                          key.begin() + (size_t)(a + 1) * ngrp);
    });
    std::vector<uint32_t> w(T.dim);
    for (int i = 0; i < T.dim; ++i) {
      w[i] = T.words[T.order[i]];
      pos[T.order[i]] = (uint32_t)i;
    }
    T.words = w;
  }
  T.off.assign(T.dim + 1, 0);
  struct E { uint32_t group, src, neg; };
  std::vector<E> row;
  for (int r = 0; r < T.dim; ++r) {
    const uint32_t y = T.words[r];
    row.clear();
    for (int b = 0; b < L.n_bonds; ++b) {
      const int p = L.p[b], q = L.q[b];
      const uint32_t bp = 1u << p, bq = 1u << q;
      const int lo = std::min(p, q), hi = std::max(p, q);
      const uint32_t between = ((1u << hi) - 1u) & ~((1u << (lo + 1)) - 1u);
      const uint32_t neg = (uint32_t)(popc(y & between) & 1);
      // orientation 0: hop p -> q produced y (q set, p clear in y)
      if ((y & bq) && !(y & bp))
        row.push_back({(uint32_t)(2 * L.bond_class[b]), pos[combinadic_rank(y ^ bp ^ bq)], neg});
      // orientation 1: hop q -> p produced y (p set, q clear in y)
      if ((y & bp) && !(y & bq))
        row.push_back({(uint32_t)(2 * L.bond_class[b] + 1), pos[combinadic_rank(y ^ bp ^ bq)], neg});
    }
    std::sort(row.begin(), row.end(), [](const E& a, const E& b) {
      return a.group != b.group ? a.group < b.group : a.src < b.src;
    });
    for (const E& e : row)
      T.ent.push_back((e.src & 0xFFFFu) | (e.group << 16) | (e.neg << 31));
    T.off[r + 1] = (int32_t)T.ent.size();
  }
  // rows padded to a multiple of 4 entries
  T.pad_off.assign(T.dim + 1, 0);
  for (int r = 0; r < T.dim; ++r) {
    const int n = T.off[r + 1] - T.off[r];
    for (int e = T.off[r]; e < T.off[r + 1]; ++e) T.pad_ent.push_back(T.ent[e]);
    if (n > 0) {
      const uint32_t last_group = T.ent[T.off[r + 1] - 1] & (0xFFu << 16);
      for (int k = n; k % 4 != 0; ++k)
        T.pad_ent.push_back((uint32_t)r | last_group | kNullEntry);
    }
    T.pad_off[r + 1] = (int32_t)T.pad_ent.size();
  }
  // warp-tiled ELL over columns (tiles of 64, two columns per lane), flat
  // slot list per tile grouped by bond group, padded to an even slot count
  const int ntile = (T.dim + 63) / 64;
  T.tslot_off.assign(ntile + 1, 0);
  int nslots = 0;
  for (int c = 0; c < ntile; ++c) {
    int maxg = -1;
    for (int l = 0; l < 64; ++l) {
      const int d = c * 64 + l;
      if (d >= T.dim) break;
      if (T.off[d + 1] > T.off[d]) maxg = std::max(maxg, (int)((T.ent[T.off[d + 1] - 1] >> 16) & 0xFFu));
    }
    int tile_slots = 0;
    for (int g = 0; g <= maxg; ++g) {
      std::vector<std::vector<uint32_t>> lists(64);   // entries (rank | sign) per column
      int K = 0;
      for (int l = 0; l < 64; ++l) {
        const int d = c * 64 + l;
        if (d >= T.dim) continue;
        for (int e = T.off[d]; e < T.off[d + 1]; ++e)
          if ((int)((T.ent[e] >> 16) & 0xFFu) == g)
            lists[l].push_back((T.ent[e] & 0xFFFFu) | (T.ent[e] & 0x80000000u));
        K = std::max(K, (int)lists[l].size());
      }
      if (K == 0) continue;
      std::vector<uint32_t> slots = assign_slots(lists, K, (uint32_t)T.dim);
      for (int k = 0; k < K; ++k) {
        T.slot_grp.push_back((uint32_t)g);
        for (int l = 0; l < 64; ++l) {   // l = 2 * lane + h
          const uint32_t e = slots[(size_t)k * 64 + l];
          T.ell.push_back(tile_offset(e & 0xFFFFu) | (e & 0x80000000u));
        }
        ++tile_slots;
      }
    }
    if (tile_slots % 2) {   // padding slot: every lane reads zero column dim
      T.slot_grp.push_back(T.slot_grp.empty() ? 0u : T.slot_grp.back());
      for (int l = 0; l < 64; ++l) T.ell.push_back(tile_offset((uint32_t)T.dim));
      ++tile_slots;
    }
    nslots += tile_slots;
    T.tslot_off[c + 1] = nslots;
  }
  if (L.has_eps) {
    T.eps_sum.resize(T.dim);
    for (int r = 0; r < T.dim; ++r) {
      double s = 0.0;
      for (int i = 0; i < L.Ns; ++i)
        if ((T.words[r] >> i) & 1u) s += L.eps[i];
      T.eps_sum[r] = s;
    }
  }
  return T;
}

std::vector<int> block_order(const SpinTable& T, int nr) {
  const int nb = nr > 0 ? (T.dim + nr - 1) / nr : 0;
  std::vector<std::vector<int>> adj(nb);
  for (int r = 0; r < T.dim; ++r)
    for (int e = T.off[r]; e < T.off[r + 1]; ++e) {
      const int b = r / nr, c = (int)(T.ent[e] & kEntRankMask) / nr;
      if (b != c) {
        adj[b].push_back(c);
        adj[c].push_back(b);
      }
    }
  std::vector<int> deg(nb);
  for (int b = 0; b < nb; ++b) {
    std::sort(adj[b].begin(), adj[b].end());
    adj[b].erase(std::unique(adj[b].begin(), adj[b].end()), adj[b].end());
    deg[b] = (int)adj[b].size();
  }
  // Cuthill-McKee: breadth-first from a block of least degree, neighbours
  // visited by increasing degree; repeated for every connected component
  std::vector<int> order;
  order.reserve(nb);
  std::vector<char> seen(nb, 0);
  while ((int)order.size() < nb) {
    int s0 = -1;
    for (int b = 0; b < nb; ++b)
      if (!seen[b] && (s0 < 0 || deg[b] < deg[s0])) s0 = b;
    seen[s0] = 1;
    size_t head = order.size();
    order.push_back(s0);
    while (head < order.size()) {
      const int b = order[head++];
      std::vector<int> nxt;
      for (int c : adj[b])
        if (!seen[c]) {
          seen[c] = 1;
          nxt.push_back(c);
        }
      std::stable_sort(nxt.begin(), nxt.end(), [&](int x, int y) { return deg[x] < deg[y]; });
      order.insert(order.end(), nxt.begin(), nxt.end());
    }
  }
  std::reverse(order.begin(), order.end());
  for (int& b : order) b *= nr;
  return order;
}

void group_coefficients(const LatticeHost& L, const double A[3], double* out) {
  for (int c = 0; c < L.n_classes; ++c) {
    const double phi = A[0] * L.class_d[3 * c] + A[1] * L.class_d[3 * c + 1] +
                       A[2] * L.class_d[3 * c + 2];
    const double tc = L.class_t[c];
    const double cs = std::cos(phi), sn = std::sin(phi);
    // -t exp(-i phi) and -t exp(+i phi)
    out[4 * c + 0] = -tc * cs;
    out[4 * c + 1] = tc * sn;
    out[4 * c + 2] = -tc * cs;
    out[4 * c + 3] = -tc * sn;
  }
}

void pulse_A(int shape, double A0, double omega, double sigma, double t0, double b,
             const double dir[3], double t, double out[3]) {
  const double s = t - t0;
  const double env = std::exp(-s * s / (2.0 * sigma * sigma));
  const double amp = shape == 1 ? -A0 * (std::cos(omega * s) - b) * env
                                : A0 * env * std::sin(omega * s);
  for (int k = 0; k < 3; ++k) out[k] = amp * dir[k];
}

std::vector<int32_t> fermion_map(int Ns, int n_up, int n_dn, int site, int spin,
                                 bool create) {
  const int n_src = spin == 0 ? n_up : n_dn;
  const int n_dst = n_src + (create ? 1 : -1);
  const std::vector<uint32_t> dst_words = spin_basis(Ns, n_dst);
  std::vector<int32_t> map(dst_words.size(), 0x7FFFFFFF);
  const uint32_t bit = 1u << site;
  const uint32_t below = bit - 1u;
  for (size_t t = 0; t < dst_words.size(); ++t) {
    const uint32_t y = dst_words[t];
    // c removes the electron: y lacks the bit; c^+ adds it: y has the bit
    if (create ? !(y & bit) : (y & bit)) continue;
    const uint32_t x = y ^ bit;  // source configuration
    int parity = popc(x & below);
    if (spin == 1) parity += n_up;
    const uint32_t src = combinadic_rank(x);
    map[t] = (int32_t)(src | ((uint32_t)(parity & 1) << 31));
  }
  return map;
}

}  // namespace ed
