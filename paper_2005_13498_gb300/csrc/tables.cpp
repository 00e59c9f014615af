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

// One quarter warp and h of assign_slots: the entries of its 8 lanes'
// lists as the edges of a bipartite multigraph (lanes x virtual bank
// groups), coloured with K colours; slot_of[i * maxlen + j] receives the
// colour (slot) of entry j of lane i.
static void colour_quarter(const std::vector<uint32_t>* lists8, int K,
                           std::vector<int>& slot_of /* [8 * maxlen] */, int maxlen) {
  struct Edge { int lane, vb, col; };
  std::vector<Edge> E;
  int occ[8] = {0};
  for (int i = 0; i < 8; ++i)
    for (size_t j = 0; j < lists8[i].size(); ++j) {
      const int b = (int)(lists8[i][j] & 7u);
      E.push_back({i, b + 8 * (occ[b] / K), -1});
      ++occ[b];
    }
  int nv = 0;
  for (const Edge& e : E) nv = std::max(nv, e.vb + 1);
  std::vector<int> atL((size_t)8 * K, -1), atV((size_t)nv * K, -1);
  std::vector<int> path;
  for (int e = 0; e < (int)E.size(); ++e) {
    const int u = E[e].lane, v = E[e].vb;
    int a = -1, b = -1;
    for (int c = 0; c < K && a < 0; ++c)
      if (atL[(size_t)u * K + c] < 0) a = c;
    for (int c = 0; c < K && b < 0; ++c)
      if (atV[(size_t)v * K + c] < 0) b = c;
    if (atV[(size_t)v * K + a] >= 0) {
      // swap colours a and b along the alternating path that leaves v by
      // its a edge; it cannot reach u (a is free there), and afterwards a
      // is free at v
      path.clear();
      int node = v, c = a;
      bool right = true;
      for (;;) {
        const int f = right ? atV[(size_t)node * K + c] : atL[(size_t)node * K + c];
        if (f < 0) break;
        path.push_back(f);
        node = right ? E[f].lane : E[f].vb;
        right = !right;
        c = c == a ? b : a;
      }
      for (int f : path) {
        atL[(size_t)E[f].lane * K + E[f].col] = -1;
        atV[(size_t)E[f].vb * K + E[f].col] = -1;
      }
      for (int f : path) {
        E[f].col = E[f].col == a ? b : a;
        atL[(size_t)E[f].lane * K + E[f].col] = f;
        atV[(size_t)E[f].vb * K + E[f].col] = f;
      }
    }
    E[e].col = a;
    atL[(size_t)u * K + a] = e;
    atV[(size_t)v * K + a] = e;
  }
  int k = 0;
  for (int i = 0; i < 8; ++i)
    for (size_t j = 0; j < lists8[i].size(); ++j, ++k) slot_of[(size_t)i * maxlen + j] = E[k].col;
}

// Distributes the entries of 64 column lists (column l = 2 * lane + h) over
// K slots, each list in its own column of the slots, so that the loads one
// gather instruction makes (one slot, one h, 32 lanes) are spread over the
// shared-memory banks.  The hardware serves a 16-byte-per-lane load a quarter
// warp (8 lanes) at a time; sources of distinct rank mod 8 fall in distinct
// 16-byte bank groups (16-byte columns: rank mod 8; 32-byte swizzled
// columns: 2 (rank mod 4) + bit 2 of rank, also a bijection of rank mod 8).
// Per quarter warp and h this is an edge colouring of a bipartite multigraph:
// lanes on one side, bank groups on the other, an edge per entry, a colour
// per slot; a slot whose entries all have distinct bank groups costs one
// shared-memory wavefront.  A bank group with more than K entries is split
// into virtual groups of at most K, so that every vertex has degree <= K and
// K colours suffice (Konig's theorem); the colouring follows the alternating
// path argument of that theorem, one edge at a time.  A lane with fewer
// entries than K leaves slots empty: it reads one of the eight zero columns
// dim .. dim + 7, the same one for every empty lane of the quarter warp (a
// broadcast), picked in a bank group the quarter warp's real entries leave
// free, so empty slots need no test in the kernel.  Returns [K][64] entries
// (rank | sign << 31).
static std::vector<uint32_t> assign_slots(const std::vector<std::vector<uint32_t>>& lists, int K,
                                          uint32_t dim) {
  std::vector<uint32_t> out((size_t)K * 64, kEllNull);
  std::vector<uint32_t> lists8[8];
  std::vector<int> slot_of((size_t)8 * K);
  for (int h = 0; h < 2; ++h) {
    for (int ph = 0; ph < 4; ++ph) {
      int cols[8];
      for (int i = 0; i < 8; ++i) {
        cols[i] = 2 * (8 * ph + i) + h;
        lists8[i] = lists[cols[i]];
      }
      colour_quarter(lists8, K, slot_of, K);
      for (int i = 0; i < 8; ++i)
        for (size_t j = 0; j < lists8[i].size(); ++j)
          out[(size_t)slot_of[(size_t)i * K + j] * 64 + cols[i]] = lists8[i][j];
      // Where several bank groups have more than K entries the colouring
      // may put their surplus entries in different slots; moving a lane's
      // entry (or empty place) from one slot to another, while that lowers
      // the two slots' wavefronts, gathers them (a slot's wavefronts: the
      // most distinct sources it reads in one bank group, at least 1).
      auto slot_cost = [&](int k) {
        uint32_t r[8];
        int n = 0, c[8] = {0}, m = 1;
        for (int i = 0; i < 8; ++i) {
          const uint32_t e = out[(size_t)k * 64 + cols[i]];
          if (e == kEllNull) continue;
          const uint32_t rank = e & 0xFFFFu;
          bool dup = false;
          for (int q = 0; q < n; ++q) dup = dup || r[q] == rank;
          if (dup) continue;
          r[n++] = rank;
          m = std::max(m, ++c[rank & 7u]);
        }
        return m;
      };
      for (bool better = true; better;) {
        better = false;
        for (int k1 = 0; k1 < K; ++k1)
          for (int k2 = k1 + 1; k2 < K; ++k2) {
            int c12 = slot_cost(k1) + slot_cost(k2);
            if (c12 == 2) continue;
            for (int i = 0; i < 8; ++i) {
              uint32_t& e1 = out[(size_t)k1 * 64 + cols[i]];
              uint32_t& e2 = out[(size_t)k2 * 64 + cols[i]];
              if (e1 == e2) continue;
              std::swap(e1, e2);
              const int c = slot_cost(k1) + slot_cost(k2);
              if (c < c12) {
                c12 = c;
                better = true;
              } else {
                std::swap(e1, e2);
              }
            }
          }
      }
      for (int k = 0; k < K; ++k) {
        // the zero column for this slot's empty lanes of the quarter warp
        bool used[8] = {false};
        for (int i = 0; i < 8; ++i) {
          const uint32_t e = out[(size_t)k * 64 + cols[i]];
          if (e != kEllNull) used[e & 7u] = true;
        }
        uint32_t zero = dim;
        for (uint32_t z = 0; z < 8; ++z)
          if (!used[(dim + z) & 7u]) {
            zero = dim + z;
            break;
          }
        for (int i = 0; i < 8; ++i)
          if (out[(size_t)k * 64 + cols[i]] == kEllNull) out[(size_t)k * 64 + cols[i]] = zero;
      }
    }
  }
  return out;
}

// Connection rows of the basis in the order given by words (position ->
// word) and pos (ascending rank -> position): for target position r every
// source x = y ^ 2^p ^ 2^q that a hop along a bond turns into y = words[r],
// packed as (pos(x), group, sign) and sorted by (group, source).
static void connection_rows(const LatticeHost& L, const std::vector<uint32_t>& words,
                            const std::vector<uint32_t>& pos, std::vector<int32_t>& off,
                            std::vector<uint32_t>& ent) {
  const int dim = (int)words.size();
  off.assign(dim + 1, 0);
  ent.clear();
  struct E { uint32_t group, src, neg; };
  std::vector<E> row;
  for (int r = 0; r < dim; ++r) {
    const uint32_t y = words[r];
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
    for (const E& e : row) ent.push_back((e.src & 0xFFFFu) | (e.group << 16) | (e.neg << 31));
    off[r + 1] = (int32_t)ent.size();
  }
}

// Permutes the columns within each 64-column ELL tile (every tile keeps its
// column set, so its slot counts per group are unchanged) to spread the
// sources that each quarter warp's gathers read over the eight 16-byte bank
// groups.  The cost of one (tile, group, h, quarter warp) is K plus, over
// the bank groups, the entries beyond K in each: the wavefronts its K slots
// take when every surplus entry costs one (the fewest is K plus the largest
// surplus; the slot assignment gets close to that, and this cost, which also
// counts how many bank groups overflow, gave fewer wavefronts in the end
// than the bound itself).  Seeded local search over swaps of two columns of one
// tile, simulated annealing with an integer acceptance rule (a swap that
// raises the cost by c is taken with probability (thr / 2^20)^c, thr falling
// linearly from about e^-1 to 0), so every host builds the same table.
// Returns perm: new position -> old position.
static std::vector<int> tile_bank_search(const std::vector<int32_t>& off,
                                         const std::vector<uint32_t>& ent, int ngrp,
                                         long iters) {
  const int dim = (int)off.size() - 1;
  const int ntile = (dim + 63) / 64;
  std::vector<int> perm(dim);
  for (int i = 0; i < dim; ++i) perm[i] = i;
  if (dim < 2 || ngrp <= 0) return perm;
  struct En { int d, s, g; };
  std::vector<En> E;
  std::vector<std::vector<int>> by_t(dim), by_s(dim);
  for (int d = 0; d < dim; ++d)
    for (int e = off[d]; e < off[d + 1]; ++e) {
      const int s = (int)(ent[e] & 0xFFFFu), g = (int)((ent[e] >> 16) & 0xFFu);
      by_t[d].push_back((int)E.size());
      by_s[s].push_back((int)E.size());
      E.push_back({d, s, g});
    }
  // K of every (tile, group), invariant under the search
  std::vector<int> K((size_t)ntile * ngrp, 0);
  std::vector<int> cnt(ngrp);
  for (int d = 0; d < dim; ++d) {
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int e : by_t[d]) cnt[E[e].g]++;
    for (int g = 0; g < ngrp; ++g)
      K[(size_t)(d / 64) * ngrp + g] = std::max(K[(size_t)(d / 64) * ngrp + g], cnt[g]);
  }
  std::vector<int> pos(dim);   // column (old position) -> current position
  for (int d = 0; d < dim; ++d) pos[d] = d;
  auto inst = [&](int d, int g) {
    const int p = pos[d];
    return (((p / 64) * ngrp + g) * 2 + (p & 1)) * 4 + (p % 64) / 16;
  };
  const size_t ninst = (size_t)ntile * ngrp * 8;
  std::vector<int> deg(ninst * 8, 0);
  auto cost = [&](int I) {
    const int k = K[(size_t)I / 8];
    int m = k;
    for (int b = 0; b < 8; ++b) m += std::max(0, deg[(size_t)I * 8 + b] - k);
    return m;
  };
  auto add = [&](int e, int dlt) { deg[(size_t)inst(E[e].d, E[e].g) * 8 + (pos[E[e].s] & 7)] += dlt; };
  for (int e = 0; e < (int)E.size(); ++e) add(e, 1);
  uint64_t rng = 0x9E3779B97F4A7C15ull;
  auto rnd = [&]() {
    rng ^= rng << 13;
    rng ^= rng >> 7;
    rng ^= rng << 17;
    return rng;
  };
  const uint64_t thr0 = 385749;   // e^-1 * 2^20
  std::vector<int> aff, touched;
  std::vector<char> emark(E.size(), 0), imark(ninst, 0);
  for (long it = 0; it < iters; ++it) {
    const int t = (int)(rnd() % (uint64_t)ntile);
    const int n_in = std::min(64, dim - 64 * t);
    if (n_in < 2) continue;
    const int pa = 64 * t + (int)(rnd() % (uint64_t)n_in), pb = 64 * t + (int)(rnd() % (uint64_t)n_in);
    if (pa == pb) continue;
    const int a = perm[pa], b = perm[pb];
    aff.clear();
    touched.clear();
    for (int x : {a, b}) {
      for (int e : by_t[x]) if (!emark[e]) { emark[e] = 1; aff.push_back(e); }
      for (int e : by_s[x]) if (!emark[e]) { emark[e] = 1; aff.push_back(e); }
    }
    for (int pass = 0; pass < 2; ++pass) {   // instances before and after the swap
      for (int e : aff) {
        const int I = inst(E[e].d, E[e].g);
        if (!imark[I]) { imark[I] = 1; touched.push_back(I); }
      }
      std::swap(pos[a], pos[b]);
    }
    long before = 0, after = 0;
    for (int I : touched) before += cost(I);
    for (int e : aff) add(e, -1);
    std::swap(pos[a], pos[b]);
    for (int e : aff) add(e, 1);
    for (int I : touched) after += cost(I);
    bool take = after <= before;
    if (!take) {
      const uint64_t thr = thr0 * (uint64_t)(iters - it) / (uint64_t)iters;
      uint64_t p = thr;
      for (long c = 1; c < after - before && p; ++c) p = (p * thr) >> 20;
      take = (rnd() & 0xFFFFFu) < p;
    }
    if (take) {
      std::swap(perm[pa], perm[pb]);
    } else {
      for (int e : aff) add(e, -1);
      std::swap(pos[a], pos[b]);
      for (int e : aff) add(e, 1);
    }
    for (int e : aff) emark[e] = 0;
    for (int I : touched) imark[I] = 0;
  }
  return perm;
}

SpinTable build_spin_table(const LatticeHost& L, int n, bool hop_order) {
  SpinTable T;
  T.n = n;
  const std::vector<uint32_t> asc = spin_basis(L.Ns, n);
  T.dim = (int)asc.size();
  T.order.resize(T.dim);
  for (int i = 0; i < T.dim; ++i) T.order[i] = i;
  // pos[rank]: position of the state of that ascending-word rank
  std::vector<uint32_t> pos(T.dim);
  auto place = [&]() {
    T.words.resize(T.dim);
    for (int i = 0; i < T.dim; ++i) {
      T.words[i] = asc[T.order[i]];
      pos[T.order[i]] = (uint32_t)i;
    }
  };
  if (hop_order) {
    const int ngrp = 2 * L.n_classes;
    std::vector<int32_t> key((size_t)T.dim * ngrp, 0);   // hops into each state, per group
    for (int r = 0; r < T.dim; ++r) {
      const uint32_t y = asc[r];
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
    // then the columns of each tile rearranged for the gathers' banks
    place();
    std::vector<int32_t> off1;
    std::vector<uint32_t> ent1;
    connection_rows(L, T.words, pos, off1, ent1);
    const std::vector<int> perm = tile_bank_search(off1, ent1, ngrp, 64L * T.dim);
    std::vector<int32_t> o2(T.dim);
    for (int i = 0; i < T.dim; ++i) o2[i] = T.order[perm[i]];
    T.order = o2;
  }
  place();
  connection_rows(L, T.words, pos, T.off, T.ent);
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
