// Host-side basis enumeration, ranks, connection tables and sector maps.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "common.h"   // kEllNull

namespace ed {

// Null entry of a padded row: contributes zero (bit 30; no rank uses it).
constexpr uint32_t kNullEntry = 0x40000000u;

// Byte offset of column `rank` in the shared-memory tile of the apply kernel
// when a column holds 32 bytes (two 16-byte chunks, swapped for columns with
// bit 2 set to spread random gathers over all bank groups); the second chunk
// is at offset ^ 16.  Layouts with other column sizes recover the rank as
// offset >> 5.
inline uint32_t tile_offset(uint32_t rank) { return 32u * rank + 16u * ((rank >> 2) & 1u); }

// Spin basis of n electrons on Ns sites: all Ns-bit words with n ones in
// ascending order (Sec. 3.1; the order of the hash of Eq. (36)).
std::vector<uint32_t> spin_basis(int Ns, int n);

// Rank of a popcount-n word in that basis by the combinatorial number system,
// sum_k C(p_k, k+1) over the 0-based sorted occupied positions p_0 < p_1 < ...
// (Eq. (36) with 0-based positions).
uint32_t combinadic_rank(uint32_t word);
uint64_t binomial(int n, int k);

struct LatticeHost {
  int Ns = 0;
  int n_bonds = 0;
  std::vector<int> p, q;
  std::vector<double> t, d;      // d: 3 per bond
  double U = 0.0;
  bool has_eps = false;
  std::vector<double> eps;       // Ns
  int n_classes = 0;             // bonds with equal (t, d) share a class
  std::vector<int> bond_class;   // per bond
  std::vector<double> class_t, class_d;
};

// Validates and fills the bond classes; returns "" or an error message.
std::string make_lattice(LatticeHost& L, int Ns, int n_bonds, const int32_t* p,
                         const int32_t* q, const double* t, const double* d,
                         double U, const double* eps);

// Connection table of one spin species (target-row major, CSR):
// for target configuration y (rank r) every source x = y ^ 2^p ^ 2^q that a
// hop along a bond turns into y, packed as (rank(x), group, sign).  Entries
// of a row are sorted by (group, source rank).
struct SpinTable {
  int n = 0, dim = 0;
  std::vector<uint32_t> words;
  std::vector<int32_t> off;
  std::vector<uint32_t> ent;
  std::vector<double> eps_sum;   // per state: sum of eps over occupied sites
  // Padded rows (used for the across-row gathers): the entries of row r,
  // sorted by group, padded to a multiple of 4 with null entries (bit 30 set,
  // sign 0, source = row r itself, group of the last real entry); row r
  // occupies pad_ent[pad_off[r] .. pad_off[r+1]).
  std::vector<int32_t> pad_off;
  std::vector<uint32_t> pad_ent;
  // Warp-tiled ELL (used for the within-row gathers): columns in tiles of 64,
  // lane l of a warp owning columns 64c + 2l and 64c + 2l + 1.  Tile c owns
  // slots tslot_off[c] .. tslot_off[c+1] (a multiple of 2, grouped by bond
  // group, slot_grp[s] = group of slot s); slot s holds for lane l the two
  // entries tile_offset(rank) | sign << 31 of its columns at
  // ell[2 * (s * 32 + l)] and [.. + 1].  A group spans as many slots as its
  // longest column list in the tile; which slot each entry of a column takes
  // is chosen so that the eight lanes of each quarter warp read sources of
  // distinct rank mod 8 where possible (distinct 16-byte shared-memory bank
  // groups for 16- and 32-byte tile columns, see assign_slots).  A slot a
  // column does not use points to one of the zero columns dim .. dim + 7 of
  // the tile, chosen in a bank group that slot's quarter warp leaves free.
  std::vector<int32_t> tslot_off;
  std::vector<uint32_t> slot_grp;
  std::vector<uint32_t> ell;
  // order[i]: the rank (ascending-word position) of the basis state at
  // position i of this table; the identity unless built in hop order
  std::vector<int32_t> order;
};
// The table of one spin species in ascending-word order (the basis order of
// the C ABI), or with hop_order in the order of decreasing per-group hop
// counts (ties by word): every quantity of the table (words, entries' source
// positions, ELL) then refers to positions in that order, whose 64-column
// ELL tiles hold columns of equal entry counts per group and so need fewer
// padded slots.  A vector whose columns are in hop order is the ascending
// one permuted by `order` (k_permute_cols in kernels.cu).
SpinTable build_spin_table(const LatticeHost& L, int n, bool hop_order = false);

// First rows of the blocks of nr consecutive rows of the target space of T
// (the apply's CTAs), in reverse Cuthill-McKee order of the graph in which
// two blocks are adjacent when a row of one has a source row in the other.
// Launched in this order, the CTAs resident at one time gather from a
// compact set of source rows (the working set the L2 must hold shrinks).
std::vector<int> block_order(const SpinTable& T, int nr);

// Per-group hopping coefficients for a vector potential A:
//   group 2c   (hop p -> q of class c): -t_c exp(-i A.d_c)
//   group 2c+1 (hop q -> p):            -t_c exp(+i A.d_c)
// written as interleaved (re, im) doubles, 2 * n_classes complex numbers.
void group_coefficients(const LatticeHost& L, const double A[3], double* out);

// Vector potential of the pump pulse at time t (shape 0: A0 e^{-s^2/2sigma^2}
// sin(omega s) dir; shape 1: -A0 [cos(omega s) - b] e^{-s^2/2sigma^2} dir,
// s = t - t0).
void pulse_A(int shape, double A0, double omega, double sigma, double t0, double b,
             const double dir[3], double t, double out[3]);

// Map for c_{i,s} (create = false) or c^+_{i,s} (create = true) from the
// sector (n_up, n_dn) to the target sector, over the target ranks of spin s:
// entry = source rank | (sign < 0) << 31, or 0x7FFFFFFF when the target
// configuration has no source.  Sign (-1)^(occupied modes before (i, s)),
// modes ordered all up then all down (so spin 1 includes (-1)^n_up).
std::vector<int32_t> fermion_map(int Ns, int n_up, int n_dn, int site, int spin,
                                 bool create);

}  // namespace ed
