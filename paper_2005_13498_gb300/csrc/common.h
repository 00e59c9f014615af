// Internal definitions shared by the host driver and the CUDA kernels.
// Not part of the public ABI (include/ed.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ed {

constexpr int kMaxKrylov = 64;      // largest supported Krylov dimension m
constexpr int kMaxSites = 16;       // Ns <= 16: spin ranks fit in 16 bits
constexpr int kMaxGroups = 256;     // 2 * bond classes (group id is 8 bits)

// Packed connection-table entry (one per allowed hop into a target state):
//   bits  0-15  rank of the source configuration (same spin basis)
//   bits 16-23  group = 2 * bond class + orientation (0: p->q, 1: q->p)
//   bit  31     fermion sign of the hop (1 = negative)
constexpr uint32_t kEntRankMask = 0xFFFFu;
constexpr int kEntGroupShift = 16;
constexpr uint32_t kEntSignBit = 0x80000000u;
constexpr uint32_t kNullEntryBit = 0x40000000u;  // padding entry of a row list
constexpr uint32_t kEllNull = 0x7FFFFFFFu;       // host marker of an unassigned ELL slot
constexpr int kZeroCols = 8;                     // zero columns past the end of a staged tile

// Device view of one sector's tables (pointers into device memory).
struct SectorDev {
  int dim_up, dim_dn;
  int n_up, n_dn;
  const int32_t* up_off;    // [dim_up + 1]
  const uint32_t* up_ent;   // packed entries, target-row major
  const int32_t* dn_off;    // [dim_dn + 1]
  const uint32_t* dn_ent;
  const uint32_t* up_word;  // [dim_up] spin configuration words
  const uint32_t* dn_word;  // [dim_dn]
  const double* up_eps;     // [dim_up] sum of eps over occupied sites, or null
  const double* dn_eps;     // [dim_dn]
  // up spin: rows padded to multiples of 4 entries (across-row gathers)
  const int32_t* up_pad_off;   // [dim_up + 1]
  const uint32_t* up_pad_ent;  // entries; bit 30 = null (contributes zero)
  const uint32_t* up_pad_row;  // element offset of the source row: rank * dim_dn
  const uint32_t* up_pad_cs;   // coefficient slot: 0 padding, else 1 + 2 group + sign
  // down spin: warp-tiled ELL over 64-column tiles (within-row gathers),
  // slot lists as in SpinTable (tables.h)
  const int32_t* dn_tslot_off; // [ceil(dim_dn/64) + 1], even slot counts
  const uint32_t* dn_slot_grp; // group of each slot
  // packed: one word per lane and slot [slots][32 lanes] with both entries
  // of the lane as 15-bit column units and signs (bits 0-14 unit of the
  // first column's entry, 15 sign of the second, 16-30 unit of the second,
  // 31 sign of the first); units of 16 bytes in 32-byte tile columns
  // (2 rank + swizzle bit), and in 16- and 8-byte columns the unit is the
  // column width, so the units are the source ranks
  const uint32_t* dn_ellp32;
  const uint32_t* dn_ellpr;
  // up spin, same tiling over 64-row tiles (the column pass of the split
  // apply), entries tile_offset(rank) | sign << 31 for 32-byte tile columns
  // and 16 rank | sign << 31 for 16-byte ones
  const int32_t* up_tslot_off;
  const uint32_t* up_slot_grp;
  const uint32_t* up_ell;
  const uint32_t* up_ell16;
};

// Per-vector Lanczos scalars, all float64, 1-based Krylov index j.
// x_j denotes the stored (unnormalised) vector, v_j = inv_scale[j] * x_j the
// Lanczos vector of Algorithm 6.  x_1 is the propagated state itself.
struct LanczosState {
  double alpha[kMaxKrylov + 2];
  double beta[kMaxKrylov + 2];
  double inv_scale[kMaxKrylov + 2];
  double comb_re[kMaxKrylov + 2];   // combine coefficients: psi = sum comb_j x_j
  double comb_im[kMaxKrylov + 2];
  double scale;      // running max(1, |alpha|, beta) for the breakdown test
  double beta0;      // |psi| at the start of the step
  double delta;      // a-posteriori estimate of the last step
  double dot_out;    // scratch result of a plain dot product
  double red[4];     // scratch results of generic reductions
  // adaptive exit of Algorithm 6 (eps_tol > 0): the check after step j
  // stores y^(j) = exp(-i tau T_j) e_1 here and sets conv_m = j once the
  // a-posteriori error epsilon drops below eps_tol
  double eps_tol;                   // 0: fixed Krylov dimension
  double sc_at[kMaxKrylov + 2];     // breakdown scale max(1,|alpha|,beta) seen by step j
  double yprev_re[kMaxKrylov];
  double yprev_im[kMaxKrylov];
  double conv_delta;                // delta of the converged step
  int m;             // requested Krylov dimension
  int m_eff;         // dimension in use (set < m on breakdown)
  int stopped;       // 1 once breakdown was detected in this step
  int step;          // time-step counter (indexes coefficient arrays)
  int status;        // 0 ok, ED_ERR_NUMERIC on a non-finite norm
  int conv_m;        // 0, or the step j at which the adaptive exit was taken
  int pad[2];
};

// One propagated vector of a batch.
struct VecDev {
  int sector;          // index into the SectorDev array
  int pad0;
  int64_t D;           // dim_up * dim_dn
  void* x1;            // the state psi (x_1)
  void* V;             // (m-1) * D slots for x_2 .. x_m
  void* w;             // scratch vector of D elements
  int apply_begin, apply_end;   // range of apply blocks of this vector
  int ew_begin, ew_end;         // range of elementwise blocks
  double* out_docc;    // device [n_steps+1] or null
  double* out_norm2;   // device [n_steps+1] or null
  double* out_energy;  // device [n_steps+1] or null
  double* out_delta;   // device [n_steps] or null
  int* out_meff;       // device [n_steps] or null
};

// Elementwise block: elements [begin, end) of vector vec.
struct EwBlock {
  int vec;
  int pad;
  int64_t begin, end;
};

// Apply block: the nrows (<= 4) rows row[0..nrows) of vector vec, not
// necessarily consecutive (row0 = row[0]); for the column pass of the split
// apply: columns [row0, row0 + nrows); for its row-gather T_up pass: the
// rows row[0..nrows) and the column pairs from pc on (one chunk).
struct ApplyBlock {
  int vec;
  int row0;
  int nrows;
  int pc;
  int row[4];
};

// Everything the batched kernels need, passed by value.
struct BatchArgs {
  const SectorDev* sec;
  VecDev* vec;
  LanczosState* st;
  const ApplyBlock* apply_map;
  const ApplyBlock* col_map;  // split apply: column blocks (row0 = first column)
  const EwBlock* ew_map;
  double* partials;       // >= 4 * max(#apply blocks, #ew blocks)
  unsigned* counters;     // [nvec], zero between kernels
  const void* coefs;      // [n_steps][n_groups] complex of the vector dtype
  const void* coefs_obs;  // [n_steps+1][n_groups] (energy at t_n) or null
  int n_groups;
  int nvec;
  int Ns;
  int max_dim_dn;
  int max_dim_up;
  int n_col_blocks;
  double U;
  double tau;
  double break_tol;
  // bounded device-side waits (TMA configurations of the apply): polls of
  // every mbarrier wait before it gives up with ED_ERR_TIMEOUT, and a test
  // hook, the index (per thread block) of the T_up row-chunk copy that the
  // producer warp stops at without issuing it (-1: none), which makes the
  // consumers' wait for that copy run out
  uint32_t wait_limit;
  int tma_withhold;
};

// Default poll limit of the bounded mbarrier waits.
constexpr uint32_t kDefaultWaitLimit = 1u << 22;

}  // namespace ed
