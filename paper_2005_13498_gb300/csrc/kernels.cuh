// Kernel launchers (host-callable), implemented in kernels.cu.
#pragma once

#include <algorithm>
#include <vector>

#include "common.h"

namespace ed {

enum KernelKind { KK_APPLY = 0, KK_UPDATE = 1, KK_EXPM = 2, KK_COMBINE = 3,
                  KK_ENERGY = 4, KK_OVERLAP = 5, KK_COUNT = 6 };

struct LaunchShape {
  int threads;   // block size of the apply kernel
  int ept;       // columns per thread per chunk in the apply kernel
  int nr;        // rows per CTA (apply blocks hold up to nr rows)
  size_t smem;   // dynamic shared memory of the apply kernel
  bool vec = false;  // complex64 rows accessed as 16-byte pairs
  int cfg = 0;       // index of the kernel configuration (rows, pairs, occupancy)
  bool split = false;  // column pass (T_up) + row pass instead of one kernel
  size_t smem_c = 0;   // dynamic shared memory of the column pass
  int cb = 32;         // column-pass block: bytes of columns per row (32 or 16);
                       // 0: the T_up pass gathers rows (k_apply_tup) instead
  int tc = 256;        // column-pass threads per CTA
  int ppc = 1;         // T_up pass: column pairs per thread (chunk = 256 ppc pairs)
  bool tma = false;    // T_up row chunks staged by TMA (one extra producer warp)
  bool mv = false;     // multi-vector blocks: one row of nr vectors of one sector
};

// Feasible apply configurations for sectors of at most max_dim_up rows of
// length max_dim_dn (the first is the default); the autotuner in engine.cpp
// times them on the real data.
std::vector<LaunchShape> apply_candidates(int max_dim_up, int max_dim_dn, bool fp64,
                                          int n_groups);

// Column blocks of the split apply: cb bytes of columns (cb / element size
// columns) covering columns [0, dim_dn) of vector vec.
inline void append_col_blocks(std::vector<ApplyBlock>& map, int vec, int dim_dn, bool fp64,
                              int cb) {
  const int nc = cb / (fp64 ? 16 : 8);
  for (int d = 0; d < dim_dn; d += nc)
    map.push_back({vec, d, dim_dn - d < nc ? dim_dn - d : nc, 0});
}

// Threads per CTA of the apply kernels (the default; a configuration may
// run its row pass with more) and rows per block of the row-gather T_up
// pass (k_apply_tup).
constexpr int kApplyThreads = 256;
constexpr int kTupRows = 4;
static_assert(kTupRows <= 4, "an ApplyBlock lists at most 4 rows");

// Blocks of the row-gather T_up pass of the split apply for one chunk of
// column pairs (from pc on) of vector vec: nr <= 4 rows per block, rows in
// the given order (natural when order is null).  The engine appends the
// chunks of all vectors chunk-major, so that the CTAs resident together
// gather from one chunk of columns of all rows.
inline void append_tup_chunk(std::vector<ApplyBlock>& map, int vec, int dim_up, int nr, int pc,
                             const std::vector<int>* order = nullptr) {
  for (int i = 0; i < dim_up; i += nr) {
    ApplyBlock b{vec, 0, dim_up - i < nr ? dim_up - i : nr, pc, {0, 0, 0, 0}};
    for (int r = 0; r < b.nrows; ++r) b.row[r] = order ? (*order)[i + r] : i + r;
    b.row0 = b.row[0];
    map.push_back(b);
  }
}

// Apply blocks of nr <= 4 rows covering rows [0, dim_up) of vector vec:
// consecutive rows in the order given (all rows once), or in natural order
// when order is null.
inline void append_apply_blocks(std::vector<ApplyBlock>& map, int vec, int dim_up, int nr,
                                const std::vector<int>* order = nullptr) {
  // every configuration of the table has nr <= 4 (the rows an ApplyBlock holds)
  for (int i = 0; i < dim_up; i += nr) {
    ApplyBlock b{vec, 0, dim_up - i < nr ? dim_up - i : nr, 0, {0, 0, 0, 0}};
    for (int r = 0; r < b.nrows; ++r) b.row[r] = order ? (*order)[i + r] : i + r;
    b.row0 = b.row[0];
    map.push_back(b);
  }
}

// Multi-vector apply blocks: for every sector, its vectors (vec_ids, in
// batch order) in subgroups of at most nr, and for each subgroup one block
// per row u in the given order (natural when order is null): row0 = u,
// nrows = vectors in the subgroup, row[r] = their batch indices, vec = the
// first of them.
inline void append_mv_blocks(std::vector<ApplyBlock>& map, const std::vector<int>& vec_ids,
                             int dim_up, int nr, const std::vector<int>* order = nullptr) {
  for (size_t g = 0; g < vec_ids.size(); g += nr) {
    const int k = (int)std::min<size_t>(nr, vec_ids.size() - g);
    for (int i = 0; i < dim_up; ++i) {
      ApplyBlock b{vec_ids[g], order ? (*order)[i] : i, k, 0, {0, 0, 0, 0}};
      for (int r = 0; r < k; ++r) b.row[r] = vec_ids[g + r];
      map.push_back(b);
    }
  }
}

// Block range [apply_begin, apply_end) of every vector: its own blocks, or
// in multi-vector maps the blocks of its subgroup (contiguous in the map).
inline void assign_apply_ranges(const std::vector<ApplyBlock>& map, bool mv,
                                VecDev* vd, int nvec) {
  for (int i = 0; i < nvec; ++i) { vd[i].apply_begin = -1; vd[i].apply_end = -1; }
  for (int b = 0; b < (int)map.size(); ++b) {
    VecDev& v = vd[map[b].vec];
    if (v.apply_begin < 0) v.apply_begin = b;
    v.apply_end = b + 1;
  }
  if (mv)
    for (const ApplyBlock& b : map)
      for (int r = 0; r < b.nrows; ++r) {
        vd[b.row[r]].apply_begin = vd[b.vec].apply_begin;
        vd[b.row[r]].apply_end = vd[b.vec].apply_end;
      }
}

// Doubles of reduction scratch per apply block (Re and Im of <x_j, w> per
// vector of the block).
inline size_t apply_partials_per_block(const LaunchShape& sh) {
  return sh.mv ? std::max(4, 2 * sh.nr) : 4;
}

// The configuration table: its size, and the precision, rows per CTA, pairs
// per thread, CTAs per SM, split, TMA and multi-vector flags of entry i
// (false if out of range).
int apply_config_count();
bool apply_config_info(int i, int* fp64, int* nr, int* pp, int* minb, int* split, int* tma,
                       int* mv);
// The default configuration (first candidate).
LaunchShape apply_shape(int max_dim_up, int max_dim_dn, bool fp64, int n_groups);
// Raise the dynamic shared-memory limit of the apply kernel for this shape
// (once, before launches or graph capture).
cudaError_t prepare_apply(bool fp64, const LaunchShape& sh);

// j >= 1: Lanczos step j; j == 0: plain apply x1 -> w with coefs row 0;
// j == -1: energy (w = H x1 with coefs_obs[step], out_energy[step] = <x1,w>/Ns).
// A split shape launches the column pass (a.col_map, a.n_col_blocks) first.
cudaError_t launch_apply(bool fp64, const BatchArgs& a, int n_apply_blocks,
                         const LaunchShape& sh, int j, cudaStream_t s);
cudaError_t launch_update(bool fp64, const BatchArgs& a, int n_ew_blocks, int j,
                          cudaStream_t s);
cudaError_t launch_expm(const BatchArgs& a, cudaStream_t s);
// y[b] = exp(-i tau T_b) e_1 for batch real symmetric tridiagonals T_b of
// order n <= kMaxKrylov (alpha: batch x n, beta: batch x (n - 1), y: batch x n
// complex as (re, im) pairs), device pointers; the routine of k_expm.
cudaError_t launch_tridiag_expm(const double* alpha, const double* beta, int n, double tau,
                                double* y, int batch, cudaStream_t s);
// Adaptive exit check after Lanczos step j (vectors with eps_tol > 0).
cudaError_t launch_conv_check(const BatchArgs& a, int j, cudaStream_t s);
cudaError_t launch_combine(bool fp64, const BatchArgs& a, int n_ew_blocks,
                           cudaStream_t s);
// Observables of x1 without combining (t_0): sets beta0, inv_scale[1], outputs.
cudaError_t launch_observe(bool fp64, const BatchArgs& a, int n_ew_blocks,
                           cudaStream_t s);

// Fermion operator: out[t] = sign * in[src(t)] through a row map (spin 0) or a
// column map (spin 1); spin 2: a column map with out stored transposed
// (dim_dn_dst x dim_up_dst).  map entries: src | (neg << 31); 0x7FFFFFFF = no
// source.
cudaError_t launch_fermion_op(bool fp64, const void* in, void* out,
                              int dim_up_src, int dim_dn_src,
                              int dim_up_dst, int dim_dn_dst, int spin,
                              const int32_t* map, cudaStream_t s);

// Overlaps <op psi | phi_b> for the phi vectors of a batch: per vector b with
// map_off[b] >= 0, psi = vec[psi_index].x1; result added to out[(step)*nb*2..]
struct OverlapArgs {
  const int32_t* maps;      // concatenated maps
  const void* psiT;         // psi transposed (dim_dn x dim_up), for map mode 2
  const int64_t* map_off;   // [nvec] offset into maps, -1 = no overlap
  const int32_t* map_spin;  // [nvec] 0 row map, 1 column map, 2 column map with the
                            // vector stored transposed (see k_fermion_op)
  int psi_index;            // vector holding psi(t_n)
  double* out;              // [n_steps+1][nvec][2] (re, im)
};
cudaError_t launch_overlap(bool fp64, const BatchArgs& a, const OverlapArgs& o,
                           int n_ew_blocks, cudaStream_t s);
// In-place column permutation of each row of a dim_up x dim_dn complex
// matrix (device): forward x[u][i] = x_old[u][order[i]], else the inverse.
// order holds 2 dim_dn entries: the permutation, then its inverse.
cudaError_t launch_permute_cols(bool fp64, void* x, int dim_up, int dim_dn, const int32_t* order,
                                bool forward, cudaStream_t s);
// The same from src to dst (distinct buffers; either may be a pinned host
// buffer's device-mapped address): forward dst[u][i] = src[u][order[i]],
// else dst[u][order[i]] = src[u][i]; dim_dn = 1 copies.
cudaError_t launch_permute_cols_copy(bool fp64, const void* src, void* dst, int dim_up,
                                     int dim_dn, const int32_t* order, bool forward,
                                     cudaStream_t s);
// out[c * rows + r] = in[r * cols + c] for a rows x cols complex matrix.
cudaError_t launch_transpose(bool fp64, const void* in, void* out, int rows, int cols,
                             cudaStream_t s);

// ---- ground-state helpers (float64 only) ---------------------------------
// partial[blk][i] = sum over block chunk of conj(V_i) w, i < k  (k <= 256)
cudaError_t launch_multidot(const double2* V, int64_t ldV, int k,
                            const double2* w, int64_t D, double2* partial,
                            int nblk, cudaStream_t s);
cudaError_t launch_reduce_cols(const double2* partial, int nblk, int k,
                               double2* out, cudaStream_t s);
// w -= sum_i c_i V_i  (c on device)
cudaError_t launch_multiaxpy(const double2* V, int64_t ldV, int k,
                             const double2* c, double2* w, int64_t D,
                             cudaStream_t s);
// y = sum_i c_i V_i (c real, on device)
cudaError_t launch_combine_real(const double2* V, int64_t ldV, int k,
                                const double* c, double2* y, int64_t D,
                                cudaStream_t s);
// partial sums of |x|^2 and optionally Re<x, y>; out[2] via deterministic
// two-pass reduction (partial has nblk*2 doubles).
cudaError_t launch_norm_dot(const double2* x, const double2* y, int64_t D,
                            double* partial, int nblk, double* out,
                            cudaStream_t s);
cudaError_t launch_scale(double2* x, int64_t D, const double* s_dev,
                         bool inverse_sqrt, cudaStream_t s);
cudaError_t launch_axpy_real(double2* y, const double2* x, int64_t D,
                             const double* a_dev, double a_sign,
                             cudaStream_t s);
cudaError_t launch_random_fill(double2* x, int64_t D, uint64_t seed,
                               cudaStream_t s);
// double occupancy: out[0] = sum_k w_d |psi|^2, out[1+i] = site i values
cudaError_t launch_docc_sites(bool fp64, const void* psi, const SectorDev* sec,
                              int dim_up, int dim_dn, int Ns, double* partial,
                              int nblk, double* out, cudaStream_t s);
// dtype conversion
cudaError_t launch_convert(const void* in, bool in_fp64, void* out,
                           bool out_fp64, int64_t n_complex, cudaStream_t s);

}  // namespace ed
