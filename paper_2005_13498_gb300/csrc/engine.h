// Batched propagation engine: owns the device workspace of one or more
// vectors propagated together by the exponential midpoint rule, and the CUDA
// graph of one time step.
#pragma once

#include <string>
#include <vector>

#include "common.h"
#include "kernels.cuh"

// Returns the failing call and CUDA's message as a string from a function
// that reports errors as std::string (empty on success).
#define ED_TRY(call)                                                    \
  do {                                                                  \
    cudaError_t e_ = (call);                                            \
    if (e_ != cudaSuccess)                                              \
      return std::string(#call) + ": " + cudaGetErrorString(e_);        \
  } while (0)

namespace ed {

struct SpinTable;   // tables.h

struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t alloc(size_t n);
  void release();
  ~DevMem() { release(); }
};

struct EngineVector {
  int sector;      // index into the engine's sector list
  int64_t D;
  void* x1;        // device pointer of the state (external or owned)
  bool owned_x1;
};

struct EngineConfig {
  int64_t workspace_limit = 0;   // > 0: cap on the engine's device allocations (bytes)
  bool fp64 = false;
  int m = 1;
  bool energy = false;
  bool overlaps = false;
  int n_steps_cap = 0;
  double eps_tol = 0.0;   // > 0: adaptive exit of Algorithm 6, m is the maximum
};

// Autotuner of the apply kernel: times the feasible configurations (rows per
// CTA, column pairs per thread, occupancy target) with plain applies on the
// caller's buffers and keeps the fastest.  Decisions are cached per
// (precision, vector shapes) for the life of the process.
struct ApplyTuneTarget {
  bool fp64 = false;
  bool vec_ok = false;          // complex64 rows may be read as 16-byte pairs
  bool tma_ok = false;          // even rows, 16-byte aligned bases (TMA row chunks)
  int max_dim_up = 1;
  int max_dim_dn = 1;
  int n_groups = 0;
  std::vector<int> dim_up;      // per vector
  std::vector<int> dim_dn;      // per vector
  std::vector<const SpinTable*> up;   // per vector: up-spin table (CTA order), or empty
  std::vector<int> sector;      // per vector: sector index (equal = same tables)
  BatchArgs args{};             // vec / sec / coefs valid; the block maps are set here
};
// Process-wide choice of the apply configuration: -1 lets the autotuner pick
// (default), otherwise the index into the configuration table is used for
// every engine and plan set up afterwards (tune_apply fails if that
// configuration does not fit the precision or sector).
void set_forced_apply_config(int cfg);
int forced_apply_config();
// Test hook of the bounded device-side waits (ed_set_wait_fault): the T_up
// copy the TMA producer stops at (-1: none) and the poll limit of every
// mbarrier wait (0: kDefaultWaitLimit); engines and plans set up afterwards
// use them.
void set_wait_fault(int withhold, uint32_t polls);
// A BatchArgs with every field zero except the wait controls, which take the
// current test-hook state (by default: no withheld copy, the default limit).
void init_batch_args(BatchArgs* a);
// Picks the apply configuration and returns its row-block map and (split
// shapes) its column-block map.
std::string tune_apply(const ApplyTuneTarget& t, cudaStream_t s, LaunchShape* shape,
                       std::vector<ApplyBlock>* map, std::vector<ApplyBlock>* cmap);

class Engine {
 public:
  ~Engine();
  // Allocate everything; sectors must stay alive while the engine exists.
  // up_tabs (optional, one per sector) give the CTA order of the apply.
  std::string setup(const EngineConfig& cfg, const std::vector<SectorDev>& sectors,
                    const std::vector<EngineVector>& vecs, int n_groups, int Ns,
                    double U, double break_tol, cudaStream_t stream,
                    const std::vector<const SpinTable*>& up_tabs = {});
  bool compatible(const EngineConfig& cfg, const std::vector<EngineVector>& vecs) const;
  int apply_config() const { return shape_.cfg; }
  // Upload per-step coefficients ([n_steps][n_groups] complex double; energy
  // coefficients [n_steps+1][n_groups] or empty) and reset the Lanczos state.
  std::string begin(const std::vector<double>& coefs, const std::vector<double>& coefs_obs,
                    int n_steps, double tau, cudaStream_t stream);
  // Observables at t_0, then n_steps steps (graph replays or profiled launches).
  std::string run(int n_steps, bool profile, double* kernel_ms, int64_t* launches,
                  cudaStream_t stream);
  // Copy per-vector outputs of the last run to host (synchronises stream).
  std::string fetch(int vec, int n_steps, double* docc, double* norm2, double* energy,
                    double* delta, int32_t* meff, int* status, cudaStream_t stream);
  std::string fetch_overlaps(int n_steps, std::vector<double>& out, cudaStream_t stream);
  // Green's-function overlaps after every step (and at t_0): vector b with
  // off[b] >= 0 is overlapped with the image of vector psi_index under its map.
  std::string set_overlap_maps(const std::vector<int32_t>& maps, const std::vector<int64_t>& off,
                               const std::vector<int32_t>& spin, int psi_index, cudaStream_t s);
  size_t device_bytes() const;
  void* vec_x1(int v) const { return vecs_[v].x1; }
  int nvec() const { return (int)vecs_.size(); }

 private:
  std::string launch_step(cudaStream_t s, bool profile, cudaEvent_t* ev, int* kind_of,
                          int* nev);
  std::string capture(cudaStream_t s);
  // psi^T for the overlaps of vectors stored transposed (map mode 2)
  cudaError_t launch_psiT(cudaStream_t s);

  EngineConfig cfg_;
  int64_t workspace_bytes_ = 0;   // owned states + Krylov slots + scratch
  std::vector<EngineVector> vecs_;
  std::vector<SectorDev> sectors_;
  int n_groups_ = 0, Ns_ = 0;
  double U_ = 0.0, break_tol_ = 0.0, tau_ = 0.0;
  int n_apply_ = 0, n_ew_ = 0;
  LaunchShape shape_{};
  // adaptive exit: side stream for the convergence checks and the events
  // that fork check j after update j and join it before pass j + 2
  cudaStream_t side_ = nullptr;
  std::vector<cudaEvent_t> ev_fork_, ev_check_;
  BatchArgs args_{};
  OverlapArgs oargs_{};
  bool have_overlaps_ = false;
  DevMem d_sec_, d_vec_, d_st_, d_amap_, d_cmap_, d_emap_, d_partials_, d_counters_;
  DevMem d_coefs_, d_coefs_obs_, d_V_, d_w_, d_out_, d_owned_x1_;
  DevMem d_maps_, d_map_off_, d_map_spin_, d_ovl_, d_psiT_;
  bool need_psiT_ = false;
  cudaGraph_t graph_ = nullptr;
  cudaGraphExec_t exec_ = nullptr;
};

}  // namespace ed
