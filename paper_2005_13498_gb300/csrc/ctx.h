// Internal context type and helpers shared by the C-ABI translation units.
#pragma once

#include "../../include/ed.h"

#include <initializer_list>
#include <memory>
#include <string>
#include <vector>

#include "common.h"
#include "engine.h"
#include "kernels.cuh"
#include "tables.h"

namespace ed {

struct SectorGPU {
  int Ns = 0, n_up = 0, n_dn = 0;
  SpinTable up, dn;
  DevMem up_off, up_ent, dn_off, dn_ent, up_word, dn_word, up_eps, dn_eps;
  DevMem up_pad_off, up_pad_ent, up_pad_row, up_pad_cs, dn_tslot_off, dn_slot_grp;
  DevMem up_tslot_off, up_slot_grp, up_ell, up_ell16;
  DevMem dn_ellp32, dn_ellpr;
  SectorDev dev{};
  // the down-spin table in hop order (build_spin_table) with its device
  // copies, and dev_hop: dev with those down-spin tables, for vectors whose
  // columns are permuted into hop order (dn_order: position -> rank, then
  // its inverse rank -> position)
  SpinTable dn_hop;
  DevMem dnh_off, dnh_ent, dnh_word, dnh_eps, dnh_tslot_off, dnh_slot_grp, dnh_ellp32,
      dnh_ellpr, dn_order;
  SectorDev dev_hop{};
  bool has_eps = false;
  bool uploaded = false;
};

struct ApplyPlan {
  int nvec = 0;
  const void* v = nullptr;
  void* w = nullptr;
  bool fp64 = false;
  DevMem sec, vec, st, amap, cmap, partials, counters, coefs;
  BatchArgs args{};
  LaunchShape shape{};
  int nblk = 0;
  double A[3] = {0, 0, 0};
  bool valid = false;
};

}  // namespace ed

struct ed_ctx {
  int Ns = 0, n_up = 0, n_dn = 0;
  int64_t dim_up = 0, dim_dn = 0;
  std::vector<uint32_t> up_words, dn_words;
  bool lattice_set = false;
  ed::LatticeHost lat;
  ed::SectorGPU sec;
  double A[3] = {0, 0, 0};
  double krylov_tol = 0.0;   // > 0: adaptive Krylov dimension (Algorithm 6)
  int64_t workspace_limit = 0;   // > 0: cap on Krylov workspace allocations (bytes)
  int integrator = 0;        // ED_MIDPOINT or ED_CFET4
  std::string err;
  cudaStream_t stream = nullptr;
  int device = 0;
  ed::ApplyPlan plan;
  std::unique_ptr<ed::Engine> engine;
  std::unique_ptr<ed::Engine> spec_engine;
  std::vector<std::unique_ptr<ed::SectorGPU>> spec_sectors;
};

namespace ed {

ed_status fail(ed_ctx* ctx, ed_status st, const std::string& msg);
ed_status cuda_fail(ed_ctx* ctx, cudaError_t e, const char* what);
cudaError_t build_sector_gpu(SectorGPU& S, const LatticeHost& L, int n_up, int n_dn);
void build_sector_host(SectorGPU& S, const LatticeHost& L, int n_up, int n_dn);
cudaError_t upload_sector(SectorGPU& S);
// Upload the context's tables and create its stream on first GPU use.
ed_status ensure_device(ed_ctx* ctx);
// Refuse to launch when the current device is not the one the context's
// tables live on (ED_ERR_STATE), or when a caller's device buffer belongs to
// another device (ED_ERR_ARG); null entries of bufs are skipped.
ed_status check_device(ed_ctx* ctx, std::initializer_list<const void*> bufs);
bool is_device_ptr(const void* p);
cudaError_t join_streams(cudaStream_t from, cudaStream_t to);
std::vector<double> step_coefficients(const LatticeHost& L, const ed_pulse* pulse,
                                      double t_start, double dt, int n_steps, bool mid);
// ED_ERR_ARG (recorded on ctx) for non-finite parameters or an unknown shape.
ed_status check_pulse(ed_ctx* ctx, const ed_pulse* pulse);
// The Krylov sub-steps of n_steps time steps of the context's integrator:
// per-sub-step group coefficients, the sub-step length, and the number of
// sub-steps per time step (1 for the midpoint rule, 2 for CFET4).
struct SubSteps {
  std::vector<double> coefs;
  double tau = 0.0;
  int per_step = 1;
};
SubSteps integrator_substeps(const ed_ctx* ctx, const ed_pulse* pulse, double t_start,
                             double dt, int n_steps);

template <typename T>
cudaError_t upload(DevMem& m, const std::vector<T>& v) {
  cudaError_t e = m.alloc(std::max<size_t>(1, v.size()) * sizeof(T));
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  return cudaMemcpy(m.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace ed

#define CK(ctx, call)                                               \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return ed::cuda_fail((ctx), e_, #call);  \
  } while (0)

#define CKS(ctx, strexpr)                                           \
  do {                                                              \
    std::string s_ = (strexpr);                                     \
    if (!s_.empty()) return ed::fail((ctx), ED_ERR_CUDA, s_);       \
  } while (0)
