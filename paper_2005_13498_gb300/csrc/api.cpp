// C ABI (include/ed.h): contexts, tables on the device, and the drivers of
// ed_apply_H, ed_propagate and the sector maps.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "ctx.h"
#include "device_guard.h"

using namespace ed;

namespace {
thread_local std::string g_last_error;
}

namespace ed {

ed_status fail(ed_ctx* ctx, ed_status st, const std::string& msg) {
  g_last_error = msg;
  if (ctx) ctx->err = msg;
  return st;
}

ed_status cuda_fail(ed_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, e == cudaErrorMemoryAllocation ? ED_ERR_OOM : ED_ERR_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

void build_sector_host(SectorGPU& S, const LatticeHost& L, int n_up, int n_dn) {
  S.Ns = L.Ns;
  S.n_up = n_up;
  S.n_dn = n_dn;
  S.up = build_spin_table(L, n_up);
  S.dn = build_spin_table(L, n_dn);
  S.dn_hop = build_spin_table(L, n_dn, true);
  S.has_eps = L.has_eps;
  S.uploaded = false;
}

cudaError_t upload_sector(SectorGPU& S) {
  cudaError_t e;
  if ((e = upload(S.up_off, S.up.off)) != cudaSuccess) return e;
  if ((e = upload(S.up_ent, S.up.ent)) != cudaSuccess) return e;
  if ((e = upload(S.dn_off, S.dn.off)) != cudaSuccess) return e;
  if ((e = upload(S.dn_ent, S.dn.ent)) != cudaSuccess) return e;
  if ((e = upload(S.up_word, S.up.words)) != cudaSuccess) return e;
  if ((e = upload(S.dn_word, S.dn.words)) != cudaSuccess) return e;
  if ((e = upload(S.up_pad_off, S.up.pad_off)) != cudaSuccess) return e;
  if ((e = upload(S.up_pad_ent, S.up.pad_ent)) != cudaSuccess) return e;
  {
    std::vector<uint32_t> rows(S.up.pad_ent.size());
    for (size_t i = 0; i < rows.size(); ++i)
      rows[i] = (S.up.pad_ent[i] & kEntRankMask) * (uint32_t)S.dn.dim;
    if ((e = upload(S.up_pad_row, rows)) != cudaSuccess) return e;
    std::vector<uint32_t> cs(S.up.pad_ent.size());
    for (size_t i = 0; i < cs.size(); ++i) {
      const uint32_t en = S.up.pad_ent[i];
      cs[i] = (en & kNullEntryBit) ? 0u
                                   : 1u + 2u * ((en >> kEntGroupShift) & 0xFFu) + (en >> 31);
    }
    if ((e = upload(S.up_pad_cs, cs)) != cudaSuccess) return e;
  }
  if ((e = upload(S.dn_tslot_off, S.dn.tslot_off)) != cudaSuccess) return e;
  if ((e = upload(S.dn_slot_grp, S.dn.slot_grp)) != cudaSuccess) return e;
  if ((e = upload(S.up_tslot_off, S.up.tslot_off)) != cudaSuccess) return e;
  if ((e = upload(S.up_slot_grp, S.up.slot_grp)) != cudaSuccess) return e;
  if ((e = upload(S.up_ell, S.up.ell)) != cudaSuccess) return e;
  {
    // 16-byte-column copy of the up ELL: the byte offset of the source
    // (rank) in tiles of 16-byte columns, from tile_offset = 32 rank + 16 sw
    auto width_copy = [](const std::vector<uint32_t>& ell, uint32_t width) {
      std::vector<uint32_t> out(ell.size());
      for (size_t i = 0; i < ell.size(); ++i)
        out[i] = (((ell[i] & 0x7FFFFFFFu) >> 5) * width) | (ell[i] & 0x80000000u);
      return out;
    };
    if ((e = upload(S.up_ell16, width_copy(S.up.ell, 16))) != cudaSuccess) return e;
    // packed copies of the down-spin ELL: lane words of two 15-bit column
    // units (unit = byte offset / 16, or / 8 for 8-byte columns) and signs
    auto packed_copy = [](const std::vector<uint32_t>& ell, int width, std::vector<uint32_t>* out) {
      out->resize(ell.size() / 2);
      for (size_t i = 0; i < out->size(); ++i) {
        uint32_t u[2], sg[2];
        for (int h = 0; h < 2; ++h) {
          const uint32_t en = ell[2 * i + h];
          const uint32_t off = en & 0x7FFFFFFFu;          // 32 rank + 16 swizzle
          u[h] = width == 32 ? off >> 4 : (off >> 5);
          sg[h] = en >> 31;
          if (u[h] > 0x7FFFu) return false;
        }
        (*out)[i] = u[0] | (sg[1] << 15) | (u[1] << 16) | (sg[0] << 31);
      }
      return true;
    };
    std::vector<uint32_t> pk;
    if (!packed_copy(S.dn.ell, 32, &pk)) return cudaErrorInvalidValue;
    if ((e = upload(S.dn_ellp32, pk)) != cudaSuccess) return e;
    if (!packed_copy(S.dn.ell, 16, &pk)) return cudaErrorInvalidValue;   // units = rank
    if ((e = upload(S.dn_ellpr, pk)) != cudaSuccess) return e;
    // the same for the hop-ordered down-spin table
    if ((e = upload(S.dnh_off, S.dn_hop.off)) != cudaSuccess) return e;
    if ((e = upload(S.dnh_ent, S.dn_hop.ent)) != cudaSuccess) return e;
    if ((e = upload(S.dnh_word, S.dn_hop.words)) != cudaSuccess) return e;
    if ((e = upload(S.dnh_tslot_off, S.dn_hop.tslot_off)) != cudaSuccess) return e;
    if ((e = upload(S.dnh_slot_grp, S.dn_hop.slot_grp)) != cudaSuccess) return e;
    {
      // the permutation and its inverse (the permutation kernel gathers both ways)
      const std::vector<int32_t>& o = S.dn_hop.order;
      std::vector<int32_t> oi(2 * o.size());
      for (size_t i = 0; i < o.size(); ++i) {
        oi[i] = o[i];
        oi[o.size() + (size_t)o[i]] = (int32_t)i;
      }
      if ((e = upload(S.dn_order, oi)) != cudaSuccess) return e;
    }
    if (!packed_copy(S.dn_hop.ell, 32, &pk)) return cudaErrorInvalidValue;
    if ((e = upload(S.dnh_ellp32, pk)) != cudaSuccess) return e;
    if (!packed_copy(S.dn_hop.ell, 16, &pk)) return cudaErrorInvalidValue;
    if ((e = upload(S.dnh_ellpr, pk)) != cudaSuccess) return e;
  }
  if (S.has_eps) {
    if ((e = upload(S.up_eps, S.up.eps_sum)) != cudaSuccess) return e;
    if ((e = upload(S.dn_eps, S.dn.eps_sum)) != cudaSuccess) return e;
    if ((e = upload(S.dnh_eps, S.dn_hop.eps_sum)) != cudaSuccess) return e;
  } else {
    S.up_eps.release();
    S.dn_eps.release();
    S.dnh_eps.release();
  }
  SectorDev& d = S.dev;
  d.dim_up = S.up.dim;
  d.dim_dn = S.dn.dim;
  d.n_up = S.n_up;
  d.n_dn = S.n_dn;
  d.up_off = static_cast<const int32_t*>(S.up_off.p);
  d.up_ent = static_cast<const uint32_t*>(S.up_ent.p);
  d.dn_off = static_cast<const int32_t*>(S.dn_off.p);
  d.dn_ent = static_cast<const uint32_t*>(S.dn_ent.p);
  d.up_word = static_cast<const uint32_t*>(S.up_word.p);
  d.dn_word = static_cast<const uint32_t*>(S.dn_word.p);
  d.up_eps = S.has_eps ? static_cast<const double*>(S.up_eps.p) : nullptr;
  d.dn_eps = S.has_eps ? static_cast<const double*>(S.dn_eps.p) : nullptr;
  d.up_pad_off = static_cast<const int32_t*>(S.up_pad_off.p);
  d.up_pad_ent = static_cast<const uint32_t*>(S.up_pad_ent.p);
  d.up_pad_row = static_cast<const uint32_t*>(S.up_pad_row.p);
  d.up_pad_cs = static_cast<const uint32_t*>(S.up_pad_cs.p);
  d.dn_tslot_off = static_cast<const int32_t*>(S.dn_tslot_off.p);
  d.dn_slot_grp = static_cast<const uint32_t*>(S.dn_slot_grp.p);
  d.up_tslot_off = static_cast<const int32_t*>(S.up_tslot_off.p);
  d.up_slot_grp = static_cast<const uint32_t*>(S.up_slot_grp.p);
  d.up_ell = static_cast<const uint32_t*>(S.up_ell.p);
  d.up_ell16 = static_cast<const uint32_t*>(S.up_ell16.p);
  d.dn_ellp32 = static_cast<const uint32_t*>(S.dn_ellp32.p);
  d.dn_ellpr = static_cast<const uint32_t*>(S.dn_ellpr.p);
  SectorDev& h = S.dev_hop;
  h = d;
  h.dn_off = static_cast<const int32_t*>(S.dnh_off.p);
  h.dn_ent = static_cast<const uint32_t*>(S.dnh_ent.p);
  h.dn_word = static_cast<const uint32_t*>(S.dnh_word.p);
  h.dn_eps = S.has_eps ? static_cast<const double*>(S.dnh_eps.p) : nullptr;
  h.dn_tslot_off = static_cast<const int32_t*>(S.dnh_tslot_off.p);
  h.dn_slot_grp = static_cast<const uint32_t*>(S.dnh_slot_grp.p);
  h.dn_ellp32 = static_cast<const uint32_t*>(S.dnh_ellp32.p);
  h.dn_ellpr = static_cast<const uint32_t*>(S.dnh_ellpr.p);
  S.uploaded = true;
  return cudaSuccess;
}

cudaError_t build_sector_gpu(SectorGPU& S, const LatticeHost& L, int n_up, int n_dn) {
  build_sector_host(S, L, n_up, n_dn);
  return upload_sector(S);
}

ed_status ensure_device(ed_ctx* ctx) {
  if (!ctx->lattice_set) return fail(ctx, ED_ERR_STATE, "ed_set_lattice has not been called");
  if (ctx->sec.uploaded) return ED_OK;
  CK(ctx, cudaGetDevice(&ctx->device));
  if (!ctx->stream) CK(ctx, cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking));
  CK(ctx, upload_sector(ctx->sec));
  return ED_OK;
}

ed_status check_device(ed_ctx* ctx, std::initializer_list<const void*> bufs) {
  int cur = -1;
  CK(ctx, cudaGetDevice(&cur));
  if (device_verdict(ctx->device, cur, -1) == kDeviceWrongCurrent)
    return fail(ctx, ED_ERR_STATE,
                "the context's tables live on device " + std::to_string(ctx->device) +
                    " but device " + std::to_string(cur) +
                    " is current; make that device current first");
  for (const void* p : bufs) {
    if (!p) continue;
    int dev = -1;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) == cudaSuccess) {
      if (a.type == cudaMemoryTypeDevice) dev = a.device;
    } else {
      cudaGetLastError();
    }
    if (device_verdict(ctx->device, cur, dev) == kDeviceForeignBuffer)
      return fail(ctx, ED_ERR_ARG,
                  "a vector lives on device " + std::to_string(dev) +
                      ", the context's tables on device " + std::to_string(ctx->device));
  }
  return ED_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// The device's address of a pinned host buffer mapped into its address space
// (cudaHostAlloc, or cudaHostRegister with mapping), or NULL for any other
// pointer.
static void* mapped_host_ptr(void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Event-based ordering between the caller's stream and the context stream.
cudaError_t join_streams(cudaStream_t from, cudaStream_t to) {
  if (from == to) return cudaSuccess;
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return e;
  e = cudaEventRecord(ev, from);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
  cudaEventDestroy(ev);
  return e;
}

ed_status check_pulse(ed_ctx* ctx, const ed_pulse* pulse) {
  if (!pulse) return ED_OK;
  if (!(std::isfinite(pulse->A0) && std::isfinite(pulse->omega) &&
        std::isfinite(pulse->sigma) && pulse->sigma != 0.0 && std::isfinite(pulse->t0) &&
        std::isfinite(pulse->b)))
    return fail(ctx, ED_ERR_ARG, "pulse parameters not finite or sigma == 0");
  if (pulse->shape != ED_PULSE_SIN_GAUSS && pulse->shape != ED_PULSE_COS_PHASE)
    return fail(ctx, ED_ERR_ARG, "unknown pulse shape");
  return ED_OK;
}

static void pulse_at(const ed_pulse& p, double t, double A[3]) {
  pulse_A(p.shape, p.A0, p.omega, p.sigma, p.t0, p.b, p.dir, t, A);
}

std::vector<double> step_coefficients(const LatticeHost& L, const ed_pulse* pulse,
                                      double t_start, double dt, int n_steps, bool mid) {
  const int ng = 2 * L.n_classes;
  std::vector<double> out((size_t)n_steps * ng * 2);
  for (int n = 0; n < n_steps; ++n) {
    const double t = t_start + (n + (mid ? 0.5 : 0.0)) * dt;
    double A[3] = {0, 0, 0};
    if (pulse) pulse_at(*pulse, t, A);
    group_coefficients(L, A, out.data() + (size_t)n * ng * 2);
  }
  return out;
}

// CFET4 (fourth-order commutator-free exponential propagator, the family
// named in Sec. 3.4; two-exponential form of Alvermann and Fehske, J. Comput.
// Phys. 230, 5930 (2011)): one step t -> t + dt is
//   exp(-i dt (a1 H1 + a2 H2)) exp(-i dt (a2 H1 + a1 H2)),
// H_k = H(t + c_k dt), c_{1,2} = 1/2 -+ sqrt(3)/6, a_{1,2} = (3 -+ 2 sqrt(3))/12.
// Since a1 + a2 = 1/2, each factor equals exp(-i (dt/2) H~) with H~ the full
// diagonal plus hopping coefficients 2 (a c_g(A1) + b c_g(A2)): a Krylov
// sub-step of length dt/2 with combined group coefficients.
SubSteps integrator_substeps(const ed_ctx* ctx, const ed_pulse* pulse, double t_start,
                             double dt, int n_steps) {
  SubSteps r;
  if (ctx->integrator != ED_CFET4) {
    r.coefs = step_coefficients(ctx->lat, pulse, t_start, dt, n_steps, true);
    r.tau = dt;
    r.per_step = 1;
    return r;
  }
  const double s3 = std::sqrt(3.0);
  const double c1 = 0.5 - s3 / 6.0, c2 = 0.5 + s3 / 6.0;
  const double a1 = (3.0 - 2.0 * s3) / 12.0, a2 = (3.0 + 2.0 * s3) / 12.0;
  const int ng = 2 * ctx->lat.n_classes;
  r.coefs.assign((size_t)2 * n_steps * ng * 2, 0.0);
  std::vector<double> g1(ng * 2), g2(ng * 2);
  for (int n = 0; n < n_steps; ++n) {
    const double t = t_start + n * dt;
    double A1[3] = {0, 0, 0}, A2[3] = {0, 0, 0};
    if (pulse) {
      pulse_at(*pulse, t + c1 * dt, A1);
      pulse_at(*pulse, t + c2 * dt, A2);
    }
    group_coefficients(ctx->lat, A1, g1.data());
    group_coefficients(ctx->lat, A2, g2.data());
    double* first = r.coefs.data() + (size_t)(2 * n) * ng * 2;     // a2 H1 + a1 H2
    double* second = r.coefs.data() + (size_t)(2 * n + 1) * ng * 2; // a1 H1 + a2 H2
    for (int k = 0; k < ng * 2; ++k) {
      first[k] = 2.0 * (a2 * g1[k] + a1 * g2[k]);
      second[k] = 2.0 * (a1 * g1[k] + a2 * g2[k]);
    }
  }
  r.tau = 0.5 * dt;
  r.per_step = 2;
  return r;
}

}  // namespace ed

extern "C" {

const char* ed_version(void) { return "hubbard_ed 0.1 (sm_103a)"; }

const char* ed_last_error(const ed_ctx* ctx) {
  if (ctx && !ctx->err.empty()) return ctx->err.c_str();
  return g_last_error.c_str();
}

ed_status ed_build_basis(ed_ctx** out, int Ns, int n_up, int n_dn) {
  if (!out) return fail(nullptr, ED_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (Ns < 1 || Ns > kMaxSites) return fail(nullptr, ED_ERR_UNSUPPORTED, "Ns must be in 1..16");
  if (n_up < 0 || n_up > Ns || n_dn < 0 || n_dn > Ns)
    return fail(nullptr, ED_ERR_ARG, "n_up and n_dn must be in 0..Ns");
  ed_ctx* c = new (std::nothrow) ed_ctx();
  if (!c) return fail(nullptr, ED_ERR_OOM, "host allocation failed");
  c->Ns = Ns;
  c->n_up = n_up;
  c->n_dn = n_dn;
  c->up_words = spin_basis(Ns, n_up);
  c->dn_words = spin_basis(Ns, n_dn);
  c->dim_up = (int64_t)c->up_words.size();
  c->dim_dn = (int64_t)c->dn_words.size();
  *out = c;
  return ED_OK;
}

ed_status ed_dims(const ed_ctx* ctx, int64_t* dim_up, int64_t* dim_dn) {
  if (!ctx || !dim_up || !dim_dn) return fail(nullptr, ED_ERR_ARG, "NULL argument");
  *dim_up = ctx->dim_up;
  *dim_dn = ctx->dim_dn;
  return ED_OK;
}

ed_status ed_get_basis(const ed_ctx* ctx, int spin, uint32_t* words) {
  if (!ctx || !words || (spin != 0 && spin != 1)) return fail(nullptr, ED_ERR_ARG, "bad argument");
  const auto& w = spin == 0 ? ctx->up_words : ctx->dn_words;
  std::memcpy(words, w.data(), w.size() * sizeof(uint32_t));
  return ED_OK;
}

ed_status ed_set_lattice(ed_ctx* ctx, int n_bonds, const int32_t* p, const int32_t* q,
                         const double* t_hop, const double* d, double U, const double* eps) {
  if (!ctx) return fail(nullptr, ED_ERR_ARG, "ctx is NULL");
  LatticeHost L;
  std::string err = make_lattice(L, ctx->Ns, n_bonds, p, q, t_hop, d, U, eps);
  if (!err.empty()) return fail(ctx, ED_ERR_ARG, err);
  ctx->lat = L;
  ctx->lattice_set = false;
  ctx->engine.reset();
  ctx->spec_engine.reset();
  ctx->spec_sectors.clear();
  ctx->plan.valid = false;
  build_sector_host(ctx->sec, ctx->lat, ctx->n_up, ctx->n_dn);
  ctx->lattice_set = true;
  return ED_OK;
}

ed_status ed_set_field(ed_ctx* ctx, const double A[3]) {
  if (!ctx || !A) return fail(nullptr, ED_ERR_ARG, "NULL argument");
  for (int k = 0; k < 3; ++k) {
    if (!std::isfinite(A[k])) return fail(ctx, ED_ERR_ARG, "A is not finite");
    ctx->A[k] = A[k];
  }
  return ED_OK;
}

ed_status ed_get_table(const ed_ctx* ctx, int spin, int32_t* off, uint32_t* ent,
                       int64_t* nnz_out, int32_t* n_classes) {
  if (!ctx || (spin != 0 && spin != 1)) return fail(nullptr, ED_ERR_ARG, "bad argument");
  if (!ctx->lattice_set) return fail(nullptr, ED_ERR_STATE, "lattice not set");
  const SpinTable& T = spin == 0 ? ctx->sec.up : ctx->sec.dn;
  if (nnz_out) *nnz_out = (int64_t)T.ent.size();
  if (n_classes) *n_classes = ctx->lat.n_classes;
  if (off) std::memcpy(off, T.off.data(), T.off.size() * sizeof(int32_t));
  if (ent) std::memcpy(ent, T.ent.data(), T.ent.size() * sizeof(uint32_t));
  return ED_OK;
}

ed_status ed_device_bytes(const ed_ctx* ctx, int64_t* bytes) {
  if (!ctx || !bytes) return fail(nullptr, ED_ERR_ARG, "NULL argument");
  const SectorGPU& S = ctx->sec;
  int64_t b = S.up_off.bytes + S.up_ent.bytes + S.dn_off.bytes + S.dn_ent.bytes +
              S.up_word.bytes + S.dn_word.bytes + S.up_eps.bytes + S.dn_eps.bytes +
              S.up_pad_off.bytes + S.up_pad_ent.bytes + S.up_pad_row.bytes + S.up_pad_cs.bytes +
              S.dn_tslot_off.bytes +
              S.dn_slot_grp.bytes + S.up_tslot_off.bytes + S.up_slot_grp.bytes +
              S.up_ell.bytes + S.up_ell16.bytes +
              S.dn_ellp32.bytes + S.dn_ellpr.bytes + S.dnh_off.bytes + S.dnh_ent.bytes +
              S.dnh_word.bytes + S.dnh_eps.bytes + S.dnh_tslot_off.bytes +
              S.dnh_slot_grp.bytes + S.dnh_ellp32.bytes + S.dnh_ellpr.bytes +
              S.dn_order.bytes;
  if (ctx->engine) b += ctx->engine->device_bytes();
  if (ctx->spec_engine) b += ctx->spec_engine->device_bytes();
  *bytes = b;
  return ED_OK;
}

ed_status ed_set_krylov_tol(ed_ctx* ctx, double tol) {
  if (!ctx) return fail(nullptr, ED_ERR_ARG, "ctx is NULL");
  if (!(tol >= 0.0) || !std::isfinite(tol))
    return fail(ctx, ED_ERR_ARG, "tol must be finite and >= 0");
  ctx->krylov_tol = tol;
  return ED_OK;
}

ed_status ed_set_workspace_limit(ed_ctx* ctx, int64_t bytes) {
  if (!ctx) return fail(nullptr, ED_ERR_ARG, "ctx is NULL");
  if (bytes < 0) return fail(ctx, ED_ERR_ARG, "bytes must be >= 0");
  ctx->workspace_limit = bytes;
  return ED_OK;
}

ed_status ed_set_wait_fault(int withhold_copy, int64_t wait_polls) {
  if (withhold_copy < -1 || wait_polls < 0 || wait_polls > 0xFFFFFFFFll)
    return fail(nullptr, ED_ERR_ARG, "withhold_copy must be >= -1, wait_polls in 0..2^32-1");
  set_wait_fault(withhold_copy, (uint32_t)wait_polls);
  return ED_OK;
}

ed_status ed_set_integrator(ed_ctx* ctx, ed_integrator scheme) {
  if (!ctx) return fail(nullptr, ED_ERR_ARG, "ctx is NULL");
  if (scheme != ED_MIDPOINT && scheme != ED_CFET4)
    return fail(ctx, ED_ERR_ARG, "unknown integrator");
  ctx->integrator = scheme;
  return ED_OK;
}

ed_status ed_step_coefficients(ed_ctx* ctx, const ed_pulse* pulse, double t_start, double dt,
                               int n_steps, double* coef, int* n_sub_out, double* tau) {
  if (!ctx) return fail(nullptr, ED_ERR_ARG, "ctx is NULL");
  if (!ctx->lattice_set) return fail(ctx, ED_ERR_STATE, "ed_set_lattice has not been called");
  if (n_steps < 1 || !std::isfinite(t_start) || !std::isfinite(dt))
    return fail(ctx, ED_ERR_ARG, "n_steps >= 1 and finite t_start, dt required");
  if (ed_status e = check_pulse(ctx, pulse)) return e;
  const SubSteps sub = integrator_substeps(ctx, pulse, t_start, dt, n_steps);
  const int ng = 2 * ctx->lat.n_classes, nb = ctx->lat.n_bonds;
  const int n_sub = n_steps * sub.per_step;
  if (n_sub_out) *n_sub_out = n_sub;
  if (tau) *tau = sub.tau;
  if (!coef) return ED_OK;
  for (int s = 0; s < n_sub; ++s)
    for (int b = 0; b < nb; ++b) {
      // group 2 c: the hop p -> q of bond class c
      const size_t g = ((size_t)s * ng + 2 * (size_t)ctx->lat.bond_class[b]) * 2;
      coef[2 * ((size_t)s * nb + b)] = sub.coefs[g];
      coef[2 * ((size_t)s * nb + b) + 1] = sub.coefs[g + 1];
    }
  return ED_OK;
}

ed_status ed_tridiag_expm(int batch, int n, const double* alpha, const double* beta,
                          double tau, double* y) {
  if (batch < 1 || n < 1 || n > kMaxKrylov)
    return fail(nullptr, ED_ERR_ARG, "batch >= 1 and 1 <= n <= 64 required");
  if (!alpha || !y || (n > 1 && !beta)) return fail(nullptr, ED_ERR_ARG, "NULL argument");
  if (!std::isfinite(tau)) return fail(nullptr, ED_ERR_ARG, "tau is not finite");
  const size_t na = (size_t)batch * n, nbeta = (size_t)batch * (n - 1);
  for (size_t i = 0; i < na; ++i)
    if (!std::isfinite(alpha[i])) return fail(nullptr, ED_ERR_ARG, "alpha is not finite");
  for (size_t i = 0; i < nbeta; ++i)
    if (!std::isfinite(beta[i])) return fail(nullptr, ED_ERR_ARG, "beta is not finite");
  DevMem da, db, dy;
  cudaError_t e = da.alloc(na * sizeof(double));
  if (e == cudaSuccess) e = db.alloc(std::max<size_t>(1, nbeta) * sizeof(double));
  if (e == cudaSuccess) e = dy.alloc(2 * na * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpy(da.p, alpha, na * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && nbeta)
    e = cudaMemcpy(db.p, beta, nbeta * sizeof(double), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = launch_tridiag_expm(static_cast<const double*>(da.p), static_cast<const double*>(db.p),
                            n, tau, static_cast<double*>(dy.p), batch, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(y, dy.p, 2 * na * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "ed_tridiag_expm");
  return ED_OK;
}

int ed_apply_config_count(void) { return apply_config_count(); }

ed_status ed_apply_config_info(int config, int* fp64, int* rows_per_cta,
                               int* pairs_per_thread, int* ctas_per_sm, int* split, int* tma,
                               int* multi_vector) {
  int f, nr, pp, mb, sp, tm, mv;
  if (!apply_config_info(config, &f, &nr, &pp, &mb, &sp, &tm, &mv))
    return fail(nullptr, ED_ERR_ARG, "no apply configuration " + std::to_string(config));
  if (fp64) *fp64 = f;
  if (rows_per_cta) *rows_per_cta = nr;
  if (pairs_per_thread) *pairs_per_thread = pp;
  if (ctas_per_sm) *ctas_per_sm = mb;
  if (split) *split = sp;
  if (tma) *tma = tm;
  if (multi_vector) *multi_vector = mv;
  return ED_OK;
}

ed_status ed_set_apply_config(int config) {
  if (config < -1 || config >= apply_config_count())
    return fail(nullptr, ED_ERR_ARG, "apply configuration must be -1 or a table index");
  set_forced_apply_config(config);
  return ED_OK;
}

ed_status ed_get_apply_config(const ed_ctx* ctx, int* propagate, int* apply) {
  if (!ctx || !propagate || !apply) return fail(nullptr, ED_ERR_ARG, "NULL argument");
  *propagate = ctx->engine ? ctx->engine->apply_config() : -1;
  *apply = ctx->plan.valid ? ctx->plan.shape.cfg : -1;
  return ED_OK;
}

ed_status ed_apply_H(ed_ctx* ctx, const void* v, void* w, ed_dtype dtype, int nvec,
                     void* stream) {
  if (!ctx) return fail(nullptr, ED_ERR_ARG, "ctx is NULL");
  if (ed_status e = ensure_device(ctx)) return e;
  if (!v || !w || nvec < 1) return fail(ctx, ED_ERR_ARG, "v, w must be non-NULL and nvec >= 1");
  if (dtype != ED_C128 && dtype != ED_C64) return fail(ctx, ED_ERR_ARG, "bad dtype");
  if (v == w) return fail(ctx, ED_ERR_ARG, "v and w must not alias");
  if (ed_status e = check_device(ctx, {v, w})) return e;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool fp64 = dtype == ED_C128;
  ApplyPlan& P = ctx->plan;
  const bool same_field = P.A[0] == ctx->A[0] && P.A[1] == ctx->A[1] && P.A[2] == ctx->A[2];
  const int forced = forced_apply_config();
  BatchArgs now;
  init_batch_args(&now);
  const bool same_cfg = (forced < 0 || forced == P.shape.cfg) &&
                        now.wait_limit == P.args.wait_limit &&
                        now.tma_withhold == P.args.tma_withhold;
  if (!(P.valid && P.nvec == nvec && P.v == v && P.w == w && P.fp64 == fp64 && same_field &&
        same_cfg)) {
    if (!is_device_ptr(v) || !is_device_ptr(w))
      return fail(ctx, ED_ERR_ARG, "ed_apply_H needs device pointers");
    P.valid = false;
    const int64_t D = ctx->dim_up * ctx->dim_dn;
    const size_t esz = fp64 ? 16 : 8;
    const int ng = 2 * ctx->lat.n_classes;
    std::vector<VecDev> vd(nvec);
    for (int b = 0; b < nvec; ++b) {
      std::memset(&vd[b], 0, sizeof(VecDev));
      vd[b].sector = 0;
      vd[b].D = D;
      vd[b].x1 = const_cast<char*>(static_cast<const char*>(v)) + (size_t)b * D * esz;
      vd[b].w = static_cast<char*>(w) + (size_t)b * D * esz;
    }
    std::vector<double> cf(std::max(1, ng) * 2, 0.0);
    group_coefficients(ctx->lat, ctx->A, cf.data());
    std::vector<float> cff(cf.begin(), cf.end());
    std::vector<SectorDev> secs = {ctx->sec.dev};
    std::vector<LanczosState> st(nvec);
    std::memset(st.data(), 0, st.size() * sizeof(LanczosState));
    CK(ctx, upload(P.sec, secs));
    CK(ctx, upload(P.vec, vd));
    CK(ctx, upload(P.st, st));
    CK(ctx, P.counters.alloc(sizeof(unsigned) * nvec));
    CK(ctx, cudaMemset(P.counters.p, 0, sizeof(unsigned) * nvec));
    if (fp64) CK(ctx, upload(P.coefs, cf));
    else CK(ctx, upload(P.coefs, cff));
    init_batch_args(&P.args);
    P.args.sec = static_cast<const SectorDev*>(P.sec.p);
    P.args.vec = static_cast<VecDev*>(P.vec.p);
    P.args.st = static_cast<LanczosState*>(P.st.p);
    P.args.apply_map = static_cast<const ApplyBlock*>(P.amap.p);
    P.args.partials = static_cast<double*>(P.partials.p);
    P.args.counters = static_cast<unsigned*>(P.counters.p);
    P.args.coefs = P.coefs.p;
    P.args.n_groups = ng;
    P.args.nvec = nvec;
    P.args.Ns = ctx->Ns;
    P.args.max_dim_dn = (int)ctx->dim_dn;
    P.args.max_dim_up = (int)ctx->dim_up;
    P.args.U = ctx->lat.U;
    ApplyTuneTarget tt;
    tt.fp64 = fp64;
    tt.vec_ok = !fp64 && (ctx->dim_dn % 2 == 0) &&
                ((((uintptr_t)v) | ((uintptr_t)w)) & 15u) == 0;
    tt.tma_ok = (ctx->dim_dn % 2 == 0) && ((((uintptr_t)v) | ((uintptr_t)w)) & 15u) == 0;
    tt.max_dim_up = (int)ctx->dim_up;
    tt.max_dim_dn = (int)ctx->dim_dn;
    tt.n_groups = ng;
    tt.dim_up.assign(nvec, (int)ctx->dim_up);
    tt.dim_dn.assign(nvec, (int)ctx->dim_dn);
    tt.up.assign(nvec, &ctx->sec.up);
    tt.sector.assign(nvec, 0);
    tt.args = P.args;
    std::vector<ApplyBlock> amap, cmap;
    CKS(ctx, tune_apply(tt, s, &P.shape, &amap, &cmap));
    CK(ctx, prepare_apply(fp64, P.shape));
    assign_apply_ranges(amap, P.shape.mv, vd.data(), nvec);
    CK(ctx, upload(P.vec, vd));
    CK(ctx, upload(P.amap, amap));
    CK(ctx, upload(P.cmap, cmap));
    CK(ctx, P.partials.alloc(sizeof(double) * apply_partials_per_block(P.shape) * amap.size()));
    P.args.vec = static_cast<VecDev*>(P.vec.p);
    P.args.apply_map = static_cast<const ApplyBlock*>(P.amap.p);
    P.args.col_map = static_cast<const ApplyBlock*>(P.cmap.p);
    P.args.n_col_blocks = (int)cmap.size();
    P.args.partials = static_cast<double*>(P.partials.p);
    P.nblk = (int)amap.size();
    P.nvec = nvec;
    P.v = v;
    P.w = w;
    P.fp64 = fp64;
    for (int k = 0; k < 3; ++k) P.A[k] = ctx->A[k];
    P.valid = true;
  }
  CK(ctx, launch_apply(fp64, P.args, P.nblk, P.shape, 0, s));
  return ED_OK;
}

ed_status ed_propagate(ed_ctx* ctx, void* psi, ed_dtype dtype, const ed_pulse* pulse,
                       double t_start, double dt, int n_steps, int m,
                       const ed_observables* obs, void* stream) {
  if (!ctx) return fail(nullptr, ED_ERR_ARG, "ctx is NULL");
  if (!ctx->lattice_set) return fail(ctx, ED_ERR_STATE, "ed_set_lattice has not been called");
  if (!psi) return fail(ctx, ED_ERR_ARG, "psi is NULL");
  if (dtype != ED_C128 && dtype != ED_C64) return fail(ctx, ED_ERR_ARG, "bad dtype");
  if (n_steps < 0) return fail(ctx, ED_ERR_ARG, "n_steps < 0");
  if (m < 1) return fail(ctx, ED_ERR_ARG, "m < 1");
  if (m > kMaxKrylov) return fail(ctx, ED_ERR_UNSUPPORTED, "m > 64");
  if (!std::isfinite(dt) || !std::isfinite(t_start)) return fail(ctx, ED_ERR_ARG, "dt/t_start not finite");
  if (ed_status e = check_pulse(ctx, pulse)) return e;
  if (ed_status e = ensure_device(ctx)) return e;
  if (ed_status e = check_device(ctx, {psi})) return e;
  cudaStream_t us = static_cast<cudaStream_t>(stream);
  cudaStream_t s = ctx->stream;
  const bool fp64 = dtype == ED_C128;
  const int64_t D = ctx->dim_up * ctx->dim_dn;
  const size_t esz = fp64 ? 16 : 8;
  const bool on_device = is_device_ptr(psi);
  const bool energy = obs && obs->energy;
  const bool profile = obs && obs->profile;

  const SubSteps sub = integrator_substeps(ctx, pulse, t_start, dt, n_steps);
  const int per = sub.per_step;
  const int n_sub = n_steps * per;

  EngineConfig cfg;
  cfg.fp64 = fp64;
  cfg.m = m;
  cfg.energy = energy;
  cfg.n_steps_cap = std::max(1, n_sub);
  cfg.eps_tol = ctx->krylov_tol;
  cfg.workspace_limit = ctx->workspace_limit;
  std::vector<EngineVector> vecs = {{0, D, on_device ? psi : nullptr, !on_device}};
  CK(ctx, join_streams(us, s));
  if (!ctx->engine || !ctx->engine->compatible(cfg, vecs)) {
    ctx->engine.reset(new Engine());
    cfg.n_steps_cap = std::max(cfg.n_steps_cap, 64);
    // the engine runs on the hop-ordered down-spin tables (fewer padded ELL
    // slots): the state's columns are permuted into that order for the call
    std::string err = ctx->engine->setup(cfg, {ctx->sec.dev_hop}, vecs, 2 * ctx->lat.n_classes,
                                         ctx->Ns, ctx->lat.U, fp64 ? 1e-13 : 1e-6, s,
                                         {&ctx->sec.up});
    if (!err.empty()) {
      ctx->engine.reset();
      return fail(ctx, err.find("memory") != std::string::npos ? ED_ERR_OOM : ED_ERR_CUDA, err);
    }
  }
  Engine& E = *ctx->engine;
  void* x1 = E.vec_x1(0);
  const int32_t* order = static_cast<const int32_t*>(ctx->sec.dn_order.p);
  // A pinned host state is read (and at the end written) by the permutation
  // kernel itself, in the same pass that puts its columns into hop order;
  // other host memory goes through a copy and the in-place permutation.
  void* host_dev = on_device ? nullptr : mapped_host_ptr(psi);
  if (host_dev) {
    CK(ctx, launch_permute_cols_copy(fp64, host_dev, x1, (int)ctx->dim_up, (int)ctx->dim_dn,
                                     order, true, s));
  } else {
    if (!on_device) CK(ctx, cudaMemcpyAsync(x1, psi, D * esz, cudaMemcpyHostToDevice, s));
    CK(ctx, launch_permute_cols(fp64, x1, (int)ctx->dim_up, (int)ctx->dim_dn, order, true, s));
  }
  int status = 0;
  // the steps; the state's columns go back to ascending-word order whatever
  // they return
  const ed_status run_st = [&]() -> ed_status {
  // energy at the time-step boundaries t_start + k dt / per of the sub-steps
  // (only every per-th entry, a whole time step, is reported)
  std::vector<double> coefs_obs;
  if (energy)
    coefs_obs = step_coefficients(ctx->lat, pulse, t_start, dt / per, n_sub + 1, false);
  CKS(ctx, E.begin(sub.coefs, coefs_obs, n_sub, sub.tau, s));
  CKS(ctx, E.run(n_sub, profile, obs ? obs->kernel_ms : nullptr,
                 obs ? obs->kernel_launches : nullptr, s));
  if (per == 1) {
    CKS(ctx, E.fetch(0, n_steps, obs ? obs->docc : nullptr, obs ? obs->norm2 : nullptr,
                     energy ? obs->energy : nullptr, obs ? obs->delta : nullptr,
                     obs ? obs->m_eff : nullptr, &status, s));
  } else {
    std::vector<double> d(n_sub + 1), n2(n_sub + 1), en(n_sub + 1), dl(std::max(1, n_sub));
    std::vector<int32_t> me(std::max(1, n_sub));
    CKS(ctx, E.fetch(0, n_sub, d.data(), n2.data(), energy ? en.data() : nullptr, dl.data(),
                     me.data(), &status, s));
    if (obs) {
      for (int n = 0; n <= n_steps; ++n) {
        if (obs->docc) obs->docc[n] = d[(size_t)n * per];
        if (obs->norm2) obs->norm2[n] = n2[(size_t)n * per];
        if (energy) obs->energy[n] = en[(size_t)n * per];
      }
      for (int n = 0; n < n_steps; ++n) {
        double dmax = 0.0;
        int mmax = 0;
        for (int k = 0; k < per; ++k) {
          dmax = std::max(dmax, dl[(size_t)n * per + k]);
          mmax = std::max(mmax, me[(size_t)n * per + k]);
        }
        if (obs->delta) obs->delta[n] = dmax;
        if (obs->m_eff) obs->m_eff[n] = mmax;
      }
    }
  }
  return ED_OK;
  }();
  const cudaError_t pe =
      host_dev ? launch_permute_cols_copy(fp64, x1, host_dev, (int)ctx->dim_up,
                                          (int)ctx->dim_dn, order, false, s)
               : launch_permute_cols(fp64, x1, (int)ctx->dim_up, (int)ctx->dim_dn, order, false, s);
  if (host_dev) {
    // the permutation kernel writes psi: done before the call returns, also
    // on an error
    const cudaError_t se = cudaStreamSynchronize(s);
    if (run_st != ED_OK) return run_st;
    CK(ctx, pe);
    CK(ctx, se);
  } else {
    if (run_st != ED_OK) return run_st;
    CK(ctx, pe);
    if (!on_device) {
      CK(ctx, cudaMemcpyAsync(psi, x1, D * esz, cudaMemcpyDeviceToHost, s));
      CK(ctx, cudaStreamSynchronize(s));
    }
  }
  CK(ctx, join_streams(s, us));
  if (status == ED_ERR_TIMEOUT)
    return fail(ctx, ED_ERR_TIMEOUT, "a bounded device-side wait of the apply kernel gave up");
  if (status != 0) return fail(ctx, ED_ERR_NUMERIC, "non-finite norm or inner product during propagation");
  return ED_OK;
}

ed_status ed_double_occupation(ed_ctx* ctx, const void* psi, ed_dtype dtype, double* d_avg,
                               double* d_site) {
  if (!ctx || !psi || !d_avg) return fail(ctx, ED_ERR_ARG, "NULL argument");
  if (dtype != ED_C128 && dtype != ED_C64) return fail(ctx, ED_ERR_ARG, "bad dtype");
  if (ed_status e = ensure_device(ctx)) return e;
  if (ed_status e = check_device(ctx, {psi})) return e;
  const bool fp64 = dtype == ED_C128;
  const int64_t D = ctx->dim_up * ctx->dim_dn;
  const size_t esz = fp64 ? 16 : 8;
  cudaStream_t s = ctx->stream;
  DevMem tmp, part, out;
  const void* p = psi;
  if (!is_device_ptr(psi)) {
    CK(ctx, tmp.alloc(D * esz));
    CK(ctx, cudaMemcpyAsync(tmp.p, psi, D * esz, cudaMemcpyHostToDevice, s));
    p = tmp.p;
  }
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(1216, (D + 1023) / 1024));
  CK(ctx, part.alloc(sizeof(double) * (kMaxSites + 1) * nblk));
  CK(ctx, out.alloc(sizeof(double) * (kMaxSites + 1)));
  CK(ctx, launch_docc_sites(fp64, p, &ctx->sec.dev, (int)ctx->dim_up, (int)ctx->dim_dn, ctx->Ns,
                            static_cast<double*>(part.p), nblk, static_cast<double*>(out.p), s));
  double h[kMaxSites + 1];
  CK(ctx, cudaMemcpyAsync(h, out.p, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  *d_avg = h[0] / ctx->Ns;
  if (d_site)
    for (int i = 0; i < ctx->Ns; ++i) d_site[i] = h[1 + i];
  return ED_OK;
}

ed_status ed_apply_fermion_op(ed_ctx* ctx, ed_ctx* dst, int site, int spin, int create,
                              const void* psi, void* out, ed_dtype dtype, void* stream) {
  if (!ctx || !dst || !psi || !out) return fail(ctx, ED_ERR_ARG, "NULL argument");
  if (site < 0 || site >= ctx->Ns || (spin != 0 && spin != 1))
    return fail(ctx, ED_ERR_ARG, "bad site or spin");
  const int dn = create ? 1 : -1;
  const int tu = ctx->n_up + (spin == 0 ? dn : 0), td = ctx->n_dn + (spin == 1 ? dn : 0);
  if (dst->Ns != ctx->Ns || dst->n_up != tu || dst->n_dn != td)
    return fail(ctx, ED_ERR_ARG, "destination context has the wrong sector");
  if (dtype != ED_C128 && dtype != ED_C64) return fail(ctx, ED_ERR_ARG, "bad dtype");
  if (ed_status e = ensure_device(ctx)) return e;
  if (!is_device_ptr(psi) || !is_device_ptr(out))
    return fail(ctx, ED_ERR_ARG, "device pointers required");
  if (ed_status e = check_device(ctx, {psi, out})) return e;
  std::vector<int32_t> map = fermion_map(ctx->Ns, ctx->n_up, ctx->n_dn, site, spin, create != 0);
  DevMem dmap;
  CK(ctx, upload(dmap, map));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  CK(ctx, launch_fermion_op(dtype == ED_C128, psi, out, (int)ctx->dim_up, (int)ctx->dim_dn,
                            (int)dst->dim_up, (int)dst->dim_dn, spin,
                            static_cast<const int32_t*>(dmap.p), s));
  CK(ctx, cudaStreamSynchronize(s));  // map buffer is freed on return
  return ED_OK;
}

ed_status ed_destroy(ed_ctx* ctx) {
  if (!ctx) return ED_OK;
  ctx->engine.reset();
  ctx->spec_engine.reset();
  ctx->spec_sectors.clear();
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
  return ED_OK;
}

}  // extern "C"
