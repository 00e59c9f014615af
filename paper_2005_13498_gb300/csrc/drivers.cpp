// Drivers of ed_ground_state and ed_spectral_propagate.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "ctx.h"

using namespace ed;

namespace {

// Number of eigenvalues of the symmetric tridiagonal T(a, b) below x
// (Sturm count from the signs of the pivots of the LDL^T factorisation of
// T - x I).
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  int cnt = 0;
  double q = 1.0;
  const double tiny = 1e-300;
  for (size_t i = 0; i < a.size(); ++i) {
    const double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
    q = (a[i] - x) - (i > 0 ? bb / q : 0.0);
    if (q == 0.0) q = -tiny;
    if (q < 0.0) ++cnt;
  }
  return cnt;
}

// Lowest eigenpair of T(a, b) by bisection on the Sturm count and inverse
// iteration with a partially pivoted tridiagonal solve.
void lowest_eigenpair(const std::vector<double>& a, const std::vector<double>& b,
                      double* theta, std::vector<double>& s) {
  const int n = (int)a.size();
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < n; ++i) {
    const double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (sturm_count(a, b, mid) >= 1) hi = mid; else lo = mid;
  }
  const double th = 0.5 * (lo + hi);
  *theta = th;
  // inverse iteration: solve (T - th I) x = s three times, s normalised
  s.assign(n, 1.0 / std::sqrt((double)n));
  const double scale = std::max(1.0, std::max(std::fabs(lo), std::fabs(hi)));
  const double shift = th - 1e-14 * scale;  // keep the system nonsingular
  for (int rep = 0; rep < 3; ++rep) {
    // Gaussian elimination with partial pivoting on the tridiagonal system;
    // U has up to two super-diagonals.
    std::vector<double> d(n), du(n, 0.0), du2(n, 0.0), dl(n, 0.0), x = s;
    for (int i = 0; i < n; ++i) d[i] = a[i] - shift;
    for (int i = 0; i < n - 1; ++i) { du[i] = b[i]; dl[i] = b[i]; }
    for (int i = 0; i < n - 1; ++i) {
      if (std::fabs(d[i]) >= std::fabs(dl[i])) {
        const double piv = d[i] != 0.0 ? d[i] : 1e-300;
        const double f = dl[i] / piv;
        d[i + 1] -= f * du[i];
        x[i + 1] -= f * x[i];
        dl[i] = 0.0;
      } else {
        // swap rows i and i+1
        const double f = d[i] / dl[i];
        d[i] = dl[i];
        const double t1 = d[i + 1];
        d[i + 1] = du[i] - f * t1;
        if (i < n - 2) {
          du2[i] = du[i + 1];
          du[i + 1] = -f * du2[i];
        }
        du[i] = t1;
        const double tx = x[i];
        x[i] = x[i + 1];
        x[i + 1] = tx - f * x[i + 1];
      }
    }
    if (d[n - 1] == 0.0) d[n - 1] = 1e-300;
    x[n - 1] /= d[n - 1];
    if (n > 1) x[n - 2] = (x[n - 2] - du[n - 2] * x[n - 1]) / d[n - 2];
    for (int i = n - 3; i >= 0; --i)
      x[i] = (x[i] - du[i] * x[i + 1] - du2[i] * x[i + 2]) / d[i];
    double nrm = 0.0;
    for (double v : x) nrm += v * v;
    nrm = std::sqrt(nrm);
    for (int i = 0; i < n; ++i) s[i] = x[i] / nrm;
  }
}

struct GsApply {
  DevMem sec, vec, st, amap, cmap, partials, counters, coefs;
  BatchArgs args{};
  LaunchShape shape{};
  int nblk = 0;
};

// x, w: device buffers of length D the autotuner may read and overwrite.
std::string gs_apply_setup(GsApply& G, ed_ctx* ctx, const double2* x, double2* w,
                           cudaStream_t s) {
  // hop-ordered down-spin tables: the Lanczos vectors keep their columns in
  // that order, and the result goes back to ascending-word order at the end
  std::vector<SectorDev> secs = {ctx->sec.dev_hop};
  std::vector<VecDev> vd(1);
  std::memset(vd.data(), 0, sizeof(VecDev));
  vd[0].D = ctx->dim_up * ctx->dim_dn;
  vd[0].x1 = const_cast<double2*>(x);
  vd[0].w = w;
  const int ng = 2 * ctx->lat.n_classes;
  std::vector<double> cf(std::max(1, ng) * 2, 0.0);
  const double A0[3] = {0, 0, 0};
  group_coefficients(ctx->lat, A0, cf.data());
  std::vector<LanczosState> st(1);
  std::memset(st.data(), 0, sizeof(LanczosState));
  ED_TRY(upload(G.sec, secs));
  ED_TRY(upload(G.vec, vd));
  ED_TRY(upload(G.st, st));
  ED_TRY(upload(G.coefs, cf));
  ED_TRY(G.counters.alloc(sizeof(unsigned)));
  ED_TRY(cudaMemset(G.counters.p, 0, sizeof(unsigned)));
  init_batch_args(&G.args);
  G.args.sec = static_cast<const SectorDev*>(G.sec.p);
  G.args.vec = static_cast<VecDev*>(G.vec.p);
  G.args.st = static_cast<LanczosState*>(G.st.p);
  G.args.counters = static_cast<unsigned*>(G.counters.p);
  G.args.coefs = G.coefs.p;
  G.args.n_groups = ng;
  G.args.nvec = 1;
  G.args.Ns = ctx->Ns;
  G.args.max_dim_dn = (int)ctx->dim_dn;
  G.args.max_dim_up = (int)ctx->dim_up;
  G.args.U = ctx->lat.U;
  ApplyTuneTarget tt;
  tt.fp64 = true;
  tt.vec_ok = false;
  tt.tma_ok = (ctx->dim_dn % 2 == 0) && ((((uintptr_t)x) | ((uintptr_t)w)) & 15u) == 0;
  tt.max_dim_up = (int)ctx->dim_up;
  tt.max_dim_dn = (int)ctx->dim_dn;
  tt.n_groups = ng;
  tt.dim_up = {(int)ctx->dim_up};
  tt.dim_dn = {(int)ctx->dim_dn};
  tt.up = {&ctx->sec.up};
  tt.sector = {0};
  tt.args = G.args;
  std::vector<ApplyBlock> amap, cmap;
  std::string err = tune_apply(tt, s, &G.shape, &amap, &cmap);
  if (!err.empty()) return err;
  assign_apply_ranges(amap, G.shape.mv, vd.data(), 1);
  ED_TRY(upload(G.vec, vd));
  ED_TRY(upload(G.amap, amap));
  ED_TRY(upload(G.cmap, cmap));
  ED_TRY(G.partials.alloc(sizeof(double) * apply_partials_per_block(G.shape) * amap.size()));
  G.args.vec = static_cast<VecDev*>(G.vec.p);
  G.args.apply_map = static_cast<const ApplyBlock*>(G.amap.p);
  G.args.col_map = static_cast<const ApplyBlock*>(G.cmap.p);
  G.args.n_col_blocks = (int)cmap.size();
  G.args.partials = static_cast<double*>(G.partials.p);
  G.nblk = (int)amap.size();
  ED_TRY(prepare_apply(true, G.shape));
  return "";
}

cudaError_t gs_apply(GsApply& G, const double2* x, double2* w, cudaStream_t s) {
  VecDev vd;
  cudaError_t e = cudaMemcpyAsync(&vd, G.vec.p, sizeof(VecDev), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  vd.x1 = const_cast<double2*>(x);
  vd.w = w;
  if ((e = cudaMemcpyAsync(G.vec.p, &vd, sizeof(VecDev), cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return e;
  if ((e = launch_apply(true, G.args, G.nblk, G.shape, 0, s)) != cudaSuccess) return e;
  return cudaStreamSynchronize(s);  // vd is a host temporary
}

}  // namespace

extern "C" {

ed_status ed_ground_state(ed_ctx* ctx, void* psi, double* E0, double tol, int max_iter,
                          uint64_t seed, double* resid_out) {
  if (!ctx || !psi || !E0) return fail(ctx, ED_ERR_ARG, "NULL argument");
  if (ed_status e = ensure_device(ctx)) return e;
  if (!(tol > 0.0) || max_iter < 1) return fail(ctx, ED_ERR_ARG, "tol must be > 0, max_iter >= 1");
  if (ed_status e = check_device(ctx, {psi})) return e;
  cudaStream_t s = ctx->stream;
  const int64_t D = ctx->dim_up * ctx->dim_dn;
  // Krylov subspace size per restart, bounded by memory and by the multi-dot
  size_t free_b = 0, total_b = 0;
  CK(ctx, cudaMemGetInfo(&free_b, &total_b));
  int64_t kfit = (int64_t)(0.5 * (double)free_b / ((double)D * 16.0)) - 4;
  // V holds K + 1 vectors, w and y one each
  if (ctx->workspace_limit > 0)
    kfit = std::min<int64_t>(kfit, ctx->workspace_limit / ((int64_t)D * 16) - 3);
  int K = (int)std::min<int64_t>(std::min<int64_t>(200, kfit), D);
  K = std::min(K, max_iter);
  if (K < 2 && D > 1)
    return fail(ctx, ED_ERR_OOM,
                "not enough device memory (or workspace limit) for two Lanczos vectors");
  if (D == 1) K = 1;
  DevMem V, w, y, part, red, cvec, cdev, sdev;
  CK(ctx, V.alloc((size_t)(K + 1) * D * 16));
  CK(ctx, w.alloc((size_t)D * 16));
  CK(ctx, y.alloc((size_t)D * 16));
  const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>(1216, (D + 2047) / 2048));
  CK(ctx, part.alloc(sizeof(double2) * (size_t)nblk * (K + 1)));
  CK(ctx, red.alloc(sizeof(double) * 2));
  CK(ctx, cdev.alloc(sizeof(double2) * (K + 1)));
  CK(ctx, sdev.alloc(sizeof(double) * (K + 1)));
  GsApply G;
  CKS(ctx, gs_apply_setup(G, ctx, static_cast<const double2*>(V.p),
                         static_cast<double2*>(w.p), s));
  double2* Vp = static_cast<double2*>(V.p);
  double2* wp = static_cast<double2*>(w.p);
  double2* yp = static_cast<double2*>(y.p);
  double* redp = static_cast<double*>(red.p);
  auto vk = [&](int k) { return Vp + (size_t)k * D; };
  auto norm_dot = [&](const double2* a, const double2* b, double out[2]) -> cudaError_t {
    cudaError_t e = launch_norm_dot(a, b, D, static_cast<double*>(part.p), nblk, redp, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(out, redp, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
  };
  // seeded start vector, normalised
  CK(ctx, launch_random_fill(vk(0), D, seed, s));
  double nd[2];
  CK(ctx, norm_dot(vk(0), nullptr, nd));
  CK(ctx, cudaMemcpyAsync(redp, &nd[0], sizeof(double), cudaMemcpyHostToDevice, s));
  CK(ctx, launch_scale(vk(0), D, redp, true, s));
  int applies = 0;
  double theta = 0.0, resid = 1e300;
  std::vector<double> al, be, sv;
  bool converged = false;
  while (applies < max_iter && !converged) {
    al.clear();
    be.clear();
    int k = 0;
    for (; k < K; ++k) {
      CK(ctx, gs_apply(G, vk(k), wp, s));
      ++applies;
      CK(ctx, norm_dot(vk(k), wp, nd));
      const double a = nd[1];
      al.push_back(a);
      double tmp = a;
      CK(ctx, cudaMemcpyAsync(redp, &tmp, sizeof(double), cudaMemcpyHostToDevice, s));
      CK(ctx, launch_axpy_real(wp, vk(k), D, redp, -1.0, s));
      if (k > 0) {
        double bprev = be.back();
        CK(ctx, cudaMemcpyAsync(redp + 1, &bprev, sizeof(double), cudaMemcpyHostToDevice, s));
        CK(ctx, launch_axpy_real(wp, vk(k - 1), D, redp + 1, -1.0, s));
      }
      // full reorthogonalisation, classical Gram-Schmidt applied twice
      for (int pass = 0; pass < 2; ++pass) {
        CK(ctx, launch_multidot(vk(0), D, k + 1, wp, D, static_cast<double2*>(part.p), nblk, s));
        CK(ctx, launch_reduce_cols(static_cast<double2*>(part.p), nblk, k + 1,
                                   static_cast<double2*>(cdev.p), s));
        CK(ctx, launch_multiaxpy(vk(0), D, k + 1, static_cast<double2*>(cdev.p), wp, D, s));
      }
      CK(ctx, norm_dot(wp, nullptr, nd));
      const double b = std::sqrt(nd[0]);
      be.push_back(b);
      lowest_eigenpair(al, be, &theta, sv);
      const double est = b * std::fabs(sv.back());
      const double sc = std::max(1.0, std::fabs(theta));
      if (est <= 0.1 * tol * sc || b <= 1e-14 * sc || k + 1 == K || applies >= max_iter) {
        ++k;
        break;
      }
      CK(ctx, cudaMemcpyAsync(vk(k + 1), wp, (size_t)D * 16, cudaMemcpyDeviceToDevice, s));
      CK(ctx, cudaMemcpyAsync(redp, &nd[0], sizeof(double), cudaMemcpyHostToDevice, s));
      CK(ctx, launch_scale(vk(k + 1), D, redp, true, s));
    }
    // Ritz vector y = V s, normalised
    CK(ctx, cudaMemcpyAsync(sdev.p, sv.data(), sizeof(double) * sv.size(), cudaMemcpyHostToDevice, s));
    CK(ctx, launch_combine_real(vk(0), D, (int)sv.size(), static_cast<double*>(sdev.p), yp, D, s));
    CK(ctx, norm_dot(yp, nullptr, nd));
    CK(ctx, cudaMemcpyAsync(redp, &nd[0], sizeof(double), cudaMemcpyHostToDevice, s));
    CK(ctx, launch_scale(yp, D, redp, true, s));
    // true residual |H y - theta' y| with theta' = <y, H y>
    CK(ctx, gs_apply(G, yp, wp, s));
    ++applies;
    CK(ctx, norm_dot(yp, wp, nd));
    theta = nd[1];
    double mth = theta;
    CK(ctx, cudaMemcpyAsync(redp, &mth, sizeof(double), cudaMemcpyHostToDevice, s));
    CK(ctx, launch_axpy_real(wp, yp, D, redp, -1.0, s));
    CK(ctx, norm_dot(wp, nullptr, nd));
    resid = std::sqrt(nd[0]);
    converged = resid <= tol * std::max(1.0, std::fabs(theta));
    // restart from the Ritz vector
    CK(ctx, cudaMemcpyAsync(vk(0), yp, (size_t)D * 16, cudaMemcpyDeviceToDevice, s));
  }
  // columns back to ascending-word order, then the phase fix on the host:
  // largest-magnitude element real and positive
  CK(ctx, launch_permute_cols(true, yp, (int)ctx->dim_up, (int)ctx->dim_dn,
                              static_cast<const int32_t*>(ctx->sec.dn_order.p), false, s));
  std::vector<std::complex<double>> h(D);
  CK(ctx, cudaMemcpyAsync(h.data(), yp, (size_t)D * 16, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  int64_t kmax = 0;
  double amax = -1.0;
  for (int64_t i = 0; i < D; ++i) {
    const double a = std::abs(h[i]);
    if (a > amax) { amax = a; kmax = i; }
  }
  const std::complex<double> ph = std::conj(h[kmax]) / std::abs(h[kmax]);
  for (auto& z : h) z *= ph;
  h[kmax] = std::complex<double>(std::abs(h[kmax]), 0.0);
  if (is_device_ptr(psi))
    CK(ctx, cudaMemcpy(psi, h.data(), (size_t)D * 16, cudaMemcpyHostToDevice));
  else
    std::memcpy(psi, h.data(), (size_t)D * 16);
  *E0 = theta;
  if (resid_out) *resid_out = resid;
  if (!std::isfinite(theta) || !std::isfinite(resid))
    return fail(ctx, ED_ERR_NUMERIC, "non-finite ground-state estimate");
  return ED_OK;
}

ed_status ed_spectral_propagate(ed_ctx* ctx, const void* psi0, ed_dtype dtype,
                                const ed_pulse* pulse, double dt, int n_steps, int m,
                                double* G_less, double* G_great, void* stream) {
  return ed_spectral_propagate_at(ctx, psi0, 0.0, dtype, pulse, dt, n_steps, m, G_less,
                                  G_great, stream);
}

ed_status ed_spectral_propagate_at(ed_ctx* ctx, const void* psi0, double t_ref,
                                   ed_dtype dtype, const ed_pulse* pulse, double dt,
                                   int n_steps, int m, double* G_less, double* G_great,
                                   void* stream) {
  if (!ctx || !psi0 || !G_less || !G_great) return fail(ctx, ED_ERR_ARG, "NULL argument");
  if (!ctx->lattice_set) return fail(ctx, ED_ERR_STATE, "ed_set_lattice has not been called");
  if (dtype != ED_C128 && dtype != ED_C64) return fail(ctx, ED_ERR_ARG, "bad dtype");
  if (n_steps < 0 || m < 1) return fail(ctx, ED_ERR_ARG, "n_steps >= 0 and m >= 1 required");
  if (m > kMaxKrylov) return fail(ctx, ED_ERR_UNSUPPORTED, "m > 64");
  if (!std::isfinite(dt) || !std::isfinite(t_ref)) return fail(ctx, ED_ERR_ARG, "dt/t_ref not finite");
  if (ed_status e = check_pulse(ctx, pulse)) return e;
  if (ed_status e = ensure_device(ctx)) return e;
  if (ed_status e = check_device(ctx, {psi0})) return e;
  cudaStream_t us = static_cast<cudaStream_t>(stream);
  cudaStream_t s = ctx->stream;
  const bool fp64 = dtype == ED_C128;
  const int Ns = ctx->Ns;
  // sector list: 0 = N, then the N -+ 1 sectors the phi vectors live in.  A
  // down-spin phi of sector (n_up, n_dn -+ 1) is stored transposed, as a
  // vector of the swapped sector (n_dn -+ 1, n_up): T_up and T_dn depend only
  // on the particle number, so the Hamiltonian of the swapped sector is the
  // same operator on the transposed matrix.  Its rows then have the length
  // C(Ns, n_up) of the up-spin phi's rows, and at half filling the two
  // operators of one kind share one sector (rows of an even length keep the
  // 16-byte accesses of the apply for every vector of the batch).
  struct Target { int n_up, n_dn; };
  const Target tg[4] = {{ctx->n_up - 1, ctx->n_dn}, {ctx->n_dn - 1, ctx->n_up},
                        {ctx->n_up + 1, ctx->n_dn}, {ctx->n_dn + 1, ctx->n_up}};
  auto exists = [&](const Target& t) {
    return t.n_up >= 0 && t.n_up <= Ns && t.n_dn >= 0 && t.n_dn <= Ns;
  };
  // k aliases the first j < k with the same sector (or is itself the first)
  int first_of[4];
  for (int k = 0; k < 4; ++k) {
    first_of[k] = k;
    for (int j = 0; j < k; ++j)
      if (tg[j].n_up == tg[k].n_up && tg[j].n_dn == tg[k].n_dn) { first_of[k] = j; break; }
  }
  int sector_of[4];
  std::vector<SectorDev> secs = {ctx->sec.dev};
  std::vector<const SpinTable*> up_tabs = {&ctx->sec.up};
  if (ctx->spec_sectors.empty()) {
    for (int k = 0; k < 4; ++k) {
      std::unique_ptr<SectorGPU> S;
      if (exists(tg[k]) && first_of[k] == k) {
        S.reset(new SectorGPU());
        CK(ctx, build_sector_gpu(*S, ctx->lat, tg[k].n_up, tg[k].n_dn));
      }
      ctx->spec_sectors.push_back(std::move(S));
    }
  }
  for (int k = 0; k < 4; ++k) {
    if (!exists(tg[k])) {
      sector_of[k] = -1;
    } else if (first_of[k] != k) {
      sector_of[k] = sector_of[first_of[k]];
    } else {
      sector_of[k] = (int)secs.size();
      secs.push_back(ctx->spec_sectors[k]->dev);
      up_tabs.push_back(&ctx->spec_sectors[k]->up);
    }
  }
  // vectors: psi, then for op (0: c, 1: c^+), spin, site; map mode 0 (row
  // map) for the up spin, 2 (column map, vector stored transposed) for down
  struct Phi { int op, spin, site, vec; };
  std::vector<Phi> phis;
  std::vector<EngineVector> vecs = {{0, ctx->dim_up * ctx->dim_dn, nullptr, true}};
  std::vector<int32_t> maps;
  std::vector<int64_t> moff = {-1};
  std::vector<int32_t> mspin = {0};
  for (int op = 0; op < 2; ++op)
    for (int spin = 0; spin < 2; ++spin) {
      const int k = op * 2 + spin;
      if (sector_of[k] < 0) continue;
      const SectorDev& sd = secs[sector_of[k]];
      for (int site = 0; site < Ns; ++site) {
        phis.push_back({op, spin, site, (int)vecs.size()});
        vecs.push_back({sector_of[k], (int64_t)sd.dim_up * sd.dim_dn, nullptr, true});
        std::vector<int32_t> mp = fermion_map(Ns, ctx->n_up, ctx->n_dn, site, spin, op == 1);
        moff.push_back((int64_t)maps.size());
        mspin.push_back(spin == 0 ? 0 : 2);
        maps.insert(maps.end(), mp.begin(), mp.end());
      }
    }
  EngineConfig cfg;
  cfg.fp64 = fp64;
  cfg.m = m;
  cfg.overlaps = true;
  const SubSteps sub = integrator_substeps(ctx, pulse, t_ref, dt, n_steps);
  const int per = sub.per_step;
  const int n_sub = n_steps * per;
  cfg.n_steps_cap = std::max(1, n_sub);
  cfg.eps_tol = ctx->krylov_tol;
  cfg.workspace_limit = ctx->workspace_limit;
  CK(ctx, join_streams(us, s));
  if (!ctx->spec_engine || !ctx->spec_engine->compatible(cfg, vecs)) {
    ctx->spec_engine.reset(new Engine());
    cfg.n_steps_cap = std::max(cfg.n_steps_cap, 64);
    std::string err = ctx->spec_engine->setup(cfg, secs, vecs, 2 * ctx->lat.n_classes, Ns,
                                              ctx->lat.U, fp64 ? 1e-13 : 1e-6, s, up_tabs);
    if (!err.empty()) {
      ctx->spec_engine.reset();
      return fail(ctx, err.find("memory") != std::string::npos ? ED_ERR_OOM : ED_ERR_CUDA, err);
    }
    CKS(ctx, ctx->spec_engine->set_overlap_maps(maps, moff, mspin, 0, s));
  }
  Engine& E = *ctx->spec_engine;
  // psi (converted to the propagation dtype), then phi = op psi
  const int64_t D0 = ctx->dim_up * ctx->dim_dn;
  DevMem tmp;
  const void* p0 = psi0;
  if (!is_device_ptr(psi0)) {
    CK(ctx, tmp.alloc((size_t)D0 * 16));
    CK(ctx, cudaMemcpyAsync(tmp.p, psi0, (size_t)D0 * 16, cudaMemcpyHostToDevice, s));
    p0 = tmp.p;
  }
  CK(ctx, launch_convert(p0, true, E.vec_x1(0), fp64, D0, s));
  DevMem dmaps;
  CK(ctx, upload(dmaps, maps));
  for (const Phi& f : phis) {
    // the target sector's shape (the stored shape transposed for spin 1)
    const SectorDev& sd = secs[vecs[f.vec].sector];
    const int du = f.spin == 0 ? sd.dim_up : sd.dim_dn, dd = f.spin == 0 ? sd.dim_dn : sd.dim_up;
    CK(ctx, launch_fermion_op(fp64, E.vec_x1(0), E.vec_x1(f.vec), (int)ctx->dim_up,
                              (int)ctx->dim_dn, du, dd, f.spin == 0 ? 0 : 2,
                              static_cast<const int32_t*>(dmaps.p) + moff[f.vec], s));
  }
  CKS(ctx, E.begin(sub.coefs, {}, n_sub, sub.tau, s));
  CKS(ctx, E.run(n_sub, false, nullptr, nullptr, s));
  std::vector<double> ov;
  CKS(ctx, E.fetch_overlaps(n_sub, ov, s));
  bool timed_out = false, non_finite = false;
  for (int v = 0; v < E.nvec(); ++v) {
    int st = 0;
    CKS(ctx, E.fetch(v, 0, nullptr, nullptr, nullptr, nullptr, nullptr, &st, s));
    timed_out |= st == ED_ERR_TIMEOUT;
    non_finite |= st != 0 && st != ED_ERR_TIMEOUT;
  }
  CK(ctx, cudaStreamSynchronize(s));
  CK(ctx, join_streams(s, us));
  std::memset(G_less, 0, sizeof(double) * 2 * (size_t)(n_steps + 1) * Ns * 2);
  std::memset(G_great, 0, sizeof(double) * 2 * (size_t)(n_steps + 1) * Ns * 2);
  const int nv = E.nvec();
  for (int n = 0; n <= n_steps; ++n)
    for (const Phi& f : phis) {
      const size_t k = (size_t)n * per;   // overlaps after whole time steps
      const double re = ov[(k * nv + f.vec) * 2], im = ov[(k * nv + f.vec) * 2 + 1];
      const size_t o = (((size_t)n * Ns + f.site) * 2 + f.spin) * 2;
      if (f.op == 0) {  // G^< = i L
        G_less[o] = -im;
        G_less[o + 1] = re;
      } else {          // G^> = -i G
        G_great[o] = im;
        G_great[o + 1] = -re;
      }
    }
  if (timed_out)
    return fail(ctx, ED_ERR_TIMEOUT, "a bounded device-side wait of the apply kernel gave up");
  if (non_finite) return fail(ctx, ED_ERR_NUMERIC, "non-finite norm during spectral propagation");
  return ED_OK;
}

// Eq. (37), Sec. 3.7: A(nu) = (1/pi) Im int_0^T e^{-eps t} e^{i nu t}
// G(t) dt over the samples G(k dt), k = 0..n_steps, by the trapezoid rule.
ed_status ed_spectral_function(const double* G, int n_steps, int n_series, double dt,
                               double eps, const double* nu, int n_nu, double* A) {
  if (!G || !nu || !A) return fail(nullptr, ED_ERR_ARG, "NULL argument");
  if (n_steps < 1 || n_series < 1 || n_nu < 1)
    return fail(nullptr, ED_ERR_ARG, "n_steps, n_series, n_nu must be >= 1");
  if (!(dt > 0.0) || !std::isfinite(dt) || !(eps >= 0.0) || !std::isfinite(eps))
    return fail(nullptr, ED_ERR_ARG, "dt > 0 and eps >= 0 required");
  for (int f = 0; f < n_nu; ++f) {
    for (int j = 0; j < n_series; ++j) {
      double sr = 0.0, si = 0.0;   // sum of weights * e^{(i nu - eps) t} G(t)
      for (int k = 0; k <= n_steps; ++k) {
        const double t = k * dt;
        const double wgt = (k == 0 || k == n_steps) ? 0.5 : 1.0;
        const double damp = wgt * std::exp(-eps * t);
        const double c = std::cos(nu[f] * t) * damp, sn = std::sin(nu[f] * t) * damp;
        const double gr = G[((size_t)k * n_series + j) * 2], gi = G[((size_t)k * n_series + j) * 2 + 1];
        sr += c * gr - sn * gi;
        si += c * gi + sn * gr;
      }
      A[(size_t)f * n_series + j] = si * dt / 3.14159265358979323846;
    }
  }
  return ED_OK;
}

}  // extern "C"
