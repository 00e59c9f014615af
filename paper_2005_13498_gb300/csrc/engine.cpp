// Batched midpoint-rule propagation engine (see engine.h).
#include "engine.h"
#include "tables.h"

#include <algorithm>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>

namespace ed {


cudaError_t DevMem::alloc(size_t n) {
  release();
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    return e;
  }
  bytes = n;
  return cudaSuccess;
}

void DevMem::release() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}

Engine::~Engine() {
  if (exec_) cudaGraphExecDestroy(exec_);
  if (graph_) cudaGraphDestroy(graph_);
  for (cudaEvent_t e : ev_fork_) cudaEventDestroy(e);
  for (cudaEvent_t e : ev_check_) cudaEventDestroy(e);
  if (side_) cudaStreamDestroy(side_);
}

size_t Engine::device_bytes() const {
  return d_sec_.bytes + d_vec_.bytes + d_st_.bytes + d_amap_.bytes + d_cmap_.bytes +
         d_emap_.bytes +
         d_partials_.bytes + d_counters_.bytes + d_coefs_.bytes + d_coefs_obs_.bytes +
         d_V_.bytes + d_w_.bytes + d_out_.bytes + d_owned_x1_.bytes + d_maps_.bytes +
         d_map_off_.bytes + d_map_spin_.bytes + d_ovl_.bytes + d_psiT_.bytes;
}

static std::atomic<int> g_forced_cfg{-1};
void set_forced_apply_config(int cfg) { g_forced_cfg.store(cfg); }
int forced_apply_config() { return g_forced_cfg.load(); }

static std::atomic<int> g_withhold{-1};
static std::atomic<uint32_t> g_wait_polls{0};
void set_wait_fault(int withhold, uint32_t polls) {
  g_withhold.store(withhold);
  g_wait_polls.store(polls);
}
void init_batch_args(BatchArgs* a) {
  std::memset(a, 0, sizeof(*a));
  const uint32_t polls = g_wait_polls.load();
  a->wait_limit = polls > 0 ? polls : kDefaultWaitLimit;
  a->tma_withhold = g_withhold.load();
}

bool Engine::compatible(const EngineConfig& cfg, const std::vector<EngineVector>& vecs) const {
  const int forced = forced_apply_config();
  if (forced >= 0 && forced != shape_.cfg) return false;
  BatchArgs now;
  init_batch_args(&now);
  if (now.wait_limit != args_.wait_limit || now.tma_withhold != args_.tma_withhold) return false;
  if (cfg.workspace_limit > 0 && workspace_bytes_ > cfg.workspace_limit) return false;
  if (cfg.fp64 != cfg_.fp64 || cfg.m != cfg_.m || cfg.energy != cfg_.energy ||
      cfg.overlaps != cfg_.overlaps || cfg.n_steps_cap > cfg_.n_steps_cap ||
      cfg.eps_tol != cfg_.eps_tol)
    return false;
  if (vecs.size() != vecs_.size()) return false;
  for (size_t i = 0; i < vecs.size(); ++i) {
    if (vecs[i].sector != vecs_[i].sector || vecs[i].D != vecs_[i].D) return false;
    if (!vecs[i].owned_x1 && (vecs_[i].owned_x1 || vecs[i].x1 != vecs_[i].x1)) return false;
    if (vecs[i].owned_x1 != vecs_[i].owned_x1) return false;
  }
  return true;
}

std::string tune_apply(const ApplyTuneTarget& t, cudaStream_t s, LaunchShape* shape,
                       std::vector<ApplyBlock>* map, std::vector<ApplyBlock>* cmap) {
  static std::mutex mu;
  static std::map<std::string, int> cache;
  std::vector<LaunchShape> cands =
      apply_candidates(t.max_dim_up, t.max_dim_dn, t.fp64, t.n_groups);
  if (!t.tma_ok)
    cands.erase(std::remove_if(cands.begin(), cands.end(),
                               [](const LaunchShape& c) { return c.tma; }),
                cands.end());
  // multi-vector configurations run only when pinned: on both spectral
  // batches they measured slower than one-vector blocks (the vectors that
  // share a block multiply the working set of the T_up row gathers)
  if (forced_apply_config() < 0)
    cands.erase(std::remove_if(cands.begin(), cands.end(),
                               [](const LaunchShape& c) { return c.mv; }),
                cands.end());
  if (cands.empty()) return "apply kernel: rows too long for shared memory";
  for (auto& c : cands) c.vec = t.vec_ok;
  // row orders of the vectors' up spaces (reverse Cuthill-McKee), computed once
  std::vector<std::vector<int>> orders(t.dim_up.size());
  for (size_t i = 0; i < t.dim_up.size(); ++i)
    if (i < t.up.size() && t.up[i] && t.up[i]->dim == t.dim_up[i])
      orders[i] = block_order(*t.up[i], 1);
  auto order_of = [&](size_t i) { return orders[i].empty() ? nullptr : &orders[i]; };
  auto build = [&](const LaunchShape& sh) {
    map->clear();
    cmap->clear();
    if (sh.mv) {   // the vectors of each sector, in batch order, nr at a time
      std::vector<int> done(t.dim_up.size(), 0);
      for (size_t i = 0; i < t.dim_up.size(); ++i) {
        if (done[i]) continue;
        std::vector<int> ids;
        for (size_t k = i; k < t.dim_up.size(); ++k)
          if (!done[k] && (k < t.sector.size() ? t.sector[k] : (int)k) ==
                              (i < t.sector.size() ? t.sector[i] : (int)i)) {
            ids.push_back((int)k);
            done[k] = 1;
          }
        append_mv_blocks(*map, ids, t.dim_up[i], sh.nr, order_of(i));
      }
      return;
    }
    for (size_t i = 0; i < t.dim_up.size(); ++i) {
      append_apply_blocks(*map, (int)i, t.dim_up[i], sh.nr, order_of(i));
      if (sh.split && sh.cb > 0) append_col_blocks(*cmap, (int)i, t.dim_dn[i], t.fp64, sh.cb);
    }
    if (sh.split && sh.cb == 0) {   // row-gather T_up pass: chunk-major over the batch
      const int chunk = kApplyThreads * sh.ppc;   // k_apply_tup runs kApplyThreads threads
      int max_pairs = 0;
      for (int d : t.dim_dn) max_pairs = std::max(max_pairs, (d + 1) / 2);
      for (int pc = 0; pc < max_pairs; pc += chunk)
        for (size_t i = 0; i < t.dim_up.size(); ++i)
          if (pc < (t.dim_dn[i] + 1) / 2)
            append_tup_chunk(*cmap, (int)i, t.dim_up[i], kTupRows, pc, order_of(i));
    }
  };
  const int forced = forced_apply_config();
  if (forced >= 0) {
    for (const LaunchShape& c : cands)
      if (c.cfg == forced) {
        *shape = c;
        build(c);
        return "";
      }
    return "apply configuration " + std::to_string(forced) +
           " does not fit this precision and sector";
  }
  std::string key = (t.fp64 ? "d" : "f") + std::string(t.vec_ok ? "v" : "s");
  for (size_t i = 0; i < t.dim_up.size(); ++i)
    key += ":" + std::to_string(t.dim_up[i]) + "x" + std::to_string(t.dim_dn[i]);
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end())
      for (auto& c : cands)
        if (c.cfg == it->second) {
          *shape = c;
          build(c);
          return "";
        }
  }
  int64_t elems = 0;
  for (size_t i = 0; i < t.dim_up.size(); ++i) elems += (int64_t)t.dim_up[i] * t.dim_dn[i];
  if (cands.size() == 1 || elems < (1 << 20)) {   // small problems: the default
    *shape = cands.front();
    build(*shape);
    std::lock_guard<std::mutex> lock(mu);
    cache[key] = shape->cfg;
    return "";
  }
  cudaEvent_t e0, e1;
  ED_TRY(cudaEventCreate(&e0));
  ED_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  LaunchShape best_sh = cands.front();
  std::string err;
  for (const LaunchShape& c : cands) {
    build(c);
    DevMem dmap, dcmap;
    if (dmap.alloc(map->size() * sizeof(ApplyBlock)) != cudaSuccess ||
        cudaMemcpy(dmap.p, map->data(), map->size() * sizeof(ApplyBlock),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        dcmap.alloc(std::max<size_t>(1, cmap->size()) * sizeof(ApplyBlock)) != cudaSuccess ||
        (!cmap->empty() &&
         cudaMemcpy(dcmap.p, cmap->data(), cmap->size() * sizeof(ApplyBlock),
                    cudaMemcpyHostToDevice) != cudaSuccess) ||
        prepare_apply(t.fp64, c) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    BatchArgs a = t.args;
    a.apply_map = static_cast<const ApplyBlock*>(dmap.p);
    a.col_map = static_cast<const ApplyBlock*>(dcmap.p);
    a.n_col_blocks = (int)cmap->size();
    const int nblk = (int)map->size();
    if (launch_apply(t.fp64, a, nblk, c, 0, s) != cudaSuccess) { cudaGetLastError(); continue; }
    cudaEventRecord(e0, s);
    for (int r = 0; r < 3; ++r) launch_apply(t.fp64, a, nblk, c, 0, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) { err = "autotune: apply failed"; break; }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best) { best = ms; best_sh = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!err.empty()) return err;
  *shape = best_sh;
  build(best_sh);
  std::lock_guard<std::mutex> lock(mu);
  cache[key] = best_sh.cfg;
  return "";
}

static int64_t ew_chunk(int64_t D) {
  int64_t c = (D + 1215) / 1216;
  c = ((c + 255) / 256) * 256;
  return std::max<int64_t>(1024, std::min<int64_t>(16384, c));
}

std::string Engine::setup(const EngineConfig& cfg, const std::vector<SectorDev>& sectors,
                          const std::vector<EngineVector>& vecs, int n_groups, int Ns,
                          double U, double break_tol, cudaStream_t stream,
                          const std::vector<const SpinTable*>& up_tabs) {
  if (exec_) { cudaGraphExecDestroy(exec_); exec_ = nullptr; }
  if (graph_) { cudaGraphDestroy(graph_); graph_ = nullptr; }
  cfg_ = cfg;
  sectors_ = sectors;
  vecs_ = vecs;
  n_groups_ = n_groups;
  Ns_ = Ns;
  U_ = U;
  break_tol_ = break_tol;
  have_overlaps_ = false;
  const size_t esz = cfg.fp64 ? 16 : 8;
  const int nv = (int)vecs.size();
  const int m = cfg.m;
  if (cfg.eps_tol > 0.0 && !side_) {
    ED_TRY(cudaStreamCreateWithFlags(&side_, cudaStreamNonBlocking));
    ev_fork_.assign(kMaxKrylov + 1, nullptr);
    ev_check_.assign(kMaxKrylov + 1, nullptr);
    for (int i = 0; i <= kMaxKrylov; ++i) {
      ED_TRY(cudaEventCreateWithFlags(&ev_fork_[i], cudaEventDisableTiming));
      ED_TRY(cudaEventCreateWithFlags(&ev_check_[i], cudaEventDisableTiming));
    }
  }

  // owned state buffers, Krylov storage and scratch: checked against the
  // context's workspace limit before anything is allocated
  int64_t owned = 0, totD = 0;
  for (auto& v : vecs_) {
    if (v.owned_x1) owned += v.D;
    totD += v.D;
  }
  const int64_t need = (owned + (int64_t)std::max(0, m - 1) * totD + totD) * (int64_t)esz;
  workspace_bytes_ = need;
  if (cfg.workspace_limit > 0 && need > cfg.workspace_limit)
    return "device memory for the Krylov workspace (" + std::to_string(need) +
           " bytes) exceeds the context's workspace limit (" +
           std::to_string(cfg.workspace_limit) + " bytes)";
  ED_TRY(d_owned_x1_.alloc((size_t)owned * esz));
  {
    int64_t o = 0;
    for (auto& v : vecs_)
      if (v.owned_x1) {
        v.x1 = static_cast<char*>(d_owned_x1_.p) + (size_t)o * esz;
        o += v.D;
      }
  }
  // Krylov storage and scratch
  ED_TRY(d_V_.alloc((size_t)std::max(0, m - 1) * totD * esz));
  ED_TRY(d_w_.alloc((size_t)totD * esz));

  // block maps
  std::vector<ApplyBlock> amap;
  std::vector<EwBlock> emap;
  std::vector<VecDev> vd(nv);
  int max_dim_dn = 1, max_dim_up = 1;
  for (int i = 0; i < nv; ++i) {
    max_dim_dn = std::max(max_dim_dn, sectors_[vecs_[i].sector].dim_dn);
    max_dim_up = std::max(max_dim_up, sectors_[vecs_[i].sector].dim_up);
  }
  int64_t voff = 0;
  const int ncap = cfg.n_steps_cap;
  // outputs per vector: docc, norm2, energy [ncap+1], delta [ncap], meff [ncap]
  const size_t per_vec_out = (size_t)4 * (ncap + 1) + (ncap + 1);
  ED_TRY(d_out_.alloc(per_vec_out * nv * sizeof(double)));
  for (int i = 0; i < nv; ++i) {
    const SectorDev& sd = sectors_[vecs_[i].sector];
    max_dim_dn = std::max(max_dim_dn, sd.dim_dn);
    VecDev& v = vd[i];
    std::memset(&v, 0, sizeof(v));
    v.sector = vecs_[i].sector;
    v.D = vecs_[i].D;
    v.x1 = vecs_[i].x1;
    v.V = static_cast<char*>(d_V_.p) + (size_t)std::max(0, m - 1) * voff * esz;
    v.w = static_cast<char*>(d_w_.p) + (size_t)voff * esz;
    voff += v.D;

    v.ew_begin = (int)emap.size();
    // one chunk size for the whole batch, from its total size: sized per
    // vector, a batch of 49 small vectors got 35,000 blocks of 1024
    // elements, each paying a block reduction
    const int64_t ch = ew_chunk(totD);
    for (int64_t b = 0; b < v.D; b += ch) emap.push_back({i, 0, b, std::min(v.D, b + ch)});
    v.ew_end = (int)emap.size();
    double* base = static_cast<double*>(d_out_.p) + per_vec_out * i;
    v.out_docc = base;
    v.out_norm2 = base + (ncap + 1);
    v.out_energy = base + 2 * (ncap + 1);
    v.out_delta = base + 3 * (ncap + 1);
    v.out_meff = reinterpret_cast<int*>(base + 4 * (ncap + 1));
  }
  n_ew_ = (int)emap.size();
  // 16-byte pair accesses for complex64 when every row and buffer allows it;
  // the same conditions allow TMA row chunks in either precision
  bool tma_ok = true;
  for (int i = 0; i < nv; ++i) {
    if (sectors_[vecs_[i].sector].dim_dn & 1) tma_ok = false;
    if (((uintptr_t)vd[i].x1 | (uintptr_t)vd[i].V | (uintptr_t)vd[i].w) & 15u) tma_ok = false;
  }
  const bool vec_ok = !cfg.fp64 && tma_ok;

  ED_TRY(d_sec_.alloc(sizeof(SectorDev) * sectors_.size()));
  ED_TRY(d_vec_.alloc(sizeof(VecDev) * nv));
  ED_TRY(d_st_.alloc(sizeof(LanczosState) * nv));
  ED_TRY(d_emap_.alloc(sizeof(EwBlock) * emap.size()));
  ED_TRY(d_counters_.alloc(sizeof(unsigned) * nv));
  ED_TRY(d_coefs_.alloc(esz * (size_t)n_groups * std::max(1, ncap)));
  if (cfg.energy) ED_TRY(d_coefs_obs_.alloc(esz * (size_t)n_groups * (ncap + 1)));
  else d_coefs_obs_.release();
  ED_TRY(cudaMemcpyAsync(d_sec_.p, sectors_.data(), sizeof(SectorDev) * sectors_.size(),
                         cudaMemcpyHostToDevice, stream));
  ED_TRY(cudaMemcpyAsync(d_vec_.p, vd.data(), sizeof(VecDev) * nv, cudaMemcpyHostToDevice,
                         stream));
  ED_TRY(cudaMemcpyAsync(d_emap_.p, emap.data(), sizeof(EwBlock) * emap.size(),
                         cudaMemcpyHostToDevice, stream));
  ED_TRY(cudaStreamSynchronize(stream));

  init_batch_args(&args_);
  args_.sec = static_cast<const SectorDev*>(d_sec_.p);
  args_.vec = static_cast<VecDev*>(d_vec_.p);
  args_.st = static_cast<LanczosState*>(d_st_.p);
  args_.apply_map = static_cast<const ApplyBlock*>(d_amap_.p);
  args_.ew_map = static_cast<const EwBlock*>(d_emap_.p);
  args_.partials = static_cast<double*>(d_partials_.p);
  args_.counters = static_cast<unsigned*>(d_counters_.p);
  args_.coefs = d_coefs_.p;
  args_.coefs_obs = d_coefs_obs_.p;
  args_.n_groups = n_groups;
  args_.nvec = nv;
  args_.Ns = Ns;
  args_.max_dim_dn = max_dim_dn;
  args_.max_dim_up = max_dim_up;
  args_.U = U;
  args_.tau = 0.0;
  args_.break_tol = break_tol;

  // apply configuration (autotuned) and its block map
  ApplyTuneTarget tt;
  tt.fp64 = cfg.fp64;
  tt.vec_ok = vec_ok;
  tt.tma_ok = tma_ok;
  tt.max_dim_up = max_dim_up;
  tt.max_dim_dn = max_dim_dn;
  tt.n_groups = n_groups;
  for (int i = 0; i < nv; ++i) {
    tt.dim_up.push_back(sectors_[vecs_[i].sector].dim_up);
    tt.dim_dn.push_back(sectors_[vecs_[i].sector].dim_dn);
    tt.up.push_back((size_t)vecs_[i].sector < up_tabs.size() ? up_tabs[vecs_[i].sector]
                                                               : nullptr);
    tt.sector.push_back(vecs_[i].sector);
  }
  tt.args = args_;
  std::vector<ApplyBlock> cmap;
  std::string err = tune_apply(tt, stream, &shape_, &amap, &cmap);
  if (!err.empty()) return err;
  ED_TRY(prepare_apply(cfg.fp64, shape_));
  n_apply_ = (int)amap.size();
  assign_apply_ranges(amap, shape_.mv, vd.data(), nv);
  ED_TRY(d_amap_.alloc(sizeof(ApplyBlock) * amap.size()));
  ED_TRY(d_cmap_.alloc(sizeof(ApplyBlock) * std::max<size_t>(1, cmap.size())));
  if (!cmap.empty())
    ED_TRY(cudaMemcpyAsync(d_cmap_.p, cmap.data(), sizeof(ApplyBlock) * cmap.size(),
                           cudaMemcpyHostToDevice, stream));
  ED_TRY(d_partials_.alloc(sizeof(double) *
                           std::max(apply_partials_per_block(shape_) * n_apply_,
                                    (size_t)4 * n_ew_)));
  ED_TRY(cudaMemcpyAsync(d_vec_.p, vd.data(), sizeof(VecDev) * nv, cudaMemcpyHostToDevice,
                         stream));
  ED_TRY(cudaMemcpyAsync(d_amap_.p, amap.data(), sizeof(ApplyBlock) * amap.size(),
                         cudaMemcpyHostToDevice, stream));
  ED_TRY(cudaMemsetAsync(d_counters_.p, 0, sizeof(unsigned) * nv, stream));
  ED_TRY(cudaStreamSynchronize(stream));
  args_.apply_map = static_cast<const ApplyBlock*>(d_amap_.p);
  args_.col_map = static_cast<const ApplyBlock*>(d_cmap_.p);
  args_.n_col_blocks = (int)cmap.size();
  args_.partials = static_cast<double*>(d_partials_.p);
  return "";
}

std::string Engine::set_overlap_maps(const std::vector<int32_t>& maps,
                                     const std::vector<int64_t>& off,
                                     const std::vector<int32_t>& spin, int psi_index,
                                     cudaStream_t s) {
  const int nv = (int)vecs_.size();
  if ((int)off.size() != nv || (int)spin.size() != nv) return "overlap map arrays: bad size";
  ED_TRY(d_maps_.alloc(std::max<size_t>(1, maps.size()) * sizeof(int32_t)));
  ED_TRY(d_map_off_.alloc(nv * sizeof(int64_t)));
  ED_TRY(d_map_spin_.alloc(nv * sizeof(int32_t)));
  ED_TRY(d_ovl_.alloc((size_t)(cfg_.n_steps_cap + 1) * nv * 2 * sizeof(double)));
  if (!maps.empty())
    ED_TRY(cudaMemcpyAsync(d_maps_.p, maps.data(), maps.size() * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s));
  ED_TRY(cudaMemcpyAsync(d_map_off_.p, off.data(), nv * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  ED_TRY(cudaMemcpyAsync(d_map_spin_.p, spin.data(), nv * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  ED_TRY(cudaMemsetAsync(d_ovl_.p, 0, d_ovl_.bytes, s));
  ED_TRY(cudaStreamSynchronize(s));
  oargs_.maps = static_cast<const int32_t*>(d_maps_.p);
  oargs_.map_off = static_cast<const int64_t*>(d_map_off_.p);
  oargs_.map_spin = static_cast<const int32_t*>(d_map_spin_.p);
  oargs_.psi_index = psi_index;
  oargs_.out = static_cast<double*>(d_ovl_.p);
  // column maps of vectors stored transposed (mode 2) read psi transposed:
  // one copy, refreshed before every overlap launch
  need_psiT_ = std::find(spin.begin(), spin.end(), 2) != spin.end();
  if (need_psiT_) {
    const size_t esz = cfg_.fp64 ? 16 : 8;
    ED_TRY(d_psiT_.alloc((size_t)vecs_[psi_index].D * esz));
  } else {
    d_psiT_.release();
  }
  oargs_.psiT = d_psiT_.p;
  have_overlaps_ = true;
  if (exec_) { cudaGraphExecDestroy(exec_); exec_ = nullptr; }
  if (graph_) { cudaGraphDestroy(graph_); graph_ = nullptr; }
  return "";
}

static std::string upload_coefs(DevMem& dst, const std::vector<double>& c, bool fp64,
                                cudaStream_t s) {
  if (c.empty()) return "";
  if (fp64) {
    if (c.size() * sizeof(double) > dst.bytes) return "coefficient buffer too small";
    ED_TRY(cudaMemcpyAsync(dst.p, c.data(), c.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  } else {
    std::vector<float> f(c.size());
    for (size_t i = 0; i < c.size(); ++i) f[i] = (float)c[i];
    if (f.size() * sizeof(float) > dst.bytes) return "coefficient buffer too small";
    ED_TRY(cudaMemcpyAsync(dst.p, f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    ED_TRY(cudaStreamSynchronize(s));  // f goes out of scope
  }
  return "";
}

std::string Engine::begin(const std::vector<double>& coefs, const std::vector<double>& coefs_obs,
                          int n_steps, double tau, cudaStream_t stream) {
  if (n_steps > cfg_.n_steps_cap) return "n_steps exceeds engine capacity";
  std::string err = upload_coefs(d_coefs_, coefs, cfg_.fp64, stream);
  if (!err.empty()) return err;
  err = upload_coefs(d_coefs_obs_, coefs_obs, cfg_.fp64, stream);
  if (!err.empty()) return err;
  std::vector<LanczosState> st(vecs_.size());
  for (auto& s : st) {
    std::memset(&s, 0, sizeof(s));
    s.m = cfg_.m;
    s.m_eff = cfg_.m;
    s.scale = 1.0;
    s.eps_tol = cfg_.eps_tol;
  }
  ED_TRY(cudaMemcpyAsync(d_st_.p, st.data(), sizeof(LanczosState) * st.size(),
                         cudaMemcpyHostToDevice, stream));
  ED_TRY(cudaStreamSynchronize(stream));
  if (tau != tau_ || args_.tau != tau) {
    tau_ = tau;
    args_.tau = tau;
    if (exec_) { cudaGraphExecDestroy(exec_); exec_ = nullptr; }
    if (graph_) { cudaGraphDestroy(graph_); graph_ = nullptr; }
  }
  return "";
}

std::string Engine::launch_step(cudaStream_t s, bool profile, cudaEvent_t* ev, int* kind_of,
                                int* nev) {
  const bool f = cfg_.fp64;
  auto mark = [&](int kind) -> std::string {
    if (!profile) return "";
    ED_TRY(cudaEventRecord(ev[*nev], s));
    kind_of[*nev] = kind;
    ++*nev;
    return "";
  };
  std::string err;
#define STEP_LAUNCH(kind, call)                         \
  do {                                                  \
    if (!(err = mark(-1)).empty()) return err;          \
    ED_TRY(call);                                       \
    if (!(err = mark(kind)).empty()) return err;        \
  } while (0)
  // With the adaptive exit, the check of step j runs on the side stream
  // while pass j + 1 proceeds on s; pass j + 2 waits for it (a converged
  // check makes the later passes return at once, see lanczos_done).
  const bool adaptive = cfg_.eps_tol > 0.0;
  for (int j = 1; j <= cfg_.m; ++j) {
    if (adaptive && j >= 3) ED_TRY(cudaStreamWaitEvent(s, ev_check_[j - 2], 0));
    STEP_LAUNCH(KK_APPLY, launch_apply(f, args_, n_apply_, shape_, j, s));
    if (j < cfg_.m) {
      STEP_LAUNCH(KK_UPDATE, launch_update(f, args_, n_ew_, j, s));
      if (adaptive) {
        ED_TRY(cudaEventRecord(ev_fork_[j], s));
        ED_TRY(cudaStreamWaitEvent(side_, ev_fork_[j], 0));
        ED_TRY(launch_conv_check(args_, j, side_));
        ED_TRY(cudaEventRecord(ev_check_[j], side_));
      }
    }
  }
  if (adaptive && cfg_.m >= 2) ED_TRY(cudaStreamWaitEvent(s, ev_check_[cfg_.m - 1], 0));
  STEP_LAUNCH(KK_EXPM, launch_expm(args_, s));
  STEP_LAUNCH(KK_COMBINE, launch_combine(f, args_, n_ew_, s));
  if (cfg_.energy) STEP_LAUNCH(KK_ENERGY, launch_apply(f, args_, n_apply_, shape_, -1, s));
  if (have_overlaps_) {
    if (need_psiT_) STEP_LAUNCH(KK_OVERLAP, launch_psiT(s));
    STEP_LAUNCH(KK_OVERLAP, launch_overlap(f, args_, oargs_, n_ew_, s));
  }
#undef STEP_LAUNCH
  return "";
}

cudaError_t Engine::launch_psiT(cudaStream_t s) {
  const SectorDev& sp = sectors_[vecs_[oargs_.psi_index].sector];
  return launch_transpose(cfg_.fp64, vecs_[oargs_.psi_index].x1, d_psiT_.p, sp.dim_up,
                          sp.dim_dn, s);
}

std::string Engine::capture(cudaStream_t s) {
  if (exec_) return "";
  ED_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  std::string err = launch_step(s, false, nullptr, nullptr, nullptr);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(s, &g);
  if (!err.empty()) {
    if (g) cudaGraphDestroy(g);
    return err;
  }
  if (e != cudaSuccess) return std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e);
  graph_ = g;
  ED_TRY(cudaGraphInstantiate(&exec_, graph_, 0));
  return "";
}

std::string Engine::run(int n_steps, bool profile, double* kernel_ms, int64_t* launches,
                        cudaStream_t s) {
  const bool f = cfg_.fp64;
  // observables at t_0 (also sets beta0 and the first scale)
  ED_TRY(launch_observe(f, args_, n_ew_, s));
  if (have_overlaps_) {
    if (need_psiT_) ED_TRY(launch_psiT(s));
    ED_TRY(launch_overlap(f, args_, oargs_, n_ew_, s));
  }
  if (cfg_.energy) ED_TRY(launch_apply(f, args_, n_apply_, shape_, -1, s));
  if (!profile) {
    std::string err = capture(s);
    if (!err.empty()) return err;
    for (int n = 0; n < n_steps; ++n) ED_TRY(cudaGraphLaunch(exec_, s));
    return "";
  }
  const int per_step = 2 * (2 * cfg_.m + 6);   // event pairs per step, every launch kind
  std::vector<cudaEvent_t> ev((size_t)per_step * std::max(1, n_steps));
  std::vector<int> kind(ev.size(), -1);
  for (auto& e : ev) ED_TRY(cudaEventCreate(&e));
  int nev = 0;
  std::string err;
  for (int n = 0; n < n_steps && err.empty(); ++n)
    err = launch_step(s, true, ev.data(), kind.data(), &nev);
  if (err.empty()) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) err = std::string("sync: ") + cudaGetErrorString(e);
  }
  if (err.empty()) {
    for (int k = 0; k < KK_COUNT; ++k) {
      if (kernel_ms) kernel_ms[k] = 0.0;
      if (launches) launches[k] = 0;
    }
    for (int i = 1; i < nev; i += 2) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i - 1], ev[i]);
      if (kind[i] >= 0) {
        if (kernel_ms) kernel_ms[kind[i]] += ms;
        if (launches) launches[kind[i]] += 1;
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  return err;
}

std::string Engine::fetch(int vec, int n_steps, double* docc, double* norm2, double* energy,
                          double* delta, int32_t* meff, int* status, cudaStream_t s) {
  VecDev v;
  ED_TRY(cudaMemcpyAsync(&v, static_cast<VecDev*>(d_vec_.p) + vec, sizeof(VecDev),
                         cudaMemcpyDeviceToHost, s));
  LanczosState st;
  ED_TRY(cudaMemcpyAsync(&st, static_cast<LanczosState*>(d_st_.p) + vec, sizeof(st),
                         cudaMemcpyDeviceToHost, s));
  ED_TRY(cudaStreamSynchronize(s));
  const size_t nb = (size_t)(n_steps + 1) * sizeof(double);
  if (docc) ED_TRY(cudaMemcpyAsync(docc, v.out_docc, nb, cudaMemcpyDeviceToHost, s));
  if (norm2) ED_TRY(cudaMemcpyAsync(norm2, v.out_norm2, nb, cudaMemcpyDeviceToHost, s));
  if (energy) ED_TRY(cudaMemcpyAsync(energy, v.out_energy, nb, cudaMemcpyDeviceToHost, s));
  if (delta && n_steps > 0)
    ED_TRY(cudaMemcpyAsync(delta, v.out_delta, n_steps * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (meff && n_steps > 0)
    ED_TRY(cudaMemcpyAsync(meff, v.out_meff, n_steps * sizeof(int), cudaMemcpyDeviceToHost, s));
  ED_TRY(cudaStreamSynchronize(s));
  if (status) *status = st.status;
  return "";
}

std::string Engine::fetch_overlaps(int n_steps, std::vector<double>& out, cudaStream_t s) {
  out.assign((size_t)(n_steps + 1) * vecs_.size() * 2, 0.0);
  if (!have_overlaps_) return "no overlaps configured";
  ED_TRY(cudaMemcpyAsync(out.data(), d_ovl_.p, out.size() * sizeof(double),
                         cudaMemcpyDeviceToHost, s));
  ED_TRY(cudaStreamSynchronize(s));
  return "";
}

}  // namespace ed
