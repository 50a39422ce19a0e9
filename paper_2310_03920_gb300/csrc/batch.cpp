// Batched execution of many independent DMRG problems on one GPU.
//
// The problems advance in lockstep: every Davidson iteration issues ONE grouped launch of
// the H_eff contraction over all problems still iterating (heff_apply_batched: the work
// items of every problem's window program in one grid), so that small windows, which alone
// would leave most SMs idle, share the GPU.  The Davidson bookkeeping of each problem is
// the single-problem algorithm (davidson in algo.cpp) split at its two host
// synchronisation points, so that one synchronisation serves every problem; per problem,
// the kernels, their arguments and their order are those of the single-problem path, so
// the results are identical to solving the problems one by one.  Sweeps advance window by
// window in lockstep too (problems with fewer sites finish their sweep earlier).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "algo.hpp"

namespace b2 {

namespace {

// pinned host slots for the scalars each problem reads back per phase
struct HostSlots {
  double* p = nullptr;
  explicit HostSlots(size_t n) {
    B2_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&p), sizeof(double) * std::max<size_t>(n, 1),
                          cudaHostAllocDefault));
  }
  ~HostSlots() {
    if (p) cudaFreeHost(p);
  }
  HostSlots(const HostSlots&) = delete;
  HostSlots& operator=(const HostSlots&) = delete;
};

struct DavState {
  b2_env_s* env = nullptr;
  int site = 0;
  double* psi = nullptr;
  int64_t n = 0;
  int kmax = 0, max_iter = 0;
  double tol = 0;
  DevBuf V, W, diag, u, hu, t, small, d_dims, d_offs;
  double *part = nullptr, *VW = nullptr, *G = nullptr, *evecs = nullptr, *evals = nullptr,
         *cvec = nullptr, *scal = nullptr;
  int k = 1, nmv = 0;
  int dims_h = 0;
  bool active = true;
  std::vector<double> hist;   // residuals so far (stagnation test of split products)
  DavidsonResult res;
};

// Lockstep Davidson over the states (see davidson_core in algo.cpp for the single-problem
// form of each step).  w0[i] (may be null): H psi_i / |psi_i| in FP64 seeding W[0].
void davidson_batched_core(Ctx* c, std::vector<DavState>& st, const b2_dav_opts& o,
                           b2_prec mv_prec, const std::vector<const double*>& w0,
                           const std::vector<double>& tol) {
  const int np = int(st.size());
  HostSlots hs(size_t(np) * 4);
  const int kPart = 256 * 16;
  std::vector<int> need;
  for (int i = 0; i < np; ++i) {
    DavState& s = st[i];
    WindowProgram& wp = window_program(s.env, s.site);
    s.n = wp.psi.size;
    B2_REQUIRE(s.n > 0, B2_EINVAL, "empty two-site wavefunction");
    s.kmax = std::max(2, std::min(o.max_subspace > 0 ? o.max_subspace : 30, 64));
    s.max_iter = o.max_iter > 0 ? o.max_iter : 30;
    s.tol = tol[i];
    s.V.reset(c, sizeof(double) * s.n * s.kmax);
    s.W.reset(c, sizeof(double) * s.n * s.kmax);
    s.diag.reset(c, sizeof(double) * s.n);
    s.u.reset(c, sizeof(double) * s.n);
    s.hu.reset(c, sizeof(double) * s.n);
    s.t.reset(c, sizeof(double) * s.n);
    s.small.reset(c, sizeof(double) * (kPart + 4 * s.kmax * s.kmax + 8 * s.kmax + 16));
    s.part = s.small.as<double>();
    s.VW = s.part + kPart;
    s.G = s.VW + s.kmax * s.kmax;
    s.evecs = s.G + s.kmax * s.kmax;
    s.evals = s.evecs + s.kmax * s.kmax;
    s.cvec = s.evals + s.kmax;
    s.scal = s.cvec + 2 * s.kmax;
    s.d_dims.reset(c, sizeof(int));
    s.d_offs.reset(c, sizeof(int64_t) * 2);
    s.k = 1;
    s.nmv = 0;
    s.active = true;
    s.hist.clear();
    s.res = DavidsonResult{};
    heff_diag(s.env, s.site, s.diag.as<double>());
    b2k::launch_multidot(1, s.psi, s.n, s.psi, s.n, s.part, s.scal + 2, 1, c->stream);
    B2_CUDA(cudaMemcpyAsync(s.V.ptr, s.psi, sizeof(double) * s.n, cudaMemcpyDeviceToDevice, c->stream));
    b2k::launch_scale_inv_sqrt(s.V.as<double>(), s.n, s.scal + 2, c->stream);
    if (w0[i])
      B2_CUDA(cudaMemcpyAsync(s.W.ptr, w0[i], sizeof(double) * s.n, cudaMemcpyDeviceToDevice, c->stream));
    else
      need.push_back(i);
  }
  auto batched_matvec = [&](const std::vector<int>& ids, int col) {
    if (ids.empty()) return;
    std::vector<b2_env_s*> envs;
    std::vector<int> sites;
    std::vector<const double*> in;
    std::vector<double*> out;
    for (int i : ids) {
      DavState& s = st[i];
      envs.push_back(s.env);
      sites.push_back(s.site);
      const int kk = col < 0 ? s.k : col;
      in.push_back(s.V.as<double>() + int64_t(kk) * s.n);
      out.push_back(s.W.as<double>() + int64_t(kk) * s.n);
    }
    double fl = 0;
    heff_apply_batched(c, int(ids.size()), envs.data(), sites.data(), in.data(), out.data(),
                       mv_prec, &fl);
    for (int i : ids) {
      // per-problem flop count of its own program
      st[i].res.flops += window_program(st[i].env, st[i].site).heff.flops;
      st[i].nmv += 1;
    }
  };
  batched_matvec(need, 0);
  const int64_t zero_offs[2] = {0, 0};
  for (auto& s : st) {
    b2k::launch_multidot(1, s.V.as<double>(), s.n, s.W.as<double>(), s.n, s.part, s.VW, 1, c->stream);
    B2_CUDA(cudaMemcpyAsync(s.d_offs.ptr, zero_offs, sizeof(zero_offs), cudaMemcpyHostToDevice,
                            c->stream));
  }
  const bool trace = std::getenv("B2_TRACE_DAVIDSON") != nullptr;
  for (;;) {
    bool any = false;
    // A: Rayleigh-Ritz, residual and preconditioned correction
    for (int i = 0; i < np; ++i) {
      DavState& s = st[i];
      if (!s.active) continue;
      any = true;
      b2k::launch_symmetrize(s.k, s.VW, s.kmax, s.G, c->stream);
      s.dims_h = s.k;
      B2_CUDA(cudaMemcpyAsync(s.d_dims.ptr, &s.dims_h, sizeof(int), cudaMemcpyHostToDevice, c->stream));
      b2k::launch_jacobi(1, s.d_dims.as<int>(), s.d_offs.as<int64_t>(), s.d_offs.as<int64_t>(), s.G,
                         s.evals, s.evecs, nullptr, s.d_offs.as<int64_t>(), s.k, c->stream);
      b2k::launch_ritz(s.k, s.V.as<double>(), s.W.as<double>(), s.n, s.evecs + (s.k - 1), s.k,
                       s.evals + (s.k - 1), s.diag.as<double>(), s.u.as<double>(), s.hu.as<double>(),
                       s.t.as<double>(), s.n, s.part, s.scal, c->stream);
      B2_CUDA(cudaMemcpyAsync(hs.p + 4 * i, s.scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      B2_CUDA(cudaMemcpyAsync(hs.p + 4 * i + 1, s.evals + (s.k - 1), sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
    }
    if (!any) break;
    B2_CUDA(cudaStreamSynchronize(c->stream));
    if (mv_prec != B2_FP64)
      B2_REQUIRE(c->take_status() == 0, B2_ETIMEOUT, "tensor-core wait ran out");
    // B: orthogonalise the corrections of the problems that continue
    for (int i = 0; i < np; ++i) {
      DavState& s = st[i];
      if (!s.active) continue;
      s.res.resid2 = hs.p[4 * i];
      s.res.energy = hs.p[4 * i + 1];
      if (trace)
        std::fprintf(stderr, "batched davidson problem %d site %d k %d nmv %d theta %.15f r2 %.3e\n",
                     i, s.site, s.k, s.nmv, s.res.energy, s.res.resid2);
      B2_REQUIRE(std::isfinite(s.res.resid2) && std::isfinite(s.res.energy), B2_ENOCONV,
                 "Davidson produced a non-finite value");
      if (s.res.resid2 <= s.tol || s.nmv >= s.max_iter) {
        s.active = false;
        continue;
      }
      // the same stagnation stop as the single-problem solver (split-precision products)
      s.hist.push_back(s.res.resid2);
      if (mv_prec != B2_FP64 && s.hist.size() > 4 && s.hist.back() > 0.5 * s.hist[s.hist.size() - 5]) {
        s.active = false;
        continue;
      }
      double* Vp = s.V.as<double>();
      double* Wp = s.W.as<double>();
      if (s.k >= s.kmax) {   // restart from the Ritz vector
        B2_CUDA(cudaMemcpyAsync(Vp, s.u.ptr, sizeof(double) * s.n, cudaMemcpyDeviceToDevice, c->stream));
        B2_CUDA(cudaMemcpyAsync(Wp, s.hu.ptr, sizeof(double) * s.n, cudaMemcpyDeviceToDevice, c->stream));
        s.k = 1;
        b2k::launch_multidot(1, Vp, s.n, Wp, s.n, s.part, s.VW, 1, c->stream);
      }
      double* tp = s.t.as<double>();
      for (int pass = 0; pass < 2; ++pass) {
        b2k::launch_multidot(s.k, Vp, s.n, tp, s.n, s.part, s.cvec, 1, c->stream);
        b2k::launch_multiaxpy(s.k, Vp, s.n, s.cvec, tp, s.n, -1.0, c->stream);
      }
      b2k::launch_multidot(1, tp, s.n, tp, s.n, s.part, s.scal + 1, 1, c->stream);
      B2_CUDA(cudaMemcpyAsync(hs.p + 4 * i + 2, s.scal + 1, sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
    }
    B2_CUDA(cudaStreamSynchronize(c->stream));
    // C: new basis vectors, one grouped product for all
    std::vector<int> mv;
    for (int i = 0; i < np; ++i) {
      DavState& s = st[i];
      if (!s.active) continue;
      if (!(std::sqrt(hs.p[4 * i + 2]) >= 1e-14)) {
        s.active = false;
        continue;
      }
      double* vk = s.V.as<double>() + int64_t(s.k) * s.n;
      B2_CUDA(cudaMemcpyAsync(vk, s.t.ptr, sizeof(double) * s.n, cudaMemcpyDeviceToDevice, c->stream));
      b2k::launch_scale_inv_sqrt(vk, s.n, s.scal + 1, c->stream);
      mv.push_back(i);
    }
    batched_matvec(mv, -1);
    for (int i : mv) {
      DavState& s = st[i];
      double* Vp = s.V.as<double>();
      double* Wp = s.W.as<double>();
      double* vk = Vp + int64_t(s.k) * s.n;
      double* wk = Wp + int64_t(s.k) * s.n;
      b2k::launch_multidot(s.k + 1, Vp, s.n, wk, s.n, s.part, s.VW + s.k, s.kmax, c->stream);
      b2k::launch_multidot(s.k, Wp, s.n, vk, s.n, s.part, s.VW + int64_t(s.k) * s.kmax, 1, c->stream);
      ++s.k;
    }
  }
  for (auto& s : st) {
    b2k::launch_multidot(1, s.u.as<double>(), s.n, s.u.as<double>(), s.n, s.part, s.scal + 2, 1,
                         c->stream);
    B2_CUDA(cudaMemcpyAsync(s.psi, s.u.ptr, sizeof(double) * s.n, cudaMemcpyDeviceToDevice, c->stream));
    b2k::launch_scale_inv_sqrt(s.psi, s.n, s.scal + 2, c->stream);
    s.res.n_matvec = s.nmv;
  }
  B2_CUDA(cudaStreamSynchronize(c->stream));
  for (auto& s : st) {   // release the work buffers now
    s.V.release(); s.W.release(); s.diag.release(); s.u.release(); s.hu.release(); s.t.release();
    s.small.release(); s.d_dims.release(); s.d_offs.release();
  }
}

}  // namespace

// Batched Davidson: the single-problem davidson for every (envs[i], sites[i], psis[i]).
std::vector<DavidsonResult> davidson_batched(Ctx* c, const std::vector<b2_env_s*>& envs,
                                             const std::vector<int>& sites,
                                             const std::vector<double*>& psis,
                                             const b2_dav_opts& o) {
  const int np = int(envs.size());
  std::vector<DavidsonResult> out(np);
  if (np == 0) return out;
  std::vector<DavState> st(np);
  for (int i = 0; i < np; ++i) {
    B2_REQUIRE(envs[i]->ctx == c, B2_EINVAL, "batched Davidson: env of another context");
    st[i].env = envs[i];
    st[i].site = sites[i];
    st[i].psi = psis[i];
  }
  if (o.prec == B2_FP64) {
    davidson_batched_core(c, st, o, B2_FP64, std::vector<const double*>(np, nullptr),
                          std::vector<double>(np, o.conv_tol));
    for (int i = 0; i < np; ++i) out[i] = st[i].res;
    return out;
  }
  B2_REQUIRE(o.prec == B2_BF16X3 || o.prec == B2_TF32X3, B2_EUNSUPPORTED,
             "precision not implemented in this build");
  // mixed-precision refinement (davidson in algo.cpp), all problems in lockstep
  const int rounds = o.refine_max > 0 ? o.refine_max : 4;
  const int max_inner = o.max_iter > 0 ? o.max_iter : 30;
  HostSlots hs(size_t(np) * 2);
  std::vector<DevBuf> w(np), sc(np), r(np);
  std::vector<int64_t> n(np);
  for (int i = 0; i < np; ++i) {
    n[i] = window_program(envs[i], sites[i]).psi.size;
    w[i].reset(c, sizeof(double) * n[i]);
    sc[i].reset(c, sizeof(double) * (256 * 16 + 8));
    r[i].reset(c, sizeof(double) * n[i]);
    double* part = sc[i].as<double>();
    b2k::launch_multidot(1, psis[i], n[i], psis[i], n[i], part, part + 256 * 16, 1, c->stream);
    b2k::launch_scale_inv_sqrt(psis[i], n[i], part + 256 * 16, c->stream);
  }
  std::vector<int> live(np);
  for (int i = 0; i < np; ++i) live[i] = i;
  for (int round = 0; !live.empty(); ++round) {
    std::vector<b2_env_s*> e;
    std::vector<int> s_;
    std::vector<const double*> in;
    std::vector<double*> o_;
    for (int i : live) {
      e.push_back(envs[i]);
      s_.push_back(sites[i]);
      in.push_back(psis[i]);
      o_.push_back(w[i].as<double>());
    }
    double fl = 0;
    heff_apply_batched(c, int(live.size()), e.data(), s_.data(), in.data(), o_.data(), B2_FP64, &fl);
    for (int i : live) {
      out[i].flops += window_program(envs[i], sites[i]).heff.flops;
      out[i].n_matvec += 1;
      double* part = sc[i].as<double>();
      double* s = part + 256 * 16;
      b2k::launch_multidot(1, psis[i], n[i], w[i].as<double>(), n[i], part, s + 1, 1, c->stream);
      B2_CUDA(cudaMemcpyAsync(hs.p + 2 * i, s + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    }
    B2_CUDA(cudaStreamSynchronize(c->stream));
    for (int i : live) {
      double* part = sc[i].as<double>();
      double* s = part + 256 * 16;
      const double th = hs.p[2 * i];
      B2_CUDA(cudaMemcpyAsync(r[i].ptr, w[i].ptr, sizeof(double) * n[i], cudaMemcpyDeviceToDevice,
                              c->stream));
      b2k::launch_axpby(r[i].as<double>(), psis[i], n[i], 1.0, -th, c->stream);
      b2k::launch_multidot(1, r[i].as<double>(), n[i], r[i].as<double>(), n[i], part, s + 2, 1, c->stream);
      B2_CUDA(cudaMemcpyAsync(hs.p + 2 * i + 1, s + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
      out[i].energy = th;
    }
    B2_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<int> next;
    std::vector<DavState> inner;
    std::vector<const double*> w0;
    std::vector<double> tol;
    for (int i : live) {
      const double r2 = hs.p[2 * i + 1];
      out[i].resid2 = r2;
      if (r2 <= o.conv_tol || round >= rounds) continue;
      next.push_back(i);
      DavState s;
      s.env = envs[i];
      s.site = sites[i];
      s.psi = psis[i];
      inner.push_back(std::move(s));
      w0.push_back(w[i].as<double>());
      tol.push_back(std::max(o.conv_tol, 1e-4 * r2));
    }
    if (next.empty()) break;
    b2_dav_opts io = o;
    io.max_iter = max_inner;
    davidson_batched_core(c, inner, io, o.prec, w0, tol);
    for (size_t j = 0; j < next.size(); ++j) {
      out[next[j]].flops += inner[j].res.flops;
      out[next[j]].n_matvec += inner[j].res.n_matvec;
    }
    live = next;
  }
  return out;
}

// Lockstep sweeps of independent problems: step t of a sweep is window t of the forward
// half (t <= n - 2) or window 2(n - 1) - 1 - t of the backward half; after each window, the
// split of the single-problem sweep.  Results per problem and sweep; seconds = wall time
// of the whole batch's sweep.
void sweep_batched(Ctx* c, const std::vector<b2_env_s*>& envs, const b2_sweep_opts& o,
                   b2_sweep_result* res, const int* dims_per_problem) {
  const int np = int(envs.size());
  if (o.dots)
    for (int sw = 0; sw < o.n_sweeps; ++sw)
      B2_REQUIRE(o.dots[sw] == 2, B2_EUNSUPPORTED, "batched sweeps are two-site only");
  if (o.noise)
    for (int sw = 0; sw < o.n_sweeps; ++sw)
      B2_REQUIRE(o.noise[sw] == 0, B2_EUNSUPPORTED, "batched sweeps take no noise");
  B2_REQUIRE(o.n_roots <= 1, B2_EUNSUPPORTED, "batched sweeps solve for one root");
  b2_dav_opts dop;
  dop.max_iter = o.dav_max_iter > 0 ? o.dav_max_iter : 30;
  dop.max_subspace = o.max_subspace > 0 ? o.max_subspace : 30;
  dop.conv_tol = o.conv_tol > 0 ? o.conv_tol : 1e-10;
  dop.prec = o.prec;
  dop.refine_max = 0;
  const double cutoff = o.trunc_cutoff >= 0 ? o.trunc_cutoff : 1e-14;
  std::vector<DevBuf> psi(np);
  int max_steps = 0;
  for (int p = 0; p < np; ++p) {
    b2_env_s* env = envs[p];
    b2_mps_s* mps = env->mps;
    const int n = mps->n;
    B2_REQUIRE(env->ctx == c, B2_EINVAL, "batched sweep: env of another context");
    B2_REQUIRE(mps->center == 0, B2_EINVAL, "sweep needs an MPS centred at site 0");
    B2_REQUIRE(env->L[0].valid, B2_EINVAL, "env not initialised at centre 0");
    for (int k = 2; k <= n; ++k) B2_REQUIRE(env->R[k].valid, B2_EINVAL, "env not initialised at centre 0");
    for (int q = 0; q < p; ++q) B2_REQUIRE(envs[q] != env, B2_EINVAL, "batched sweep: the same env twice");
    WindowProgram& wp = window_program(env, 0);
    psi[p].reset(c, sizeof(double) * std::max<int64_t>(wp.psi.size, 1));
    double fl = 0;
    contract_two_sites(c, mps->bonds[0], mps->bonds[1], mps->sites[0], mps->sites[0].data.as<double>(),
                       mps->sites[1], mps->sites[1].data.as<double>(), wp.psi, psi[p].as<double>(), &fl);
    max_steps = std::max(max_steps, 2 * (n - 1));
  }
  for (int sw = 0; sw < o.n_sweeps; ++sw) {
    B2_CUDA(cudaStreamSynchronize(c->stream));
    const auto t0 = std::chrono::steady_clock::now();
    std::vector<int> Mp(np);
    for (int p = 0; p < np; ++p) {
      Mp[p] = dims_per_problem ? dims_per_problem[size_t(p) * o.n_sweeps + sw] : o.bond_dims[sw];
      B2_REQUIRE(Mp[p] >= 1, B2_EINVAL, "bond dimension must be positive");
    }
    std::vector<b2_sweep_result> r(np);
    double t_dav = 0, t_split = 0;
    for (int t = 0; t < max_steps; ++t) {
      std::vector<b2_env_s*> e;
      std::vector<int> sites, ids;
      std::vector<double*> ps;
      for (int p = 0; p < np; ++p) {
        const int n = envs[p]->mps->n;
        if (t >= 2 * (n - 1)) continue;
        const int i = t <= n - 2 ? t : 2 * (n - 1) - 1 - t;
        ids.push_back(p);
        e.push_back(envs[p]);
        sites.push_back(i);
        ps.push_back(psi[p].as<double>());
      }
      const auto ta = std::chrono::steady_clock::now();
      std::vector<DavidsonResult> d = davidson_batched(c, e, sites, ps, dop);
      const auto tb = std::chrono::steady_clock::now();
      t_dav += std::chrono::duration<double>(tb - ta).count();
      for (size_t j = 0; j < ids.size(); ++j) {
        const int p = ids[j];
        const int n = envs[p]->mps->n;
        const int i = sites[j];
        r[p].matvec_flops += d[j].flops;
        r[p].n_matvec += d[j].n_matvec;
        r[p].energy = d[j].energy;
        double dw = 0;
        if (t <= n - 2) {
          if (i < n - 2) split_left(envs[p], i, psi[p], Mp[p], cutoff, &dw, &r[p].other_flops);
        } else if (i > 0) {
          split_right(envs[p], i, psi[p], Mp[p], cutoff, &dw, &r[p].other_flops, true);
        }
        r[p].discarded_weight = std::max(r[p].discarded_weight, dw);
      }
      B2_CUDA(cudaStreamSynchronize(c->stream));
      t_split += std::chrono::duration<double>(std::chrono::steady_clock::now() - tb).count();
    }
    B2_CUDA(cudaStreamSynchronize(c->stream));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int p = 0; p < np; ++p) {
      r[p].seconds = secs;
      r[p].t_davidson = t_dav;
      r[p].t_split = t_split;
      for (auto& b : envs[p]->mps->bonds) r[p].max_bond = std::max(r[p].max_bond, b.total);
      if (res) res[size_t(p) * o.n_sweeps + sw] = r[p];
    }
  }
  // leave every MPS centred at site 0 (as the single-problem sweep does)
  for (int p = 0; p < np; ++p) {
    double dw = 0, fl = 0;
    split_right(envs[p], 0, psi[p], 1 << 30, cutoff, &dw, &fl, false);
  }
  B2_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace b2
