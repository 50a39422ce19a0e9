// Davidson eigensolver, density-matrix truncation and the two-site sweep (block2 paper,
// Sec. 2.1.2 two-site algorithm, Sec. 2.1.3 (iv) standard Davidson solver, Listing 1 for
// thrds / dav_max_iter).  The host only sequences kernels and reads back scalars needed
// for control flow (residual norms, kept-state counts).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "algo.hpp"

namespace b2 {

using b2k::BufTable;
using b2k::GemmTerm;
using b2k::kTransP;
using b2k::kTransQ;
using b2k::kTwoOp;

static void sync(Ctx* c) { B2_CUDA(cudaStreamSynchronize(c->stream)); }

// Phase timing for diagnosis: with B2_TRACE_TIME set, each mark synchronises the stream
// and prints the wall time since the previous mark.
struct Tracer {
  Ctx* c;
  const char* name;
  int site;
  bool on;
  std::chrono::steady_clock::time_point t;
  Tracer(Ctx* c_, const char* n, int s) : c(c_), name(n), site(s), on(std::getenv("B2_TRACE_TIME")) {
    if (on) {
      sync(c);
      t = std::chrono::steady_clock::now();
    }
  }
  void mark(const char* what) {
    if (!on) return;
    sync(c);
    auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "trace %s %d %s %.3f ms\n", name, site, what,
                 std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

void eigh_batched(Ctx* c, const std::vector<int>& dims, const std::vector<int64_t>& offs,
                  const std::vector<int64_t>& eoffs, const double* a, double* evals,
                  double* evecs, double* flop_counter, int* unconverged) {
  const int n = int(dims.size());
  if (n == 0) return;
  const b2k::JacobiPlan plan = b2k::plan_jacobi(dims);
  std::vector<int64_t> woffs(n, 0);
  int64_t tot_w = 0;
  for (int j = 0; j < n; ++j)
    if (b2k::jacobi_needs_work(dims[j], plan.csize[j])) {
      woffs[j] = tot_w;
      tot_w += 2 * int64_t(dims[j]) * dims[j];
    }
  DevBuf d_dims, d_offs, d_eoffs, d_woffs, d_ids, work;
  upload(c, d_dims, dims);
  upload(c, d_offs, offs);
  upload(c, d_eoffs, eoffs);
  upload(c, d_woffs, woffs);
  upload(c, d_ids, plan.ids);
  if (tot_w > 0) work.reset(c, sizeof(double) * tot_w);
  c->side_init();
  static_assert(Ctx::kSides >= b2k::kJacobiClasses - 1, "one side stream per extra class");
  b2k::JacobiStreams side{};
  for (int k = 0; k < b2k::kJacobiClasses - 1; ++k) {
    side.stream[k] = c->side[k];
    side.join[k] = c->side_join[k];
  }
  side.fork = c->side_fork;
  b2k::launch_jacobi_plan(plan, d_ids.as<int>(), d_dims.as<int>(), d_offs.as<int64_t>(),
                          d_eoffs.as<int64_t>(), a, evals, evecs, work.as<double>(),
                          d_woffs.as<int64_t>(), c->stream, &side,
                          b2k::JacobiCtl{flop_counter, unconverged, c->jacobi_max_sweeps});
  B2_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------ two-site contraction
// out(jl, s1, s2) = sum_jm X(jl, s1 -> jm) Y(jm, s2 -> jr) for a psi layout on bonds (a, c);
// X on bonds (a, b), Y on bonds (b, c).
void contract_two_sites(Ctx* c, const Bond& ba, const Bond& bb, const SiteTensor& X,
                        const double* xd, const SiteTensor& Y, const double* yd,
                        const PsiLayout& lay, double* out, double* flops) {
  GemmProgram prog;
  for (const auto& pb : lay.blocks) {
    int o = prog.add_out(1, pb.off, pb.ml, pb.mr, pb.mr, false);
    int jm = bb.find(ba.q[pb.jl] + kSiteQ[pb.s1]);
    if (jm < 0) continue;
    int xb = X.find(pb.jl, pb.s1), yb = Y.find(jm, pb.s2);
    if (xb < 0 || yb < 0) continue;
    const SiteBlock& Xb = X.blocks[xb];
    const SiteBlock& Yb = Y.blocks[yb];
    if (Xb.jr != jm || Yb.jr != pb.jr) continue;
    GemmTerm t{};
    t.offP = Xb.off; t.bufP = 0; t.ldP = Xb.mr;
    t.offX = Yb.off; t.bufX = 2; t.ldX = Yb.mr;
    t.K1 = Xb.mr;
    t.flags = kTwoOp;
    t.alpha = 1.0;
    prog.add_term(o, t);
  }
  prog.finalize(c);
  BufTable bt{};
  bt.p[0] = const_cast<double*>(xd);
  bt.p[1] = out;
  bt.p[2] = const_cast<double*>(yd);
  prog.launch(c, bt);
  if (flops) *flops += prog.flops;
}

// ------------------------------------------------------------------- Davidson
// Davidson with products in precision mv_prec.  When w0 is given it is H psi / |psi| (an
// FP64 product of the normalised start vector, computed by the caller) and seeds W[0].
static DavidsonResult davidson_core(b2_env_s* env, int site, double* psi, const b2_dav_opts& o,
                                    b2_prec mv_prec, const double* w0, double tol) {
  Ctx* c = env->ctx;
  WindowProgram& wp = window_program(env, site);
  const int64_t n = wp.psi.size;
  B2_REQUIRE(n > 0, B2_EINVAL, "empty two-site wavefunction");
  const int kmax = std::max(2, std::min(o.max_subspace > 0 ? o.max_subspace : 30, 64));
  const int max_iter = o.max_iter > 0 ? o.max_iter : 30;
  DevBuf V(c, sizeof(double) * n * kmax), W(c, sizeof(double) * n * kmax);
  DevBuf diag(c, sizeof(double) * n), u(c, sizeof(double) * n), hu(c, sizeof(double) * n),
      t(c, sizeof(double) * n);
  // small work: partial sums, VW (kmax^2), G (kmax^2), evals, evecs, coefficient vectors
  const int kPart = 256 * 16;
  DevBuf small(c, sizeof(double) * (kPart + 4 * kmax * kmax + 8 * kmax + 16));
  double* part = small.as<double>();
  double* VW = part + kPart;
  double* G = VW + kmax * kmax;
  double* evecs = G + kmax * kmax;
  double* evals = evecs + kmax * kmax;
  double* cvec = evals + kmax;
  double* scal = cvec + 2 * kmax;    // [0] |r|^2, [1] |t|^2, [2] norm of input, [3] breakdown
  DevBuf meta(c, sizeof(int64_t) * 4);
  double* Vp = V.as<double>();
  double* Wp = W.as<double>();
  DavidsonResult res;
  double fl = 0;

  heff_diag(env, site, diag.as<double>());
  // v0 = psi / |psi|
  b2k::launch_multidot(1, psi, n, psi, n, part, scal + 2, 1, c->stream);
  B2_CUDA(cudaMemcpyAsync(Vp, psi, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  b2k::launch_scale_inv_sqrt(Vp, n, scal + 2, c->stream);
  int nmv = 0, k = 1;
  if (w0) {
    B2_CUDA(cudaMemcpyAsync(Wp, w0, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    heff_apply(env, site, Vp, Wp, 0.0, &fl, mv_prec);
    res.flops += fl;
    nmv = 1;
  }
  b2k::launch_multidot(1, Vp, n, Wp, n, part, VW, 1, c->stream);
  // small eigensolver metadata: dims / offsets for the single k x k problem
  // (dims: a table 0..kmax on the device, so that no copy is needed per iteration)
  std::vector<int> dims_h(kmax + 1);
  for (int i = 0; i <= kmax; ++i) dims_h[i] = i;
  int64_t offs_h[2] = {0, 0};
  DevBuf d_dims, d_offs(c, sizeof(int64_t) * 2);
  upload(c, d_dims, dims_h);
  B2_CUDA(cudaMemcpyAsync(d_offs.ptr, offs_h, sizeof(offs_h), cudaMemcpyHostToDevice, c->stream));
  // The extension of the basis is not checked on the host: a correction of norm < 1e-14
  // (breakdown) is zeroed on the device and flags scal[3]; the flag is read with the
  // residual of the next Rayleigh-Ritz step, which is then redone without that vector.
  // One host synchronisation per iteration instead of two.
  B2_CUDA(cudaMemsetAsync(scal + 3, 0, sizeof(double), c->stream));
  double host_sc[2];
  double brk = 0;
  bool stop_after_ritz = false;
  std::vector<double> hist;   // residuals of the iterations so far
  for (;;) {
    cudaEvent_t r0 = nullptr, r1 = nullptr;
    if (c->prof) {
      B2_CUDA(cudaEventCreate(&r0));
      B2_CUDA(cudaEventCreate(&r1));
      B2_CUDA(cudaEventRecord(r0, c->stream));
    }
    b2k::launch_symmetrize(k, VW, kmax, G, c->stream);
    b2k::launch_jacobi(1, d_dims.as<int>() + k, d_offs.as<int64_t>(), d_offs.as<int64_t>(), G,
                       evals, evecs, nullptr, d_offs.as<int64_t>(), k, c->stream);
    if (c->prof) {
      B2_CUDA(cudaEventRecord(r1, c->stream));
      c->rr_events.push_back({r0, r1});
    }
    // lowest Ritz pair: last of the descending eigenvalues, column k-1
    b2k::launch_ritz(k, Vp, Wp, n, evecs + (k - 1), k, evals + (k - 1), diag.as<double>(),
                     u.as<double>(), hu.as<double>(), t.as<double>(), n, part, scal, c->stream);
    B2_CUDA(cudaMemcpyAsync(host_sc, scal, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    B2_CUDA(cudaMemcpyAsync(&res.energy, evals + (k - 1), sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
    B2_CUDA(cudaMemcpyAsync(&brk, scal + 3, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    sync(c);
    if (brk != 0.0) {   // the last vector added was a breakdown: drop it, redo Rayleigh-Ritz
      --k;
      --nmv;
      res.flops -= fl;
      brk = 0.0;
      B2_CUDA(cudaMemsetAsync(scal + 3, 0, sizeof(double), c->stream));
      stop_after_ritz = true;
      continue;
    }
    res.resid2 = host_sc[0];
    if (std::getenv("B2_TRACE_DAVIDSON"))
      std::fprintf(stderr, "davidson site %d k %d nmv %d theta %.15f r2 %.3e\n", site, k, nmv,
                   res.energy, res.resid2);
    B2_REQUIRE(std::isfinite(res.resid2) && std::isfinite(res.energy), B2_ENOCONV,
               "Davidson produced a non-finite value");
    if (mv_prec != B2_FP64)
      B2_REQUIRE(c->take_status() == 0, B2_ETIMEOUT, "tensor-core wait ran out");
    if (stop_after_ritz || res.resid2 <= tol || nmv >= max_iter) break;
    // split-precision products resolve the residual only down to their own error: once it
    // has stopped falling (less than a factor 2 over four products), hand back to the FP64
    // refinement instead of spending products on rounding noise
    hist.push_back(res.resid2);
    if (mv_prec != B2_FP64 && hist.size() > 4 && hist.back() > 0.5 * hist[hist.size() - 5]) break;
    if (k >= kmax) {   // restart from the Ritz vector
      B2_CUDA(cudaMemcpyAsync(Vp, u.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
      B2_CUDA(cudaMemcpyAsync(Wp, hu.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
      k = 1;
      b2k::launch_multidot(1, Vp, n, Wp, n, part, VW, 1, c->stream);
    }
    double* tp = t.as<double>();
    for (int pass = 0; pass < 2; ++pass) {
      b2k::launch_multidot(k, Vp, n, tp, n, part, cvec, 1, c->stream);
      b2k::launch_multiaxpy(k, Vp, n, cvec, tp, n, -1.0, c->stream);
    }
    b2k::launch_multidot(1, tp, n, tp, n, part, scal + 1, 1, c->stream);
    double* vk = Vp + int64_t(k) * n;
    double* wk = Wp + int64_t(k) * n;
    B2_CUDA(cudaMemcpyAsync(vk, tp, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    b2k::launch_scale_inv_sqrt(vk, n, scal + 1, c->stream, scal + 3);
    heff_apply(env, site, vk, wk, 0.0, &fl, mv_prec);
    res.flops += fl;
    ++nmv;
    // VW[j][k] = V_j . W_k (j <= k), VW[k][j] = V_k . W_j (j < k)
    b2k::launch_multidot(k + 1, Vp, n, wk, n, part, VW + k, kmax, c->stream);
    b2k::launch_multidot(k, Wp, n, vk, n, part, VW + int64_t(k) * kmax, 1, c->stream);
    ++k;
  }
  // psi = u / |u|
  b2k::launch_multidot(1, u.as<double>(), n, u.as<double>(), n, part, scal + 2, 1, c->stream);
  B2_CUDA(cudaMemcpyAsync(psi, u.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  b2k::launch_scale_inv_sqrt(psi, n, scal + 2, c->stream);
  res.n_matvec = nmv;
  sync(c);
  return res;
}

// Davidson for H_eff.  FP64: the textbook iteration.  Split precision (mixed-precision
// refinement): each round forms one FP64 product w = H u of the current unit vector u,
// the FP64 Rayleigh quotient theta = u.w and residual r = w - theta u; it stops when
// |r|^2 <= conv_tol.  Otherwise a Davidson solve seeded with the exact pair (u, w) runs with
// split-precision products until its own residual drops by 1e-4 relative to |r|^2 (or
// conv_tol) or max_iter products, and its Ritz vector becomes the next u.  At most
// refine_max (default 4) rounds.  The returned energy and residual are the FP64 ones of
// the returned vector.
DavidsonResult davidson(b2_env_s* env, int site, double* psi, const b2_dav_opts& o) {
  if (o.prec == B2_FP64) return davidson_core(env, site, psi, o, B2_FP64, nullptr, o.conv_tol);
  B2_REQUIRE(o.prec == B2_BF16X3 || o.prec == B2_TF32X3, B2_EUNSUPPORTED,
             "precision not implemented in this build");
  Ctx* c = env->ctx;
  WindowProgram& wp = window_program(env, site);
  const int64_t n = wp.psi.size;
  const int rounds = o.refine_max > 0 ? o.refine_max : 4;
  const int max_inner = o.max_iter > 0 ? o.max_iter : 30;
  DevBuf w(c, sizeof(double) * n), sc(c, sizeof(double) * (256 * 16 + 8));
  double* part = sc.as<double>();
  double* s = part + 256 * 16;
  DavidsonResult total;
  double fl = 0;
  // normalise the guess
  b2k::launch_multidot(1, psi, n, psi, n, part, s, 1, c->stream);
  b2k::launch_scale_inv_sqrt(psi, n, s, c->stream);
  for (int round = 0;; ++round) {
    heff_apply(env, site, psi, w.as<double>(), 0.0, &fl, B2_FP64);
    total.flops += fl;
    total.n_matvec += 1;
    b2k::launch_multidot(1, psi, n, w.as<double>(), n, part, s + 1, 1, c->stream);   // theta
    double th = 0;
    B2_CUDA(cudaMemcpyAsync(&th, s + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    sync(c);
    // r = w - theta u into the scratch of the inner solve's first correction
    DevBuf r(c, sizeof(double) * n);
    B2_CUDA(cudaMemcpyAsync(r.ptr, w.ptr, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    b2k::launch_axpby(r.as<double>(), psi, n, 1.0, -th, c->stream);
    b2k::launch_multidot(1, r.as<double>(), n, r.as<double>(), n, part, s + 2, 1, c->stream);
    double r2 = 0;
    B2_CUDA(cudaMemcpyAsync(&r2, s + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    sync(c);
    total.energy = th;
    total.resid2 = r2;
    if (std::getenv("B2_TRACE_DAVIDSON"))
      std::fprintf(stderr, "refine site %d round %d theta %.15f r2 %.3e\n", site, round, th, r2);
    if (r2 <= o.conv_tol || round >= rounds) break;
    b2_dav_opts inner = o;
    inner.max_iter = max_inner;
    DavidsonResult d = davidson_core(env, site, psi, inner, o.prec, w.as<double>(),
                                     std::max(o.conv_tol, 1e-4 * r2));
    total.flops += d.flops;
    total.n_matvec += d.n_matvec;
  }
  return total;
}

// --------------------------------------------------------------- density matrices
namespace {
struct RhoSector {
  QN q;
  int dim = 0;
  int64_t off = 0, eoff = 0;
  // contributing index groups: (sector of the open bond, site state) -> row offset
  std::vector<std::pair<int, int>> parts;
  std::vector<int> part_off;
};
}  // namespace

// Signature of a density-matrix sector: its quantum numbers and its parts with their
// dimensions (the warm-start cache matches sectors on it).
static std::vector<int64_t> rho_signature(const RhoSector& r) {
  std::vector<int64_t> sig{r.q.key(), r.dim};
  for (size_t a = 0; a < r.parts.size(); ++a) {
    const int end = a + 1 < r.parts.size() ? r.part_off[a + 1] : r.dim;
    sig.push_back((int64_t(r.parts[a].first) << 8) | r.parts[a].second);
    sig.push_back(end - r.part_off[a]);
  }
  return sig;
}

// Eigen-decomposition of the sector density matrices rho into evals / evecs (layout of
// secs), warm-started where the cache holds a basis of the same sector: rho' = V^T rho V,
// Jacobi on rho' (eigenvectors W), evecs = V W.  The cache then holds evecs.
static void eig_warm(Ctx* c, std::vector<RhoSector>& secs, DevBuf& rho, DevBuf& evals,
                     DevBuf& evecs, RhoCache* cache, int* unconv) {
  const int ns = int(secs.size());
  std::vector<int> dims(ns);
  std::vector<int64_t> offs(ns), eoffs(ns), warm(ns, -1);
  int64_t tot = 0;
  std::vector<std::vector<int64_t>> sigs(ns);
  bool any_warm = false;
  for (int j = 0; j < ns; ++j) {
    dims[j] = secs[j].dim;
    offs[j] = secs[j].off;
    eoffs[j] = secs[j].eoff;
    tot = std::max(tot, secs[j].off + int64_t(secs[j].dim) * secs[j].dim);
    sigs[j] = rho_signature(secs[j]);
    if (cache && cache->V.ptr) {
      auto it = cache->by_sig.find(sigs[j]);
      if (it != cache->by_sig.end() && it->second.second == dims[j] && dims[j] > 1) {
        warm[j] = it->second.first;
        any_warm = true;
      }
    }
  }
  double* flops_ctr = c->prof ? c->d_eig_flops : nullptr;
  if (!any_warm) {
    eigh_batched(c, dims, offs, eoffs, rho.as<double>(), evals.as<double>(), evecs.as<double>(),
                 flops_ctr, unconv);
  } else {
    DevBuf rho2(c, sizeof(double) * std::max<int64_t>(tot, 1));
    DevBuf W(c, sizeof(double) * std::max<int64_t>(tot, 1));
    BufTable bt{};
    bt.p[0] = rho.as<double>();
    bt.p[1] = rho2.as<double>();
    bt.p[2] = W.as<double>();
    bt.p[3] = cache->V.as<double>();
    bt.p[4] = evecs.as<double>();
    GemmProgram p1, p2;
    std::vector<b2k::CopyTask> cold_in;
    for (int j = 0; j < ns; ++j) {
      const int d = dims[j];
      if (warm[j] < 0) {
        cold_in.push_back({offs[j], offs[j], d, d, d, d, 0, 0, 1});
        continue;
      }
      GemmTerm t{};
      t.K1 = d;
      t.alpha = 1.0;
      // W = rho V
      t.offP = offs[j]; t.bufP = 0; t.ldP = d;
      t.offX = warm[j]; t.bufX = 3; t.ldX = d;
      t.flags = kTwoOp;
      p1.add_term(p1.add_out(2, offs[j], d, d, d, false), t);
      // rho' = V^T W
      t.offP = warm[j]; t.bufP = 3; t.ldP = d;
      t.offX = offs[j]; t.bufX = 2; t.ldX = d;
      t.flags = kTwoOp | kTransP;
      p2.add_term(p2.add_out(1, offs[j], d, d, d, false), t);
    }
    p1.finalize(c);
    p2.finalize(c);
    p1.launch(c, bt);
    p2.launch(c, bt);
    DevBuf d_cin;
    if (!cold_in.empty()) {
      upload(c, d_cin, cold_in);
      b2k::launch_copy(int(cold_in.size()), d_cin.as<b2k::CopyTask>(), bt, c->stream);
    }
    eigh_batched(c, dims, offs, eoffs, rho2.as<double>(), evals.as<double>(), W.as<double>(),
                 flops_ctr, unconv);
    // evecs = V W (warm sectors), W (cold sectors)
    GemmProgram p3;
    std::vector<b2k::CopyTask> cold_out;
    for (int j = 0; j < ns; ++j) {
      const int d = dims[j];
      if (warm[j] < 0) {
        cold_out.push_back({offs[j], offs[j], d, d, d, d, 0, 2, 4});
        continue;
      }
      GemmTerm t{};
      t.K1 = d;
      t.alpha = 1.0;
      t.offP = warm[j]; t.bufP = 3; t.ldP = d;
      t.offX = offs[j]; t.bufX = 2; t.ldX = d;
      t.flags = kTwoOp;
      p3.add_term(p3.add_out(4, offs[j], d, d, d, false), t);
    }
    p3.finalize(c);
    p3.launch(c, bt);
    DevBuf d_cout;
    if (!cold_out.empty()) {
      upload(c, d_cout, cold_out);
      b2k::launch_copy(int(cold_out.size()), d_cout.as<b2k::CopyTask>(), bt, c->stream);
    }
    B2_CUDA(cudaGetLastError());
  }
  if (cache) {
    cache->by_sig.clear();
    for (int j = 0; j < ns; ++j) cache->by_sig[sigs[j]] = {offs[j], dims[j]};
    cache->V.reset(c, sizeof(double) * std::max<int64_t>(tot, 1));
    B2_CUDA(cudaMemcpyAsync(cache->V.ptr, evecs.ptr, sizeof(double) * std::max<int64_t>(tot, 1),
                            cudaMemcpyDeviceToDevice, c->stream));
  }
}

// Batched eigen-decomposition of the sector density matrices, then the global selection.
// Returns kept counts per sector (host) and the discarded weight.
static std::vector<int> eig_and_select(Ctx* c, std::vector<RhoSector>& secs, DevBuf& rho,
                                       DevBuf& evals, DevBuf& evecs, int M, double cutoff,
                                       double* discarded, RhoCache* cache = nullptr) {
  int ns = int(secs.size());
  std::vector<int> dims(ns), sec_of;
  std::vector<int64_t> offs(ns), eoffs(ns);
  int64_t tot_e = 0;
  int max_dim = 0;
  for (int j = 0; j < ns; ++j) {
    dims[j] = secs[j].dim;
    offs[j] = secs[j].off;
    eoffs[j] = secs[j].eoff;
    tot_e += dims[j];
    max_dim = std::max(max_dim, dims[j]);
    for (int t = 0; t < dims[j]; ++t) sec_of.push_back(j);
  }
  if (std::getenv("B2_TRACE_TIME")) {
    std::vector<int> sd(dims.begin(), dims.end());
    std::sort(sd.rbegin(), sd.rend());
    double cubes = 0;
    for (int d : sd) cubes += double(d) * d * d;
    std::fprintf(stderr, "trace rho sectors %d dims %d %d %d %d sum_m3 %.3g\n", ns,
                 sd.size() > 0 ? sd[0] : 0, sd.size() > 1 ? sd[1] : 0, sd.size() > 2 ? sd[2] : 0,
                 sd.size() > 3 ? sd[3] : 0, cubes);
  }
  B2_REQUIRE(max_dim <= 1024, B2_EUNSUPPORTED, "density-matrix sector larger than 1024");
  B2_REQUIRE(tot_e <= b2k::kSelectMax, B2_EUNSUPPORTED, "too many density-matrix eigenvalues");
  DevBuf d_sec, d_kept(c, sizeof(int) * ns + 16), d_w(c, 2 * sizeof(double));
  upload(c, d_sec, sec_of);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->prof) {
    B2_CUDA(cudaEventCreate(&e0));
    B2_CUDA(cudaEventCreate(&e1));
    B2_CUDA(cudaEventRecord(e0, c->stream));
  }
  int* unconv = c->status() + 1;   // status word 1: Jacobi sweep limit reached
  eig_warm(c, secs, rho, evals, evecs, cache, unconv);
  if (c->prof) {
    B2_CUDA(cudaEventRecord(e1, c->stream));
    c->eig_events.push_back({e0, e1});
  }
  b2k::launch_select(int(tot_e), evals.as<double>(), d_sec.as<int>(), ns, M, cutoff,
                     d_kept.as<int>(), d_w.as<double>(), c->stream);
  B2_CUDA(cudaGetLastError());
  std::vector<int> kept(ns);
  double w[2];
  int n_unconv = 0;
  B2_CUDA(cudaMemcpyAsync(kept.data(), d_kept.ptr, sizeof(int) * ns, cudaMemcpyDeviceToHost, c->stream));
  B2_CUDA(cudaMemcpyAsync(w, d_w.ptr, sizeof(w), cudaMemcpyDeviceToHost, c->stream));
  B2_CUDA(cudaMemcpyAsync(&n_unconv, unconv, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  sync(c);
  if (n_unconv != 0) {
    B2_CUDA(cudaMemsetAsync(unconv, 0, sizeof(int), c->stream));
    B2_REQUIRE(false, B2_ENOCONV,
               "density-matrix eigensolver: " + std::to_string(n_unconv) +
                   " sector(s) still rotating after the sweep limit");
  }
  *discarded = w[0];
  return kept;
}

// Forward split of window i: psi -> A_i (left-orthonormal, new bond i+1) and the guess for
// window i+1.  Updates mps->bonds[i+1], mps->sites[i], L_{i+1}; writes the new psi.
void split_left(b2_env_s* env, int i, DevBuf& psi, int M, double cutoff, double* discarded,
                double* flops) {
  Ctx* c = env->ctx;
  Tracer tr(c, "split_left", i);
  b2_mps_s* mps = env->mps;
  WindowProgram& wp = window_program(env, i);
  const PsiLayout lay = wp.psi;
  const Bond& bl = mps->bonds[i];
  // sectors of bond i+1 from (jl, s1)
  std::map<int64_t, int> sidx;
  std::vector<RhoSector> secs;
  std::vector<QN> qs;
  for (int jl = 0; jl < bl.size(); ++jl)
    for (int s1 = 0; s1 < 4; ++s1) {
      bool any = false;
      for (int s2 = 0; s2 < 4; ++s2) any |= lay.find(jl, s1, s2) >= 0;
      if (any) qs.push_back(bl.q[jl] + kSiteQ[s1]);
    }
  std::sort(qs.begin(), qs.end());
  qs.erase(std::unique(qs.begin(), qs.end()), qs.end());
  for (auto& q : qs) {
    sidx[q.key()] = int(secs.size());
    RhoSector r;
    r.q = q;
    secs.push_back(r);
  }
  for (int jl = 0; jl < bl.size(); ++jl)
    for (int s1 = 0; s1 < 4; ++s1) {
      auto it = sidx.find((bl.q[jl] + kSiteQ[s1]).key());
      if (it == sidx.end()) continue;
      RhoSector& r = secs[it->second];
      r.parts.push_back({jl, s1});
      r.part_off.push_back(r.dim);
      r.dim += bl.m[jl];
    }
  int64_t tot = 0, tote = 0;
  for (auto& r : secs) {
    r.off = tot;
    r.eoff = tote;
    tot += int64_t(r.dim) * r.dim;
    tote += r.dim;
  }
  DevBuf rho(c, sizeof(double) * std::max<int64_t>(tot, 1));
  DevBuf evals(c, sizeof(double) * std::max<int64_t>(tote, 1));
  DevBuf evecs(c, sizeof(double) * std::max<int64_t>(tot, 1));
  // rho_q[(jl,s1),(jl',s1')] = sum_s2 psi(jl,s1,s2) psi(jl',s1',s2)^T
  GemmProgram prog;
  for (auto& r : secs)
    for (size_t a = 0; a < r.parts.size(); ++a)
      for (size_t b = 0; b < r.parts.size(); ++b) {
        int ja = r.parts[a].first, sa = r.parts[a].second;
        int jb = r.parts[b].first, sb = r.parts[b].second;
        int o = prog.add_out(1, r.off + int64_t(r.part_off[a]) * r.dim + r.part_off[b], bl.m[ja],
                             bl.m[jb], r.dim, false);
        for (int s2 = 0; s2 < 4; ++s2) {
          int pa = lay.find(ja, sa, s2), pb = lay.find(jb, sb, s2);
          if (pa < 0 || pb < 0) continue;
          const PsiBlock& A = lay.blocks[pa];
          const PsiBlock& B = lay.blocks[pb];
          GemmTerm t{};
          t.offP = A.off; t.bufP = 0; t.ldP = A.mr;
          t.offX = B.off; t.bufX = 0; t.ldX = B.mr;     // op(X) = B^T
          t.K1 = A.mr;
          t.flags = kTwoOp | kTransQ;
          t.alpha = 1.0;
          prog.add_term(o, t);
        }
      }
  prog.finalize(c);
  BufTable bt{};
  bt.p[0] = psi.as<double>();
  bt.p[1] = rho.as<double>();
  prog.launch(c, bt);
  *flops += prog.flops;
  tr.mark("rho");
  std::vector<int> kept = eig_and_select(c, secs, rho, evals, evecs, M, cutoff, discarded,
                                         &env->rho_cache[2 * i]);
  tr.mark("eig+select");

  // new bond i+1 and A_i
  Bond nb;
  std::vector<int> new_idx(secs.size(), -1);
  for (size_t j = 0; j < secs.size(); ++j)
    if (kept[j] > 0) {
      new_idx[j] = nb.size();
      nb.q.push_back(secs[j].q);
      nb.m.push_back(kept[j]);
    }
  B2_REQUIRE(nb.size() > 0, B2_ENOCONV, "truncation kept no state");
  nb.finalize();
  SiteTensor A;
  A.build(bl, nb);
  A.data.reset(c, sizeof(double) * std::max<int64_t>(A.size, 1));
  std::vector<b2k::CopyTask> copies;
  for (size_t j = 0; j < secs.size(); ++j) {
    if (new_idx[j] < 0) continue;
    const RhoSector& r = secs[j];
    for (size_t a = 0; a < r.parts.size(); ++a) {
      int ab = A.find(r.parts[a].first, r.parts[a].second);
      B2_REQUIRE(ab >= 0, B2_EINVAL, "internal: split layout");
      const SiteBlock& blk = A.blocks[ab];
      b2k::CopyTask ct{};
      ct.src = r.off + int64_t(r.part_off[a]) * r.dim;
      ct.dst = blk.off;
      ct.rows = blk.ml;
      ct.cols = blk.mr;
      ct.lds = r.dim;
      ct.ldd = blk.mr;
      ct.trans = 0;
      ct.bsrc = 0;
      ct.bdst = 1;
      copies.push_back(ct);
    }
  }
  DevBuf d_copies;
  upload(c, d_copies, copies);
  BufTable cb{};
  cb.p[0] = evecs.as<double>();
  cb.p[1] = A.data.as<double>();
  b2k::launch_copy(int(copies.size()), d_copies.as<b2k::CopyTask>(), cb, c->stream);
  B2_CUDA(cudaGetLastError());

  // C(jt, s2 -> jr) = sum_{(jl,s1) in jt} A(jl,s1,jt)^T psi(jl,s1,s2)
  const Bond& br = mps->bonds[i + 2];
  SiteTensor C;
  C.build(nb, br);
  C.data.reset(c, sizeof(double) * std::max<int64_t>(C.size, 1));
  GemmProgram pc;
  for (const auto& cbk : C.blocks) {
    int o = pc.add_out(1, cbk.off, cbk.ml, cbk.mr, cbk.mr, false);
    int j = -1;
    for (size_t x = 0; x < secs.size(); ++x)
      if (new_idx[x] == cbk.jl) j = int(x);
    const RhoSector& r = secs[j];
    for (size_t a = 0; a < r.parts.size(); ++a) {
      int jl = r.parts[a].first, s1 = r.parts[a].second;
      int pb = lay.find(jl, s1, cbk.s);
      if (pb < 0) continue;
      const PsiBlock& P = lay.blocks[pb];
      if (P.jr != cbk.jr) continue;
      const SiteBlock& Ab = A.blocks[A.find(jl, s1)];
      GemmTerm t{};
      t.offP = Ab.off; t.bufP = 2; t.ldP = Ab.mr;    // op(P) = A^T [m_jt x m_jl]
      t.offX = P.off; t.bufX = 0; t.ldX = P.mr;
      t.K1 = Ab.ml;
      t.flags = kTwoOp | kTransP;
      t.alpha = 1.0;
      pc.add_term(o, t);
    }
  }
  pc.finalize(c);
  BufTable bc{};
  bc.p[0] = psi.as<double>();
  bc.p[1] = C.data.as<double>();
  bc.p[2] = A.data.as<double>();
  pc.launch(c, bc);
  *flops += pc.flops;

  // commit: site i, bond i+1; environments on bond i+1 change
  mps->bonds[i + 1] = nb;
  mps->sites[i] = std::move(A);
  env->R[i + 1].valid = false;
  tr.mark("site+C");
  env_update_left(env, i);
  tr.mark("env");
  // guess for window i+1: C . B_{i+2}
  if (i + 2 < mps->n) {
    PsiLayout nl;
    nl.build(mps->bonds[i + 1], mps->bonds[i + 3]);
    DevBuf np(c, sizeof(double) * std::max<int64_t>(nl.size, 1));
    contract_two_sites(c, mps->bonds[i + 1], mps->bonds[i + 2], C, C.data.as<double>(),
                       mps->sites[i + 2], mps->sites[i + 2].data.as<double>(), nl, np.as<double>(),
                       flops);
    psi = std::move(np);
  }
}

// Backward split of window i: psi -> B_{i+1} (right-orthonormal, new bond i+1) and the guess
// for window i-1.  Updates mps->bonds[i+1], mps->sites[i+1], R_{i+1}; writes the new psi.
// With i == 0 and guess == false it only re-canonicalises (site 0 := C).
void split_right(b2_env_s* env, int i, DevBuf& psi, int M, double cutoff, double* discarded,
                 double* flops, bool make_guess) {
  Ctx* c = env->ctx;
  Tracer tr(c, "split_right", i);
  b2_mps_s* mps = env->mps;
  WindowProgram& wp = window_program(env, i);
  const PsiLayout lay = wp.psi;
  const Bond& bl = mps->bonds[i];
  const Bond& br = mps->bonds[i + 2];
  std::map<int64_t, int> sidx;
  std::vector<RhoSector> secs;
  std::vector<QN> qs;
  for (int jr = 0; jr < br.size(); ++jr)
    for (int s2 = 0; s2 < 4; ++s2) {
      bool any = false;
      for (const auto& pb : lay.blocks) any |= (pb.jr == jr && pb.s2 == s2);
      if (any) qs.push_back(br.q[jr] - kSiteQ[s2]);
    }
  std::sort(qs.begin(), qs.end());
  qs.erase(std::unique(qs.begin(), qs.end()), qs.end());
  for (auto& q : qs) {
    sidx[q.key()] = int(secs.size());
    RhoSector r;
    r.q = q;
    secs.push_back(r);
  }
  // rows of rho_q: (s2, jr) in (s2, jr) order
  for (int s2 = 0; s2 < 4; ++s2)
    for (int jr = 0; jr < br.size(); ++jr) {
      auto it = sidx.find((br.q[jr] - kSiteQ[s2]).key());
      if (it == sidx.end()) continue;
      RhoSector& r = secs[it->second];
      r.parts.push_back({jr, s2});
      r.part_off.push_back(r.dim);
      r.dim += br.m[jr];
    }
  int64_t tot = 0, tote = 0;
  for (auto& r : secs) {
    r.off = tot;
    r.eoff = tote;
    tot += int64_t(r.dim) * r.dim;
    tote += r.dim;
  }
  DevBuf rho(c, sizeof(double) * std::max<int64_t>(tot, 1));
  DevBuf evals(c, sizeof(double) * std::max<int64_t>(tote, 1));
  DevBuf evecs(c, sizeof(double) * std::max<int64_t>(tot, 1));
  // rho_q[(s2,jr),(s2',jr')] = sum_{(jl,s1) in q} psi(jl,s1,s2)^T psi(jl,s1,s2')
  GemmProgram prog;
  for (auto& r : secs)
    for (size_t a = 0; a < r.parts.size(); ++a)
      for (size_t b = 0; b < r.parts.size(); ++b) {
        int jra = r.parts[a].first, sa = r.parts[a].second;
        int jrb = r.parts[b].first, sb = r.parts[b].second;
        int o = prog.add_out(1, r.off + int64_t(r.part_off[a]) * r.dim + r.part_off[b], br.m[jra],
                             br.m[jrb], r.dim, false);
        for (int jl = 0; jl < bl.size(); ++jl)
          for (int s1 = 0; s1 < 4; ++s1) {
            if (!(bl.q[jl] + kSiteQ[s1] == r.q)) continue;
            int pa = lay.find(jl, s1, sa), pb = lay.find(jl, s1, sb);
            if (pa < 0 || pb < 0) continue;
            const PsiBlock& A = lay.blocks[pa];
            const PsiBlock& B = lay.blocks[pb];
            if (A.jr != jra || B.jr != jrb) continue;
            GemmTerm t{};
            t.offP = A.off; t.bufP = 0; t.ldP = A.mr;    // op(P) = A^T [m_jra x m_jl]
            t.offX = B.off; t.bufX = 0; t.ldX = B.mr;    // X [m_jl x m_jrb]
            t.K1 = A.ml;
            t.flags = kTwoOp | kTransP;
            t.alpha = 1.0;
            prog.add_term(o, t);
          }
      }
  prog.finalize(c);
  BufTable bt{};
  bt.p[0] = psi.as<double>();
  bt.p[1] = rho.as<double>();
  prog.launch(c, bt);
  *flops += prog.flops;
  tr.mark("rho");
  std::vector<int> kept = eig_and_select(c, secs, rho, evals, evecs, M, cutoff, discarded,
                                         &env->rho_cache[2 * i + 1]);
  tr.mark("eig+select");

  Bond nb;
  std::vector<int> new_idx(secs.size(), -1);
  for (size_t j = 0; j < secs.size(); ++j)
    if (kept[j] > 0) {
      new_idx[j] = nb.size();
      nb.q.push_back(secs[j].q);
      nb.m.push_back(kept[j]);
    }
  B2_REQUIRE(nb.size() > 0, B2_ENOCONV, "truncation kept no state");
  nb.finalize();
  // B_{i+1}(jt, s2 -> jr) = V_q[rows (s2, jr), kept]^T
  SiteTensor Bt;
  Bt.build(nb, br);
  Bt.data.reset(c, sizeof(double) * std::max<int64_t>(Bt.size, 1));
  std::vector<b2k::CopyTask> copies;
  for (size_t j = 0; j < secs.size(); ++j) {
    if (new_idx[j] < 0) continue;
    const RhoSector& r = secs[j];
    for (size_t a = 0; a < r.parts.size(); ++a) {
      int jr = r.parts[a].first, s2 = r.parts[a].second;
      int bb = Bt.find(new_idx[j], s2);
      B2_REQUIRE(bb >= 0 && Bt.blocks[bb].jr == jr, B2_EINVAL, "internal: split layout");
      const SiteBlock& blk = Bt.blocks[bb];
      b2k::CopyTask ct{};
      ct.src = r.off + int64_t(r.part_off[a]) * r.dim;   // V rows of (s2, jr), columns kept
      ct.dst = blk.off;
      ct.rows = blk.ml;     // kept
      ct.cols = blk.mr;     // m_jr
      ct.lds = r.dim;
      ct.ldd = blk.mr;
      ct.trans = 1;         // dst[t][x] = V[(row x) * dim + t]
      ct.bsrc = 0;
      ct.bdst = 1;
      copies.push_back(ct);
    }
  }
  DevBuf d_copies;
  upload(c, d_copies, copies);
  BufTable cb{};
  cb.p[0] = evecs.as<double>();
  cb.p[1] = Bt.data.as<double>();
  b2k::launch_copy(int(copies.size()), d_copies.as<b2k::CopyTask>(), cb, c->stream);
  B2_CUDA(cudaGetLastError());

  // C(jl, s1 -> jt) = sum_s2 psi(jl,s1,s2) B(jt,s2,jr)^T
  SiteTensor C;
  C.build(bl, nb);
  C.data.reset(c, sizeof(double) * std::max<int64_t>(C.size, 1));
  GemmProgram pc;
  for (const auto& cbk : C.blocks) {
    int o = pc.add_out(1, cbk.off, cbk.ml, cbk.mr, cbk.mr, false);
    for (int s2 = 0; s2 < 4; ++s2) {
      int pb = lay.find(cbk.jl, cbk.s, s2);
      if (pb < 0) continue;
      const PsiBlock& P = lay.blocks[pb];
      int bb = Bt.find(cbk.jr, s2);
      if (bb < 0 || Bt.blocks[bb].jr != P.jr) continue;
      const SiteBlock& Bb = Bt.blocks[bb];
      GemmTerm t{};
      t.offP = P.off; t.bufP = 0; t.ldP = P.mr;
      t.offX = Bb.off; t.bufX = 2; t.ldX = Bb.mr;   // op(X) = B^T [m_jr x m_jt]
      t.K1 = P.mr;
      t.flags = kTwoOp | kTransQ;
      t.alpha = 1.0;
      pc.add_term(o, t);
    }
  }
  pc.finalize(c);
  BufTable bc{};
  bc.p[0] = psi.as<double>();
  bc.p[1] = C.data.as<double>();
  bc.p[2] = Bt.data.as<double>();
  pc.launch(c, bc);
  *flops += pc.flops;

  mps->bonds[i + 1] = nb;
  mps->sites[i + 1] = std::move(Bt);
  env->L[i + 1].valid = false;
  tr.mark("site+C");
  env_update_right(env, i + 1);
  tr.mark("env");
  if (make_guess && i > 0) {
    PsiLayout nl;
    nl.build(mps->bonds[i - 1], mps->bonds[i + 1]);
    DevBuf np(c, sizeof(double) * std::max<int64_t>(nl.size, 1));
    contract_two_sites(c, mps->bonds[i - 1], mps->bonds[i], mps->sites[i - 1],
                       mps->sites[i - 1].data.as<double>(), C, C.data.as<double>(), nl,
                       np.as<double>(), flops);
    psi = std::move(np);
  } else {
    // centre stays on site i: it holds C
    mps->sites[i] = std::move(C);
    mps->center = i;
  }
}

// ------------------------------------------------------------------------ sweep
void sweep(b2_env_s* env, const b2_sweep_opts& o, b2_sweep_result* res) {
  Ctx* c = env->ctx;
  b2_mps_s* mps = env->mps;
  const int n = mps->n;
  B2_REQUIRE(mps->center == 0, B2_EINVAL, "sweep needs an MPS centred at site 0");
  B2_REQUIRE(env->L[0].valid, B2_EINVAL, "env not initialised at centre 0");
  for (int k = 2; k <= n; ++k) B2_REQUIRE(env->R[k].valid, B2_EINVAL, "env not initialised at centre 0");
  b2_dav_opts dop;
  dop.max_iter = o.dav_max_iter > 0 ? o.dav_max_iter : 30;
  dop.max_subspace = o.max_subspace > 0 ? o.max_subspace : 30;
  dop.conv_tol = o.conv_tol > 0 ? o.conv_tol : 1e-10;
  dop.prec = o.prec;
  dop.refine_max = 0;
  const double cutoff = o.trunc_cutoff >= 0 ? o.trunc_cutoff : 1e-14;
  // psi of window 0
  DevBuf psi;
  {
    WindowProgram& wp = window_program(env, 0);
    psi.reset(c, sizeof(double) * std::max<int64_t>(wp.psi.size, 1));
    double fl = 0;
    contract_two_sites(c, mps->bonds[0], mps->bonds[1], mps->sites[0], mps->sites[0].data.as<double>(),
                       mps->sites[1], mps->sites[1].data.as<double>(), wp.psi, psi.as<double>(), &fl);
  }
  for (int sw = 0; sw < o.n_sweeps; ++sw) {
    B2_CUDA(cudaStreamSynchronize(c->stream));
    auto t0 = std::chrono::steady_clock::now();
    const int M = o.bond_dims[sw];
    B2_REQUIRE(M >= 1, B2_EINVAL, "bond dimension must be positive");
    b2_sweep_result r{};
    double dw = 0, e = 0;
    auto now = [] { return std::chrono::steady_clock::now(); };
    auto secs = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
      return std::chrono::duration<double>(b - a).count();
    };
    auto solve = [&](int i) {
      auto ta = now();
      DavidsonResult d = davidson(env, i, psi.as<double>(), dop);
      r.t_davidson += secs(ta, now());
      r.matvec_flops += d.flops;
      r.n_matvec += d.n_matvec;
      e = d.energy;
    };
    for (int i = 0; i <= n - 2; ++i) {
      solve(i);
      if (i < n - 2) {
        auto ta = now();
        split_left(env, i, psi, M, cutoff, &dw, &r.other_flops);
        r.t_split += secs(ta, now());
        r.discarded_weight = std::max(r.discarded_weight, dw);
      }
    }
    for (int i = n - 2; i >= 0; --i) {
      solve(i);
      if (i > 0) {
        auto ta = now();
        split_right(env, i, psi, M, cutoff, &dw, &r.other_flops, true);
        r.t_split += secs(ta, now());
        r.discarded_weight = std::max(r.discarded_weight, dw);
      }
    }
    B2_CUDA(cudaStreamSynchronize(c->stream));
    r.energy = e;
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (auto& b : mps->bonds) r.max_bond = std::max(r.max_bond, b.total);
    if (res) res[sw] = r;
  }
  // leave the MPS centred at site 0: B_1 from psi of window 0 without truncation
  double dw = 0, fl = 0;
  split_right(env, 0, psi, 1 << 30, 0.0, &dw, &fl, false);
  sync(c);
}

}  // namespace b2
