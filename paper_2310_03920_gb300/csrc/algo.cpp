// Davidson eigensolver, density-matrix truncation and the two-site sweep (block2 paper,
// Sec. 2.1.2 two-site algorithm, Sec. 2.1.3 (iv) standard Davidson solver, Listing 1 for
// thrds / dav_max_iter).  The host only sequences kernels and reads back scalars needed
// for control flow (residual norms, kept-state counts).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <unordered_map>

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

// Lowest n_roots eigenpairs of H_eff (FP64 products): the block form of the Davidson method
// (several roots, Liu 1978).  psis: n_roots vectors of the window layout, one after the
// other; in: guesses, out: unit eigenvectors.  Guesses are orthonormalised in order (two
// Gram-Schmidt passes); one whose remainder has norm <= 1e-8 is replaced by the unit vector at
// the smallest diagonal element not used yet (ties by position).  Rayleigh-Ritz on V^T H V;
// the n_roots lowest Ritz pairs; stop when every |r_j|^2 <= conv_tol or after max_iter
// products; else the corrections r_j / (D - theta_j) of the unconverged roots, in root order,
// are orthogonalised twice against the subspace and added unless their norm is <= 1e-14; a
// subspace that cannot take them restarts from the Ritz vectors.  One host synchronisation
// per iteration and per added vector (its norm decides whether it is kept).
std::vector<double> davidson_roots(b2_env_s* env, int win, double* psis, int n_roots,
                                   const b2_dav_opts& o, int* n_matvec, double* max_resid2,
                                   double* flops_out) {
  Ctx* c = env->ctx;
  WindowProgram& wp = window_program(env, win);
  const int64_t n = wp.psi.size;
  const int k = n_roots;
  B2_REQUIRE(n > 0, B2_EINVAL, "empty wavefunction");
  B2_REQUIRE(k >= 1 && k <= 16 && int64_t(k) <= n, B2_EINVAL, "n_roots must be in [1, 16] and <= size");
  const int kmax = std::max(2 * k, std::min(o.max_subspace > 0 ? o.max_subspace : 40, 64));
  const int max_iter = o.max_iter > 0 ? o.max_iter : 100;
  const double tol = o.conv_tol > 0 ? o.conv_tol : 1e-10;
  DevBuf V(c, sizeof(double) * n * kmax), W(c, sizeof(double) * n * kmax);
  DevBuf diag(c, sizeof(double) * n), U(c, sizeof(double) * n * k), HU(c, sizeof(double) * n * k),
      T(c, sizeof(double) * n * k), tmp(c, sizeof(double) * n);
  const int kPart = 256 * 16;
  DevBuf small(c, sizeof(double) * (kPart + 4 * kmax * kmax + 8 * kmax + 4 * 16 + 16));
  double* part = small.as<double>();
  double* VW = part + kPart;
  double* G = VW + kmax * kmax;
  double* evecs = G + kmax * kmax;
  double* evals = evecs + kmax * kmax;
  double* cvec = evals + kmax;
  double* r2d = cvec + 2 * kmax;     // |r_j|^2
  double* nrm = r2d + 16;            // norms^2 of vectors being added
  double* Vp = V.as<double>();
  double* Wp = W.as<double>();
  double fl = 0, flops = 0;
  int nmv = 0, m = 0;
  heff_diag(env, win, diag.as<double>());
  auto orthonormal_add = [&](const double* x, double thresh2) -> bool {
    // x -> V[m] after two passes against V[0..m); kept if |remainder|^2 > thresh2
    double* vm = Vp + int64_t(m) * n;
    B2_CUDA(cudaMemcpyAsync(vm, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    for (int pass = 0; pass < 2 && m > 0; ++pass) {
      b2k::launch_multidot(m, Vp, n, vm, n, part, cvec, 1, c->stream);
      b2k::launch_multiaxpy(m, Vp, n, cvec, vm, n, -1.0, c->stream);
    }
    b2k::launch_multidot(1, vm, n, vm, n, part, nrm, 1, c->stream);
    double h2 = 0;
    B2_CUDA(cudaMemcpyAsync(&h2, nrm, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    sync(c);
    if (!(h2 > thresh2)) return false;
    b2k::launch_scale_inv_sqrt(vm, n, nrm, c->stream);
    return true;
  };
  auto add_product = [&]() {   // W[m] = H V[m]; VW updated; m += 1
    double* vm = Vp + int64_t(m) * n;
    double* wm = Wp + int64_t(m) * n;
    heff_apply(env, win, vm, wm, 0.0, &fl, B2_FP64);
    flops += fl;
    ++nmv;
    b2k::launch_multidot(m + 1, Vp, n, wm, n, part, VW + m, kmax, c->stream);
    if (m > 0) b2k::launch_multidot(m, Wp, n, vm, n, part, VW + int64_t(m) * kmax, 1, c->stream);
    ++m;
  };
  // guesses, completed by unit vectors at the smallest unused diagonal elements
  std::vector<int64_t> order;
  size_t next_unit = 0;
  for (int j = 0; j < k; ++j) {
    if (orthonormal_add(psis + int64_t(j) * n, 1e-16)) {
      add_product();
      continue;
    }
    if (order.empty()) {
      std::vector<double> dh(n);
      B2_CUDA(cudaMemcpyAsync(dh.data(), diag.ptr, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
      sync(c);
      order.resize(n);
      for (int64_t x = 0; x < n; ++x) order[x] = x;
      std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) { return dh[a] < dh[b]; });
    }
    bool ok = false;
    while (!ok && next_unit < order.size()) {
      B2_CUDA(cudaMemsetAsync(tmp.ptr, 0, sizeof(double) * n, c->stream));
      const double one = 1.0;
      B2_CUDA(cudaMemcpyAsync(tmp.as<double>() + order[next_unit++], &one, sizeof(double),
                              cudaMemcpyHostToDevice, c->stream));
      ok = orthonormal_add(tmp.as<double>(), 1e-16);
    }
    B2_REQUIRE(ok, B2_ENOCONV, "no independent start vector");
    add_product();
  }
  // dims table 0..kmax on the device for the small eigensolver
  std::vector<int> dims_h(kmax + 1);
  for (int x = 0; x <= kmax; ++x) dims_h[x] = x;
  int64_t offs_h[2] = {0, 0};
  DevBuf d_dims, d_offs(c, sizeof(int64_t) * 2);
  upload(c, d_dims, dims_h);
  B2_CUDA(cudaMemcpyAsync(d_offs.ptr, offs_h, sizeof(offs_h), cudaMemcpyHostToDevice, c->stream));
  std::vector<double> theta(k), r2(k);
  for (;;) {
    b2k::launch_symmetrize(m, VW, kmax, G, c->stream);
    b2k::launch_jacobi(1, d_dims.as<int>() + m, d_offs.as<int64_t>(), d_offs.as<int64_t>(), G,
                       evals, evecs, nullptr, d_offs.as<int64_t>(), m, c->stream);
    for (int j = 0; j < k; ++j)   // root j: eigenvalue m-1-j of the descending list
      b2k::launch_ritz(m, Vp, Wp, n, evecs + (m - 1 - j), m, evals + (m - 1 - j), diag.as<double>(),
                       U.as<double>() + int64_t(j) * n, HU.as<double>() + int64_t(j) * n,
                       T.as<double>() + int64_t(j) * n, n, part, r2d + j, c->stream);
    B2_CUDA(cudaMemcpyAsync(r2.data(), r2d, sizeof(double) * k, cudaMemcpyDeviceToHost, c->stream));
    for (int j = 0; j < k; ++j)
      B2_CUDA(cudaMemcpyAsync(&theta[j], evals + (m - 1 - j), sizeof(double), cudaMemcpyDeviceToHost,
                              c->stream));
    sync(c);
    for (int j = 0; j < k; ++j)
      B2_REQUIRE(std::isfinite(r2[j]) && std::isfinite(theta[j]), B2_ENOCONV,
                 "Davidson produced a non-finite value");
    std::vector<int> todo;
    for (int j = 0; j < k; ++j)
      if (r2[j] > tol) todo.push_back(j);
    if (std::getenv("B2_TRACE_DAVIDSON")) {
      std::fprintf(stderr, "roots win %d m %d nmv %d", win, m, nmv);
      for (int j = 0; j < k; ++j) std::fprintf(stderr, " (%.12f %.2e)", theta[j], r2[j]);
      std::fprintf(stderr, "\n");
    }
    if (todo.empty() || nmv >= max_iter) break;
    if (m + int(todo.size()) > kmax) {   // restart from the Ritz vectors
      for (int j = 0; j < k; ++j) {
        double* uj = U.as<double>() + int64_t(j) * n;
        b2k::launch_multidot(1, uj, n, uj, n, part, nrm, 1, c->stream);
        B2_CUDA(cudaMemcpyAsync(Vp + int64_t(j) * n, uj, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        B2_CUDA(cudaMemcpyAsync(Wp + int64_t(j) * n, HU.as<double>() + int64_t(j) * n,
                                sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
        b2k::launch_scale_inv_sqrt(Vp + int64_t(j) * n, n, nrm, c->stream);
        b2k::launch_scale_inv_sqrt(Wp + int64_t(j) * n, n, nrm, c->stream);
      }
      m = k;
      for (int j = 0; j < k; ++j)
        b2k::launch_multidot(k, Vp, n, Wp + int64_t(j) * n, n, part, VW + j, kmax, c->stream);
    }
    int added = 0;
    for (int j : todo) {
      if (!orthonormal_add(T.as<double>() + int64_t(j) * n, 1e-28)) continue;
      add_product();
      ++added;
    }
    if (added == 0) break;
  }
  double mx = 0;
  for (int j = 0; j < k; ++j) {
    double* uj = U.as<double>() + int64_t(j) * n;
    b2k::launch_multidot(1, uj, n, uj, n, part, nrm, 1, c->stream);
    B2_CUDA(cudaMemcpyAsync(psis + int64_t(j) * n, uj, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    b2k::launch_scale_inv_sqrt(psis + int64_t(j) * n, n, nrm, c->stream);
    mx = std::max(mx, r2[j]);
  }
  sync(c);
  if (n_matvec) *n_matvec = nmv;
  if (max_resid2) *max_resid2 = mx;
  if (flops_out) *flops_out = flops;
  return theta;
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

// ------------------------------------------------------------- perturbative noise
// The MPO factorises exactly across the bond being split, H = sum_w S_w (x) E_w (channels w
// of that bond; S_w = sum_a (-1)^{p(a) N(l)} L_a (x) W[a, w] diag((-1)^{p(w) n(s)}) on the
// left part, E_w = sum_b W[w, b] diag((-1)^{p(b) n(s)}) (x) R_b on the right part).  The
// perturbative noise (White 2005) adds to the kept part's density matrix the weight that the
// kept part's operators move psi into: N = sum_w P_w P_w^T, P_w = S_w psi (forward split) or
// E_w psi (backward split), normalised so that it adds total weight `noise`:
// rho' = rho + noise * N / tr N.  Sign factors on the other part's indices cancel in N and
// are left out.  Rows of sectors the new bond cannot hold get no noise.  The products P_w
// are blocks of their own (one per (w, row block, column block)); tr N = |P|^2.
struct NoiseBlock {
  int w, row, col;      // channel, row part index, column part index (meaning per direction)
  int64_t off;
  int m_row, m_col;
};

static double norm2_device(Ctx* c, const double* x, int64_t n) {
  if (n <= 0) return 0.0;
  DevBuf sc(c, sizeof(double) * (256 * 16 + 1));
  double* part = sc.as<double>();
  b2k::launch_multidot(1, x, n, x, n, part, part + 256 * 16, 1, c->stream);
  double v = 0;
  B2_CUDA(cudaMemcpyAsync(&v, part + 256 * 16, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  sync(c);
  return v;
}

// Forward split of window win (site i): psi -> A_i (left-orthonormal, new bond i+1) and the
// guess for the next window of the same width.  Updates mps->bonds[i+1], mps->sites[i],
// L_{i+1}; writes the new psi.  Rows of the density matrix are (jl, s1) in both widths; a
// one-site psi has only s2 = 0, so its columns are the right bond alone.
void split_left(b2_env_s* env, int win, DevBuf& psi, int M, double cutoff, double* discarded,
                double* flops, double noise, int nroot, bool keep_centre) {
  Ctx* c = env->ctx;
  const int i = win_site(win), ns = win_nsite(win);
  Tracer tr(c, "split_left", i);
  b2_mps_s* mps = env->mps;
  WindowProgram& wp = window_program(env, win);
  const PsiLayout lay = wp.psi;
  const int64_t n = lay.size;               // psi holds nroot states of this layout
  const double wr = 1.0 / nroot;            // state-average weight
  const Bond bl = mps->bonds[i];
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
  std::vector<std::vector<int>> out_of(secs.size());
  std::vector<std::pair<int, int>> part_of(size_t(bl.size()) * 4, {-1, -1});   // (sector, part)
  for (size_t j = 0; j < secs.size(); ++j)
    for (size_t a = 0; a < secs[j].parts.size(); ++a)
      part_of[size_t(secs[j].parts[a].first) * 4 + secs[j].parts[a].second] = {int(j), int(a)};
  for (size_t j = 0; j < secs.size(); ++j)
    for (size_t a = 0; a < secs[j].parts.size(); ++a)
      for (size_t b = 0; b < secs[j].parts.size(); ++b) {
        const RhoSector& r = secs[j];
        int ja = r.parts[a].first, sa = r.parts[a].second;
        int jb = r.parts[b].first, sb = r.parts[b].second;
        int o = prog.add_out(1, r.off + int64_t(r.part_off[a]) * r.dim + r.part_off[b], bl.m[ja],
                             bl.m[jb], r.dim, false);
        out_of[j].push_back(o);
        for (int s2 = 0; s2 < 4; ++s2) {
          int pa = lay.find(ja, sa, s2), pb = lay.find(jb, sb, s2);
          if (pa < 0 || pb < 0) continue;
          const PsiBlock& A = lay.blocks[pa];
          const PsiBlock& B = lay.blocks[pb];
          for (int rt = 0; rt < nroot; ++rt) {
            GemmTerm t{};
            t.offP = A.off + rt * n; t.bufP = 0; t.ldP = A.mr;
            t.offX = B.off + rt * n; t.bufX = 0; t.ldX = B.mr;     // op(X) = B^T
            t.K1 = A.mr;
            t.flags = kTwoOp | kTransQ;
            t.alpha = wr;
            prog.add_term(o, t);
          }
        }
      }
  // noise: P_w(jl', s1'; s2, jr) = sum_{a, s1} c (-1)^{p(a) N(jl)} L_a(jl' <- jl) psi(jl, s1, s2, jr)
  DevBuf pbuf;
  if (noise > 0) {
    const EnvBond& L = env->L[i];
    b2_mpo_s* mpo = env->mpo;
    std::vector<NoiseBlock> nb_;
    std::vector<std::pair<int, GemmTerm>> pterms;   // (block, term) of one state
    std::unordered_map<int64_t, int> nidx;
    const int64_t ncol = int64_t(4) * mps->bonds[i + ns].size();
    GemmProgram pp;
    int64_t psize = 0;                              // per state
    for (const auto& e : mpo->W[i]) {
      const int a = e.w, w = e.w2;
      const bool pw = mpo->parity[i + 1][w] != 0, pa = mpo->parity[i][a] != 0;
      for (int u = 0; u < 16; ++u) {
        if (e.m[u] == 0) continue;
        const int s1p = u / 4, s1 = u % 4;
        const double sg = (pw && (kSiteN[s1] & 1)) ? -1.0 : 1.0;
        for (int jl = 0; jl < bl.size(); ++jl) {
          const int lb = L.find(a, jl);
          if (lb < 0) continue;
          const int jlp = L.blocks[lb].jb;
          const int row = jlp * 4 + s1p;
          if (part_of[row].first < 0) continue;
          for (int s2 = 0; s2 < 4; ++s2) {
            const int ib = lay.find(jl, s1, s2);
            if (ib < 0) continue;
            const PsiBlock& P = lay.blocks[ib];
            const int col = P.jr * 4 + s2;
            const int64_t key = (int64_t(w) * bl.size() * 4 + row) * ncol + col;
            auto it = nidx.find(key);
            int o;
            if (it == nidx.end()) {
              o = int(nb_.size());
              nidx.emplace(key, o);
              nb_.push_back({w, row, col, psize, bl.m[jlp], P.mr});
              psize += int64_t(bl.m[jlp]) * P.mr;
            } else {
              o = it->second;
            }
            GemmTerm t{};
            t.offP = L.blocks[lb].off; t.bufP = 2; t.ldP = P.ml;   // L_a [m_jl' x m_jl]
            t.offX = P.off; t.bufX = 0; t.ldX = P.mr;               // psi [m_jl x m_jr]
            t.K1 = P.ml;
            t.flags = kTwoOp;
            t.alpha = e.m[u] * sg * ((pa && (bl.q[jl].n & 1)) ? -1.0 : 1.0);
            pterms.push_back({o, t});
          }
        }
      }
    }
    if (psize > 0) {
      // the states' products side by side, each scaled by sqrt(w): N = sum_j w_j N_j
      const double sw = std::sqrt(wr);
      for (int rt = 0; rt < nroot; ++rt)
        for (const auto& b : nb_) pp.add_out(1, rt * psize + b.off, b.m_row, b.m_col, b.m_col, false);
      for (int rt = 0; rt < nroot; ++rt)
        for (auto bt : pterms) {
          bt.second.offX += rt * n;
          bt.second.alpha *= sw;
          pp.add_term(rt * int(nb_.size()) + bt.first, bt.second);
        }
      pp.finalize(c);
      pbuf.reset(c, sizeof(double) * size_t(psize) * nroot);
      BufTable pt{};
      pt.p[0] = psi.as<double>();
      pt.p[1] = pbuf.as<double>();
      pt.p[2] = L.data.as<double>();
      pp.launch(c, pt);
      *flops += pp.flops;
      const double trN = norm2_device(c, pbuf.as<double>(), psize * nroot);
      if (trN > 0) {
        // Gram terms per environment column: rho[(row x), (row y)] += scale P_x P_y^T
        std::map<int64_t, std::vector<int>> by_col;   // key: w * ncol + col
        for (size_t x = 0; x < nb_.size(); ++x) by_col[nb_[x].w * ncol + nb_[x].col].push_back(int(x));
        for (auto& kv : by_col)
          for (int x : kv.second)
            for (int y : kv.second) {
              const auto px = part_of[nb_[x].row], py = part_of[nb_[y].row];
              if (px.first != py.first) continue;
              const int np_ = int(secs[px.first].parts.size());
              for (int rt = 0; rt < nroot; ++rt) {
                GemmTerm t{};
                t.offP = rt * psize + nb_[x].off; t.bufP = 2; t.ldP = nb_[x].m_col;
                t.offX = rt * psize + nb_[y].off; t.bufX = 2; t.ldX = nb_[y].m_col;   // P_y^T
                t.K1 = nb_[x].m_col;
                t.flags = kTwoOp | kTransQ;
                t.alpha = noise / trN;
                prog.add_term(out_of[px.first][size_t(px.second) * np_ + py.second], t);
              }
            }
      }
    }
  }
  prog.finalize(c);
  BufTable bt{};
  bt.p[0] = psi.as<double>();
  bt.p[1] = rho.as<double>();
  bt.p[2] = pbuf.as<double>();
  prog.launch(c, bt);
  *flops += prog.flops;
  tr.mark("rho");
  std::vector<int> kept = eig_and_select(c, secs, rho, evals, evecs, M, cutoff, discarded,
                                         &env->rho_cache[4 * i + 2 * (ns == 1)]);
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

  // C(jt, s2 -> jr) = sum_{(jl,s1) in jt} A(jl,s1,jt)^T psi(jl,s1,s2)  (one-site: s2 = 0,
  // C is the matrix from the new bond i+1 to the old one; its blocks s2 > 0 stay unused)
  const Bond br = mps->bonds[i + ns];
  SiteTensor C;
  C.build(nb, br);
  C.data.reset(c, sizeof(double) * std::max<int64_t>(C.size * nroot, 1));   // one C per state
  GemmProgram pc;
  for (int rt = 0; rt < nroot; ++rt)
  for (const auto& cbk : C.blocks) {
    int o = pc.add_out(1, rt * C.size + cbk.off, cbk.ml, cbk.mr, cbk.mr, false);
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
      t.offX = P.off + rt * n; t.bufX = 0; t.ldX = P.mr;
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

  // commit: site i, bond i+1; environments on bond i+1 change.  br_mid: the bond between
  // C and the next site tensor (bond i+2 for two sites, the old bond i+1 for one)
  const Bond br_mid = ns == 2 ? mps->bonds[i + 2] : br;
  mps->bonds[i + 1] = nb;
  mps->sites[i] = std::move(A);
  env->R[i + 1].valid = false;
  tr.mark("site+C");
  env_update_left(env, i);
  tr.mark("env");
  // keep_centre (two sites): psi := C, the one-site psi of site i+1 on bonds (i+1, i+2)
  // (a site tensor's layout is the one-site layout)
  if (keep_centre) {
    B2_REQUIRE(ns == 2 && nroot == 1, B2_EINVAL, "internal: keep_centre");
    psi = std::move(C.data);
    return;
  }
  // guess for the next window: C . B_{i+ns}.  One-site: C(jt, 0 -> jr) B_{i+1}(jr, s -> jr')
  // lands in the layout with the trivial site first, i.e. at the one-site offsets.
  if (i + ns < mps->n) {
    PsiLayout nl;
    nl.build(mps->bonds[i + 1], mps->bonds[i + 1 + ns], ns, ns == 1);
    DevBuf np(c, sizeof(double) * std::max<int64_t>(nl.size * nroot, 1));
    for (int rt = 0; rt < nroot; ++rt)
      contract_two_sites(c, mps->bonds[i + 1], br_mid, C, C.data.as<double>() + rt * C.size,
                         mps->sites[i + ns], mps->sites[i + ns].data.as<double>(), nl,
                         np.as<double>() + rt * nl.size, flops);
    psi = std::move(np);
  }
}

// Backward split of window win (site i): psi -> B_k (right-orthonormal, new bond k) with
// k = i+1 for two sites and k = i for one, and the guess for the previous window of the same
// width.  Updates mps->bonds[k], mps->sites[k], R_k; writes the new psi.  Two sites: rows
// (jl, s1), columns (s2, jr).  One site: psi read with the trivial site first, (jl, 0, s, jr),
// so the same code takes rows (jl) and columns (s, jr).  With a two-site window 0 and
// guess == false it only re-canonicalises (site 0 := C).
void split_right(b2_env_s* env, int win, DevBuf& psi, int M, double cutoff, double* discarded,
                 double* flops, bool make_guess, double noise, int nroot, bool keep_centre) {
  Ctx* c = env->ctx;
  const int i = win_site(win), ns = win_nsite(win);
  const int k = i + ns - 1;
  Tracer tr(c, "split_right", i);
  b2_mps_s* mps = env->mps;
  B2_REQUIRE(ns == 2 || (make_guess && i > 0), B2_EINVAL, "internal: one-site split at site 0");
  WindowProgram& wp = window_program(env, win);
  PsiLayout lay = wp.psi;
  const Bond bl = mps->bonds[i];
  const Bond br = mps->bonds[i + ns];
  if (ns == 1) lay.build(bl, br, 1, true);
  const int64_t n = lay.size;               // psi holds nroot states of this layout
  const double wr = 1.0 / nroot;            // state-average weight
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
  std::vector<std::vector<int>> out_of(secs.size());
  std::vector<std::pair<int, int>> part_of(size_t(br.size()) * 4, {-1, -1});   // (sector, part)
  for (size_t j = 0; j < secs.size(); ++j)
    for (size_t a = 0; a < secs[j].parts.size(); ++a)
      part_of[size_t(secs[j].parts[a].first) * 4 + secs[j].parts[a].second] = {int(j), int(a)};
  for (size_t j = 0; j < secs.size(); ++j)
    for (size_t a = 0; a < secs[j].parts.size(); ++a)
      for (size_t b = 0; b < secs[j].parts.size(); ++b) {
        const RhoSector& r = secs[j];
        int jra = r.parts[a].first, sa = r.parts[a].second;
        int jrb = r.parts[b].first, sb = r.parts[b].second;
        int o = prog.add_out(1, r.off + int64_t(r.part_off[a]) * r.dim + r.part_off[b], br.m[jra],
                             br.m[jrb], r.dim, false);
        out_of[j].push_back(o);
        for (int jl = 0; jl < bl.size(); ++jl)
          for (int s1 = 0; s1 < 4; ++s1) {
            if (!(bl.q[jl] + kSiteQ[s1] == r.q)) continue;
            int pa = lay.find(jl, s1, sa), pb = lay.find(jl, s1, sb);
            if (pa < 0 || pb < 0) continue;
            const PsiBlock& A = lay.blocks[pa];
            const PsiBlock& B = lay.blocks[pb];
            if (A.jr != jra || B.jr != jrb) continue;
            for (int rt = 0; rt < nroot; ++rt) {
              GemmTerm t{};
              t.offP = A.off + rt * n; t.bufP = 0; t.ldP = A.mr;    // op(P) = A^T [m_jra x m_jl]
              t.offX = B.off + rt * n; t.bufX = 0; t.ldX = B.mr;    // X [m_jl x m_jrb]
              t.K1 = A.ml;
              t.flags = kTwoOp | kTransP;
              t.alpha = wr;
              prog.add_term(o, t);
            }
          }
      }
  // noise: P_w(jl, s1; s2', jr') = sum_{b, s2} c (-1)^{p(b) n(s2)} psi(jl, s1, s2, jr) R_b(jr' <- jr)^T
  // with W of the kept site k (channels w on bond k, b on bond i+ns)
  DevBuf pbuf;
  if (noise > 0) {
    const EnvBond& R = env->R[i + ns];
    b2_mpo_s* mpo = env->mpo;
    std::vector<NoiseBlock> nb_;
    std::vector<std::pair<int, GemmTerm>> pterms;   // (block, term) of one state
    std::unordered_map<int64_t, int> nidx;
    const int64_t ncol = int64_t(4) * br.size();
    GemmProgram pp;
    int64_t psize = 0;                              // per state
    for (const auto& e : mpo->W[k]) {
      const int w = e.w, b = e.w2;
      const bool pb = mpo->parity[i + ns][b] != 0;
      for (int u = 0; u < 16; ++u) {
        if (e.m[u] == 0) continue;
        const int s2p = u / 4, s2 = u % 4;
        const double sg = (pb && (kSiteN[s2] & 1)) ? -1.0 : 1.0;
        for (const auto& P : lay.blocks) {
          if (P.s2 != s2) continue;
          const int rb = R.find(b, P.jr);
          if (rb < 0) continue;
          const int jrp = R.blocks[rb].jb;
          const int col = jrp * 4 + s2p;
          if (part_of[col].first < 0) continue;
          const int row = P.jl * 4 + P.s1;
          const int64_t key = (int64_t(w) * bl.size() * 4 + row) * ncol + col;
          auto it = nidx.find(key);
          int o;
          if (it == nidx.end()) {
            o = int(nb_.size());
            nidx.emplace(key, o);
            nb_.push_back({w, row, col, psize, P.ml, br.m[jrp]});
            psize += int64_t(P.ml) * br.m[jrp];
          } else {
            o = it->second;
          }
          GemmTerm t{};
          t.offP = P.off; t.bufP = 0; t.ldP = P.mr;                      // psi [m_jl x m_jr]
          t.offX = R.blocks[rb].off; t.bufX = 3; t.ldX = P.mr;           // R_b [m_jr' x m_jr]
          t.K1 = P.mr;
          t.flags = kTwoOp | kTransQ;
          t.alpha = e.m[u] * sg;
          pterms.push_back({o, t});
        }
      }
    }
    if (psize > 0) {
      const double sw = std::sqrt(wr);
      for (int rt = 0; rt < nroot; ++rt)
        for (const auto& b : nb_) pp.add_out(1, rt * psize + b.off, b.m_row, b.m_col, b.m_col, false);
      for (int rt = 0; rt < nroot; ++rt)
        for (auto bt : pterms) {
          bt.second.offP += rt * n;
          bt.second.alpha *= sw;
          pp.add_term(rt * int(nb_.size()) + bt.first, bt.second);
        }
      pp.finalize(c);
      pbuf.reset(c, sizeof(double) * size_t(psize) * nroot);
      BufTable pt{};
      pt.p[0] = psi.as<double>();
      pt.p[1] = pbuf.as<double>();
      pt.p[3] = R.data.as<double>();
      pp.launch(c, pt);
      *flops += pp.flops;
      const double trN = norm2_device(c, pbuf.as<double>(), psize * nroot);
      if (trN > 0) {
        // Gram terms per environment row: rho[(col x), (col y)] += scale P_x^T P_y
        std::map<int64_t, std::vector<int>> by_row;   // key: w * (4 |bond i|) + row
        for (size_t x = 0; x < nb_.size(); ++x)
          by_row[int64_t(nb_[x].w) * bl.size() * 4 + nb_[x].row].push_back(int(x));
        for (auto& kv : by_row)
          for (int x : kv.second)
            for (int y : kv.second) {
              const auto px = part_of[nb_[x].col], py = part_of[nb_[y].col];
              if (px.first != py.first) continue;
              const int np_ = int(secs[px.first].parts.size());
              for (int rt = 0; rt < nroot; ++rt) {
                GemmTerm t{};
                t.offP = rt * psize + nb_[x].off; t.bufP = 2; t.ldP = nb_[x].m_col;   // P_x^T
                t.offX = rt * psize + nb_[y].off; t.bufX = 2; t.ldX = nb_[y].m_col;
                t.K1 = nb_[x].m_row;
                t.flags = kTwoOp | kTransP;
                t.alpha = noise / trN;
                prog.add_term(out_of[px.first][size_t(px.second) * np_ + py.second], t);
              }
            }
      }
    }
  }
  prog.finalize(c);
  BufTable bt{};
  bt.p[0] = psi.as<double>();
  bt.p[1] = rho.as<double>();
  bt.p[2] = pbuf.as<double>();
  prog.launch(c, bt);
  *flops += prog.flops;
  tr.mark("rho");
  std::vector<int> kept = eig_and_select(c, secs, rho, evals, evecs, M, cutoff, discarded,
                                         &env->rho_cache[4 * i + 2 * (ns == 1) + 1]);
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
  C.data.reset(c, sizeof(double) * std::max<int64_t>(C.size * nroot, 1));   // one C per state
  GemmProgram pc;
  for (int rt = 0; rt < nroot; ++rt)
  for (const auto& cbk : C.blocks) {
    int o = pc.add_out(1, rt * C.size + cbk.off, cbk.ml, cbk.mr, cbk.mr, false);
    for (int s2 = 0; s2 < 4; ++s2) {
      int pb = lay.find(cbk.jl, cbk.s, s2);
      if (pb < 0) continue;
      const PsiBlock& P = lay.blocks[pb];
      int bb = Bt.find(cbk.jr, s2);
      if (bb < 0 || Bt.blocks[bb].jr != P.jr) continue;
      const SiteBlock& Bb = Bt.blocks[bb];
      GemmTerm t{};
      t.offP = P.off + rt * n; t.bufP = 0; t.ldP = P.mr;
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

  mps->bonds[k] = nb;
  mps->sites[k] = std::move(Bt);
  env->L[k].valid = false;
  tr.mark("site+C");
  env_update_right(env, k);
  tr.mark("env");
  if (keep_centre) {   // two sites: psi := C, the one-site psi of site i on bonds (i, i+1)
    B2_REQUIRE(ns == 2 && nroot == 1, B2_EINVAL, "internal: keep_centre");
    psi = std::move(C.data);
  } else if (make_guess && i > 0) {
    // A_{i-1} . C on bonds (i-1, i+ns-1); bl is bond i as A_{i-1} and C knew it
    PsiLayout nl;
    nl.build(mps->bonds[i - 1], mps->bonds[k], ns);
    DevBuf np(c, sizeof(double) * std::max<int64_t>(nl.size * nroot, 1));
    for (int rt = 0; rt < nroot; ++rt)
      contract_two_sites(c, mps->bonds[i - 1], bl, mps->sites[i - 1],
                         mps->sites[i - 1].data.as<double>(), C, C.data.as<double>() + rt * C.size,
                         nl, np.as<double>() + rt * nl.size, flops);
    psi = std::move(np);
  } else {
    // centre stays on site i: it holds C
    mps->sites[i] = std::move(C);
    mps->center = i;
  }
}

// ------------------------------------------------------------------- TDVP
// psi <- exp(-t H_eff) psi / |exp(-t H_eff) psi| for window win by the Krylov (Lanczos)
// method: orthonormal basis V of span{psi, H psi, ...} (each new vector orthogonalised twice
// against all previous ones), T = V^T H V (FP64 products; T from the same V.W dot products as
// Davidson's Rayleigh-Ritz), its eigen-decomposition by the Jacobi kernel, and
// c = exp(-t (T - lambda_min)) e_1 (k_krylov_coef).  Stops when the next vector's weight
// beta_k |c_k| is <= tol |c|, when the space is exhausted (beta <= 1e-14 max(1, |lambda|))
// or at max_k vectors; psi = V c normalised (imaginary time does not keep the norm and only
// the direction is used).  One host synchronisation per Krylov vector.
static void krylov_exp(b2_env_s* env, int win, double* psi, double t, double tol, int max_k,
                       double* flops, int* n_matvec) {
  Ctx* c = env->ctx;
  WindowProgram& wp = window_program(env, win);
  const int64_t n = wp.psi.size;
  B2_REQUIRE(n > 0, B2_EINVAL, "empty wavefunction");
  const int kmax = std::max(2, std::min(max_k > 0 ? max_k : 40, 64));
  DevBuf V(c, sizeof(double) * n * kmax), W(c, sizeof(double) * n * kmax);
  const int kPart = 256 * 16;
  DevBuf small(c, sizeof(double) * (kPart + 4 * kmax * kmax + 4 * kmax + 16));
  double* part = small.as<double>();
  double* VW = part + kPart;
  double* G = VW + kmax * kmax;
  double* evecs = G + kmax * kmax;
  double* evals = evecs + kmax * kmax;
  double* cvec = evals + kmax;
  double* stats = cvec + 2 * kmax;   // |c|^2, lambda_min, max |lambda|, beta^2, c_last
  double* Vp = V.as<double>();
  double* Wp = W.as<double>();
  std::vector<int> dims_h(kmax + 1);
  for (int x = 0; x <= kmax; ++x) dims_h[x] = x;
  int64_t offs_h[2] = {0, 0};
  DevBuf d_dims, d_offs(c, sizeof(int64_t) * 2);
  upload(c, d_dims, dims_h);
  B2_CUDA(cudaMemcpyAsync(d_offs.ptr, offs_h, sizeof(offs_h), cudaMemcpyHostToDevice, c->stream));
  b2k::launch_multidot(1, psi, n, psi, n, part, stats + 3, 1, c->stream);
  B2_CUDA(cudaMemcpyAsync(Vp, psi, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
  b2k::launch_scale_inv_sqrt(Vp, n, stats + 3, c->stream);
  int m = 0;
  double fl = 0;
  for (;;) {
    double* vm = Vp + int64_t(m) * n;
    double* wm = Wp + int64_t(m) * n;
    heff_apply(env, win, vm, wm, 0.0, &fl, B2_FP64);
    if (flops) *flops += fl;
    if (n_matvec) ++*n_matvec;
    b2k::launch_multidot(m + 1, Vp, n, wm, n, part, VW + m, kmax, c->stream);
    if (m > 0) b2k::launch_multidot(m, Wp, n, vm, n, part, VW + int64_t(m) * kmax, 1, c->stream);
    ++m;
    b2k::launch_symmetrize(m, VW, kmax, G, c->stream);
    b2k::launch_jacobi(1, d_dims.as<int>() + m, d_offs.as<int64_t>(), d_offs.as<int64_t>(), G,
                       evals, evecs, nullptr, d_offs.as<int64_t>(), m, c->stream);
    b2k::launch_krylov_coef(m, evecs, evals, t, cvec, stats, c->stream);
    if (m >= kmax) break;
    // next direction: H v_{m-1} orthogonalised twice against V
    double* vn = Vp + int64_t(m) * n;
    B2_CUDA(cudaMemcpyAsync(vn, wm, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    for (int pass = 0; pass < 2; ++pass) {
      b2k::launch_multidot(m, Vp, n, vn, n, part, cvec + kmax, 1, c->stream);
      b2k::launch_multiaxpy(m, Vp, n, cvec + kmax, vn, n, -1.0, c->stream);
    }
    b2k::launch_multidot(1, vn, n, vn, n, part, stats + 3, 1, c->stream);
    double h[4];
    B2_CUDA(cudaMemcpyAsync(h, stats, sizeof(double) * 4, cudaMemcpyDeviceToHost, c->stream));
    double clast = 0;
    B2_CUDA(cudaMemcpyAsync(&clast, cvec + (m - 1), sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    sync(c);
    B2_REQUIRE(std::isfinite(h[0]) && std::isfinite(h[3]), B2_ENOCONV, "Krylov exponential: non-finite value");
    const double beta = std::sqrt(std::max(h[3], 0.0));
    if (beta * std::fabs(clast) <= tol * std::sqrt(h[0]) || beta <= 1e-14 * std::max(1.0, h[2]))
      break;
    b2k::launch_scale_inv_sqrt(vn, n, stats + 3, c->stream);
  }
  B2_CUDA(cudaMemsetAsync(psi, 0, sizeof(double) * n, c->stream));
  b2k::launch_multiaxpy(m, Vp, n, cvec, psi, n, 1.0, c->stream);
  b2k::launch_multidot(1, psi, n, psi, n, part, stats + 3, 1, c->stream);
  b2k::launch_scale_inv_sqrt(psi, n, stats + 3, c->stream);
  B2_CUDA(cudaGetLastError());
}

// Imaginary-time two-site TDVP (projector splitting, second order; Sec. 2.7.3): per step a
// forward half over windows 0..n-2 and a backward half n-2..0, each evolving the two-site psi
// by exp(-tau/2 H2), splitting it (truncated like a sweep split) and evolving the one-site
// remainder backwards by exp(+tau/2 H1) on the one-site window before contracting it with the
// next site tensor.  Starts from and returns to an MPS centred at site 0.
void tdvp(b2_env_s* env, const b2_tdvp_opts& o, b2_tdvp_result* res) {
  Ctx* c = env->ctx;
  b2_mps_s* mps = env->mps;
  const int n = mps->n;
  B2_REQUIRE(n >= 3, B2_EINVAL, "TDVP needs at least three sites");
  B2_REQUIRE(mps->center == 0, B2_EINVAL, "TDVP needs an MPS centred at site 0");
  B2_REQUIRE(env->L[0].valid, B2_EINVAL, "env not initialised at centre 0");
  for (int k = 2; k <= n; ++k) B2_REQUIRE(env->R[k].valid, B2_EINVAL, "env not initialised at centre 0");
  B2_REQUIRE(o.bond_dim >= 1 && std::isfinite(o.tau) && o.tau > 0, B2_EINVAL, "bad TDVP options");
  const double cutoff = o.trunc_cutoff >= 0 ? o.trunc_cutoff : 1e-14;
  const double ktol = o.krylov_tol > 0 ? o.krylov_tol : 1e-12;
  const int kmax = o.krylov_max > 0 ? o.krylov_max : 40;
  const double h = 0.5 * o.tau;
  auto two_site_from = [&](int i, const SiteTensor& X, const double* xd, const SiteTensor& Y,
                           const double* yd, double* fl) {
    WindowProgram& wp = window_program(env, i);
    DevBuf np(c, sizeof(double) * std::max<int64_t>(wp.psi.size, 1));
    contract_two_sites(c, mps->bonds[i], mps->bonds[i + 1], X, xd, Y, yd, wp.psi, np.as<double>(), fl);
    return np;
  };
  double fl0 = 0;
  DevBuf psi = two_site_from(0, mps->sites[0], mps->sites[0].data.as<double>(), mps->sites[1],
                             mps->sites[1].data.as<double>(), &fl0);
  for (int step = 0; step < o.n_steps; ++step) {
    B2_CUDA(cudaStreamSynchronize(c->stream));
    auto t0 = std::chrono::steady_clock::now();
    b2_tdvp_result r{};
    double dw = 0, other = 0;
    for (int i = 0; i <= n - 2; ++i) {
      krylov_exp(env, i, psi.as<double>(), h, ktol, kmax, &r.matvec_flops, &r.n_matvec);
      if (i < n - 2) {
        split_left(env, i, psi, o.bond_dim, cutoff, &dw, &other, 0.0, 1, true);
        r.discarded_weight = std::max(r.discarded_weight, dw);
        krylov_exp(env, (i + 1) | kOneSite, psi.as<double>(), -h, ktol, kmax, &r.matvec_flops,
                   &r.n_matvec);
        SiteTensor X;   // layout of the one-site psi of site i+1
        X.build(mps->bonds[i + 1], mps->bonds[i + 2]);
        psi = two_site_from(i + 1, X, psi.as<double>(), mps->sites[i + 2],
                            mps->sites[i + 2].data.as<double>(), &other);
      }
    }
    for (int i = n - 2; i >= 0; --i) {
      krylov_exp(env, i, psi.as<double>(), h, ktol, kmax, &r.matvec_flops, &r.n_matvec);
      if (i > 0) {
        split_right(env, i, psi, o.bond_dim, cutoff, &dw, &other, false, 0.0, 1, true);
        r.discarded_weight = std::max(r.discarded_weight, dw);
        krylov_exp(env, i | kOneSite, psi.as<double>(), -h, ktol, kmax, &r.matvec_flops,
                   &r.n_matvec);
        SiteTensor Y;   // layout of the one-site psi of site i
        Y.build(mps->bonds[i], mps->bonds[i + 1]);
        psi = two_site_from(i - 1, mps->sites[i - 1], mps->sites[i - 1].data.as<double>(), Y,
                            psi.as<double>(), &other);
      }
    }
    // energy of the (normalised) window-0 psi
    {
      WindowProgram& wp = window_program(env, 0);
      const int64_t nn = wp.psi.size;
      DevBuf hp(c, sizeof(double) * std::max<int64_t>(nn, 1)), sc(c, sizeof(double) * (256 * 16 + 1));
      double fl = 0;
      heff_apply(env, 0, psi.as<double>(), hp.as<double>(), 0.0, &fl, B2_FP64);
      b2k::launch_multidot(1, psi.as<double>(), nn, hp.as<double>(), nn, sc.as<double>(),
                           sc.as<double>() + 256 * 16, 1, c->stream);
      B2_CUDA(cudaMemcpyAsync(&r.energy, sc.as<double>() + 256 * 16, sizeof(double),
                              cudaMemcpyDeviceToHost, c->stream));
      sync(c);
    }
    r.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (auto& b : mps->bonds) r.max_bond = std::max(r.max_bond, b.total);
    if (res) res[step] = r;
  }
  double dw = 0, fl = 0;
  split_right(env, 0, psi, 1 << 30, cutoff, &dw, &fl, false);
  sync(c);
}

// ------------------------------------------------------------------------ sweep
// Between sweeps the centre is at site 0: the two-site psi of window 0 (width 2; R_2 and
// L_0 exist) or the one-site psi of site 0 (width 1; R_1 exists), which has the layout of
// site tensor 0 on bonds (0, 1).  Changing the width at the start of a sweep (Sec. 2.1.2:
// mixing the one-site and two-site algorithms): 2 -> 1 splits the window-0 psi backward with
// the entering sweep's M and cutoff (B_1, R_1, centre C); 1 -> 2 contracts psi with B_1.
void sweep(b2_env_s* env, const b2_sweep_opts& o, b2_sweep_result* res) {
  Ctx* c = env->ctx;
  b2_mps_s* mps = env->mps;
  const int n = mps->n;
  B2_REQUIRE(mps->center == 0, B2_EINVAL, "sweep needs an MPS centred at site 0");
  B2_REQUIRE(env->L[0].valid, B2_EINVAL, "env not initialised at centre 0");
  for (int k = 2; k <= n; ++k) B2_REQUIRE(env->R[k].valid, B2_EINVAL, "env not initialised at centre 0");
  if (o.dots)
    for (int sw = 0; sw < o.n_sweeps; ++sw)
      B2_REQUIRE(o.dots[sw] == 1 || o.dots[sw] == 2, B2_EINVAL, "dots entries must be 1 or 2");
  if (o.noise)
    for (int sw = 0; sw < o.n_sweeps; ++sw)
      B2_REQUIRE(o.noise[sw] >= 0 && std::isfinite(o.noise[sw]), B2_EINVAL, "noise must be >= 0");
  const int nr = o.n_roots > 1 ? o.n_roots : 1;   // state-averaged roots
  B2_REQUIRE(nr <= B2_MAX_ROOTS, B2_EINVAL, "n_roots above B2_MAX_ROOTS");
  if (nr > 1) {
    B2_REQUIRE(o.prec == B2_FP64, B2_EUNSUPPORTED, "state averaging runs FP64 products only");
    if (o.dots)
      for (int sw = 0; sw < o.n_sweeps; ++sw)
        B2_REQUIRE(o.dots[sw] == 2, B2_EUNSUPPORTED, "state averaging runs two-site sweeps only");
  }
  b2_dav_opts dop;
  dop.max_iter = o.dav_max_iter > 0 ? o.dav_max_iter : 30;
  dop.max_subspace = o.max_subspace > 0 ? o.max_subspace : 30;
  dop.conv_tol = o.conv_tol > 0 ? o.conv_tol : 1e-10;
  dop.prec = o.prec;
  dop.refine_max = 0;
  const double cutoff = o.trunc_cutoff >= 0 ? o.trunc_cutoff : 1e-14;
  DevBuf psi;
  int width = 0;   // width of the centre psi (0: none formed yet, the MPS holds it)
  auto enter = [&](int ns, int M) {
    if (ns == width) return;
    double dw = 0, fl = 0;
    if (ns == 2) {
      WindowProgram& wp = window_program(env, 0);
      DevBuf np(c, sizeof(double) * std::max<int64_t>(wp.psi.size * nr, 1));
      if (nr > 1)   // further states start from zero (completed by the Davidson rule)
        B2_CUDA(cudaMemsetAsync(np.ptr, 0, np.bytes, c->stream));
      SiteTensor X;   // layout of the centre on bonds (0, 1); data: the MPS's or psi
      X.build(mps->bonds[0], mps->bonds[1]);
      const double* xd = width == 1 ? psi.as<double>() : mps->sites[0].data.as<double>();
      contract_two_sites(c, mps->bonds[0], mps->bonds[1], X, xd, mps->sites[1],
                         mps->sites[1].data.as<double>(), wp.psi, np.as<double>(), &fl);
      psi = std::move(np);
    } else {
      if (width == 2) split_right(env, 0, psi, M, cutoff, &dw, &fl, false);   // site 0 := C
      if (!env->R[1].valid) env_update_right(env, 1);
      const SiteTensor& s0 = mps->sites[0];
      DevBuf np(c, sizeof(double) * std::max<int64_t>(s0.size, 1));
      if (s0.size > 0)
        B2_CUDA(cudaMemcpyAsync(np.ptr, s0.data.ptr, sizeof(double) * size_t(s0.size),
                                cudaMemcpyDeviceToDevice, c->stream));
      psi = std::move(np);
    }
    width = ns;
  };
  for (int sw = 0; sw < o.n_sweeps; ++sw) {
    B2_CUDA(cudaStreamSynchronize(c->stream));
    auto t0 = std::chrono::steady_clock::now();
    const int M = o.bond_dims[sw];
    B2_REQUIRE(M >= 1, B2_EINVAL, "bond dimension must be positive");
    const int ns = o.dots ? o.dots[sw] : 2;
    const int flag = ns == 1 ? kOneSite : 0;
    const double nz = o.noise ? o.noise[sw] : 0.0;
    enter(ns, M);
    b2_sweep_result r{};
    double dw = 0, e = 0;
    auto now = [] { return std::chrono::steady_clock::now(); };
    auto secs = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
      return std::chrono::duration<double>(b - a).count();
    };
    auto solve = [&](int i) {
      auto ta = now();
      if (nr > 1) {
        int nmv = 0;
        double r2 = 0, fl = 0;
        std::vector<double> th = davidson_roots(env, i, psi.as<double>(), nr, dop, &nmv, &r2, &fl);
        r.matvec_flops += fl;
        r.n_matvec += nmv;
        e = th[0];
        for (int j = 0; j < nr; ++j) r.root_energy[j] = th[j];
      } else {
        DavidsonResult d = davidson(env, i | flag, psi.as<double>(), dop);
        r.matvec_flops += d.flops;
        r.n_matvec += d.n_matvec;
        e = d.energy;
        r.root_energy[0] = e;
      }
      r.t_davidson += secs(ta, now());
    };
    // A window's program (precombined operators, split planes) is used only until its split:
    // the split changes one of its environments, so it is released then instead of holding
    // device memory for every window of the chain (gigabytes per window at n = 36).
    const int last = n - ns;   // last window site
    for (int i = 0; i <= last; ++i) {
      solve(i);
      if (i < last) {
        auto ta = now();
        split_left(env, i | flag, psi, M, cutoff, &dw, &r.other_flops, nz, nr);
        env->windows.erase(i | flag);
        r.t_split += secs(ta, now());
        r.discarded_weight = std::max(r.discarded_weight, dw);
      }
    }
    for (int i = last; i >= 0; --i) {
      solve(i);
      if (i > 0) {
        auto ta = now();
        split_right(env, i | flag, psi, M, cutoff, &dw, &r.other_flops, true, nz, nr);
        env->windows.erase(i | flag);
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
  // leave the MPS centred at site 0: two sites, B_1 from psi of window 0 without a bond
  // limit (states of relative weight <= cutoff, numerically zero, dropped as in every
  // split); one site, psi is site tensor 0
  if (width == 2) {
    double dw = 0, fl = 0;
    split_right(env, 0, psi, 1 << 30, cutoff, &dw, &fl, false, 0.0, nr);
  } else if (width == 1) {
    SiteTensor s0;
    s0.build(mps->bonds[0], mps->bonds[1]);
    s0.data = std::move(psi);
    mps->sites[0] = std::move(s0);
    mps->center = 0;
  }
  sync(c);
}

}  // namespace b2
