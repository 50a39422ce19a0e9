// extern "C" entry points of libb2 (declared and documented in include/b2.h).  Each one
// validates its arguments, runs the work on the context stream and maps exceptions to
// status codes; nothing here aborts the process.
#include <cmath>
#include <new>

#include "algo.hpp"

b2_mpo_s* b2_build_mpo_impl(int n, const double* h1, const double* eri, double e_core, int n_elec,
                            int two_sz, double cutoff);
double mpo_compress(b2_mpo_s* mpo, double tol, std::vector<int>* dims_out);
b2_mps_s* b2_mps_import_impl(b2::Ctx* ctx, int n, int n_elec, int two_sz, const int* n_sectors,
                             const int* sectors, const double* site_data, int center);
void b2_mps_export_impl(b2::Ctx* ctx, b2_mps_s* mps, int* n_sectors, int* sectors,
                        double* site_data);
b2_mps_s* b2_mps_random_impl(b2::Ctx* ctx, b2_mpo_s* mpo, int M, const double* occ,
                             uint64_t seed);

namespace {
thread_local std::string g_error;

void set_error(b2_ctx ctx, const std::string& m) {
  if (ctx)
    ctx->c.last_error = m;
  else
    g_error = m;
}

template <class F>
int guarded(b2_ctx ctx, F&& f) {
  try {
    if (ctx) ctx->c.last_error.clear();
    f();
    return B2_OK;
  } catch (const b2::Error& e) {
    set_error(ctx, e.what());
    return e.code;
  } catch (const std::bad_alloc&) {
    set_error(ctx, "host allocation failed");
    return B2_ENOMEM;
  } catch (const std::exception& e) {
    set_error(ctx, e.what());
    return B2_EINVAL;
  }
}

void ensure_device(b2_ctx ctx) { B2_CUDA(cudaSetDevice(ctx->c.device)); }

void check_env(b2_ctx ctx, b2_env env) {
  B2_REQUIRE(ctx && env, B2_EINVAL, "null handle");
  B2_REQUIRE(env->ctx == &ctx->c, B2_EINVAL, "env belongs to another context");
}

bool overlap(const void* a, const void* b, int64_t n) {
  auto x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
  uintptr_t bytes = uintptr_t(n) * sizeof(double);
  return x < y + bytes && y < x + bytes;
}
}  // namespace

extern "C" {

int b2_create(b2_ctx* out, int device, void* stream, b2_alloc_fn alloc, b2_free_fn free_fn,
              void* user) {
  return guarded(nullptr, [&] {
    B2_REQUIRE(out != nullptr, B2_EINVAL, "out is null");
    B2_REQUIRE((alloc == nullptr) == (free_fn == nullptr), B2_EINVAL,
               "give both allocator callbacks or neither");
    int count = 0;
    B2_CUDA(cudaGetDeviceCount(&count));
    B2_REQUIRE(device >= 0 && device < count, B2_EINVAL, "no such device");
    B2_CUDA(cudaSetDevice(device));
    auto* c = new b2_ctx_s;
    c->c.device = device;
    c->c.stream = static_cast<cudaStream_t>(stream);
    c->c.alloc = alloc;
    c->c.free_fn = free_fn;
    c->c.user = user;
    *out = c;
  });
}

void b2_destroy(b2_ctx ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->c.stream);
  ctx->c.prof_clear();
  if (ctx->c.d_status) ctx->c.raw_free(ctx->c.d_status);
  if (ctx->c.d_eig_flops) ctx->c.raw_free(ctx->c.d_eig_flops);
  ctx->c.side_destroy();
  delete ctx;
}

const char* b2_last_error(b2_ctx ctx) { return ctx ? ctx->c.last_error.c_str() : g_error.c_str(); }

int b2_build_mpo(b2_ctx ctx, int n_orb, const double* h1, const double* eri, double e_core,
                 int n_elec, int two_sz, double cutoff, b2_mpo* out) {
  return guarded(ctx, [&] {
    B2_REQUIRE(h1 && eri && out, B2_EINVAL, "null argument");   // ctx may be NULL: host work
    B2_REQUIRE(std::isfinite(cutoff) && cutoff >= 0, B2_EINVAL, "cutoff must be >= 0");
    *out = b2_build_mpo_impl(n_orb, h1, eri, e_core, n_elec, two_sz, cutoff);
  });
}

int b2_mpo_compress(b2_ctx ctx, b2_mpo mpo, double tol, double* discarded) {
  return guarded(ctx, [&] {
    B2_REQUIRE(mpo, B2_EINVAL, "null mpo");
    B2_REQUIRE(std::isfinite(tol) && tol >= 0 && tol < 1, B2_EINVAL, "tol must be in [0, 1)");
    const double d = mpo_compress(mpo, tol, nullptr);
    if (discarded) *discarded = d;
  });
}

int b2_mpo_export(b2_mpo mpo, int64_t* n_entries, int* entry_chan, double* entry_ops,
                  int* chan_info) {
  return guarded(nullptr, [&] {
    B2_REQUIRE(mpo && n_entries, B2_EINVAL, "null argument");
    int64_t e = 0, c = 0;
    for (int k = 0; k < mpo->n; ++k) {
      n_entries[k] = int64_t(mpo->W[k].size());
      for (const auto& x : mpo->W[k]) {
        if (entry_chan) {
          entry_chan[2 * e] = x.w;
          entry_chan[2 * e + 1] = x.w2;
        }
        if (entry_ops)
          for (int u = 0; u < 16; ++u) entry_ops[16 * e + u] = x.m[u];
        ++e;
      }
    }
    if (chan_info)
      for (int k = 0; k <= mpo->n; ++k)
        for (int w = 0; w < mpo->D[k]; ++w, ++c) {
          chan_info[3 * c] = mpo->parity[k][w];
          chan_info[3 * c + 1] = mpo->dq[k][w].n;
          chan_info[3 * c + 2] = mpo->dq[k][w].tsz;
        }
  });
}

int b2_mpo_info(b2_mpo mpo, int* n_orb, int* bond_dims) {
  if (!mpo) return B2_EINVAL;
  if (n_orb) *n_orb = mpo->n;
  if (bond_dims)
    for (int k = 0; k <= mpo->n; ++k) bond_dims[k] = mpo->D[k];
  return B2_OK;
}

int b2_mps_import(b2_ctx ctx, int n, int n_elec, int two_sz, const int* n_sectors,
                  const int* sectors, const double* site_data, int center, b2_mps* out) {
  return guarded(ctx, [&] {
    B2_REQUIRE(ctx && out, B2_EINVAL, "null argument");
    ensure_device(ctx);
    *out = b2_mps_import_impl(&ctx->c, n, n_elec, two_sz, n_sectors, sectors, site_data, center);
  });
}

int b2_mps_size(b2_mps mps, int64_t* n_sector_total, int64_t* n_elem_total, int* center) {
  if (!mps) return B2_EINVAL;
  int64_t ns = 0, ne = 0;
  for (auto& b : mps->bonds) ns += b.size();
  for (auto& s : mps->sites) ne += s.size;
  if (n_sector_total) *n_sector_total = ns;
  if (n_elem_total) *n_elem_total = ne;
  if (center) *center = mps->center;
  return B2_OK;
}

int b2_mps_export(b2_ctx ctx, b2_mps mps, int* n_sectors, int* sectors, double* site_data) {
  return guarded(ctx, [&] {
    B2_REQUIRE(ctx && mps && n_sectors && sectors && site_data, B2_EINVAL, "null argument");
    ensure_device(ctx);
    b2_mps_export_impl(&ctx->c, mps, n_sectors, sectors, site_data);
  });
}

int b2_mps_random(b2_ctx ctx, b2_mpo mpo, int bond_dim, const double* occ, uint64_t seed,
                  b2_mps* out) {
  return guarded(ctx, [&] {
    B2_REQUIRE(ctx && mpo && out, B2_EINVAL, "null argument");
    B2_REQUIRE(bond_dim >= 1, B2_EINVAL, "bond_dim must be positive");
    ensure_device(ctx);
    *out = b2_mps_random_impl(&ctx->c, mpo, bond_dim, occ, seed);
  });
}

int b2_env_init(b2_ctx ctx, b2_mpo mpo, b2_mps mps, int center, b2_env* out) {
  return guarded(ctx, [&] {
    B2_REQUIRE(ctx && mpo && mps && out, B2_EINVAL, "null argument");
    B2_REQUIRE(mps->ctx == &ctx->c, B2_EINVAL, "mps belongs to another context");
    B2_REQUIRE(mpo->n == mps->n && mpo->n_elec == mps->n_elec && mpo->two_sz == mps->two_sz,
               B2_EINVAL, "mpo and mps describe different systems");
    B2_REQUIRE(center >= 0 && center + 1 < mps->n, B2_EINVAL, "center out of range");
    ensure_device(ctx);
    std::unique_ptr<b2_env_s> env(new b2_env_s);
    env->ctx = &ctx->c;
    env->mpo = mpo;
    env->mps = mps;
    const int n = mps->n;
    env->L.resize(n + 1);
    env->R.resize(n + 1);
    const double one = 1.0;
    auto boundary = [&](b2::EnvBond& e, const b2::Bond& b, const std::vector<b2::QN>& dq) {
      e.layout(b, dq);
      B2_REQUIRE(e.size == 1, B2_EINVAL, "internal: boundary environment");
      e.data.reset(&ctx->c, sizeof(double));
      B2_CUDA(cudaMemcpyAsync(e.data.ptr, &one, sizeof(double), cudaMemcpyHostToDevice,
                              ctx->c.stream));
      e.valid = true;
      e.version = ++env->version_counter;
    };
    boundary(env->L[0], mps->bonds[0], mpo->dq[0]);
    boundary(env->R[n], mps->bonds[n], mpo->dq[n]);
    for (int k = 0; k < center; ++k) b2::env_update_left(env.get(), k);
    for (int k = n - 1; k >= center + 2; --k) b2::env_update_right(env.get(), k);
    B2_CUDA(cudaStreamSynchronize(ctx->c.stream));
    *out = env.release();
  });
}

int b2_env_update(b2_ctx ctx, b2_env env, int site, int dir) {
  return guarded(ctx, [&] {
    check_env(ctx, env);
    B2_REQUIRE(dir == 1 || dir == -1, B2_EINVAL, "dir must be +1 or -1");
    ensure_device(ctx);
    if (dir == 1)
      b2::env_update_left(env, site);
    else
      b2::env_update_right(env, site);
  });
}

int b2_psi_layout(b2_ctx ctx, b2_env env, int site, int64_t* n_elem, int64_t* n_blocks) {
  return guarded(ctx, [&] {
    check_env(ctx, env);
    ensure_device(ctx);
    auto& wp = b2::window_program(env, site);
    if (n_elem) *n_elem = wp.psi.size;
    if (n_blocks) *n_blocks = int64_t(wp.psi.blocks.size());
  });
}

int b2_psi_blocks(b2_ctx ctx, b2_env env, int site, int64_t* table) {
  return guarded(ctx, [&] {
    check_env(ctx, env);
    B2_REQUIRE(table, B2_EINVAL, "null table");
    ensure_device(ctx);
    auto& wp = b2::window_program(env, site);
    for (size_t b = 0; b < wp.psi.blocks.size(); ++b) {
      const auto& p = wp.psi.blocks[b];
      int64_t* r = table + 6 * b;
      r[0] = p.jl; r[1] = p.s1; r[2] = p.s2; r[3] = p.jr; r[4] = p.off;
      r[5] = int64_t(p.ml) * p.mr;
    }
  });
}

int b2_psi_from_mps(b2_ctx ctx, b2_env env, int site, double* psi) {
  return guarded(ctx, [&] {
    check_env(ctx, env);
    B2_REQUIRE(psi, B2_EINVAL, "null psi");
    ensure_device(ctx);
    auto& wp = b2::window_program(env, site);
    b2_mps_s* mps = env->mps;
    const int i = b2::win_site(site);
    if (b2::win_nsite(site) == 1) {
      // the one-site psi has the layout of the site tensor itself
      const b2::SiteTensor& st = mps->sites[i];
      B2_REQUIRE(st.size == wp.psi.size, B2_EINVAL, "internal: one-site layout");
      if (st.size > 0)
        B2_CUDA(cudaMemcpyAsync(psi, st.data.ptr, sizeof(double) * size_t(st.size),
                                cudaMemcpyDeviceToDevice, ctx->c.stream));
    } else {
      b2::contract_two_sites(&ctx->c, mps->bonds[i], mps->bonds[i + 1], mps->sites[i],
                             mps->sites[i].data.as<double>(), mps->sites[i + 1],
                             mps->sites[i + 1].data.as<double>(), wp.psi, psi, nullptr);
    }
  });
}

int b2_heff_apply(b2_ctx ctx, b2_env env, int site, const double* psi, double* out,
                  b2_prec prec, double e_shift, double* algo_flops) {
  return guarded(ctx, [&] {
    check_env(ctx, env);
    B2_REQUIRE(psi && out, B2_EINVAL, "null vector");
    B2_REQUIRE(std::isfinite(e_shift), B2_EINVAL, "non-finite shift");
    B2_REQUIRE(prec == B2_FP64 || prec == B2_BF16X3 || prec == B2_TF32X3, B2_EINVAL,
               "unknown precision (B2_FP64, B2_BF16X3, B2_TF32X3)");
    ensure_device(ctx);
    auto& wp = b2::window_program(env, site);
    B2_REQUIRE(!overlap(psi, out, wp.psi.size), B2_EINVAL, "psi and out overlap");
    b2::heff_apply(env, site, psi, out, e_shift, algo_flops, prec);
  });
}

int b2_heff_diag(b2_ctx ctx, b2_env env, int site, double* diag) {
  return guarded(ctx, [&] {
    check_env(ctx, env);
    B2_REQUIRE(diag, B2_EINVAL, "null diag");
    ensure_device(ctx);
    b2::heff_diag(env, site, diag);
  });
}

int b2_davidson(b2_ctx ctx, b2_env env, int site, double* psi, const b2_dav_opts* opts,
                double* energy, int* n_matvec, double* resid2) {
  return guarded(ctx, [&] {
    check_env(ctx, env);
    B2_REQUIRE(psi && opts, B2_EINVAL, "null argument");
    B2_REQUIRE(opts->conv_tol >= 0 && std::isfinite(opts->conv_tol), B2_EINVAL, "bad conv_tol");
    ensure_device(ctx);
    b2::DavidsonResult r = b2::davidson(env, site, psi, *opts);
    if (energy) *energy = r.energy;
    if (n_matvec) *n_matvec = r.n_matvec;
    if (resid2) *resid2 = r.resid2;
  });
}

int b2_sweep(b2_ctx ctx, b2_mpo mpo, b2_mps mps, b2_env env, const b2_sweep_opts* opts,
             b2_sweep_result* per_sweep) {
  return guarded(ctx, [&] {
    check_env(ctx, env);
    B2_REQUIRE(opts && opts->bond_dims && opts->n_sweeps >= 0, B2_EINVAL, "bad sweep options");
    B2_REQUIRE(env->mpo == mpo && env->mps == mps, B2_EINVAL, "env was made for another mpo/mps");
    ensure_device(ctx);
    b2::sweep(env, *opts, per_sweep);
  });
}

int b2_tdvp(b2_ctx ctx, b2_mpo mpo, b2_mps mps, b2_env env, const b2_tdvp_opts* opts,
            b2_tdvp_result* per_step) {
  return guarded(ctx, [&] {
    check_env(ctx, env);
    B2_REQUIRE(opts && opts->n_steps >= 0, B2_EINVAL, "bad TDVP options");
    B2_REQUIRE(env->mpo == mpo && env->mps == mps, B2_EINVAL, "env was made for another mpo/mps");
    ensure_device(ctx);
    b2::tdvp(env, *opts, per_step);
  });
}

int b2_eigh_batched(b2_ctx ctx, int n_mat, const int* dims, const double* a, double* evals,
                    double* evecs) {
  return guarded(ctx, [&] {
    B2_REQUIRE(ctx && dims && a && evals && evecs, B2_EINVAL, "null argument");
    B2_REQUIRE(n_mat >= 0, B2_EINVAL, "n_mat < 0");
    ensure_device(ctx);
    b2::Ctx* c = &ctx->c;
    std::vector<int> d(dims, dims + n_mat);
    std::vector<int64_t> offs(n_mat), eoffs(n_mat);
    int64_t o = 0, e = 0;
    for (int i = 0; i < n_mat; ++i) {
      B2_REQUIRE(d[i] >= 1 && d[i] <= 1024, B2_EINVAL, "dims must be in [1, 1024]");
      offs[i] = o;
      eoffs[i] = e;
      o += int64_t(d[i]) * d[i];
      e += d[i];
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->prof) {
      B2_CUDA(cudaEventCreate(&e0));
      B2_CUDA(cudaEventCreate(&e1));
      B2_CUDA(cudaEventRecord(e0, c->stream));
    }
    b2::eigh_batched(c, d, offs, eoffs, a, evals, evecs, c->prof ? c->d_eig_flops : nullptr);
    if (c->prof) {
      B2_CUDA(cudaEventRecord(e1, c->stream));
      c->eig_events.push_back({e0, e1});
    }
    B2_CUDA(cudaGetLastError());
    B2_CUDA(cudaStreamSynchronize(c->stream));
  });
}

int b2_heff_apply_batched(b2_ctx ctx, int n, const b2_env* envs, const int* sites,
                          const double* const* psis, double* const* outs, b2_prec prec,
                          double* algo_flops) {
  return guarded(ctx, [&] {
    B2_REQUIRE(n >= 0, B2_EINVAL, "n < 0");
    if (n == 0) return;
    B2_REQUIRE(envs && sites && psis && outs, B2_EINVAL, "null argument");
    B2_REQUIRE(prec == B2_FP64 || prec == B2_BF16X3 || prec == B2_TF32X3, B2_EINVAL,
               "unknown precision (B2_FP64, B2_BF16X3, B2_TF32X3)");
    for (int i = 0; i < n; ++i) check_env(ctx, envs[i]);
    ensure_device(ctx);
    b2::heff_apply_batched(&ctx->c, n, envs, sites, psis, outs, prec, algo_flops);
  });
}

int b2_davidson_batched(b2_ctx ctx, int n, const b2_env* envs, const int* sites,
                        double* const* psis, const b2_dav_opts* opts, double* energies,
                        int* n_matvec, double* resid2) {
  return guarded(ctx, [&] {
    B2_REQUIRE(n >= 0, B2_EINVAL, "n < 0");
    if (n == 0) return;
    B2_REQUIRE(envs && sites && psis && opts, B2_EINVAL, "null argument");
    for (int i = 0; i < n; ++i) {
      check_env(ctx, envs[i]);
      B2_REQUIRE(psis[i] != nullptr, B2_EINVAL, "null psi");
    }
    ensure_device(ctx);
    std::vector<b2_env_s*> e(envs, envs + n);
    std::vector<int> s(sites, sites + n);
    std::vector<double*> p(psis, psis + n);
    std::vector<b2::DavidsonResult> r = b2::davidson_batched(&ctx->c, e, s, p, *opts);
    for (int i = 0; i < n; ++i) {
      if (energies) energies[i] = r[i].energy;
      if (n_matvec) n_matvec[i] = r[i].n_matvec;
      if (resid2) resid2[i] = r[i].resid2;
    }
  });
}

int b2_sweep_batched(b2_ctx ctx, int n, const b2_env* envs, const b2_sweep_opts* opts,
                     b2_sweep_result* results) {
  return guarded(ctx, [&] {
    B2_REQUIRE(n >= 0, B2_EINVAL, "n < 0");
    if (n == 0) return;
    B2_REQUIRE(envs && opts && opts->bond_dims && opts->n_sweeps >= 0, B2_EINVAL,
               "bad batched sweep arguments");
    for (int i = 0; i < n; ++i) check_env(ctx, envs[i]);
    ensure_device(ctx);
    std::vector<b2_env_s*> e(envs, envs + n);
    b2::sweep_batched(&ctx->c, e, *opts, results);
  });
}

int b2_sweep_batched_dims(b2_ctx ctx, int n, const b2_env* envs, const b2_sweep_opts* opts,
                          const int* bond_dims, b2_sweep_result* results) {
  return guarded(ctx, [&] {
    B2_REQUIRE(n >= 0, B2_EINVAL, "n < 0");
    if (n == 0) return;
    B2_REQUIRE(envs && opts && bond_dims && opts->n_sweeps >= 0, B2_EINVAL,
               "bad batched sweep arguments");
    for (int i = 0; i < n; ++i) check_env(ctx, envs[i]);
    ensure_device(ctx);
    std::vector<b2_env_s*> e(envs, envs + n);
    b2::sweep_batched(&ctx->c, e, *opts, results, bond_dims);
  });
}

int b2_rdm_grad(b2_ctx ctx, b2_mpo mpo, b2_mps mps, double* h1_grad, double* eri_grad) {
  return guarded(ctx, [&] {
    B2_REQUIRE(ctx && mpo && mps && h1_grad && eri_grad, B2_EINVAL, "null argument");
    B2_REQUIRE(!mpo->compressed, B2_EUNSUPPORTED,
               "the gradient needs the exact MPO (a compressed one has no coefficient Jacobian)");
    B2_REQUIRE(mps->ctx == &ctx->c, B2_EINVAL, "mps belongs to another context");
    ensure_device(ctx);
    b2::rdm_grad(&ctx->c, mpo, mps, h1_grad, eri_grad);
  });
}

int b2_debug_limits(b2_ctx ctx, int stuck_wait_polls, int jacobi_max_sweeps) {
  return guarded(ctx, [&] {
    B2_REQUIRE(ctx, B2_EINVAL, "null context");
    B2_REQUIRE(stuck_wait_polls >= 0 && jacobi_max_sweeps >= 0, B2_EINVAL, "limits must be >= 0");
    ctx->c.stuck_polls = uint32_t(stuck_wait_polls);
    ctx->c.jacobi_max_sweeps = jacobi_max_sweeps;
  });
}

int b2_sync(b2_ctx ctx) {
  return guarded(ctx, [&] {
    B2_REQUIRE(ctx, B2_EINVAL, "null context");
    ensure_device(ctx);
    B2_CUDA(cudaStreamSynchronize(ctx->c.stream));
    B2_CUDA(cudaGetLastError());
    B2_REQUIRE(ctx->c.take_status() == 0, B2_ETIMEOUT,
               "a bounded device-side wait ran out since the last check");
  });
}

int b2_profile(b2_ctx ctx, int enable) {
  return guarded(ctx, [&] {
    B2_REQUIRE(ctx, B2_EINVAL, "null context");
    B2_CUDA(cudaStreamSynchronize(ctx->c.stream));
    ensure_device(ctx);
    if (enable && !ctx->c.d_eig_flops)
      ctx->c.d_eig_flops = static_cast<double*>(ctx->c.raw_alloc(256));
    ctx->c.prof_clear();
    ctx->c.prof = enable != 0;
    ctx->c.launch_base = b2k::launch_count();
  });
}

int b2_profile_read(b2_ctx ctx, b2_profile_data* out) {
  return guarded(ctx, [&] {
    B2_REQUIRE(ctx && out, B2_EINVAL, "null argument");
    B2_CUDA(cudaStreamSynchronize(ctx->c.stream));
    double ms = 0;
    for (auto& e : ctx->c.prof_events) {
      float t = 0;
      B2_CUDA(cudaEventElapsedTime(&t, e.first, e.second));
      ms += t;
    }
    out->launches = b2k::launch_count() - ctx->c.launch_base;
    out->heff_launches = int64_t(ctx->c.prof_events.size());
    out->heff_ms = ms;
    out->heff_flops = ctx->c.prof_flops;
    double ems = 0, ef = 0;
    for (auto& e : ctx->c.eig_events) {
      float t = 0;
      B2_CUDA(cudaEventElapsedTime(&t, e.first, e.second));
      ems += t;
    }
    if (ctx->c.d_eig_flops)
      B2_CUDA(cudaMemcpy(&ef, ctx->c.d_eig_flops, sizeof(double), cudaMemcpyDeviceToHost));
    out->eig_launches = int64_t(ctx->c.eig_events.size());
    out->eig_ms = ems;
    out->eig_flops = ef;
    double rms = 0;
    for (auto& e : ctx->c.rr_events) {
      float t = 0;
      B2_CUDA(cudaEventElapsedTime(&t, e.first, e.second));
      rms += t;
    }
    out->rr_launches = int64_t(ctx->c.rr_events.size());
    out->rr_ms = rms;
  });
}

void b2_free_mpo(b2_mpo mpo) { delete mpo; }
void b2_free_mps(b2_mps mps) {
  if (mps && mps->ctx) cudaStreamSynchronize(mps->ctx->stream);
  delete mps;
}
void b2_free_env(b2_env env) {
  if (env && env->ctx) cudaStreamSynchronize(env->ctx->stream);
  delete env;
}

}  // extern "C"
