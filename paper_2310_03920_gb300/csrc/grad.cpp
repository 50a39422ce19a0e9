// Energy gradient with respect to the integrals at a fixed MPS: the 1- and 2-particle
// density matrices (block2 paper, Sec. 2.5.1 N-PDMs; the gradient pattern of Sec. 2.4.2's
// automatic differentiation applied to the MPO coefficients).
//
// For E(h, eri) = <Psi|H(h, eri)|Psi>, E is linear in every MPO coefficient.  Each
// site-ordered operator string s has one MPO entry W_k[w, w2] where its coefficient c_s
// enters as c_s * op_s, with a plain (coefficient-free) left channel w and right channel
// w2, so dE/dc_s = <s> = sum_{s' s} G_k[w, w2]_{s' s} (op_s)_{s' s}, where
//   G_k[w, w2]_{s' s} = sum (-1)^{sign} conj(psi)[l' s' r'] L_w[l', l] psi[l s r] R_w2[r', r]
// is the adjoint of the one-site effective Hamiltonian with respect to that entry (psi the
// MPS with its orthogonality centre on site k).  The chain rule through the builder's
// Jacobian gives dE/dh_pq = sum of signed <s> over the strings h_pq feeds (= gamma_pq) and
// dE/d(pq|rs) = 1/2 of the same sum for (pq|rs) (= Gamma_pqrs / 2).
//
// The computation runs on a private copy of the MPS with an MPO built from generic
// integrals of the same symmetry (so that every string and channel exists, also for
// integrals that are zero in the caller's Hamiltonian): a right-to-left pass builds all
// right environments, then the centre moves left to right; at site k the kernels form
// M_{w2 s' s} = psi_{s'} R_w2 psi_s^T block by block (3-operand block GEMMs) and G as
// signed Frobenius products of M with the left environments, grouped into one FP64 GEMM per
// quantum-number class (site_expectations).
#include <algorithm>
#include <cmath>
#include <map>

#include "algo.hpp"

b2_mpo_s* b2_build_mpo_impl(int n, const double* h1, const double* eri, double e_core, int n_elec,
                            int two_sz, double cutoff);

namespace b2 {

using b2k::GemmTerm;

namespace {

std::unique_ptr<b2_mps_s> copy_mps(Ctx* c, const b2_mps_s* m) {
  std::unique_ptr<b2_mps_s> out(new b2_mps_s);
  out->ctx = c;
  out->n = m->n;
  out->n_elec = m->n_elec;
  out->two_sz = m->two_sz;
  out->center = m->center;
  out->bonds = m->bonds;
  out->sites.resize(m->n);
  for (int k = 0; k < m->n; ++k) {
    const SiteTensor& s = m->sites[k];
    SiteTensor& d = out->sites[k];
    d.blocks = s.blocks;
    d.lookup = s.lookup;
    d.size = s.size;
    d.data.reset(c, sizeof(double) * std::max<int64_t>(s.size, 1));
    B2_CUDA(cudaMemcpyAsync(d.data.ptr, s.data.ptr, sizeof(double) * s.size,
                            cudaMemcpyDeviceToDevice, c->stream));
  }
  return out;
}

// Eigen-decompose the m_j x m_j Gram matrices G_j (stored consecutively at goff) and write
// U diag(lam^-1/2) to U1 and U diag(lam^1/2) to U2.
void gram_factors(Ctx* c, const std::vector<int>& dims, const std::vector<int64_t>& goff,
                  const std::vector<int64_t>& eoff, DevBuf& G, DevBuf& U, DevBuf& lam, DevBuf& U1,
                  DevBuf& U2) {
  for (size_t j = 0; j < dims.size(); ++j)
    B2_REQUIRE(dims[j] <= 1024, B2_EUNSUPPORTED, "gradient: bond sector larger than 1024 states");
  eigh_batched(c, dims, goff, eoff, G.as<double>(), lam.as<double>(), U.as<double>());
  // Directions with Gram eigenvalue below kNullGram carry at most sqrt(kNullGram) of the
  // (normalised) state; they are dropped from both factors rather than blown up by lam^-1/2.
  constexpr double kNullGram = 1e-28;
  for (size_t j = 0; j < dims.size(); ++j) {
    b2k::launch_scale_cols(dims[j], U.as<double>() + goff[j], lam.as<double>() + eoff[j], -0.5,
                           kNullGram, U1.as<double>() + goff[j], c->stream, true);
    b2k::launch_scale_cols(dims[j], U.as<double>() + goff[j], lam.as<double>() + eoff[j], 0.5,
                           kNullGram, U2.as<double>() + goff[j], c->stream, true);
  }
  B2_CUDA(cudaGetLastError());
  // wait before the host-side metadata vectors go out of scope
  B2_CUDA(cudaStreamSynchronize(c->stream));
}

// Move the orthogonality centre from site k to k+1: for each right sector r of bond k+1,
// X_r = the (jl, s) rows of site k with that sector, G = X_r^T X_r = V lam V^T,
// site k <- X V lam^-1/2 (left-orthonormal), site k+1 <- lam^1/2 V^T site k+1.
void move_center_right(Ctx* c, b2_mps_s* mps, int k) {
  SiteTensor& st = mps->sites[k];
  SiteTensor& nx = mps->sites[k + 1];
  const Bond& br = mps->bonds[k + 1];
  std::vector<int> dims(br.size());
  std::vector<int64_t> goff(br.size()), eoff(br.size());
  int64_t gsize = 0, esize = 0;
  for (int j = 0; j < br.size(); ++j) {
    dims[j] = br.m[j];
    goff[j] = gsize;
    eoff[j] = esize;
    gsize += int64_t(br.m[j]) * br.m[j];
    esize += br.m[j];
  }
  DevBuf G(c, sizeof(double) * gsize), U(c, sizeof(double) * gsize), lam(c, sizeof(double) * esize),
      U1(c, sizeof(double) * gsize), U2(c, sizeof(double) * gsize);
  GemmProgram pg;
  std::vector<int> outs(br.size());
  for (int j = 0; j < br.size(); ++j) outs[j] = pg.add_out(1, goff[j], br.m[j], br.m[j], br.m[j], false);
  for (const auto& blk : st.blocks) {
    GemmTerm t{};
    t.offP = blk.off; t.bufP = 0; t.ldP = blk.mr;   // op(P) = X^T
    t.offX = blk.off; t.bufX = 0; t.ldX = blk.mr;
    t.K1 = blk.ml;
    t.flags = b2k::kTwoOp | b2k::kTransP;
    t.alpha = 1.0;
    pg.add_term(outs[blk.jr], t);
  }
  pg.finalize(c);
  b2k::BufTable bt{};
  bt.p[0] = st.data.as<double>();
  bt.p[1] = G.as<double>();
  pg.launch(c, bt);
  gram_factors(c, dims, goff, eoff, G, U, lam, U1, U2);
  // A = X U1 ; new next = U2^T next
  DevBuf na(c, sizeof(double) * std::max<int64_t>(st.size, 1));
  GemmProgram pa;
  for (const auto& blk : st.blocks) {
    int o = pa.add_out(1, blk.off, blk.ml, blk.mr, blk.mr, false);
    GemmTerm t{};
    t.offP = blk.off; t.bufP = 0; t.ldP = blk.mr;
    t.offX = goff[blk.jr]; t.bufX = 2; t.ldX = blk.mr;
    t.K1 = blk.mr;
    t.flags = b2k::kTwoOp;
    t.alpha = 1.0;
    pa.add_term(o, t);
  }
  pa.finalize(c);
  b2k::BufTable ba{};
  ba.p[0] = st.data.as<double>();
  ba.p[1] = na.as<double>();
  ba.p[2] = U1.as<double>();
  pa.launch(c, ba);
  DevBuf nn(c, sizeof(double) * std::max<int64_t>(nx.size, 1));
  GemmProgram pn;
  for (const auto& blk : nx.blocks) {
    int o = pn.add_out(1, blk.off, blk.ml, blk.mr, blk.mr, false);
    GemmTerm t{};
    t.offP = goff[blk.jl]; t.bufP = 2; t.ldP = blk.ml;   // op(P) = U2^T
    t.offX = blk.off; t.bufX = 0; t.ldX = blk.mr;
    t.K1 = blk.ml;
    t.flags = b2k::kTwoOp | b2k::kTransP;
    t.alpha = 1.0;
    pn.add_term(o, t);
  }
  pn.finalize(c);
  b2k::BufTable bn{};
  bn.p[0] = nx.data.as<double>();
  bn.p[1] = nn.as<double>();
  bn.p[2] = U2.as<double>();
  pn.launch(c, bn);
  B2_CUDA(cudaGetLastError());
  B2_CUDA(cudaStreamSynchronize(c->stream));
  st.data = std::move(na);
  nx.data = std::move(nn);
  mps->center = k + 1;
}

// <string> for every string whose coefficient enters at site k (centre on site k).
//
// With ket sector j of bond k and bra sector j', the one-site adjoint of entry (w, w2) is
//   G[w, w2]_{s' s} = sum_j sign_j <L_w[j' <- j], M_{w2 s' s}[j' <- j]>  (Frobenius),
//   M_{w2 s' s}[j' <- j] = psi(j', s') R_w2[jr' <- jr] psi(j, s)^T,
//   sign_j = (-1)^(p(s' <- s) N(j) + p(w2) (N(j) + n(s)))   (fermion order l, s, r).
// Only pairs with dq(w) = q(s) + dq(w2) - q(s') =: D can be nonzero, and then j' is fixed
// by j and D.  For each class D the requested channels w become rows and the requested
// (w2, s', s) columns of one matrix G_D = sum_j Lg_{D,j} Mg_{D,j}^T, where Lg_{D,j} gathers
// the L blocks (j' <- j) of the rows, flattened, and Mg_{D,j} holds the signed M blocks of
// the columns: one grouped FP64 GEMM per site instead of one reduction per element.
void site_expectations(b2_env_s* env, int k, const std::vector<int>& strs, std::vector<double>& ev) {
  Ctx* c = env->ctx;
  b2_mpo_s* mpo = env->mpo;
  b2_mps_s* mps = env->mps;
  const SiteTensor& psi = mps->sites[k];
  const Bond& bk = mps->bonds[k];
  const Bond& bk1 = mps->bonds[k + 1];
  const EnvBond& L = env->L[k];
  const EnvBond& R = env->R[k + 1];
  B2_REQUIRE(L.valid && R.valid, B2_EINVAL, "internal: gradient environments");
  auto op_elem = [&](const b2_mpo_s::StringEntry& e, int a) {
    return e.op < 0 ? (a / 4 == a % 4 ? 1.0 : 0.0) : mpo->ops[e.op][a];
  };
  // columns m = (w2, s', s) and their classes D
  std::map<std::tuple<int, int, int>, int> midx;
  std::vector<std::tuple<int, int, int>> mkeys;
  for (int si : strs) {
    const auto& e = mpo->str_entry[si];
    for (int a = 0; a < 16; ++a) {
      if (op_elem(e, a) == 0) continue;
      auto key = std::make_tuple(e.w2, a / 4, a % 4);
      if (!midx.count(key)) {
        midx[key] = int(mkeys.size());
        mkeys.push_back(key);
      }
    }
  }
  std::map<int64_t, int> cls_of_d;   // QN key of D -> class
  std::vector<QN> cls_d;
  std::vector<int> m_cls(mkeys.size()), m_col(mkeys.size());
  std::vector<int> n_cols;
  for (size_t mi = 0; mi < mkeys.size(); ++mi) {
    int w2 = std::get<0>(mkeys[mi]), sp = std::get<1>(mkeys[mi]), s_ = std::get<2>(mkeys[mi]);
    QN d = kSiteQ[s_] + mpo->dq[k + 1][w2] - kSiteQ[sp];
    auto it = cls_of_d.find(d.key());
    int cl;
    if (it == cls_of_d.end()) {
      cl = int(cls_d.size());
      cls_of_d[d.key()] = cl;
      cls_d.push_back(d);
      n_cols.push_back(0);
    } else {
      cl = it->second;
    }
    m_cls[mi] = cl;
    m_col[mi] = n_cols[cl]++;
  }
  // rows: requested channels w whose dq matches the class of the column they pair with
  const int ncls = int(cls_d.size());
  std::vector<std::map<int, int>> rows(ncls);
  for (int si : strs) {
    const auto& e = mpo->str_entry[si];
    for (int a = 0; a < 16; ++a) {
      if (op_elem(e, a) == 0) continue;
      int mi = midx[std::make_tuple(e.w2, a / 4, a % 4)];
      int cl = m_cls[mi];
      if (!(mpo->dq[k][e.w] == cls_d[cl])) continue;
      if (!rows[cl].count(e.w)) {
        int r = int(rows[cl].size());
        rows[cl][e.w] = r;
      }
    }
  }
  // offsets of Lg, Mg (per class, per ket sector) and G (per class)
  std::vector<std::vector<int>> bra(ncls, std::vector<int>(bk.size(), -1));
  std::vector<std::vector<int64_t>> lg_off(ncls, std::vector<int64_t>(bk.size(), 0)),
      mg_off(ncls, std::vector<int64_t>(bk.size(), 0));
  std::vector<int64_t> g_off(ncls, 0);
  int64_t lg_size = 0, mg_size = 0, g_size = 0;
  for (int cl = 0; cl < ncls; ++cl) {
    const int nr = int(rows[cl].size()), nc = n_cols[cl];
    g_off[cl] = g_size;
    g_size += int64_t(nr) * nc;
    if (nr == 0) continue;
    for (int j = 0; j < bk.size(); ++j) {
      int jp = bk.find(bk.q[j] + cls_d[cl]);
      if (jp < 0) continue;
      bra[cl][j] = jp;
      const int64_t x = int64_t(bk.m[jp]) * bk.m[j];
      lg_off[cl][j] = lg_size;
      lg_size += nr * x;
      mg_off[cl][j] = mg_size;
      mg_size += nc * x;
    }
  }
  std::vector<double> g(std::max<int64_t>(g_size, 1), 0.0);
  if (lg_size > 0) {
    DevBuf Lg(c, sizeof(double) * lg_size), Mg(c, sizeof(double) * mg_size),
        G(c, sizeof(double) * g_size);
    B2_CUDA(cudaMemsetAsync(Mg.ptr, 0, sizeof(double) * mg_size, c->stream));
    // gather the L blocks
    std::vector<b2k::CopyTask> cp;
    for (int cl = 0; cl < ncls; ++cl)
      for (const auto& wr : rows[cl])
        for (int j = 0; j < bk.size(); ++j) {
          if (bra[cl][j] < 0) continue;
          int lb = L.blk[wr.first][j];
          B2_REQUIRE(lb >= 0 && L.blocks[lb].jb == bra[cl][j], B2_EINVAL,
                     "internal: gradient environment block");
          const int mb = L.blocks[lb].mb, mk = L.blocks[lb].mk;
          b2k::CopyTask t{};
          t.src = L.blocks[lb].off;
          t.dst = lg_off[cl][j] + int64_t(wr.second) * mb * mk;
          t.rows = mb;
          t.cols = mk;
          t.lds = mk;
          t.ldd = mk;
          t.trans = 0;
          t.bsrc = 0;
          t.bdst = 1;
          cp.push_back(t);
        }
    DevBuf d_cp;
    upload(c, d_cp, cp);
    b2k::BufTable bc{};
    bc.p[0] = L.data.as<double>();
    bc.p[1] = Lg.as<double>();
    b2k::launch_copy(int(cp.size()), d_cp.as<b2k::CopyTask>(), bc, c->stream);
    // signed M blocks
    GemmProgram pm;
    for (size_t mi = 0; mi < mkeys.size(); ++mi) {
      const int cl = m_cls[mi];
      if (rows[cl].empty()) continue;
      const int w2 = std::get<0>(mkeys[mi]), sp = std::get<1>(mkeys[mi]), s_ = std::get<2>(mkeys[mi]);
      const int pop = (kSiteN[sp] + kSiteN[s_]) & 1;
      const int pw2 = mpo->parity[k + 1][w2];
      for (int j = 0; j < bk.size(); ++j) {
        const int jp = bra[cl][j];
        if (jp < 0) continue;
        const int b = psi.find(j, s_);
        if (b < 0) continue;
        const SiteBlock& kb = psi.blocks[b];
        const int rb = R.blk[w2][kb.jr];
        if (rb < 0) continue;
        const int jrp = R.blocks[rb].jb;
        const int bb = psi.find(jp, sp);
        if (bb < 0 || psi.blocks[bb].jr != jrp) continue;
        const SiteBlock& pb = psi.blocks[bb];
        const int64_t x = int64_t(pb.ml) * kb.ml;
        int o = pm.add_out(1, mg_off[cl][j] + int64_t(m_col[mi]) * x, pb.ml, kb.ml, kb.ml, false);
        const int par = pop * (bk.q[j].n & 1) + pw2 * ((bk.q[j].n + kSiteN[s_]) & 1);
        GemmTerm t{};
        t.offP = pb.off; t.bufP = 0; t.ldP = pb.mr;             // psi(j', s') [m_j' x m_jr']
        t.offX = R.blocks[rb].off; t.bufX = 2; t.ldX = kb.mr;   // R_w2 [m_jr' x m_jr]
        t.offQ = kb.off; t.bufQ = 0; t.ldQ = kb.mr;             // psi(j, s)^T [m_jr x m_j]
        t.K1 = pb.mr;
        t.K2 = kb.mr;
        t.flags = b2k::kTransQ;
        t.alpha = (par & 1) ? -1.0 : 1.0;
        pm.add_term(o, t);
      }
    }
    pm.finalize(c);
    b2k::BufTable bt{};
    bt.p[0] = psi.data.as<double>();
    bt.p[1] = Mg.as<double>();
    bt.p[2] = R.data.as<double>();
    pm.launch(c, bt);
    // G_D = sum_j Lg_{D,j} Mg_{D,j}^T
    GemmProgram pg;
    for (int cl = 0; cl < ncls; ++cl) {
      const int nr = int(rows[cl].size()), nc = n_cols[cl];
      if (nr == 0 || nc == 0) continue;
      int o = pg.add_out(1, g_off[cl], nr, nc, nc, false);
      for (int j = 0; j < bk.size(); ++j) {
        const int jp = bra[cl][j];
        if (jp < 0) continue;
        const int x = bk.m[jp] * bk.m[j];
        GemmTerm t{};
        t.offP = lg_off[cl][j]; t.bufP = 0; t.ldP = x;
        t.offX = mg_off[cl][j]; t.bufX = 2; t.ldX = x;
        t.K1 = x;
        t.flags = b2k::kTwoOp | b2k::kTransQ;
        t.alpha = 1.0;
        pg.add_term(o, t);
      }
    }
    pg.finalize(c);
    b2k::BufTable bg{};
    bg.p[0] = Lg.as<double>();
    bg.p[1] = G.as<double>();
    bg.p[2] = Mg.as<double>();
    B2_CUDA(cudaMemsetAsync(G.ptr, 0, sizeof(double) * g_size, c->stream));
    pg.launch(c, bg);
    B2_CUDA(cudaGetLastError());
    B2_CUDA(cudaMemcpyAsync(g.data(), G.ptr, sizeof(double) * g_size, cudaMemcpyDeviceToHost,
                            c->stream));
    B2_CUDA(cudaStreamSynchronize(c->stream));
  }
  for (int si : strs) {
    const auto& e = mpo->str_entry[si];
    double v = 0;
    for (int a = 0; a < 16; ++a) {
      const double x = op_elem(e, a);
      if (x == 0) continue;
      const int mi = midx[std::make_tuple(e.w2, a / 4, a % 4)];
      const int cl = m_cls[mi];
      auto it = rows[cl].find(e.w);
      if (it == rows[cl].end()) continue;   // dq mismatch: this element of G is zero
      v += x * g[g_off[cl] + int64_t(it->second) * n_cols[cl] + m_col[mi]];
    }
    ev[si] = v;
  }
}

// generic integrals with the symmetry of a real Hamiltonian (every string present)
void generic_integrals(int n, std::vector<double>& h, std::vector<double>& eri) {
  auto u = [](uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return 0.5 + double(x >> 11) * (1.0 / 9007199254740992.0);
  };
  h.assign(size_t(n) * n, 0.0);
  for (int p = 0; p < n; ++p)
    for (int q = p; q < n; ++q) h[size_t(p) * n + q] = h[size_t(q) * n + p] = u(uint64_t(p) * 131 + q);
  eri.assign(size_t(n) * n * n * n, 0.0);
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s) {
          int a = std::min(p, q), b = std::max(p, q), cc = std::min(r, s), d = std::max(r, s);
          int x = a * n + b, y = cc * n + d;
          uint64_t key = uint64_t(std::min(x, y)) * 1000003ull + uint64_t(std::max(x, y)) + 7777;
          eri[((size_t(p) * n + q) * n + r) * n + s] = u(key);
        }
}

}  // namespace

void rdm_grad(Ctx* c, b2_mpo_s* ham, b2_mps_s* mps_in, double* h1_grad, double* eri_grad) {
  B2_REQUIRE(ham->n == mps_in->n && ham->n_elec == mps_in->n_elec && ham->two_sz == mps_in->two_sz,
             B2_EINVAL, "mpo and mps describe different systems");
  B2_REQUIRE(mps_in->center == 0, B2_EINVAL, "b2_rdm_grad needs an MPS centred at site 0");
  const int n = mps_in->n;
  std::vector<double> gh, geri;
  generic_integrals(n, gh, geri);
  std::unique_ptr<b2_mpo_s> gm(b2_build_mpo_impl(n, gh.data(), geri.data(), 0.0, mps_in->n_elec,
                                                 mps_in->two_sz, 0.0));
  std::unique_ptr<b2_mps_s> mps = copy_mps(c, mps_in);
  // <psi|psi> from the centre site
  double norm2 = 0.0;
  {
    const SiteTensor& s0 = mps->sites[0];
    B2_REQUIRE(s0.size > 0 && s0.size < (int64_t(1) << 31), B2_EINVAL, "internal: centre site size");
    std::vector<b2k::DotOut> o{{0, 1}};
    std::vector<b2k::DotTerm> t{{0, 0, int(s0.size), 1.0}};
    DevBuf d_o, d_t, d_n(c, sizeof(double));
    upload(c, d_o, o);
    upload(c, d_t, t);
    b2k::launch_dots(1, d_o.as<b2k::DotOut>(), d_t.as<b2k::DotTerm>(), s0.data.as<double>(),
                     s0.data.as<double>(), d_n.as<double>(), c->stream);
    B2_CUDA(cudaGetLastError());
    B2_CUDA(cudaMemcpyAsync(&norm2, d_n.ptr, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    B2_CUDA(cudaStreamSynchronize(c->stream));
    B2_REQUIRE(norm2 > 0 && std::isfinite(norm2), B2_EINVAL, "MPS has zero or non-finite norm");
  }
  b2_env_s env;
  env.ctx = c;
  env.mpo = gm.get();
  env.mps = mps.get();
  env.L.resize(n + 1);
  env.R.resize(n + 1);
  const double one = 1.0;
  auto boundary = [&](EnvBond& e, const Bond& b, const std::vector<QN>& dq) {
    e.layout(b, dq);
    e.data.reset(c, sizeof(double));
    B2_CUDA(cudaMemcpyAsync(e.data.ptr, &one, sizeof(double), cudaMemcpyHostToDevice, c->stream));
    e.valid = true;
    e.version = ++env.version_counter;
  };
  boundary(env.L[0], mps->bonds[0], gm->dq[0]);
  boundary(env.R[n], mps->bonds[n], gm->dq[n]);
  for (int k = n - 1; k >= 1; --k) env_update_right(&env, k);
  // strings by the site where their coefficient enters
  std::vector<std::vector<int>> at(n);
  for (size_t si = 0; si < gm->str_entry.size(); ++si) {
    const auto& e = gm->str_entry[si];
    B2_REQUIRE(e.site >= 0, B2_EINVAL, "internal: string without an MPO entry");
    at[e.site].push_back(int(si));
  }
  std::vector<double> ev(gm->str_entry.size(), 0.0);
  for (int k = 0; k < n; ++k) {
    site_expectations(&env, k, at[k], ev);
    if (k + 1 < n) {
      move_center_right(c, mps.get(), k);
      env_update_left(&env, k);
      env.R[k + 1].data.release();   // no longer needed
    }
  }
  // chain rule through the builder's Jacobian
  const size_t n2 = size_t(n) * n, n4 = n2 * n2;
  std::fill(h1_grad, h1_grad + n2, 0.0);
  std::fill(eri_grad, eri_grad + n4, 0.0);
  const double inv = 1.0 / norm2;
  for (const auto& t : gm->terms) {
    if (t.kind == 0)
      h1_grad[t.integral] += t.sign * ev[t.str] * inv;
    else
      eri_grad[t.integral] += 0.5 * t.sign * ev[t.str] * inv;
  }
  B2_CUDA(cudaStreamSynchronize(c->stream));
}

}  // namespace b2
