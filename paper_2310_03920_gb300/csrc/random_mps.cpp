// Random initial MPS (block2 paper, Sec. 2.1.6 "Initial guesses": (i) a random MPS of the
// requested bond dimension; (ii) the initial quantum-number distribution from occupancies
// of each site assumed independent).
//
// Sector sizes: every spin orbital p is occupied with probability f_p independently, so the
// (N_alpha, N_beta) content of the left block at bond k follows a product of two
// Poisson-binomial distributions; m_q = max(1, round(M P(q))) over sectors compatible with
// the remaining sites and with P(q) >= 1e-12, capped by the Fock dimension of both blocks,
// scaled down until sum_q m_q <= M, then made consistent between neighbouring bonds.
// Entries: standard normal numbers from a counter-based generator (SplitMix64 of
// seed + counter, Box-Muller), counter = position of the entry in the concatenated site
// data.  Right-orthonormal form on the GPU: for site k = n-1 .. 1 and each left sector j,
// G = X X^T over the sector's row block X, G = U diag(lam) U^T (batched Jacobi kernel),
// B = diag(lam^-1/2) U^T X, and U diag(lam^1/2) is multiplied into site k-1; done twice per
// site, so that the orthonormality error is not the first pass's 1e-15 / min(lam).  Site 0 is
// scaled to unit norm.
#include <algorithm>
#include <cmath>
#include <map>

#include "algo.hpp"

namespace {

using b2::Bond;
using b2::QN;

std::vector<double> poisson_binomial(const double* f, int k) {
  std::vector<double> pmf(k + 1, 0.0);
  pmf[0] = 1.0;
  for (int i = 0; i < k; ++i) {
    for (int c = i + 1; c >= 1; --c) pmf[c] = pmf[c] * (1.0 - f[i]) + pmf[c - 1] * f[i];
    pmf[0] *= (1.0 - f[i]);
  }
  return pmf;
}

double comb(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return std::round(r);
}

std::vector<std::map<std::pair<int, int>, int>> sector_sizes(int n, int n_elec, int two_sz, int M,
                                                             const std::vector<double>& f) {
  const int na = (n_elec + two_sz) / 2, nb = (n_elec - two_sz) / 2;
  std::vector<std::map<std::pair<int, int>, int>> bonds(n + 1);   // key (N, 2Sz)
  bonds[0][{0, 0}] = 1;
  bonds[n][{n_elec, two_sz}] = 1;
  for (int k = 1; k < n; ++k) {
    std::vector<double> pa = poisson_binomial(f.data(), k);
    std::map<std::pair<int, int>, double> prob;
    double tot = 0;
    for (int xa = std::max(0, na - (n - k)); xa <= std::min(k, na); ++xa)
      for (int xb = std::max(0, nb - (n - k)); xb <= std::min(k, nb); ++xb) {
        prob[{xa, xb}] = pa[xa] * pa[xb];
        tot += pa[xa] * pa[xb];
      }
    std::map<std::pair<int, int>, int> ms;
    std::map<std::pair<int, int>, double> pk;
    for (auto& kv : prob) {
      double p = kv.second / tot;
      if (p < 1e-12) continue;
      int xa = kv.first.first, xb = kv.first.second;
      double cap = std::min(comb(k, xa) * comb(k, xb), comb(n - k, na - xa) * comb(n - k, nb - xb));
      ms[kv.first] = int(std::min(cap, std::max(1.0, std::round(M * p))));
      pk[kv.first] = p;
    }
    auto total = [&] {
      long s = 0;
      for (auto& kv : ms) s += kv.second;
      return s;
    };
    while (total() > M) {
      double scale = double(M) / double(total());
      bool changed = false;
      for (auto& kv : ms) {
        int v = std::max(1, int(std::floor(kv.second * scale)));
        changed |= v != kv.second;
        kv.second = v;
      }
      if (!changed) {   // only single states left: drop the least probable sectors
        std::vector<std::pair<double, std::pair<int, int>>> order;
        for (auto& kv : ms) order.push_back({pk[kv.first], kv.first});
        std::sort(order.begin(), order.end());
        for (size_t i = 0; i < order.size() && total() > M; ++i) ms.erase(order[i].second);
      }
    }
    for (auto& kv : ms)
      bonds[k][{kv.first.first + kv.first.second, kv.first.first - kv.first.second}] = kv.second;
  }
  const int dn[4] = {0, 1, 1, 2}, ds[4] = {0, 1, -1, 0};
  for (bool changed = true; changed;) {
    changed = false;
    for (int k = 1; k <= n; ++k)
      for (auto it = bonds[k].begin(); it != bonds[k].end();) {
        int lim = 0;
        for (int s = 0; s < 4; ++s) {
          auto f2 = bonds[k - 1].find({it->first.first - dn[s], it->first.second - ds[s]});
          if (f2 != bonds[k - 1].end()) lim += f2->second;
        }
        if (lim < it->second) {
          changed = true;
          if (lim == 0) {
            it = bonds[k].erase(it);
            continue;
          }
          it->second = lim;
        }
        ++it;
      }
    for (int k = n - 1; k >= 0; --k)
      for (auto it = bonds[k].begin(); it != bonds[k].end();) {
        int lim = 0;
        for (int s = 0; s < 4; ++s) {
          auto f2 = bonds[k + 1].find({it->first.first + dn[s], it->first.second + ds[s]});
          if (f2 != bonds[k + 1].end()) lim += f2->second;
        }
        if (lim < it->second) {
          changed = true;
          if (lim == 0) {
            it = bonds[k].erase(it);
            continue;
          }
          it->second = lim;
        }
        ++it;
      }
  }
  return bonds;
}

uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

double gaussian(uint64_t seed, uint64_t counter) {
  // Box-Muller on two uniforms in (0, 1] from two generator outputs
  const uint64_t a = splitmix64(seed ^ splitmix64(2 * counter));
  const uint64_t b = splitmix64(seed ^ splitmix64(2 * counter + 1));
  const double u1 = (double((a >> 11) + 1)) * (1.0 / 9007199254740992.0);
  const double u2 = double(b >> 11) * (1.0 / 9007199254740992.0);
  return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
}

}  // namespace

b2_mps_s* b2_mps_random_impl(b2::Ctx* ctx, b2_mpo_s* mpo, int M, const double* occ,
                             uint64_t seed) {
  const int n = mpo->n;
  std::vector<double> f(n);
  for (int p = 0; p < n; ++p) {
    f[p] = occ ? occ[p] : 1.0 / (1.0 + std::exp((p + 0.5 - mpo->n_elec / 2.0) / 2.0));
    B2_REQUIRE(std::isfinite(f[p]) && f[p] >= 0 && f[p] <= 1, B2_EINVAL, "occupancies must be in [0, 1]");
  }
  auto sizes = sector_sizes(n, mpo->n_elec, mpo->two_sz, M, f);
  std::unique_ptr<b2_mps_s> mps(new b2_mps_s);
  mps->ctx = ctx;
  mps->n = n;
  mps->n_elec = mpo->n_elec;
  mps->two_sz = mpo->two_sz;
  mps->center = 0;
  mps->bonds.resize(n + 1);
  for (int k = 0; k <= n; ++k) {
    B2_REQUIRE(!sizes[k].empty(), B2_EINVAL, "no consistent sector on bond " + std::to_string(k));
    for (auto& kv : sizes[k]) {   // std::map orders by (N, 2Sz)
      mps->bonds[k].q.push_back(QN{kv.first.first, kv.first.second});
      mps->bonds[k].m.push_back(kv.second);
    }
    mps->bonds[k].finalize();
  }
  mps->sites.resize(n);
  uint64_t counter = 0;
  for (int k = 0; k < n; ++k) {
    auto& st = mps->sites[k];
    st.build(mps->bonds[k], mps->bonds[k + 1]);
    std::vector<double> h(size_t(std::max<int64_t>(st.size, 1)));
    for (int64_t i = 0; i < st.size; ++i) h[size_t(i)] = gaussian(seed, counter++);
    b2::upload(ctx, st.data, h);
  }
  // right-orthonormalise sites n-1 .. 1; two passes per site: the first leaves B B^T - I at
  // about 1e-15 / lam_min of the Gram matrix, the second (Gram matrix ~ I) at rounding level
  using b2k::GemmTerm;
  for (int k = n - 1; k >= 1; --k)
  for (int pass = 0; pass < 2; ++pass) {
    auto& st = mps->sites[k];
    const Bond& bl = mps->bonds[k];
    // G_j = X_j X_j^T for every left sector j, stored consecutively
    std::vector<int64_t> goff(bl.size());
    std::vector<int> dims(bl.size());
    int64_t gsize = 0, esize = 0;
    std::vector<int64_t> eoff(bl.size());
    for (int j = 0; j < bl.size(); ++j) {
      goff[j] = gsize;
      eoff[j] = esize;
      dims[j] = bl.m[j];
      gsize += int64_t(bl.m[j]) * bl.m[j];
      esize += bl.m[j];
    }
    b2::DevBuf G(ctx, sizeof(double) * gsize), U(ctx, sizeof(double) * gsize),
        lam(ctx, sizeof(double) * esize), U1(ctx, sizeof(double) * gsize),
        U2(ctx, sizeof(double) * gsize);
    b2::GemmProgram pg;
    for (int j = 0; j < bl.size(); ++j) {
      int o = pg.add_out(1, goff[j], bl.m[j], bl.m[j], bl.m[j], false);
      for (int s = 0; s < 4; ++s) {
        int b = st.find(j, s);
        if (b < 0) continue;
        const auto& blk = st.blocks[b];
        GemmTerm t{};
        t.offP = blk.off; t.bufP = 0; t.ldP = blk.mr;
        t.offX = blk.off; t.bufX = 0; t.ldX = blk.mr;    // op(X) = X^T
        t.K1 = blk.mr;
        t.flags = b2k::kTwoOp | b2k::kTransQ;
        t.alpha = 1.0;
        pg.add_term(o, t);
      }
    }
    pg.finalize(ctx);
    b2k::BufTable bt{};
    bt.p[0] = st.data.as<double>();
    bt.p[1] = G.as<double>();
    pg.launch(ctx, bt);
    // eigen-decomposition of every G_j
    b2::eigh_batched(ctx, dims, goff, eoff, G.as<double>(), lam.as<double>(), U.as<double>());
    for (int j = 0; j < bl.size(); ++j) {
      b2k::launch_scale_cols(dims[j], U.as<double>() + goff[j], lam.as<double>() + eoff[j], -0.5,
                             1e-300, U1.as<double>() + goff[j], ctx->stream);
      b2k::launch_scale_cols(dims[j], U.as<double>() + goff[j], lam.as<double>() + eoff[j], 0.5,
                             0.0, U2.as<double>() + goff[j], ctx->stream);
    }
    // B = U1^T X (new data of site k), site k-1 <- site k-1 . U2
    b2::DevBuf nb(ctx, sizeof(double) * std::max<int64_t>(st.size, 1));
    b2::GemmProgram pb;
    for (const auto& blk : st.blocks) {
      int o = pb.add_out(1, blk.off, blk.ml, blk.mr, blk.mr, false);
      GemmTerm t{};
      t.offP = goff[blk.jl]; t.bufP = 2; t.ldP = blk.ml;    // op(P) = U1^T
      t.offX = blk.off; t.bufX = 0; t.ldX = blk.mr;
      t.K1 = blk.ml;
      t.flags = b2k::kTwoOp | b2k::kTransP;
      t.alpha = 1.0;
      pb.add_term(o, t);
    }
    pb.finalize(ctx);
    b2k::BufTable bb{};
    bb.p[0] = st.data.as<double>();
    bb.p[1] = nb.as<double>();
    bb.p[2] = U1.as<double>();
    pb.launch(ctx, bb);
    auto& prev = mps->sites[k - 1];
    b2::DevBuf np(ctx, sizeof(double) * std::max<int64_t>(prev.size, 1));
    b2::GemmProgram pp;
    for (const auto& blk : prev.blocks) {
      int o = pp.add_out(1, blk.off, blk.ml, blk.mr, blk.mr, false);
      GemmTerm t{};
      t.offP = blk.off; t.bufP = 0; t.ldP = blk.mr;
      t.offX = goff[blk.jr]; t.bufX = 2; t.ldX = blk.mr;   // U2 of the right sector of site k-1
      t.K1 = blk.mr;
      t.flags = b2k::kTwoOp;
      t.alpha = 1.0;
      pp.add_term(o, t);
    }
    pp.finalize(ctx);
    b2k::BufTable bq{};
    bq.p[0] = prev.data.as<double>();
    bq.p[1] = np.as<double>();
    bq.p[2] = U2.as<double>();
    pp.launch(ctx, bq);
    B2_CUDA(cudaGetLastError());
    B2_CUDA(cudaStreamSynchronize(ctx->stream));
    st.data = std::move(nb);
    prev.data = std::move(np);
  }
  // unit norm on site 0
  auto& s0 = mps->sites[0];
  b2::DevBuf sc(ctx, sizeof(double) * (256 * 16 + 8));
  b2k::launch_multidot(1, s0.data.as<double>(), s0.size, s0.data.as<double>(), s0.size,
                       sc.as<double>(), sc.as<double>() + 256 * 16, 1, ctx->stream);
  b2k::launch_scale_inv_sqrt(s0.data.as<double>(), s0.size, sc.as<double>() + 256 * 16, ctx->stream);
  B2_CUDA(cudaGetLastError());
  B2_CUDA(cudaStreamSynchronize(ctx->stream));
  return mps.release();
}
