// Environments (renormalized operators), the two-site effective Hamiltonian and its
// diagonal, expressed as block-GEMM programs for the FP64 kernels (block2 paper: Sec.
// 2.1.2 for the two-site wavefunction, Sec. 2.3 for the MPO / renormalized-operator
// view).
//
// Fermion signs.  Every MPO channel w carries the parity p(w) of its left part.  On a ket
// |l>|s> the product (left part)(site operator) costs (-1)^{p(op) N(l)}; on |s>|r> the
// product (site operator)(right part w') costs (-1)^{p(w') n(s)}.  For the window (i, i+1)
// the operator L_a (x) O1 (x) O2 (x) R_b on |l s1 s2 r> costs
//   (-1)^{p(a) N(l)} * (-1)^{p(O2) n(s1)} * (-1)^{p(b) (n(s1) + n(s2))}
// (the parities of the four factors add up to an even number).
#include "engine.hpp"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <map>

namespace b2 {

using b2k::BufTable;
using b2k::GemmTerm;
using b2k::kTransP;
using b2k::kTransQ;
using b2k::kTwoOp;

static inline int par_n(int n) { return n & 1; }

// --------------------------------------------------------------- GemmProgram
int GemmProgram::add_out(uint8_t buf, int64_t off, int M, int N, int ld, bool accumulate) {
  b2k::GemmOut o;
  o.off = off;
  o.M = M;
  o.N = N;
  o.ld = ld;
  o.t0 = o.t1 = 0;
  o.buf = buf;
  o.accumulate = accumulate ? 1 : 0;
  outs.push_back(o);
  by_out.emplace_back();
  return int(outs.size()) - 1;
}

void GemmProgram::add_term(int out, const GemmTerm& t) {
  by_out[out].push_back(t);
  const auto& o = outs[out];
  if (t.flags & kTwoOp)
    flops += 2.0 * o.M * t.K1 * o.N;
  else
    flops += 2.0 * o.M * t.K1 * t.K2 + 2.0 * o.M * double(t.K2) * o.N;
}

// Work distribution of the FP64 kernel.  The cost of a 32 x 32 tile is the flops its CTA
// performs (operands padded to 32): 2*32*32*K1 for a 2-operand term, 2*32*K1*K2 +
// 2*32*32*K2 for a 3-operand one.  Tiles are split into term ranges of about equal cost
// when the program would otherwise leave SMs idle: the target cost of an item is the total
// over kSplitItems items, at least kMinItemFlops.
namespace {
constexpr double kSplitItems = 4.0 * 152;
constexpr double kMinItemFlops = 1.0e5;
inline int pad32(int x) { return (x + 31) & ~31; }
double term_tile_flops(const GemmTerm& t) {
  if (t.flags & kTwoOp) return 2.0 * 32 * 32 * pad32(t.K1);
  return 2.0 * 32 * pad32(t.K1) * pad32(t.K2) + 2.0 * 32 * 32 * pad32(t.K2);
}
}  // namespace

void GemmProgram::finalize(Ctx* c) {
  terms.clear();
  tasks.clear();
  reds.clear();
  std::vector<double> tcost;   // per term
  double total = 0;
  for (size_t i = 0; i < outs.size(); ++i) {
    auto& o = outs[i];
    o.t0 = int(terms.size());
    terms.insert(terms.end(), by_out[i].begin(), by_out[i].end());
    o.t1 = int(terms.size());
    double per_tile = 0;
    for (const auto& t : by_out[i]) {
      tcost.push_back(term_tile_flops(t));
      per_tile += tcost.back();
    }
    if (o.M > 0 && o.N > 0 && !(o.accumulate && o.t0 == o.t1))
      total += per_tile * double((o.M + 31) / 32) * double((o.N + 31) / 32);
  }
  const double target = std::max(total / kSplitItems, kMinItemFlops);
  int slots = 0;
  for (size_t i = 0; i < outs.size(); ++i) {
    const auto& o = outs[i];
    if (o.M == 0 || o.N == 0) continue;
    if (o.accumulate && o.t0 == o.t1) continue;
    // term ranges of about equal cost (the same for every tile of this output)
    std::vector<std::pair<int, int>> ranges;
    double per_tile = 0;
    for (int t = o.t0; t < o.t1; ++t) per_tile += tcost[t];
    const int n_split = std::max(1, std::min(o.t1 - o.t0, int(std::ceil(per_tile / target))));
    if (n_split == 1) {
      ranges.push_back({o.t0, o.t1});
    } else {
      const double chunk = per_tile / n_split;
      double accum = 0;
      int start = o.t0;
      for (int t = o.t0; t < o.t1; ++t) {
        accum += tcost[t];
        if (accum >= chunk * double(ranges.size() + 1) && int(ranges.size()) + 1 < n_split) {
          ranges.push_back({start, t + 1});
          start = t + 1;
        }
      }
      ranges.push_back({start, o.t1});
    }
    for (int r = 0; r < o.M; r += b2k::kTile)
      for (int cc = 0; cc < o.N; cc += b2k::kTile) {
        if (ranges.size() == 1) {
          tasks.push_back({int(i), r, cc, ranges[0].first, ranges[0].second, -1});
        } else {
          reds.push_back({int(i), r, cc, slots, int(ranges.size())});
          for (const auto& rg : ranges) tasks.push_back({int(i), r, cc, rg.first, rg.second, slots++});
        }
      }
  }
  // most expensive items first (they are dispatched first)
  std::vector<double> cost(tasks.size());
  for (size_t k = 0; k < tasks.size(); ++k) {
    double x = 0;
    for (int t = tasks[k].t0; t < tasks[k].t1; ++t) x += tcost[t];
    cost[k] = x;
  }
  std::vector<int> order(tasks.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = int(k);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<b2k::GemmTask> sorted(tasks.size());
  for (size_t k = 0; k < order.size(); ++k) sorted[k] = tasks[order[k]];
  tasks.swap(sorted);
  B2_REQUIRE(terms.size() < (1u << 31), B2_EUNSUPPORTED, "too many contraction terms");
  by_out.clear();
  by_out.shrink_to_fit();
  upload(c, d_terms, terms);
  upload(c, d_outs, outs);
  upload(c, d_tasks, tasks);
  upload(c, d_reds, reds);
  if (slots > 0) d_partial.reset(c, sizeof(double) * size_t(slots) * b2k::kTile * b2k::kTile);
}

void GemmProgram::launch(Ctx* c, const BufTable& bt) const {
  b2k::launch_gemm(d_tasks.as<b2k::GemmTask>(), int(tasks.size()), d_reds.as<b2k::GemmReduce>(),
                   int(reds.size()), d_partial.as<double>(), d_outs.as<b2k::GemmOut>(),
                   d_terms.as<GemmTerm>(), bt, c->stream);
  B2_CUDA(cudaGetLastError());
}

void CombProgram::finalize(Ctx* c) {
  tiles.clear();
  for (size_t i = 0; i < outs.size(); ++i)
    for (int64_t e = 0; e < outs[i].n; e += b2k::kCombChunk) tiles.push_back({int(i), e});
  upload(c, d_terms, terms);
  upload(c, d_outs, outs);
  upload(c, d_tiles, tiles);
}

void CombProgram::launch(Ctx* c, const BufTable& bt) const {
  b2k::launch_comb(d_tiles.as<b2k::CombTile>(), int(tiles.size()), d_outs.as<b2k::CombOut>(),
                   d_terms.as<b2k::CombTerm>(), bt, c->stream);
  B2_CUDA(cudaGetLastError());
}

// ------------------------------------------------------------------- layouts
void EnvBond::layout(const Bond& b, const std::vector<QN>& dq) {
  blocks.clear();
  blk.assign(dq.size(), std::vector<int>(b.size(), -1));
  size = 0;
  for (size_t w = 0; w < dq.size(); ++w)
    for (int jk = 0; jk < b.size(); ++jk) {
      int jb = b.find(b.q[jk] + dq[w]);
      if (jb < 0) continue;
      blk[w][jk] = int(blocks.size());
      blocks.push_back({jb, jk, b.m[jb], b.m[jk], size});
      size += int64_t(b.m[jb]) * b.m[jk];
    }
}

void PsiLayout::build(const Bond& bl, const Bond& br, int nsite, bool trivial_first) {
  blocks.clear();
  lookup.assign(size_t(bl.size()) * 16, -1);
  size = 0;
  if (nsite == 1) {
    for (int jl = 0; jl < bl.size(); ++jl)
      for (int s = 0; s < 4; ++s) {
        int jr = br.find(bl.q[jl] + kSiteQ[s]);
        if (jr < 0) continue;
        const int s1 = trivial_first ? 0 : s, s2 = trivial_first ? s : 0;
        lookup[(size_t(jl) * 4 + s1) * 4 + s2] = int(blocks.size());
        blocks.push_back({jl, s1, s2, jr, bl.m[jl], br.m[jr], size});
        size += int64_t(bl.m[jl]) * br.m[jr];
      }
    return;
  }
  for (int jl = 0; jl < bl.size(); ++jl)
    for (int s1 = 0; s1 < 4; ++s1)
      for (int s2 = 0; s2 < 4; ++s2) {
        int jr = br.find(bl.q[jl] + kSiteQ[s1] + kSiteQ[s2]);
        if (jr < 0) continue;
        lookup[(size_t(jl) * 4 + s1) * 4 + s2] = int(blocks.size());
        blocks.push_back({jl, s1, s2, jr, bl.m[jl], br.m[jr], size});
        size += int64_t(bl.m[jl]) * br.m[jr];
      }
}

static int op_parity(const double* m) {
  for (int i = 0; i < 16; ++i)
    if (m[i] != 0) return (kSiteN[i / 4] + kSiteN[i % 4]) & 1;
  return 0;
}

// ----------------------------------------------------- operand precombination
// An operand of a contraction: either one environment channel scaled by coef, or the
// linear combination sum_c coef_c env[c] stored once in the combination buffer.  All
// channels of one operand share their quantum-number shift, hence their block layout.
struct Operand {
  uint8_t buf;                   // 2/3: environment data, 4: combination buffer
  std::vector<int64_t> off;      // per ket sector: block offset, -1 if absent
  std::vector<int> bra;          // per ket sector: bra sector
  double coef = 1.0;
};

struct Combiner {
  CombProgram prog;
  int64_t size = 0;
  std::map<std::vector<std::pair<int, double>>, Operand> cache;

  // env: the environment, buf its data id; list: (channel, coefficient)
  Operand make(const EnvBond& env, uint8_t buf, const std::vector<std::pair<int, double>>& list) {
    Operand op;
    int ref = list[0].first;
    const int nk = int(env.blk[ref].size());
    op.off.assign(nk, -1);
    op.bra.assign(nk, -1);
    if (list.size() == 1) {
      op.buf = buf;
      op.coef = list[0].second;
      for (int jk = 0; jk < nk; ++jk) {
        int b = env.blk[ref][jk];
        if (b < 0) continue;
        op.off[jk] = env.blocks[b].off;
        op.bra[jk] = env.blocks[b].jb;
      }
      return op;
    }
    auto key = list;
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    op.buf = 4;
    for (int jk = 0; jk < nk; ++jk) {
      int b = env.blk[ref][jk];
      if (b < 0) continue;
      const auto& blk = env.blocks[b];
      op.off[jk] = size;
      op.bra[jk] = blk.jb;
      b2k::CombOut o;
      o.off = size;
      o.n = int64_t(blk.mb) * blk.mk;
      o.buf = 4;
      o.t0 = int(prog.terms.size());
      for (auto& cw : list) {
        int bb = env.blk[cw.first][jk];
        B2_REQUIRE(bb >= 0 && env.blocks[bb].jb == blk.jb, B2_EINVAL,
                   "internal: combined channels with different layouts");
        prog.terms.push_back({env.blocks[bb].off, cw.second, buf});
      }
      o.t1 = int(prog.terms.size());
      prog.outs.push_back(o);
      size += o.n;
    }
    cache[key] = op;
    return op;
  }
};

// ------------------------------------------------------------ env updates
static void check_env(const EnvBond& e, const char* what) {
  B2_REQUIRE(e.valid, B2_EINVAL, std::string("environment not available: ") + what);
}

void env_update_left(b2_env_s* env, int k) {
  b2_mpo_s* mpo = env->mpo;
  b2_mps_s* mps = env->mps;
  Ctx* c = env->ctx;
  B2_REQUIRE(k >= 0 && k < mpo->n, B2_EINVAL, "site out of range");
  EnvBond& Lk = env->L[k];
  check_env(Lk, "L_site");
  EnvBond& Lo = env->L[k + 1];
  const Bond& bk = mps->bonds[k];
  const Bond& bk1 = mps->bonds[k + 1];
  const SiteTensor& A = mps->sites[k];
  Lo.layout(bk1, mpo->dq[k + 1]);
  Lo.data.reset(c, size_t(std::max<int64_t>(Lo.size, 1)) * sizeof(double));

  std::map<std::tuple<int, int, int>, std::vector<std::pair<int, double>>> groups;
  for (const auto& e : mpo->W[k])
    for (int sp = 0; sp < 4; ++sp)
      for (int s = 0; s < 4; ++s) {
        double v = e.m[sp * 4 + s];
        if (v != 0) groups[{e.w2, sp, s}].push_back({e.w, v});
      }
  GemmProgram prog;
  std::vector<int> out_of(Lo.blocks.size());
  for (size_t b = 0; b < Lo.blocks.size(); ++b) {
    const auto& blk = Lo.blocks[b];
    out_of[b] = prog.add_out(3, blk.off, blk.mb, blk.mk, blk.mk, false);
  }
  Combiner comb;
  for (auto& g : groups) {
    int w2 = std::get<0>(g.first), sp = std::get<1>(g.first), s = std::get<2>(g.first);
    Operand op = comb.make(Lk, 2, g.second);
    int odd = par_n(kSiteN[sp] + kSiteN[s]);
    for (int jk = 0; jk < bk.size(); ++jk) {
      if (op.off[jk] < 0) continue;
      int jb = op.bra[jk];
      int ab = A.find(jb, sp), ak = A.find(jk, s);
      if (ab < 0 || ak < 0) continue;
      const SiteBlock& Ab = A.blocks[ab];
      const SiteBlock& Ak = A.blocks[ak];
      int ob = Lo.find(w2, Ak.jr);
      B2_REQUIRE(ob >= 0 && Lo.blocks[ob].jb == Ab.jr, B2_EINVAL, "internal: env layout");
      double sign = (odd && par_n(bk.q[jk].n)) ? -1.0 : 1.0;
      GemmTerm t{};
      t.offP = Ab.off; t.bufP = 5; t.ldP = Ab.mr;        // op(P) = A^T  [m_jt' x m_jb]
      t.offX = op.off[jk]; t.bufX = op.buf; t.ldX = bk.m[jk];   // X [m_jb x m_jk]
      t.offQ = Ak.off; t.bufQ = 5; t.ldQ = Ak.mr;        // Q = A  [m_jk x m_jt]
      t.K1 = bk.m[jb];
      t.K2 = bk.m[jk];
      t.flags = kTransP;
      t.alpha = op.coef * sign;
      prog.add_term(out_of[ob], t);
    }
  }
  DevBuf cbuf;
  BufTable bt{};
  bt.p[2] = Lk.data.as<double>();
  bt.p[3] = Lo.data.as<double>();
  bt.p[5] = A.data.as<double>();
  if (comb.size > 0) {
    cbuf.reset(c, size_t(comb.size) * sizeof(double));
    bt.p[4] = cbuf.as<double>();
    comb.prog.finalize(c);
    comb.prog.launch(c, bt);
  }
  prog.finalize(c);
  prog.launch(c, bt);
  Lo.valid = true;
  Lo.version = ++env->version_counter;
}

void env_update_right(b2_env_s* env, int k) {
  b2_mpo_s* mpo = env->mpo;
  b2_mps_s* mps = env->mps;
  Ctx* c = env->ctx;
  B2_REQUIRE(k >= 0 && k < mpo->n, B2_EINVAL, "site out of range");
  EnvBond& Rk1 = env->R[k + 1];
  check_env(Rk1, "R_{site+1}");
  EnvBond& Ro = env->R[k];
  const Bond& bk = mps->bonds[k];
  const Bond& bk1 = mps->bonds[k + 1];
  const SiteTensor& B = mps->sites[k];
  Ro.layout(bk, mpo->dq[k]);
  Ro.data.reset(c, size_t(std::max<int64_t>(Ro.size, 1)) * sizeof(double));
  // site blocks by (jr, s)
  std::vector<int> rev(size_t(bk1.size()) * 4, -1);
  for (size_t b = 0; b < B.blocks.size(); ++b) rev[size_t(B.blocks[b].jr) * 4 + B.blocks[b].s] = int(b);

  std::map<std::tuple<int, int, int>, std::vector<std::pair<int, double>>> groups;
  for (const auto& e : mpo->W[k])
    for (int sp = 0; sp < 4; ++sp)
      for (int s = 0; s < 4; ++s) {
        double v = e.m[sp * 4 + s];
        if (v != 0) groups[{e.w, sp, s}].push_back({e.w2, v});
      }
  GemmProgram prog;
  std::vector<int> out_of(Ro.blocks.size());
  for (size_t b = 0; b < Ro.blocks.size(); ++b) {
    const auto& blk = Ro.blocks[b];
    out_of[b] = prog.add_out(3, blk.off, blk.mb, blk.mk, blk.mk, false);
  }
  Combiner comb;
  for (auto& g : groups) {
    int w = std::get<0>(g.first), sp = std::get<1>(g.first), s = std::get<2>(g.first);
    Operand op = comb.make(Rk1, 2, g.second);
    int pw2 = mpo->parity[k + 1][g.second[0].first];
    double sign = (pw2 && par_n(kSiteN[s])) ? -1.0 : 1.0;
    for (int jrk = 0; jrk < bk1.size(); ++jrk) {
      if (op.off[jrk] < 0) continue;
      int jrb = op.bra[jrk];
      int bb = rev[size_t(jrb) * 4 + sp], bkk = rev[size_t(jrk) * 4 + s];
      if (bb < 0 || bkk < 0) continue;
      const SiteBlock& Bb = B.blocks[bb];
      const SiteBlock& Bk = B.blocks[bkk];
      int ob = Ro.find(w, Bk.jl);
      B2_REQUIRE(ob >= 0 && Ro.blocks[ob].jb == Bb.jl, B2_EINVAL, "internal: env layout");
      GemmTerm t{};
      t.offP = Bb.off; t.bufP = 5; t.ldP = Bb.mr;            // P = B [m_j' x m_jr']
      t.offX = op.off[jrk]; t.bufX = op.buf; t.ldX = bk1.m[jrk];   // X [m_jr' x m_jr]
      t.offQ = Bk.off; t.bufQ = 5; t.ldQ = Bk.mr;            // op(Q) = B^T [m_jr x m_j]
      t.K1 = bk1.m[jrb];
      t.K2 = bk1.m[jrk];
      t.flags = kTransQ;
      t.alpha = op.coef * sign;
      prog.add_term(out_of[ob], t);
    }
  }
  DevBuf cbuf;
  BufTable bt{};
  bt.p[2] = Rk1.data.as<double>();
  bt.p[3] = Ro.data.as<double>();
  bt.p[5] = B.data.as<double>();
  if (comb.size > 0) {
    cbuf.reset(c, size_t(comb.size) * sizeof(double));
    bt.p[4] = cbuf.as<double>();
    comb.prog.finalize(c);
    comb.prog.launch(c, bt);
  }
  prog.finalize(c);
  prog.launch(c, bt);
  Ro.valid = true;
  Ro.version = ++env->version_counter;
}

// ------------------------------------------------------------- window program
namespace {
struct Edge {
  int a, b;
  double v;
};
}  // namespace

static void build_window(b2_env_s* env, int win, WindowProgram& wp) {
  b2_mpo_s* mpo = env->mpo;
  b2_mps_s* mps = env->mps;
  Ctx* c = env->ctx;
  const int i = win_site(win), ns = win_nsite(win);
  const EnvBond& L = env->L[i];
  const EnvBond& R = env->R[i + ns];
  const Bond& bl = mps->bonds[i];
  const Bond& br = mps->bonds[i + ns];
  wp = WindowProgram();
  wp.win = win;
  wp.site = i;
  wp.nsite = ns;
  wp.ver_l = L.version;
  wp.ver_r = R.version;
  wp.psi.build(bl, br, ns);

  // Two-site operator entries grouped by local pattern (u, v), u = 4 s1' + s2',
  // v = 4 s1 + s2: sum over w' of W_i[a,w']_{s1's1} W_{i+1}[w',b]_{s2's2}, with the sign of
  // moving the site-(i+1) operator past s1 and the right part past s1 s2 folded in.  Flat
  // edge lists per pattern; duplicates (several w' joining the same a, b) are merged after
  // a stable sort, so they are summed in generation order.
  // One-site window: W_i[a,b]_{s's} alone with the sign of moving the right part past s,
  // at patterns (4 s', 4 s) (the trivial second site in state 0).
  std::vector<std::vector<Edge>> pat(256);
  if (ns == 1)
    for (const auto& e1 : mpo->W[i]) {
      const int pb = mpo->parity[i + 1][e1.w2];
      for (int a1 = 0; a1 < 16; ++a1) {
        if (e1.m[a1] == 0) continue;
        const int s1p = a1 / 4, s1 = a1 % 4;
        const double sign = (pb && par_n(kSiteN[s1])) ? -1.0 : 1.0;
        pat[(s1p * 4) * 16 + s1 * 4].push_back({e1.w, e1.w2, sign * e1.m[a1]});
      }
    }
  std::vector<std::vector<int>> byw(ns == 2 ? mpo->D[i + 1] : 0);
  if (ns == 2)
    for (size_t e = 0; e < mpo->W[i + 1].size(); ++e) byw[mpo->W[i + 1][e].w].push_back(int(e));
  static const std::vector<b2_mpo_s::Entry> kNoEntries;
  for (const auto& e1 : ns == 2 ? mpo->W[i] : kNoEntries) {
    int nz1[16], n1 = 0;
    for (int a1 = 0; a1 < 16; ++a1)
      if (e1.m[a1] != 0) nz1[n1++] = a1;
    for (int e2i : byw[e1.w2]) {
      const auto& e2 = mpo->W[i + 1][e2i];
      const int p2 = op_parity(e2.m);
      const int pb = mpo->parity[i + ns][e2.w2];
      for (int k1 = 0; k1 < n1; ++k1) {
        const int a1 = nz1[k1];
        const double x1 = e1.m[a1];
        const int s1p = a1 / 4, s1 = a1 % 4;
        for (int a2 = 0; a2 < 16; ++a2) {
          const double x2 = e2.m[a2];
          if (x2 == 0) continue;
          const int s2p = a2 / 4, s2 = a2 % 4;
          double sign = 1.0;
          if (p2 && par_n(kSiteN[s1])) sign = -sign;
          if (pb && par_n(kSiteN[s1] + kSiteN[s2])) sign = -sign;
          pat[(s1p * 4 + s2p) * 16 + s1 * 4 + s2].push_back({e1.w, e2.w2, sign * x1 * x2});
        }
      }
    }
  }
  for (auto& edges : pat) {
    std::stable_sort(edges.begin(), edges.end(), [](const Edge& x, const Edge& y) {
      return x.a != y.a ? x.a < y.a : x.b < y.b;
    });
    size_t w = 0;
    for (size_t r = 0; r < edges.size();) {
      Edge m = edges[r];
      size_t q = r + 1;
      while (q < edges.size() && edges[q].a == m.a && edges[q].b == m.b) m.v += edges[q++].v;
      if (m.v != 0) edges[w++] = m;
      r = q;
    }
    edges.resize(w);
  }

  // outputs: every psi block, overwritten
  GemmProgram& prog = wp.heff;
  for (const auto& pb : wp.psi.blocks) prog.add_out(1, pb.off, pb.ml, pb.mr, pb.mr, false);
  Combiner combL, combR;   // separate so the two combination regions can be concatenated
  struct Pending {
    Operand lop, rop;
    int u, v;
    int pL;
    double coef;
    bool block_h = false;
  };
  std::vector<Pending> pending;
  const int Da = mpo->D[i], Db = mpo->D[i + ns];
  // The two block-Hamiltonian terms, L_H (x) 1 (x) R_H (left block's Hamiltonian, right
  // block's identity) and L_I (x) 1 (x) R_I (the reverse), carry the energy scale of H_eff;
  // they are kept out of the precombination as terms of their own (flag kBlockH) so that the
  // split-precision path can evaluate them in FP64 (normal-ordering idea of Sec. 2.1.5: the
  // low-precision products then carry only the coupling between the blocks and the sites).
  std::vector<std::vector<Edge>> block_h_edges(16);   // kept for the diagonal
  for (int v = 0; v < 16; ++v) {
    auto& edges = pat[v * 16 + v];
    for (int which = 0; which < 2; ++which) {
      const int a = which ? mpo->chan_H[i] : mpo->chan_I[i];
      const int b = which ? mpo->chan_H[i + ns] : mpo->chan_I[i + ns];
      if (a < 0 || b < 0) continue;
      for (size_t k = 0; k < edges.size(); ++k)
        if (edges[k].a == a && edges[k].b == b) {
          Pending p;
          p.u = p.v = v;
          p.lop = combL.make(L, 2, {{a, edges[k].v}});
          p.rop = combR.make(R, 3, {{b, 1.0}});
          p.pL = mpo->parity[i][a];
          p.coef = p.lop.coef * p.rop.coef;
          p.block_h = true;
          pending.push_back(std::move(p));
          block_h_edges[v].push_back(edges[k]);
          edges.erase(edges.begin() + k);
          break;
        }
    }
  }
  std::vector<int> dega(Da, 0), degb(Db, 0), posa(Da, -1), posb(Db, -1);
  for (int pv = 0; pv < 256; ++pv) {
    auto& edges = pat[pv];
    if (edges.empty()) continue;
    const int u = pv / 16, v = pv % 16;
    // greedy vertex cover: highest degree first; each chosen vertex takes its remaining
    // edges as one group (the other side is precombined)
    std::vector<int> ta, tb;
    for (auto& e : edges) {
      if (dega[e.a]++ == 0) ta.push_back(e.a);
      if (degb[e.b]++ == 0) tb.push_back(e.b);
    }
    // incidence: edges are sorted by a; by_b holds edge indices sorted by (b, a)
    for (size_t k = 0; k < edges.size(); ++k)
      if (posa[edges[k].a] < 0) posa[edges[k].a] = int(k);
    std::vector<int> by_b(edges.size());
    for (size_t k = 0; k < edges.size(); ++k) by_b[k] = int(k);
    std::stable_sort(by_b.begin(), by_b.end(), [&](int x, int y) { return edges[x].b < edges[y].b; });
    for (size_t k = 0; k < by_b.size(); ++k)
      if (posb[edges[by_b[k]].b] < 0) posb[edges[by_b[k]].b] = int(k);
    struct Vert {
      int deg, side, id;
    };
    std::vector<Vert> verts;
    verts.reserve(ta.size() + tb.size());
    for (int x : ta) verts.push_back({dega[x], 0, x});
    for (int x : tb) verts.push_back({degb[x], 1, x});
    std::sort(verts.begin(), verts.end(), [](const Vert& x, const Vert& y) {
      if (x.deg != y.deg) return x.deg > y.deg;
      if (x.side != y.side) return x.side < y.side;
      return x.id < y.id;
    });
    std::vector<char> used(edges.size(), 0);
    for (auto& vt : verts) {
      std::vector<std::pair<int, double>> others;
      if (vt.side == 0) {
        for (int k = posa[vt.id]; k < int(edges.size()) && edges[k].a == vt.id; ++k)
          if (!used[k]) {
            used[k] = 1;
            others.push_back({edges[k].b, edges[k].v});
          }
      } else {
        for (int k = posb[vt.id]; k < int(by_b.size()) && edges[by_b[k]].b == vt.id; ++k)
          if (!used[by_b[k]]) {
            used[by_b[k]] = 1;
            others.push_back({edges[by_b[k]].a, edges[by_b[k]].v});
          }
      }
      if (others.empty()) continue;
      Pending p;
      p.u = u;
      p.v = v;
      if (vt.side == 0) {
        p.lop = combL.make(L, 2, {{vt.id, 1.0}});
        p.rop = combR.make(R, 3, others);
        p.pL = mpo->parity[i][vt.id];
      } else {
        p.lop = combL.make(L, 2, others);
        p.rop = combR.make(R, 3, {{vt.id, 1.0}});
        p.pL = mpo->parity[i][others[0].first];
      }
      p.coef = p.lop.coef * p.rop.coef;
      pending.push_back(std::move(p));
    }
    for (int x : ta) dega[x] = 0, posa[x] = -1;
    for (int x : tb) degb[x] = 0, posb[x] = -1;
  }
  // the R combinations live after the L ones in the same buffer
  int64_t shiftR = combL.size;
  for (auto& o : combR.prog.outs) o.off += shiftR;
  CombProgram& cp = wp.comb;
  cp.outs = combL.prog.outs;
  cp.terms = combL.prog.terms;
  int tbase = int(cp.terms.size());
  for (auto o : combR.prog.outs) {
    o.t0 += tbase;
    o.t1 += tbase;
    cp.outs.push_back(o);
  }
  cp.terms.insert(cp.terms.end(), combR.prog.terms.begin(), combR.prog.terms.end());
  for (auto& p : pending) {
    if (p.rop.buf == 4)
      for (auto& x : p.rop.off)
        if (x >= 0) x += shiftR;
    int s1p = p.u / 4, s2p = p.u % 4, s1 = p.v / 4, s2 = p.v % 4;
    for (int jl = 0; jl < bl.size(); ++jl) {
      int ib = wp.psi.find(jl, s1, s2);
      if (ib < 0) continue;
      const PsiBlock& in = wp.psi.blocks[ib];
      if (p.lop.off[jl] < 0 || p.rop.off[in.jr] < 0) continue;
      int jlp = p.lop.bra[jl], jrp = p.rop.bra[in.jr];
      int ob = wp.psi.find(jlp, s1p, s2p);
      if (ob < 0 || wp.psi.blocks[ob].jr != jrp) continue;
      double sign = (p.pL && par_n(bl.q[jl].n)) ? -1.0 : 1.0;
      GemmTerm t{};
      t.offP = p.lop.off[jl]; t.bufP = p.lop.buf; t.ldP = in.ml;      // L [m_l' x m_l]
      t.offX = in.off; t.bufX = 0; t.ldX = in.mr;                       // psi [m_l x m_r]
      t.offQ = p.rop.off[in.jr]; t.bufQ = p.rop.buf; t.ldQ = in.mr;    // R [m_r' x m_r]
      t.K1 = in.ml;
      t.K2 = in.mr;
      t.flags = kTransQ | (p.block_h ? b2k::kBlockH : uint8_t(0));
      t.alpha = p.coef * sign;
      prog.add_term(ob, t);
    }
  }
  if (std::getenv("B2_TRACE_WINDOW")) {
    // structure of the contraction: term shapes (rows m_l', K1 = m_l, K2 = m_r, cols m_r')
    // weighted by their flops, and the 128-row / 64-wide padding of the tensor-core tiles
    double fl = 0, fl_pad = 0, n_terms = 0;
    std::map<int, double> by_rows;   // flops by rows of the output block (bucketed)
    for (size_t o = 0; o < prog.outs.size(); ++o) {
      const auto& out = prog.outs[o];
      for (const auto& t : prog.by_out[o]) {
        const double f = 2.0 * out.M * t.K1 * t.K2 + 2.0 * out.M * double(t.K2) * out.N;
        fl += f;
        n_terms += 1;
        const double mp = 128.0 * ((out.M + 127) / 128), k1 = 16.0 * ((t.K1 + 15) / 16),
                     k2 = 16.0 * ((t.K2 + 15) / 16), np_ = 16.0 * ((out.N + 15) / 16);
        fl_pad += 2.0 * mp * k1 * k2 + 2.0 * mp * k2 * np_;
        by_rows[out.M <= 16 ? 16 : out.M <= 32 ? 32 : out.M <= 64 ? 64 : out.M <= 128 ? 128 : 256] += f;
      }
    }
    std::fprintf(stderr, "window %d: outs %zu terms %.0f flops %.4g padded128 %.4g L %lld R %lld comb %lld psi %lld\n",
                 i, prog.outs.size(), n_terms, fl, fl_pad, (long long)L.size, (long long)R.size,
                 (long long)(combL.size + combR.size), (long long)wp.psi.size);
    for (auto& kv : by_rows) std::fprintf(stderr, "  rows<=%d: %.3f of flops\n", kv.first, kv.second / fl);
  }
  prog.finalize(c);
  int64_t comb_size = combL.size + combR.size;
  if (comb_size > 0) {
    wp.comb_buf.reset(c, size_t(comb_size) * sizeof(double));
    cp.finalize(c);
  }

  // diagonal: diagonal patterns whose channels keep the sector (dq = 0 on both sides)
  std::vector<std::vector<Edge>> dedges(16);
  for (int v = 0; v < 16; ++v)
    for (const auto& e : block_h_edges[v]) dedges[v].push_back(e);
  for (int v = 0; v < 16; ++v)
    for (const auto& e : pat[v * 16 + v])
      if (mpo->dq[i][e.a] == QN{0, 0} && mpo->dq[i + ns][e.b] == QN{0, 0}) dedges[v].push_back(e);
  {
    // channel rows of the diagonal buffers
    std::vector<int> ka(Da, -1), kb(Db, -1);
    int KA = 0, KB = 0;
    for (int v = 0; v < 16; ++v)
      for (const auto& e : dedges[v]) {
        B2_REQUIRE(mpo->parity[i][e.a] == 0 && mpo->parity[i + ns][e.b] == 0, B2_EINVAL,
                   "internal: odd channel on the diagonal");
        if (ka[e.a] < 0) ka[e.a] = KA++;
        if (kb[e.b] < 0) kb[e.b] = KB++;
      }
    const int64_t SL = bl.total, SR = br.total;
    const int64_t offDR = int64_t(KA) * SL, offS = offDR + int64_t(KB) * SR;
    wp.dg_size = offS + int64_t(16) * KA * SR;
    // diagonals of the blocks (dst row = channel, columns = the bond's states)
    for (int a = 0; a < Da; ++a) {
      if (ka[a] < 0) continue;
      for (int j = 0; j < bl.size(); ++j) {
        const int b = L.blk[a][j];
        if (b < 0) continue;
        B2_REQUIRE(L.blocks[b].jb == j, B2_EINVAL, "internal: diagonal block");
        wp.dg_copy.push_back({L.blocks[b].off, int64_t(ka[a]) * SL + bl.off[j], bl.m[j], 1,
                              bl.m[j] + 1, 1, 0, 2, 5});
      }
    }
    for (int b = 0; b < Db; ++b) {
      if (kb[b] < 0) continue;
      for (int j = 0; j < br.size(); ++j) {
        const int rb = R.blk[b][j];
        if (rb < 0) continue;
        B2_REQUIRE(R.blocks[rb].jb == j, B2_EINVAL, "internal: diagonal block");
        wp.dg_copy.push_back({R.blocks[rb].off, offDR + int64_t(kb[b]) * SR + br.off[j], br.m[j], 1,
                              br.m[j] + 1, 1, 0, 3, 5});
      }
    }
    // S rows: per pattern v and left channel a, sum over its edges of c * dR_b
    std::vector<int> order;
    for (int v = 0; v < 16; ++v) {
      auto& ed = dedges[v];
      order.resize(ed.size());
      for (size_t k = 0; k < ed.size(); ++k) order[k] = int(k);
      std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ed[x].a < ed[y].a; });
      for (size_t k = 0; k < order.size();) {
        const int a = ed[order[k]].a;
        b2k::CombOut co;
        co.off = offS + (int64_t(v) * KA + ka[a]) * SR;
        co.n = SR;
        co.buf = 5;
        co.t0 = int(wp.dg_comb.terms.size());
        for (; k < order.size() && ed[order[k]].a == a; ++k) {
          const Edge& e = ed[order[k]];
          wp.dg_comb.terms.push_back({offDR + int64_t(kb[e.b]) * SR, e.v, 5});
        }
        co.t1 = int(wp.dg_comb.terms.size());
        wp.dg_comb.outs.push_back(co);
      }
    }
    // one product per psi block: diag[l][r] = sum_k dL[k][l] S_v[k][r]
    for (const auto& pb : wp.psi.blocks) {
      const int v = pb.s1 * 4 + pb.s2;
      const int o = wp.dg_gemm.add_out(1, pb.off, pb.ml, pb.mr, pb.mr, false);
      if (dedges[v].empty() || KA == 0) continue;
      GemmTerm t{};
      t.offP = bl.off[pb.jl]; t.bufP = 5; t.ldP = int(SL);
      t.offX = offS + int64_t(v) * KA * SR + br.off[pb.jr]; t.bufX = 5; t.ldX = int(SR);
      t.K1 = KA;
      t.flags = kTwoOp | kTransP;
      t.alpha = 1.0;
      wp.dg_gemm.add_term(o, t);
    }
    upload(c, wp.d_dg_copy, wp.dg_copy);
    if (!wp.dg_comb.outs.empty()) wp.dg_comb.finalize(c);
    wp.dg_gemm.finalize(c);
  }
  wp.comb_done = false;
}

WindowProgram& window_program(b2_env_s* env, int win) {
  B2_REQUIRE(win >= 0 && (win & ~(kOneSite | (kOneSite - 1))) == 0, B2_EINVAL, "bad window id");
  const int site = win_site(win), ns = win_nsite(win);
  B2_REQUIRE(site + ns <= env->mpo->n, B2_EINVAL, "window site out of range");
  check_env(env->L[site], "L_site");
  check_env(env->R[site + ns], ns == 2 ? "R_{site+2}" : "R_{site+1}");
  auto& slot = env->windows[win];
  if (!slot) slot.reset(new WindowProgram());
  WindowProgram& wp = *slot;
  if (wp.win != win || wp.ver_l != env->L[site].version || wp.ver_r != env->R[site + ns].version)
    build_window(env, win, wp);
  return wp;
}

// ----------------------------------------------------- split-precision program
namespace {
inline int pad16(int x) { return (x + 15) & ~15; }
inline int elem_bytes(b2_prec p) { return p == B2_TF32X3 ? 4 : 2; }

// Host tables of the tensor-core form of the window's contraction (see TcProgram): the
// block-Hamiltonian terms go to an FP64 program that overwrites every output, the others
// to the tensor-core tables, whose outputs then accumulate.
void build_tc(Ctx* c, WindowProgram& wp) {
  TcProgram& tp = wp.tc;
  const GemmProgram& g = wp.heff;
  for (const auto& o : g.outs) tp.block_h.add_out(o.buf, o.off, o.M, o.N, o.ld, false);
  std::map<std::pair<int, int64_t>, int64_t> env_dst;
  auto env_operand = [&](int buf, int64_t off, int rows, int cols, int ld) -> int64_t {
    B2_REQUIRE(ld == cols, B2_EINVAL, "internal: operand block not contiguous");
    auto key = std::make_pair(buf, off);
    auto it = env_dst.find(key);
    if (it != env_dst.end()) return it->second;
    const int rp = pad16(rows), kp = pad16(cols);
    const int64_t dst = tp.env_elems;
    tp.env_elems += int64_t(rp) * kp;
    tp.env_tasks.push_back({off, dst, rows, cols, ld, 0, rp, kp, buf});
    env_dst[key] = dst;
    return dst;
  };
  // psi^T blocks: rows m_r, contraction index m_l
  std::map<int64_t, int64_t> psi_dst;
  for (const auto& pb : wp.psi.blocks) {
    const int rp = pad16(pb.mr), kp = pad16(pb.ml);
    psi_dst[pb.off] = tp.psi_elems;
    tp.psi_tasks.push_back({pb.off, tp.psi_elems, pb.mr, pb.ml, pb.mr, 1, rp, kp, 0});
    tp.psi_elems += int64_t(rp) * kp;
  }
  std::vector<double> cost;
  for (size_t i = 0; i < g.outs.size(); ++i) {
    const b2k::GemmOut& o = g.outs[i];
    b2k::TcOut to{};
    to.off = o.off;
    to.M = o.M;
    to.N = o.N;
    to.accumulate = 1;
    to.t0 = int(tp.terms.size());
    double cst = 0;
    for (int t = o.t0; t < o.t1; ++t) {
      const GemmTerm& gt = g.terms[t];
      B2_REQUIRE((gt.flags & ~b2k::kBlockH) == kTransQ && gt.bufX == 0 && !o.accumulate,
                 B2_EINVAL, "internal: H_eff term form");
      if (gt.flags & b2k::kBlockH) {
        tp.block_h.add_term(int(i), gt);
        continue;
      }
      auto ip = psi_dst.find(gt.offX);
      B2_REQUIRE(ip != psi_dst.end(), B2_EINVAL, "internal: psi block of a term");
      b2k::TcTerm tt{};
      tt.offA = env_operand(gt.bufP, gt.offP, o.M, gt.K1, gt.ldP);
      tt.offB1 = ip->second;
      tt.offB2 = env_operand(gt.bufQ, gt.offQ, o.N, gt.K2, gt.ldQ);
      B2_REQUIRE(gt.K1 < 65536 && gt.K2 < 65536, B2_EUNSUPPORTED, "sector dimension above 65535");
      tt.K1 = uint16_t(gt.K1);
      tt.K2 = uint16_t(gt.K2);
      tt.alpha = static_cast<float>(gt.alpha);
      tp.terms.push_back(tt);
      cst += double(pad16(gt.K2)) * (pad16(gt.K1) + pad16(std::min(o.N, b2k::kTcTileN)));
    }
    to.t1 = int(tp.terms.size());
    tp.outs.push_back(to);
    if (to.t1 == to.t0) continue;   // nothing to add to the block-Hamiltonian part
    for (int r = 0; r < o.M; r += b2k::kTcTileM)
      for (int cc = 0; cc < o.N; cc += b2k::kTcTileN) {
        tp.tiles.push_back({int(i), r, cc});
        cost.push_back(cst);
      }
  }
  tp.block_h.finalize(c);
  // most expensive tiles first
  std::vector<int> order(tp.tiles.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = int(k);
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  std::vector<b2k::TcTile> sorted(tp.tiles.size());
  for (size_t k = 0; k < order.size(); ++k) sorted[k] = tp.tiles[order[k]];
  tp.tiles.swap(sorted);
  B2_REQUIRE(tp.terms.size() < (1u << 31), B2_EUNSUPPORTED, "too many contraction terms");
  tp.built = true;
}

BufTable window_buffers(b2_env_s* env, WindowProgram& wp, const double* psi, double* out) {
  BufTable bt{};
  bt.p[0] = const_cast<double*>(psi);
  bt.p[1] = out;
  bt.p[2] = env->L[wp.site].data.as<double>();
  bt.p[3] = env->R[wp.site + wp.nsite].data.as<double>();
  bt.p[4] = wp.comb_buf.as<double>();
  return bt;
}

// precombined operators of the window, once
void ensure_comb(Ctx* c, WindowProgram& wp, const BufTable& bt) {
  if (!wp.comb_done) {
    if (wp.comb_buf.ptr) wp.comb.launch(c, bt);
    wp.comb_done = true;
  }
}

// split psi (once per product) into the psi planes of the window's tensor-core program
void split_psi(Ctx* c, TcProgram& tp, const double* psi, b2_prec prec) {
  const size_t plane = size_t(std::max<int64_t>(tp.psi_elems, 1)) * elem_bytes(prec);
  if (tp.psi_planes.bytes < 2 * plane) tp.psi_planes.reset(c, 2 * plane);
  BufTable bt{};
  bt.p[0] = const_cast<double*>(psi);
  uint8_t* hi = tp.psi_planes.as<uint8_t>();
  b2k::launch_split(tp.d_psi_tasks.as<b2k::SplitTask>(), int(tp.psi_tasks.size()), bt, hi,
                    hi + plane, prec == B2_TF32X3, c->stream);
  B2_CUDA(cudaGetLastError());
}

b2k::TcGroup tc_group(TcProgram& tp, b2_prec prec, double* out) {
  const size_t eplane = size_t(std::max<int64_t>(tp.env_elems, 1)) * elem_bytes(prec);
  const size_t pplane = size_t(std::max<int64_t>(tp.psi_elems, 1)) * elem_bytes(prec);
  b2k::TcGroup g{};
  g.tiles = tp.d_tiles.as<b2k::TcTile>();
  g.outs = tp.d_outs.as<b2k::TcOut>();
  g.terms = tp.d_terms.as<b2k::TcTerm>();
  g.env_hi = tp.env_planes.as<uint8_t>();
  g.env_lo = g.env_hi + eplane;
  g.psi_hi = tp.psi_planes.as<uint8_t>();
  g.psi_lo = g.psi_hi + pplane;
  g.out = out;
  g.tile0 = 0;
  return g;
}
}  // namespace

TcProgram& tc_program(b2_env_s* env, int site, b2_prec prec) {
  B2_REQUIRE(prec == B2_BF16X3 || prec == B2_TF32X3, B2_EUNSUPPORTED, "precision not implemented");
  WindowProgram& wp = window_program(env, site);
  Ctx* c = env->ctx;
  TcProgram& tp = wp.tc;
  if (!tp.built) {
    build_tc(c, wp);
    upload(c, tp.d_outs, tp.outs);
    upload(c, tp.d_terms, tp.terms);
    upload(c, tp.d_tiles, tp.tiles);
    upload(c, tp.d_env_tasks, tp.env_tasks);
    upload(c, tp.d_psi_tasks, tp.psi_tasks);
  }
  if (tp.env_prec != int(prec)) {
    BufTable bt = window_buffers(env, wp, nullptr, nullptr);
    ensure_comb(c, wp, bt);
    const size_t plane = size_t(std::max<int64_t>(tp.env_elems, 1)) * elem_bytes(prec);
    tp.env_planes.reset(c, 2 * plane);
    uint8_t* hi = tp.env_planes.as<uint8_t>();
    b2k::launch_split(tp.d_env_tasks.as<b2k::SplitTask>(), int(tp.env_tasks.size()), bt, hi,
                      hi + plane, prec == B2_TF32X3, c->stream);
    B2_CUDA(cudaGetLastError());
    tp.env_prec = int(prec);
  }
  return tp;
}

void heff_apply(b2_env_s* env, int site, const double* psi, double* out, double e_shift,
                double* flops, b2_prec prec) {
  WindowProgram& wp = window_program(env, site);
  Ctx* c = env->ctx;
  BufTable bt = window_buffers(env, wp, psi, out);
  ensure_comb(c, wp, bt);
  TcProgram* tp = prec == B2_FP64 ? nullptr : &tc_program(env, site, prec);
  if (tp) split_psi(c, *tp, psi, prec);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->prof) {
    B2_CUDA(cudaEventCreate(&e0));
    B2_CUDA(cudaEventCreate(&e1));
    B2_CUDA(cudaEventRecord(e0, c->stream));
  }
  if (!tp) {
    wp.heff.launch(c, bt);
  } else {
    tp->block_h.launch(c, bt);   // FP64 block-Hamiltonian terms write the output
    b2k::launch_heff_tc(tc_group(*tp, prec, out), nullptr, 1, int(tp->tiles.size()),
                        prec == B2_TF32X3, c->status(), c->stuck_polls, c->stream);
    B2_CUDA(cudaGetLastError());
  }
  if (e0) {
    B2_CUDA(cudaEventRecord(e1, c->stream));
    c->prof_events.push_back({e0, e1});
    c->prof_flops += wp.heff.flops;
  }
  if (e_shift != 0.0) b2k::launch_axpby(out, psi, wp.psi.size, 1.0, -e_shift, c->stream);
  if (flops) *flops = wp.heff.flops;
}

void heff_apply_batched(Ctx* c, int n, b2_env_s* const* envs, const int* sites,
                        const double* const* psis, double* const* outs, b2_prec prec,
                        double* flops) {
  std::vector<b2k::GemmGroup> groups;
  std::vector<b2k::TcGroup> groups_tc;
  int items = 0, reds = 0, tiles = 0;
  double fl = 0;
  for (int i = 0; i < n; ++i) {
    b2_env_s* env = envs[i];
    B2_REQUIRE(env->ctx == c, B2_EINVAL, "batched H_eff: env of another context");
    for (int j = 0; j < i; ++j)
      B2_REQUIRE(envs[j] != env, B2_EINVAL, "batched H_eff: the same env twice");
    const int site = sites[i];
    WindowProgram& wp = window_program(env, site);
    B2_REQUIRE(psis[i] != outs[i], B2_EINVAL, "batched H_eff: out aliases psi");
    BufTable bt = window_buffers(env, wp, psis[i], outs[i]);
    ensure_comb(c, wp, bt);
    if (prec == B2_FP64) {
      groups.push_back({wp.heff.d_tasks.as<b2k::GemmTask>(), wp.heff.d_reds.as<b2k::GemmReduce>(),
                        wp.heff.d_outs.as<b2k::GemmOut>(), wp.heff.d_terms.as<GemmTerm>(),
                        wp.heff.d_partial.as<double>(), bt, items, reds});
      items += int(wp.heff.tasks.size());
      reds += int(wp.heff.reds.size());
    } else {
      TcProgram& tp = tc_program(env, site, prec);
      split_psi(c, tp, psis[i], prec);
      tp.block_h.launch(c, bt);   // FP64 block-Hamiltonian terms write the output
      b2k::TcGroup g = tc_group(tp, prec, outs[i]);
      g.tile0 = tiles;
      groups_tc.push_back(g);
      tiles += int(tp.tiles.size());
    }
    fl += wp.heff.flops;
  }
  DevBuf d_groups;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (c->prof) {
    B2_CUDA(cudaEventCreate(&e0));
    B2_CUDA(cudaEventCreate(&e1));
  }
  if (prec == B2_FP64) {
    upload(c, d_groups, groups);
    if (e0) B2_CUDA(cudaEventRecord(e0, c->stream));
    b2k::launch_gemm_grouped(d_groups.as<b2k::GemmGroup>(), int(groups.size()), items, reds,
                             c->stream);
  } else {
    upload(c, d_groups, groups_tc);
    if (e0) B2_CUDA(cudaEventRecord(e0, c->stream));
    b2k::launch_heff_tc(b2k::TcGroup{}, d_groups.as<b2k::TcGroup>(), int(groups_tc.size()), tiles,
                        prec == B2_TF32X3, c->status(), c->stuck_polls, c->stream);
  }
  B2_CUDA(cudaGetLastError());
  if (e0) {
    B2_CUDA(cudaEventRecord(e1, c->stream));
    c->prof_events.push_back({e0, e1});
    c->prof_flops += fl;
  }
  if (flops) *flops = fl;
}

void heff_diag(b2_env_s* env, int site, double* diag) {
  WindowProgram& wp = window_program(env, site);
  Ctx* c = env->ctx;
  // the diagonal depends only on the window's environments: computed once per window
  // program, copied out on later calls (the Davidson solver asks for it every solve)
  if (!wp.diag_done) {
    wp.diag.reset(c, sizeof(double) * size_t(std::max<int64_t>(wp.psi.size, 1)));
    DevBuf work(c, sizeof(double) * size_t(std::max<int64_t>(wp.dg_size, 1)));
    B2_CUDA(cudaMemsetAsync(work.ptr, 0, work.bytes, c->stream));
    BufTable bt{};
    bt.p[1] = wp.diag.as<double>();
    bt.p[2] = env->L[wp.site].data.as<double>();
    bt.p[3] = env->R[wp.site + wp.nsite].data.as<double>();
    bt.p[5] = work.as<double>();
    b2k::launch_copy(int(wp.dg_copy.size()), wp.d_dg_copy.as<b2k::CopyTask>(), bt, c->stream);
    if (!wp.dg_comb.outs.empty()) wp.dg_comb.launch(c, bt);
    wp.dg_gemm.launch(c, bt);
    B2_CUDA(cudaGetLastError());
    wp.diag_done = true;
  }
  if (wp.psi.size > 0)
    B2_CUDA(cudaMemcpyAsync(diag, wp.diag.ptr, sizeof(double) * size_t(wp.psi.size),
                            cudaMemcpyDeviceToDevice, c->stream));
}

}  // namespace b2
