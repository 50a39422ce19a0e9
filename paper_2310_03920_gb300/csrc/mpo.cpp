// MPO of the ab initio Hamiltonian (block2 paper, Sec. 2.1.1 for the Hamiltonian,
// Sec. 2.3 for the automatic MPO construction from operator strings and the
// normal/complementary partition with the NC -> CN switch at the middle site).
//
// Every Hamiltonian term is rewritten as a site-ordered string of local operators (the
// product of the elementary a+/a acting on one site, in their original order, with the
// fermionic sign of the reordering).  On bond k a term is carried by one channel:
//   "I"   no operator of the term on sites < k
//   "H"   the whole term on sites < k
//   L(prefix)  normal operator: the term's left part, when that part holds at most two
//              elementary operators (bonds k <= n/2) or the right part holds at least
//              three (bonds k > n/2); the coefficient is applied further right
//   R(suffix)  otherwise: the right part keys the channel and the left side carries the
//              coefficient-weighted sum of left parts (a complementary operator)
// W_k[w, w'] is the local operator taking channel w on bond k to w' on bond k+1; it
// picks up the coefficient where a term leaves the "plain" (I or L) channels.
#include <algorithm>
#include <array>
#include <cmath>
#include <map>
#include <tuple>

#include "common.hpp"

namespace b2 {

const QN kSiteQ[4] = {{0, 0}, {1, 1}, {1, -1}, {2, 0}};
const int kSiteN[4] = {0, 1, 1, 2};

namespace {

using Mat4 = std::array<double, 16>;

// Listing 1, Part A: alpha+, alpha, beta+, beta in the basis [0, a, b, ab]; row = output.
const Mat4 kCreA = {0, 0, 0, 0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0};
const Mat4 kAnnA = {0, 1, 0, 0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0};
const Mat4 kCreB = {0, 0, 0, 0, 0, 0, 0, 0, 1, 0, 0, 0, 0, -1, 0, 0};
const Mat4 kAnnB = {0, 0, 1, 0, 0, 0, 0, -1, 0, 0, 0, 0, 0, 0, 0, 0};

Mat4 matmul4(const Mat4& a, const Mat4& b) {
  Mat4 c{};
  for (int i = 0; i < 4; ++i)
    for (int k = 0; k < 4; ++k) {
      double x = a[i * 4 + k];
      if (x == 0) continue;
      for (int j = 0; j < 4; ++j) c[i * 4 + j] += x * b[k * 4 + j];
    }
  return c;
}

bool is_zero(const Mat4& a) {
  for (double x : a)
    if (x != 0) return false;
  return true;
}

// Table of distinct local operators (entries are small integers, compared exactly).
struct OpTable {
  std::vector<Mat4> mats;
  std::vector<QN> dq;
  std::unordered_map<uint64_t, int> index;
  static uint64_t hash(const Mat4& m) {
    uint64_t h = 0;
    for (double x : m) h = h * 3 + uint64_t(int(x) + 1);   // entries in {-1, 0, 1}
    return h;
  }
  int get(const Mat4& m) {
    for (double x : m)
      B2_REQUIRE(x == 0 || x == 1 || x == -1, B2_EINVAL, "local operator outside {-1,0,1}");
    uint64_t h = hash(m);
    auto it = index.find(h);
    if (it != index.end()) return it->second;
    int id = int(mats.size());
    B2_REQUIRE(id < 64, B2_EINVAL, "too many distinct local operators");
    mats.push_back(m);
    QN d{0, 0};
    bool set = false;
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        if (m[i * 4 + j] != 0) {
          QN x = kSiteQ[i] - kSiteQ[j];
          if (set) B2_REQUIRE(x == d, B2_EINVAL, "local operator without definite dq");
          d = x;
          set = true;
        }
    dq.push_back(d);
    index[h] = id;
    return id;
  }
};

// A site-ordered string of up to four (site, op, count) elements, packed 16 bits each:
// bits 10..15 site, 3..9 op id, 0..2 count.  Element 0 in the low bits.
struct Str {
  int len = 0;
  int site[4], op[4], cnt[4];
  uint64_t pack(int from, int to) const {   // elements [from, to)
    uint64_t k = 0;
    for (int i = from; i < to; ++i)
      k |= uint64_t((site[i] << 10) | (op[i] << 3) | cnt[i]) << (16 * (i - from));
    return k;
  }
};

struct ElemOp {
  int mode;
  bool dag;
};

}  // namespace

struct MpoBuilder {
  int n;
  OpTable table;
  // distinct site-ordered strings in first-seen order, with their summed coefficients
  std::unordered_map<uint64_t, int> index;
  std::vector<uint64_t> keys;
  std::vector<double> coefs;
  // for gradients: every spin-orbital term, its string and sign, and the integral it reads
  std::vector<b2_mpo_s::TermRec> terms;
  int cur_integral = 0;
  int8_t cur_kind = 0;

  explicit MpoBuilder(int n_) : n(n_) {}

  void add(double coef, const ElemOp* ops, int nops) {
    int sites[4];
    for (int i = 0; i < nops; ++i) sites[i] = ops[i].mode / 2;
    double sign = 1.0;
    for (int i = 0; i < nops; ++i)
      for (int j = i + 1; j < nops; ++j)
        if (sites[i] > sites[j]) sign = -sign;
    int order[4] = {0, 1, 2, 3};
    std::stable_sort(order, order + nops, [&](int a, int b) { return sites[a] < sites[b]; });
    Str s;
    Mat4 cur{};
    int cur_site = -1, cur_cnt = 0;
    auto flush = [&]() -> bool {
      if (cur_site < 0) return true;
      if (is_zero(cur)) return false;
      s.site[s.len] = cur_site;
      s.op[s.len] = table.get(cur);
      s.cnt[s.len] = cur_cnt;
      ++s.len;
      return true;
    };
    for (int t = 0; t < nops; ++t) {
      const ElemOp& e = ops[order[t]];
      const Mat4& m = (e.mode & 1) ? (e.dag ? kCreB : kAnnB) : (e.dag ? kCreA : kAnnA);
      if (sites[order[t]] == cur_site) {
        cur = matmul4(cur, m);
        ++cur_cnt;
      } else {
        if (!flush()) return;
        cur = m;
        cur_site = sites[order[t]];
        cur_cnt = 1;
      }
    }
    if (!flush()) return;
    const uint64_t key = s.pack(0, s.len);
    auto it = index.find(key);
    int idx;
    if (it == index.end()) {
      idx = int(keys.size());
      index.emplace(key, idx);
      keys.push_back(key);
      coefs.push_back(0.0);
    } else {
      idx = it->second;
    }
    coefs[idx] += sign * coef;
    terms.push_back({idx, cur_integral, cur_kind, int8_t(sign > 0 ? 1 : -1)});
  }

  static Str unpack(uint64_t k) {
    Str s;
    for (int i = 0; i < 4; ++i) {
      uint64_t e = (k >> (16 * i)) & 0xFFFF;
      if (e == 0) break;
      s.site[i] = int(e >> 10);
      s.op[i] = int((e >> 3) & 127);
      s.cnt[i] = int(e & 7);
      s.len = i + 1;
    }
    return s;
  }
};

}  // namespace b2

using b2::MpoBuilder;
using b2::QN;

namespace {

// channel key on a bond: 2-bit type in the top bits, packed substring below
constexpr uint64_t kTypeI = 1ull << 62, kTypeH = 2ull << 62, kTypeL = 0, kTypeR = 3ull << 62;

struct BondChans {
  std::unordered_map<uint64_t, int> index;
  std::vector<uint64_t> keys;
  int get(uint64_t key) {
    auto it = index.find(key);
    if (it != index.end()) return it->second;
    int id = int(keys.size());
    index[key] = id;
    keys.push_back(key);
    return id;
  }
};

}  // namespace

// Builds the MPO (throws b2::Error).
b2_mpo_s* b2_build_mpo_impl(int n, const double* h1, const double* eri, double e_core, int n_elec,
                            int two_sz, double cutoff) {
  B2_REQUIRE(n >= 2 && n <= 63, B2_EINVAL, "n_orb must be in [2, 63]");
  B2_REQUIRE(n_elec >= 0 && n_elec <= 2 * n, B2_EINVAL, "n_elec out of range");
  B2_REQUIRE(((n_elec + two_sz) % 2) == 0 && std::abs(two_sz) <= n_elec &&
                 (n_elec + two_sz) / 2 <= n && (n_elec - two_sz) / 2 <= n,
             B2_EINVAL, "(n_elec, two_sz) impossible");
  B2_REQUIRE(std::isfinite(e_core), B2_EINVAL, "non-finite e_core");
  size_t n2 = size_t(n) * n, n4 = n2 * n2;
  for (size_t i = 0; i < n2; ++i) B2_REQUIRE(std::isfinite(h1[i]), B2_EINVAL, "non-finite h1");
  for (size_t i = 0; i < n4; ++i) B2_REQUIRE(std::isfinite(eri[i]), B2_EINVAL, "non-finite eri");

  MpoBuilder bld(n);
  b2::ElemOp ops[4];
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q) {
      double v = h1[size_t(p) * n + q];
      if (std::abs(v) <= cutoff || v == 0) continue;
      bld.cur_integral = p * n + q;
      bld.cur_kind = 0;
      for (int s = 0; s < 2; ++s) {
        ops[0] = {2 * p + s, true};
        ops[1] = {2 * q + s, false};
        bld.add(v, ops, 2);
      }
    }
  for (int p = 0; p < n; ++p)
    for (int q = 0; q < n; ++q)
      for (int r = 0; r < n; ++r)
        for (int s = 0; s < n; ++s) {
          double v = eri[((size_t(p) * n + q) * n + r) * n + s];
          if (std::abs(v) <= cutoff || v == 0) continue;
          bld.cur_integral = int(((p * n + q) * n + r) * n + s);
          bld.cur_kind = 1;
          for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) {
              ops[0] = {2 * p + a, true};
              ops[1] = {2 * r + b, true};
              ops[2] = {2 * s + b, false};
              ops[3] = {2 * q + a, false};
              bld.add(0.5 * v, ops, 4);
            }
        }

  std::vector<BondChans> chans(n + 1);
  for (int k = 0; k < n; ++k) chans[k].get(kTypeI);
  for (int k = 1; k <= n; ++k) chans[k].get(kTypeH);
  // W accumulation: per site, (w << 32 | w2) -> entry index
  std::vector<std::unordered_map<uint64_t, int>> windex(n);
  auto* mpo = new b2_mpo_s;
  mpo->n = n;
  mpo->n_elec = n_elec;
  mpo->two_sz = two_sz;
  mpo->e_core = e_core;
  mpo->W.resize(n);
  auto entry = [&](int k, int w, int w2) -> b2_mpo_s::Entry& {
    uint64_t key = (uint64_t(uint32_t(w)) << 32) | uint32_t(w2);
    auto it = windex[k].find(key);
    if (it != windex[k].end()) return mpo->W[k][it->second];
    windex[k][key] = int(mpo->W[k].size());
    b2_mpo_s::Entry e;
    e.w = w;
    e.w2 = w2;
    std::fill(e.m, e.m + 16, 0.0);
    mpo->W[k].push_back(e);
    return mpo->W[k].back();
  };
  const double eye[16] = {1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1};
  for (int k = 0; k + 1 < n; ++k) std::copy(eye, eye + 16, entry(k, 0, 0).m);   // I -> I
  for (int k = 1; k < n; ++k) {
    int hk = chans[k].get(kTypeH), hk1 = chans[k + 1].get(kTypeH);
    std::copy(eye, eye + 16, entry(k, hk, hk1).m);                               // H -> H
  }
  if (e_core != 0) {
    auto& e = entry(0, 0, chans[1].get(kTypeH));
    for (int i = 0; i < 16; ++i) e.m[i] += e_core * eye[i];
  }

  auto key_of = [&](const b2::Str& s, int k) -> uint64_t {
    int nl = 0, nr = 0, split = 0;
    for (int i = 0; i < s.len; ++i) {
      if (s.site[i] < k) {
        nl += s.cnt[i];
        split = i + 1;
      } else {
        nr += s.cnt[i];
      }
    }
    if (nl == 0) return kTypeI;
    if (nr == 0) return kTypeH;
    bool left_keyed = (k <= n / 2) ? (nl <= 2) : (nr >= 3);
    if (left_keyed) return kTypeL | s.pack(0, split);
    return kTypeR | s.pack(split, s.len);
  };

  mpo->str_entry.assign(bld.keys.size(), b2_mpo_s::StringEntry{-1, -1, -1, -1});
  for (size_t si = 0; si < bld.keys.size(); ++si) {
    double coef = bld.coefs[si];
    if (coef == 0) continue;
    b2::Str s = MpoBuilder::unpack(bld.keys[si]);
    int first = s.site[0], last = s.site[s.len - 1];
    int el = 0;
    for (int k = first; k <= last; ++k) {
      uint64_t src_key = key_of(s, k), dst_key = key_of(s, k + 1);
      int src = chans[k].get(src_key), dst = chans[k + 1].get(dst_key);
      const double* mat = eye;
      int op_id = -1;
      if (el < s.len && s.site[el] == k) {
        op_id = s.op[el];
        mat = bld.table.mats[op_id].data();
        ++el;
      }
      bool src_plain = (src_key >> 62) == (kTypeI >> 62) || (src_key >> 62) == 0;
      bool dst_plain = (dst_key >> 62) == 0;
      auto& e = entry(k, src, dst);
      if (src_plain && !dst_plain) {
        for (int i = 0; i < 16; ++i) e.m[i] += coef * mat[i];
        mpo->str_entry[si] = {k, src, dst, op_id};   // where this string's coefficient enters
      } else {
        B2_REQUIRE(src_plain || !dst_plain, B2_EINVAL, "internal: channel order");
        for (int i = 0; i < 16; ++i) e.m[i] = mat[i];
      }
    }
  }

  mpo->D.resize(n + 1);
  mpo->parity.resize(n + 1);
  mpo->dq.resize(n + 1);
  mpo->chan_I.assign(n + 1, -1);
  mpo->chan_H.assign(n + 1, -1);
  for (int k = 0; k < n; ++k) mpo->chan_I[k] = chans[k].get(kTypeI);
  for (int k = 1; k <= n; ++k) mpo->chan_H[k] = chans[k].get(kTypeH);
  for (int k = 0; k <= n; ++k) {
    int d = int(chans[k].keys.size());
    mpo->D[k] = d;
    mpo->parity[k].assign(d, 0);
    mpo->dq[k].assign(d, QN{0, 0});
    for (int w = 0; w < d; ++w) {
      uint64_t key = chans[k].keys[w];
      uint64_t type = key >> 62;
      if (type == 1 || type == 2) continue;
      b2::Str s = MpoBuilder::unpack(key & ((1ull << 62) - 1));
      int par = 0;
      QN q{0, 0};
      for (int i = 0; i < s.len; ++i) {
        par += s.cnt[i];
        q = q + bld.table.dq[s.op[i]];
      }
      mpo->parity[k][w] = par & 1;
      mpo->dq[k][w] = (type == 0) ? q : QN{-q.n, -q.tsz};
    }
  }
  mpo->terms = std::move(bld.terms);
  mpo->ops.resize(bld.table.mats.size());
  for (size_t i = 0; i < bld.table.mats.size(); ++i)
    std::copy(bld.table.mats[i].begin(), bld.table.mats[i].end(), mpo->ops[i].begin());
  // drop W entries that cancelled exactly
  for (int k = 0; k < n; ++k) {
    auto& v = mpo->W[k];
    v.erase(std::remove_if(v.begin(), v.end(),
                           [](const b2_mpo_s::Entry& e) {
                             for (double x : e.m)
                               if (x != 0) return false;
                             return true;
                           }),
            v.end());
  }
  return mpo;
}

// ------------------------------------------------------------------ MPO compression
namespace {

// Eigen-decomposition of the symmetric n x n matrix a (row-major, overwritten) by cyclic
// Jacobi rotations (Golub & Van Loan, sym.schur2): eigenvalues in w, eigenvectors as the
// columns of v.  Stops when the off-diagonal mass is below 1e-30 of the matrix's.
void host_jacobi(int n, std::vector<double>& a, std::vector<double>& w, std::vector<double>& v) {
  v.assign(size_t(n) * n, 0.0);
  for (int i = 0; i < n; ++i) v[size_t(i) * n + i] = 1.0;
  double total = 0;
  for (double x : a) total += x * x;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += 2 * a[size_t(p) * n + q] * a[size_t(p) * n + q];
    if (off <= 1e-30 * total || off == 0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = a[size_t(p) * n + q];
        if (apq == 0) continue;
        const double app = a[size_t(p) * n + p], aqq = a[size_t(q) * n + q];
        const double tau = (aqq - app) / (2 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
        const double c = 1 / std::sqrt(1 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {   // A <- A J (columns p, q)
          const double akp = a[size_t(k) * n + p], akq = a[size_t(k) * n + q];
          a[size_t(k) * n + p] = c * akp - s * akq;
          a[size_t(k) * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
          const double apk = a[size_t(p) * n + k], aqk = a[size_t(q) * n + k];
          a[size_t(p) * n + k] = c * apk - s * aqk;
          a[size_t(q) * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {   // V <- V J
          const double vkp = v[size_t(k) * n + p], vkq = v[size_t(k) * n + q];
          v[size_t(k) * n + p] = c * vkp - s * vkq;
          v[size_t(k) * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = a[size_t(i) * n + i];
}

// A channel's incoming column (entries of W[site left of the bond] ending in it, keyed
// (w, local element)) or outgoing row (entries of W[site right of the bond] starting in
// it, keyed (w2, local element)), as a sparse vector.
using Sparse = std::vector<std::pair<int64_t, double>>;

}  // namespace

namespace {

double dot16(const double* a, const double* b) {
  double s = 0;
  for (int u = 0; u < 16; ++u) s += a[u] * b[u];
  return s;
}

// Gram matrix (dense D2 x D2) of the operators a site tensor's entries build on the next
// bond, from the Gram matrix G (D1 x D1) of the operators on the previous bond: for the
// left parts, entries (w1 -> w2) and G of bond b-1 give G of bond b; for the right parts,
// entries read the other way round.  Channels of different quantum numbers or parity are
// orthogonal (their operators have zero trace products), so only pairs within one group
// are formed; the parity factors of the fermion convention cancel within a group.
std::vector<double> next_gram(const std::vector<b2_mpo_s::Entry>& W, bool left_to_right, int D1,
                              const std::vector<double>& G, int D2, const std::vector<int>& group) {
  std::vector<std::vector<const b2_mpo_s::Entry*>> by(D2);
  for (const auto& e : W) by[left_to_right ? e.w2 : e.w].push_back(&e);
  std::vector<double> out(size_t(D2) * D2, 0.0);
  for (int x = 0; x < D2; ++x)
    for (int y = x; y < D2; ++y) {
      if (group[x] != group[y]) continue;
      double s = 0;
      for (const auto* e1 : by[x]) {
        const int a1 = left_to_right ? e1->w : e1->w2;
        for (const auto* e2 : by[y]) {
          const int a2 = left_to_right ? e2->w : e2->w2;
          const double g = G[size_t(a1) * D1 + a2];
          if (g != 0) s += g * dot16(e1->m, e2->m);
        }
      }
      out[size_t(x) * D2 + y] = out[size_t(y) * D2 + x] = s;
    }
  return out;
}

// Groups of a bond's channels: with isolate_ends, the groups that may be combined (same
// left-part quantum numbers and parity; the identity and whole-Hamiltonian channels alone);
// without, the classes of mutually non-orthogonal operators (same quantum numbers and
// parity), which the Gram recursions use.
std::vector<int> channel_groups(const b2_mpo_s* mpo, int b, int* n_groups, bool isolate_ends) {
  std::map<std::tuple<int, int, int>, int> id;
  std::vector<int> g(mpo->D[b]);
  int next = 0;
  for (int w = 0; w < mpo->D[b]; ++w) {
    if (isolate_ends && (w == mpo->chan_I[b] || w == mpo->chan_H[b])) {
      g[w] = next++;
      continue;
    }
    auto key = std::make_tuple(mpo->dq[b][w].n, mpo->dq[b][w].tsz, mpo->parity[b][w]);
    auto it = id.find(key);
    if (it == id.end()) it = id.emplace(key, next++).first;
    g[w] = it->second;
  }
  *n_groups = next;
  return g;
}

}  // namespace

// Bond-by-bond compression of the MPO (Sec. 2.3, the SVD construction with its controlled
// error; see b2_mpo_compress).  H = sum_w L_w (x) R_w across bond b.  Gram matrices of the
// complete left parts (built left to right on the current tensors) and right parts (built
// right to left on the original ones, which the pass has not touched yet) give, per group
// of channels, orthonormal left and right bases and the coefficient matrix X of the group's
// part of H in them; the SVD X = Y S Z^T truncated at tol * s_max is the best approximation
// of that part in the Frobenius norm.  New channel c: left part sum_w alpha_wc L_w, right
// part sum_w beta_wc R_w with alpha = U_A L_A^-1/2 Y and beta = U_C L_C^-1/2 Z S (A, C the
// group's left and right Grams), i.e. new columns of W[b-1] and rows of W[b].
double mpo_compress(b2_mpo_s* mpo, double tol, std::vector<int>* dims_out) {
  const int n = mpo->n;
  // right Grams of every bond, right to left
  std::vector<std::vector<double>> GR(n + 1);
  GR[n] = std::vector<double>(size_t(mpo->D[n]) * mpo->D[n], 0.0);
  for (int w = 0; w < mpo->D[n]; ++w) GR[n][size_t(w) * mpo->D[n] + w] = 1.0;
  for (int b = n - 1; b >= 1; --b) {
    int ng = 0;
    std::vector<int> cls = channel_groups(mpo, b, &ng, false);
    GR[b] = next_gram(mpo->W[b], false, mpo->D[b + 1], GR[b + 1], mpo->D[b], cls);
  }
  std::vector<double> GL(size_t(mpo->D[0]) * mpo->D[0], 0.0);
  for (int w = 0; w < mpo->D[0]; ++w) GL[size_t(w) * mpo->D[0] + w] = 1.0;
  double worst = 0;
  const double rank_eps = 1e-13;
  for (int b = 1; b < n; ++b) {
    auto& Wl = mpo->W[b - 1];
    auto& Wr = mpo->W[b];
    const int D = mpo->D[b];
    int ng = 0, ncls = 0;
    std::vector<int> grp = channel_groups(mpo, b, &ng, true);
    const std::vector<double> GLb = next_gram(Wl, true, mpo->D[b - 1], GL, D,
                                              channel_groups(mpo, b, &ncls, false));
    std::vector<Sparse> col(D), row(D);
    for (const auto& e : Wl)
      for (int u = 0; u < 16; ++u)
        if (e.m[u] != 0) col[e.w2].push_back({int64_t(e.w) * 16 + u, e.m[u]});
    for (const auto& e : Wr)
      for (int u = 0; u < 16; ++u)
        if (e.m[u] != 0) row[e.w].push_back({int64_t(e.w2) * 16 + u, e.m[u]});
    std::vector<std::vector<int>> members(ng);
    for (int w = 0; w < D; ++w) members[grp[w]].push_back(w);
    std::vector<Sparse> ncol, nrow;
    std::vector<int> npar;
    std::vector<b2::QN> ndq;
    int nI = -1, nH = -1;
    // sum_x coef[x][c] vecs[mem[x]] for a coefficient matrix of m rows and ld columns
    auto combine = [](const std::vector<Sparse>& vecs, const std::vector<int>& mem,
                      const std::vector<double>& coef, int m, int ld, int c) {
      std::map<int64_t, double> acc;
      for (int x = 0; x < m; ++x) {
        const double a = coef[size_t(x) * ld + c];
        if (a == 0) continue;
        for (const auto& kv : vecs[mem[x]]) acc[kv.first] += a * kv.second;
      }
      return Sparse(acc.begin(), acc.end());
    };
    for (int gi = 0; gi < ng; ++gi) {
      const auto& mem = members[gi];
      const int m = int(mem.size());
      const bool special = m == 1 && (mem[0] == mpo->chan_I[b] || mem[0] == mpo->chan_H[b]);
      if (special) {
        if (mem[0] == mpo->chan_I[b]) nI = int(ncol.size());
        if (mem[0] == mpo->chan_H[b]) nH = int(ncol.size());
        ncol.push_back(col[mem[0]]);
        nrow.push_back(row[mem[0]]);
        npar.push_back(mpo->parity[b][mem[0]]);
        ndq.push_back(mpo->dq[b][mem[0]]);
        continue;
      }
      // the group's left and right Grams and their eigen-decompositions
      std::vector<double> A(size_t(m) * m), C(size_t(m) * m), la, Ua, lc, Uc;
      for (int x = 0; x < m; ++x)
        for (int y = 0; y < m; ++y) {
          A[size_t(x) * m + y] = GLb[size_t(mem[x]) * D + mem[y]];
          C[size_t(x) * m + y] = GR[b][size_t(mem[x]) * D + mem[y]];
        }
      host_jacobi(m, A, la, Ua);
      host_jacobi(m, C, lc, Uc);
      double amax = 0, cmax = 0;
      for (double v : la) amax = std::max(amax, v);
      for (double v : lc) cmax = std::max(cmax, v);
      std::vector<int> ka, kc;
      for (int i = 0; i < m; ++i) {
        if (la[i] > rank_eps * amax) ka.push_back(i);
        if (lc[i] > rank_eps * cmax) kc.push_back(i);
      }
      const int ra = int(ka.size()), rc = int(kc.size());
      if (ra == 0 || rc == 0) continue;   // the group's part of H is zero
      // X = La^1/2 Ua^T Uc Lc^1/2 (ra x rc), its SVD through X^T X = Z S^2 Z^T
      std::vector<double> X(size_t(ra) * rc, 0.0);
      for (int i = 0; i < ra; ++i)
        for (int j = 0; j < rc; ++j) {
          double s2 = 0;
          for (int x = 0; x < m; ++x) s2 += Ua[size_t(x) * m + ka[i]] * Uc[size_t(x) * m + kc[j]];
          X[size_t(i) * rc + j] = std::sqrt(la[ka[i]]) * s2 * std::sqrt(lc[kc[j]]);
        }
      std::vector<double> XtX(size_t(rc) * rc, 0.0), s2v, Z;
      for (int p = 0; p < rc; ++p)
        for (int q = 0; q < rc; ++q) {
          double v = 0;
          for (int i = 0; i < ra; ++i) v += X[size_t(i) * rc + p] * X[size_t(i) * rc + q];
          XtX[size_t(p) * rc + q] = v;
        }
      host_jacobi(rc, XtX, s2v, Z);
      double smax2 = 0, tot = 0;
      for (double v : s2v) {
        smax2 = std::max(smax2, v);
        tot += std::max(v, 0.0);
      }
      std::vector<int> keep;
      double dropped = 0;
      for (int c = 0; c < rc; ++c) {
        if (s2v[c] > std::max(tol * tol, 1e-26) * smax2) keep.push_back(c);
        else dropped += std::max(s2v[c], 0.0);
      }
      if (tot > 0) worst = std::max(worst, std::sqrt(dropped / tot));
      const int r = int(keep.size());
      // alpha (m x r) = Ua_k La^-1/2 Y, Y = X Z S^-1; beta (m x r) = Uc_k Lc^-1/2 Z S
      std::vector<double> alpha(size_t(m) * std::max(r, 1), 0.0), beta(size_t(m) * std::max(r, 1), 0.0);
      for (int c = 0; c < r; ++c) {
        const int zc = keep[c];
        const double sc = std::sqrt(s2v[zc]);
        for (int i = 0; i < ra; ++i) {
          double y = 0;   // Y[i][c]
          for (int j = 0; j < rc; ++j) y += X[size_t(i) * rc + j] * Z[size_t(j) * rc + zc];
          y /= sc;
          const double f = y / std::sqrt(la[ka[i]]);
          for (int x = 0; x < m; ++x) alpha[size_t(x) * r + c] += Ua[size_t(x) * m + ka[i]] * f;
        }
        for (int j = 0; j < rc; ++j) {
          const double f = Z[size_t(j) * rc + zc] * sc / std::sqrt(lc[kc[j]]);
          for (int x = 0; x < m; ++x) beta[size_t(x) * r + c] += Uc[size_t(x) * m + kc[j]] * f;
        }
      }
      for (int c = 0; c < r; ++c) {
        ncol.push_back(combine(col, mem, alpha, m, r, c));
        nrow.push_back(combine(row, mem, beta, m, r, c));
        npar.push_back(mpo->parity[b][mem[0]]);
        ndq.push_back(mpo->dq[b][mem[0]]);
      }
    }
    // rebuild W[b-1] (columns) and W[b] (rows) from the new channels
    auto rebuild = [](const std::vector<Sparse>& vecs, bool as_col) {
      std::map<std::pair<int, int>, std::array<double, 16>> acc;
      for (size_t k = 0; k < vecs.size(); ++k)
        for (const auto& kv : vecs[k]) {
          const int other = int(kv.first / 16), u = int(kv.first % 16);
          auto key = as_col ? std::make_pair(other, int(k)) : std::make_pair(int(k), other);
          auto it = acc.find(key);
          if (it == acc.end()) it = acc.emplace(key, std::array<double, 16>{}).first;
          it->second[u] += kv.second;
        }
      std::vector<b2_mpo_s::Entry> out;
      for (const auto& kv : acc) {
        b2_mpo_s::Entry e;
        e.w = kv.first.first;
        e.w2 = kv.first.second;
        bool any = false;
        for (int u = 0; u < 16; ++u) {
          e.m[u] = kv.second[u];
          any |= e.m[u] != 0;
        }
        if (any) out.push_back(e);
      }
      return out;
    };
    Wl = rebuild(ncol, true);
    Wr = rebuild(nrow, false);
    mpo->D[b] = int(ncol.size());
    mpo->parity[b] = npar;
    mpo->dq[b] = ndq;
    mpo->chan_I[b] = nI;
    mpo->chan_H[b] = nH;
    // left Gram of the new channels, for the next bond
    int ng2 = 0;
    GL = next_gram(Wl, true, mpo->D[b - 1], GL, mpo->D[b], channel_groups(mpo, b, &ng2, false));
  }
  mpo->compressed = true;
  mpo->str_entry.clear();
  mpo->terms.clear();
  if (dims_out) *dims_out = mpo->D;
  return worst;
}
