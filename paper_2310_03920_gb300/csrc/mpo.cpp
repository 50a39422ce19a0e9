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
