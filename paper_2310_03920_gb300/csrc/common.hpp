// Internal declarations shared by the host-side translation units of libb2.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <cstring>
#include <memory>
#include <stdexcept>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/b2.h"

namespace b2 {

// ------------------------------------------------------------------ errors
struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};
#define B2_REQUIRE(cond, code, msg)                                   \
  do {                                                                \
    if (!(cond)) throw ::b2::Error((code), std::string(msg));         \
  } while (0)
#define B2_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      throw ::b2::Error(B2_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------- quantum numbers
struct QN {
  int n = 0, tsz = 0;
  bool operator==(const QN& o) const { return n == o.n && tsz == o.tsz; }
  bool operator<(const QN& o) const { return n < o.n || (n == o.n && tsz < o.tsz); }
  QN operator+(const QN& o) const { return {n + o.n, tsz + o.tsz}; }
  QN operator-(const QN& o) const { return {n - o.n, tsz - o.tsz}; }
  int64_t key() const { return (int64_t(n) << 32) ^ int64_t(uint32_t(tsz)); }
};
extern const QN kSiteQ[4];    // |0>, |a>, |b>, |ab>
extern const int kSiteN[4];

// --------------------------------------------------------------------- context
struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  b2_alloc_fn alloc = nullptr;
  b2_free_fn free_fn = nullptr;
  void* user = nullptr;
  std::string last_error;
  int* d_status = nullptr;   // device status words: [0] bounded waits, [1] Jacobi limit (0 = ok)
  // failure-path test settings (b2_debug_limits); 0 = off / the built-in defaults
  int jacobi_max_sweeps = 0;
  uint32_t stuck_polls = 0;
  // side streams and fork/join events (created on first use) for concurrent kernels
  static constexpr int kSides = 4;
  cudaStream_t side[kSides] = {};
  cudaEvent_t side_fork = nullptr;
  cudaEvent_t side_join[kSides] = {};
  void side_init() {
    if (side_fork) return;
    // side stream 0 at the device's highest priority (see b2k::JacobiStreams)
    int lo = 0, hi = 0;
    B2_CUDA(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    for (int k = 0; k < kSides; ++k) {
      B2_CUDA(cudaStreamCreateWithPriority(&side[k], cudaStreamNonBlocking, k == 0 ? hi : lo));
      B2_CUDA(cudaEventCreateWithFlags(&side_join[k], cudaEventDisableTiming));
    }
    B2_CUDA(cudaEventCreateWithFlags(&side_fork, cudaEventDisableTiming));
  }
  void side_destroy() {
    for (int k = 0; k < kSides; ++k) {
      if (side[k]) cudaStreamDestroy(side[k]);
      if (side_join[k]) cudaEventDestroy(side_join[k]);
      side[k] = nullptr;
      side_join[k] = nullptr;
    }
    if (side_fork) cudaEventDestroy(side_fork);
    side_fork = nullptr;
  }
  // benchmark profiling (b2_profile): events around H_eff kernel launches
  bool prof = false;
  long long launch_base = 0;
  double prof_flops = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_events;
  // ... and around the truncation eigensolver launches, with its applied-rotation flops
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> eig_events;
  double* d_eig_flops = nullptr;   // device counter (allocated by b2_profile)
  // ... and around the Davidson Rayleigh-Ritz eigensolver (k x k projected matrix)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> rr_events;
  void* raw_alloc(size_t bytes);
  void raw_free(void* p);
  // device status word of bounded waits: allocated and zeroed on first use
  int* status();
  // read (synchronising the stream) and clear the status word; nonzero = a wait ran out
  int take_status();
  void prof_clear() {
    for (auto* v : {&prof_events, &eig_events, &rr_events}) {
      for (auto& e : *v) {
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
      }
      v->clear();
    }
    prof_flops = 0;
    if (d_eig_flops) cudaMemsetAsync(d_eig_flops, 0, sizeof(double), stream);
  }
};

// Device buffer owned by the library, allocated through the context.
struct DevBuf {
  Ctx* ctx = nullptr;
  void* ptr = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(Ctx* c, size_t b) { reset(c, b); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { *this = std::move(o); }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      ctx = o.ctx; ptr = o.ptr; bytes = o.bytes;
      o.ptr = nullptr; o.bytes = 0;
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void reset(Ctx* c, size_t b) {
    release();
    ctx = c;
    bytes = b;
    ptr = b ? c->raw_alloc(b) : nullptr;
  }
  void release() {
    if (ptr && ctx) ctx->raw_free(ptr);
    ptr = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

// Upload a host vector into a (re)sized device buffer on the context stream.
template <class T>
void upload(Ctx* c, DevBuf& buf, const std::vector<T>& v) {
  size_t b = v.size() * sizeof(T);
  if (buf.bytes < b || buf.ptr == nullptr) buf.reset(c, b ? b : sizeof(T));
  if (b) B2_CUDA(cudaMemcpyAsync(buf.ptr, v.data(), b, cudaMemcpyHostToDevice, c->stream));
}

// ---------------------------------------------------------------- bond table
struct Bond {
  std::vector<QN> q;
  std::vector<int> m;
  std::vector<int64_t> off;   // state offset of each sector (prefix sums of m)
  std::unordered_map<int64_t, int> index;
  int total = 0;
  void finalize() {
    off.assign(q.size() + 1, 0);
    index.clear();
    for (size_t j = 0; j < q.size(); ++j) {
      off[j + 1] = off[j] + m[j];
      index[q[j].key()] = int(j);
    }
    total = int(off.back());
  }
  int find(const QN& x) const {
    auto it = index.find(x.key());
    return it == index.end() ? -1 : it->second;
  }
  int size() const { return int(q.size()); }
};

// ---------------------------------------------------------- site tensor table
struct SiteBlock {
  int jl, s, jr;
  int ml, mr;
  int64_t off;   // element offset in the site buffer
};
struct SiteTensor {
  std::vector<SiteBlock> blocks;
  std::vector<int> lookup;   // lookup[jl * 4 + s] -> block index or -1
  int64_t size = 0;
  DevBuf data;
  void build(const Bond& left, const Bond& right);   // all allowed blocks, sorted
  int find(int jl, int s) const { return lookup[size_t(jl) * 4 + s]; }
};

}  // namespace b2

// -------------------------------------------------------------- public handles
struct b2_ctx_s {
  b2::Ctx c;
};

struct b2_mpo_s {
  int n = 0, n_elec = 0, two_sz = 0;
  double e_core = 0.0;
  std::vector<int> D;                                // channels per bond
  std::vector<int> chan_I, chan_H;                   // per bond: the "nothing applied yet" and
                                                     // "whole term applied" channels (-1: none)
  std::vector<std::vector<int>> parity;              // per bond, per channel
  std::vector<std::vector<b2::QN>> dq;               // per bond, per channel (left part)
  struct Entry {
    int w, w2;
    double m[16];   // local operator, row = output state
  };
  std::vector<std::vector<Entry>> W;                 // per site
  // Coefficient Jacobian (for energy gradients).  Every distinct site-ordered operator
  // string s has one MPO entry where its coefficient c_s enters, W_site[w, w2] += c_s * op;
  // every spin-orbital term of the Hamiltonian adds sign * (h_pq or eri_pqrs / 2) to one
  // string's coefficient.
  struct StringEntry {
    int site, w, w2, op;   // op: index into ops, -1 = identity; site -1: coefficient zero
  };
  std::vector<StringEntry> str_entry;
  struct TermRec {
    int32_t str;
    int32_t integral;      // p*n+q (h) or ((p*n+q)*n+r)*n+s (eri)
    int8_t kind;           // 0: h, 1: eri (coefficient eri / 2)
    int8_t sign;
  };
  std::vector<TermRec> terms;
  std::vector<std::array<double, 16>> ops;           // local operator table
  bool compressed = false;   // b2_mpo_compress ran: channels are combinations, no Jacobian
};

struct b2_mps_s {
  b2::Ctx* ctx = nullptr;
  int n = 0, n_elec = 0, two_sz = 0, center = 0;
  std::vector<b2::Bond> bonds;          // n + 1
  std::vector<b2::SiteTensor> sites;    // n
};
