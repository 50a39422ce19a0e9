// Block-sparse MPS storage: bond sector tables, site tensor block tables, host import and
// export (layout documented in include/b2.h).
#include <algorithm>
#include <cmath>

#include "common.hpp"

namespace b2 {

void* Ctx::raw_alloc(size_t bytes) {
  void* p = nullptr;
  if (alloc) {
    p = alloc(bytes, user);
    B2_REQUIRE(p != nullptr, B2_ENOMEM, "allocator callback failed for " + std::to_string(bytes) + " bytes");
  } else {
    cudaError_t e = cudaMallocAsync(&p, bytes, stream);
    B2_REQUIRE(e == cudaSuccess, B2_ENOMEM,
               std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
  }
  B2_REQUIRE((reinterpret_cast<uintptr_t>(p) & 255) == 0 || bytes < 256, B2_ENOMEM,
             "allocation not 256-byte aligned");
  return p;
}

void Ctx::raw_free(void* p) {
  if (!p) return;
  if (free_fn)
    free_fn(p, user);
  else
    cudaFreeAsync(p, stream);
}

int* Ctx::status() {
  if (!d_status) {
    d_status = static_cast<int*>(raw_alloc(256));
    B2_CUDA(cudaMemsetAsync(d_status, 0, 256, stream));
  }
  return d_status;
}

int Ctx::take_status() {
  if (!d_status) return 0;
  int h = 0;
  B2_CUDA(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, stream));
  B2_CUDA(cudaStreamSynchronize(stream));
  if (h) B2_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), stream));
  return h;
}

void SiteTensor::build(const Bond& left, const Bond& right) {
  blocks.clear();
  lookup.assign(size_t(left.size()) * 4, -1);
  size = 0;
  for (int jl = 0; jl < left.size(); ++jl)
    for (int s = 0; s < 4; ++s) {
      int jr = right.find(left.q[jl] + kSiteQ[s]);
      if (jr < 0) continue;
      lookup[size_t(jl) * 4 + s] = int(blocks.size());
      blocks.push_back({jl, s, jr, left.m[jl], right.m[jr], size});
      size += int64_t(left.m[jl]) * right.m[jr];
    }
}

}  // namespace b2

using b2::Bond;
using b2::QN;

b2_mps_s* b2_mps_import_impl(b2::Ctx* ctx, int n, int n_elec, int two_sz, const int* n_sectors,
                             const int* sectors, const double* site_data, int center) {
  B2_REQUIRE(n >= 2 && n <= 63, B2_EINVAL, "n must be in [2, 63]");
  B2_REQUIRE(center >= 0 && center < n, B2_EINVAL, "center out of range");
  B2_REQUIRE(n_sectors && sectors && site_data, B2_EINVAL, "null array");
  auto* mps = new b2_mps_s;
  std::unique_ptr<b2_mps_s> guard(mps);
  mps->ctx = ctx;
  mps->n = n;
  mps->n_elec = n_elec;
  mps->two_sz = two_sz;
  mps->center = center;
  mps->bonds.resize(n + 1);
  int64_t pos = 0;
  for (int k = 0; k <= n; ++k) {
    B2_REQUIRE(n_sectors[k] >= 1, B2_EINVAL, "every bond needs a sector");
    Bond& b = mps->bonds[k];
    for (int j = 0; j < n_sectors[k]; ++j, ++pos) {
      QN q{sectors[3 * pos], sectors[3 * pos + 1]};
      int m = sectors[3 * pos + 2];
      B2_REQUIRE(m >= 1, B2_EINVAL, "sector size must be positive");
      if (!b.q.empty()) B2_REQUIRE(b.q.back() < q, B2_EINVAL, "sectors not sorted by (N, 2Sz)");
      b.q.push_back(q);
      b.m.push_back(m);
    }
    b.finalize();
  }
  B2_REQUIRE((mps->bonds[0].size() == 1 && mps->bonds[0].q[0] == QN{0, 0} && mps->bonds[0].m[0] == 1),
             B2_EINVAL, "bond 0 must be the single sector (0, 0) of size 1");
  B2_REQUIRE((mps->bonds[n].size() == 1 && mps->bonds[n].q[0] == QN{n_elec, two_sz} &&
              mps->bonds[n].m[0] == 1),
             B2_EINVAL, "bond n must be the single target sector of size 1");
  mps->sites.resize(n);
  const double* src = site_data;
  for (int k = 0; k < n; ++k) {
    auto& st = mps->sites[k];
    st.build(mps->bonds[k], mps->bonds[k + 1]);
    B2_REQUIRE(st.size > 0, B2_EINVAL, "site tensor " + std::to_string(k) + " has no blocks");
    for (int64_t i = 0; i < st.size; ++i)
      B2_REQUIRE(std::isfinite(src[i]), B2_EINVAL, "non-finite MPS entry");
    st.data.reset(ctx, size_t(st.size) * sizeof(double));
    B2_CUDA(cudaMemcpyAsync(st.data.ptr, src, size_t(st.size) * sizeof(double),
                            cudaMemcpyHostToDevice, ctx->stream));
    src += st.size;
  }
  B2_CUDA(cudaStreamSynchronize(ctx->stream));
  return guard.release();
}

void b2_mps_export_impl(b2::Ctx* ctx, b2_mps_s* mps, int* n_sectors, int* sectors,
                        double* site_data) {
  int64_t pos = 0;
  for (int k = 0; k <= mps->n; ++k) {
    const Bond& b = mps->bonds[k];
    n_sectors[k] = b.size();
    for (int j = 0; j < b.size(); ++j, ++pos) {
      sectors[3 * pos] = b.q[j].n;
      sectors[3 * pos + 1] = b.q[j].tsz;
      sectors[3 * pos + 2] = b.m[j];
    }
  }
  double* dst = site_data;
  for (int k = 0; k < mps->n; ++k) {
    auto& st = mps->sites[k];
    B2_CUDA(cudaMemcpyAsync(dst, st.data.ptr, size_t(st.size) * sizeof(double),
                            cudaMemcpyDeviceToHost, ctx->stream));
    dst += st.size;
  }
  B2_CUDA(cudaStreamSynchronize(ctx->stream));
}
