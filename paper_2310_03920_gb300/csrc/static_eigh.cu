// Batched Jacobi eigensolver that allocates nothing: its scratch (the matrix metadata and
// the global-memory work space of matrices too large for shared memory) lives in one
// fixed device array defined in this file.
//
// The array is a file-scope __device__ variable, so every GPU that loads the library
// holds it (kScratchBytes) until the process exits.  Host code cannot use the array's name
// as a device address: the address is looked up once per device with
// cudaGetSymbolAddress (on the first call made on that device, with the device current)
// and passed to the kernels.  The cached address belongs to the device's primary context;
// a cudaDeviceReset tears that context down and is not supported between calls.
//
// The matrix sizes reach the device as a kernel argument (by value), and a one-block
// kernel writes the offsets into the array, so nothing is staged through host memory
// that outlives the call.  All calls share the array and it keeps the last call's
// contents; nothing in it has to start at zero (every call writes its metadata, and the
// eigensolver initialises its work space).  Calls whose work overlaps on the GPU (for
// example on two streams at once) race on the array.
#include <mutex>

#include "common.hpp"
#include "kernels.cuh"

namespace {

constexpr int kMaxMats = 1024;
constexpr int kShmemDim = b2k::kJacobiSmemAV;   // larger matrices need global work space
constexpr int64_t kWorkDoubles = int64_t(1) << 19;   // 4 MiB of Jacobi work space
constexpr int64_t kMetaDoubles = 4096;               // dims + three offset tables
constexpr int64_t kScratchDoubles = kMetaDoubles + kWorkDoubles;

static __device__ __align__(256) double g_b2_static_scratch[kScratchDoubles];

std::mutex g_mutex;
void* g_address[64] = {};

double* scratch_address(int device) {
  std::lock_guard<std::mutex> lock(g_mutex);
  B2_REQUIRE(device >= 0 && device < 64, B2_EINVAL, "device index out of range");
  if (!g_address[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_b2_static_scratch);
    B2_REQUIRE(e == cudaSuccess && p != nullptr, B2_ECUDA,
               std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
    g_address[device] = p;
  }
  return static_cast<double*>(g_address[device]);
}

// Layout of the metadata region at the start of the array.
struct Meta {
  int dims[kMaxMats];
  int pad[kMaxMats];   // keeps the int64 tables 8-byte aligned at a fixed offset
  int64_t offs[kMaxMats], eoffs[kMaxMats], woffs[kMaxMats];
};
static_assert(sizeof(Meta) <= kMetaDoubles * sizeof(double), "metadata exceeds its region");

// The sizes of one call, passed by value (2 KiB of kernel arguments).
struct Dims {
  int n;
  uint16_t d[kMaxMats];
};

// One thread writes the sizes and the prefix sums of dim^2 (matrices and eigenvectors),
// dim (eigenvalues) and 2 dim^2 over the matrices with dim > kShmemDim (work space).
__global__ void k_static_meta(const __grid_constant__ Dims p, Meta* m) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t o = 0, e = 0, w = 0;
  for (int i = 0; i < p.n; ++i) {
    const int d = p.d[i];
    m->dims[i] = d;
    m->offs[i] = o;
    m->eoffs[i] = e;
    m->woffs[i] = d > kShmemDim ? w : 0;
    o += int64_t(d) * d;
    e += d;
    if (d > kShmemDim) w += 2 * int64_t(d) * d;
  }
}

}  // namespace

extern "C" int b2_eigh_batched_static(b2_ctx ctx, int n_mat, const int* dims, const double* a,
                                      double* evals, double* evecs) {
  if (!ctx) return B2_EINVAL;
  try {
    ctx->c.last_error.clear();
    B2_REQUIRE(dims && a && evals && evecs, B2_EINVAL, "null argument");
    B2_REQUIRE(n_mat >= 0 && n_mat <= kMaxMats, B2_EINVAL,
               "b2_eigh_batched_static takes at most 1024 matrices");
    B2_CUDA(cudaSetDevice(ctx->c.device));
    Dims p;
    p.n = n_mat;
    int64_t w = 0;
    int max_dim = 0;
    for (int i = 0; i < n_mat; ++i) {
      B2_REQUIRE(dims[i] >= 1 && dims[i] <= 1024, B2_EINVAL, "dims must be in [1, 1024]");
      p.d[i] = uint16_t(dims[i]);
      if (dims[i] > kShmemDim) w += 2 * int64_t(dims[i]) * dims[i];
      max_dim = dims[i] > max_dim ? dims[i] : max_dim;
    }
    B2_REQUIRE(w <= kWorkDoubles, B2_EINVAL,
               "matrices larger than 112 need 2*dim^2 doubles each of static work space; "
               "their sum exceeds the 524288 available (4 MiB)");
    if (n_mat == 0) return B2_OK;
    double* base = scratch_address(ctx->c.device);
    Meta* meta = reinterpret_cast<Meta*>(base);
    k_static_meta<<<1, 32, 0, ctx->c.stream>>>(p, meta);
    b2k::count_launches(1);
    B2_CUDA(cudaGetLastError());
    // device addresses of the tables (offsets into the array; nothing is dereferenced here)
    char* mb = reinterpret_cast<char*>(base);
    const int* d_dims = reinterpret_cast<const int*>(mb + offsetof(Meta, dims));
    const int64_t* d_offs = reinterpret_cast<const int64_t*>(mb + offsetof(Meta, offs));
    const int64_t* d_eoffs = reinterpret_cast<const int64_t*>(mb + offsetof(Meta, eoffs));
    const int64_t* d_woffs = reinterpret_cast<const int64_t*>(mb + offsetof(Meta, woffs));
    b2k::launch_jacobi(n_mat, d_dims, d_offs, d_eoffs, a, evals, evecs, base + kMetaDoubles,
                       d_woffs, max_dim, ctx->c.stream);
    B2_CUDA(cudaGetLastError());
    return B2_OK;
  } catch (const b2::Error& err) {
    ctx->c.last_error = err.what();
    return err.code;
  } catch (const std::exception& err) {
    ctx->c.last_error = err.what();
    return B2_EINVAL;
  }
}
