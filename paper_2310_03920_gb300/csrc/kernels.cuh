// Device-side task formats and launchers of libb2's FP64 kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

namespace b2k {

// Number of kernels launched by this library in this process (all threads).
long long launch_count();
void count_launches(int n);

constexpr int kMaxBufs = 8;
struct BufTable {
  double* p[kMaxBufs];
};

// One contribution to an output block:
//   3-operand: out += alpha * op(P) [M x K1] * X [K1 x K2] * op(Q) [K2 x N]
//   2-operand (flags & kTwoOp): out += alpha * op(P) [M x K1] * op(X) [K1 x N]
// op(P) = P^T when flags & kTransP, op(Q) = Q^T when flags & kTransQ (2-operand: op(X) =
// X^T when flags & kTransQ).  Matrices are row-major with leading dimensions ld*.
// kBlockH marks the two block-Hamiltonian terms of an H_eff output (L_H (x) 1 (x) R_H and
// L_I (x) 1 (x) R_I: the energy scale of the product); the kernels ignore it.
enum : uint8_t { kTransP = 1, kTransQ = 2, kTwoOp = 4, kBlockH = 8 };
struct GemmTerm {
  int64_t offP, offX, offQ;
  int ldP, ldX, ldQ;
  int K1, K2;
  double alpha;
  uint8_t bufP, bufX, bufQ, flags;
};
// An output block [M x N] (row-major, leading dimension ld) and its terms [t0, t1).
struct GemmOut {
  int64_t off;
  int M, N, ld;
  int t0, t1;
  uint8_t buf, accumulate;   // accumulate = 0: out is overwritten
};
constexpr int kTile = 32;
// Work item of the FP64 kernel: the 32 x 32 tile (r0, c0) of output out, summed over the
// terms [t0, t1) of that output.  slot < 0: the item owns the tile and writes the output;
// slot >= 0: the item is one of several term ranges of the tile and writes its partial sum
// to partial[slot] (32 x 32), and a reduction task adds the slots in order.
struct GemmTask {
  int out, r0, c0;
  int t0, t1;
  int slot;
};
struct GemmReduce {
  int out, r0, c0;
  int slot0, n;
};

// out[i] (+)= sum_t c_t * in_t[i] for i < n: precombination of operator blocks.
struct CombTerm {
  int64_t off;
  double c;
  int buf;
};
struct CombOut {
  int64_t off, n;
  int t0, t1;
  int buf;
};
constexpr int kCombChunk = 2048;
struct CombTile {
  int out;
  int64_t e0;
};

// Strided block copy: dst[r*ldd + c] = src[r*lds + c] (or src[c*lds + r] when trans).
struct CopyTask {
  int64_t src, dst;
  int rows, cols, lds, ldd;
  int trans;
  uint8_t bsrc, bdst;
};

void launch_gemm(const GemmTask* tasks, int n_tasks, const GemmReduce* reds, int n_reds,
                 double* partial, const GemmOut* outs, const GemmTerm* terms, const BufTable& bt,
                 cudaStream_t s);
// One problem of a grouped launch (many independent problems in one grid): its work
// items, reductions, outputs, terms, partial tiles and buffers; item0 / red0 are the
// grid indices of its first work item / reduction (groups in increasing order).
struct GemmGroup {
  const GemmTask* tasks;
  const GemmReduce* reds;
  const GemmOut* outs;
  const GemmTerm* terms;
  double* partial;
  BufTable bt;
  int item0, red0;
};
void launch_gemm_grouped(const GemmGroup* groups, int n_groups, int n_items, int n_reds,
                         cudaStream_t s);
// ------------------------------------------------ split-precision tensor-core contraction
// An operand block split into hi / lo planes in the pre-tiled layout of tc_heff.cu: rows
// padded to rp = round16(rows), columns (the contraction index) to kp = round16(cols).
// Element (r, k) of the block is src[r * ld + k], or src[k * ld + r] with trans.  dst: the
// block's offset in elements of the planes (a multiple of 256).
struct SplitTask {
  int64_t src, dst;
  int rows, cols, ld, trans;
  int rp, kp;
  int buf;
};
void launch_split(const SplitTask* tasks, int n_tasks, const BufTable& bt, uint8_t* hi,
                  uint8_t* lo, bool tf32, cudaStream_t s);
// H_eff output block [M x N] (row-major, ld = N) at element offset off of the output
// vector, its terms [t0, t1); every term's L operand has M rows and R operand N rows.
struct TcOut {
  int64_t off;
  int M, N;
  int t0, t1;
  int accumulate;
};
// out += alpha * L [M x K1] psi [K1 x K2] R^T [K2 x N]; offA / offB2: element offsets of the
// split L and R operands (rows M / N, K = K1 / K2) in the environment planes, offB1: of the
// split psi^T block (rows K2, K = K1) in the psi planes.
struct TcTerm {   // 32 bytes: batches of them are copied into shared memory
  int64_t offA, offB1, offB2;
  uint16_t K1, K2;
  float alpha;
};
static_assert(sizeof(TcTerm) == 32, "TcTerm is moved in 16-byte units");
// Output tiles of the tensor-core contraction: kTcTileM rows x kTcTileN columns of a psi
// block (two CTAs per SM).
constexpr int kTcTileM = 64, kTcTileN = 64;
struct TcTile {
  int out, r0, c0;
};
// One problem of a launch: tiles, outputs and terms, the split planes and the FP64 output;
// tile0 is the grid index of its first tile (groups in increasing order).
struct TcGroup {
  const TcTile* tiles;
  const TcOut* outs;
  const TcTerm* terms;
  const uint8_t *env_hi, *env_lo, *psi_hi, *psi_lo;
  double* out;
  int tile0;
};
// One CTA per 128 x 128 output tile, over all groups' tiles (groups: device table of
// n_groups problems, or nullptr for the single problem g0); tf32: tf32 x3, else bf16 x3.
// A bounded wait that runs out writes 1 to *status; stuck_polls > 0 (tests) injects one.
void launch_heff_tc(const TcGroup& g0, const TcGroup* groups, int n_groups, int n_tiles, bool tf32,
                    int* status, uint32_t stuck_polls, cudaStream_t s);
void launch_comb(const CombTile* tiles, int n_tiles, const CombOut* outs, const CombTerm* terms,
                 const BufTable& bt, cudaStream_t s);
void launch_copy(int n_tasks, const CopyTask* tasks, const BufTable& bt, cudaStream_t s);
// Batched symmetric eigensolver (cyclic Jacobi); offs/eoffs: element offsets of each
// matrix (dims^2 each) and of its eigenvalues; work/woffs: global work space of 2 dims^2
// doubles for each matrix with jacobi_needs_work(dims, cluster size) (the others work in
// shared memory).  A matrix is solved either by one CTA or by a cluster of 2 to 16 CTAs;
// every cluster size applies the same rotations in the same order, so the results are
// identical (bitwise) whichever size solves a matrix.
constexpr int kJacobiSmemAV = 112;
inline bool jacobi_needs_work(int dim, int csize) { return csize > 1 || dim > kJacobiSmemAV; }
// Optional controls of a launch: flop_counter (device) += 12 m_active + 6 m per applied
// rotation; unconverged (device) += 1 for every matrix that used up max_sweeps sweeps
// (0 = the default of 60) with rotations still above the threshold.
struct JacobiCtl {
  double* flop_counter = nullptr;
  int* unconverged = nullptr;
  int max_sweeps = 0;
};
// One CTA per matrix, on stream s.
void launch_jacobi(int n_mat, const int* dims, const int64_t* offs, const int64_t* eoffs,
                   const double* a, double* evals, double* evecs, double* work,
                   const int64_t* woffs, int max_dim, cudaStream_t s,
                   const JacobiCtl& ctl = JacobiCtl());
// Host-side plan of a batch: a cluster size per matrix and the matrices grouped by size
// (ids, class by class).  GB300 runs FP64 at ~1.75 FMA per clock per SM, so one CTA is
// arithmetic-bound on a large matrix; the plan starts from one CTA per matrix and keeps
// doubling the cluster of the matrix with the longest modelled time while the CTAs still
// fit one per SM.  With more matrices than SMs every matrix keeps one CTA.
constexpr int kJacobiClasses = 5;   // cluster sizes 1, 2, 4, 8, 16
struct JacobiPlan {
  std::vector<int> csize;   // per matrix
  std::vector<int> ids;     // matrix ids ordered by class
  int n_cls = 0;
  int cls_csize[kJacobiClasses] = {};
  int cls_begin[kJacobiClasses + 1] = {};
  size_t cls_smem[kJacobiClasses] = {};   // dynamic shared memory of each class's launch
  bool spread = false;      // total CTAs <= SMs: launched one CTA per SM
};
JacobiPlan plan_jacobi(const std::vector<int>& dims);
// Streams for the classes of a plan, forked from the caller's stream s and joined back into
// it: class 0 (largest clusters) on stream[0], which should have the highest priority, class
// 1 on s, class k >= 2 on stream[k - 1].
struct JacobiStreams {
  cudaStream_t stream[kJacobiClasses - 1];
  cudaEvent_t fork;
  cudaEvent_t join[kJacobiClasses - 1];
};
// ids: device copy of plan.ids.  Without side streams the classes run one after another
// on s.
void launch_jacobi_plan(const JacobiPlan& plan, const int* ids, const int* dims,
                        const int64_t* offs, const int64_t* eoffs, const double* a,
                        double* evals, double* evecs, double* work, const int64_t* woffs,
                        cudaStream_t s, const JacobiStreams* side = nullptr,
                        const JacobiCtl& ctl = JacobiCtl());
// Global top-M selection over n eigenvalues (sector-major, descending in each sector).
// sector[i], index[i]: sector id and position in sector of value i.  Writes kept[sector]
// (counts, zeroed first, n_sec entries) and out[0] = discarded weight, out[1] = kept weight.
// n <= kSelectMax.
constexpr int kSelectMax = 16384;
void launch_select(int n, const double* vals, const int* sector, int n_sec, int M,
                   double cutoff, int* kept, double* out, cudaStream_t s);

// Davidson vector kernels (n-long FP64 vectors, k <= 64 of them).
// partial[j * nblk + b] = block b's part of dot(vs[j], x); then reduce to out[j] (with
// out_stride).
void launch_multidot(int k, const double* vs, int64_t ld, const double* x, int64_t n,
                     double* partial, double* out, int out_stride, cudaStream_t s);
// c = U exp(-t (Lambda - lambda_min)) U^T e_1 of a k x k eigen-decomposition (k <= 64; evecs
// row-major with eigenvector j in column j); stats: |c|^2, lambda_min, max |lambda|.
void launch_krylov_coef(int k, const double* evecs, const double* evals, double t, double* c,
                        double* stats, cudaStream_t s);
// y = y - sum_j c[j] vs[j]   (c on device)
void launch_multiaxpy(int k, const double* vs, int64_t ld, const double* c, double* y,
                      int64_t n, double sign, cudaStream_t s);
// u = V s, hu = W s, r = hu - theta u; t = r / (D - theta) (|den| < 1e-8 -> 1e-8);
// partial sums of |r|^2 into partial, reduced into out[0].  theta = evals[0], s = evec col 0.
void launch_ritz(int k, const double* V, const double* W, int64_t ld, const double* small_evecs,
                 int small_ld, const double* theta, const double* diag, double* u, double* hu,
                 double* t, int64_t n, double* partial, double* out, cudaStream_t s);
// x *= 1 / sqrt(*norm2); with flag (device), a norm below 1e-14 zeroes x and sets *flag = 1
void launch_scale_inv_sqrt(double* x, int64_t n, const double* norm2, cudaStream_t s,
                           double* flag = nullptr);
// x = alpha * y
void launch_axpby(double* x, const double* y, int64_t n, double a, double b, cudaStream_t s);
// Build the symmetric k x k Rayleigh matrix from the stored overlaps: g[i*k+j] =
// 0.5 (VW[i][j] + VW[j][i]), VW row-major with stride kmax.
void launch_symmetrize(int k, const double* vw, int kmax, double* g, cudaStream_t s);
// out[r][c] = u[r][c] * max(lam[c], floor)^power for an m x m row-major matrix; with
// drop_below, columns with lam[c] < floor are set to zero instead.
void launch_scale_cols(int m, const double* u, const double* lam, double power, double floor,
                       double* out, cudaStream_t s, bool drop_below = false);

// out[k] = sum_t sign_t * dot(A[offA_t : +n_t], B[offB_t : +n_t]) over the tasks t of output k
// (one CTA per output, fixed summation order).
struct DotTerm {
  int64_t offA, offB;
  int n;
  double sign;
};
struct DotOut {
  int t0, t1;
};
void launch_dots(int n_out, const DotOut* outs, const DotTerm* terms, const double* A,
                 const double* B, double* out, cudaStream_t s);

}  // namespace b2k
