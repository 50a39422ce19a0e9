// FP64 kernels of libb2: block-sparse contractions, precombination of operators, the
// H_eff diagonal, the batched Jacobi eigensolver, truncation selection, block copies and
// the Davidson vector operations.  All loops over data are bounded by sizes passed in;
// there are no device-side waits.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <climits>
#include <cmath>
#include <mutex>

#include <cooperative_groups.h>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace b2k {

static std::atomic<long long> g_launches{0};
long long launch_count() { return g_launches.load(); }
void count_launches(int n) { g_launches += n; }

// ============================================================ block GEMM (FP64)
// One CTA of 128 threads takes one work item: a 32 x 32 tile of one output block and a
// range of that block's terms, added in order.  Items that own their tile write it; tiles
// whose terms are split over several items (so that small programs still fill the GPU)
// get per-item partial tiles that k_gemm_reduce adds in a fixed order: no atomics,
// deterministic.  A 3-operand term is evaluated as sum over 32-wide chunks c of K2 of
// (op(P) X[:, c]) op(Q)[c, :], keeping the intermediate chunk in shared memory.
__device__ __forceinline__ void load_tile(double (*S)[kTile + 1], const double* M, int ld,
                                          int rows, int cols, int r0, int c0, bool trans,
                                          int tid) {
  // S[i][j] = op(M)[r0 + i][c0 + j] (0 outside rows x cols); op(M) = M^T when trans
  if (!trans) {
    for (int e = tid; e < kTile * kTile; e += 128) {
      int i = e >> 5, j = e & 31;
      int r = r0 + i, c = c0 + j;
      S[i][j] = (r < rows && c < cols) ? M[int64_t(r) * ld + c] : 0.0;
    }
  } else {
    for (int e = tid; e < kTile * kTile; e += 128) {
      int j = e >> 5, i = e & 31;
      int r = r0 + i, c = c0 + j;
      S[i][j] = (r < rows && c < cols) ? M[int64_t(c) * ld + r] : 0.0;
    }
  }
}

// A tile staged through registers: fetch issues the thread's 8 global loads of a tile (the
// elements load_tile would store), put stores them to shared memory.  Fetching the next K
// chunk right after a barrier lets those loads run under the current chunk's FMAs.
struct TileRegs {
  double v[kTile * kTile / 128];
};
__device__ __forceinline__ void fetch_tile(TileRegs& R, const double* M, int ld, int rows, int cols,
                                           int r0, int c0, bool trans, int tid) {
#pragma unroll
  for (int q = 0; q < kTile * kTile / 128; ++q) {
    const int e = tid + 128 * q;
    const int i = trans ? (e & 31) : (e >> 5), j = trans ? (e >> 5) : (e & 31);
    const int r = r0 + i, c = c0 + j;
    R.v[q] = (r < rows && c < cols) ? (trans ? M[int64_t(c) * ld + r] : M[int64_t(r) * ld + c]) : 0.0;
  }
}
__device__ __forceinline__ void put_tile(double (*S)[kTile + 1], const TileRegs& R, bool trans, int tid) {
#pragma unroll
  for (int q = 0; q < kTile * kTile / 128; ++q) {
    const int e = tid + 128 * q;
    const int i = trans ? (e & 31) : (e >> 5), j = trans ? (e >> 5) : (e & 31);
    S[i][j] = R.v[q];
  }
}

// acc[a][b] += sum_{kk < kn} A[ry + a][kk] * B[kk][cx + b] (ry, cx: the thread's first row
// and column in the tile), kn rounded up to 8 (the tiles are zero there, so the sums equal
// the full-width ones exactly)
__device__ __forceinline__ void tile_fma(const double (*As)[kTile + 1], const double (*Bs)[kTile + 1],
                                         int kn, int cx, int ry, double (&acc)[2][4]) {
  const int kn8 = (kn + 7) & ~7;
  for (int k8 = 0; k8 < kn8; k8 += 8) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int kk = k8 + u;
      const double a0 = As[ry][kk], a1 = As[ry + 1][kk];
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const double x = Bs[kk][cx + b];
        acc[0][b] = fma(a0, x, acc[0][b]);
        acc[1][b] = fma(a1, x, acc[1][b]);
      }
    }
  }
}

__device__ __forceinline__ void gemm_item(const GemmTask& tile, const GemmOut* __restrict__ outs,
                                          const GemmTerm* __restrict__ terms, const BufTable& bt,
                                          double* __restrict__ partial) {
  __shared__ double Ps[kTile][kTile + 1], Xs[kTile][kTile + 1];
  __shared__ double Ts[kTile][kTile + 1], Qs[kTile][kTile + 1];
  const GemmOut o = outs[tile.out];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int r0 = tile.r0, c0 = tile.c0;
  // warp w owns the 16 x 16 quadrant (rows 16 (w >> 1), columns 16 (w & 1)) of the tile;
  // lane l its rows ry, ry + 1 and columns cx .. cx + 3.  Warps whose quadrant lies past
  // the block's rows or columns (or, for the intermediate, the K2 chunk) only load: the FP64
  // pipe is the bottleneck, and padded quadrants would spend it on zeros.
  const int qr = 16 * (warp >> 1), qc = 16 * (warp & 1);
  const int ry = qr + 2 * (lane >> 2), cx = qc + 4 * (lane & 3);
  const bool live_r = r0 + qr < o.M;
  const bool live = live_r && c0 + qc < o.N;
  double acc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  for (int t = tile.t0; t < tile.t1; ++t) {
    const GemmTerm g = terms[t];
    const double* P = bt.p[g.bufP] + g.offP;
    const double* X = bt.p[g.bufX] + g.offX;
    const bool tP = g.flags & kTransP, tQ = g.flags & kTransQ;
    double tacc[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
    TileRegs rp, rx;
    if (g.flags & kTwoOp) {
      fetch_tile(rp, P, g.ldP, o.M, g.K1, r0, 0, tP, tid);
      fetch_tile(rx, X, g.ldX, g.K1, o.N, 0, c0, tQ, tid);
      for (int k0 = 0; k0 < g.K1; k0 += kTile) {
        put_tile(Ps, rp, tP, tid);
        put_tile(Xs, rx, tQ, tid);
        __syncthreads();
        if (k0 + kTile < g.K1) {   // next chunk in flight during this chunk's FMAs
          fetch_tile(rp, P, g.ldP, o.M, g.K1, r0, k0 + kTile, tP, tid);
          fetch_tile(rx, X, g.ldX, g.K1, o.N, k0 + kTile, c0, tQ, tid);
        }
        if (live) tile_fma(Ps, Xs, min(kTile, g.K1 - k0), cx, ry, tacc);
        __syncthreads();
      }
    } else {
      const double* Q = bt.p[g.bufQ] + g.offQ;
      fetch_tile(rp, P, g.ldP, o.M, g.K1, r0, 0, tP, tid);
      fetch_tile(rx, X, g.ldX, g.K1, g.K2, 0, 0, false, tid);
      for (int k2 = 0; k2 < g.K2; k2 += kTile) {
        double tt[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
        for (int k1 = 0; k1 < g.K1; k1 += kTile) {
          put_tile(Ps, rp, tP, tid);
          put_tile(Xs, rx, false, tid);
          __syncthreads();
          if (k1 + kTile < g.K1) {
            fetch_tile(rp, P, g.ldP, o.M, g.K1, r0, k1 + kTile, tP, tid);
            fetch_tile(rx, X, g.ldX, g.K1, g.K2, k1 + kTile, k2, false, tid);
          } else {   // X is done for this K2 chunk: its registers stage the Q chunk
            fetch_tile(rx, Q, g.ldQ, g.K2, o.N, k2, c0, tQ, tid);
          }
          if (live_r && qc < g.K2 - k2) tile_fma(Ps, Xs, min(kTile, g.K1 - k1), cx, ry, tt);
          __syncthreads();
        }
        // every warp writes its quadrant of T (zeros where it skipped), so columns past the
        // chunk are zero for the second product
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          Ts[ry][cx + b] = tt[0][b];
          Ts[ry + 1][cx + b] = tt[1][b];
        }
        put_tile(Qs, rx, tQ, tid);
        __syncthreads();
        if (k2 + kTile < g.K2) {   // the next K2 chunk's first operand chunks
          fetch_tile(rp, P, g.ldP, o.M, g.K1, r0, 0, tP, tid);
          fetch_tile(rx, X, g.ldX, g.K1, g.K2, 0, k2 + kTile, false, tid);
        }
        if (live) tile_fma(Ts, Qs, min(kTile, g.K2 - k2), cx, ry, tacc);
        __syncthreads();
      }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(g.alpha, tacc[a][b], acc[a][b]);
  }
  if (tile.slot >= 0) {
    double* pt = partial + int64_t(tile.slot) * (kTile * kTile);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) pt[(ry + a) * kTile + cx + b] = acc[a][b];
    return;
  }
  double* out = bt.p[o.buf] + o.off;
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    int r = r0 + ry + a;
    if (r >= o.M) continue;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      int c = c0 + cx + b;
      if (c >= o.N) continue;
      double* p = out + int64_t(r) * o.ld + c;
      *p = o.accumulate ? *p + acc[a][b] : acc[a][b];
    }
  }
}

__global__ void __launch_bounds__(128, 4) k_gemm(const GemmTask* __restrict__ tasks,
                                              const GemmOut* __restrict__ outs,
                                              const GemmTerm* __restrict__ terms, BufTable bt,
                                              double* __restrict__ partial) {
  gemm_item(tasks[blockIdx.x], outs, terms, bt, partial);
}

// Grouped launch over the programs of several independent problems: CTA b takes item
// b - item0 of the group g with item0(g) <= b < item0(g + 1).
__device__ __forceinline__ int find_group(const GemmGroup* __restrict__ groups, int n_groups,
                                          int b, bool reds) {
  int lo = 0, hi = n_groups - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    const int start = reds ? groups[mid].red0 : groups[mid].item0;
    if (start <= b) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(128, 4) k_gemm_grouped(const GemmGroup* __restrict__ groups,
                                                      int n_groups) {
  const int g = find_group(groups, n_groups, blockIdx.x, false);
  const GemmGroup& G = groups[g];
  const BufTable bt = G.bt;
  gemm_item(G.tasks[blockIdx.x - G.item0], G.outs, G.terms, bt, G.partial);
}

__device__ __forceinline__ void reduce_item(const GemmReduce& rd, const GemmOut* __restrict__ outs,
                                            const BufTable& bt, const double* __restrict__ partial) {
  const GemmOut o = outs[rd.out];
  double* out = bt.p[o.buf] + o.off;
  for (int e = threadIdx.x; e < kTile * kTile; e += 128) {
    const int r = rd.r0 + e / kTile, c = rd.c0 + e % kTile;
    if (r >= o.M || c >= o.N) continue;
    double v = 0.0;
    for (int k = 0; k < rd.n; ++k) v += partial[int64_t(rd.slot0 + k) * (kTile * kTile) + e];
    double* p = out + int64_t(r) * o.ld + c;
    *p = o.accumulate ? *p + v : v;
  }
}

__global__ void __launch_bounds__(128) k_gemm_reduce(const GemmReduce* __restrict__ reds,
                                                     const GemmOut* __restrict__ outs, BufTable bt,
                                                     const double* __restrict__ partial) {
  reduce_item(reds[blockIdx.x], outs, bt, partial);
}

__global__ void __launch_bounds__(128) k_gemm_reduce_grouped(const GemmGroup* __restrict__ groups,
                                                             int n_groups) {
  const int g = find_group(groups, n_groups, blockIdx.x, true);
  const GemmGroup& G = groups[g];
  const BufTable bt = G.bt;
  reduce_item(G.reds[blockIdx.x - G.red0], G.outs, bt, G.partial);
}

void launch_gemm_grouped(const GemmGroup* groups, int n_groups, int n_items, int n_reds,
                         cudaStream_t s) {
  if (n_groups <= 0 || n_items <= 0) return;
  k_gemm_grouped<<<n_items, 128, 0, s>>>(groups, n_groups);
  g_launches += 1;
  if (n_reds <= 0) return;
  k_gemm_reduce_grouped<<<n_reds, 128, 0, s>>>(groups, n_groups);
  g_launches += 1;
}

void launch_gemm(const GemmTask* tasks, int n_tasks, const GemmReduce* reds, int n_reds,
                 double* partial, const GemmOut* outs, const GemmTerm* terms, const BufTable& bt,
                 cudaStream_t s) {
  if (n_tasks <= 0) return;
  k_gemm<<<n_tasks, 128, 0, s>>>(tasks, outs, terms, bt, partial);
  g_launches += 1;
  if (n_reds <= 0) return;
  k_gemm_reduce<<<n_reds, 128, 0, s>>>(reds, outs, bt, partial);
  g_launches += 1;
}

// =============================================================== precombination
__global__ void __launch_bounds__(256) k_comb(const CombTile* __restrict__ tiles,
                                              const CombOut* __restrict__ outs,
                                              const CombTerm* __restrict__ terms, BufTable bt) {
  const CombTile tile = tiles[blockIdx.x];
  const CombOut o = outs[tile.out];
  int64_t end = tile.e0 + kCombChunk;
  if (end > o.n) end = o.n;
  for (int64_t e = tile.e0 + threadIdx.x; e < end; e += 256) {
    double acc = 0.0;
    for (int t = o.t0; t < o.t1; ++t) {
      const CombTerm c = terms[t];
      acc = fma(c.c, bt.p[c.buf][c.off + e], acc);
    }
    bt.p[o.buf][o.off + e] = acc;
  }
}

void launch_comb(const CombTile* tiles, int n_tiles, const CombOut* outs, const CombTerm* terms,
                 const BufTable& bt, cudaStream_t s) {
  if (n_tiles <= 0) return;
  k_comb<<<n_tiles, 256, 0, s>>>(tiles, outs, terms, bt);
  g_launches += 1;
}

// =========================================================================== copy
__global__ void __launch_bounds__(128) k_copy(const CopyTask* __restrict__ tasks, BufTable bt) {
  const CopyTask c = tasks[blockIdx.x];
  const double* src = bt.p[c.bsrc] + c.src;
  double* dst = bt.p[c.bdst] + c.dst;
  const int n = c.rows * c.cols;
  for (int e = threadIdx.x; e < n; e += 128) {
    int r = e / c.cols, k = e % c.cols;
    dst[int64_t(r) * c.ldd + k] = c.trans ? src[int64_t(k) * c.lds + r] : src[int64_t(r) * c.lds + k];
  }
}

void launch_copy(int n_tasks, const CopyTask* tasks, const BufTable& bt, cudaStream_t s) {
  if (n_tasks <= 0) return;
  k_copy<<<n_tasks, 128, 0, s>>>(tasks, bt);
  g_launches += 1;
}

// ================================================================ batched Jacobi
// Cyclic Jacobi for a real symmetric matrix (Golub & Van Loan, Matrix Computations,
// Alg. 8.5.2 / 8.5.3 "sym.schur2" rotation), one CTA per matrix.  Each sweep visits every
// pair of its active rows (rows that still hold an off-diagonal element above the
// threshold) once in round-robin order, disjoint pairs per round, so one round applies the
// block-diagonal rotation J (2 x 2 blocks on the pairs) as A <- J^T A J.  Element blocks
// A[{p_i, q_i}][{p_j, q_j}] depend only on their own four entries, so a round is one pass
// over the 2 x 2 blocks of the upper triangle (mirrored below), and the eigenvector matrix
// is kept transposed (V^T) so that its rotations update two contiguous rows.  A rotation is
// skipped when the off-diagonal element is below kJacobiAbsTol times the largest input
// element or negligible next to both diagonal entries (binary exponent at least 61 below
// each); the iteration stops after a sweep without rotations or without two active rows
// (at most kMaxSweeps sweeps).  A lives in shared memory for dim <= kJacobiSmemA, V^T too
// for dim <= kJacobiSmemAV; larger matrices use global work space (2 dim^2 doubles).
constexpr int kJacobiSmemA = 160;
// A rotation is skipped when |a_pq| <= kJacobiAbsTol * max |a_ij| of the input: the
// eigen-decomposition is then accurate to about that fraction of the largest element
// (the accuracy of a backward-stable solver), and graded or rank-deficient density
// matrices, whose smallest eigenvalues are rounding noise, stop after about 10 to 30
// sweeps (dims 16 to 300) instead of chasing that noise up to kMaxSweeps.
constexpr double kJacobiAbsTol = 1e-15;
// Algorithmic flops of one applied rotation in a sweep over ms active rows of an m x m
// problem (textbook count: the two rows and two columns of A within the active rows,
// 12 ms, and two columns of V, 6 m), for the profiling counter.
constexpr double kJacobiRotFlopsA = 12.0, kJacobiRotFlopsV = 6.0;
constexpr int kMaxSweeps = 60;
constexpr int kJacobiThreads = 512;

// dynamic shared memory needed by a matrix of dimension m: A (dim <= kJacobiSmemA) and
// V^T (dim <= kJacobiSmemAV), then the round's rotations (c, s, pair rows p, q), the list
// of the pairs that rotate and the sweep's active rows (flags, list, positions)
__host__ __device__ inline size_t jacobi_smem_bytes(int m) {
  const int half = (m + (m & 1)) / 2;
  size_t aux = size_t(half) * (2 * sizeof(double) + 3 * sizeof(int)) + size_t(3 * m) * sizeof(int);
  size_t mat = 0;
  if (m <= kJacobiSmemAV)
    mat = 2 * size_t(m) * m * sizeof(double);
  else if (m <= kJacobiSmemA)
    mat = size_t(m) * m * sizeof(double);
  return mat + aux;
}

// Round-robin ("tournament") pairing of the cyclic sweep for an even count mp: index 0 stays
// at position 0 and indices 1..mp-1 move one position on per round, so in round r position
// i holds jacobi_at(i, r) and index x sits at jacobi_pos(x, r); pair k of the round is
// (positions k and mp-1-k).  Rounds are taken modulo mp-1 (a sweep has mp-1 rounds).
__device__ __forceinline__ int jacobi_at(int i, int r, int mp) {
  return i == 0 ? 0 : 1 + (i - 1 - r + (mp - 1)) % (mp - 1);
}
__device__ __forceinline__ int jacobi_pos(int x, int r, int mp) {
  return x == 0 ? 0 : 1 + (x - 1 + r) % (mp - 1);
}

// Deflation: a sweep pairs only the rows that still hold an off-diagonal element above tol
// (|a_xy| compared as bit patterns); the converged rows keep their last values and their
// entries against the active rows (all <= tol) are not rotated any more -- a perturbation at
// the stopping threshold, the accuracy the stopping rule gives anyway.  In a CPU re-enactment
// this removes a fifth of the rounds of graded density matrices (dim 64: 1134 -> 869,
// dim 147: 3087 -> 2499) at the same residual and orthogonality.
__device__ __forceinline__ int jacobi_row_active(const double* row, int x, int m,
                                                 long long tol_bits) {
  for (int y = 0; y < m; ++y)
    if (y != x && (__double_as_longlong(row[y]) & 0x7fffffffffffffffLL) > tol_bits) return 1;
  return 0;
}

// Block-wide compaction of flag[0..m): sidx = the flagged x in increasing order, spos[x] =
// its position there or -1; returns the count to every thread.  flag must be complete
// (a barrier before the call); wsum: >= 33 ints of shared memory.
__device__ int block_compact(const int* flag, int m, int* sidx, int* spos, int* wsum) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int per = (m + nt - 1) / nt;
  const int x0 = min(m, tid * per), x1 = min(m, x0 + per);
  int cnt = 0;
  for (int x = x0; x < x1; ++x) cnt += flag[x];
  int incl = cnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const int w = lane < nw ? wsum[lane] : 0;
    int wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += v;
    }
    if (lane < nw) wsum[lane] = wi - w;   // exclusive prefix of the warp totals
    if (lane == 31) wsum[32] = wi;        // total
  }
  __syncthreads();
  int off = wsum[warp] + incl - cnt;
  for (int x = x0; x < x1; ++x) {
    if (flag[x]) {
      sidx[off] = x;
      spos[x] = off++;
    } else {
      spos[x] = -1;
    }
  }
  const int total = wsum[32];
  __syncthreads();
  return total;
}

// max |src[e]| over e < n, returned to every thread of the block (red: >= 32 doubles)
__device__ double block_max_abs(const double* __restrict__ src, int n, double* red) {
  double v = 0.0;
  for (int e = threadIdx.x; e < n; e += blockDim.x) v = fmax(v, fabs(src[e]));
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  v = 0.0;
  for (int w = 0; w < int(blockDim.x >> 5); ++w) v = fmax(v, red[w]);
  __syncthreads();
  return v;
}

// Rotation (c, s) annihilating a_pq of the 2 x 2 pivot [app apq; apq aqq] (the smaller of
// the two angles, t = tan = s / c the root of apq t^2 + (aqq - app) t - apq = 0 with
// |t| <= 1).  The kernels scale the matrix by a power of two on entry so that max |a| lies
// in [0.5, 1): every pivot that rotates (|a_pq| above 1e-15 of that) is then a normal FP32
// number.  GB300 runs FP64 at about 1.75 operations per clock per SM, and this dependent
// chain sits on the critical path of every round, so t comes from FP32 arithmetic and is
// refined by two chord-Newton steps in FP64 that reuse one FP32 reciprocal of the derivative
// 2 apq t + (aqq - app) (each step multiplies the error by ~1e-7), and c = (1 + t^2)^(-1/2)
// from an FP32 reciprocal square root refined by two FP64 Newton steps y(3 - x y^2)/2:
// 16 FP64 operations, and the rotation equals the exactly computed one to rounding and is
// orthogonal to rounding.
__device__ __forceinline__ void jacobi_rotation(double app, double aqq, double apq, double& c,
                                                double& s) {
  const double d = aqq - app;
  const float d32 = static_cast<float>(d), p32 = static_cast<float>(apq);
  const float tau = d32 / (2.0f * p32);
  const float t32 = fabsf(tau) > 1e18f ? 0.5f / tau
                                        : copysignf(1.0f, tau) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
  const double r = 1.0f / fmaf(2.0f * p32, t32, d32);
  double t = t32;
#pragma unroll
  for (int it = 0; it < 2; ++it) t = fma(-fma(fma(apq, t, d), t, -apq), r, t);
  const double hx = 0.5 * fma(t, t, 1.0);
  double y = rsqrtf(fmaf(t32, t32, 1.0f));
#pragma unroll
  for (int it = 0; it < 2; ++it) y = y * fma(-hx * y, y, 1.5);
  c = y;
  s = t * y;
}

// Pivot test of the sweep: rotate unless |a_pq| <= tol (tol_bits: the bit pattern of tol >= 0)
// or a_pq is negligible next to both diagonal entries (binary exponent at least 61 below
// each).  Integer operations on the bit patterns, none on the FP64 pipe.
__device__ __forceinline__ bool jacobi_rotates(double app, double aqq, double apq,
                                               long long tol_bits) {
  const long long bp = __double_as_longlong(apq) & 0x7fffffffffffffffLL;
  if (bp <= tol_bits) return false;
  const int ep = int(bp >> 52);
  const int e1 = int((__double_as_longlong(app) >> 52) & 0x7ff);
  const int e2 = int((__double_as_longlong(aqq) >> 52) & 0x7ff);
  return !(ep + 61 <= e1 && ep + 61 <= e2);
}

// Binary exponent k with max_abs * 2^-k in [0.5, 1) (0 for a zero or non-finite maximum),
// clamped so that 2^k and 2^-k are finite
__device__ __forceinline__ int jacobi_scale_exp(double max_abs) {
  if (!(max_abs > 0.0) || !isfinite(max_abs)) return 0;
  return min(1000, max(-1000, ilogb(max_abs) + 1));
}

// row-major rank e of the upper triangle (i <= j < half) -> (i, j); the float estimate
// is corrected with exact integer arithmetic
__device__ __forceinline__ void unrank_upper(int e, int half, int& i, int& j) {
  const float h = 2.0f * half + 1.0f;
  i = int((h - sqrtf(fmaxf(h * h - 8.0f * float(e), 0.0f))) * 0.5f);
  i = max(0, min(i, half - 1));
  while (i > 0 && i * half - i * (i - 1) / 2 > e) --i;
  while ((i + 1) * half - (i + 1) * i / 2 <= e) ++i;
  j = i + (e - (i * half - i * (i - 1) / 2));
}

__global__ void __launch_bounds__(kJacobiThreads) k_jacobi(const int* __restrict__ dims,
                                                           const int64_t* __restrict__ offs,
                                                           const int64_t* __restrict__ eoffs,
                                                           const double* __restrict__ a,
                                                           double* evals, double* evecs,
                                                           double* work,
                                                           const int64_t* __restrict__ woffs,
                                                           const int* __restrict__ ids,
                                                           JacobiCtl ctl) {
  extern __shared__ double smem[];
  __shared__ int nact[2];    // rotating pairs of the round (double-buffered by round parity)
  __shared__ int nrot;       // rotations applied in the sweep
  double rot_flops = 0.0;    // thread 0: flops of the rotations applied
  const int b = ids ? ids[blockIdx.x] : int(blockIdx.x), tid = threadIdx.x, nt = blockDim.x;
  const int m = dims[b];
  const int mp = m + (m & 1), half = mp / 2;
  double *A, *Vt;
  double* next = smem;
  if (m <= kJacobiSmemAV) {
    A = smem;
    Vt = smem + size_t(m) * m;
    next = Vt + size_t(m) * m;
  } else if (m <= kJacobiSmemA) {
    A = smem;
    Vt = work + woffs[b] + size_t(m) * m;
    next = smem + size_t(m) * m;
  } else {
    A = work + woffs[b];
    Vt = A + size_t(m) * m;
  }
  double* cs = next;
  double* sn = cs + half;
  int* pi_ = reinterpret_cast<int*>(sn + half);
  int* qi_ = pi_ + half;
  int* act = qi_ + half;
  int* uc = act + half;     // row x active in this sweep
  int* sidx = uc + m;       // active rows, increasing
  int* spos = sidx + m;     // position of row x in sidx, or -1
  __shared__ int wsum[33];
  const double* src = a + offs[b];
  if (tid == 0) nact[0] = nact[1] = 0;
  __shared__ double red[kJacobiThreads / 32];
  // A scaled by 2^-ksc (exact) so that max |a| is in [0.5, 1); undone on the eigenvalues
  const double amax = block_max_abs(src, m * m, red);
  const int ksc = jacobi_scale_exp(amax);
  const double sc = scalbn(1.0, -ksc);
  for (int e = tid; e < m * m; e += nt) {
    A[e] = src[e] * sc;
    Vt[e] = (e / m == e % m) ? 1.0 : 0.0;
  }
  const long long tol_bits = __double_as_longlong(kJacobiAbsTol * (amax * sc));
  __syncthreads();
  int gr = 0;                               // rounds so far, over all sweeps
  const int max_sweeps = ctl.max_sweeps > 0 ? ctl.max_sweeps : kMaxSweeps;
  bool done = m <= 1;                       // stopped by the threshold, not the sweep limit
  for (int sweep = 0; sweep < max_sweeps && m > 1; ++sweep) {
    // the sweep pairs the active rows only (round-robin over their positions in sidx)
    for (int x = tid; x < m; x += nt) uc[x] = jacobi_row_active(A + x * m, x, m, tol_bits);
    __syncthreads();
    const int ms = block_compact(uc, m, sidx, spos, wsum);
    if (ms < 2) {
      done = true;
      break;
    }
    const int msp = ms + (ms & 1), hs = msp / 2;
    const int nblk = hs * (hs + 1) / 2;   // upper-triangle 2x2 blocks (i <= j) of the pairs
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int round = 0; round < msp - 1; ++round, ++gr) {
      const int par = gr & 1;
      for (int i = tid; i < hs; i += nt) {
        int pa = jacobi_at(i, round, msp), pb = jacobi_at(msp - 1 - i, round, msp);
        if (pa > pb) { int x = pa; pa = pb; pb = x; }
        const int p = sidx[pa], q = pb < ms ? sidx[pb] : -1;   // -1: p unpaired (odd count)
        double c = 1.0, s = 0.0;
        if (q >= 0) {
          const double apq = A[p * m + q], app = A[p * m + p], aqq = A[q * m + q];
          if (jacobi_rotates(app, aqq, apq, tol_bits)) {
            jacobi_rotation(app, aqq, apq, c, s);
            act[atomicAdd(&nact[par], 1)] = i;
          }
        }
        cs[i] = c;
        sn[i] = s;
        pi_[i] = p;
        qi_[i] = q;
      }
      __syncthreads();
      const int na = nact[par];
      if (tid == 0) {
        nrot += na;
        nact[par ^ 1] = 0;   // the next round's counter; its last reader was two rounds ago
      }
      if (na > 0) {
        // A <- J^T A J, one 2x2 block (pair i rows, pair j columns) per work item, i <= j
        for (int e = tid; e < nblk; e += nt) {
          // unrank e -> (i, j), 0 <= i <= j < hs, row-major over the upper triangle
          int i, j;
          unrank_upper(e, hs, i, j);
          const double ci = cs[i], si = sn[i], cj = cs[j], sj = sn[j];
          if (si == 0.0 && sj == 0.0) continue;   // identity on this block: nothing changes
          const int p = pi_[i], q = qi_[i], r = pi_[j], u = qi_[j];
          if (q >= 0 && u >= 0) {
            double app = A[p * m + r], apq = A[p * m + u], aqp = A[q * m + r], aqq = A[q * m + u];
            // rows: [c -s; s c] applied on (p, q); columns likewise on (r, u)
            double b11 = ci * app - si * aqp, b12 = ci * apq - si * aqq;
            double b21 = si * app + ci * aqp, b22 = si * apq + ci * aqq;
            double n11 = cj * b11 - sj * b12, n12 = sj * b11 + cj * b12;
            double n21 = cj * b21 - sj * b22, n22 = sj * b21 + cj * b22;
            if (i == j && si != 0.0) { n12 = 0.0; n21 = 0.0; }
            A[p * m + r] = n11; A[p * m + u] = n12; A[q * m + r] = n21; A[q * m + u] = n22;
            if (i != j) {
              A[r * m + p] = n11; A[u * m + p] = n12; A[r * m + q] = n21; A[u * m + q] = n22;
            }
          } else if (q >= 0) {   // column pair j is a single index r
            double ap = A[p * m + r], aq = A[q * m + r];
            double np = ci * ap - si * aq, nq = si * ap + ci * aq;
            A[p * m + r] = np; A[q * m + r] = nq;
            if (i != j) { A[r * m + p] = np; A[r * m + q] = nq; }
          } else if (u >= 0) {   // row pair i is a single index p
            double ar = A[p * m + r], au = A[p * m + u];
            double nr = cj * ar - sj * au, nu = sj * ar + cj * au;
            A[p * m + r] = nr; A[p * m + u] = nu;
            if (i != j) { A[r * m + p] = nr; A[u * m + p] = nu; }
          }
        }
        // V <- V J: rows p, q of V^T, one (rotating pair, column) per work item
        for (int t = tid; t < na * m; t += nt) {
          const int i = act[t / m], k = t % m;
          const int p = pi_[i], q = qi_[i];
          const double c = cs[i], s = sn[i];
          double vp = Vt[p * m + k], vq = Vt[q * m + k];
          Vt[p * m + k] = c * vp - s * vq;
          Vt[q * m + k] = s * vp + c * vq;
        }
      }
      __syncthreads();
    }
    if (tid == 0) rot_flops += double(nrot) * (kJacobiRotFlopsA * ms + kJacobiRotFlopsV * m);
    if (nrot == 0) {
      done = true;
      break;
    }
    __syncthreads();   // every thread has read nrot before it is reset
  }
  if (ctl.flop_counter && tid == 0) atomicAdd(ctl.flop_counter, rot_flops);
  if (!done && ctl.unconverged && tid == 0) atomicAdd(ctl.unconverged, 1);
  // descending order, ties by index
  double* ev = evals + eoffs[b];
  double* vec = evecs + offs[b];
  const double unsc = scalbn(1.0, ksc);
  for (int i = tid; i < m; i += nt) {
    double di = A[i * m + i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      double dj = A[j * m + j];
      rank += (dj > di) || (dj == di && j < i);
    }
    ev[rank] = di * unsc;
    for (int k = 0; k < m; ++k) vec[int64_t(k) * m + rank] = Vt[i * m + k];
  }
}

// The same rotation sequence for one matrix spread over a cluster of CTAs: GB300's FP64
// rate per SM is low (about 1.75 operations per clock), so one SM per large matrix bounds the
// whole truncation.  A is distributed over the cluster's shared memory by rows (row x in CTA
// x mod C) where it fits, else it stays in the global work space (L2 resident); V^T is split
// in column slices, one per CTA (shared memory where it fits).  Each sweep first marks the
// active rows (deflation: rows with an off-diagonal element above the threshold; every CTA
// checks its rows and writes the flags into all CTAs) and pairs only those.  Every round,
// each CTA computes all the round's rotations from its own copy of the round's pivots
// (diagonal entries and pair off-diagonals, identical in every CTA); the 2 x 2 blocks of A
// are dealt out round-robin over the CTAs (block e to CTA e mod C), so every CTA carries
// 1/C of the round's FP64 work; the thread that writes a pivot element of the NEXT round
// also writes it into every CTA's pivot copy (double-buffered by round parity); one cluster
// barrier per round then orders everything, and the CTA's own V^T slice is rotated between
// its arrive and wait.  Each element sees the same operations in the same order as in
// k_jacobi, so the results are identical.  One cluster per matrix: cluster k of the grid
// solves matrix ids[k].
// barrier.cluster.arrive (release) + barrier.cluster.wait (acquire): orders the global
// and distributed-shared-memory accesses of the cluster's threads around the barrier
__device__ __forceinline__ void cluster_barrier(const cg::cluster_group& cl) { cl.sync(); }
// the same barrier split in two: work between arrive and wait overlaps the other CTAs'
// arrival (it must not touch memory that other CTAs read after the barrier)
__device__ __forceinline__ void cluster_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_acquire() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared memory of one CTA: rotations (c, s, p, q), the rotating-pair list, the pivot
// copies of two rounds, the next round's pairing (partner and pair index of each row), the
// eigenvalue ranks, the sweep's active rows (flags, list, positions), this CTA's column
// slice of V^T where it fits in kJacobiVsliceMax and its rows of A where they fit in
// kJacobiAsliceMax
constexpr size_t kJacobiVsliceMax = 100 * 1024;
__host__ __device__ inline size_t jacobi_cluster_aux_bytes(int m) {
  const int mp = m + (m & 1), half = mp / 2;
  return size_t(half) * (2 * sizeof(double) + 3 * sizeof(int)) +
         size_t(2 * mp + 2 * half) * sizeof(double) + size_t(6 * mp) * sizeof(int);
}
__host__ __device__ inline size_t jacobi_vslice_bytes(int m, int C) {
  return size_t(m) * size_t((m + C - 1) / C) * sizeof(double);
}
__host__ __device__ inline bool jacobi_vslice_in_smem(int m, int C) {
  return jacobi_vslice_bytes(m, C) <= kJacobiVsliceMax;
}
// A distributed over the cluster's shared memory by rows (row x in CTA x mod C, local row
// x / C) where the slice fits in kJacobiAsliceMax; else A stays in the global work space
constexpr size_t kJacobiAsliceMax = 96 * 1024;
__host__ __device__ inline size_t jacobi_aslice_bytes(int m, int C) {
  return size_t((m + C - 1) / C) * size_t(m) * sizeof(double);
}
__host__ __device__ inline bool jacobi_aslice_in_smem(int m, int C) {
  return jacobi_aslice_bytes(m, C) <= kJacobiAsliceMax;
}
__host__ __device__ inline size_t jacobi_cluster_smem_bytes(int m, int C) {
  const size_t aux = (jacobi_cluster_aux_bytes(m) + 15) / 16 * 16;
  return aux + (jacobi_vslice_in_smem(m, C) ? jacobi_vslice_bytes(m, C) : 0) +
         (jacobi_aslice_in_smem(m, C) ? jacobi_aslice_bytes(m, C) : 0);
}

__global__ void __launch_bounds__(kJacobiThreads) k_jacobi_cluster(
    const int* __restrict__ dims, const int64_t* __restrict__ offs,
    const int64_t* __restrict__ eoffs, const double* __restrict__ a, double* evals,
    double* evecs, double* work, const int64_t* __restrict__ woffs,
    const int* __restrict__ ids, JacobiCtl ctl) {
  extern __shared__ double smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = int(cl.num_blocks());
  const int crank = int(cl.block_rank());
  const int b = ids[blockIdx.x / C];
  const int m = dims[b];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mp = m + (m & 1), half = mp / 2;
  double* Ag = work + woffs[b];
  double* cs = smem;
  double* sn = cs + half;
  double* snd = sn + half;        // [2][mp]: diagonal entries, by round parity
  double* sno = snd + 2 * mp;     // [2][half]: pair off-diagonals, by round parity
  int* pi_ = reinterpret_cast<int*>(sno + 2 * half);
  int* qi_ = pi_ + half;
  int* act = qi_ + half;
  int* partner = act + half;      // partner of row x in the next round
  int* pidx = partner + mp;       // index of x's pair in the next round
  int* rnk = pidx + mp;           // eigenvalue rank of row x (output)
  int* uc = rnk + mp;             // row x active in this sweep (written by every CTA)
  int* sidx = uc + mp;            // active rows, increasing
  int* spos = sidx + mp;          // position of row x in sidx, or -1
  __shared__ int wsum[33];
  // this CTA's columns [k0, k0 + ncol) of V^T: in shared memory (row x at Vs + x * ncol)
  // where the slice fits, else in the global work space (row x at Vt + x * m + k0)
  const int cw = (m + C - 1) / C;
  const int k0 = min(m, crank * cw), ncol = min(m, k0 + cw) - k0;
  const bool vs_smem = jacobi_vslice_in_smem(m, C);
  double* Vs = smem + (jacobi_cluster_aux_bytes(m) + 15) / 16 * 2;
  double* Vt = Ag + size_t(m) * m;
  double* vrow = vs_smem ? Vs : Vt + k0;   // V^T[x][k0 + kk] = vrow[x * vld + kk]
  const int vld = vs_smem ? ncol : m;
  // element (x, y) of A: row x of CTA x mod C in distributed shared memory, or global
  const bool as_smem = jacobi_aslice_in_smem(m, C);
  double* As = Vs + (vs_smem ? size_t(m) * cw : 0);   // the same offset in every CTA
  auto aref = [&](int x, int y) -> double* {
    if (as_smem) return cl.map_shared_rank(As + size_t(x / C) * m + y, x % C);
    return Ag + size_t(x) * m + y;
  };
  __shared__ int nact[2];
  __shared__ int nrot;
  double rot_flops = 0.0;    // thread 0: flops of the rotations applied
  const double* src = a + offs[b];
  const int gt = crank * nt + tid, gn = C * nt;
  if (tid == 0) nact[0] = nact[1] = 0;
  __shared__ double red[kJacobiThreads / 32];
  // A scaled by 2^-ksc (exact) so that max |a| is in [0.5, 1); the same in every CTA
  const double amax = block_max_abs(src, m * m, red);
  const int ksc = jacobi_scale_exp(amax);
  const double sc = scalbn(1.0, -ksc);
  const long long tol_bits = __double_as_longlong(kJacobiAbsTol * (amax * sc));
  if (as_smem) {   // this CTA's rows x = crank, crank + C, ...
    const int nr = (m - crank + C - 1) / C;
    for (int t = tid; t < nr * m; t += nt) {
      const int lx = t / m, y = t % m;
      As[size_t(lx) * m + y] = src[size_t(lx * C + crank) * m + y] * sc;
    }
  } else {
    for (int e = gt; e < m * m; e += gn) Ag[e] = src[e] * sc;
  }
  for (int t = tid; t < m * ncol; t += nt) {
    const int x = t / ncol, kk = t % ncol;
    vrow[x * vld + kk] = (x == k0 + kk) ? 1.0 : 0.0;
  }
  cluster_barrier(cl);   // A and V^T initialised by every CTA
  // element (x, y) of the updated A, v, into the next round's pivots of every CTA
  auto emit = [&](int np, int x, int y, double v) {
    double* dst = nullptr;
    if (x == y)
      dst = snd + np * mp + x;
    else if (partner[x] == y)
      dst = sno + np * half + pidx[x];
    if (!dst) return;
    for (int rk = 0; rk < C; ++rk) *cl.map_shared_rank(dst, rk) = v;
  };
  auto is_pivot = [&](int x, int y) { return x == y || partner[x] == y; };
  int gr = 0;   // rounds so far, over all sweeps
  const int max_sweeps = ctl.max_sweeps > 0 ? ctl.max_sweeps : kMaxSweeps;
  bool done = false;   // stopped by the threshold (uniform over the cluster)
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // active rows (deflation): this CTA checks rows crank, crank + C, ... and writes the
    // flags into every CTA; all CTAs then hold the same flags and build the same list
    for (int x = crank + C * tid; x < m; x += C * nt) {
      const int u = jacobi_row_active(as_smem ? As + size_t(x / C) * m : Ag + size_t(x) * m,
                                      x, m, tol_bits);
      for (int rk = 0; rk < C; ++rk) *cl.map_shared_rank(uc + x, rk) = u;
    }
    cluster_barrier(cl);
    const int ms = block_compact(uc, m, sidx, spos, wsum);
    if (ms < 2) {   // uniform: the same flags in every CTA
      done = true;
      break;
    }
    const int msp = ms + (ms & 1), hs = msp / 2;
    const int nblk = hs * (hs + 1) / 2;
    // pivots of the sweep's first round from A, in every CTA
    {
      const int par = gr & 1;
      for (int x = tid; x < m; x += nt) snd[par * mp + x] = *aref(x, x);
      for (int k = tid; k < hs; k += nt) {
        int pa = jacobi_at(k, 0, msp), pb = jacobi_at(msp - 1 - k, 0, msp);
        if (pa > pb) { int x = pa; pa = pb; pb = x; }
        sno[par * half + k] = pb < ms ? *aref(sidx[pa], sidx[pb]) : 0.0;
      }
    }
    if (tid == 0) nrot = 0;
    cluster_barrier(cl);   // every CTA has read its first pivots before any CTA updates A
    for (int round = 0; round < msp - 1; ++round, ++gr) {
      const int par = gr & 1, np = par ^ 1;
      // rotations of the round from the local pivot copy (same values in every CTA)
      for (int i = tid; i < hs; i += nt) {
        int pa = jacobi_at(i, round, msp), pb = jacobi_at(msp - 1 - i, round, msp);
        if (pa > pb) { int x = pa; pa = pb; pb = x; }
        const int p = sidx[pa], q = pb < ms ? sidx[pb] : -1;
        double c = 1.0, s = 0.0;
        if (q >= 0) {
          const double apq = sno[par * half + i];
          const double app = snd[par * mp + p], aqq = snd[par * mp + q];
          if (jacobi_rotates(app, aqq, apq, tol_bits)) {
            jacobi_rotation(app, aqq, apq, c, s);
            act[atomicAdd(&nact[par], 1)] = i;
          }
        }
        cs[i] = c;
        sn[i] = s;
        pi_[i] = p;
        qi_[i] = q;
      }
      // pairing of the next round, by row (rows outside the active list pair with none)
      for (int x = tid; x < m; x += nt) {
        const int sp = spos[x];
        if (sp < 0) {
          partner[x] = -1;
          continue;
        }
        const int pos = jacobi_pos(sp, round + 1, msp);
        const int ps = jacobi_at(msp - 1 - pos, round + 1, msp);
        partner[x] = ps < ms ? sidx[ps] : -1;
        pidx[x] = min(pos, msp - 1 - pos);
      }
      __syncthreads();
      const int na = nact[par];
      if (tid == 0) {
        nrot += na;
        nact[np] = 0;   // the next round's counter; its last reader was two rounds ago
      }
      for (int e = crank + C * tid; e < nblk; e += C * nt) {
        int i, j;
        unrank_upper(e, hs, i, j);
        const double ci = cs[i], si = sn[i], cj = cs[j], sj = sn[j];
        const int p = pi_[i], q = qi_[i], r = pi_[j], u = qi_[j];
        if (si == 0.0 && sj == 0.0) {   // identity on this block: only pass on its pivots
          if (is_pivot(p, r)) emit(np, p, r, *aref(p, r));
          if (u >= 0 && is_pivot(p, u)) emit(np, p, u, *aref(p, u));
          if (q >= 0 && is_pivot(q, r)) emit(np, q, r, *aref(q, r));
          if (q >= 0 && u >= 0 && i != j && is_pivot(q, u)) emit(np, q, u, *aref(q, u));
          if (i == j && q >= 0) emit(np, q, q, *aref(q, q));
          continue;
        }
        if (q >= 0 && u >= 0) {
          double* const ppr = aref(p, r);
          double* const ppu = aref(p, u);
          double* const pqr = aref(q, r);
          double* const pqu = aref(q, u);
          double app = *ppr, apq = *ppu, aqp = *pqr, aqq = *pqu;
          double b11 = ci * app - si * aqp, b12 = ci * apq - si * aqq;
          double b21 = si * app + ci * aqp, b22 = si * apq + ci * aqq;
          double n11 = cj * b11 - sj * b12, n12 = sj * b11 + cj * b12;
          double n21 = cj * b21 - sj * b22, n22 = sj * b21 + cj * b22;
          if (i == j && si != 0.0) { n12 = 0.0; n21 = 0.0; }
          *ppr = n11; *ppu = n12; *pqr = n21; *pqu = n22;
          if (i != j) {
            *aref(r, p) = n11; *aref(u, p) = n12; *aref(r, q) = n21; *aref(u, q) = n22;
          }
          emit(np, p, r, n11);
          emit(np, p, u, n12);
          if (i != j) emit(np, q, r, n21);   // (q, p) of a diagonal block is (p, q)
          emit(np, q, u, n22);
        } else if (q >= 0) {
          double* const ppr = aref(p, r);
          double* const pqr = aref(q, r);
          double ap = *ppr, aq = *pqr;
          double np_ = ci * ap - si * aq, nq = si * ap + ci * aq;
          *ppr = np_; *pqr = nq;
          if (i != j) { *aref(r, p) = np_; *aref(r, q) = nq; }
          emit(np, p, r, np_);
          emit(np, q, r, nq);
        } else if (u >= 0) {
          double* const ppr = aref(p, r);
          double* const ppu = aref(p, u);
          double ar = *ppr, au = *ppu;
          double nr = cj * ar - sj * au, nu = sj * ar + cj * au;
          *ppr = nr; *ppu = nu;
          if (i != j) { *aref(r, p) = nr; *aref(u, p) = nu; }
          emit(np, p, r, nr);
          emit(np, p, u, nu);
        }
      }
      // one barrier per round: the next round reads only its own pivot copy, complete once
      // every CTA has passed this barrier, before any CTA updates A again.  The V^T slice
      // is this CTA's alone, so its update runs between arrive and wait; the CTA barrier
      // after it keeps the next round's rotations from overwriting what it still reads.
      cluster_arrive_release();
      // V <- V J on this CTA's columns, one (rotating pair, column) per work item
      for (int t = tid; t < na * ncol; t += nt) {
        const int i = act[t / ncol], kk = t % ncol;
        const int p = pi_[i], q = qi_[i];
        const double c = cs[i], s = sn[i];
        double vp = vrow[p * vld + kk], vq = vrow[q * vld + kk];
        vrow[p * vld + kk] = c * vp - s * vq;
        vrow[q * vld + kk] = s * vp + c * vq;
      }
      __syncthreads();
      cluster_wait_acquire();
    }
    // the count is the same in every CTA (same rotations), so the exit is uniform
    if (tid == 0) rot_flops += double(nrot) * (kJacobiRotFlopsA * ms + kJacobiRotFlopsV * m);
    if (nrot == 0) {
      done = true;
      break;
    }
    __syncthreads();   // every thread has read nrot before it is reset
  }
  if (ctl.flop_counter && crank == 0 && tid == 0) atomicAdd(ctl.flop_counter, rot_flops);
  if (!done && ctl.unconverged && crank == 0 && tid == 0) atomicAdd(ctl.unconverged, 1);
  // descending order, ties by index; every CTA ranks all rows and writes its own columns
  double* ev = evals + eoffs[b];
  double* vec = evecs + offs[b];
  const double unsc = scalbn(1.0, ksc);
  // the diagonal, gathered into the pivot buffer (all of it read by every thread); the
  // barrier keeps every CTA's rows of A alive until all CTAs have read them
  double* dg = snd;
  for (int x = tid; x < m; x += nt) dg[x] = *aref(x, x);
  cluster_barrier(cl);
  for (int i = tid; i < m; i += nt) {
    double di = dg[i];
    int rank = 0;
    for (int j = 0; j < m; ++j) {
      double dj = dg[j];
      rank += (dj > di) || (dj == di && j < i);
    }
    rnk[i] = rank;
    if (crank == 0) ev[rank] = di * unsc;
  }
  __syncthreads();
  for (int t = tid; t < m * ncol; t += nt) {
    const int x = t / ncol, kk = t % ncol;
    vec[int64_t(k0 + kk) * m + rnk[x]] = vrow[x * vld + kk];
  }
}

// Both kernels' dynamic shared memory limits, set once: k_jacobi up to the largest
// per-matrix need (dim 160: A in shared memory), k_jacobi_cluster up to the largest need
// (a V^T slice of up to kJacobiVsliceMax) or the one-CTA-per-SM floor.  kJacobiSpreadSmem > half of an SM's 228 KB keeps a second CTA off the SM, so that
// each CTA of a spread plan has an FP64 pipe to itself.
constexpr size_t kJacobiSpreadSmem = 116 * 1024;
static size_t jacobi_smem_limit() {
  size_t smem = 0;
  for (int m = 1; m <= 1024; ++m) smem = smem > jacobi_smem_bytes(m) ? smem : jacobi_smem_bytes(m);
  return smem > kJacobiSpreadSmem ? smem : kJacobiSpreadSmem;
}
static size_t jacobi_cluster_smem_limit() {
  size_t smem = kJacobiSpreadSmem;   // at most aux + kJacobiVsliceMax + kJacobiAsliceMax
  for (int C = 2; C <= 16; C *= 2)
    for (int m = 1; m <= 1024; ++m) smem = std::max(smem, jacobi_cluster_smem_bytes(m, C));
  return smem;
}

// Largest cluster size the device runs for k_jacobi_cluster with spread shared memory: 16
// (non-portable) where possible, else 8.
static int jacobi_max_cluster() {
  static std::once_flag once;
  static int csize = 8;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(jacobi_smem_limit()));
    cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(jacobi_cluster_smem_limit()));
    if (cudaFuncSetAttribute(k_jacobi_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
        cudaSuccess) {
      cudaGetLastError();
      return;
    }
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(16, 1, 1);
    q.blockDim = dim3(kJacobiThreads, 1, 1);
    q.dynamicSmemBytes = kJacobiSpreadSmem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    q.attrs = at;
    q.numAttrs = 1;
    int n_clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&n_clusters, k_jacobi_cluster, &q) == cudaSuccess &&
        n_clusters > 0)
      csize = 16;
    cudaGetLastError();
  });
  return csize;
}

void launch_jacobi(int n_mat, const int* dims, const int64_t* offs, const int64_t* eoffs,
                   const double* a, double* evals, double* evecs, double* work,
                   const int64_t* woffs, int max_dim, cudaStream_t s, const JacobiCtl& ctl) {
  if (n_mat <= 0) return;
  jacobi_max_cluster();   // sets the shared memory limits
  // the need is not monotonic in the dimension (V^T leaves shared memory above
  // kJacobiSmemAV, A above kJacobiSmemA): the largest over every dimension up to max_dim
  size_t smem = 0;
  for (int m = 1; m <= max_dim; ++m) smem = std::max(smem, jacobi_smem_bytes(m));
  k_jacobi<<<n_mat, kJacobiThreads, smem, s>>>(dims, offs, eoffs, a, evals, evecs, work, woffs,
                                               nullptr, ctl);
  g_launches += 1;
}

// Modelled time of one Jacobi round (us) of an m x m matrix on a cluster of C CTAs, one
// per SM: the A and V^T updates (about 4 m^2 FP64 operations, split over the CTAs), the
// m/2 rotations that every CTA computes (about 35 operations each), at 1.75 operations per
// clock at 2.07 GHz, plus the round's synchronisation (a cluster barrier, or __syncthreads).
static double jacobi_round_us(int m, int C) {
  const double ops = 4.0 * m * m / C + 17.5 * m;
  return ops / 3600.0 + (C > 1 ? 1.0 : 0.3);
}

JacobiPlan plan_jacobi(const std::vector<int>& dims) {
  JacobiPlan p;
  const int n = int(dims.size());
  p.csize.assign(n, 1);
  int dev = 0, n_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  const int cmax = jacobi_max_cluster();
  // CTAs left for doubling: a seventh of the SMs stays free, as clusters must be packed
  // into GPCs (up to 16 SMs of one GPC per cluster)
  const long long budget = n_sm - n_sm / 7;
  long long used = n;
  if (used <= budget) {
    // rounds per sweep (m - 1) x round time: the sweep count is similar across a batch.
    // Double the cluster of the slowest matrix that still gains from it, while the CTAs fit.
    auto t = [&](int b, int C) { return double(dims[b]) * jacobi_round_us(dims[b], C); };
    for (;;) {
      int w = -1;
      double tw = -1.0;
      for (int b = 0; b < n; ++b) {
        const int C = p.csize[b];
        const double tb = t(b, C);
        if (C < cmax && used + C <= budget && t(b, 2 * C) < tb && tb > tw) {
          tw = tb;
          w = b;
        }
      }
      if (w < 0) break;
      used += p.csize[w];
      p.csize[w] *= 2;
    }
    p.spread = true;
  }
  static const int kSizes[kJacobiClasses] = {16, 8, 4, 2, 1};   // launch order
  for (int k = 0; k < kJacobiClasses; ++k) {
    const int begin = int(p.ids.size());
    size_t smem = 0;
    for (int b = 0; b < n; ++b)
      if (p.csize[b] == kSizes[k]) {
        p.ids.push_back(b);
        smem = std::max(smem, kSizes[k] == 1 ? jacobi_smem_bytes(dims[b])
                                             : jacobi_cluster_smem_bytes(dims[b], kSizes[k]));
      }
    if (int(p.ids.size()) == begin) continue;
    if (p.spread) smem = std::max(smem, kJacobiSpreadSmem);
    p.cls_csize[p.n_cls] = kSizes[k];
    p.cls_begin[p.n_cls] = begin;
    p.cls_smem[p.n_cls] = smem;
    ++p.n_cls;
  }
  p.cls_begin[p.n_cls] = int(p.ids.size());
  return p;
}

void launch_jacobi_plan(const JacobiPlan& p, const int* ids, const int* dims, const int64_t* offs,
                        const int64_t* eoffs, const double* a, double* evals, double* evecs,
                        double* work, const int64_t* woffs, cudaStream_t s,
                        const JacobiStreams* side, const JacobiCtl& ctl) {
  if (p.n_cls == 0) return;
  jacobi_max_cluster();
  // With side streams, class 0 (the largest clusters) runs on side stream 0, which has the
  // highest priority so that its clusters find whole GPCs free, class 1 on s, class k >= 2 on
  // side stream k - 1: they touch disjoint matrices and outputs.
  const bool fork = side && p.n_cls > 1;
  auto stream_of = [&](int k) { return !fork ? s : (k == 1 ? s : side->stream[k == 0 ? 0 : k - 1]); };
  if (fork) {
    cudaEventRecord(side->fork, s);
    for (int k = 0; k < p.n_cls; ++k)
      if (k != 1) cudaStreamWaitEvent(stream_of(k), side->fork, 0);
  }
  for (int k = 0; k < p.n_cls; ++k) {
    cudaStream_t sk = stream_of(k);
    const int C = p.cls_csize[k];
    const int cnt = p.cls_begin[k + 1] - p.cls_begin[k];
    const int* cids = ids + p.cls_begin[k];
    const size_t smem = p.cls_smem[k];
    if (C == 1) {
      k_jacobi<<<cnt, kJacobiThreads, smem, sk>>>(dims, offs, eoffs, a, evals, evecs, work, woffs,
                                                  cids, ctl);
    } else {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(unsigned(cnt) * unsigned(C), 1, 1);
      cfg.blockDim = dim3(kJacobiThreads, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = sk;
      cudaLaunchAttribute attr_c[1];
      attr_c[0].id = cudaLaunchAttributeClusterDimension;
      attr_c[0].val.clusterDim.x = unsigned(C);
      attr_c[0].val.clusterDim.y = 1;
      attr_c[0].val.clusterDim.z = 1;
      cfg.attrs = attr_c;
      cfg.numAttrs = 1;
      cudaLaunchKernelEx(&cfg, k_jacobi_cluster, dims, offs, eoffs, a, evals, evecs, work, woffs,
                         cids, ctl);
    }
    g_launches += 1;
  }
  if (fork) {   // join: s waits for every class on a side stream
    for (int k = 0; k < p.n_cls; ++k) {
      if (k == 1) continue;
      const int j = k == 0 ? 0 : k - 1;
      cudaEventRecord(side->join[j], side->stream[j]);
      cudaStreamWaitEvent(s, side->join[j], 0);
    }
  }
}

// ======================================================================= selection
// Single CTA: bitonic sort of (value desc, id asc); chain neighbours closer than
// 1e-14 * max into groups; re-sort by (group, id); keep the first M above cutoff * max.
__device__ void bitonic_desc_val(double* key, int* id, int n2, int tid, int nt) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < n2; i += nt) {
        int l = i ^ j;
        if (l > i) {
          bool up = (i & k) == 0;   // "up" segment sorted descending by value
          // a comes before b when (value larger) or (equal value and smaller id)
          bool i_first = (key[i] > key[l]) || (key[i] == key[l] && id[i] < id[l]);
          if (up != i_first) {
            double tk = key[i]; key[i] = key[l]; key[l] = tk;
            int ti = id[i]; id[i] = id[l]; id[l] = ti;
          }
        }
      }
      __syncthreads();
    }
}

__device__ void bitonic_asc_int(long long* key, int n2, int tid, int nt) {
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < n2; i += nt) {
        int l = i ^ j;
        if (l > i) {
          bool up = (i & k) == 0;
          if (up == (key[i] > key[l])) {
            long long t = key[i]; key[i] = key[l]; key[l] = t;
          }
        }
      }
      __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_select(int n, const double* __restrict__ vals,
                                                 const int* __restrict__ sector, int n_sec,
                                                 int M, double cutoff, int* kept, double* out) {
  extern __shared__ unsigned char sm_raw[];
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  double* key = reinterpret_cast<double*>(sm_raw);
  int* id = reinterpret_cast<int*>(key + n2);
  long long* key2 = reinterpret_cast<long long*>(key);   // reused after the first sort
  __shared__ double red[1024];
  __shared__ double vmax_s;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int i = tid; i < n_sec; i += nt) kept[i] = 0;
  double vmax = -DBL_MAX, tot = 0.0;
  for (int i = tid; i < n2; i += nt) {
    key[i] = i < n ? vals[i] : -DBL_MAX;
    id[i] = i;
    if (i < n) {
      vmax = fmax(vmax, vals[i]);
      tot += vals[i];
    }
  }
  red[tid] = vmax;
  __syncthreads();
  for (int st = nt / 2; st > 0; st >>= 1) {
    if (tid < st) red[tid] = fmax(red[tid], red[tid + st]);
    __syncthreads();
  }
  if (tid == 0) vmax_s = red[0];
  __syncthreads();
  vmax = vmax_s;
  // total weight in a fixed order (thread 0 sums sequentially for reproducibility)
  __syncthreads();
  bitonic_desc_val(key, id, n2, tid, nt);
  // group ids by chaining neighbours: flag[i] = 1 if a new group starts at i
  // prefix sum of flags -> group; store composite (group << 20 | id) in key2 afterwards
  __shared__ int chunk_sum[1025];
  int per = (n + nt - 1) / nt;
  int lo = tid * per, hi = min(n, lo + per);
  const double tol = 1e-14 * vmax;
  int cnt = 0;
  for (int i = lo; i < hi; ++i) cnt += (i == 0) || (key[i - 1] - key[i] > tol);
  chunk_sum[tid + 1] = cnt;
  if (tid == 0) chunk_sum[0] = 0;
  __syncthreads();
  if (tid == 0)
    for (int i = 1; i <= nt; ++i) chunk_sum[i] += chunk_sum[i - 1];
  __syncthreads();
  // compute groups into registers first (key is overwritten by key2 afterwards)
  long long comp[32];
  int g = chunk_sum[tid];
  int nloc = 0;
  for (int i = lo; i < hi && nloc < 32; ++i) {
    g += (i == 0) || (key[i - 1] - key[i] > tol);
    comp[nloc++] = ((long long)(g - 1) << 20) | (long long)id[i];
  }
  __syncthreads();
  for (int i = lo, c = 0; i < hi && c < 32; ++i, ++c) key2[i] = comp[c];
  for (int i = n + tid; i < n2; i += nt) key2[i] = LLONG_MAX;
  __syncthreads();
  bitonic_asc_int(key2, n2, tid, nt);
  if (tid == 0) {
    double kw = 0.0, all = 0.0;
    for (int i = 0; i < n; ++i) all += vals[i];
    for (int r = 0; r < n && r < M; ++r) {
      int j = int(key2[r] & ((1 << 20) - 1));
      if (vals[j] > cutoff * vmax) {
        kept[sector[j]] += 1;
        kw += vals[j];
      }
    }
    out[0] = all - kw;
    out[1] = kw;
  }
  (void)tot;
}

void launch_select(int n, const double* vals, const int* sector, int n_sec, int M,
                   double cutoff, int* kept, double* out, cudaStream_t s) {
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  size_t smem = size_t(n2) * (sizeof(double) + sizeof(int));
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         kSelectMax * int(sizeof(double) + sizeof(int)));
  });
  k_select<<<1, 1024, smem, s>>>(n, vals, sector, n_sec, M, cutoff, kept, out);
  g_launches += 1;
}

// ================================================================ Davidson vectors
constexpr int kDotBlocks = 256;
constexpr int kDotChunk = 16;

__global__ void __launch_bounds__(256) k_multidot(int k, const double* __restrict__ vs, int64_t ld,
                                                  const double* __restrict__ x, int64_t n,
                                                  double* partial) {
  __shared__ double red[kDotChunk][256 / 32];
  const int tid = threadIdx.x;
  double acc[kDotChunk];
#pragma unroll
  for (int j = 0; j < kDotChunk; ++j) acc[j] = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * 256 + tid; i < n; i += int64_t(gridDim.x) * 256) {
    double xi = x[i];
#pragma unroll
    for (int j = 0; j < kDotChunk; ++j)
      if (j < k) acc[j] = fma(vs[j * ld + i], xi, acc[j]);
  }
#pragma unroll
  for (int j = 0; j < kDotChunk; ++j) {
    double v = acc[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[j][tid >> 5] = v;
  }
  __syncthreads();
  if (tid < kDotChunk && tid < k) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += red[tid][w];
    partial[int64_t(tid) * gridDim.x + blockIdx.x] = v;
  }
}

__global__ void k_reduce_partials(int k, const double* __restrict__ partial, int nblk, double* out,
                                  int stride) {
  __shared__ double red[256];
  int j = blockIdx.x;
  double v = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 256) v += partial[int64_t(j) * nblk + b];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[int64_t(j) * stride] = red[0];
}

void launch_multidot(int k, const double* vs, int64_t ld, const double* x, int64_t n,
                     double* partial, double* out, int out_stride, cudaStream_t s) {
  for (int j0 = 0; j0 < k; j0 += kDotChunk) {
    int kk = k - j0 < kDotChunk ? k - j0 : kDotChunk;
    k_multidot<<<kDotBlocks, 256, 0, s>>>(kk, vs + j0 * ld, ld, x, n, partial);
    g_launches += 1;
    k_reduce_partials<<<kk, 256, 0, s>>>(kk, partial, kDotBlocks, out + int64_t(j0) * out_stride,
                                         out_stride);
    g_launches += 1;
  }
}

__global__ void k_multiaxpy(int k, const double* __restrict__ vs, int64_t ld,
                            const double* __restrict__ c, double* y, int64_t n, double sign) {
  __shared__ double cc[64];
  if (threadIdx.x < k) cc[threadIdx.x] = c[threadIdx.x];
  __syncthreads();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma(cc[j], vs[j * ld + i], acc);
    y[i] = fma(sign, acc, y[i]);
  }
}

void launch_multiaxpy(int k, const double* vs, int64_t ld, const double* c, double* y,
                      int64_t n, double sign, cudaStream_t s) {
  k_multiaxpy<<<1024, 256, 0, s>>>(k, vs, ld, c, y, n, sign);
  g_launches += 1;
}

// Krylov exponential coefficients: c = U exp(-t (Lambda - lambda_min)) U^T e_1 for the
// k x k eigen-decomposition (evecs row-major, eigenvector j in column j; evals in any
// order).  stats[0] = |c|^2, stats[1] = lambda_min, stats[2] = max |lambda|.  One block.
__global__ void k_krylov_coef(int k, const double* __restrict__ evecs, const double* __restrict__ evals,
                              double t, double* c, double* stats) {
  __shared__ double f[64];
  __shared__ double lmin, lmax;
  if (threadIdx.x == 0) {
    double a = evals[0], b = fabs(evals[0]);
    for (int j = 1; j < k; ++j) {
      a = fmin(a, evals[j]);
      b = fmax(b, fabs(evals[j]));
    }
    lmin = a;
    lmax = b;
  }
  __syncthreads();
  if (threadIdx.x < k) f[threadIdx.x] = exp(-t * (evals[threadIdx.x] - lmin)) * evecs[threadIdx.x];
  __syncthreads();
  if (threadIdx.x < k) {
    double acc = 0.0;
    for (int j = 0; j < k; ++j) acc = fma(evecs[threadIdx.x * k + j], f[j], acc);
    c[threadIdx.x] = acc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int j = 0; j < k; ++j) s2 = fma(c[j], c[j], s2);
    stats[0] = s2;
    stats[1] = lmin;
    stats[2] = lmax;
  }
}

void launch_krylov_coef(int k, const double* evecs, const double* evals, double t, double* c,
                        double* stats, cudaStream_t s) {
  k_krylov_coef<<<1, 64, 0, s>>>(k, evecs, evals, t, c, stats);
  g_launches += 1;
}

__global__ void __launch_bounds__(256) k_ritz(int k, const double* __restrict__ V,
                                              const double* __restrict__ W, int64_t ld,
                                              const double* __restrict__ sv, int sld,
                                              const double* __restrict__ theta_p,
                                              const double* __restrict__ diag, double* u,
                                              double* hu, double* t, int64_t n, double* partial) {
  __shared__ double cc[64];
  __shared__ double red[8];
  if (threadIdx.x < k) cc[threadIdx.x] = sv[threadIdx.x * sld];
  __syncthreads();
  const double theta = *theta_p;
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * 256 + threadIdx.x; i < n; i += int64_t(gridDim.x) * 256) {
    double a = 0.0, b = 0.0;
    for (int j = 0; j < k; ++j) {
      a = fma(cc[j], V[j * ld + i], a);
      b = fma(cc[j], W[j * ld + i], b);
    }
    u[i] = a;
    hu[i] = b;
    double r = b - theta * a;
    acc = fma(r, r, acc);
    double den = diag[i] - theta;
    if (fabs(den) < 1e-8) den = 1e-8;
    t[i] = r / den;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int w = 0; w < 8; ++w) v += red[w];
    partial[blockIdx.x] = v;
  }
}

void launch_ritz(int k, const double* V, const double* W, int64_t ld, const double* small_evecs,
                 int small_ld, const double* theta, const double* diag, double* u, double* hu,
                 double* t, int64_t n, double* partial, double* out, cudaStream_t s) {
  k_ritz<<<kDotBlocks, 256, 0, s>>>(k, V, W, ld, small_evecs, small_ld, theta, diag, u, hu, t, n,
                                    partial);
  g_launches += 1;
  k_reduce_partials<<<1, 256, 0, s>>>(1, partial, kDotBlocks, out, 1);
  g_launches += 1;
}

// x *= |x|^-1 given |x|^2; the factor is formed once per block (FP64 division and square
// root are long sequences on GB300's FP64 pipe).  With flag: a norm below 1e-14 (a
// breakdown of the Davidson basis extension) zeroes x and sets *flag = 1.
__global__ void k_scale_inv_sqrt(double* x, int64_t n, const double* norm2, double* flag) {
  __shared__ double f;
  if (threadIdx.x == 0) {
    const double nn = *norm2;
    const bool ok = !flag || sqrt(nn) >= 1e-14;
    f = ok ? 1.0 / sqrt(nn) : 0.0;
    if (!ok && blockIdx.x == 0) *flag = 1.0;
  }
  __syncthreads();
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[i] *= f;
}

static int vec_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256;
  return int(b < 1 ? 1 : (b > 1024 ? 1024 : b));
}

void launch_scale_inv_sqrt(double* x, int64_t n, const double* norm2, cudaStream_t s,
                           double* flag) {
  k_scale_inv_sqrt<<<vec_blocks(n), 256, 0, s>>>(x, n, norm2, flag);
  g_launches += 1;
}

__global__ void k_axpby(double* x, const double* y, int64_t n, double a, double b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    x[i] = a * x[i] + b * y[i];
}

void launch_axpby(double* x, const double* y, int64_t n, double a, double b, cudaStream_t s) {
  k_axpby<<<1024, 256, 0, s>>>(x, y, n, a, b);
  g_launches += 1;
}

__global__ void k_symmetrize(int k, const double* vw, int kmax, double* g) {
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    int i = e / k, j = e % k;
    g[e] = 0.5 * (vw[i * kmax + j] + vw[j * kmax + i]);
  }
}

void launch_symmetrize(int k, const double* vw, int kmax, double* g, cudaStream_t s) {
  k_symmetrize<<<1, 256, 0, s>>>(k, vw, kmax, g);
  g_launches += 1;
}

}  // namespace b2k

namespace b2k {

__global__ void k_scale_cols(int m, const double* __restrict__ u, const double* __restrict__ lam,
                             double power, double floor_, int drop, double* out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x) {
    int c = e % m;
    const double l = lam[c];
    out[e] = (drop && l < floor_) ? 0.0 : u[e] * pow(fmax(l, floor_), power);
  }
}

void launch_scale_cols(int m, const double* u, const double* lam, double power, double floor_,
                       double* out, cudaStream_t s, bool drop_below) {
  int blocks = (m * m + 255) / 256;
  if (blocks > 1024) blocks = 1024;
  k_scale_cols<<<blocks, 256, 0, s>>>(m, u, lam, power, floor_, drop_below ? 1 : 0, out);
  g_launches += 1;
}

}  // namespace b2k

namespace b2k {

__global__ void __launch_bounds__(256) k_dots(const DotOut* __restrict__ outs,
                                              const DotTerm* __restrict__ terms,
                                              const double* __restrict__ A,
                                              const double* __restrict__ B, double* out) {
  __shared__ double red[256];
  const DotOut o = outs[blockIdx.x];
  double acc = 0.0;
  for (int t = o.t0; t < o.t1; ++t) {
    const DotTerm d = terms[t];
    double part = 0.0;
    for (int e = threadIdx.x; e < d.n; e += 256) part = fma(A[d.offA + e], B[d.offB + e], part);
    acc = fma(d.sign, part, acc);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

void launch_dots(int n_out, const DotOut* outs, const DotTerm* terms, const double* A,
                 const double* B, double* out, cudaStream_t s) {
  if (n_out <= 0) return;
  k_dots<<<n_out, 256, 0, s>>>(outs, terms, A, B, out);
  g_launches += 1;
}

}  // namespace b2k
