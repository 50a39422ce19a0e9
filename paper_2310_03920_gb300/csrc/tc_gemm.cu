// Split-precision block contraction on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Same task lists as the FP64 kernel (kernels.cuh): each output block receives
//   3-operand terms  alpha * op(P) X op(Q)      or   2-operand terms  alpha * op(P) op(X).
// Every FP64 operand element a is split into bf16 hi = bf16(a) and lo = bf16(a - hi) (formed
// in FP32 after one rounding of a to FP32, see split()); a
// product a*b is formed as hi*hi + hi*lo + lo*hi on the tensor cores with FP32
// accumulation in tensor memory (TMEM); the FP32 tile is added to the FP64 output at the
// end.  One CTA (8 warps) owns a 128 x 128 output tile:
//   3-operand term, per 64-wide chunk c of K2:
//     T  = op(P)[tile rows, :] X[:, c]        (tcgen05.mma, TMEM columns [0, 64))
//     T  -> registers, times alpha, split, back to shared memory (A operand)
//     acc += T op(Q)[c, tile cols]            (tcgen05.mma, TMEM columns [128, 256))
//   2-operand term: acc += (alpha op(P)) op(X) directly.
// Operands are staged by the threads (converting while they store) into the canonical
// K-major no-swizzle layout: 8 x 16-byte core matrices, consecutive along K at 128 bytes
// (LBO), 8-row groups at 1024 bytes (SBO) for a 64-wide K chunk.  One thread issues the
// MMAs; completion is signalled through an mbarrier whose waits are bounded: a wait that
// runs out sets the status word, waits (bounded) once more for the MMAs in flight, frees
// TMEM and returns.
#include <cuda_bf16.h>

#include <cstdint>

#include <mutex>

#include "kernels.cuh"

namespace b2k {

namespace {

constexpr int kRows = 128;       // output tile rows (MMA M)
constexpr int kCols = 128;       // output tile columns (max MMA N of the second product)
constexpr int kKc = 64;          // K chunk staged in shared memory
constexpr int kTmemCols = 256;   // T at [0, 64), accumulator at [128, 256)
constexpr int kTileBytes = kRows * kKc * 2;   // one bf16 [128 x 64] K-major tile
constexpr uint32_t kWaitLimit = 1u << 26;
// 8 warps: all stage operands (twice the loads in flight of 4 warps); TMEM is read by warp w
// in lane quarter w % 4, the two warpgroups taking alternate 16-column chunks
constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major no-swizzle offset of element (r, k) in a [rows x 64] tile
__device__ __forceinline__ uint32_t koff(int r, int k) {
  return uint32_t((r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = uint64_t((addr >> 4) & 0x3FFF);
  d |= uint64_t(128 >> 4) << 16;    // LBO: next core matrix along K
  d |= uint64_t(1024 >> 4) << 32;   // SBO: next 8-row group
  d |= uint64_t(1) << 46;           // tcgen05 descriptor version
  return d;                         // base offset 0, no swizzle
}

__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(kRows >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                    uint32_t accum) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(bar)));
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t phase) {
  uint32_t done = 0;
  for (uint32_t it = 0; it < kWaitLimit && !done; ++it) {
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(phase));
  }
  return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// hi = bf16(x), lo = bf16(x - hi), formed in FP32: x is rounded to FP32 once (relative
// error 2^-24, far below the 2^-17 that hi + lo resolves), then f - hi is exact in FP32.
// GB300's FP64 pipe is narrow, so the staging loops keep FP64 work to the one conversion.
__device__ __forceinline__ void split(float f, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(f);
  lo = __float2bfloat16_rn(f - __bfloat162float(hi));
}

// Stage op(M)[r0 + i][c0 + k] (i < rows_tile, k < kw; zero outside rows x cols) as the
// K-major operand (row i, K index k), scaled by s, into hi/lo tiles.  kw (a multiple of 16)
// covers the K-steps the MMA will read; rows >= rows_tile are left as they are (zero).
// Each thread loads kStageBatch elements before converting any of them, so that many L2 /
// HBM loads are in flight per thread (the staging is bound by load latency).
constexpr int kStageBatch = 4;
__device__ __forceinline__ void stage_rowmajor(unsigned char* hi, unsigned char* lo, const double* M,
                                               int ld, int rows, int cols, int r0, int c0,
                                               bool trans, int rows_tile, int kw, double s,
                                               int tid) {
  const int n = rows_tile * kw;
  const float sf = static_cast<float>(s);
  for (int e0 = tid; e0 < n; e0 += kThreads * kStageBatch) {
    double v[kStageBatch];
    uint32_t off[kStageBatch];
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      const int e = e0 + u * kThreads;
      int i = 0, k = 0;
      if (!trans) {
        i = e / kw;
        k = e - i * kw;
      } else {
        k = e / rows_tile;
        i = e - k * rows_tile;
      }
      const int r = r0 + i, c = c0 + k;
      const bool in = e < n && r < rows && c < cols;
      v[u] = in ? (trans ? M[int64_t(c) * ld + r] : M[int64_t(r) * ld + c]) : 0.0;
      off[u] = e < n ? koff(i, k) : 0xffffffffu;
    }
#pragma unroll
    for (int u = 0; u < kStageBatch; ++u) {
      if (off[u] == 0xffffffffu) continue;
      __nv_bfloat16 h, l;
      split(sf * static_cast<float>(v[u]), h, l);
      *reinterpret_cast<__nv_bfloat16*>(hi + off[u]) = h;
      *reinterpret_cast<__nv_bfloat16*>(lo + off[u]) = l;
    }
  }
}

}  // namespace

__device__ __forceinline__ void gemm_tc_item(const GemmTile& tile, const GemmOut* __restrict__ outs,
                                             const GemmTerm* __restrict__ terms, const BufTable& bt,
                                             int* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* a_hi = base;                       // A operand (128 x 64)
  unsigned char* a_lo = base + kTileBytes;
  unsigned char* b_hi = base + 2 * kTileBytes;      // B operand (<= 128 x 64)
  unsigned char* b_lo = base + 3 * kTileBytes;
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_slot;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const GemmOut o = outs[tile.out];
  const int r0 = tile.r0, c0 = tile.c0;
  const int nt = min(kCols, o.N - c0);
  const int n_acc = ((nt + 15) / 16) * 16;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;
  const uint32_t tmem_t = tmem, tmem_acc = tmem + 128;
  const int quad = warp & 3, wg = warp >> 2;   // TMEM lane quarter, warpgroup
  const uint32_t lane_off = uint32_t(quad * 32) << 16;

  // rows of the A operand beyond the output block stay zero for every term
  const int m_rows = min(kRows, o.M - r0);
  for (int e = tid; e < kTileBytes / 16; e += kThreads) {
    reinterpret_cast<uint4*>(a_hi)[e] = make_uint4(0, 0, 0, 0);
    reinterpret_cast<uint4*>(a_lo)[e] = make_uint4(0, 0, 0, 0);
  }
  uint32_t phase = 0;
  bool ok = true, started = false;
  const uint32_t ia = smem_u32(a_hi), ial = smem_u32(a_lo), ib = smem_u32(b_hi), ibl = smem_u32(b_lo);

  // issue hi*hi + hi*lo + lo*hi over ksteps K-steps into tmem_d, then wait
  auto run_mma = [&](uint32_t tmem_d, int n, int ksteps, bool accum_first) -> bool {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (tid == 0) {
      const uint32_t id = idesc_bf16(n);
      for (int ks = 0; ks < ksteps; ++ks) {
        const uint32_t off = uint32_t(ks) * 256;
        mma(tmem_d, sdesc(ia + off), sdesc(ib + off), id, (accum_first || ks > 0) ? 1u : 0u);
        mma(tmem_d, sdesc(ia + off), sdesc(ibl + off), id, 1u);
        mma(tmem_d, sdesc(ial + off), sdesc(ib + off), id, 1u);
      }
      commit(&bar);
    }
    // every thread waits; the outcome is made uniform so that no barrier diverges
    const int done = __syncthreads_and(wait_bar(&bar, phase) ? 1 : 0);
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;");
    return done != 0;
  };

  for (int t = o.t0; t < o.t1 && ok; ++t) {
    const GemmTerm g = terms[t];
    const double* P = bt.p[g.bufP] + g.offP;
    const double* X = bt.p[g.bufX] + g.offX;
    const bool tP = g.flags & kTransP, tQ = g.flags & kTransQ;
    if (g.flags & kTwoOp) {
      for (int k0 = 0; k0 < g.K1 && ok; k0 += kKc) {
        const int kc = min(kKc, g.K1 - k0);
        const int kw = ((kc + 15) / 16) * 16;
        stage_rowmajor(a_hi, a_lo, P, g.ldP, o.M, g.K1, r0, k0, tP, m_rows, kw, g.alpha, tid);
        // B operand row n = output column c0 + n, K index k: op(X)[k0 + k][c0 + n]
        stage_rowmajor(b_hi, b_lo, X, g.ldX, o.N, g.K1, c0, k0, !tQ, n_acc, kw, 1.0, tid);
        ok = run_mma(tmem_acc, n_acc, (kc + 15) / 16, started);
        started = true;
      }
    } else {
      const double* Q = bt.p[g.bufQ] + g.offQ;
      for (int k2 = 0; k2 < g.K2 && ok; k2 += kKc) {
        const int kc2 = min(kKc, g.K2 - k2);
        const int n_t = ((kc2 + 15) / 16) * 16;
        // T = op(P)[rows, :] X[:, k2:k2+64]
        for (int k1 = 0; k1 < g.K1 && ok; k1 += kKc) {
          const int kc1 = min(kKc, g.K1 - k1);
          const int kw1 = ((kc1 + 15) / 16) * 16;
          stage_rowmajor(a_hi, a_lo, P, g.ldP, o.M, g.K1, r0, k1, tP, m_rows, kw1, 1.0, tid);
          // B operand row n = column k2 + n of X, K index k = row k1 + k of X
          stage_rowmajor(b_hi, b_lo, X, g.ldX, g.K2, g.K1, k2, k1, true, n_t, kw1, 1.0, tid);
          ok = run_mma(tmem_t, n_t, (kc1 + 15) / 16, k1 > 0);
        }
        if (!ok) break;
        // T (FP32, row = thread) -> alpha * T split into the A operand
        if (quad * 32 < m_rows) {   // warps holding only rows past the block: T is zero there
          const int row = quad * 32 + lane;
          const float af = static_cast<float>(g.alpha);
          for (int cc = wg * 16; cc < n_t; cc += 32) {
            float v[16];
            tmem_ld16(tmem_t + lane_off + uint32_t(cc), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
              __nv_bfloat16 h, l;
              split(af * v[j], h, l);
              uint32_t off = koff(row, cc + j);
              *reinterpret_cast<__nv_bfloat16*>(a_hi + off) = h;
              *reinterpret_cast<__nv_bfloat16*>(a_lo + off) = l;
            }
          }
        }
        // B operand row n = output column c0 + n, K index k: op(Q)[k2 + k][c0 + n]
        stage_rowmajor(b_hi, b_lo, Q, g.ldQ, o.N, g.K2, c0, k2, !tQ, n_acc, n_t, 1.0, tid);
        ok = run_mma(tmem_acc, n_acc, (kc2 + 15) / 16, started);
        started = true;
      }
    }
  }

  if (ok) {
    double* out = bt.p[o.buf] + o.off;
    const int row = quad * 32 + lane;
    const int r = r0 + row;
    for (int cc = wg * 16; cc < n_acc; cc += 32) {
      float v[16];
      if (started) {
        tmem_ld16(tmem_acc + lane_off + uint32_t(cc), v);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = 0.f;
      }
      if (r < o.M) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          int c = c0 + cc + j;
          if (cc + j < nt) {
            double* p = out + int64_t(r) * o.ld + c;
            *p = o.accumulate ? *p + double(v[j]) : double(v[j]);
          }
        }
      }
    }
  } else {
    if (tid == 0) atomicExch(status, 1);
    wait_bar(&bar, phase);   // bounded: let MMAs in flight finish before freeing TMEM
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

__global__ void __launch_bounds__(kThreads, 2) k_gemm_tc(const GemmTile* __restrict__ tiles,
                                                 const GemmOut* __restrict__ outs,
                                                 const GemmTerm* __restrict__ terms, BufTable bt,
                                                 int* status) {
  gemm_tc_item(tiles[blockIdx.x], outs, terms, bt, status);
}

// Grouped launch over several problems: CTA b takes tile b - tile0 of the group g with
// tile0(g) <= b < tile0(g + 1).
__global__ void __launch_bounds__(kThreads, 2) k_gemm_tc_grouped(const GemmGroupTc* __restrict__ groups,
                                                         int n_groups, int* status) {
  int lo = 0, hi = n_groups - 1;
  const int b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (groups[mid].tile0 <= b) lo = mid; else hi = mid - 1;
  }
  const GemmGroupTc& G = groups[lo];
  const BufTable bt = G.bt;
  gemm_tc_item(G.tiles[b - G.tile0], G.outs, G.terms, bt, status);
}

size_t gemm_tc_smem() { return size_t(4) * kTileBytes + 1024; }

void launch_gemm_tc(const GemmTile* tiles, int n_tiles, const GemmOut* outs, const GemmTerm* terms,
                    const BufTable& bt, int* status, cudaStream_t s) {
  if (n_tiles <= 0) return;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(gemm_tc_smem()));
  });
  k_gemm_tc<<<n_tiles, kThreads, gemm_tc_smem(), s>>>(tiles, outs, terms, bt, status);
  count_launches(1);
}

void launch_gemm_tc_grouped(const GemmGroupTc* groups, int n_groups, int n_tiles, int* status,
                            cudaStream_t s) {
  if (n_groups <= 0 || n_tiles <= 0) return;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_gemm_tc_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         int(gemm_tc_smem()));
  });
  k_gemm_tc_grouped<<<n_tiles, kThreads, gemm_tc_smem(), s>>>(groups, n_groups, status);
  count_launches(1);
}

}  // namespace b2k
