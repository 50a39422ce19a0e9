// Split-precision H_eff contraction on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// Operands.  Every FP64 operand a is split once into hi + lo (bf16 x3: hi = bf16(a),
// lo = bf16(a - hi); tf32 x3: the same with tf32, i.e. FP32 with 13 low mantissa bits
// dropped) and stored "pre-tiled": a block of R rows (the M or N index of the product) and
// K columns (the contraction index) is padded with zeros to Rp = round16(R) rows and
// Kp = round16(K) columns and laid out in 128-byte chunks of K; chunk c holds, for every
// 8-row group, the 16-byte pieces of its kg_c k-groups ([row group][k-group][row][16 B]).
// This is the canonical K-major no-swizzle operand layout of tcgen05 (8 x 16-byte core
// matrices, LBO = 128 bytes between k-groups, SBO = kg_c * 128 bytes between row groups),
// so a 128-row sub-tile of one K chunk is one contiguous run of bytes that a single
// cp.async.bulk moves into shared memory.  The environments (and their precombined
// operators) are split once per window and reused by every Davidson product; psi is split
// (transposed: rows = its columns m_r, K = its rows m_l) once per product.
//
// Contraction.  An output tile (64 rows x <= 64 columns of one psi block; two CTAs per SM)
// receives
//   sum over terms t, over 128-byte chunks c of K2 = m_r:
//     T   = L_t[tile rows, :] psi_t[:, c]          (MMA1, FP32 in TMEM, K = m_l)
//     T'  = split(alpha_t * T)                     (TMEM -> registers -> shared memory)
//     acc += T' R_t[tile cols, c]^T                 (MMA2, FP32 in TMEM)
// each product formed as hi*hi + hi*lo + lo*hi; the FP32 accumulator is added to the FP64
// output block every kGroup chain units.
//
// Roles (6 warps): the producer warp streams operand chunks through a byte ring of shared
// memory with cp.async.bulk (completion on the item's mbarrier) and is the only reader of
// the term list; one thread of the MMA warp issues the MMAs; four converter warps (TMEM lane
// quarters 0 and 1, two warps per quarter on the two column halves) convert T into T' and
// add the accumulators to the output.  The MMA thread computes T of the next chain unit
// while the converters work on the current one (two T buffers in TMEM, two T' buffers in
// shared memory); the sum over a tile's units runs in groups of kGroup units in two TMEM
// accumulators, each group added to the FP64 output by the converter warps while the other
// accumulator fills.  Every wait is bounded: a wait that runs out sets the CTA's abort flag
// and the status word; the other roles then stop, the producer waits (with the full limit)
// for its copies in flight, the MMA thread for its MMAs, TMEM is freed and the CTA returns.
// For tests of that path, stuck_polls > 0 makes the MMA thread first wait that many polls on
// a barrier nothing arrives on.
#include <cuda_bf16.h>

#include <cstdint>
#include <mutex>

#include "kernels.cuh"

namespace b2k {

namespace {

// Operand chunks stream through a byte ring of shared memory: each item (the chunks one
// MMA group reads: L and psi^T for MMA1, R for MMA2, hi and lo planes) takes exactly its
// size, so many small blocks are in flight at once; at most kSlots items are outstanding.
constexpr int kSlots = 16;
// Two CTAs per SM (two MMA-issuing threads): an output tile is kTcTileM x kTcTileN (the
// MMAs keep M = 128; accumulator rows past the tile are discarded)
constexpr int kTileM = kTcTileM, kTileN = kTcTileN;
constexpr int kPBytes = 128 * 128;                   // 128 rows x one 128-byte K chunk
constexpr int kTpBytes = 2 * kPBytes;                // T' hi + lo (follows the ring: an A
                                                     // operand read past its item's rows stays
                                                     // inside shared memory)
constexpr int kRingBytes = 40 * 1024;
constexpr int kDynSmem = kRingBytes + 2 * kTpBytes + 1024;
// warps: 2 producer, 3 MMA issuer, 0 1 4 5 converters (TMEM lane quarters 0 and 1 hold the
// tile's rows; the two warps of a quarter take the two halves of the columns)
constexpr int kThreads = 192;
constexpr int kProducerWarp = 2, kMmaWarp = 3;
constexpr int kConv = 128;                           // converter threads (4 warps)
// TMEM columns: T0 [0,64), T1 [64,128), acc0 [128,192), acc1 [192,256)
constexpr int kTmemCols = 256;
// chain units summed in one FP32 accumulator before it is added to the FP64 output: bounds
// the FP32 rounding error of the long term sums (thousands of terms per output block)
constexpr int kGroup = 64;
constexpr uint32_t kDefaultWait = 1u << 22;
constexpr uint32_t kDrainWait = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// K-major no-swizzle shared-memory descriptor: start, LBO = 128 (k-groups), SBO (row groups)
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t sbo) {
  uint64_t d = uint64_t((addr >> 4) & 0x3FFF);
  d |= uint64_t(128 >> 4) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFF) << 32;
  d |= uint64_t(1) << 46;   // descriptor version of tcgen05
  return d;
}

// instruction descriptor: FP32 accumulator, A and B K-major, M = 128, N = n;
// operand type 1 = bf16 (kind::f16), 2 = tf32 (kind::tf32)
__device__ __forceinline__ uint32_t idesc(int n, bool tf32) {
  const uint32_t ty = tf32 ? 2u : 1u;
  return (1u << 4) | (ty << 7) | (ty << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(128 >> 4) << 24);
}

__device__ __forceinline__ void mma(bool tf32, uint32_t tmem, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t accum) {
  if (tf32)
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(accum));
  else
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem),
        "l"(a), "l"(b), "r"(id), "r"(accum));
}

// hi*hi + hi*lo + lo*hi of one K-step into tmem (descriptors of the hi and lo planes)
__device__ __forceinline__ void mma3(bool tf32, uint32_t tmem, uint64_t ah, uint64_t al,
                                     uint64_t bh, uint64_t bl, uint32_t id, uint32_t accum) {
  mma(tf32, tmem, ah, bh, id, accum);
  mma(tf32, tmem, ah, bl, id, 1u);
  mma(tf32, tmem, al, bh, id, 1u);
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void bar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void bar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool bar_try(uint64_t* bar, uint32_t parity) {
  uint32_t done = 0;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait that also gives up once another role has aborted the CTA
__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, uint32_t limit,
                                         volatile int* abort_flag) {
  for (uint32_t it = 0; it < limit; ++it) {
    if (bar_try(bar, parity)) return true;
    if (*abort_flag) return false;
  }
  return false;
}

// bounded wait used while draining: never cut short
__device__ __forceinline__ bool bar_drain(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kDrainWait; ++it)
    if (bar_try(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
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

// tf32 rounding of an FP32 value: nearest on the magnitude (ties away from zero), the 13
// low mantissa bits cleared
__device__ __forceinline__ uint32_t tf32_bits(float f) {
  return (__float_as_uint(f) + 0x1000u) & 0xFFFFE000u;
}

// split f into (hi, lo) of the operand type, packed as raw bits: bf16 -> 16 bits each
__device__ __forceinline__ void split_bf16(float f, uint16_t& hi, uint16_t& lo) {
  const __nv_bfloat16 h = __float2bfloat16_rn(f);
  const __nv_bfloat16 l = __float2bfloat16_rn(f - __bfloat162float(h));
  hi = __bfloat16_as_ushort(h);
  lo = __bfloat16_as_ushort(l);
}
__device__ __forceinline__ void split_tf32(float f, uint32_t& hi, uint32_t& lo) {
  hi = tf32_bits(f);
  lo = tf32_bits(f - __uint_as_float(hi));
}

__host__ __device__ __forceinline__ int pad16(int x) { return (x + 15) & ~15; }

}  // namespace

// byte offset of chunk c of a pre-tiled block of rp rows (chunks before c are full)
__host__ __device__ __forceinline__ int64_t tc_chunk_off(int rp, int c) {
  return int64_t(c) * rp * 128;
}
// k-groups (16 bytes) of chunk c of a block with kp padded columns of es-byte elements
__host__ __device__ __forceinline__ int tc_chunk_kg(int kp, int es, int c) {
  const int rem = kp * es / 16 - 8 * c;
  return rem < 8 ? rem : 8;
}

// ------------------------------------------------------------------ operand split
// One CTA per block: every 16-byte piece (row r, k-group j) of the padded pre-tiled block,
// rows fastest so that consecutive threads read consecutive rows.
__global__ void __launch_bounds__(256) k_split(const SplitTask* __restrict__ tasks,
                                               BufTable bt, uint8_t* hi, uint8_t* lo, int tf32) {
  const SplitTask tk = tasks[blockIdx.x];
  const double* src = bt.p[tk.buf] + tk.src;
  const int es = tf32 ? 4 : 2;
  const int per = 16 / es;                     // elements per 16-byte piece
  const int kgt = tk.kp * es / 16;             // k-groups over all chunks
  const int64_t n_units = int64_t(tk.rp) * kgt;
  const int64_t base = tk.dst * es;
  for (int64_t u = threadIdx.x; u < n_units; u += blockDim.x) {
    const int r = int(u % tk.rp), j = int(u / tk.rp);
    const int c = j >> 3, jj = j & 7;
    const int kg = tc_chunk_kg(tk.kp, es, c);
    const int64_t off = base + tc_chunk_off(tk.rp, c) + int64_t(r >> 3) * kg * 128 + jj * 128 + (r & 7) * 16;
    float f[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int k = j * per + e;
      double v = 0.0;
      if (e < per && r < tk.rows && k < tk.cols)
        v = tk.trans ? src[int64_t(k) * tk.ld + r] : src[int64_t(r) * tk.ld + k];
      f[e] = static_cast<float>(v);
    }
    uint4 h, l;
    if (tf32) {
      uint32_t hh[4], ll[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) split_tf32(f[e], hh[e], ll[e]);
      h = make_uint4(hh[0], hh[1], hh[2], hh[3]);
      l = make_uint4(ll[0], ll[1], ll[2], ll[3]);
    } else {
      uint16_t hh[8], ll[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) split_bf16(f[e], hh[e], ll[e]);
      h = make_uint4(hh[0] | (uint32_t(hh[1]) << 16), hh[2] | (uint32_t(hh[3]) << 16),
                     hh[4] | (uint32_t(hh[5]) << 16), hh[6] | (uint32_t(hh[7]) << 16));
      l = make_uint4(ll[0] | (uint32_t(ll[1]) << 16), ll[2] | (uint32_t(ll[3]) << 16),
                     ll[4] | (uint32_t(ll[5]) << 16), ll[6] | (uint32_t(ll[7]) << 16));
    }
    *reinterpret_cast<uint4*>(hi + off) = h;
    *reinterpret_cast<uint4*>(lo + off) = l;
  }
}

// ------------------------------------------------------------------ the contraction
namespace {
constexpr int kTermBatch = 64;   // terms copied into shared memory per bulk copy
constexpr int kUnitRing = 32;    // unit descriptors in flight between producer and converter
// what the MMA thread needs of one ring item (written by the producer before the item's
// copies are armed, so the full barrier orders it)
struct ItemMeta {
  uint32_t pos;      // ring offset of the item
  uint32_t a, b;     // bytes of one plane of the first / second operand
  uint16_t kg, n1;   // k-groups of the chunk, T columns of the unit
  uint8_t kind;      // 0: MMA1 chunk, 1: MMA2
  uint8_t first, last;   // MMA1: first / last K1 chunk of the unit; MMA2: last unit of the tile
};
// what the converter needs of one chain unit
struct UnitMeta {
  float alpha;
  int n1;
  int last;          // last unit of the tile
};
}  // namespace

__device__ __forceinline__ void heff_tc_tile(const TcGroup& G, const TcTile tile, int* status,
                                             uint32_t stuck_polls, bool tf32) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t full[kSlots], empty[kSlots];
  __shared__ __align__(8) uint64_t tfull[2], tempty[2], tpready[2], tpempty[2], drainb;
  __shared__ __align__(8) uint64_t accfull[2], accempty[2];
  __shared__ __align__(8) uint64_t ufull[kUnitRing], uempty[kUnitRing], tbfull[2];
  __shared__ __align__(8) uint64_t neverb;   // nothing arrives on it (failure-path tests)
  __shared__ __align__(16) TcTerm tbatch[2][kTermBatch];
  __shared__ ItemMeta imeta[kSlots];
  __shared__ UnitMeta umeta[kUnitRing];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* ring = base;
  unsigned char* tp_mem = base + kRingBytes;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int es = tf32 ? 4 : 2;
  const int wk = 128 / es;   // elements in one 128-byte K chunk (= T columns per unit)
  const TcOut o = G.outs[tile.out];
  const int r0 = tile.r0, c0 = tile.c0;
  const int n2 = pad16(min(kTileN, o.N - c0));        // MMA2 N (acc columns)
  const int rowsA = min(kTileM, pad16(o.M) - r0);     // L rows loaded for this tile
  const int rowsB2 = min(kTileN, pad16(o.N) - c0);    // R rows loaded for this tile
  const uint32_t limit = kDefaultWait;

  if (tid == 0) {
    for (int s = 0; s < kSlots; ++s) {
      bar_init(&full[s], 1);
      bar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      bar_init(&tfull[b], 1);
      bar_init(&tempty[b], kConv);
      bar_init(&tpready[b], kConv);
      bar_init(&tpempty[b], 1);
      bar_init(&accfull[b], 1);
      bar_init(&accempty[b], kConv);
      bar_init(&tbfull[b], 1);
    }
    for (int k = 0; k < kUnitRing; ++k) {
      bar_init(&ufull[k], 1);
      bar_init(&uempty[k], kConv);
    }
    bar_init(&drainb, 1);
    bar_init(&neverb, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_slot;

  auto fail = [&]() {
    abort_flag = 1;
    atomicExch(status, 1);
  };
  auto nchunks = [&](int k) { return (pad16(k) * es + 127) / 128; };
  const int n_terms = o.t1 - o.t0;

  if (warp == kProducerWarp) {
    // ------------------------------------------------------------ producer
    // The only role that reads the term list: batches of kTermBatch terms are copied into
    // shared memory two ahead; every item carries what the MMA thread needs (imeta), every
    // unit what the converter needs (umeta).
    if (lane == 0) {
      uint32_t item = 0, oldest = 0;   // items issued / first item not known consumed
      uint32_t head = 0, used = 0;     // next ring offset, bytes held by in-flight items
      uint32_t foot[kSlots];           // ring bytes of the in-flight item of each slot
      bool ok = true;
      const int n_batches = (n_terms + kTermBatch - 1) / kTermBatch;
      auto issue_batch = [&](int bt) {
        const int cnt = min(kTermBatch, n_terms - bt * kTermBatch);
        const uint32_t bytes = uint32_t(cnt) * uint32_t(sizeof(TcTerm));
        bar_expect_tx(&tbfull[bt & 1], bytes);
        bulk_g2s(smem_u32(&tbatch[bt & 1][0]), G.terms + o.t0 + bt * kTermBatch, bytes,
                 &tbfull[bt & 1]);
      };
      int cur_batch = -1;
      // term t (relative to o.t0), waiting for its batch and arming the one after it (the
      // slot it goes to held the batch before this one, which this thread has finished)
      auto term = [&](int t, TcTerm& tm) -> bool {
        const int bt = t / kTermBatch;
        if (bt != cur_batch) {
          if (!bar_wait(&tbfull[bt & 1], (bt >> 1) & 1, limit, &abort_flag)) {
            if (!abort_flag) fail();
            return false;
          }
          cur_batch = bt;
          if (bt + 1 < n_batches && bt >= 1) {
            // this thread's reads of the slot (batch bt - 1) come before the copy's writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue_batch(bt + 1);
          }
        }
        tm = tbatch[bt & 1][t % kTermBatch];
        return true;
      };
      // the oldest in-flight item has been consumed: its bytes are free again
      auto retire = [&]() -> bool {
        const int s = int(oldest % kSlots);
        if (!bar_wait(&empty[s], (oldest / kSlots) & 1, limit, &abort_flag)) {
          if (!abort_flag) fail();
          return false;
        }
        used -= foot[s];
        ++oldest;
        return true;
      };
      // a slot and sz contiguous ring bytes (wrapping to offset 0 when the end is too close;
      // the skipped bytes count with the item until it is consumed)
      auto acquire = [&](uint32_t sz, int& s, uint32_t& pos) -> bool {
        while (item - oldest >= uint32_t(kSlots))
          if (!retire()) return false;
        for (;;) {
          if (oldest == item) head = 0;   // empty ring: start at 0, so any item fits
          const bool fits = head + sz <= uint32_t(kRingBytes);
          const uint32_t fp = fits ? sz : (uint32_t(kRingBytes) - head) + sz;
          if (fp <= uint32_t(kRingBytes) - used) {
            pos = fits ? head : 0;
            s = int(item % kSlots);
            foot[s] = fp;
            used += fp;
            head = pos + sz;
            return true;
          }
          if (oldest == item || !retire()) {   // (an item never exceeds the ring)
            if (!abort_flag) fail();
            return false;
          }
        }
      };
      // Y item of a unit (R chunk), from the values kept when its X items were produced
      struct PendY {
        int64_t offB2;
        int K2, c;
        bool last;
      };
      auto produce_y = [&](const PendY& py) -> bool {
        const int kg = tc_chunk_kg(pad16(py.K2), es, py.c);
        const uint32_t b = uint32_t(rowsB2) * kg * 16;
        int s;
        uint32_t pos;
        if (!acquire(2 * b, s, pos)) return false;
        imeta[s] = ItemMeta{pos, b, 0, uint16_t(kg), uint16_t(pad16(min(wk, py.K2 - py.c * wk))),
                            1, 0, uint8_t(py.last ? 1 : 0)};
        const int64_t oR = py.offB2 * es + tc_chunk_off(pad16(o.N), py.c) + int64_t(c0 >> 3) * kg * 128;
        const uint32_t st = smem_u32(ring + pos);
        bar_expect_tx(&full[s], 2 * b);
        bulk_g2s(st, G.env_hi + oR, b, &full[s]);
        bulk_g2s(st + b, G.env_lo + oR, b, &full[s]);
        ++item;
        return true;
      };
      issue_batch(0);
      if (n_batches > 1) issue_batch(1);
      // item order: X(0), X(1), then X(u+2), Y(u): T of a unit is computed two units before
      // its product with R, so the MMA thread never waits for a conversion to start the
      // next T (two T buffers)
      uint32_t ui = 0;   // units produced
      PendY pend[2] = {};
      for (int t = 0; t < n_terms && ok && !abort_flag; ++t) {
        TcTerm tm;
        if (!(ok = term(t, tm))) break;
        const int nch2 = nchunks(tm.K2), nch1 = nchunks(tm.K1);
        const int kp1 = pad16(tm.K1), rp1 = pad16(tm.K2);
        for (int c2 = 0; c2 < nch2 && ok; ++c2, ++ui) {
          const bool last_unit = (t == n_terms - 1) && (c2 == nch2 - 1);
          const int n1 = pad16(min(wk, int(tm.K2) - c2 * wk));
          // the converter's descriptor of this unit
          const int k = int(ui % kUnitRing);
          if (ui >= uint32_t(kUnitRing) &&
              !bar_wait(&uempty[k], ((ui / kUnitRing) & 1) ^ 1, limit, &abort_flag)) {
            if (!abort_flag) fail();
            ok = false;
            break;
          }
          umeta[k] = UnitMeta{tm.alpha, n1, last_unit ? 1 : 0};
          bar_arrive(&ufull[k]);
          // X items: the K1 chunks of L and psi^T
          const int rowsB1 = min(wk, rp1 - c2 * wk);
          for (int c = 0; c < nch1; ++c) {
            const int kg = tc_chunk_kg(kp1, es, c);
            const uint32_t bA = uint32_t(rowsA) * kg * 16, bB = uint32_t(rowsB1) * kg * 16;
            int s;
            uint32_t pos;
            if (!(ok = acquire(2 * (bA + bB), s, pos))) break;
            imeta[s] = ItemMeta{pos, bA, bB, uint16_t(kg), uint16_t(n1), 0, uint8_t(c == 0),
                                uint8_t(c == nch1 - 1)};
            const int64_t oA = tm.offA * es + tc_chunk_off(pad16(o.M), c) + int64_t(r0 >> 3) * kg * 128;
            const int64_t oB = tm.offB1 * es + tc_chunk_off(rp1, c) + int64_t((c2 * wk) >> 3) * kg * 128;
            const uint32_t st = smem_u32(ring + pos);
            bar_expect_tx(&full[s], 2 * (bA + bB));
            bulk_g2s(st, G.env_hi + oA, bA, &full[s]);
            bulk_g2s(st + bA, G.env_lo + oA, bA, &full[s]);
            bulk_g2s(st + 2 * bA, G.psi_hi + oB, bB, &full[s]);
            bulk_g2s(st + 2 * bA + bB, G.psi_lo + oB, bB, &full[s]);
            ++item;
          }
          if (!ok) break;
          // then the Y item of the unit two back
          if (ui >= 2 && !(ok = produce_y(pend[ui & 1]))) break;
          pend[ui & 1] = PendY{tm.offB2, int(tm.K2), c2, last_unit};
        }
      }
      // the last two units' Y items
      for (uint32_t u = ui >= 2 ? ui - 2 : 0; u < ui && ok && !abort_flag; ++u)
        ok = produce_y(pend[u & 1]);
      // drain: every copy issued has landed before the CTA can exit (items already
      // consumed complete at once); the term batches too
      for (uint32_t i = oldest; i < item; ++i)
        if (!bar_drain(&full[i % kSlots], (i / kSlots) & 1)) fail();
      if (cur_batch + 1 < n_batches) {   // batches armed but never waited for
        for (int bt = cur_batch + 1; bt < min(n_batches, max(cur_batch, 0) + 2); ++bt)
          if (!bar_drain(&tbfull[bt & 1], (bt >> 1) & 1)) fail();
      }
    }
    __syncwarp();
  } else if (warp == kMmaWarp) {
    // ------------------------------------------------------------ MMA issuer
    // Items in the producer's order.  Descriptors are formed once per item and stepped by
    // 256 bytes (16 in descriptor units) per K-step: this single thread issues every MMA,
    // so its instruction count per unit bounds the kernel.
    if (lane == 0) {
      uint32_t item = 0, ix = 0, iy = 0;
      bool ok = true;
      if (stuck_polls) {
        // failure-path test: a bounded wait on a barrier nothing arrives on runs out
        if (!bar_wait(&neverb, 0, stuck_polls, &abort_flag) && !abort_flag) fail();
        ok = false;
      }
      const uint32_t id2 = idesc(n2, tf32);
      const uint64_t tp0 = sdesc(smem_u32(tp_mem), 1024);   // T' buffer 0, hi plane
      constexpr uint64_t kTpStep = uint64_t(kTpBytes) >> 4, kLoStep = uint64_t(kPBytes) >> 4;
      bool done = false;
      while (ok && !done) {
        const int s = int(item % kSlots);
        if (!bar_wait(&full[s], (item / kSlots) & 1, limit, &abort_flag)) {
          if (!abort_flag) fail();
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const ItemMeta im = imeta[s];
        const uint32_t st = smem_u32(ring + im.pos);
        const uint32_t sbo = uint32_t(im.kg) * 128;
        if (im.kind == 0) {
          // MMA1 chunk of unit ix: T[ix & 1] (+)= L psi^T chunk
          const int b = ix & 1;
          if (im.first && ix >= 2 && !bar_wait(&tempty[b], ((ix >> 1) & 1) ^ 1, limit, &abort_flag)) {
            if (!abort_flag) fail();
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t id1 = idesc(im.n1, tf32);
          const uint32_t tT = tmem + uint32_t(b * 64);
          const uint64_t ah = sdesc(st, sbo), al = sdesc(st + im.a, sbo);
          const uint64_t bh = sdesc(st + 2 * im.a, sbo), bl = sdesc(st + 2 * im.a + im.b, sbo);
          const int kss = im.kg / 2;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            if (ks < kss) {
              const uint64_t d = uint64_t(ks) * 16;
              mma3(tf32, tT, ah + d, al + d, bh + d, bl + d, id1, (!im.first || ks > 0) ? 1u : 0u);
            }
          commit(&empty[s]);
          if (im.last) {
            commit(&tfull[b]);
            ++ix;
          }
        } else {
          // MMA2 of unit iy into accumulator (iy / kGroup) & 1: the first unit of a group
          // overwrites it (after the converter has added the group two back to the output)
          const int b = iy & 1;
          const uint32_t g = iy / kGroup;
          const int ab = int(g & 1);
          const bool gstart = (iy % kGroup) == 0;
          if (gstart && g >= 2 && !bar_wait(&accempty[ab], ((g >> 1) & 1) ^ 1, limit, &abort_flag)) {
            if (!abort_flag) fail();
            break;
          }
          if (!bar_wait(&tpready[b], (iy >> 1) & 1, limit, &abort_flag)) {
            if (!abort_flag) fail();
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t acc_tm = tmem + 128u + uint32_t(ab * kTileN);
          const uint64_t th = tp0 + uint64_t(b) * kTpStep, tl = th + kLoStep;
          const uint64_t rh = sdesc(st, sbo), rl = sdesc(st + im.a, sbo);
          const int kss = im.n1 * es / 32;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks)
            if (ks < kss) {
              const uint64_t d = uint64_t(ks) * 16;
              mma3(tf32, acc_tm, th + d, tl + d, rh + d, rl + d, id2, (!gstart || ks > 0) ? 1u : 0u);
            }
          commit(&empty[s]);
          commit(&tpempty[b]);
          if (im.last || iy % kGroup == kGroup - 1) commit(&accfull[ab]);
          done = im.last;
          ++iy;
        }
        ++item;
      }
      // every MMA issued has finished before TMEM is freed
      commit(&drainb);
      if (!bar_drain(&drainb, 0)) fail();
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ converter and flushes
    // warp w reads TMEM lane quarter w % 4 (tile rows 32 (w % 4) ..), the two warps of a
    // quarter take the two halves of the columns
    const int quad = warp & 3;
    const int half = warp >> 2;
    const int row = quad * 32 + lane;       // tile row = TMEM lane
    const uint32_t lane_off = uint32_t(quad * 32) << 16;
    const int hw = wk / 2;                  // T columns per half (32 bf16, 16 tf32)
    const uint32_t rbase = uint32_t(row >> 3) * 1024 + uint32_t(row & 7) * 16;
    double* out = G.out + o.off;
    const int r = r0 + row;
    // warps whose 32 rows all lie past the output block skip the arithmetic: their T' rows
    // only feed accumulator rows that are never written
    const bool live = r0 + quad * 32 < o.M;
    bool ok = true;
    // add accumulator group g to the FP64 output; every decision is uniform over the warp
    // (__all_sync) so that the warp-collective TMEM loads never run in part of a warp
    auto flush = [&](uint32_t g) -> bool {
      const int ab = int(g & 1);
      if (!__all_sync(0xffffffffu, bar_wait(&accfull[ab], (g >> 1) & 1, limit, &abort_flag))) {
        if (!abort_flag) fail();
        return false;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      constexpr int kHalfN = kTileN / 2;
      uint32_t v[kHalfN];
      const int cb = half * kHalfN;
      if (live) {
#pragma unroll
        for (int j = 0; j < kHalfN / 16; ++j)
          if (cb + 16 * j < n2) tmem_ld16_async(tmem + lane_off + 128u + uint32_t(ab * kTileN + cb + 16 * j), v + 16 * j);
        tmem_wait_ld();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      bar_arrive(&accempty[ab]);
      if (live && r < o.M) {
        double* p = out + int64_t(r) * o.N + c0 + cb;
#pragma unroll
        for (int j = 0; j < kHalfN; ++j)
          if (cb + j < n2 && c0 + cb + j < o.N) p[j] += double(__uint_as_float(v[j]));
      }
      return true;
    };
    uint32_t idx = 0;
    bool last = false;
    while (!last) {
      const int b = idx & 1;
      const int k = int(idx % kUnitRing);
      bool w = bar_wait(&ufull[k], (idx / kUnitRing) & 1, limit, &abort_flag);
      if (w) w = bar_wait(&tfull[b], (idx >> 1) & 1, limit, &abort_flag);
      if (w && idx >= 2) w = bar_wait(&tpempty[b], ((idx >> 1) & 1) ^ 1, limit, &abort_flag);
      if (!__all_sync(0xffffffffu, w)) {
        if (!abort_flag) fail();
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const UnitMeta um = umeta[k];
      bar_arrive(&uempty[k]);
      last = um.last != 0;
      const float alpha = um.alpha;
      const int n1 = um.n1;
      const int cb = half * hw;
      unsigned char* tpH = tp_mem + b * kTpBytes;
      unsigned char* tpL = tpH + kPBytes;
      uint32_t v[32];
      if (live) {
#pragma unroll
        for (int j = 0; j < 2; ++j)
          if (16 * j < hw && cb + 16 * j < n1) tmem_ld16_async(tmem + lane_off + uint32_t(b * 64 + cb + 16 * j), v + 16 * j);
        tmem_wait_ld();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      bar_arrive(&tempty[b]);   // T of this buffer is in registers
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int cc = cb + 16 * j;
        if (!live || 16 * j >= hw || cc >= n1) continue;
        if (tf32) {
#pragma unroll
          for (int q = 0; q < 4; ++q) {   // 4 k-groups of 4 elements
            uint32_t hh[4], ll[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) split_tf32(alpha * __uint_as_float(v[16 * j + 4 * q + e]), hh[e], ll[e]);
            const uint32_t off = rbase + uint32_t((cc >> 2) + q) * 128;
            *reinterpret_cast<uint4*>(tpH + off) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
            *reinterpret_cast<uint4*>(tpL + off) = make_uint4(ll[0], ll[1], ll[2], ll[3]);
          }
        } else {
#pragma unroll
          for (int q = 0; q < 2; ++q) {   // 2 k-groups of 8 elements
            uint16_t hh[8], ll[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) split_bf16(alpha * __uint_as_float(v[16 * j + 8 * q + e]), hh[e], ll[e]);
            const uint32_t off = rbase + uint32_t((cc >> 3) + q) * 128;
            *reinterpret_cast<uint4*>(tpH + off) =
                make_uint4(hh[0] | (uint32_t(hh[1]) << 16), hh[2] | (uint32_t(hh[3]) << 16),
                           hh[4] | (uint32_t(hh[5]) << 16), hh[6] | (uint32_t(hh[7]) << 16));
            *reinterpret_cast<uint4*>(tpL + off) =
                make_uint4(ll[0] | (uint32_t(ll[1]) << 16), ll[2] | (uint32_t(ll[3]) << 16),
                           ll[4] | (uint32_t(ll[5]) << 16), ll[6] | (uint32_t(ll[7]) << 16));
          }
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_arrive(&tpready[b]);
      // the group before this one is complete once this unit's T' is handed over
      if (idx % kGroup == 0 && idx > 0 && !flush(idx / kGroup - 1)) {
        ok = false;
        break;
      }
      ++idx;
    }
    if (ok && idx > 0 && !flush((idx - 1) / kGroup)) ok = false;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// One problem (g0, passed by value) or several (groups in device memory): CTA b takes tile
// b - tile0 of the group g with tile0(g) <= b < tile0(g + 1).
__global__ void __launch_bounds__(kThreads, 2) k_heff_tc(const __grid_constant__ TcGroup g0,
                                                          const TcGroup* __restrict__ groups,
                                                          int n_groups, int* status,
                                                          uint32_t stuck_polls, int tf32) {
  const int b = blockIdx.x;
  if (!groups) {
    heff_tc_tile(g0, g0.tiles[b], status, stuck_polls, tf32 != 0);
    return;
  }
  int lo = 0, hi = n_groups - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (groups[mid].tile0 <= b) lo = mid; else hi = mid - 1;
  }
  const TcGroup& G = groups[lo];
  heff_tc_tile(G, G.tiles[b - G.tile0], status, stuck_polls, tf32 != 0);
}

void launch_split(const SplitTask* tasks, int n_tasks, const BufTable& bt, uint8_t* hi, uint8_t* lo,
                  bool tf32, cudaStream_t s) {
  if (n_tasks <= 0) return;
  k_split<<<n_tasks, 256, 0, s>>>(tasks, bt, hi, lo, tf32 ? 1 : 0);
  count_launches(1);
}

void launch_heff_tc(const TcGroup& g0, const TcGroup* groups, int n_groups, int n_tiles, bool tf32,
                    int* status, uint32_t stuck_polls, cudaStream_t s) {
  if (n_tiles <= 0 || (groups && n_groups <= 0)) return;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_heff_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kDynSmem);
  });
  k_heff_tc<<<n_tiles, kThreads, kDynSmem, s>>>(g0, groups, n_groups, status, stuck_polls,
                                                tf32 ? 1 : 0);
  count_launches(1);
}

}  // namespace b2k
