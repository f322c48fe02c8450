// tc_gemm.cuh -- the three passes over A on the 5th-generation tensor cores:
// tcgen05.mma (kind::tf32) with the accumulator in tensor memory (TMEM),
// operands staged in shared memory by TMA (cp.async.bulk.tensor), a persistent
// stream-K schedule over (128-row tile, K-block) units, warp-specialised roles.
//
//   D (M x N, row-major, FP32) = sum_k Aop(m, k) Bop(k, n)
//   Aop(m, k): the big matrix A, either stored with m contiguous (A_MN:
//              element (m,k) at A[k*lda + m]; passes 1 and 2, where the
//              contraction runs over A's rows) or with k contiguous (element
//              (m,k) at A[m*lda + k]; pass 3).
//   Bop(k, n): a thin operand stored K-major as Bt[n*ldb + k] (Omega, Q1^T,
//              V'^T), N <= 256 columns.
//   NPROD = 1: one TF32 product (the sketch, pass 1).
//   NPROD = 3: the split A = Ah + Al, B = Bh + Bl with Ah, Bh exactly
//              representable in TF32 (low 13 mantissa bits cleared) and
//              D = Ah Bh + Ah Bl + Al Bh (dropping Al Bl ~ 2^-22 |A||B|), which
//              restores FP32-level accuracy from TF32 products.  Bh / Bl are
//              prepared by split_tf32_kernel; Ah / Al are formed in shared
//              memory by the converter warps.
//
// The MMA always reads both operands K-major (the tf32 MMA is used without its
// transpose mode).  For A_MN the TMA lands the tile m-contiguous (four boxes of
// 32 m x BK k, 128-byte swizzle) and the converter warps transpose it in shared
// memory into the K-major swizzled layout the MMA reads (splitting it into
// Ah / Al on the way when NPROD = 3); for pass 3 the TMA lands A K-major and
// the converters only split it in place.
//
// Accumulation: the tensor core adds each MMA's products into the FP32 TMEM
// accumulator without round-to-nearest (the sum is biased toward zero by up
// to one unit in the last place per MMA), which over K = 20000 (2500 MMAs)
// shrank results by ~1e-4 relative.  So the MMA accumulates only TC_CHUNK
// K-blocks into a TMEM buffer; the epilogue warps add each chunk into FP32
// registers (round-to-nearest) and write the sum once per segment.  Two TMEM
// buffers (256 columns each) let the MMA fill one chunk while the epilogue
// drains the other.
//
// Warp roles (16 warps, by warpgroup; see TC_THREADS below): the TMA
// producer and the MMA issuer (one thread each) share the first warpgroup
// with two converter warps, two warpgroups drain TMEM (epilogue), and a
// fourth warpgroup converts.  Registers move from the converter groups to the
// epilogue groups with setmaxnreg, so six converter warps fit beside
// epilogue warps that hold up to 112 accumulators each.
//
// BF16 operands (kind::f16, the split-BF16 mode): A lands as FP32 and the
// converters write its BF16 head and tail (round to nearest even) as K-major
// rows of 32 BF16 values; the thin operand comes split to BF16 from global
// memory; D = Ah Bh + Ah Bl + Al Bh with FP32 accumulation (about 2^-16 per
// product).  The one-product BF16 sketch keeps the head only.
//
// Schedule (unit u = tile*KB + kb): the first dpt = tiles - tiles mod G tiles
// are data-parallel, block c taking dpt/G consecutive whole tiles; the last
// tiles mod G tiles are stream-K over all blocks, block c owning their units
// [S*c/G, S*(c+1)/G) (S of them).  A block's first and last stream-K
// segments may cover part of a tile's K range; those partial tiles go to
// part[(2c + slot)] and tc_fixup_kernel adds the pieces of each such tile in
// block order (deterministic).  All other tiles are written directly.  (With
// fewer tiles than blocks, a Gram, everything is stream-K.)  With a short K (sc.whole_tiles) block c owns the whole tiles
// [tiles*c/G, tiles*(c+1)/G) instead: every tile is written directly and no
// fixup runs.  Every mbarrier wait is bounded (~1 s); on expiry the block
// records STATUS_TIMEOUT, drains what it issued, frees its TMEM and exits.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace ffq {

constexpr int TC_BM = 128;
// Warp roles, by warpgroup (four warps each):
//   WG0: warp 0 TMA producer, warp 1 TMEM owner and MMA issuer, warps 2-3 converters;
//   WG1, WG2: epilogue (warp w reads TMEM lanes 32 (w % 4) .. + 31; WG1 takes
//             the first half of the columns, WG2 the second);
//   WG3: converters.
// The block is launched with 128 registers per thread (65536 / 512); WG0 and
// WG3 give theirs down to TC_REG_LOW, WG1 and WG2 take TC_REG_HIGH (the
// epilogue holds up to 112 FP32 accumulators per thread):
// 128 (2 TC_REG_LOW + 2 TC_REG_HIGH) = 128 * 512 = 65536, the launch's total.
constexpr int TC_CONV_WARPS = 6;
constexpr int TC_THREADS = 512;
constexpr int TC_REG_LOW = 88;
constexpr int TC_REG_HIGH = 168;
static_assert(128 * (2 * TC_REG_LOW + 2 * TC_REG_HIGH) == 65536, "register split must equal the launch's total");
static_assert(TC_THREADS * 128 == 65536, "launched at 128 registers per thread");
constexpr int TC_CHUNK = 8;      // K-blocks per TMEM accumulation chunk (3-product kernels)
constexpr int TC_MAX_NT = 224;   // widest N tile (columns) the epilogue registers hold
constexpr int TC_EPI_WARPS = 8;
constexpr int TC_MAX_STAGES = 8;
constexpr long long TC_SPIN = 4000000;

struct TcSched {
  int M, N, K;      // problem
  int KB;           // K blocks
  int tiles;        // ceil(M / 128)
  long long U;      // tiles * KB
  int G;            // grid
  int ntile;        // N rounded up to a multiple of 16 (MMA N)
  int stages;       // pipeline depth (<= TC_MAX_STAGES)
  int64_t ldc;
  float *C;
  float *part;      // [2G][128][ntile]
  int *ctl;
  int vec4;         // C rows are 16-byte aligned (C % 16 == 0, ldc % 4 == 0)
  int fix_rows;     // rows of a tile per fixup block (divides TC_BM)
  int whole_tiles;  // 1: block c takes tiles [tiles c / G, tiles (c+1) / G) whole (no partials)
  int dpt;          // data-parallel tiles (a multiple of G; the rest are stream-K)
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bounded wait (~1 s of wall time, whatever try_wait's internal suspend time
// is); returns false and flags the timeout if it expires, or returns false at
// once if another role already flagged one.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          int *ctl) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  long long spins = 0;
  while (!mbar_try(bar, parity)) {
    if (*abort_flag) return false;
    if ((++spins & 255) == 0 && (globaltimer_ns() - t0 > 1000000000ull || spins > TC_SPIN)) {
      *abort_flag = 1;
      atomicExch(ctl + CTL_TIMEOUT, 1);
      set_status(ctl, STATUS_TIMEOUT);
      return false;
    }
  }
  return true;
}

// Wait (at most ~1 s) without touching the abort state: used while draining.
__device__ __forceinline__ void mbar_wait_quiet(uint64_t *bar, uint32_t parity) {
  const unsigned long long t0 = globaltimer_ns();
  long long spins = 0;
  while (!mbar_try(bar, parity)) {
    if ((++spins & 255) == 0 && (globaltimer_ns() - t0 > 1000000000ull || spins > TC_SPIN)) return;
  }
}

__device__ __forceinline__ void tma_load_2d(void *smem_dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(smem_dst)), "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// tcgen05 shared-memory matrix descriptor: start address, leading / stride
// byte offsets (>> 4), version 1, swizzle mode (2 = 128B, 4 = 64B).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t swz) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | ((uint64_t)swz << 61);
}

// Instruction descriptor, kind::tf32, FP32 accumulate, M = 128, both operands
// K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

// Instruction descriptor, kind::f16 with BF16 A and B, FP32 accumulate,
// M = 128, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
      ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 32 consecutive 32-bit TMEM columns -> 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 8 consecutive 32-bit TMEM columns -> 8 registers per thread.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                 "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// Block c's units: range 0 its data-parallel tiles (or, with sc.whole_tiles,
// its whole tiles), range 1 its stream-K units.
__device__ __forceinline__ void tc_range(const TcSched &sc, int c, int r, int &a, int &b) {
  if (sc.whole_tiles) {
    a = (r == 0) ? (int)(((long long)sc.tiles * c) / sc.G) * sc.KB : 0;
    b = (r == 0) ? (int)(((long long)sc.tiles * (c + 1)) / sc.G) * sc.KB : 0;
  } else if (r == 0) {
    const int per = (sc.dpt / sc.G) * sc.KB;
    a = c * per;
    b = a + per;
  } else {
    const long long base = (long long)sc.dpt * sc.KB, sk = sc.U - base;
    a = (int)(base + (sk * c) / sc.G);
    b = (int)(base + (sk * (c + 1)) / sc.G);
  }
}

// Segment iterator shared by all roles: block c walks its range 0, then its
// range 1 (units < 2^31); the second range is formed from the launch's
// parameters when the first runs out, so a role holds only two counters.
struct SegIter {
  int u, u1, r;
  __device__ bool next(const TcSched &sc, int &tile, int &kb0, int &kb1) {
    if (u >= u1) {
      if (r != 0) return false;
      r = 1;
      tc_range(sc, (int)blockIdx.x, 1, u, u1);
      if (u >= u1) return false;
    }
    tile = u / sc.KB;
    kb0 = u - tile * sc.KB;
    const int left = u1 - u;
    kb1 = (kb0 + left < sc.KB) ? kb0 + left : sc.KB;
    u += kb1 - kb0;
    return true;
  }
};

// Byte offset of element (row r, column k) in a K-major tile whose rows are
// BK FP32 values (128 B for BK = 32 with the 128B swizzle, 64 B for BK = 16
// with the 64B swizzle): the 16-byte chunk index is XORed with address bits
// 7..9 (128B) or 7..8 (64B), as TMA writes and the MMA reads it.
template <int BK>
__device__ __forceinline__ uint32_t kmajor_off(int r, int k) {
  if (BK == 32) return (uint32_t)(r * 128 + ((((k >> 2) ^ (r & 7)) & 7) << 4) + ((k & 3) << 2));
  return (uint32_t)(r * 64 + ((((k >> 2) ^ ((r >> 1) & 3)) & 3) << 4) + ((k & 3) << 2));
}
// Byte offset of element (k, m) in the m-contiguous TMA landing tile: four
// boxes of 32 m x BK k rows of 128 B, 128B swizzle.
template <int BK>
__device__ __forceinline__ uint32_t mn_off(int k, int m) {
  const int q = m >> 5, ml = m & 31;
  return (uint32_t)(q * (BK * 128) + k * 128 + ((((ml >> 2) ^ (k & 7)) & 7) << 4) + ((ml & 3) << 2));
}

__device__ __forceinline__ float tf32_head(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Named barrier 1 over the TC_CONV_WARPS converter warps: a plain barrier,
// and one that returns whether any participant passed a true condition (so
// that all converter warps leave their loop together).
template <int NTHR>
__device__ __forceinline__ void conv_sync() {
  asm volatile("bar.sync 1, %0;" ::"n"(NTHR) : "memory");
}
template <int NTHR>
__device__ __forceinline__ bool conv_any(bool c) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred pi, po;\n setp.ne.u32 pi, %1, 0;\n bar.red.or.pred po, 1, %2, pi;\n selp.u32 %0, 1, 0, po;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)c), "n"(NTHR)
      : "memory");
  return r != 0;
}

// Byte offset of the 16-byte chunk holding BF16 elements (r, 8 c .. 8 c + 7)
// of a K-major tile whose rows are 32 BF16 values (64 bytes, 64B swizzle:
// the chunk index XORed with address bits 7..8, as the MMA reads it).
__device__ __forceinline__ uint32_t kmajor_bf16_chunk(int r, int c) {
  return (uint32_t)(r * 64 + (((c ^ (r >> 1)) & 3) << 4));
}

// Eight FP32 values -> their BF16 heads (round to nearest even) and, with
// TAIL, the BF16 of what the heads leave (x - head, exact in FP32), each
// packed as one 16-byte chunk.
template <bool TAIL>
__device__ __forceinline__ void bf16_split8(const float *x, uint4 &h, uint4 &l) {
  uint32_t hw[4], lw[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    hw[i] = *reinterpret_cast<const uint32_t *>(&hb);
    if (TAIL) {
      const float2 hf = __bfloat1622float2(hb);
      const __nv_bfloat162 lb = __floats2bfloat162_rn(x[2 * i] - hf.x, x[2 * i + 1] - hf.y);
      lw[i] = *reinterpret_cast<const uint32_t *>(&lb);
    }
  }
  h = make_uint4(hw[0], hw[1], hw[2], hw[3]);
  if (TAIL) l = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}

// Shared memory of one stage: [raw A landing (A_MN only)] [Ah] [Al (NPROD 3)]
// [Bh] [Bl (NPROD 3)]; every piece is a multiple of 1024 bytes.
// BF: the operands are BF16 (kind::f16): A lands as FP32 (BK columns, 128 B
// rows) and the converters write its BF16 head (and tail) as K-major rows of
// BK = 32 BF16 values (64 bytes); the thin operand comes as BF16 from global
// memory.
// With BF the conversion is in place: the converter warps read the whole FP32
// landing tile into registers, meet at a named barrier, and write the BF16
// head (and tail) over it, so a stage is the landing tile plus B (which lets
// five stages fit instead of three).
template <int BK, int NPROD, bool A_MN, bool BF = false>
struct TcStage {
  static constexpr int EL = BF ? 2 : 4;                    // operand element bytes
  static constexpr int A_BYTES = TC_BM * BK * EL;          // one operand tile of A
  static constexpr int RAW_BYTES = TC_BM * BK * 4;         // the FP32 landing tile
  static constexpr int RAW = (A_MN && !BF) ? RAW_BYTES : 0;
  static constexpr int AH = RAW;
  static constexpr int AL = AH + A_BYTES;
  static constexpr int BH = BF ? RAW_BYTES : AH + A_BYTES * (NPROD == 3 ? 2 : 1);
  __host__ __device__ static constexpr int b_bytes(int nt) { return nt * BK * EL; }
  __host__ __device__ static constexpr int bytes(int nt) { return BH + b_bytes(nt) * (NPROD == 3 ? 2 : 1); }
  __host__ __device__ static constexpr int tx(int nt) { return RAW_BYTES + b_bytes(nt) * (NPROD == 3 ? 2 : 1); }
  static constexpr bool CONVERT = A_MN || NPROD == 3 || BF;
};

template <int BK, int NPROD, bool A_MN, bool BF = false>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmBl, TcSched sc) {
  using S = TcStage<BK, NPROD, A_MN, BF>;
  // the single-product sketch keeps whole segments in TMEM: its accuracy is
  // set by the TF32 operands, not by the accumulation
  constexpr int CHUNK = (NPROD == 3) ? TC_CHUNK : (1 << 30);
  constexpr int A_BYTES = S::A_BYTES;
  constexpr int KROW = BK * S::EL;             // bytes of a K-major operand row
  constexpr int KSWZ = (KROW == 128) ? 2 : 4;  // 128B / 64B swizzle of K-major rows
  const int NT = sc.ntile;
  const int STAGES = sc.stages;
  const int B_BYTES = S::b_bytes(NT);
  const int STAGE_BYTES = S::bytes(NT);
  const uint32_t TX_BYTES = (uint32_t)S::tx(NT);

  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                          ~(uintptr_t)1023);
  __shared__ __align__(8) uint64_t full_bar[TC_MAX_STAGES], conv_bar[TC_MAX_STAGES], empty_bar[TC_MAX_STAGES];
  __shared__ __align__(8) uint64_t accf_bar[2], acce_bar[2], drain_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x;
  SegIter it;
  tc_range(sc, c, 0, it.u, it.u1);
  it.r = 0;
  int first_tile;  // the first stream-K tile (partial slot 0)
  {
    int a, b;
    tc_range(sc, c, 1, a, b);
    first_tile = a / sc.KB;
  }

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&conv_bar[s], TC_CONV_WARPS);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf_bar[b], 1);
      mbar_init(&acce_bar[b], TC_EPI_WARPS);
    }
    mbar_init(&drain_bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(&tmem_base))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  volatile int *abortp = &abort_flag;


  auto stage_ptr = [&](int s) { return smem + (size_t)s * STAGE_BYTES; };

  // Roles by warpgroup; each warpgroup's branch starts with its register
  // share (setmaxnreg is warpgroup-wide, so all four warps of a group execute
  // the same instruction).
  auto converters = [&]() {
    // ---------------- converters (warps 2-3 and 12-15) ----------------
    constexpr int NCT = 32 * TC_CONV_WARPS;
    const int ct = ((warp < 4) ? warp - 2 : warp - 10) * 32 + lane;  // 0..NCT-1
    int s = 0;
    uint32_t ph = 0;
    int tile, kb0, kb1;
    SegIter my = it;
    bool ok = true;
    while (ok && my.next(sc, tile, kb0, kb1)) {
      for (int kb = kb0; kb < kb1; ++kb) {
        if constexpr (BF) {
          // all converter warps take the same decision: leave together on a
          // timeout or abort seen by any of them (the named barriers below
          // must be reached by all of them)
          const bool bad = !mbar_wait(&full_bar[s], ph, abortp, sc.ctl);
          if (conv_any<NCT>(bad)) {
            ok = false;
            break;
          }
        } else if (!mbar_wait(&full_bar[s], ph, abortp, sc.ctl)) {
          ok = false;
          break;
        }
        unsigned char *st = stage_ptr(s);
        if constexpr (BF) {
          // FP32 landing -> K-major BF16 head (and tail), in place: task =
          // (row m, 8 consecutive k), 128 rows x BK / 8 chunks per stage,
          // consecutive threads on consecutive m (conflict-free landing
          // reads).  Every task's values are read before any is written.
          constexpr int NTASK = TC_BM * (BK / 8);
          constexpr int TPT = (NTASK + NCT - 1) / NCT;  // tasks per thread
          float x[TPT][8];
#pragma unroll
          for (int u = 0; u < TPT; ++u) {
            const int task = ct + u * NCT;
            if (task < NTASK) {
              const int m = task % TC_BM, c8 = task / TC_BM;
              if (A_MN) {
#pragma unroll
                for (int j = 0; j < 8; ++j)
                  x[u][j] = *reinterpret_cast<const float *>(st + mn_off<BK>(8 * c8 + j, m));
              } else {
                const float4 v0 = *reinterpret_cast<const float4 *>(st + kmajor_off<32>(m, 8 * c8));
                const float4 v1 = *reinterpret_cast<const float4 *>(st + kmajor_off<32>(m, 8 * c8 + 4));
                x[u][0] = v0.x;
                x[u][1] = v0.y;
                x[u][2] = v0.z;
                x[u][3] = v0.w;
                x[u][4] = v1.x;
                x[u][5] = v1.y;
                x[u][6] = v1.z;
                x[u][7] = v1.w;
              }
            }
          }
          conv_sync<NCT>();
#pragma unroll
          for (int u = 0; u < TPT; ++u) {
            const int task = ct + u * NCT;
            if (task < NTASK) {
              const int m = task % TC_BM, c8 = task / TC_BM;
              uint4 h, l;
              bf16_split8<NPROD == 3>(x[u], h, l);
              const uint32_t o = kmajor_bf16_chunk(m, c8);
              *reinterpret_cast<uint4 *>(st + S::AH + o) = h;
              if (NPROD == 3) *reinterpret_cast<uint4 *>(st + S::AL + o) = l;
            }
          }
        } else if (A_MN) {
          // transpose rows m = ct, ct + NCT, ... of the m-contiguous tile
          // into K-major rows
#pragma unroll 1
          for (int m = ct; m < TC_BM; m += NCT)
#pragma unroll 4
          for (int k4 = 0; k4 < BK; k4 += 4) {
            float x[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = *reinterpret_cast<const float *>(st + mn_off<BK>(k4 + j, m));
            const uint32_t o = kmajor_off<BK>(m, k4);
            if (NPROD == 3) {
              float4 h, l;
              h.x = tf32_head(x[0]);
              h.y = tf32_head(x[1]);
              h.z = tf32_head(x[2]);
              h.w = tf32_head(x[3]);
              l.x = x[0] - h.x;
              l.y = x[1] - h.y;
              l.z = x[2] - h.z;
              l.w = x[3] - h.w;
              *reinterpret_cast<float4 *>(st + S::AH + o) = h;
              *reinterpret_cast<float4 *>(st + S::AL + o) = l;
            } else {
              *reinterpret_cast<float4 *>(st + S::AH + o) = make_float4(x[0], x[1], x[2], x[3]);
            }
          }
        } else {
          // split the K-major tile in place: Ah (TF32 head) and Al (tail)
          float4 *a4 = reinterpret_cast<float4 *>(st + S::AH);
          float4 *l4 = reinterpret_cast<float4 *>(st + S::AL);
#pragma unroll 4
          for (int i = ct; i < A_BYTES / 16; i += NCT) {
            const float4 x = a4[i];
            float4 h, l;
            h.x = tf32_head(x.x);
            h.y = tf32_head(x.y);
            h.z = tf32_head(x.z);
            h.w = tf32_head(x.w);
            l.x = x.x - h.x;
            l.y = x.y - h.y;
            l.z = x.z - h.z;
            l.w = x.w - h.w;
            a4[i] = h;
            l4[i] = l;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv_bar[s]);
        if (++s == STAGES) {
          s = 0;
          ph ^= 1u;
        }
      }
    }
    };
  const int wg = warp >> 2;
  if (wg == 0) {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(TC_REG_LOW));
    if (warp == 0) {
      // ---------------- TMA producer ----------------
      if (lane == 0) {
        int s = 0;
        uint32_t ph = 0;
        int tile, kb0, kb1;
        SegIter my = it;
        bool ok = true;
        uint32_t issued = 0, issued_ph = 0;  // per stage: a load in flight, and its phase parity
        while (ok && my.next(sc, tile, kb0, kb1)) {
          for (int kb = kb0; kb < kb1 && ok; ++kb) {
            if (!mbar_wait(&empty_bar[s], ph ^ 1u, abortp, sc.ctl)) {
              ok = false;
              break;
            }
            issued |= 1u << s;
            issued_ph = (issued_ph & ~(1u << s)) | (ph << s);
            unsigned char *st = stage_ptr(s);
            mbar_expect_tx(&full_bar[s], TX_BYTES);
            const int k0 = kb * BK, m0 = tile * TC_BM;
            if (A_MN) {
  #pragma unroll
              for (int q = 0; q < TC_BM / 32; ++q)
                tma_load_2d(st + q * (BK * 128), &tmA, m0 + 32 * q, k0, &full_bar[s]);
            } else {
              tma_load_2d(st + (BF ? 0 : S::AH), &tmA, k0, m0, &full_bar[s]);
            }
            tma_load_2d(st + S::BH, &tmB, k0, 0, &full_bar[s]);
            if (NPROD == 3) tma_load_2d(st + S::BH + B_BYTES, &tmBl, k0, 0, &full_bar[s]);
            if (++s == STAGES) {
              s = 0;
              ph ^= 1u;
            }
          }
        }
        if (!ok) {
          for (int d = 0; d < STAGES; ++d)
            if (issued & (1u << d)) mbar_wait_quiet(&full_bar[d], (issued_ph >> d) & 1u);
        }
      }
      __syncwarp();
    } else if (warp == 1) {
      // ---------------- MMA issuer ----------------
      if (lane == 0) {
        int s = 0;
        uint32_t ph = 0;
        int chunk = 0;
        int tile, kb0, kb1;
        SegIter my = it;
        const uint32_t IDESC = BF ? idesc_bf16(NT) : idesc_tf32(NT);
        bool ok = true;
        while (ok && my.next(sc, tile, kb0, kb1)) {
          for (int kc = kb0; kc < kb1 && ok; kc += CHUNK) {
            const int kc1 = (kb1 - kc > CHUNK) ? kc + CHUNK : kb1;
            const int b = chunk & 1;
            const uint32_t acc_ph = (uint32_t)((chunk >> 1) & 1);
            if (!mbar_wait(&acce_bar[b], acc_ph ^ 1u, abortp, sc.ctl)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t dt = tmem + (uint32_t)(b * 256);
            for (int kb = kc; kb < kc1; ++kb) {
              uint64_t *wb = S::CONVERT ? &conv_bar[s] : &full_bar[s];
              if (!mbar_wait(wb, ph, abortp, sc.ctl)) {
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t base = smem_u32(stage_ptr(s));
              const uint32_t ah = base + S::AH, al = base + S::AL, bh = base + S::BH, bl = bh + B_BYTES;
              // K-major operands: rows of KROW bytes in 8-row groups; the K step
              // of one MMA (8 TF32 or 16 BF16 values) is 32 bytes within the
              // swizzled row.
  #pragma unroll
              for (int kk = 0; kk < KROW / 32; ++kk) {
                const uint64_t da = smem_desc(ah + kk * 32, 16, 8 * KROW, KSWZ);
                const uint64_t db = smem_desc(bh + kk * 32, 16, 8 * KROW, KSWZ);
                const uint32_t acc = (kb > kc || kk > 0) ? 1u : 0u;
                if constexpr (BF) mma_bf16(dt, da, db, IDESC, acc);
                else mma_tf32(dt, da, db, IDESC, acc);
                if (NPROD == 3) {
                  const uint64_t dal = smem_desc(al + kk * 32, 16, 8 * KROW, KSWZ);
                  const uint64_t dbl = smem_desc(bl + kk * 32, 16, 8 * KROW, KSWZ);
                  if constexpr (BF) {
                    mma_bf16(dt, da, dbl, IDESC, 1u);
                    mma_bf16(dt, dal, db, IDESC, 1u);
                  } else {
                    mma_tf32(dt, da, dbl, IDESC, 1u);
                    mma_tf32(dt, dal, db, IDESC, 1u);
                  }
                }
              }
              mma_commit(&empty_bar[s]);
              if (++s == STAGES) {
                s = 0;
                ph ^= 1u;
              }
            }
            if (!ok) break;
            mma_commit(&accf_bar[b]);
            ++chunk;
          }
        }
        if (*abortp) {
          // make sure no MMA is still writing TMEM before it is freed
          mma_commit(&drain_bar);
          mbar_wait_quiet(&drain_bar, 0);
        }
      }
      __syncwarp();
    } else if (S::CONVERT) {
      converters();
    }
  } else if (wg <= 2) {
    asm volatile("setmaxnreg.inc.sync.aligned.u32 %0;" ::"n"(TC_REG_HIGH));
    // ---------------- epilogue ----------------
    const int q = warp & 3;                        // TMEM lane quadrant
    const int half = NT >> 1;                      // columns per warp (multiple of 8)
    const int col0 = (warp >= 8) ? half : 0;       // WG1: first half of the columns, WG2: second
    constexpr int NACC = TC_MAX_NT / 2;
    int chunk = 0;
    int tile, kb0, kb1;
    SegIter my = it;
    bool ok = true;
    while (ok && my.next(sc, tile, kb0, kb1)) {
      float acc[NACC];
#pragma unroll
      for (int i = 0; i < NACC; ++i) acc[i] = 0.f;
      for (int kc = kb0; kc < kb1; kc += CHUNK) {
        const int b = chunk & 1;
        const uint32_t acc_ph = (uint32_t)((chunk >> 1) & 1);
        if (!mbar_wait(&accf_bar[b], acc_ph, abortp, sc.ctl)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t ta = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * 256 + col0);
#pragma unroll
        for (int g = 0; g < NACC / 8; ++g) {
          if (g * 8 < half) {
            float v[8];
            tmem_ld8(ta + (uint32_t)(g * 8), v);
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[g * 8 + i] += v[i];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acce_bar[b]);
        ++chunk;
      }
      if (!ok) break;
      const int row_in_tile = q * 32 + lane;
      const int row = tile * TC_BM + row_in_tile;
      const bool full = (kb0 == 0 && kb1 == sc.KB);
      float *dst;
      int ncols;
      if (full) {
        dst = (row < sc.M) ? sc.C + (int64_t)row * sc.ldc : nullptr;
        ncols = sc.N;
      } else {
        const int slot = (tile == first_tile) ? 0 : 1;
        dst = sc.part + ((int64_t)(2 * c + slot) * TC_BM + row_in_tile) * sc.ntile;
        ncols = sc.ntile;
      }
      if (dst) {
        const bool v4 = !full || sc.vec4;
#pragma unroll
        for (int g = 0; g < NACC / 4; ++g) {
          const int cc = col0 + 4 * g;
          if (4 * g < half) {
            if (v4 && cc + 4 <= ncols) {
              *reinterpret_cast<float4 *>(dst + cc) =
                  make_float4(acc[4 * g], acc[4 * g + 1], acc[4 * g + 2], acc[4 * g + 3]);
            } else {
#pragma unroll
              for (int i = 0; i < 4; ++i)
                if (cc + i < ncols) dst[cc + i] = acc[4 * g + i];
            }
          }
        }
      }
    }
  } else {
    asm volatile("setmaxnreg.dec.sync.aligned.u32 %0;" ::"n"(TC_REG_LOW));
    if (S::CONVERT) converters();
  }
  // teardown
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
  }
}

constexpr int TC_MAX_GRID = 1024;  // upper bound of the persistent grid (fixup slot table)

// Sum the partial pieces of the stream-K tiles that several blocks share, in
// block order (deterministic), and write them to C.  Grid (tiles - dpt,
// TC_BM / sc.fix_rows): one block per sc.fix_rows rows of a stream-K tile.
__global__ void tc_fixup_kernel(TcSched sc) {
  __shared__ int s_lo, s_hi;
  __shared__ unsigned char s_slot[TC_MAX_GRID];
  const int tile = sc.dpt + blockIdx.x;
  const long long base = (long long)sc.dpt * sc.KB, sk = sc.U - base;
  if (threadIdx.x == 0) {
    const long long ua = (long long)tile * sc.KB, ub = ua + sc.KB - 1;
    auto owner = [&](long long u) {  // the block whose stream-K units hold u
      long long lo = 0, hi = sc.G - 1;
      while (lo < hi) {
        const long long mid = (lo + hi + 1) / 2;
        if (base + (sk * mid) / sc.G <= u) lo = mid;
        else hi = mid - 1;
      }
      return (int)lo;
    };
    s_lo = owner(ua);
    s_hi = owner(ub);
  }
  __syncthreads();
  const int c_lo = s_lo, c_hi = s_hi;
  if (c_lo == c_hi) return;  // written directly by its only owner
  // slot of this tile in each contributor's partial buffer: 0 if it is the
  // contributor's first tile, else 1
  for (int cb = c_lo + threadIdx.x; cb <= c_hi; cb += blockDim.x)
    s_slot[cb - c_lo] = (tile == (int)((base + (sk * cb) / sc.G) / sc.KB)) ? 0 : 1;
  __syncthreads();
  const int r0 = blockIdx.y * sc.fix_rows;
  for (int e = threadIdx.x; e < sc.fix_rows * sc.N; e += blockDim.x) {
    const int rr = r0 + e / sc.N, col = e % sc.N;
    const int row = tile * TC_BM + rr;
    if (row >= sc.M) continue;
    // added in block order (deterministic); many contributors (a Gram):
    // thirty-two loads in flight at a time
    float acc = 0.f;
    if (c_hi - c_lo < 7) {
      for (int cb = c_lo; cb <= c_hi; ++cb)
        acc += sc.part[((int64_t)(2 * cb + s_slot[cb - c_lo]) * TC_BM + rr) * sc.ntile + col];
    } else {
      for (int cb0 = c_lo; cb0 <= c_hi; cb0 += 32) {
        float pv[32];
#pragma unroll
        for (int u = 0; u < 32; ++u) {
          const int cb = cb0 + u;
          pv[u] = (cb <= c_hi) ? sc.part[((int64_t)(2 * cb + s_slot[cb - c_lo]) * TC_BM + rr) * sc.ntile + col]
                               : 0.f;
        }
#pragma unroll
        for (int u = 0; u < 32; ++u)
          if (cb0 + u <= c_hi) acc += pv[u];
      }
    }
    sc.C[(int64_t)row * sc.ldc + col] = acc;
  }
}

// Bh = TF32-exact head of B (low 13 mantissa bits cleared), Bl = B - Bh
// (exact in FP32), over a rows x cols block with leading dimension ld.
__global__ void split_tf32_kernel(const float *__restrict__ B, int64_t ld, int64_t rows, int64_t cols,
                                  float *__restrict__ Bh, float *__restrict__ Bl) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    const float x = B[i * ld + j];
    const float h = tf32_head(x);
    Bh[i * ld + j] = h;
    Bl[i * ld + j] = x - h;
  }
}

// Dh / Dl (cols x rows, leading dimension ldd) = TF32 head / tail of Src^T,
// Src rows x cols with leading dimension lds: the K-major thin operand of a
// tensor-core product.  32 x 32 tiles through shared memory, block (32, 8).
__global__ void transpose_split_kernel(const float *__restrict__ Src, int64_t lds, int64_t rows, int64_t cols,
                                       float *__restrict__ Dh, float *__restrict__ Dl, int64_t ldd) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t r = r0 + yy, c = c0 + threadIdx.x;
    tile[yy][threadIdx.x] = (r < rows && c < cols) ? Src[r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t dr = c0 + yy, dc = r0 + threadIdx.x;  // Dst row = Src column
    if (dr < cols && dc < rows) {
      const float x = tile[threadIdx.x][yy];
      const float h = tf32_head(x);
      Dh[dr * ldd + dc] = h;
      Dl[dr * ldd + dc] = x - h;
    }
  }
}

// Dst (rows x cols, leading dimension ldd, BF16) = Src (FP32, leading
// dimension lds) rounded to nearest even.
__global__ void to_bf16_kernel(const float *__restrict__ Src, int64_t lds, int64_t rows, int64_t cols,
                               __nv_bfloat16 *__restrict__ Dst, int64_t ldd) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / cols, j = e - i * cols;
    Dst[i * ldd + j] = __float2bfloat16_rn(Src[i * lds + j]);
  }
}

// Dh / Dl (cols x rows, leading dimension ldd, BF16) = head (round to nearest
// even) and tail (BF16 of x - head) of Src^T, Src rows x cols (FP32, leading
// dimension lds): the K-major split-BF16 thin operand of a pass.  32 x 32
// tiles through shared memory, block (32, 8).
__global__ void transpose_split_bf16_kernel(const float *__restrict__ Src, int64_t lds, int64_t rows,
                                            int64_t cols, __nv_bfloat16 *__restrict__ Dh,
                                            __nv_bfloat16 *__restrict__ Dl, int64_t ldd) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t r = r0 + yy, c = c0 + threadIdx.x;
    tile[yy][threadIdx.x] = (r < rows && c < cols) ? Src[r * lds + c] : 0.f;
  }
  __syncthreads();
  for (int yy = threadIdx.y; yy < 32; yy += blockDim.y) {
    const int64_t dr = c0 + yy, dc = r0 + threadIdx.x;  // Dst row = Src column
    if (dr < cols && dc < rows) {
      const float x = tile[threadIdx.x][yy];
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      Dh[dr * ldd + dc] = h;
      Dl[dr * ldd + dc] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
  }
}

}  // namespace ffq
