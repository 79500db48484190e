// Streaming row-local update of the split iteration for KP = 32 (17 <= k <=
// 32) on sm_103a: one thread per row, tiles of 128 rows moved by TMA, both
// dense contractions on the fifth-generation tensor cores.
//
// Same mathematics as update_kernel / update_tc_kernel, per row i:
//   y_i  = xbar^{n-1}_i + beta (xbar^{n-1}_i - xbar^{n-2}_i)          (X^n, Alg. 4)
//   SY_i = z_i + beta (z_i - z^{prev}_i)                             (S X^n by linearity)
//   xbar^n_i = P_simplex(y_i + 4 tau (SY_i - y_i G(Y)))              (Eq. "gradient_column", Alg. 1)
// with the trace term <xbar^{n-1}_i, z_i> of the loss update (Sect. 3), the
// projected-gradient norm ||y_i - xbar^n_i||^2 and the Gram partials of
// Xbar^n and of Y^{n+1} = Xbar^n + beta_{n+1} (Xbar^n - Xbar^{n-1}).
//
// Layout and roles (one CTA per SM, persistent over a contiguous range of
// tiles; 320 threads):
//   * two compute warpgroups (warps 0-3 and 4-7) take the CTA's tiles in turn;
//     thread t of a warpgroup owns row t of its tile and keeps the row's 32
//     features in registers, so the projection, the trace term and the norm
//     are sums inside one thread (no shuffles);
//   * one helper thread per warpgroup (warps 8 and 9) issues its TMA loads of
//     the four input tiles (z, xbar^{n-1}, xbar^{n-2}, z^{prev}: 4 x 16 KB,
//     128-byte swizzle, which makes every thread's 16-byte reads of its own
//     row conflict-free) and its tcgen05.mma instructions, sleeping in
//     mbarrier waits between them (no polling loop taking issue slots from
//     the compute warps).
//   * y G(Y): kind::tf32, 3xTF32 (hi/lo split), M = 128 = the tile's rows, so
//     row r of the accumulator is TMEM lane r and each thread reads its own
//     row back (tcgen05.ld 32x32b).  Each thread writes its row of the y
//     operand (hi, lo) over its own rows of the stage's xbar^{n-2} and
//     xbar^{n-1} tiles, just read: the next tile's z tiles load as soon as the
//     warpgroup has read its rows, its xbar tiles once y G has completed, and
//     the previous tile's Gram is read back while y G runs, so neither
//     tensor-core round trip of a tile waits on the other.
//   * Gram of [Xbar^n | Y^{n+1}] (64 features): kind::f16 with both operands
//     MN-major, i.e. the row-major tile itself (no transpose).  Each value is
//     scaled by 2^13 and split into two float16 parts h + l (h = s x rounded
//     to 11 significant bits, l = f16(s x - h)); h h + h l + l h carries the
//     product to about 2^-22
//     relative, like 3xTF32, and values below the float16 normal range lose
//     only an absolute 2^-38 after the scale.  The accumulator is read back
//     per tile and added into float pairs (Fast2Sum) in the threads, so the
//     partial of a CTA does not drift over thousands of tiles; the h h
//     products of the tile's two row halves go to two accumulators, which
//     halves the bias of the tensor core's truncating accumulation.
//
// Every wait is bounded (polls of bounded length, about one second in all);
// a warpgroup whose wait gives up raises an abort flag that ends every role's
// loop, the helper waits (bounded) for its loads and MMAs still in flight, and
// the fold ends the run with CLUSTER_ETIMEOUT.  Test hook bit 0 withholds the
// commit of y G, which drives that path without any fault.
#pragma once
#include <cuda.h>
#include <cuda_fp16.h>

#include "tc_update.cuh"

namespace fc {

// Tensor maps of the four n x 32 float32 buffers the streaming update reads
// (box 32 x 128 rows, 128-byte swizzle, rows beyond n read as zero).
struct StreamMaps {
  CUtensorMap X[2];
  CUtensorMap Z[2];
};

namespace ts {

constexpr int R = 128;                  // rows per tile
constexpr int NT = 320;                 // 2 x 128 compute threads + one helper warp per warpgroup
constexpr int TILE_B = R * 128;         // one tile of one input: 16 KB
constexpr int STAGE_B = 4 * TILE_B;     // z, xbar^{n-1}, xbar^{n-2}, z^{prev}
constexpr int GOP_B = 2 * R * 128;      // Gram operand: h and l, 128 rows x 64 float16
constexpr int OFF_GH = 0, OFF_GL = 4096, OFF_WG = 8192;
constexpr int WG_B = STAGE_B + GOP_B;   // 96 KB per warpgroup
constexpr size_t SMEM = (size_t)OFF_WG + 2 * (size_t)WG_B + 1024;  // + alignment slack
constexpr int TMEM_COLS = 512;
// TMEM columns per warpgroup w (base 256 w): y G (32), Gram accumulators A, B
// (64 each), 32 columns in which each thread keeps its 16 float pairs of the
// running Gram partial, and 32 that hold its row of xbar^{n-1} between the
// loads and the Gram operand (its own lane; registers are the scarce resource)
constexpr int COL_YG = 0, COL_GA = 64, COL_GB = 128, COL_ACC = 192, COL_PV = 224, COL_WG = 256;
constexpr float kScale = 8192.0f;                          // 2^13
constexpr float kUnscale2 = 1.0f / (8192.0f * 8192.0f);   // 2^-26, exact
// mbarriers of warpgroup w: w * 5 + {full, yready, ygdone, gready, grdone}; 10 + w: its helper's final commit
constexpr int BAR_FULL = 0, BAR_YREADY = 1, BAR_YGDONE = 2, BAR_GREADY = 3, BAR_GRDONE = 4, NBARS = 12;

static_assert(SMEM <= 232448, "shared memory of the streaming update");

__host__ __device__ constexpr uint32_t idesc_tf32_m128() { return tc::idesc_tf32(128, 32); }
// kind::f16: float32 accumulator (bits 4-5 = 1), A and B float16 (bits 7-9,
// 10-12 = 0), both MN-major (bits 15, 16), N / 8 at bit 17, M / 16 at bit 24
__host__ __device__ constexpr uint32_t idesc_f16_mn(int M, int N) {
  return (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// MN-major operand with 128-byte swizzle whose MN extent is one 128-byte atom
// (64 float16): groups of 8 K-rows 1024 bytes apart.  The byte offset between
// atoms along MN is not used at this width; it is set to the same 1024.
__device__ __forceinline__ uint64_t desc_mn128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(1024 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_init_n(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
// 2-D tiled TMA load of the box at (x, y) into shared memory, completing on bar
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(map) : "memory");
}
// b rounded to 11 significant bits (the sign, 8 exponent and 10 stored
// fraction bits of TF32), to nearest with ties away from zero, in integer
// arithmetic: add half of the 13 dropped bits' weight, then drop them.  The
// rounding cvt.rna.tf32.f32 performs, without the conversion pipe.
__device__ __forceinline__ uint32_t round11(uint32_t b) { return (b + 0x1000u) & 0xFFFFE000u; }
// 3xTF32 split of four values: hi = round11(x), lo = x - hi, exact and at most
// 2^-11 |x|; lo is not rounded: the tensor core reads its leading 11 bits, so
// it drops at most 2^-21 |x| (2^-22 with a rounded lo)
__device__ __forceinline__ void split11_store4(float* hi, float* lo, const float* v) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    h[q] = round11(__float_as_uint(v[q]));
    l[q] = __float_as_uint(v[q] - __uint_as_float(h[q]));
  }
  *reinterpret_cast<uint4*>(hi) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo) = make_uint4(l[0], l[1], l[2], l[3]);
}

// float pairs g[8 CG + j] (high) / g[16 + 8 CG + j] (low), kept as bits, += v[j]
// by Fast2Sum (Dekker): s = h + x, the add's rounding error x - (s - h) into
// the low part.  Exact when |h| >= |x|, which holds for these running sums:
// the entries of Xbar^T Xbar are sums of products of non-negative values, so
// the running sum of the tile partials only grows (and Y^{n+1} differs from
// Xbar^n by the small momentum term); the first tile adds to zero exactly.
template <int CG>
__device__ __forceinline__ void pair_acc8(uint32_t (&g)[32], const uint32_t (&v)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float h = __uint_as_float(g[8 * CG + j]), x = __uint_as_float(v[j]);
    const float sum = h + x;
    const float err = x - (sum - h);
    g[8 * CG + j] = __float_as_uint(sum);
    g[16 + 8 * CG + j] = __float_as_uint(__uint_as_float(g[16 + 8 * CG + j]) + err);
  }
}

// 32-byte store (one whole sector; p 32-byte aligned)
__device__ __forceinline__ void st_v8(void* p, const uint32_t* v) {
  asm volatile("st.global.v8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(v[0]), "r"(v[1]), "r"(v[2]),
               "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7])
               : "memory");
}
__device__ __forceinline__ void named_sync(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// TMEM -> registers, no wait: the calling thread's lane (of its warp's
// quarter), 32 consecutive columns from taddr; the values may be used only
// after wait_ld().  Several loads can be in flight under one wait.
__device__ __forceinline__ void ld32x32_async(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
// 16 lanes x 16 columns (shape 16x32bx2, half offset 8), no wait: thread t gets
// lane base + (t & 15), columns col + 8 (t >> 4) + j, j < 8
__device__ __forceinline__ void ld16x16_async(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.16x32bx2.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], 8;"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// After wait_ld(): make every later use of the loaded registers depend on a
// point ordered after the wait (an empty volatile asm that "rewrites" them),
// so the compiler cannot move a use above the wait.
__device__ __forceinline__ void pin8(uint32_t* r) {
  asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]));
}
__device__ __forceinline__ void pin32(uint32_t* r) {
  pin8(r);
  pin8(r + 8);
  pin8(r + 16);
  pin8(r + 24);
}
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
// registers -> TMEM, no wait (wait_st() before the columns are read again)
__device__ __forceinline__ void st32x32_async(uint32_t taddr, const uint32_t* r) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]), "r"(r[9]),
      "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]),
      "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]),
      "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

// Shared state of one CTA of the streaming update.
struct StreamCta {
  uint8_t* sm;       // 1024-aligned dynamic shared memory
  uint32_t sb;       // its shared-window address
  uint32_t tmem;     // TMEM base (512 columns)
  uint32_t bars;     // shared address of the NBARS mbarriers (8 bytes each)
  int* flags;        // [0] abort (a wait gave up), [1] test hooks
  int64_t t0;        // first tile of this CTA
  int cnt;           // tiles of this CTA (warpgroup w takes local tiles w, w + 2, ...)
  __device__ __forceinline__ uint32_t bar(int w, int i) const { return bars + 8u * (uint32_t)(w * 5 + i); }
  __device__ __forceinline__ bool aborted() const { return *reinterpret_cast<volatile int*>(flags) != 0; }
};

// The helper thread of warpgroup w, in the warpgroup's order: the first
// tile's loads; then per tile, once the warpgroup has read its rows and
// written its y operand over the stage's xbar^{n-1} and xbar^{n-2} tiles
// (y-ready): the next tile's z and z^{prev} tiles into the freed slots and
// y G; once y G has completed: the next tile's xbar^{n-1} and xbar^{n-2}
// tiles over the y operand; once the warpgroup has written the Gram operand
// (G-ready): the Gram.  Every wait is bounded and also ends on the abort flag.
// Returns after its MMAs have completed and its issued loads have landed
// (each bounded).
__device__ __forceinline__ void stream_helper(const StreamCta& c, const StreamMaps& m, int64_t pass, int w) {
  const CUtensorMap* mz = &m.Z[(pass + 1) & 1];   // S Xbar^{pass}
  const CUtensorMap* mp = &m.X[pass & 1];         // Xbar^{pass}
  const CUtensorMap* mq = &m.X[(pass + 1) & 1];   // Xbar^{pass-1}
  const CUtensorMap* mzp = &m.Z[pass & 1];        // S Xbar^{pass-1}
  prefetch_map(mz);
  prefetch_map(mp);
  prefetch_map(mq);
  prefetch_map(mzp);
  const bool hook = (c.flags[1] & 1) != 0;
  const int ntw = (c.cnt + 1 - w) / 2;
  const uint32_t st = c.sb + OFF_WG + (uint32_t)w * WG_B;
  const uint32_t full = c.bar(w, BAR_FULL);
  auto tile_row = [&](int jj) { return (int)((c.t0 + 2 * jj + w) * R); };
  // slots 0 and 3 (z, z^{prev}); the stage's whole byte count is expected here
  auto load_z = [&](int jj) {
    expect_tx(full, STAGE_B);
    tma_load_2d(st + 0 * TILE_B, mz, 0, tile_row(jj), full);
    tma_load_2d(st + 3 * TILE_B, mzp, 0, tile_row(jj), full);
  };
  // slots 1 and 2 (xbar^{n-1}, xbar^{n-2})
  auto load_x = [&](int jj) {
    tma_load_2d(st + 1 * TILE_B, mp, 0, tile_row(jj), full);
    tma_load_2d(st + 2 * TILE_B, mq, 0, tile_row(jj), full);
  };
  auto wait = [&](uint32_t bar, uint32_t par) -> bool {
    for (uint32_t i = 0; i < tc::kWaitPolls; ++i) {
      if (tc::bar_try(bar, par)) return true;
      if (c.aborted()) return false;
    }
    *reinterpret_cast<volatile int*>(c.flags) = 1;
    return false;
  };
  int nl = 0;          // tiles whose loads were (at least in part) issued
  bool half = false;   // the last of them still lacks its x tiles
  if (ntw > 0) {
    load_z(0);
    load_x(0);
    nl = 1;
  }
  for (int jj = 0; jj < ntw; ++jj) {
    if (!wait(c.bar(w, BAR_YREADY), (uint32_t)jj & 1u)) break;
    if (jj + 1 < ntw) {
      load_z(jj + 1);
      ++nl;
      half = true;
    }
    // y G(Y): A = y hi / lo (stage slots 2 / 1), B = G(Y) hi / lo
    tc::fence_after_sync();
    {
      const uint32_t d = c.tmem + (uint32_t)(w * COL_WG + COL_YG);
      const uint32_t yh = st + 2 * TILE_B, yl = st + 1 * TILE_B;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t ah = tc::desc_k128(yh + 32 * ks), al = tc::desc_k128(yl + 32 * ks);
        const uint64_t bh = tc::desc_k128(c.sb + OFF_GH + 32 * ks), bl = tc::desc_k128(c.sb + OFF_GL + 32 * ks);
        tc::mma(d, al, bh, idesc_tf32_m128(), ks > 0);
        tc::mma(d, ah, bl, idesc_tf32_m128(), 1);
        tc::mma(d, ah, bh, idesc_tf32_m128(), 1);
      }
      if (!hook) tc::commit(c.bar(w, BAR_YGDONE));
    }
    if (half) {
      if (!wait(c.bar(w, BAR_YGDONE), (uint32_t)jj & 1u)) break;
      load_x(jj + 1);
      half = false;
    }
    if (!wait(c.bar(w, BAR_GREADY), (uint32_t)jj & 1u)) break;
    // Gram of [Xbar^n | Y^{n+1}] over the tile's rows (K = 128, 8 steps of 16):
    // the small cross products first, then h h: rows 0-63 into A, 64-127 into B
    tc::fence_after_sync();
    {
      const uint32_t da = c.tmem + (uint32_t)(w * COL_WG + COL_GA), db = c.tmem + (uint32_t)(w * COL_WG + COL_GB);
      const uint32_t g = st + STAGE_B;
      constexpr uint32_t ID = idesc_f16_mn(64, 64);
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        const uint64_t h = desc_mn128(g + 2048 * ks), l = desc_mn128(g + TILE_B + 2048 * ks);
        mma_f16(da, l, h, ID, ks > 0);
        mma_f16(da, h, l, ID, 1);
      }
#pragma unroll
      for (int ks = 0; ks < 8; ++ks) {
        const uint64_t h = desc_mn128(g + 2048 * ks);
        if (ks < 4) mma_f16(da, h, h, ID, 1);
        else mma_f16(db, h, h, ID, ks > 4);
      }
      tc::commit(c.bar(w, BAR_GRDONE));
    }
  }
  // nothing of this thread may be in flight when the CTA exits: its MMAs
  // first (they may still read the y operand), then the rest of a half-issued
  // stage, so that the stage's phase can complete, then the loads
  const uint32_t fin = c.bars + 8u * (uint32_t)(10 + w);
  tc::commit(fin);
  tc::bar_wait(fin, 0);
  if (half) load_x(nl - 1);
  if (nl > 0) tc::bar_wait(full, (uint32_t)(nl - 1) & 1u);
}

// One compute thread: row t of each tile of warpgroup w.  Per tile: the four
// input rows from the stage (conflict-free swizzled reads), the trace term,
// y and SY; the y operand over the rows just read; y G back from TMEM; step
// and projection onto the simplex inside the thread (Michelot's active-set
// iteration, the same threshold as Algorithm 1); the Gram operand of
// [Xbar^n | Y^{n+1}], so that its MMAs start at once; then the new row and
// its bfloat16 copy to global memory (stores that wait on the memory system
// no longer delay the Gram: 8.48 -> 8.20 ms mixed at n = 70M).  Partial
// results go to slots slot0 + 2 w (the float pairs' high parts and the
// scalars) and slot0 + 2 w + 1 (the low parts).
// FULL: k = 32 (no padded feature to exclude from the projection).
template <bool MIXED, bool FULL>
__device__ __forceinline__ void stream_compute(const PassArgs& a, const StreamCta& c, int64_t pass, int slot0,
                                               double (*red)[4]) {
  const int tid = threadIdx.x, w = tid >> 7, t = tid & 127, qw = (tid >> 5) & 3, lane = tid & 31;
  const FistaState* st = a.st;
  const float beta = (float)st->beta, beta_next = (float)st->beta_next;
  const float tau4 = (float)(4.0 * st->tau);
  float* Qx = (pass & 1) ? a.X0 : a.X1;              // Xbar^{pass+1} out (over Xbar^{pass-1})
  __nv_bfloat16* XSo = (pass & 1) ? a.XS0 : a.XS1;
  const int k = a.k;
  uint8_t* stp = c.sm + OFF_WG + w * WG_B;
  uint8_t* gp = stp + STAGE_B;
  // this warp's TMEM lane quarter, this warpgroup's columns
  const uint32_t tw = c.tmem + ((uint32_t)(32 * qw) << 16) + (uint32_t)(w * COL_WG);
  const int gm = qw >> 1;  // Gram rows of this warp's quarter: matrix 0 (Xbar^n) or 1 (Y^{n+1})
  {
    uint32_t z[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) z[i] = 0u;
    st32x32_async(tw + COL_ACC, z);  // running Gram partial: [0, 16) high parts, [16, 32) low parts
  }
  float tr_hi = 0.f, tr_lo = 0.f, pg_hi = 0.f, pg_lo = 0.f;
  int bad = 0;
  bool dead = false;
  const int ntw = (c.cnt + 1 - w) / 2;
  const int swz = t & 7;

  // bounded wait, the same outcome on every lane of the warp (every lane
  // polls: a single polling lane with a warp shuffle measured 0.35 ms slower)
  auto wait = [&](uint32_t bar, uint32_t par) -> bool {
    bool ok = false;
    for (uint32_t i = 0; i < tc::kWaitPolls && !ok; ++i) {
      ok = tc::bar_try(bar, par);
      if (!ok && c.aborted()) break;
    }
    ok = __all_sync(kFull, ok);
    if (!ok) {
      dead = true;
      *reinterpret_cast<volatile int*>(c.flags) = 1;
    }
    tc::fence_after_sync();
    return ok;
  };
  // the previous tile's Gram (both accumulators) into the float pairs: all
  // TMEM loads under one wait, the store's completion awaited only before the
  // next load of the same columns
  // (warps holding Gram rows 16-31 of a block skip its columns 0-15: entries
  // below the diagonal, which the fold never reads)
  const bool below = (qw & 1) != 0;
  auto gram_back = [&]() {
    uint32_t g[32], v0[8], v1[8], v2[8], v3[8];
    wait_st();
    ld32x32_async(tw + COL_ACC, g);
    if (below) {
      ld16x16_async(tw + COL_GA + 32 * gm + 16, v1);
      ld16x16_async(tw + COL_GB + 32 * gm + 16, v3);
      wait_ld();
      pin32(g);
      pin8(v1);
      pin8(v3);
      pair_acc8<1>(g, v1);
      pair_acc8<1>(g, v3);
    } else {
      ld16x16_async(tw + COL_GA + 32 * gm, v0);
      ld16x16_async(tw + COL_GA + 32 * gm + 16, v1);
      ld16x16_async(tw + COL_GB + 32 * gm, v2);
      ld16x16_async(tw + COL_GB + 32 * gm + 16, v3);
      wait_ld();
      pin32(g);
      pin8(v0);
      pin8(v1);
      pin8(v2);
      pin8(v3);
      pair_acc8<0>(g, v0);
      pair_acc8<1>(g, v1);
      pair_acc8<0>(g, v2);
      pair_acc8<1>(g, v3);
    }
    st32x32_async(tw + COL_ACC, g);
  };

  for (int jj = 0; jj < ntw; ++jj) {
    const int64_t row = (c.t0 + 2 * jj + w) * R + t;
    const bool active = row < a.n;
    if (!wait(c.bar(w, BAR_FULL), (uint32_t)jj & 1u)) break;
    float y[32], sy[32], pv[32];
    float dq[4] = {0.f, 0.f, 0.f, 0.f};  // four partial sums: short dependency chains
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
      const int off = t * 128 + ((ch ^ swz) << 4);
      const float4 z4 = *reinterpret_cast<const float4*>(stp + 0 * TILE_B + off);
      const float4 p4 = *reinterpret_cast<const float4*>(stp + 1 * TILE_B + off);
      const float4 q4 = *reinterpret_cast<const float4*>(stp + 2 * TILE_B + off);
      const float4 r4 = *reinterpret_cast<const float4*>(stp + 3 * TILE_B + off);
      const float zv[4] = {z4.x, z4.y, z4.z, z4.w}, pvv[4] = {p4.x, p4.y, p4.z, p4.w};
      const float qv[4] = {q4.x, q4.y, q4.z, q4.w}, zp[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int f = 4 * ch + q;
        pv[f] = pvv[q];
        dq[q] = fmaf(pvv[q], zv[q], dq[q]);
        y[f] = fmaf(beta, pvv[q] - qv[q], pvv[q]);
        sy[f] = fmaf(beta, zv[q] - zp[q], zv[q]);
      }
      // y operand (row t, 128-byte swizzle, K-major) over the row's chunk of
      // xbar^{n-2} (hi) and xbar^{n-1} (lo), both just read into y
      split11_store4(reinterpret_cast<float*>(stp + 2 * TILE_B + off), reinterpret_cast<float*>(stp + 1 * TILE_B + off),
                     &y[4 * ch]);
    }
    {
      uint32_t pu[32];
#pragma unroll
      for (int f = 0; f < 32; ++f) pu[f] = __float_as_uint(pv[f]);
      st32x32_async(tw + COL_PV, pu);
    }
    const float d = (dq[0] + dq[1]) + (dq[2] + dq[3]);
    if (!isfinite(d)) bad = 1;  // d is finite exactly when every z of the row is
    if (active) two_sum_acc(tr_hi, tr_lo, d);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    arrive(c.bar(w, BAR_YREADY));
    // while y G runs: the previous tile's Gram into the float pairs (which
    // also frees the Gram operand's area for this tile)
    if (jj > 0) {
      if (!wait(c.bar(w, BAR_GRDONE), (uint32_t)(jj - 1) & 1u)) break;
      gram_back();
    }
    if (!wait(c.bar(w, BAR_YGDONE), (uint32_t)jj & 1u)) break;

    float v[32];
    {
      uint32_t qu[32];
      ld32x32_async(tw + COL_YG, qu);  // (y G(Y))_i of this row
      wait_ld();
      pin32(qu);
#pragma unroll
      for (int f = 0; f < 32; ++f) v[f] = __uint_as_float(qu[f]);
    }
    float sq[4] = {0.f, 0.f, 0.f, 0.f}, mn[4];
#pragma unroll
    for (int f = 0; f < 32; ++f) {
      v[f] = fmaf(tau4, sy[f] - v[f], y[f]);
      sq[f & 3] += v[f];  // padded features are exactly zero
      mn[f & 3] = f < 4 ? v[f] : fminf(mn[f & 3], v[f]);
    }
    const float s = (sq[0] + sq[1]) + (sq[2] + sq[3]);
    const float vmin = fminf(fminf(mn[0], mn[1]), fminf(mn[2], mn[3]));
    // this row of xbar^{n-1} back from TMEM, landing while the row is projected
    uint32_t pvu[32];
    wait_st();
    ld32x32_async(tw + COL_PV, pvu);
    if constexpr (!FULL) {
#pragma unroll
      for (int f = 0; f < 32; ++f)
        if (f >= k) v[f] = -INFINITY;
    }
    // Michelot: theta = (sum over A of v - 1) / |A|, A = {v > theta}, until |A| is stable.
    // With k = 32 the first set is stable when every feature exceeds the
    // first threshold (min v > theta): then no pass over the features is
    // needed (the same theta the loop would stop at)
    float cnt = FULL ? 32.0f : (float)k;
    float theta = __fdividef(s - 1.0f, cnt);
    const bool settled = FULL && vmin > theta;
    for (int it = 0; it <= 32 && !settled; ++it) {
      float s4[4] = {0.f, 0.f, 0.f, 0.f}, c4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int f = 0; f < 32; ++f) {
        const bool on = v[f] > theta;
        s4[f & 3] += on ? v[f] : 0.f;
        c4[f & 3] += on ? 1.f : 0.f;
      }
      const float s2 = (s4[0] + s4[1]) + (s4[2] + s4[3]), c2 = (c4[0] + c4[1]) + (c4[2] + c4[3]);
      if (c2 == cnt) break;
      cnt = c2;
      theta = __fdividef(s2 - 1.0f, cnt);
    }
    float pq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int f = 0; f < 32; ++f) {
      v[f] = fmaxf(v[f] - theta, 0.0f);  // xbar^n_i
      const float dd = y[f] - v[f];
      pq[f & 3] = fmaf(dd, dd, pq[f & 3]);
    }
    const float pg = (pq[0] + pq[1]) + (pq[2] + pq[3]);
    if (!isfinite(pg)) bad = 1;
    // the Gram operand's area (the previous tile's Gram has completed):
    // s [xbar^n | y^{n+1}] as float16 h + l, row t, chunk ch = features 8 ch ..
    wait_ld();
    pin32(pvu);
#pragma unroll
    for (int f = 0; f < 32; ++f) pv[f] = __uint_as_float(pvu[f]);
    // the scale 2^13, or 0 for a row past n (its operand row must be zero);
    // s y^{n+1} = s xbar^n + (s beta_{n+1}) (xbar^n - xbar^{n-1})
    const float rs = active ? kScale : 0.f, bs = beta_next * rs;
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
      uint32_t hu[4], lu[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        // h = the scaled value rounded to float16's 11 significant bits (exact
        // in float16 in its normal range), l = the exact remainder
        float hv[2], lv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int f = 8 * (ch & 3) + 2 * e + h;
          const float xs = v[f] * rs;
          const float val = ch < 4 ? xs : fmaf(bs, v[f] - pv[f], xs);
          hv[h] = __uint_as_float(round11(__float_as_uint(val)));
          lv[h] = val - hv[h];
        }
        const __half2 hh = __floats2half2_rn(hv[0], hv[1]);
        const __half2 ll = __floats2half2_rn(lv[0], lv[1]);
        hu[e] = *reinterpret_cast<const uint32_t*>(&hh);
        lu[e] = *reinterpret_cast<const uint32_t*>(&ll);
      }
      const int off = t * 128 + ((ch ^ swz) << 4);
      *reinterpret_cast<uint4*>(gp + off) = make_uint4(hu[0], hu[1], hu[2], hu[3]);
      *reinterpret_cast<uint4*>(gp + TILE_B + off) = make_uint4(lu[0], lu[1], lu[2], lu[3]);
    }
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    arrive(c.bar(w, BAR_GREADY));
    if (active) {
      two_sum_acc(pg_hi, pg_lo, pg);
      // whole 32-byte sectors: 4 stores per float32 row, 2 per bfloat16 row
      float* xo = Qx + row * 32;
#pragma unroll
      for (int ch = 0; ch < 4; ++ch) {
        uint32_t u[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) u[e] = __float_as_uint(v[8 * ch + e]);
        st_v8(xo + 8 * ch, u);
      }
      if constexpr (MIXED) {
        __nv_bfloat16* bo = XSo + row * 32;
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          uint32_t u[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const __nv_bfloat162 b2 = __floats2bfloat162_rn(v[16 * ch + 2 * e], v[16 * ch + 2 * e + 1]);
            u[e] = *reinterpret_cast<const uint32_t*>(&b2);
          }
          st_v8(bo + 16 * ch, u);
        }
      }
    }
  }
  if (!dead && ntw > 0 && wait(c.bar(w, BAR_GRDONE), (uint32_t)(ntw - 1) & 1u)) gram_back();

  // ---- partial results (fixed order: bit-reproducible) ----
  double trd = (double)tr_hi + (double)tr_lo, pgd = (double)pg_hi + (double)pg_lo;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    trd += __shfl_down_sync(kFull, trd, o);
    pgd += __shfl_down_sync(kFull, pgd, o);
  }
  bad = __reduce_or_sync(kFull, bad);
  if (lane == 0) {
    red[4 * w + qw][0] = trd;
    red[4 * w + qw][1] = pgd;
    red[4 * w + qw][2] = (double)bad;
    red[4 * w + qw][3] = dead ? 1.0 : 0.0;
  }
  named_sync(1 + w, 128);
  const int shi = slot0 + 2 * w, slo = shi + 1;
  if (t == 0) {
    double acc[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; ++i)
      for (int q = 0; q < 4; ++q) acc[q] += red[4 * w + i][q];
    for (int q = 0; q < 4; ++q) {
      a.sc_part[shi * 4 + q] = acc[q];
      a.sc_part[slo * 4 + q] = 0.0;
    }
  }
  constexpr int E2 = 32 * 32;
  const int r = 16 * (qw & 1) + (lane & 15);
  float g[32];
  {
    uint32_t gu[32];
    wait_st();
    ld32x32_async(tw + COL_ACC, gu);
    wait_ld();
    pin32(gu);
#pragma unroll
    for (int j = 0; j < 32; ++j) g[j] = __uint_as_float(gu[j]);
  }
#pragma unroll
  for (int cg = 0; cg < 2; ++cg) {
    if (cg == 0 && below) continue;  // below the diagonal: never read by the fold
    const size_t o = (size_t)gm * E2 + (size_t)r * 32 + 16 * cg + 8 * (lane >> 4);
    float* hi = a.gram_part + (size_t)shi * 2 * E2 + o;
    float* lo = a.gram_part + (size_t)slo * 2 * E2 + o;
    const float* H = g + 8 * cg;
    const float* Lw = g + 16 + 8 * cg;
    reinterpret_cast<float4*>(hi)[0] = make_float4(H[0] * kUnscale2, H[1] * kUnscale2, H[2] * kUnscale2, H[3] * kUnscale2);
    reinterpret_cast<float4*>(hi)[1] = make_float4(H[4] * kUnscale2, H[5] * kUnscale2, H[6] * kUnscale2, H[7] * kUnscale2);
    reinterpret_cast<float4*>(lo)[0] =
        make_float4(Lw[0] * kUnscale2, Lw[1] * kUnscale2, Lw[2] * kUnscale2, Lw[3] * kUnscale2);
    reinterpret_cast<float4*>(lo)[1] =
        make_float4(Lw[4] * kUnscale2, Lw[5] * kUnscale2, Lw[6] * kUnscale2, Lw[7] * kUnscale2);
  }
}

}  // namespace ts

// Split iteration, step 3, streaming form for KP = 32: CTA b takes tiles
// [b T / G, (b+1) T / G) of the T = ceil(n / 128) row tiles and partial slots
// 4 b .. 4 b + 3 (warpgroup w: 4 b + 2 w high parts and scalars, 4 b + 2 w + 1
// low parts).  Launch with ts::NT threads, ts::SMEM bytes of dynamic shared
// memory and at most one CTA per SM (it allocates all 512 TMEM columns).
// FULL: launched only for k = 32.
template <bool MIXED, bool FULL>
__global__ void __launch_bounds__(ts::NT, 1) update_stream_kernel(PassArgs a, const __grid_constant__ StreamMaps maps) {
  using namespace ts;
  volatile FistaState* vs = a.st;
  const int64_t pass = pass_to_run(a.st);
  if (pass < 0) return;
  extern __shared__ __align__(1024) uint8_t ts_smem_raw[];
  __shared__ __align__(8) uint64_t bars[NBARS];
  __shared__ uint32_t tslot;
  __shared__ int flags[2];
  __shared__ double red[8][4];
  StreamCta c;
  c.sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(ts_smem_raw) + 1023) & ~(uintptr_t)1023);
  c.sb = tc::saddr(c.sm);
  c.bars = tc::saddr(bars);
  c.flags = flags;
  const int64_t T = (a.n + R - 1) / R;
  c.t0 = T * (int64_t)blockIdx.x / gridDim.x;
  c.cnt = (int)(T * (int64_t)(blockIdx.x + 1) / gridDim.x - c.t0);
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::saddr(&tslot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int w = 0; w < 2; ++w) {
      bar_init_n(c.bar(w, BAR_FULL), 1);
      bar_init_n(c.bar(w, BAR_YREADY), 128);
      bar_init_n(c.bar(w, BAR_YGDONE), 1);
      bar_init_n(c.bar(w, BAR_GREADY), 128);
      bar_init_n(c.bar(w, BAR_GRDONE), 1);
    }
    bar_init_n(c.bars + 8u * 10u, 1);
    bar_init_n(c.bars + 8u * 11u, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    flags[0] = 0;
    flags[1] = vs->hooks;
  }
  // G(Y) (symmetric: its rows serve as the K-major B operand of y G), hi / lo
  if (tid < 256) {
    const int n = tid >> 3, ch = tid & 7;
    float g[4];
    load_row<4>(a.Gy + n * 32 + 4 * ch, g);
    split_store4(reinterpret_cast<float*>(c.sm + OFF_GH + tc::sw_chunk(n, ch)),
                 reinterpret_cast<float*>(c.sm + OFF_GL + tc::sw_chunk(n, ch)), g);
  }
  tc::fence_smem_to_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  c.tmem = tslot;
  if (warp < 8) {
    stream_compute<MIXED, FULL>(a, c, pass, 4 * (int)blockIdx.x, red);
  } else {
    if ((tid & 31) == 0) stream_helper(c, maps, pass, warp - 8);
    __syncwarp();
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) {
    tc::fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(c.tmem), "r"(TMEM_COLS) : "memory");
  }
}

}  // namespace fc
