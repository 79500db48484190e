// Row-local update of the split iteration on the fifth-generation tensor
// cores (tcgen05, sm_103a) for KP = 32 (17 <= k <= 32) and KP = 64 (33 <= k
// <= 64).
//
// Same arithmetic as update_kernel in pass_kernels.cuh, per row i:
//   y_i  = xbar^{n-1}_i + beta (xbar^{n-1}_i - xbar^{n-2}_i)          (X^n, Alg. 4)
//   SY_i = z_i + beta (z_i - z^{prev}_i)                             (S X^n by linearity)
//   q_i  = y_i G(Y)                                                  (share^n = Y^T Y)
//   xbar^n_i = P_simplex(y_i + 4 tau (SY_i - q_i))                   (Eq. "gradient_column", Alg. 1)
// with the trace term <xbar^{n-1}_i, z_i> of the loss update (Sect. 3), the
// projected-gradient norm ||y_i - xbar^n_i||^2, and the Gram partials of
// Xbar^n (the loss of the next pass) and of Y^{n+1} = Xbar^n + beta_{n+1}
// (Xbar^n - Xbar^{n-1}) (the share of the next pass).
//
// The two dense contractions of a tile of 32 rows are tcgen05.mma kind::tf32
// with the 3xTF32 split (x = hi + lo, products lo*hi + hi*lo + hi*hi), the
// operands read from shared memory through matrix descriptors and the
// accumulators in tensor memory (TMEM):
//   Y G   M = 64 tile rows (the operand's rows 32..63 are whatever follows the
//         tile in shared memory; those accumulator rows are never read), N = 32,
//         K = 32; Y and G in the K-major layout with 128-byte swizzle (a row of
//         32 floats fills 128 bytes, its 16-byte chunk c sits at chunk c ^ (row & 7),
//         groups of 8 rows 1024 bytes apart)
//   Gram  M = N = 64 features [Xbar^n | Y^{n+1}], K = the tile's 32 rows, A = B =
//         the transposed tile in K-major core matrices without swizzle; the
//         diagonal 32 x 32 blocks of the 64 x 64 result are the two Gram matrices.
// With M = 64, accumulator row r lives in TMEM lane 32 (r / 16) + r % 16.
// Each tile's products are the ones the warp-level form (mma.sync, 3xTF32,
// same K order) computes, so both forms give the same bits.
//
// One thread issues the MMAs and tcgen05.commit signals an mbarrier that the
// block waits on.  Per tile: wait for Y G, stage it, project the rows, then
// (after reading back the previous tile's Gram) write this tile's transposed
// rows and the next tile's extrapolated rows, and after one barrier issue the
// next tile's Y G and this tile's Gram together: two block barriers per tile.
// Every wait is bounded (a count of polls of bounded length, about one second
// in all): a block whose wait gives up records a timeout,
// issues no further MMAs, and the fold ends the run with status
// CLUSTER_ETIMEOUT.  Each tile's Gram starts from zero and is read back
// (tcgen05.ld) into float sums with round-to-nearest adds: the tensor core's
// accumulation does not round to nearest, and a long sum in TMEM drifts.
#pragma once
#include <algorithm>

#include "pass_kernels.cuh"

#ifndef FC_TC_UPDATE
#define FC_TC_UPDATE 1  // 0: KP = 32 uses the warp-level mma.sync update as well
#endif

namespace fc {
namespace tc {

// A wait gives up after kWaitPolls polls of at most kPollNs each (about one
// second; a tile's MMAs take microseconds).  A count, unlike a clock, does not
// run out while the kernel is not scheduled.
constexpr uint32_t kWaitPolls = 1u << 20, kPollNs = 1000u;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: start address / 16 (bits 0-13), leading
// byte offset / 16 (bits 16-29; unused by a swizzled K-major operand whose K
// slice lies inside one 128-byte row), stride byte offset / 16 (bits 32-45:
// 1024 bytes between groups of 8 rows), version 1 (bit 46), 128-byte swizzle
// (layout 2 in bits 61-63).
__device__ __forceinline__ uint64_t desc_k128(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(16 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46) | (2ull << 61);
}

// Descriptor of a K-major operand without swizzle, built from "core matrices"
// of 8 rows x 16 bytes (128 contiguous bytes): lbo = byte distance between
// core matrices adjacent in K, sbo = between core matrices adjacent in M / N.
__device__ __forceinline__ uint64_t desc_core(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: float32 accumulator (bits 4-5 = 1), A
// and B in TF32 (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N / 8
// in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
// arrive on the mbarrier once every MMA this thread issued so far has completed
__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
// poll: true if the phase with this parity has completed; the thread may
// suspend up to kPollNs waiting for it
__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kPollNs)
      : "memory");
  return ok != 0;
}
// true once the phase with this parity has completed; false when the wait gives up
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (uint32_t i = 0; i < kWaitPolls; ++i)
    if (bar_try(bar, parity)) return true;
  return false;
}
// ordinary shared-memory stores -> visible to the MMA's (async proxy) reads
__device__ __forceinline__ void fence_smem_to_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 TMEM lanes x 16 columns into a warp: thread t gets lane base + (t & 15),
// columns col + 8 (t >> 4) + j, j < 8 (shape 16x32bx2, half offset 8).
__device__ __forceinline__ void ld16x16(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.16x32bx2.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8], 8;"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// 32 TMEM lanes (this warp's quarter) x 32 columns: thread t gets lane base +
// t, columns col .. col + 31
__device__ __forceinline__ void ld32x32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16)
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// byte offset of 16-byte chunk c of row r in a 128-byte-swizzled tile
__device__ __forceinline__ int sw_chunk(int r, int c) { return r * 128 + ((c ^ (r & 7)) << 4); }

}  // namespace tc

template <int KP>
struct TcUpd {
  static constexpr bool ON = FC_TC_UPDATE && (KP == 32 || KP == 64);
  static constexpr int R = Lay<KP>::R;  // tile rows: 32 (KP = 32), 16 (KP = 64)
  // Operands in the K-major layout with 128-byte swizzle: a row of KP TF32
  // values spans KP / 32 atoms of 128 bytes; atom a of all the rows first
  // (the y tile: ATOM_Y bytes per atom; G(Y): ATOM_G), then atom a + 1.
  static constexpr int ATOMS = KP / 32;
  static constexpr int ATOM_Y = R * 128, ATOM_G = KP * 128;
  // Gram operand (the transposed tile, 2 KP feature rows x R tile rows, hi
  // and lo): K-major core matrices of 8 features x 4 tile rows; the one for
  // features 8 g.. and rows 4 c.. at g * CM_SBO + c * CM_LBO.  CM_SBO = 144
  // (36 words = 4 mod 32) spreads a warp's scalar stores over the banks (all
  // 32 for KP = 32; two lanes per bank for KP = 64).
  static constexpr int CM_SBO = 144, CM_LBO = (2 * KP / 8) * CM_SBO, TBYTES = (R / 4) * CM_LBO;
  // byte offsets from the 1024-aligned base: G hi / lo, Y hi / lo (the M = 64
  // read of the last Y lo atom runs up to 8 KB past its start, into TH: rows
  // that are ignored), the transposed tile hi / lo, the Y G staging rows
  // (stride QS floats)
  static constexpr int QS = KP + 4;
  static constexpr int GH = 0, GL = ATOMS * ATOM_G, YH = 2 * ATOMS * ATOM_G, YL = YH + ATOMS * ATOM_Y;
  static constexpr int TH = YL + ATOMS * ATOM_Y, TL = TH + TBYTES;
  static constexpr int QO = TL + TBYTES;
  static constexpr int BYTES = QO + R * QS * 4;
  __host__ __device__ static constexpr size_t smem() { return (size_t)BYTES + 1024; }  // + alignment slack
  // TMEM: y G (M = 64: the tile's rows in lanes 16 q + r, N = KP) at column 0,
  // the Gram (M = N = 2 KP) at D_GR
  static constexpr int TMEM_COLS = KP == 32 ? 128 : 256, D_YG = 0, D_GR = KP == 32 ? 64 : 128;
  static constexpr uint32_t ID_YG = tc::idesc_tf32(64, KP);
  static constexpr uint32_t ID_GR = tc::idesc_tf32(2 * KP, 2 * KP);
  static_assert(YL + (ATOMS - 1) * ATOM_Y + 8 * 1024 <= BYTES, "the M = 64 read of Y lo stays inside the allocation");
  static_assert(KP == 32 ? (TH == 16384 && TBYTES == 9216) : true, "KP = 32 layout unchanged");
};

// Per-block resources of the tcgen05 update: the 1024-aligned operand area,
// TMEM columns, two mbarriers (Y G done, Gram done), and the count of tiles the
// block has run (both barriers complete one phase per tile).
struct TcBlock {
  uint8_t* sm;
  uint32_t sbase;   // shared-window address of sm
  uint32_t tmem;
  uint32_t bar_yg, bar_gr;
  int* tmo_flag;    // [0] set when a wait gave up: no further MMAs are issued; [1] test hooks
  uint32_t tiles;
  bool dead;        // this warp saw a wait give up: no more waits or TMEM reads
};

// Allocate TMEM (warp 0) and initialise the barriers; all threads of the block.
template <int KP>
__device__ __forceinline__ void tc_begin(TcBlock& b, uint8_t* raw, uint64_t* bars, uint32_t* tslot, int* flag) {
  using U = TcUpd<KP>;
  b.sm = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
  b.sbase = tc::saddr(b.sm);
  b.bar_yg = tc::saddr(&bars[0]);
  b.bar_gr = tc::saddr(&bars[1]);
  b.tmo_flag = flag;
  b.tiles = 0;
  b.dead = false;
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc::saddr(tslot)),
                 "r"(U::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    tc::bar_init(b.bar_yg);
    tc::bar_init(b.bar_gr);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    flag[0] = flag[1] = 0;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  b.tmem = *tslot;
}

// Release TMEM once every thread's TMEM reads have completed.
template <int KP>
__device__ __forceinline__ void tc_end(const TcBlock& b) {
  tc::fence_before_sync();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    tc::fence_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(b.tmem), "r"(TcUpd<KP>::TMEM_COLS)
                 : "memory");
  }
}

// The row-local inputs of one tile row: loads, trace term, extrapolation.
struct TcRow {
  int64_t row;
  bool active;
  float y[4], sy[4], pv[4];
};

// One block's share of a pass: rows [p0, p1) in index order, partial results
// into slot `slot` of gram_part / sc_part (the layout update_kernel writes).
template <int KP, bool MIXED>
__device__ __forceinline__ void tc_update_range(const PassArgs& a, int64_t pass, int64_t p0, int64_t p1, int slot,
                                                TcBlock& b) {
  using L = Lay<KP>;
  using U = TcUpd<KP>;
  static_assert((KP == 32 || KP == 64) && L::R == U::R && L::VEC == 4 && L::T == KP / 4,
                "tile layout of the tcgen05 update");
  constexpr int KS = KP / 8;
  // Gram sums per thread: KP = 32, 8 entries (M = 64 accumulator read as 16
  // lanes x 16 columns); KP = 64, 32 entries (M = 128: 32 lanes x 32 columns)
  constexpr int GS = KP == 32 ? 8 : 32;
  uint8_t* sm = b.sm;
  const uint32_t sbase = b.sbase, tmem = b.tmem;

  const float* Zcur = ((pass + 1) & 1) ? a.Z1 : a.Z0;  // S Xbar^{pass}
  const float* Zprv = (pass & 1) ? a.Z1 : a.Z0;        // S Xbar^{pass-1}
  const FistaState* st = a.st;
  const float beta = (float)st->beta, beta_next = (float)st->beta_next;
  const float tau4 = (float)(4.0 * st->tau);
  const float* P = (pass & 1) ? a.X1 : a.X0;  // Xbar^{pass}
  float* Qx = (pass & 1) ? a.X0 : a.X1;       // Xbar^{pass-1} in, Xbar^{pass+1} out
  __nv_bfloat16* XSo = (pass & 1) ? a.XS0 : a.XS1;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int tiw = lane / L::T, lt = lane % L::T;
  const int team = warp * L::TPW + tiw;  // tile row of this team
  const int f0 = lt * L::VEC;            // = 4 lt: this lane's 16-byte chunk of the row
  const int k = a.k;

  // TMEM read-back roles: lane quarter qd (the lanes this warp may access) and
  // column group cg.  Y G: warps with qd < 2 read accumulator rows
  // 16 qd + (lane & 15), columns 16 cg + 8 (lane >> 4) + j.  Gram: matrix
  // gm = qd / 2 (0: Xbar^n, 1: Y^{n+1}), its row 16 (qd & 1) + (lane & 15),
  // columns 16 cg + 8 (lane >> 4) + j of that diagonal block.
  const int qd = warp & 3, cg = warp >> 2, gm = qd >> 1;
  const uint32_t t_lanes = (uint32_t)(32 * qd) << 16;
  float gsum[GS];
#pragma unroll
  for (int j = 0; j < GS; ++j) gsum[j] = 0.f;
  // KP = 64: Gram rows 32-63 of a block against its columns 0-31 lie below the
  // diagonal, which the fold never reads: those warps skip them
  const bool gskip = KP == 64 && (qd & 1) && cg == 0;

  float tr_hi = 0.f, tr_lo = 0.f, pg_hi = 0.f, pg_lo = 0.f;
  int bad = 0;
  bool dead = b.dead;
  const uint32_t ph0 = b.tiles;
  const uint32_t ntiles = (uint32_t)((p1 - p0 + L::R - 1) / L::R);

  auto wait_bar = [&](uint32_t bar, uint32_t phase) {
    if (!dead) {
      dead = !tc::bar_wait(bar, phase & 1u);
      dead = __any_sync(kFull, dead);
      if (dead) *b.tmo_flag = 1;
    }
    tc::fence_after_sync();
  };
  // loads of tile `tile`, its trace term, y and SY; y into the Y G operand
  auto load_tile = [&](uint32_t tile, TcRow& t) {
    const int64_t base = p0 + (int64_t)tile * L::R;
    const int64_t pos = base + team;
    t.active = pos < p1;
    t.row = t.active ? pos : base;
    float acc[4], qv[4], zp[4];
    load_row<4>(Zcur + t.row * KP + f0, acc);
    load_row<4>(P + t.row * KP + f0, t.pv);
    load_row<4>(Qx + t.row * KP + f0, qv);
    load_row<4>(Zprv + t.row * KP + f0, zp);
    float d = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      d = fmaf(t.pv[q], acc[q], d);
      if (!isfinite(acc[q])) bad = 1;
    }
    d = team_sum<L::T>(d);
    if (t.active && lt == 0) two_sum_acc(tr_hi, tr_lo, d);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      t.y[q] = fmaf(beta, t.pv[q] - qv[q], t.pv[q]);
      t.sy[q] = fmaf(beta, acc[q] - zp[q], acc[q]);
    }
    const int yo = (lt >> 3) * U::ATOM_Y + tc::sw_chunk(team, lt & 7);
    split_store4(reinterpret_cast<float*>(sm + U::YH + yo), reinterpret_cast<float*>(sm + U::YL + yo), t.y);
  };
  auto issue_yg = [&]() {
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      // K step ks: atom ks / 4, 32 bytes (8 TF32) per step inside the atom
      const int oy = (ks >> 2) * U::ATOM_Y + 32 * (ks & 3), og = (ks >> 2) * U::ATOM_G + 32 * (ks & 3);
      const uint64_t ah = tc::desc_k128(sbase + U::YH + oy), al = tc::desc_k128(sbase + U::YL + oy);
      const uint64_t bh = tc::desc_k128(sbase + U::GH + og), bl = tc::desc_k128(sbase + U::GL + og);
      tc::mma(tmem + U::D_YG, al, bh, U::ID_YG, ks > 0);
      tc::mma(tmem + U::D_YG, ah, bl, U::ID_YG, 1);
      tc::mma(tmem + U::D_YG, ah, bh, U::ID_YG, 1);
    }
    // test hook (cluster_test_hooks bit 0): withhold the commit, so the waits on it give up
    if (!(b.tmo_flag[1] & 1)) tc::commit(b.bar_yg);
  };
  auto issue_gram = [&]() {
#pragma unroll
    for (int ks = 0; ks < L::R / 8; ++ks) {
      const uint64_t th = tc::desc_core(sbase + U::TH + 2 * U::CM_LBO * ks, U::CM_LBO, U::CM_SBO);
      const uint64_t tl = tc::desc_core(sbase + U::TL + 2 * U::CM_LBO * ks, U::CM_LBO, U::CM_SBO);
      tc::mma(tmem + U::D_GR, tl, th, U::ID_GR, ks > 0);
      tc::mma(tmem + U::D_GR, th, tl, U::ID_GR, 1);
      tc::mma(tmem + U::D_GR, th, th, U::ID_GR, 1);
    }
    tc::commit(b.bar_gr);
  };

  // this tile's Gram into the float sums (round-to-nearest adds).  KP = 32:
  // M = 64 accumulator, Gram row 16 (qd & 1) + (lane & 15) of matrix gm in
  // lane 32 qd + (lane & 15), columns 16 cg + 8 (lane >> 4) + j of its diagonal
  // block; KP = 64: M = 128, Gram row 32 (qd & 1) + lane of matrix gm in lane
  // 32 qd + lane, columns 32 cg + j of its diagonal block
  auto gram_read = [&]() {
    if constexpr (KP == 32) {
      float g[8];
      tc::ld16x16(tmem + t_lanes + U::D_GR + 32 * gm + 16 * cg, g);
#pragma unroll
      for (int j = 0; j < 8; ++j) gsum[j] += g[j];
    } else {
      if (!gskip) {
        float g[32];
        tc::ld32x32(tmem + t_lanes + U::D_GR + KP * gm + 32 * cg, g);
#pragma unroll
        for (int j = 0; j < GS; ++j) gsum[j] += g[j];
      }
    }
  };

  if (tid == 0) b.tmo_flag[1] = ((const volatile FistaState*)st)->hooks;  // read by tid 0 only
  TcRow cur;
  if (ntiles > 0) {
    // G(Y), B operand of Y G: row n holds G[n][.] (= column n: G(Y) is
    // symmetric), hi / lo.  No MMA is in flight: the previous range waited for
    // all of its MMAs.
    for (int e = tid; e < KP * KP / 4; e += L::NT) {
      const int n = e / (KP / 4), c = e % (KP / 4);
      float v[4];
      load_row<4>(a.Gy + n * KP + 4 * c, v);
      const int go = (c >> 3) * U::ATOM_G + tc::sw_chunk(n, c & 7);
      split_store4(reinterpret_cast<float*>(sm + U::GH + go), reinterpret_cast<float*>(sm + U::GL + go), v);
    }
    load_tile(0, cur);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      if (!*reinterpret_cast<volatile int*>(b.tmo_flag)) issue_yg();
    }
  }
  for (uint32_t it = 0; it < ntiles; ++it) {
    // the next tile's rows (4 arrays of up to 32 consecutive rows) into L2, a
    // tile ahead of their loads
    if (tid == 0 && it + 1 < ntiles) {
      const int64_t r0 = p0 + (int64_t)(it + 1) * L::R;
      const int64_t rows = (p1 - r0 < L::R) ? p1 - r0 : L::R;
      const uint32_t bytes = (uint32_t)(rows * KP * sizeof(float));
      tc::prefetch_l2(Zcur + r0 * KP, bytes);
      tc::prefetch_l2(P + r0 * KP, bytes);
      tc::prefetch_l2(Qx + r0 * KP, bytes);
      tc::prefetch_l2(Zprv + r0 * KP, bytes);
    }
    // y G of this tile -> staging rows
    wait_bar(b.bar_yg, ph0 + it);
    // the tile's R rows sit in lane quarters 0 .. R/16 - 1; the two warps of a
    // quarter take KP / 2 columns each, 16 per load
    if (qd < U::R / 16 && !dead) {
#pragma unroll
      for (int i = 0; i < KP / 32; ++i) {
        float v[8];
        tc::ld16x16(tmem + t_lanes + U::D_YG + (KP / 2) * cg + 16 * i, v);
        float* qo = reinterpret_cast<float*>(sm + U::QO) + (16 * qd + (lane & 15)) * U::QS + (KP / 2) * cg + 16 * i +
                    8 * (lane >> 4);
        *reinterpret_cast<float4*>(qo) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4*>(qo + 4) = make_float4(v[4], v[5], v[6], v[7]);
      }
    }
    tc::fence_before_sync();
    __syncthreads();
    float qq[4];
    load_row<4>(reinterpret_cast<const float*>(sm + U::QO) + team * U::QS + f0, qq);

    float v[4], x[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) v[q] = fmaf(tau4, cur.sy[q] - qq[q], cur.y[q]);
    project_simplex<KP>(v, x, f0, k);
    float pg = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float dd = cur.y[q] - x[q];
      pg = fmaf(dd, dd, pg);
      if (!isfinite(x[q])) bad = 1;
    }
    pg = team_sum<L::T>(pg);
    if (cur.active && lt == 0) two_sum_acc(pg_hi, pg_lo, pg);
    if (cur.active) {
      store_row<4>(Qx + cur.row * KP + f0, x);
      if constexpr (MIXED) store_row_bf16<4>(XSo + cur.row * KP + f0, x);
    }
    // the previous tile's Gram is complete once its barrier phase is: read it
    // back before this tile's transposed rows overwrite the operand
    if (it > 0) {
      wait_bar(b.bar_gr, ph0 + it - 1);
      if (!dead) gram_read();
    }
    // transposed tile: Xbar^n in feature rows 0..KP-1, Y^{n+1} = xbar^n +
    // beta_{n+1} (xbar^n - xbar^{n-1}) in KP..2KP-1 (KP / 8 core-matrix groups further)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float xv = cur.active ? x[q] : 0.f;
      const float yv = cur.active ? fmaf(beta_next, x[q] - cur.pv[q], x[q]) : 0.f;
      uint32_t hx, lx, hy, ly;
      split_tf32(xv, hx, lx);
      split_tf32(yv, hy, ly);
      const int m = f0 + q;
      const int o = (m >> 3) * U::CM_SBO + (team >> 2) * U::CM_LBO + (m & 7) * 16 + (team & 3) * 4;
      *reinterpret_cast<uint32_t*>(sm + U::TH + o) = hx;
      *reinterpret_cast<uint32_t*>(sm + U::TL + o) = lx;
      *reinterpret_cast<uint32_t*>(sm + U::TH + o + (KP / 8) * U::CM_SBO) = hy;
      *reinterpret_cast<uint32_t*>(sm + U::TL + o + (KP / 8) * U::CM_SBO) = ly;
    }
    // the next tile's rows (its Y G operand is free: this tile's Y G completed)
    const bool more = it + 1 < ntiles;
    if (more) load_tile(it + 1, cur);
    tc::fence_smem_to_async();
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      if (!*reinterpret_cast<volatile int*>(b.tmo_flag)) {
        if (more) issue_yg();
        issue_gram();
      }
    }
  }
  if (ntiles > 0) {
    wait_bar(b.bar_gr, ph0 + ntiles - 1);
    if (!dead) gram_read();
  }
  b.tiles = ph0 + ntiles;
  b.dead = dead;

  // ---- block reductions (fixed order => bit-reproducible) ----
  double* dred = reinterpret_cast<double*>(sm + U::QO);
  double tr_acc = (double)tr_hi + (double)tr_lo, pg_acc = (double)pg_hi + (double)pg_lo;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tr_acc += __shfl_down_sync(kFull, tr_acc, o);
    pg_acc += __shfl_down_sync(kFull, pg_acc, o);
  }
  bad = __reduce_or_sync(kFull, bad);
  if (lane == 0) {
    dred[warp * 4 + 0] = tr_acc;
    dred[warp * 4 + 1] = pg_acc;
    dred[warp * 4 + 2] = (double)bad;
    dred[warp * 4 + 3] = dead ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0, p = 0, bd = 0, w = 0;
    for (int i = 0; i < L::WARPS; ++i) {
      t += dred[i * 4 + 0];
      p += dred[i * 4 + 1];
      bd += dred[i * 4 + 2];
      w += dred[i * 4 + 3];
    }
    a.sc_part[slot * 4 + 0] = t;
    a.sc_part[slot * 4 + 1] = p;
    a.sc_part[slot * 4 + 2] = bd;
    a.sc_part[slot * 4 + 3] = w;  // warps whose wait gave up (fold: CLUSTER_ETIMEOUT)
  }
  if constexpr (KP == 32) {
    float* go = a.gram_part + (size_t)slot * 2 * L::E2 + gm * L::E2 + (16 * (qd & 1) + (lane & 15)) * KP + 16 * cg +
                8 * (lane >> 4);
    *reinterpret_cast<float4*>(go) = make_float4(gsum[0], gsum[1], gsum[2], gsum[3]);
    *reinterpret_cast<float4*>(go + 4) = make_float4(gsum[4], gsum[5], gsum[6], gsum[7]);
  } else if (!gskip) {
    // (skipped: below the diagonal, never read by the fold)
    float* go = a.gram_part + (size_t)slot * 2 * L::E2 + gm * L::E2 + (32 * (qd & 1) + lane) * KP + 32 * cg;
#pragma unroll
    for (int j = 0; j < GS; j += 4)
      *reinterpret_cast<float4*>(go + j) = make_float4(gsum[j], gsum[j + 1], gsum[j + 2], gsum[j + 3]);
  }
  // the staging rows (dred) are written again only after the next range's
  // first barrier, which every thread reaches after tid 0 has read them
}

// Split iteration, step 3, for KP = 32: block b = upd_block0 + blockIdx.x takes
// rows [b n / parts, (b+1) n / parts) and partial slot b (as update_kernel).
template <int KP, bool MIXED>
__global__ void __launch_bounds__(Lay<KP>::NT, Lay<KP>::MINB) update_tc_kernel(PassArgs a) {
  const int64_t pass = pass_to_run(a.st);
  if (pass < 0) return;
  const int parts = a.upd_parts > 0 ? a.upd_parts : (int)gridDim.x;
  const int blk = a.upd_block0 + (int)blockIdx.x;
  const int64_t p0 = a.n * (int64_t)blk / parts;
  const int64_t p1 = a.n * (int64_t)(blk + 1) / parts;
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  __shared__ uint64_t bars[2];
  __shared__ uint32_t tslot;
  __shared__ int tmo_flag[2];
  TcBlock b;
  tc_begin<KP>(b, tc_smem_raw, bars, &tslot, tmo_flag);
  tc_update_range<KP, MIXED>(a, pass, p0, p1, blk, b);
  tc_end<KP>(b);
}

// Resident blocks per SM of a kernel that allocates tmem_cols TMEM columns per
// block, from its registers, shared memory and threads.  The runtime's
// occupancy query reports one block per SM for any kernel that uses tcgen05
// (it cannot know how many TMEM columns the kernel allocates), which would
// leave three quarters of every SM idle.
inline int tc_blocks_per_sm(const void* fn, int threads, size_t dyn_smem, int tmem_cols) {
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 1;
  int dev = 0, regs_sm = 0, smem_sm = 0, smem_res = 0, thr_sm = 0, blk_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&smem_res, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  cudaDeviceGetAttribute(&blk_sm, cudaDevAttrMaxBlocksPerMultiprocessor, dev);
  const int warps = (threads + 31) / 32;
  const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;  // per-warp allocation unit of 256 registers
  int occ = 512 / tmem_cols;
  if (regs_warp > 0) occ = std::min(occ, (regs_sm / regs_warp) / warps);
  occ = std::min(occ, smem_sm / (int)(fa.sharedSizeBytes + dyn_smem + (size_t)smem_res));
  occ = std::min(occ, thr_sm / threads);
  occ = std::min(occ, blk_sm);
  return occ < 1 ? 1 : occ;
}

}  // namespace fc
