// Fused FISTA pass for similarity-based fuzzy clustering on sm_103a.
//
// One launch of fista_pass_kernel is one iteration of the paper's parallel
// FISTA (Algorithm 4) with its loss evaluation, restructured so that S is
// streamed once per iteration:
//
//   z_i   = (S Xbar^{n-1})_i                       product with S (gather)
//   p_i   = <xbar^{n-1}_i, z_i>                    trace term of f(Xbar^{n-1})
//   y_i   = xbar^{n-1}_i + beta (xbar^{n-1}_i - xbar^{n-2}_i)       (X^n)
//   (SY)_i = z_i + beta (z_i - z^{prev}_i)         linearity: S X^n without a
//                                                  second product with S
//   q_i   = y_i G(Y)                               G(Y) = Y^T Y = share^n
//   xbar^n_i = P_simplex(y_i + 4 tau ((SY)_i - q_i))   gradient step of
//                                                  Eq. "gradient_column"
//   Gram partials of Xbar^n^T Xbar^n (for the loss) and of Y^{n+1}^T Y^{n+1},
//   where y^{n+1}_i = xbar^n_i + beta_{n+1} (xbar^n_i - xbar^{n-1}_i) is the
//   next pass's extrapolated row: the momentum schedule t_n does not depend
//   on the data, so beta_{n+1} is known one pass ahead
//   ||y_i - xbar^n_i||^2                           projected-gradient norm
//
// fold_kernel sums the Gram partials in float64 and hands G(Y^{n+1}) (the
// "share" of the next iteration of Algorithm 4) to the next pass;
// f(Xbar^{n-1}) = ||S||^2 - 2 sum_i p_i + ||Xbar^{n-1 T} Xbar^{n-1}||^2 is the
// trace identity of Sect. 3 ("Loss Update").
//
// Rows are grouped into tiles of R rows per block (team layout: iter_common.cuh).
// For 16 <= KP <= 64 the tile's dense contractions (Y G and the two Gram
// accumulations) run on the tensor cores (warp-level mma, 3xTF32); otherwise
// each thread accumulates float32 blocks of the upper Gram triangle.  Rows of
// very high degree are split into chunks whose partial products are computed
// before the row's update (heavy_kernel, or spmm_kernel in the split form).
#pragma once
#include "iter_common.cuh"
#include "spmm_kernels.cuh"

namespace fc {

// Symmetric Gram accumulation: the KP x KP matrix is cut into BS x BS blocks
// and only blocks (I, J) with I <= J are accumulated ("tasks"); the fold
// mirrors them.  Two matrices per pass (Gram of Xbar^n and of Y^{n+1}), one in
// an objective-only pass.  Threads take one task each and split the tile's
// rows into GROUPS interleaved groups (or several tasks each when there are
// more tasks than threads).
template <int KP, bool EVAL>
struct GramLay {
  static constexpr int NT = Lay<KP>::NT;
  static constexpr int BS = KP < 4 ? KP : 4;
  static constexpr int NB1 = KP / BS;
  static constexpr int NBLK = NB1 * (NB1 + 1) / 2;
  static constexpr int MATS = EVAL ? 1 : 2;
  static constexpr int TASKS = MATS * NBLK;
  static constexpr int TPT = TASKS <= NT ? 1 : (TASKS + NT - 1) / NT;
  static constexpr int GROUPS = TASKS <= NT ? NT / TASKS : 1;
  static constexpr int ACTIVE = TASKS <= NT ? GROUPS * TASKS : NT;
};

// Task t of a GramLay -> (matrix m, block row I, block column J >= I).
__device__ __forceinline__ void gram_task(int t, int nblk, int nb1, int& m, int& I, int& J) {
  m = t / nblk;
  int bi = t % nblk;
  I = 0;
  while (bi >= nb1 - I) {
    bi -= nb1 - I;
    ++I;
  }
  J = I + bi;
}

// Block b (row order) of the 16 x 8 blocks (mi, nj) with nj >= 2 mi of a
// matrix with nbj block columns: the blocks holding entries on or above the
// diagonal.
__device__ __forceinline__ void tri_block(int b, int nbj, int& mi, int& nj) {
  mi = 0;
  while (b >= nbj - 2 * mi) {
    b -= nbj - 2 * mi;
    ++mi;
  }
  nj = 2 * mi + b;
}

// ---- warp-level tensor-core helpers (mma.sync m16n8k8, TF32 inputs, FP32 accumulate) ----
// Fragment layout (lane = 4 g + t): A 16x8 row-major a0 = A[g][t], a1 = A[g+8][t],
// a2 = A[g][t+4], a3 = A[g+8][t+4]; B 8x8 b0 = B[t][g], b1 = B[t+4][g];
// D 16x8 d0 = D[g][2t], d1 = D[g][2t+1], d2 = D[g+8][2t], d3 = D[g+8][2t+1].
__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x ~ hi + lo with both parts TF32 values (the 3xTF32 split; hi keeps the top
// 11 significant bits, lo the next 11, so hi + lo carries about 22 bits of x)
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x) & 0xffffe000u;
  lo = to_tf32(x - __uint_as_float(hi));
}
__device__ __forceinline__ void mma_tf32(float* d, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Tensor-core layout of the update for 16 <= KP <= 64.  Y G: the R x KP tile
// of extrapolated rows times G(Y) as (R/16) x (KP/8) output blocks, one per
// warp.  Gram matrices: 16 x 8 feature blocks, TB of them, spread over the
// warps (BPW per warp, consecutive blocks sharing their A fragment); when
// there are fewer blocks than warps the tile rows are split KSPLIT ways and the
// partial blocks summed at the end in a fixed order.  Every product is 3xTF32
// (x = hi + lo, hi*hi + hi*lo + lo*hi), with the split done once when a value
// is written to shared memory.  Strides: TSA (= 4 mod 32 in words) makes the
// row-major fragment reads conflict-free, TSB (= 8 mod 16) the transposed
// Gram reads and the float2 stores of Y G.
//
// KP = 64 and 128 (the update only, not the objective-only pass): the same
// Y G; the Gram blocks are only those on or above the diagonal (16 x 8
// blocks (mi, nj) with nj >= 2 mi: the fold reads the upper triangle), TRIB
// per matrix, spread evenly over the warps (TPW_B per warp, in (matrix, mi,
// nj) order, so a warp's A fragment changes at most once or twice).  Each
// block's products and their order are those of the full square, so the
// entries the fold reads keep their bits; at KP = 64 the triangle is 40 of
// the square's 64 blocks, at KP = 128 the square would need 16 blocks of
// accumulators per warp, beyond the register budget of a 512-thread block.
// KP = 128 also splits Y G's 16 K steps into two accumulation chains (YG2).
template <int KP, bool EVAL>
struct MmaLay {
  static constexpr bool TRI = (KP == 64 || KP == 128) && !EVAL;
  static constexpr bool YG2 = KP == 128 && !EVAL;
  static constexpr bool ON = (KP >= 16 && KP <= 64) || TRI;
  static constexpr int TSA = KP + 4;
  static constexpr int TSB = KP + 8;
  static constexpr int KS = KP / 8;                     // K steps of Y G
  static constexpr int MATS = EVAL ? 1 : 2;
  static constexpr int GBLK = ON ? (KP / 16) * (KP / 8) : 1;  // 16x8 blocks per matrix
  static constexpr int TRIB = (KP / 16) * (KP / 16 + 1);        // blocks with nj >= 2 mi per matrix
  static constexpr int TPW_B = TRI ? MATS * TRIB / Lay<KP>::WARPS : 1;
  static_assert(!TRI || TPW_B * Lay<KP>::WARPS == MATS * TRIB, "triangle blocks per warp");
  static constexpr int TB = TRI ? Lay<KP>::WARPS : MATS * GBLK;
  static constexpr int WARPS = Lay<KP>::WARPS;
  static constexpr int KSPLIT = TB >= WARPS ? 1 : WARPS / TB;
  static constexpr int BPW = TB >= WARPS ? TB / WARPS : 1;
  static constexpr int RS = Lay<KP>::R / 8;             // K steps of a Gram over one tile
  static_assert(!ON || (Lay<KP>::R % 16 == 0 && (Lay<KP>::R / 16) * KS == WARPS), "Y G blocks != warps");
  static_assert(!ON || (TB % WARPS == 0 || WARPS % TB == 0), "Gram blocks do not tile the warps");
  static_assert(!ON || RS % KSPLIT == 0, "row split");
  static_assert(!ON || BPW == 1 || (KP / 8) % BPW == 0, "blocks of a warp share one A fragment");
  // shared floats: G fragments (2 KP^2 unless eval), Y hi/lo (TSA), Y G and
  // four hi/lo tiles of Xbar^n and Y^{n+1} (TSB)
  __host__ __device__ static constexpr size_t floats(bool eval) {
    return (eval ? 0 : 2 * (size_t)KP * KP) + 2 * (size_t)Lay<KP>::R * TSA + 5 * (size_t)Lay<KP>::R * TSB;
  }
};

__device__ __forceinline__ void split_store4(float* hi, float* lo, const float* v) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) split_tf32(v[q], h[q], l[q]);
  *reinterpret_cast<uint4*>(hi) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(lo) = make_uint4(l[0], l[1], l[2], l[3]);
}

__device__ __forceinline__ void mma3_tf32(float* d, const uint32_t* ah, const uint32_t* al, const uint32_t* bh,
                                          const uint32_t* bl) {
  mma_tf32(d, al, bh);
  mma_tf32(d, ah, bl);
  mma_tf32(d, ah, bh);
}

// hi + lo += x with the rounding error of the add kept in lo (Knuth's TwoSum)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bp = s - hi;
  const float err = (hi - (s - bp)) + (x - bp);
  hi = s;
  lo += err;
}

// Euclidean projection of one row onto the unit simplex (the row's KP values
// spread over the T lanes of a team, VEC per lane; features >= k are padding).
// Michelot's active-set iteration: theta = (sum_{a in A} v_a - 1) / |A|, then
// drop every a with v_a <= theta, until A is stable.  It reaches the same
// threshold as Algorithm 1 (sort + cumulative sums) without sorting.  The
// loop runs until every team of the warp is stable.
template <int KP>
__device__ __forceinline__ void project_simplex(const float* v, float* x, int f0, int k) {
  using L = Lay<KP>;
  bool act[L::VEC];
  float s = 0.f, c = 0.f;
#pragma unroll
  for (int q = 0; q < L::VEC; ++q) {
    act[q] = (f0 + q) < k;
    s += act[q] ? v[q] : 0.f;
    c += act[q] ? 1.f : 0.f;
  }
  s = team_sum<L::T>(s);
  c = team_sum<L::T>(c);
  // c counts at most KP entries; the approximate quotient (2 ulp) is ample for
  // a threshold that only needs float32 accuracy
  float theta = __fdividef(s - 1.0f, c);
  for (int it = 0; it <= KP; ++it) {
    float s2 = 0.f, c2 = 0.f;
#pragma unroll
    for (int q = 0; q < L::VEC; ++q) {
      act[q] = act[q] && (v[q] > theta);
      s2 += act[q] ? v[q] : 0.f;
      c2 += act[q] ? 1.f : 0.f;
    }
    s2 = team_sum<L::T>(s2);
    c2 = team_sum<L::T>(c2);
    const bool changed = c2 != c;
    if (changed) {
      s = s2;
      c = c2;
      theta = __fdividef(s - 1.0f, c);
    }
    if (!__any_sync(kFull, changed)) break;
  }
#pragma unroll
  for (int q = 0; q < L::VEC; ++q) x[q] = ((f0 + q) < k) ? fmaxf(v[q] - theta, 0.0f) : 0.0f;
}

template <int KP>
__host__ __device__ constexpr size_t pass_smem_bytes(bool eval) {
  using L = Lay<KP>;
  // Gy (KP*KP) unless eval, then the R-row tiles (xn, yn, ys [, q]), which the
  // end-of-kernel reductions reuse
  if (MmaLay<KP, false>::ON) return sizeof(float) * MmaLay<KP, false>::floats(eval) + 64;
  const size_t tiles = 3 * (size_t)L::R * KP;
  const size_t red = eval ? (size_t)GramLay<KP, true>::ACTIVE * GramLay<KP, true>::BS * GramLay<KP, true>::BS
                          : (size_t)GramLay<KP, false>::ACTIVE * GramLay<KP, false>::BS * GramLay<KP, false>::BS;
  return sizeof(float) * ((eval ? 0 : (size_t)L::E2) + (tiles > red ? tiles : red)) + 64;
}

// Split update (update_kernel, batch_update_kernel) for KP >= 64: the next
// tile's four input rows (z, xbar^{n}, xbar^{n-1}, z^{prev}; 16 bytes per
// lane) are staged in shared memory by cp.async while the current tile is
// computed, behind the pass's own shared memory (the k = 64 class of the
// batched workload: update 2.91 -> 2.78 ms; for KP = 16 and 32 the extra 16
// KB cost a resident block per SM and time)
template <int KP>
__host__ __device__ constexpr bool update_prefetch() { return Lay<KP>::VEC == 4 && KP >= 64; }
template <int KP>
__host__ __device__ constexpr size_t update_stage_offset() { return (pass_smem_bytes<KP>(false) + 15) / 16 * 16; }
template <int KP>
__host__ __device__ constexpr size_t update_smem_bytes() {
  return update_prefetch<KP>() ? update_stage_offset<KP>() + 4 * sizeof(float) * (size_t)Lay<KP>::R * KP
                               : pass_smem_bytes<KP>(false);
}

__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// One block's share of a pass: positions [p0, p1) of the row order, partial
// results into slot `slot` of gram_part / sc_part.  `pass` is the index of the
// newest iterate (the buffer parity), or the evaluated buffer when EVAL.
// EVAL: objective-only (z = S X, p_i, Gram of X; no update).
template <int KP, bool MIXED, bool EVAL, bool SPLIT = false>
__device__ __forceinline__ void pass_range(const PassArgs& a, int64_t pass, int64_t p0, int64_t p1, int slot,
                                           float* smem) {
  static_assert(!(SPLIT && EVAL), "the split update has no objective-only form");
  // SPLIT: rows in index order, z_i read from the product spmm_kernel stored
  // (Z_{(pass+1)&1}), the previous product from Z_{pass&1}; nothing gathered here
  const float* Zcur = ((pass + 1) & 1) ? a.Z1 : a.Z0;
  const float* Zprv = (pass & 1) ? a.Z1 : a.Z0;
  using L = Lay<KP>;
  FistaState* st = a.st;
  const float beta = EVAL ? 0.f : (float)st->beta;
  const float beta_next = EVAL ? 0.f : (float)st->beta_next;
  const float tau4 = EVAL ? 0.f : (float)(4.0 * st->tau);
  const float* P = (pass & 1) ? a.X1 : a.X0;          // Xbar^{pass}
  float* Q = (pass & 1) ? a.X0 : a.X1;                 // Xbar^{pass-1} in, Xbar^{pass+1} out
  const void* Xg = MIXED ? (const void*)((pass & 1) ? a.XS1 : a.XS0) : (const void*)P;
  __nv_bfloat16* XSo = (pass & 1) ? a.XS0 : a.XS1;

  using M = MmaLay<KP, EVAL>;
  constexpr int TS = M::ON ? M::TSB : KP;  // stride of the xn / yn tiles
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tiw = lane / L::T, lt = lane % L::T;
  const int team = warp * L::TPW + tiw;
  const int f0 = lt * L::VEC;
  const int k = a.k;
  const int mg = lane >> 2, mt = lane & 3;  // mma fragment coordinates (lane = 4 mg + mt)

  // shared memory.  FFMA path: Gs | xn | yn | ys.  MMA path: G fragments |
  // Y hi | Y lo | Y G | Xbar^n hi | lo | Y^{n+1} hi | lo.
  float* Gs = smem;
  uint4* Gf = reinterpret_cast<uint4*>(smem);
  float* tiles = smem + (EVAL ? 0 : (M::ON ? 2 * L::E2 : L::E2));
  float* ys = tiles + (M::ON ? 0 : 2 * L::R * KP);
  float* ysl = ys + L::R * M::TSA;
  float* qs = ysl + L::R * M::TSA;
  float* xn_t = M::ON ? qs + L::R * TS : tiles;
  float* xn_l = xn_t + L::R * TS;
  float* yn_t = M::ON ? xn_l + L::R * TS : tiles + L::R * KP;
  float* yn_l = yn_t + L::R * TS;

  // Y G block of this warp (MMA path): rows 16 ym .. +16, columns 8 yn .. +8
  const int ym = M::ON ? warp / M::KS : 0, yn = M::ON ? warp % M::KS : 0;
  if constexpr (!EVAL) {
    if constexpr (M::ON) {
      // B fragments of G(Y), split hi/lo once: Gf[(yb * KS + ks) * 32 + lane]
      for (int e = tid; e < M::KS * M::KS * 32; e += L::NT) {
        const int ln = e & 31, ks = (e >> 5) % M::KS, yb = (e >> 5) / M::KS;
        const int r0 = 8 * ks + (ln & 3), c0 = 8 * yb + (ln >> 2);
        uint32_t h0, l0, h1, l1;
        split_tf32(a.Gy[r0 * KP + c0], h0, l0);
        split_tf32(a.Gy[(r0 + 4) * KP + c0], h1, l1);
        Gf[e] = make_uint4(h0, h1, l0, l1);
      }
    } else {
      for (int e = tid; e < L::E2; e += L::NT) Gs[e] = a.Gy[e];
    }
  }
  __syncthreads();

  // KP = 128: this warp's triangle blocks, decoded once: mat << 16 | mi << 8 | nj
  __shared__ int tri_tab[M::TRI ? L::WARPS * M::TPW_B : 1];
  if constexpr (M::TRI) {
    if (lane < M::TPW_B) {
      const int bb = warp * M::TPW_B + lane;
      int mi, nj;
      tri_block(bb % M::TRIB, KP / 8, mi, nj);
      tri_tab[warp * M::TPW_B + lane] = ((bb / M::TRIB) << 16) | (mi << 8) | nj;
    }
    __syncwarp();
  }
  // Gram blocks of this warp (MMA path)
  const int mb0 = M::ON ? (warp % (M::TB / M::BPW)) * M::BPW : 0;   // first block
  const int mks = M::ON ? warp / (M::TB / M::BPW) : 0;                // row-split part
  const bool mon = M::ON && mb0 < M::TB;
  const int mmat = mb0 / (M::GBLK > 0 ? M::GBLK : 1);
  const int mrem = mb0 % (M::GBLK > 0 ? M::GBLK : 1);
  const int mmi = mrem / (KP / 8 > 0 ? KP / 8 : 1), mnj0 = mrem % (KP / 8 > 0 ? KP / 8 : 1);
  constexpr int MACC = M::ON ? (M::TRI ? M::TPW_B : M::BPW) : 1;
  float macc[MACC][4];
#pragma unroll
  for (int j = 0; j < MACC; ++j) macc[j][0] = macc[j][1] = macc[j][2] = macc[j][3] = 0.f;

  // Gram tasks of this thread (see GramLay)
  using G = GramLay<KP, EVAL>;
  constexpr int BS = G::BS;
  const int ggrp = (G::TASKS <= L::NT) ? tid / G::TASKS : 0;
  const bool gact = ggrp < G::GROUPS;
  int gI[G::TPT], gJ[G::TPT], gM[G::TPT], gT[G::TPT];
  bool gOn[G::TPT];
#pragma unroll
  for (int j = 0; j < G::TPT; ++j) {
    const int t = (G::TASKS <= L::NT) ? tid % G::TASKS : tid + j * L::NT;
    gT[j] = t;
    gOn[j] = gact && t < G::TASKS;
    gram_task(gOn[j] ? t : 0, G::NBLK, G::NB1, gM[j], gI[j], gJ[j]);
  }
  float gacc[G::TPT][BS * BS];
#pragma unroll
  for (int j = 0; j < G::TPT; ++j)
#pragma unroll
    for (int q = 0; q < BS * BS; ++q) gacc[j][q] = 0.f;

  // running sums of the trace and PG terms over this range's rows as unevaluated
  // float pairs (hi + lo, TwoSum), folded into float64 once at the end: the
  // float64 pipe of this part is narrow
  float tr_hi = 0.f, tr_lo = 0.f, pg_hi = 0.f, pg_lo = 0.f;
  int bad = 0;

  const int32_t* order = SPLIT ? nullptr : a.order;
  int64_t next_row = (p0 + team < p1) ? (order ? (int64_t)order[p0 + team] : p0 + team) : 0;
  // split update: this lane's 16 bytes of the four input rows of the next tile
  constexpr bool PF = SPLIT && update_prefetch<KP>();
  float* stg = smem + update_stage_offset<KP>() / sizeof(float) + team * KP + f0;
  constexpr int SSTR = L::R * KP;  // floats between the four staged arrays
  auto stage = [&](int64_t r) {
    cp_async16(stg, Zcur + r * KP + f0);
    cp_async16(stg + SSTR, P + r * KP + f0);
    cp_async16(stg + 2 * SSTR, Q + r * KP + f0);
    cp_async16(stg + 3 * SSTR, Zprv + r * KP + f0);
    cp_async_commit();
  };
  if constexpr (PF) {
    if (p0 < p1) stage(next_row);
  }
  for (int64_t base = p0; base < p1; base += L::R) {
    const int64_t pos = base + team;
    const bool active = pos < p1;
    const int64_t row = active ? next_row : 0;
    {  // row id of the next tile, fetched one tile ahead
      const int64_t np = pos + L::R;
      next_row = (np < p1) ? (order ? (int64_t)order[np] : np) : 0;
    }
    float acc[L::VEC];
#pragma unroll
    for (int q = 0; q < L::VEC; ++q) acc[q] = 0.f;

    int64_t lo = 0, hi = 0;
    // own-row loads are independent of the gather: issue them first
    float pv[L::VEC];
    float qv[L::VEC], zp[L::VEC];
    if constexpr (PF) {
      // this tile's rows, staged during the previous tile (each lane reads back
      // only the bytes its own copies wrote); then the next tile's copies
      cp_async_wait_all();
      load_row<L::VEC>(stg, acc);
      load_row<L::VEC>(stg + SSTR, pv);
      load_row<L::VEC>(stg + 2 * SSTR, qv);
      load_row<L::VEC>(stg + 3 * SSTR, zp);
      if (base + L::R < p1) stage(next_row);
    } else if constexpr (SPLIT) {
      load_row<L::VEC>(Zcur + row * KP + f0, acc);
    } else if (active && pos < a.n_heavy) {
      // chunked row: sum the partial products in chunk order
      const int64_t c0 = a.chunk_ptr[pos], c1 = a.chunk_ptr[pos + 1];
      for (int64_t c = c0; c < c1; ++c) {
        float pv[L::VEC];
        load_row<L::VEC>(a.hv_part + c * KP + f0, pv);
#pragma unroll
        for (int q = 0; q < L::VEC; ++q) acc[q] += pv[q];
      }
    } else if (active) {
      lo = a.row_ptr[row];
      hi = a.row_ptr[row + 1];
    }
    if constexpr (!PF) {
      load_row<L::VEC>(P + row * KP + f0, pv);
      if constexpr (!EVAL) {
        load_row<L::VEC>(Q + row * KP + f0, qv);
        load_row<L::VEC>((SPLIT ? Zprv : a.Zp) + row * KP + f0, zp);
      }
    }
    if constexpr (!SPLIT) {
      const int nb = (int)((hi - lo + L::NB - 1) / L::NB);
      const int batches = __reduce_max_sync(kFull, nb);
      gather<KP, MIXED>(a.col, a.val, Xg, lo, hi, batches, lt, f0, acc);
    }

    float d = 0.f;
#pragma unroll
    for (int q = 0; q < L::VEC; ++q) d = fmaf(pv[q], acc[q], d);
    d = team_sum<L::T>(d);
    if (active && lt == 0) two_sum_acc(tr_hi, tr_lo, d);

    if constexpr (!EVAL) {
      float y[L::VEC], sy[L::VEC];
#pragma unroll
      for (int q = 0; q < L::VEC; ++q) {
        y[q] = fmaf(beta, pv[q] - qv[q], pv[q]);
        sy[q] = fmaf(beta, acc[q] - zp[q], acc[q]);
      }
      // q_b = sum_a y_a G[a][b] for this lane's b in [f0, f0 + VEC)
      float qq[L::VEC];
      if constexpr (M::ON) {
        // tile product Y G on tensor cores (3xTF32)
        split_store4(ys + team * M::TSA + f0, ysl + team * M::TSA + f0, y);
        __syncthreads();
        float dq[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t* yh = reinterpret_cast<const uint32_t*>(ys) + (16 * ym + mg) * M::TSA + mt;
        const uint32_t* yl = reinterpret_cast<const uint32_t*>(ysl) + (16 * ym + mg) * M::TSA + mt;
        // KP = 128: the K steps alternate between two accumulators (two
        // dependency chains of 24 MMAs instead of one of 48), added at the end
        float dq2[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < M::KS; ++ks) {
          const uint32_t ah[4] = {yh[8 * ks], yh[8 * M::TSA + 8 * ks], yh[8 * ks + 4], yh[8 * M::TSA + 8 * ks + 4]};
          const uint32_t al[4] = {yl[8 * ks], yl[8 * M::TSA + 8 * ks], yl[8 * ks + 4], yl[8 * M::TSA + 8 * ks + 4]};
          const uint4 g = Gf[(yn * M::KS + ks) * 32 + lane];
          const uint32_t bh[2] = {g.x, g.y}, bl[2] = {g.z, g.w};
          mma3_tf32((M::YG2 && (ks & 1)) ? dq2 : dq, ah, al, bh, bl);
        }
        if constexpr (M::YG2) {
#pragma unroll
          for (int q = 0; q < 4; ++q) dq[q] += dq2[q];
        }
        float* qo = qs + (16 * ym + mg) * TS + 8 * yn + 2 * mt;
        *reinterpret_cast<float2*>(qo) = make_float2(dq[0], dq[1]);
        *reinterpret_cast<float2*>(qo + 8 * TS) = make_float2(dq[2], dq[3]);
        __syncthreads();
        load_row<L::VEC>(qs + team * TS + f0, qq);
      } else {
        float* yrow = ys + team * KP;
#pragma unroll
        for (int q = 0; q < L::VEC; ++q) yrow[f0 + q] = y[q];
        __syncwarp();
#pragma unroll
        for (int q = 0; q < L::VEC; ++q) qq[q] = 0.f;
#pragma unroll 4
        for (int a4 = 0; a4 < KP; a4 += L::VEC) {
          float ya[L::VEC];
          load_row<L::VEC>(yrow + a4, ya);
#pragma unroll
          for (int aa = 0; aa < L::VEC; ++aa) {
            float g[L::VEC];
            load_row<L::VEC>(Gs + (a4 + aa) * KP + f0, g);
#pragma unroll
            for (int q = 0; q < L::VEC; ++q) qq[q] = fmaf(ya[aa], g[q], qq[q]);
          }
        }
      }
      float v[L::VEC], x[L::VEC];
#pragma unroll
      for (int q = 0; q < L::VEC; ++q) v[q] = fmaf(tau4, sy[q] - qq[q], y[q]);
      project_simplex<KP>(v, x, f0, k);
      float pg = 0.f;
#pragma unroll
      for (int q = 0; q < L::VEC; ++q) {
        const float dd = y[q] - x[q];
        pg = fmaf(dd, dd, pg);
        if (!isfinite(x[q]) || !isfinite(acc[q])) bad = 1;
      }
      pg = team_sum<L::T>(pg);
      if (active && lt == 0) two_sum_acc(pg_hi, pg_lo, pg);
      if (active) {
        store_row<L::VEC>(Q + row * KP + f0, x);
        if constexpr (!SPLIT) store_row<L::VEC>(a.Zp + row * KP + f0, acc);
        if constexpr (MIXED) store_row_bf16<L::VEC>(XSo + row * KP + f0, x);
      }
      // next pass's extrapolated row y^{n+1} = xbar^n + beta_{n+1} (xbar^n - xbar^{n-1}),
      // formed exactly as the next pass will form it, feeds G(Y^{n+1})
      float xv[L::VEC], yv[L::VEC];
#pragma unroll
      for (int q = 0; q < L::VEC; ++q) {
        xv[q] = active ? x[q] : 0.f;
        yv[q] = active ? fmaf(beta_next, x[q] - pv[q], x[q]) : 0.f;
      }
      if constexpr (M::ON) {
        split_store4(xn_t + team * TS + f0, xn_l + team * TS + f0, xv);
        split_store4(yn_t + team * TS + f0, yn_l + team * TS + f0, yv);
      } else {
        store_row<L::VEC>(xn_t + team * TS + f0, xv);
        store_row<L::VEC>(yn_t + team * TS + f0, yv);
      }
    } else {
      float xv[L::VEC];
#pragma unroll
      for (int q = 0; q < L::VEC; ++q) {
        xv[q] = active ? pv[q] : 0.f;
        if (active && !isfinite(acc[q])) bad = 1;
      }
      if constexpr (M::ON) split_store4(xn_t + team * TS + f0, xn_l + team * TS + f0, xv);
      else store_row<L::VEC>(xn_t + team * TS + f0, xv);
    }
    __syncthreads();
    if constexpr (M::ON) {
      // Gram blocks on tensor cores: D[m][n] += sum_r T[r][m] T[r][n] over this
      // warp's share of the tile rows (A = T^T rows 16 mmi.., B = T columns 8 nj..)
      // The tensor core's accumulator addition does not round to nearest, so a
      // long running sum in it drifts; each tile's blocks start from zero and
      // are added to the running sums with ordinary float adds.
      if constexpr (M::TRI) {
        // this warp's TPW_B blocks of the upper triangles, the A fragment
        // reloaded only when the block row changes
        float dt[M::TPW_B][4];
#pragma unroll
        for (int j = 0; j < M::TPW_B; ++j) dt[j][0] = dt[j][1] = dt[j][2] = dt[j][3] = 0.f;
        uint32_t ah[M::RS][4], al[M::RS][4];
        int cur = -1;
#pragma unroll
        for (int j = 0; j < M::TPW_B; ++j) {
          const int info = tri_tab[warp * M::TPW_B + j];
          const int mat = info >> 16, mi = (info >> 8) & 0xff, nj = info & 0xff;
          const uint32_t* th = reinterpret_cast<const uint32_t*>(mat ? yn_t : xn_t);
          const uint32_t* tl = reinterpret_cast<const uint32_t*>(mat ? yn_l : xn_l);
          if ((info >> 8) != cur) {  // warp-uniform: (mat, mi) changed
            cur = info >> 8;
#pragma unroll
            for (int rs = 0; rs < M::RS; ++rs) {
              const int o0 = (8 * rs + mt) * TS, o4 = o0 + 4 * TS, ca = 16 * mi + mg;
              ah[rs][0] = th[o0 + ca];
              ah[rs][1] = th[o0 + ca + 8];
              ah[rs][2] = th[o4 + ca];
              ah[rs][3] = th[o4 + ca + 8];
              al[rs][0] = tl[o0 + ca];
              al[rs][1] = tl[o0 + ca + 8];
              al[rs][2] = tl[o4 + ca];
              al[rs][3] = tl[o4 + ca + 8];
            }
          }
#pragma unroll
          for (int rs = 0; rs < M::RS; ++rs) {
            const int o0 = (8 * rs + mt) * TS, o4 = o0 + 4 * TS, cb = 8 * nj + mg;
            const uint32_t bh[2] = {th[o0 + cb], th[o4 + cb]}, bl[2] = {tl[o0 + cb], tl[o4 + cb]};
            mma3_tf32(dt[j], ah[rs], al[rs], bh, bl);
          }
        }
#pragma unroll
        for (int j = 0; j < M::TPW_B; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q) macc[j][q] += dt[j][q];
      } else if (mon) {
        const uint32_t* th = reinterpret_cast<const uint32_t*>(mmat ? yn_t : xn_t);
        const uint32_t* tl = reinterpret_cast<const uint32_t*>(mmat ? yn_l : xn_l);
        float dt[M::BPW][4];
#pragma unroll
        for (int j = 0; j < M::BPW; ++j) dt[j][0] = dt[j][1] = dt[j][2] = dt[j][3] = 0.f;
#pragma unroll
        for (int rs = mks * (M::RS / M::KSPLIT); rs < (mks + 1) * (M::RS / M::KSPLIT); ++rs) {
          const int o0 = (8 * rs + mt) * TS, o4 = o0 + 4 * TS;
          const int ca = 16 * mmi + mg;
          const uint32_t ah[4] = {th[o0 + ca], th[o0 + ca + 8], th[o4 + ca], th[o4 + ca + 8]};
          const uint32_t al[4] = {tl[o0 + ca], tl[o0 + ca + 8], tl[o4 + ca], tl[o4 + ca + 8]};
#pragma unroll
          for (int j = 0; j < M::BPW; ++j) {
            const int cb = 8 * (mnj0 + j) + mg;
            const uint32_t bh[2] = {th[o0 + cb], th[o4 + cb]}, bl[2] = {tl[o0 + cb], tl[o4 + cb]};
            mma3_tf32(dt[j], ah, al, bh, bl);
          }
        }
#pragma unroll
        for (int j = 0; j < M::BPW; ++j)
#pragma unroll
          for (int q = 0; q < 4; ++q) macc[j][q] += dt[j][q];
      }
    } else if (gact) {
      // symmetric Gram blocks: M[I-block][J-block] += m_r[I-block] (x) m_r[J-block]
      for (int r = ggrp; r < L::R; r += G::GROUPS) {
#pragma unroll
        for (int j = 0; j < G::TPT; ++j) {
          if (!gOn[j]) continue;
          const float* src = (gM[j] ? yn_t : xn_t) + r * TS;
          float xa[BS], xb[BS];
          load_row<BS>(src + gI[j] * BS, xa);
          load_row<BS>(src + gJ[j] * BS, xb);
#pragma unroll
          for (int p = 0; p < BS; ++p)
#pragma unroll
            for (int q = 0; q < BS; ++q) gacc[j][p * BS + q] = fmaf(xa[p], xb[q], gacc[j][p * BS + q]);
        }
      }
    }
    // MMA update path: the next tile's first two barriers already order its
    // tile writes after these Gram reads
    if constexpr (!M::ON || EVAL) __syncthreads();
  }
  if constexpr (M::ON && !EVAL) __syncthreads();

  // ---- block reductions (fixed order => bit-reproducible) ----
  double* dred = reinterpret_cast<double*>(xn_t);  // reuse tile memory
  double tr_acc = (double)tr_hi + (double)tr_lo, pg_acc = (double)pg_hi + (double)pg_lo;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    tr_acc += __shfl_down_sync(kFull, tr_acc, o);
    pg_acc += __shfl_down_sync(kFull, pg_acc, o);
  }
  bad = __reduce_or_sync(kFull, bad);
  if (lane == 0) {
    dred[warp * 3 + 0] = tr_acc;
    dred[warp * 3 + 1] = pg_acc;
    dred[warp * 3 + 2] = (double)bad;
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0, p = 0, b = 0;
    for (int w = 0; w < L::WARPS; ++w) {
      t += dred[w * 3 + 0];
      p += dred[w * 3 + 1];
      b += dred[w * 3 + 2];
    }
    a.sc_part[slot * 4 + 0] = t;
    a.sc_part[slot * 4 + 1] = p;
    a.sc_part[slot * 4 + 2] = b;
    a.sc_part[slot * 4 + 3] = 0.0;
  }
  __syncthreads();
  float* gout = a.gram_part + (size_t)slot * 2 * L::E2;
  if constexpr (M::ON) {
    // block (mat, 16 mi.., 8 nj..) of fragment lane (mg, mt): rows mg, mg + 8, columns 2 mt, 2 mt + 1
    if constexpr (M::TRI) {
#pragma unroll
      for (int j = 0; j < M::TPW_B; ++j) {
        const int bb = warp * M::TPW_B + j;
        const int mat = bb / M::TRIB;
        int mi, nj;
        tri_block(bb % M::TRIB, KP / 8, mi, nj);
        float* o = gout + mat * L::E2 + (16 * mi + mg) * KP + 8 * nj + 2 * mt;
        *reinterpret_cast<float2*>(o) = make_float2(macc[j][0], macc[j][1]);
        *reinterpret_cast<float2*>(o + 8 * KP) = make_float2(macc[j][2], macc[j][3]);
      }
    } else if constexpr (M::KSPLIT == 1) {
#pragma unroll
      for (int j = 0; j < M::BPW; ++j) {
        float* o = gout + mmat * L::E2 + (16 * mmi + mg) * KP + 8 * (mnj0 + j) + 2 * mt;
        *reinterpret_cast<float2*>(o) = make_float2(macc[j][0], macc[j][1]);
        *reinterpret_cast<float2*>(o + 8 * KP) = make_float2(macc[j][2], macc[j][3]);
      }
    } else {
      // row-split partials: stage [part][block][lane][4], then sum parts in order
      float* red = tiles;
      if (mon) *reinterpret_cast<float4*>(red + ((mks * M::TB + mb0) * 32 + lane) * 4) =
          make_float4(macc[0][0], macc[0][1], macc[0][2], macc[0][3]);
      __syncthreads();
      for (int e = tid; e < M::TB * 32; e += L::NT) {
        float4 sum = *reinterpret_cast<const float4*>(red + e * 4);
#pragma unroll
        for (int pp = 1; pp < M::KSPLIT; ++pp) {
          const float4 v = *reinterpret_cast<const float4*>(red + ((pp * M::TB) * 32 + e) * 4);
          sum.x += v.x; sum.y += v.y; sum.z += v.z; sum.w += v.w;
        }
        const int blk = e >> 5, ln = e & 31;
        const int mat = blk / M::GBLK, rem = blk % M::GBLK;
        float* o = gout + mat * L::E2 + (16 * (rem / (KP / 8)) + (ln >> 2)) * KP + 8 * (rem % (KP / 8)) + 2 * (ln & 3);
        *reinterpret_cast<float2*>(o) = make_float2(sum.x, sum.y);
        *reinterpret_cast<float2*>(o + 8 * KP) = make_float2(sum.z, sum.w);
      }
    }
  } else if constexpr (G::GROUPS == 1) {
#pragma unroll
    for (int j = 0; j < G::TPT; ++j) {
      if (!gOn[j]) continue;
#pragma unroll
      for (int p = 0; p < BS; ++p)
#pragma unroll
        for (int q = 0; q < BS; ++q)
          gout[gM[j] * L::E2 + (gI[j] * BS + p) * KP + gJ[j] * BS + q] = gacc[j][p * BS + q];
    }
  } else {
    // groups -> one sum per entry, group order fixed
    float* gred = xn_t;  // ACTIVE * BS^2 floats
    if (gact) {
#pragma unroll
      for (int q = 0; q < BS * BS; ++q) gred[(ggrp * G::TASKS + gT[0]) * BS * BS + q] = gacc[0][q];
    }
    __syncthreads();
    for (int e = tid; e < G::TASKS * BS * BS; e += L::NT) {
      float sum = 0.f;
#pragma unroll 1
      for (int g = 0; g < G::GROUPS; ++g) sum += gred[g * G::TASKS * BS * BS + e];
      int m, I, J;
      gram_task(e / (BS * BS), G::NBLK, G::NB1, m, I, J);
      const int p = (e % (BS * BS)) / BS, q = e % BS;
      gout[m * L::E2 + (I * BS + p) * KP + J * BS + q] = sum;
    }
  }
}

// One pass of one instance: block b takes positions [cta_pos[b], cta_pos[b+1])
// (an even split when cta_pos is null) and partial slot b.
template <int KP, bool MIXED, bool EVAL>
__global__ void __launch_bounds__(Lay<KP>::NT, Lay<KP>::MINB) fista_pass_kernel(PassArgs a) {
  int64_t pass;
  if constexpr (!EVAL) {
    pass = pass_to_run(a.st);
    if (pass < 0) return;
  } else {
    pass = a.eval_sel;
  }
  int64_t p0, p1;
  if (a.cta_pos) {
    p0 = a.cta_pos[blockIdx.x];
    p1 = a.cta_pos[blockIdx.x + 1];
  } else {
    p0 = a.n * (int64_t)blockIdx.x / gridDim.x;
    p1 = a.n * (int64_t)(blockIdx.x + 1) / gridDim.x;
  }
  extern __shared__ __align__(16) float smem[];
  pass_range<KP, MIXED, EVAL>(a, pass, p0, p1, blockIdx.x, smem);
}

// Split iteration, step 3: the row-local update (extrapolation, y G, step,
// projection, writes, Gram and scalar partials) over rows in index order,
// block b taking rows [b n / parts, (b+1) n / parts) and partial slot b
// (b = upd_block0 + blockIdx.x; parts = upd_parts, or the grid).
template <int KP, bool MIXED>
__global__ void __launch_bounds__(Lay<KP>::NT, Lay<KP>::MINB) update_kernel(PassArgs a) {
  const int64_t pass = pass_to_run(a.st);
  if (pass < 0) return;
  const int parts = a.upd_parts > 0 ? a.upd_parts : (int)gridDim.x;
  const int b = a.upd_block0 + (int)blockIdx.x;
  const int64_t p0 = a.n * (int64_t)b / parts;
  const int64_t p1 = a.n * (int64_t)(b + 1) / parts;
  extern __shared__ __align__(16) float smem[];
  pass_range<KP, MIXED, false, true>(a, pass, p0, p1, b, smem);
}

// Partial products of chunked (very high degree) rows: hv_part[c] = sum over
// chunk c's nonzeros of s_ij * xbar_j.  Teams stride over chunks in rounds so
// that the gather stays warp-uniform.  EVAL: for an objective-only pass over
// buffer eval_sel (float32 iterate and values).
template <int KP, bool MIXED, bool EVAL>
__global__ void __launch_bounds__(Lay<KP>::NT) heavy_kernel(PassArgs a) {
  using L = Lay<KP>;
  int64_t pass;
  if constexpr (!EVAL) {
    pass = pass_to_run(a.st);
    if (pass < 0) return;
  } else {
    pass = a.eval_sel;
  }
  const float* P = (pass & 1) ? a.X1 : a.X0;
  const void* Xg = MIXED ? (const void*)((pass & 1) ? a.XS1 : a.XS0) : (const void*)P;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tiw = lane / L::T, lt = lane % L::T, f0 = lt * L::VEC;
  const int64_t teams = (int64_t)gridDim.x * L::R;
  const int64_t gteam = (int64_t)blockIdx.x * L::R + warp * L::TPW + tiw;
  const int64_t rounds = (a.n_chunks + teams - 1) / teams;
  for (int64_t r = 0; r < rounds; ++r) {
    const int64_t c = gteam + r * teams;
    const bool active = c < a.n_chunks;
    const int64_t lo = active ? a.chunk_e0[c] : 0, hi = active ? a.chunk_e1[c] : 0;
    float acc[L::VEC];
#pragma unroll
    for (int q = 0; q < L::VEC; ++q) acc[q] = 0.f;
    const int nb = (int)((hi - lo + L::NB - 1) / L::NB);
    const int batches = __reduce_max_sync(kFull, nb);
    gather<KP, MIXED>(a.col, a.val, Xg, lo, hi, batches, lt, f0, acc);
    if (active) store_row<L::VEC>(a.hv_part + c * KP + f0, acc);
  }
}

struct FoldArgs {
  FistaState* st;
  const float* gram_part;   // [parts][2][KP][KP], upper BS x BS blocks written
  const double* sc_part;    // [parts][4]
  int32_t parts;
  int32_t eval;             // 1: objective-only pass (Gram of the evaluated iterate only)
  int32_t eval_init;        // 1: also seed the solver (G(Y^1) = Gram of Xbar^0, gram2_cur)
  int32_t pad_;
  unsigned long long* work; // spmm work counters, reset for the next pass (may be null)
  int32_t n_work;           // how many (one per gather launch of a pass)
  int32_t pad2_;
  double* A;                // KP x KP float64: Gram of the newest iterate (scratch)
  double* G;                // KP x KP float64: Gram of the next extrapolated point (scratch)
  float* Gy;                // KP x KP float32 for the next pass
  double* bpart;            // [fold blocks][2] block partials of an iteration's fold (||A||^2, sum of G(Y))
};

// Sums the per-block partials in block order (float64), evaluates the loss of
// Xbar^{n-1}, applies the stop rule, advances t and the momentum factors, and
// stores G(Y^{n+1}) minus its mean entry in float32 (the mean shift leaves the
// projection unchanged because rows of Y sum to one: P(v + c 1) = P(v)).
// First stage: each block sums the partials of FOLD_EPB entries, its 256
// threads split into 256 / FOLD_EPB groups that take every group-th partial
// (in four interleaved float-pair chains); the group sums are then added in
// float64 in group order (a fixed tree: deterministic).
template <int KP>
__host__ __device__ constexpr int fold_epb() {
  return KP <= 32 ? 32 : (KP == 64 ? 64 : 128);
}
template <int KP>
__host__ __device__ constexpr int fold_blocks(bool eval) {
  return ((eval ? 1 : 2) * KP * KP + fold_epb<KP>() - 1) / fold_epb<KP>();
}

// Block `blk` of the `nblocks` blocks folding one instance (256 threads).
template <int KP>
__device__ __forceinline__ void fold_body(const FoldArgs& f, int blk, int nblocks) {
  constexpr int E2 = KP * KP;
  FistaState* st = f.st;
  volatile FistaState* vs = st;
  const int64_t pass = f.eval ? (int64_t)vs->pass : pass_to_run(st);
  if (pass < 0) return;
  const int64_t nnew = pass + 1;
  const int tid = threadIdx.x;
  const int nent = f.eval ? E2 : 2 * E2;
  // issued with the partials' loads rather than after them (only the last
  // block writes shift, after every block has passed this point)
  const int k = st->k;
  const double shift = f.eval ? 0.0 : st->shift;
  {
    constexpr int EPB = fold_epb<KP>(), GR = 256 / EPB;
    __shared__ double gsum[256];
    const int el = tid % EPB, g = tid / EPB;
    const int e = blk * EPB + el;
    double s = 0.0;
    int src = 0;
    if (e < nent) {
      const int m = e / E2, r = (e % E2) / KP, c = e % KP;
      src = m * E2 + ((r <= c) ? r * KP + c : c * KP + r);
      // four chains over this group's partials (p, p + GR, p + 2 GR, p + 3 GR),
      // each a float pair (TwoSum: the rounding error of every add kept,
      // about 48 significant bits), converted to float64 once: float64 adds
      // and conversions per partial saturated B300's narrow float64 pipe
      const float* gp = f.gram_part + src;
      const size_t pstr = (size_t)2 * E2 * GR;
      float h[4] = {0.f, 0.f, 0.f, 0.f}, l[4] = {0.f, 0.f, 0.f, 0.f};
      int p = g;
      for (; p + 3 * GR < f.parts; p += 4 * GR) {
        const float* q = gp + (size_t)p * 2 * E2;
        two_sum_acc(h[0], l[0], q[0]);
        two_sum_acc(h[1], l[1], q[pstr]);
        two_sum_acc(h[2], l[2], q[2 * pstr]);
        two_sum_acc(h[3], l[3], q[3 * pstr]);
      }
      for (; p < f.parts; p += GR) two_sum_acc(h[0], l[0], gp[(size_t)p * 2 * E2]);
      s = (((double)h[0] + (double)l[0]) + ((double)h[1] + (double)l[1])) +
          (((double)h[2] + (double)l[2]) + ((double)h[3] + (double)l[3]));
    }
    gsum[tid] = s;
    __syncthreads();
    // an iteration's fold (not an objective-only one) also writes its entries
    // of the float32 G(Y) for the next pass here, shifted by the previous
    // pass's mean entry (any constant shift leaves the projection unchanged;
    // the mean keeps the float32 values small), and block partials of
    // ||A||_F^2 and of the sum of G(Y)'s entries, from which the last block
    // forms the loss and the next shift without a pass over the entries
    double a2 = 0.0, gs = 0.0;
    if (g == 0 && e < nent) {
      double t = gsum[el];
      for (int q = 1; q < GR; ++q) t += gsum[q * EPB + el];
      const int m = e / E2, r = (e % E2) / KP, c = e % KP;
      (m == 0 ? f.A : f.G)[r * KP + c] = t;
      if (!f.eval) {
        if (m == 0) {
          a2 = t * t;
        } else {
          const bool in = r < k && c < k;
          gs = in ? t : 0.0;
          f.Gy[r * KP + c] = in ? (float)(t - shift) : 0.0f;
        }
      }
    }
    if (!f.eval) {
      // only the group-0 threads (the first EPB / 32 warps) hold entries
      constexpr int W0 = (EPB + 31) / 32;
      __shared__ double bred[2][W0];
      const int warp = tid >> 5, lane = tid & 31;
      if (warp < W0) {
        a2 = warp_sum_f64(a2);
        gs = warp_sum_f64(gs);
        if (lane == 0) {
          bred[0][warp] = a2;
          bred[1][warp] = gs;
        }
      }
      __syncthreads();
      if (tid == 0) {
        double x = 0.0, y = 0.0;
#pragma unroll
        for (int w = 0; w < W0; ++w) x += bred[0][w], y += bred[1][w];
        f.bpart[2 * blk] = x;
        f.bpart[2 * blk + 1] = y;
      }
    }
  }
  __threadfence();
  __syncthreads();
  __shared__ int is_last;
  if (tid == 0) is_last = (atomicAdd(&st->ticket, 1u) == (unsigned)nblocks - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();

  const int warp = tid >> 5, lane = tid & 31;
  // Six sums, each thread's share in index order (t, t + 256, ...), then a
  // fixed butterfly across the lanes and the warps in warp order
  // (deterministic): [0..3] the scalar partials (trace, squared PG norm,
  // non-finite count, waits given up), [4] ||A||_F^2 (an iteration's fold
  // takes it from the block partials, an objective-only one from the entries,
  // in four chains), [5] the sum of G(Y)'s k x k entries (iteration only).
  double v[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  if (!f.eval) {
    for (int b = tid; b < nblocks; b += 256) {
      v[4] += __ldcg(f.bpart + 2 * b);
      v[5] += __ldcg(f.bpart + 2 * b + 1);
    }
  } else {
    constexpr int PT = (E2 + 255) / 256;
    double p4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int j = 0; j < PT; ++j) {
      const int i = tid + j * 256;
      const double x = i < E2 ? __ldcg(f.A + i) : 0.0;
      p4[j & 3] = fma(x, x, p4[j & 3]);
    }
    v[4] = (p4[0] + p4[1]) + (p4[2] + p4[3]);
  }
  {
    const double2* sp = reinterpret_cast<const double2*>(f.sc_part);  // [parts][2] pairs
    int c = tid;
    for (; c + 256 < f.parts; c += 512) {  // two partials' loads in flight
      const double2 x0 = __ldcg(sp + 2 * c), x1 = __ldcg(sp + 2 * c + 1);
      const double2 y0 = __ldcg(sp + 2 * (c + 256)), y1 = __ldcg(sp + 2 * (c + 256) + 1);
      v[0] += x0.x, v[1] += x0.y, v[2] += x1.x, v[3] += x1.y;
      v[0] += y0.x, v[1] += y0.y, v[2] += y1.x, v[3] += y1.y;
    }
    if (c < f.parts) {
      const double2 x0 = __ldcg(sp + 2 * c), x1 = __ldcg(sp + 2 * c + 1);
      v[0] += x0.x, v[1] += x0.y, v[2] += x1.x, v[3] += x1.y;
    }
  }
  __shared__ double wred[6][8];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    v[q] = warp_sum_f64(v[q]);
    if (lane == 0) wred[q][warp] = v[q];
  }
  __syncthreads();
  if (tid == 0) {
    double tot[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      double x = 0.0;
#pragma unroll
      for (int w = 0; w < 8; ++w) x += wred[q][w];
      tot[q] = x;
    }
    const double tr = tot[0], pg = tot[1], bad = tot[2], tmo = tot[3], gram2_new = tot[4];
    if (f.eval) {
      st->eval_trace = tr;
      st->eval_gram2 = gram2_new;
      st->eval_f = st->S2 - 2.0 * tr + gram2_new;
      if (f.eval_init) st->gram2_cur = gram2_new;
    } else {
      // every field this update reads, loaded before any store (one round
      // trip instead of one per read: a store may alias a later load)
      const double S2 = st->S2, gram2_cur = st->gram2_cur, tau = st->tau, tol = st->tol;
      const double loss_prev = st->loss_prev, pg_first_old = st->pg_first, t0 = st->t;
      const int64_t max_iter = st->max_iter;
      const int stop_rule = st->stop_rule, accel = st->accel;
      // loss of Xbar^{pass} (= Xbar^{n-1} for this pass n = pass + 1)
      const double loss = S2 - 2.0 * tr + gram2_cur;
      const double r = sqrt(pg) / tau;
      const double pg_first = nnew == 1 ? r : pg_first_old;
      int done = 0, status = 0;
      int64_t out = nnew;
      if (tmo > 0.0) {
        // a bounded wait of the update gave up: Xbar^{pass} is the last
        // complete iterate
        done = 1;
        status = 6;
        out = pass;
      } else if (bad > 0.0 || !isfinite(loss)) {
        done = 1;
        status = 4;
        out = pass;
      } else if (stop_rule == 0) {
        if (pass >= 1 && loss_prev - loss <= tol) {
          done = 1;
          out = pass;
        }
      } else if (stop_rule == 1) {
        if (r <= tol * pg_first) done = 1;
      } else if (stop_rule == 2) {
        if (r <= tol) done = 1;
      }
      if (!done && nnew >= max_iter) {
        done = 1;
        status = 5;
      }
      // t_{n+1}, t_{n+2} and the momentum factors of the next two passes
      const double t1 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t0 * t0));
      const double t2 = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t1 * t1));
      st->trace_last = tr;
      st->gram2_last = gram2_cur;
      st->loss_last = loss;
      st->f_iter = pass;
      st->pg_last = r;
      st->pg_first = pg_first;
      st->loss_prev = loss;
      st->gram2_cur = gram2_new;
      st->t = t1;
      st->beta = accel ? (t0 - 1.0) / t1 : 0.0;
      st->beta_next = accel ? (t1 - 1.0) / t2 : 0.0;
      // the mean of G(Y)'s entries: the shift of the next pass's float32 G(Y)
      st->shift = tot[5] / ((double)k * (double)k);
      st->out_iter = out;
      st->status = status;
      st->done = done;
      st->pass = nnew;
    }
  }
  // float32 G(Y) for the next pass, minus its mean over the k x k block: an
  // iteration's fold wrote it above (with the previous pass's mean) and its
  // last block only keeps this pass's mean for the next one (above); the
  // start's objective-only fold writes it here
  if (f.eval && f.eval_init) {
    __shared__ double red[256];
    const double* Gsrc = f.A;
    double msum = 0.0;
    {
      constexpr int PT = (E2 + 255) / 256;
      double m4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int j = 0; j < PT; ++j) {
        const int i = tid + j * 256;
        const int r = i / KP, c = i % KP;
        if (i < E2 && r < k && c < k) m4[j & 3] += __ldcg(Gsrc + i);
      }
      msum = (m4[0] + m4[1]) + (m4[2] + m4[3]);
    }
    red[tid] = msum;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (tid < o) red[tid] += red[tid + o];
      __syncthreads();
    }
    const double mean = red[0] / ((double)k * (double)k);
#pragma unroll 8
    for (int i = tid; i < E2; i += 256) {
      const int r = i / KP, c = i % KP;
      f.Gy[i] = (r < k && c < k) ? (float)(__ldcg(Gsrc + i) - mean) : 0.0f;
    }
    if (tid == 0) st->shift = mean;
  }
  if (tid == 0) {
    st->ticket = 0u;
    if (f.work)
      for (int w = 0; w < f.n_work; ++w) f.work[w] = 0ull;
  }
}

// Gram partials of one iterate buffer without any product with S (the solver's
// start: G(Y^1) = Xbar^0^T Xbar^0 and ||Xbar^0^T Xbar^0||^2; the loss of Xbar^0
// comes from the first pass, whose product with S forms its trace term).
// Block b takes rows [b n / grid, (b+1) n / grid) in tiles of TR rows, staged in
// shared memory by cp.async two tiles deep (16 KB per tile at k = 32, so that
// enough bytes are in flight), rows past the block's range read as zero.  The
// KP x KP matrix is cut into B x B register blocks (B = 4; KP = 2: one 2 x 2
// block); the 256 threads are NBLK blocks x GRP row groups, and thread (g, blk)
// sums rows g, g + GRP, ... of each tile for its block: per row two short
// shared-memory reads feed B^2 FMAs (one read per FMA was the shared-memory
// bandwidth bound: 17 ms at n = 70M, k = 32).  Float32 sums over 32 rows of a
// thread, added into float pairs by Fast2Sum (exact here: the entries are sums
// of products of non-negative values, so the running sums only grow; float64
// adds, on B300's narrow float64 pipe, were the next bound); the row groups
// are added in float64 in group order (fixed: deterministic); the block's
// partial goes to gram_part[b][0] (sc_part[b] = 0: no trace term).
template <int KP>
__host__ __device__ constexpr int gram0_rows_per_tile() {
  return (256 / ((KP / (KP >= 4 ? 4 : KP)) * (KP / (KP >= 4 ? 4 : KP)))) > 128
             ? 256 / ((KP / (KP >= 4 ? 4 : KP)) * (KP / (KP >= 4 ? 4 : KP)))
             : (KP == 64 ? 64 : 128);
}
template <int KP>
__global__ void __launch_bounds__(256) gram0_kernel(const float* __restrict__ X, int64_t n, float* gram_part,
                                                    double* sc_part) {
  static_assert(KP <= 64, "register blocks");
  constexpr int E2 = KP * KP;
  constexpr int B = KP >= 4 ? 4 : KP;
  constexpr int NBS = KP / B, NBLK = NBS * NBS, GRP = 256 / NBLK;
  static_assert(NBLK * GRP == 256, "blocks x row groups = threads");
  constexpr int TR = gram0_rows_per_tile<KP>();     // rows per tile
  static_assert(TR % GRP == 0, "row groups tile the rows");
  constexpr int RPT = TR / GRP;                     // rows of a tile per thread
  constexpr int TPF = 32 / RPT > 0 ? 32 / RPT : 1;  // tiles summed in float32 between float64 adds
  constexpr int CB = KP * 4 >= 16 ? 16 : KP * 4;    // bytes per cp.async (whole rows' pieces)
  constexpr int CF = CB / 4;                        // floats per cp.async
  constexpr int NCH = TR * KP / CF;                 // cp.async per tile
  constexpr int TILE_F = TR * KP;
  constexpr int BUF_B = 2 * TILE_F * 4 > 256 * B * B * 8 ? 2 * TILE_F * 4 : 256 * B * B * 8;
  __shared__ __align__(16) unsigned char smem_raw[BUF_B];
  float* tiles = reinterpret_cast<float*>(smem_raw);
  double* red = reinterpret_cast<double*>(smem_raw);   // after the last tile
  const int tid = threadIdx.x;
  const int g = tid / NBLK, blk = tid % NBLK, bi = blk / NBS, bj = blk % NBS;
  const int64_t p0 = n * (int64_t)blockIdx.x / gridDim.x, p1 = n * (int64_t)(blockIdx.x + 1) / gridDim.x;
  float ah[B * B], al[B * B], t[B * B];
#pragma unroll
  for (int q = 0; q < B * B; ++q) ah[q] = 0.0f, al[q] = 0.0f, t[q] = 0.0f;
  // tile at row base into buffer b: rows below p1 copied, the rest zero-filled
  auto stage = [&](int64_t base, int b) {
    float* dst = tiles + b * TILE_F;
    for (int c = tid; c < NCH; c += 256) {
      const int64_t row = base + (c * CF) / KP;
      const bool in = row < p1;
      const float* src = in ? X + base * KP + (int64_t)c * CF : X;
      const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst + c * CF);
      if constexpr (CB == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(in ? 16 : 0) : "memory");
      else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"(CB), "r"(in ? CB : 0)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  int since = 0, cur = 0;
  if (p0 < p1) stage(p0, 0);
  for (int64_t base = p0; base < p1; base += TR) {
    if (base + TR < p1) {
      stage(base + TR, cur ^ 1);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
    const float* tile = tiles + cur * TILE_F;
#pragma unroll 4
    for (int rr = 0; rr < RPT; ++rr) {
      const float* row = tile + (g + rr * GRP) * KP;
      float a[B], b[B];
      if constexpr (B == 4) {  // 16-byte reads (rows and blocks are 16-byte aligned)
        const float4 va = *reinterpret_cast<const float4*>(row + bi * B);
        const float4 vb = *reinterpret_cast<const float4*>(row + bj * B);
        a[0] = va.x, a[1] = va.y, a[2] = va.z, a[3] = va.w;
        b[0] = vb.x, b[1] = vb.y, b[2] = vb.z, b[3] = vb.w;
      } else {
#pragma unroll
        for (int p = 0; p < B; ++p) {
          a[p] = row[bi * B + p];
          b[p] = row[bj * B + p];
        }
      }
#pragma unroll
      for (int p = 0; p < B; ++p)
#pragma unroll
        for (int q = 0; q < B; ++q) t[p * B + q] = fmaf(a[p], b[q], t[p * B + q]);
    }
    if (++since == TPF) {
#pragma unroll
      for (int q = 0; q < B * B; ++q) {
        const float sum = ah[q] + t[q];
        al[q] += t[q] - (sum - ah[q]);
        ah[q] = sum;
        t[q] = 0.0f;
      }
      since = 0;
    }
    __syncthreads();   // the buffer just read is staged into two tiles from now
    cur ^= 1;
  }
#pragma unroll
  for (int q = 0; q < B * B; ++q) red[tid * B * B + q] = ((double)ah[q] + (double)al[q]) + (double)t[q];
  __syncthreads();
  float* go = gram_part + (size_t)blockIdx.x * 2 * E2;
  for (int e = tid; e < E2; e += 256) {
    const int i = e / KP, j = e % KP;
    const int eb = (i / B) * NBS + j / B, ep = (i % B) * B + j % B;
    double sum = 0.0;
    for (int gg = 0; gg < GRP; ++gg) sum += red[(gg * NBLK + eb) * B * B + ep];
    go[e] = (float)sum;
  }
  if (tid < 4) sc_part[blockIdx.x * 4 + tid] = 0.0;
}

template <int KP>
__global__ void __launch_bounds__(256) fold_kernel(FoldArgs f) {
  fold_body<KP>(f, blockIdx.x, gridDim.x);
}

}  // namespace fc
