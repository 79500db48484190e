// Shared pieces of the iteration kernels on sm_103a: the team layout, the
// per-pass argument block, row loads/stores, team reductions and the gather
// acc += sum_e s_ie x_{col(e)} that both the product with S and the fused pass
// use.
//
// Layout: a "team" of T lanes owns one row; lane t holds VEC consecutive
// features of the row (KP padded features, rows of KP floats in HBM).  Teams
// of one warp take rows of similar degree (neighbouring positions of the
// processing order have similar degrees), so the gather loop is warp-uniform.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "state.h"

namespace fc {

constexpr unsigned kFull = 0xffffffffu;

// Sum over the 32 lanes of a warp by a fixed xor butterfly (every lane gets
// the same, deterministic result).
__device__ __forceinline__ double warp_sum_f64(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

#ifndef FC_MINB32
#define FC_MINB32 4  // resident 256-thread blocks per SM the k <= 32 pass is sized for
#endif

template <int KP>
struct Lay {
  static constexpr int VEC = KP < 4 ? KP : 4;      // features per lane
  static constexpr int T = KP / VEC;                // lanes per team (row)
  static constexpr int TPW = 32 / T;                // teams per warp
  static constexpr int NT = KP >= 128 ? 512 : 256;  // threads per block
  static constexpr int WARPS = NT / 32;
  static constexpr int R = WARPS * TPW;             // rows per tile
  static constexpr int NB = T > 8 ? T : 8;          // nonzeros per gather batch per team
  static constexpr int PER = NB / T;                // (col, val) pairs each lane fetches per batch
  static constexpr int E2 = KP * KP;
  // resident blocks per SM the register budget is sized for
  static constexpr int MINB = KP <= 4 ? 2 : (KP == 8 ? 3 : (KP == 16 ? 4 : (KP == 32 ? FC_MINB32 : (KP == 64 ? 2 : 1))));
};

// The pass a kernel of the iteration runs, or -1 when the solve is done or
// past its step limit.  The three fields are read together (independent
// volatile loads: one round trip to L2 instead of one per field).
__device__ __forceinline__ int64_t pass_to_run(const FistaState* st) {
  const volatile FistaState* vs = st;
  const int32_t done = vs->done;
  const int64_t pass = vs->pass;
  const int64_t limit = vs->limit;
  return (done != 0 || pass >= limit) ? -1 : pass;
}

struct PassArgs {
  const int64_t* row_ptr;    // [n+1]
  const int32_t* col;        // [nnz]
  const void* val;           // [nnz] float32 (FP32) or bfloat16 (mixed)
  const int32_t* order;      // rows in processing order (nullptr: identity)
  const int64_t* cta_pos;    // [gridDim.x + 1] position ranges (nullptr: even split)
  int64_t n_heavy;           // positions [0, n_heavy) are chunked rows
  const int64_t* chunk_ptr;  // [n_heavy + 1]
  const int64_t* chunk_e0;   // [n_chunks]
  const int64_t* chunk_e1;   // [n_chunks]
  int64_t n_chunks;
  float* hv_part;            // [n_chunks][KP] partial products of chunked rows
  float* X0;                 // iterate buffers, n x KP float32 (Xbar^j in X_{j&1})
  float* X1;
  __nv_bfloat16* XS0;        // bfloat16 gather copies (mixed precision)
  __nv_bfloat16* XS1;
  float* Zp;                 // fused pass: n x KP S Xbar^{pass-1}, replaced by S Xbar^{pass}
  float* Z0;                 // split pass: S Xbar^j in Z_{(j+1)&1}, n x KP float32
  float* Z1;
  unsigned long long* work;  // split pass: work counter of spmm_kernel (reset by the fold)
  int64_t unit_lo;           // split pass: gather units [unit_lo, unit_hi) (unit_hi < 0: all)
  int64_t unit_hi;
  int32_t upd_block0;        // split pass: first block of this update launch among
  int32_t upd_parts;         //   upd_parts blocks (0: the launch is all of them)
  const float* Gy;           // KP x KP float32, G(Y) minus its mean entry
  float* gram_part;          // [gridDim.x][2][KP][KP]
  double* sc_part;           // [gridDim.x][4]: trace, pg, nonfinite, waits given up
  FistaState* st;
  int64_t n;
  int32_t k;
  int32_t eval_sel;          // objective-only pass: buffer index to evaluate
};

template <bool MIXED>
struct GatherT;
template <>
struct GatherT<false> {
  using V = float;
};
template <>
struct GatherT<true> {
  using V = __nv_bfloat16;
};

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

// Load VEC consecutive features of the gathered iterate at element offset off.
template <int VEC, bool MIXED>
__device__ __forceinline__ void load_feat(const void* Xg, int64_t off, float* out) {
  if constexpr (!MIXED) {
    const float* p = reinterpret_cast<const float*>(Xg) + off;
    if constexpr (VEC == 4) {
      float4 v = __ldg(reinterpret_cast<const float4*>(p));
      out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    } else if constexpr (VEC == 2) {
      float2 v = __ldg(reinterpret_cast<const float2*>(p));
      out[0] = v.x; out[1] = v.y;
    } else {
      out[0] = __ldg(p);
    }
  } else {
    const __nv_bfloat16* p = reinterpret_cast<const __nv_bfloat16*>(Xg) + off;
    if constexpr (VEC == 4) {
      uint2 raw = __ldg(reinterpret_cast<const uint2*>(p));
      __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&raw.x);
      __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&raw.y);
      float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
      out[0] = fa.x; out[1] = fa.y; out[2] = fb.x; out[3] = fb.y;
    } else if constexpr (VEC == 2) {
      unsigned raw = __ldg(reinterpret_cast<const unsigned*>(p));
      float2 f = __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&raw));
      out[0] = f.x; out[1] = f.y;
    } else {
      out[0] = __bfloat162float(p[0]);
    }
  }
}

template <int VEC>
__device__ __forceinline__ void load_row(const float* base, float* out) {
  if constexpr (VEC == 4) {
    float4 v = *reinterpret_cast<const float4*>(base);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  } else if constexpr (VEC == 2) {
    float2 v = *reinterpret_cast<const float2*>(base);
    out[0] = v.x; out[1] = v.y;
  } else {
    out[0] = base[0];
  }
}

template <int VEC>
__device__ __forceinline__ void store_row(float* base, const float* v) {
  if constexpr (VEC == 4) {
    *reinterpret_cast<float4*>(base) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (VEC == 2) {
    *reinterpret_cast<float2*>(base) = make_float2(v[0], v[1]);
  } else {
    base[0] = v[0];
  }
}

template <int VEC>
__device__ __forceinline__ void store_row_bf16(__nv_bfloat16* base, const float* v) {
  if constexpr (VEC == 4) {
    __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
    __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
    uint2 raw;
    raw.x = *reinterpret_cast<unsigned*>(&a);
    raw.y = *reinterpret_cast<unsigned*>(&b);
    *reinterpret_cast<uint2*>(base) = raw;
  } else if constexpr (VEC == 2) {
    *reinterpret_cast<__nv_bfloat162*>(base) = __floats2bfloat162_rn(v[0], v[1]);
  } else {
    base[0] = __float2bfloat16_rn(v[0]);
  }
}

// Sum over the T lanes of a team (teams are aligned groups of T lanes).
template <int T>
__device__ __forceinline__ float team_sum(float v) {
#pragma unroll
  for (int o = T / 2; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// acc += sum_{e in [lo, hi)} val[e] * Xg[col[e], f0 .. f0+VEC).  `batches` must
// be the same on every lane of the warp (the maximum over its teams).  The
// (col, val) pairs of batch j+1 are fetched while the gathers of batch j are in
// flight, so a batch costs one memory round trip.
template <int KP, bool MIXED>
__device__ __forceinline__ void gather(const int32_t* __restrict__ col, const void* __restrict__ valp,
                                       const void* __restrict__ Xg, int64_t lo, int64_t hi, int batches,
                                       int lt, int f0, float* acc) {
  using L = Lay<KP>;
  using VT = typename GatherT<MIXED>::V;
  const VT* val = reinterpret_cast<const VT*>(valp);
  int ci[L::PER];
  float cv[L::PER];
#pragma unroll
  for (int p = 0; p < L::PER; ++p) {
    const int64_t e = lo + lt + p * L::T;
    const bool ok = batches > 0 && e < hi;
    ci[p] = ok ? __ldg(col + e) : 0;
    cv[p] = ok ? to_f(__ldg(val + e)) : 0.0f;
  }
  for (int j = 0; j < batches; ++j) {
    float xv[L::NB][L::VEC];
#pragma unroll
    for (int u = 0; u < L::NB; ++u) {
      const int c = L::T > 1 ? __shfl_sync(kFull, ci[u / L::T], u % L::T, L::T) : ci[u];
      load_feat<L::VEC, MIXED>(Xg, (int64_t)c * KP + f0, xv[u]);
    }
    int ni[L::PER];
    float nv[L::PER];
    const int64_t e1 = lo + (int64_t)(j + 1) * L::NB;
#pragma unroll
    for (int p = 0; p < L::PER; ++p) {
      const int64_t e = e1 + lt + p * L::T;
      const bool ok = e < hi;
      ni[p] = ok ? __ldg(col + e) : 0;
      nv[p] = ok ? to_f(__ldg(val + e)) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < L::NB; ++u) {
      const float v = L::T > 1 ? __shfl_sync(kFull, cv[u / L::T], u % L::T, L::T) : cv[u];
#pragma unroll
      for (int q = 0; q < L::VEC; ++q) acc[q] = fmaf(v, xv[u][q], acc[q]);
    }
#pragma unroll
    for (int p = 0; p < L::PER; ++p) {
      ci[p] = ni[p];
      cv[p] = nv[p];
    }
  }
}

// ---- wide gather (the split iteration's product with S) ----
// Each lane loads LB = min(16, row bytes) bytes of a gathered row per nonzero,
// GT = row bytes / LB lanes share a row, and a warp keeps TPW * NB rows in
// flight (64 rows for the bf16 copy at k = 32, 32 rows of 128 bytes for the
// float32 iterate).  Rows of at most 64 bytes are loaded with the 64-byte L2
// fetch hint: a random 64-byte row otherwise costs a 128-byte DRAM read.
// (256-bit loads were slower here: twice the batches per row for the same
// bytes in flight.)
template <int KP, bool MIXED>
struct WLay {
  static constexpr int ES = MIXED ? 2 : 4;       // bytes per gathered element
  static constexpr int RB = KP * ES;             // bytes per gathered row
  static constexpr bool HINT64 = RB <= 64;
  static constexpr int LB = RB < 16 ? RB : 16;   // bytes per lane per nonzero
  static constexpr int GT = RB / LB;             // lanes per row
  static constexpr int FEAT = LB / ES;           // features per lane
  static constexpr int TPW = 32 / GT;            // rows per warp
  // nonzeros per batch per row: 8, except 6 for the float32 k <= 32 gather,
  // whose 5-blocks-per-SM register budget (48) spilled with 8 rows of 16 bytes
  // in flight per lane (gather 43.3 -> 42.1 ms at n = 70M; each row's sum runs
  // over its nonzeros in index order whatever the batch, so no value changes)
  static constexpr int NB = (KP == 32 && !MIXED) ? 6 : (GT > 8 ? GT : 8);
  static constexpr int PER = (NB + GT - 1) / GT; // (col, val) pairs each lane fetches per batch
};

// The layout with NBX nonzeros per batch per row (0 = WLay's NB).
template <int KP, bool MIXED, int NBX>
struct WShape : WLay<KP, MIXED> {
  static constexpr int NB = NBX > 0 ? NBX : WLay<KP, MIXED>::NB;
  static constexpr int PER = (NB + WLay<KP, MIXED>::GT - 1) / WLay<KP, MIXED>::GT;
};

// out[0 .. FEAT) = the LB bytes at p, widened to float
template <int KP, bool MIXED>
__device__ __forceinline__ void load_wide(const void* p, float* out) {
  using W = WLay<KP, MIXED>;
  uint32_t r[W::LB / 4 > 0 ? W::LB / 4 : 1];
  if constexpr (W::LB == 16 && !W::HINT64) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    r[0] = v.x;
    r[1] = v.y;
    r[2] = v.z;
    r[3] = v.w;
  } else if constexpr (W::LB == 16) {
    asm volatile("ld.global.nc.L2::64B.v4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "l"(p));
  } else if constexpr (W::LB == 8) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    r[0] = v.x;
    r[1] = v.y;
  } else {
    static_assert(W::LB == 4, "row of fewer than 4 bytes");
    r[0] = __ldg(reinterpret_cast<const unsigned*>(p));
  }
#pragma unroll
  for (int w = 0; w < (W::LB / 4 > 0 ? W::LB / 4 : 1); ++w) {
    if constexpr (MIXED) {
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&r[w]));
      out[2 * w] = f.x;
      out[2 * w + 1] = f.y;
    } else {
      out[w] = __uint_as_float(r[w]);
    }
  }
}

// acc[0 .. FEAT) += sum_{e in [lo, hi)} val[e] * Xg[col[e], lt FEAT .. (lt+1) FEAT),
// nonzeros in index order (the same order, and so the same sums, as gather).
// `batches` (batches of NBX nonzeros; 0 = the layout's NB) must be the same
// on every lane of the warp.  The batch size changes no value: each row's sum
// runs over its nonzeros in index order.
template <int KP, bool MIXED, int NBX = 0>
__device__ __forceinline__ void gather_wide(const int32_t* __restrict__ col, const void* __restrict__ valp,
                                            const void* __restrict__ Xg, int64_t lo, int64_t hi, int batches,
                                            int lt, float* acc) {
  using W = WShape<KP, MIXED, NBX>;
  using VT = typename GatherT<MIXED>::V;
  const VT* val = reinterpret_cast<const VT*>(valp);
  const char* xb = reinterpret_cast<const char*>(Xg) + lt * W::LB;
  int ci[W::PER];
  float cv[W::PER];
#pragma unroll
  for (int p = 0; p < W::PER; ++p) {
    const int u = lt + p * W::GT;
    const int64_t e = lo + u;
    const bool ok = batches > 0 && u < W::NB && e < hi;
    ci[p] = ok ? __ldg(col + e) : 0;
    cv[p] = ok ? to_f(__ldg(val + e)) : 0.0f;
  }
  for (int j = 0; j < batches; ++j) {
    float xv[W::NB][W::FEAT];
#pragma unroll
    for (int u = 0; u < W::NB; ++u) {
      const int c = W::GT > 1 ? __shfl_sync(kFull, ci[u / W::GT], u % W::GT, W::GT) : ci[u];
      load_wide<KP, MIXED>(xb + (int64_t)c * W::RB, xv[u]);
    }
    int ni[W::PER];
    float nv[W::PER];
    const int64_t e1 = lo + (int64_t)(j + 1) * W::NB;
#pragma unroll
    for (int p = 0; p < W::PER; ++p) {
      const int u = lt + p * W::GT;
      const int64_t e = e1 + u;
      const bool ok = u < W::NB && e < hi;
      ni[p] = ok ? __ldg(col + e) : 0;
      nv[p] = ok ? to_f(__ldg(val + e)) : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < W::NB; ++u) {
      const float v = W::GT > 1 ? __shfl_sync(kFull, cv[u / W::GT], u % W::GT, W::GT) : cv[u];
#pragma unroll
      for (int q = 0; q < W::FEAT; ++q) acc[q] = fmaf(v, xv[u][q], acc[q]);
    }
#pragma unroll
    for (int p = 0; p < W::PER; ++p) {
      ci[p] = ni[p];
      cv[p] = nv[p];
    }
  }
}

template <int N>
__device__ __forceinline__ void store_feats(float* base, const float* v) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int q = 0; q < N; q += 4) *reinterpret_cast<float4*>(base + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
  } else if constexpr (N == 2) {
    *reinterpret_cast<float2*>(base) = make_float2(v[0], v[1]);
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) base[q] = v[q];
  }
}

}  // namespace fc
