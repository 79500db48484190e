// Split iteration, steps 1 and 2: the product Z = S Xbar of the newest iterate
// (spmm_kernel, a pure gather) and the sums of the partial products of
// chunked rows (heavy_finalize_kernel).
#pragma once
#include "iter_common.cuh"

namespace fc {

// Split iteration, step 1: z_i = (S Xbar^{pass})_i for every row, stored in
// Z_{(pass+1)&1}, plus the partial products of chunked rows (units
// [unit_lo, unit_hi) of the work list when the pass is chunked).  Pure gather, no
// per-tile barrier: warps take work units from a global counter (units of
// TPW chunks first, then units of TPW * kRowsPerUnit consecutive positions of
// the processing order, whose neighbouring positions hold rows of similar
// degree, so the teams of a warp have about equal trip counts).  Each row's
// result is computed by exactly one team in a fixed order, so the dynamic
// schedule does not change any value.
constexpr int kRowsPerUnit = 4;

// Work units of one instance's gather: chunk units, then row units of
// TPW * RPU consecutive positions.
template <int KP, bool MIXED>
__host__ __device__ __forceinline__ int64_t spmm_chunk_units(int64_t n_chunks) {
  return (n_chunks + WLay<KP, MIXED>::TPW - 1) / WLay<KP, MIXED>::TPW;
}
template <int KP, bool MIXED, int RPU = kRowsPerUnit>
__host__ __device__ __forceinline__ int64_t spmm_units(int64_t n, int64_t n_heavy, int64_t n_chunks) {
  const int64_t per = (int64_t)WLay<KP, MIXED>::TPW * RPU;
  return spmm_chunk_units<KP, MIXED>(n_chunks) + (n - n_heavy + per - 1) / per;
}

// One warp processes gather unit u of an instance (see spmm_kernel); the
// GT lanes of a row each own FEAT consecutive features of z.  Tile shape:
// NBX nonzeros per batch (0 = the layout's), RPU rows per team per unit; the
// shape changes no value (each row is summed by one team in index order).
template <int KP, bool MIXED, int NBX = 0, int RPU = kRowsPerUnit>
__device__ __forceinline__ void spmm_unit(const PassArgs& a, int64_t pass, int64_t u, int lane) {
  using W = WShape<KP, MIXED, NBX>;
  const float* P = (pass & 1) ? a.X1 : a.X0;
  const void* Xg = MIXED ? (const void*)((pass & 1) ? a.XS1 : a.XS0) : (const void*)P;
  float* Zc = ((pass + 1) & 1) ? a.Z1 : a.Z0;
  const int tiw = lane / W::GT, lt = lane % W::GT, f0 = lt * W::FEAT;
  const int64_t n_cu = spmm_chunk_units<KP, MIXED>(a.n_chunks);
  if (u < n_cu) {
    const int64_t c = u * W::TPW + tiw;
    const bool act = c < a.n_chunks;
    const int64_t lo = act ? a.chunk_e0[c] : 0, hi = act ? a.chunk_e1[c] : 0;
    float acc[W::FEAT];
#pragma unroll
    for (int q = 0; q < W::FEAT; ++q) acc[q] = 0.f;
    const int batches = __reduce_max_sync(kFull, (int)((hi - lo + W::NB - 1) / W::NB));
    gather_wide<KP, MIXED, W::NB>(a.col, a.val, Xg, lo, hi, batches, lt, acc);
    if (act) store_feats<W::FEAT>(a.hv_part + c * KP + f0, acc);
    return;
  }
  const int64_t base = a.n_heavy + (u - n_cu) * W::TPW * RPU;
  int64_t nrow = (base + tiw < a.n) ? (int64_t)a.order[base + tiw] : 0;
#pragma unroll 1
  for (int m = 0; m < RPU; ++m) {
    const int64_t pos = base + (int64_t)m * W::TPW + tiw;
    const bool act = pos < a.n;
    const int64_t row = nrow;
    const int64_t npos = pos + W::TPW;
    nrow = (m + 1 < RPU && npos < a.n) ? (int64_t)a.order[npos] : 0;
    const int64_t lo = act ? a.row_ptr[row] : 0, hi = act ? a.row_ptr[row + 1] : 0;
    float acc[W::FEAT];
#pragma unroll
    for (int q = 0; q < W::FEAT; ++q) acc[q] = 0.f;
    const int batches = __reduce_max_sync(kFull, (int)((hi - lo + W::NB - 1) / W::NB));
    gather_wide<KP, MIXED, W::NB>(a.col, a.val, Xg, lo, hi, batches, lt, acc);
    if (act) store_feats<W::FEAT>(Zc + row * KP + f0, acc);
  }
}

// Resident blocks per SM the gather's register budget is sized for: the
// float32 k <= 32 gather (128-byte rows) ran 1.8% faster with 5 blocks (48
// registers) than with 4 (58); the bfloat16 one (64-byte rows) 7% slower, and
// 6 blocks were slower for both.  0: no bound (the compiler's choice).
template <int KP, bool MIXED>
__host__ __device__ constexpr int spmm_min_blocks() {
  return (KP == 32 && !MIXED) ? 5 : 0;
}

// RPU rows per team per unit: kRowsPerUnit, or 1 for an instance too small to
// give every resident warp a unit of kRowsPerUnit rows (a unit's rows are
// gathered one after another, so at a few thousand rows the last unit's chain
// of dependent loads sets the launch's time).
template <int KP, bool MIXED, int RPU = kRowsPerUnit>
__global__ void __launch_bounds__(Lay<KP>::NT, spmm_min_blocks<KP, MIXED>()) spmm_kernel(PassArgs a) {
  const int64_t pass = pass_to_run(a.st);
  if (pass < 0) return;
  const int lane = threadIdx.x & 31;
  const int64_t units = a.unit_hi < 0 ? spmm_units<KP, MIXED, RPU>(a.n, a.n_heavy, a.n_chunks) : a.unit_hi;
  for (;;) {
    unsigned long long u = 0;
    if (lane == 0) u = atomicAdd(a.work, 1ull);
    u = __shfl_sync(kFull, u, 0);
    const int64_t unit = a.unit_lo + (int64_t)u;
    if (unit >= units) break;
    spmm_unit<KP, MIXED, 0, RPU>(a, pass, unit, lane);
  }
}

// Split iteration, step 2: z of every chunked row = sum of its chunk partials
// in chunk order.
template <int KP>
__device__ __forceinline__ void finalize_row(const PassArgs& a, int64_t pass, int64_t p, int lt) {
  using L = Lay<KP>;
  float* Zc = ((pass + 1) & 1) ? a.Z1 : a.Z0;
  const int f0 = lt * L::VEC;
  const int64_t row = a.order[p];
  float acc[L::VEC];
#pragma unroll
  for (int q = 0; q < L::VEC; ++q) acc[q] = 0.f;
  for (int64_t c = a.chunk_ptr[p]; c < a.chunk_ptr[p + 1]; ++c) {
    float pv[L::VEC];
    load_row<L::VEC>(a.hv_part + c * KP + f0, pv);
#pragma unroll
    for (int q = 0; q < L::VEC; ++q) acc[q] += pv[q];
  }
  store_row<L::VEC>(Zc + row * KP + f0, acc);
}

template <int KP>
__global__ void __launch_bounds__(256) heavy_finalize_kernel(PassArgs a) {
  using L = Lay<KP>;
  const int64_t pass = pass_to_run(a.st);
  if (pass < 0) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t teams = (int64_t)gridDim.x * blockDim.x / L::T;
  for (int64_t p = t / L::T; p < a.n_heavy; p += teams) finalize_row<KP>(a, pass, p, (int)(t % L::T));
}

}  // namespace fc
