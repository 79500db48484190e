// Segmented kernels: one launch advances every instance of a batch class (all
// instances with the same padded cluster count KP and precision) by one
// iteration.  Each kernel is persistent and takes work from a counter that
// spans all instances; every unit of work is the same unit the instance's own
// solver would run (same row ranges, partial slots and reduction order), so a
// batched instance computes bit for bit what it computes alone.
#pragma once
#include "pass_kernels.cuh"
#include "tc_update.cuh"

namespace fc {

struct BatchMeta {
  const PassArgs* args;        // [m] per-instance pass arguments (device)
  const FoldArgs* folds;       // [m] per-instance fold arguments (device)
  const int64_t* unit_base;    // [m + 1] prefix sums of gather units
  const int64_t* heavy_base;   // [m + 1] prefix sums of chunked rows
  const int32_t* item_inst;    // [n_items] update item -> instance
  const int32_t* item_slot;    // [n_items] update item -> partial slot (= solo block index)
  const int32_t* parts_upd;    // [m] update blocks of each instance when run alone
  FistaState* const* states;   // [m]
  int32_t m;
  int32_t n_items;
  unsigned long long* work;    // [2]: gather units taken, update items taken (zeroed per iteration)
};

// index j with base[j] <= x < base[j + 1]
__device__ __forceinline__ int find_segment(const int64_t* base, int m, int64_t x) {
  int lo = 0, hi = m;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (base[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Gather tile shapes the batch autotuner chooses from, per class: nonzeros per
// batch per row (NB) and rows per team per work unit (RPU).  Shape 0 is the
// solo solver's; 1 takes single-row units (finer dynamic balance over many
// small instances); 2 halves the batch (fewer idle lanes on short rows).  No
// shape changes a value: every row is summed by one team in index order.
constexpr int kGatherShapes = 3;
template <int KP, bool MIXED, int S>
struct BShape {
  static constexpr int NB0 = WLay<KP, MIXED>::NB;
  static constexpr int NB = S == 2 ? (NB0 > 1 ? NB0 / 2 : 1) : NB0;
  static constexpr int RPU = S == 1 ? 1 : kRowsPerUnit;
};

template <int KP, bool MIXED, int S = 0>
__global__ void __launch_bounds__(Lay<KP>::NT) batch_spmm_kernel(BatchMeta b) {
  const int lane = threadIdx.x & 31;
  const int64_t total = b.unit_base[b.m];
  for (;;) {
    unsigned long long u = 0;
    if (lane == 0) u = atomicAdd(&b.work[0], 1ull);
    u = __shfl_sync(kFull, u, 0);
    if ((int64_t)u >= total) break;
    const int j = find_segment(b.unit_base, b.m, (int64_t)u);
    const PassArgs& a = b.args[j];
    const int64_t pass = pass_to_run(a.st);
    if (pass < 0) continue;
    spmm_unit<KP, MIXED, BShape<KP, MIXED, S>::NB, BShape<KP, MIXED, S>::RPU>(a, pass, (int64_t)u - b.unit_base[j],
                                                                             lane);
  }
}

template <int KP>
__global__ void __launch_bounds__(256) batch_finalize_kernel(BatchMeta b) {
  using L = Lay<KP>;
  const int64_t total = b.heavy_base[b.m];
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t teams = (int64_t)gridDim.x * blockDim.x / L::T;
  for (int64_t h = t / L::T; h < total; h += teams) {
    const int j = find_segment(b.heavy_base, b.m, h);
    const PassArgs& a = b.args[j];
    const int64_t pass = pass_to_run(a.st);
    if (pass < 0) continue;
    finalize_row<KP>(a, pass, h - b.heavy_base[j], (int)(t % L::T));
  }
}

// Update items in a persistent loop: item -> (instance, partial slot), the
// rows [n slot / parts, n (slot + 1) / parts) the instance's solo block of that
// slot takes.
__device__ __forceinline__ bool next_update_item(const BatchMeta& b, int& item_s, const PassArgs*& a, int& slot,
                                                 int64_t& pass, int64_t& p0, int64_t& p1, bool& idle) {
  if (threadIdx.x == 0) item_s = (int)atomicAdd(&b.work[1], 1ull);
  __syncthreads();
  const int item = item_s;
  __syncthreads();
  if (item >= b.n_items) return false;
  const int j = b.item_inst[item];
  slot = b.item_slot[item];
  a = &b.args[j];
  pass = pass_to_run(a->st);
  idle = pass < 0;
  if (idle) return true;
  const int parts = b.parts_upd[j];
  p0 = a->n * (int64_t)slot / parts;
  p1 = a->n * (int64_t)(slot + 1) / parts;
  return true;
}

// TC: the tcgen05 update (KP = 32; TMEM and barriers held across items), else
// the warp-level one.
template <int KP, bool MIXED, bool TC>
__global__ void __launch_bounds__(Lay<KP>::NT, Lay<KP>::MINB) batch_update_kernel(BatchMeta b) {
  __shared__ int item_s;
  const PassArgs* a = nullptr;
  int slot = 0;
  int64_t pass = 0, p0 = 0, p1 = 0;
  bool idle = false;
  if constexpr (TC && TcUpd<KP>::ON) {
    extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
    __shared__ uint64_t bars[2];
    __shared__ uint32_t tslot;
    __shared__ int tmo_flag[2];
    TcBlock tb;
    tc_begin<KP>(tb, tc_smem_raw, bars, &tslot, tmo_flag);
    while (next_update_item(b, item_s, a, slot, pass, p0, p1, idle)) {
      if (idle) continue;
      tc_update_range<KP, MIXED>(*a, pass, p0, p1, slot, tb);
      __syncthreads();
    }
    tc_end<KP>(tb);
  } else {
    extern __shared__ __align__(16) float smem[];
    while (next_update_item(b, item_s, a, slot, pass, p0, p1, idle)) {
      if (idle) continue;
      pass_range<KP, MIXED, false, true>(*a, pass, p0, p1, slot, smem);
      __syncthreads();
    }
  }
}

template <int KP>
__global__ void __launch_bounds__(256) batch_fold_kernel(BatchMeta b) {
  constexpr int nb = fold_blocks<KP>(false);
  fold_body<KP>(b.folds[blockIdx.x / nb], blockIdx.x % nb, nb);
}

__global__ void batch_set_limit_kernel(FistaState* const* states, int m, int64_t iters) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) states[j]->limit = states[j]->pass + iters;
}

__global__ void batch_collect_kernel(FistaState* const* states, int m, FistaState* out) {
  const int j = blockIdx.x;
  if (j >= m) return;
  const unsigned* src = reinterpret_cast<const unsigned*>(states[j]);
  unsigned* dst = reinterpret_cast<unsigned*>(out + j);
  for (int w = threadIdx.x; w < (int)(sizeof(FistaState) / 4); w += blockDim.x) dst[w] = src[w];
}

}  // namespace fc
