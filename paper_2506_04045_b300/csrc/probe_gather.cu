// Random-row gather rate on sm_103a: the access pattern of the product S X
// (one row of the iterate per nonzero of S, rows chosen by the column index)
// isolated from everything else.  Two ways to bring the rows in:
//   * plain loads: row_bytes / 16 lanes share a row, each lane one 16-byte
//     load (ld.global.nc, optionally with the 64-byte L2 fetch hint), eight
//     rows per lane group in flight (a batch's indices first, then its rows);
//   * TMA tile::gather4: one elected lane per warp issues cp.async.bulk.tensor
//     gathers of 4 rows into a ring of shared-memory stages (mbarrier per
//     stage), and the warp consumes each stage from shared memory.
// Both reduce what they read into a per-thread checksum, so no load is dead.
// Built as its own library (libgather_probe.so) for bench.py's "rowrate"
// workload; the solver does not use it.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <mutex>

#define PROBE_API extern "C" __attribute__((visibility("default")))

namespace {

constexpr unsigned kFull = 0xffffffffu;

template <int RB, bool HINT64>
__device__ __forceinline__ uint4 load16(const uint8_t* p) {
  uint4 v;
  if constexpr (HINT64) {
    asm volatile("ld.global.nc.L2::64B.v4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
  } else {
    v = __ldg(reinterpret_cast<const uint4*>(p));
  }
  return v;
}

// Plain loads: GT = RB / 16 lanes per row, TPW = 32 / GT rows per warp and
// NB rows per lane group in flight; warps take chunks of TPW * NB indices.
template <int RB, bool HINT64>
__global__ void __launch_bounds__(256) probe_ldg_kernel(const uint8_t* __restrict__ table,
                                                        const int32_t* __restrict__ idx, int64_t m,
                                                        uint32_t* __restrict__ sink) {
  constexpr int GT = RB / 16, TPW = 32 / GT, NB = 8, CH = TPW * NB;
  const int lane = threadIdx.x & 31, g = lane / GT, lt = lane % GT;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  uint32_t acc = 0;
  for (int64_t base = warp * CH; base < m; base += nwarps * CH) {
    int r[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int64_t e = base + (int64_t)u * TPW + g;
      r[u] = e < m ? __ldg(idx + e) : -1;
    }
    uint4 v[NB];
#pragma unroll
    for (int u = 0; u < NB; ++u)
      v[u] = r[u] >= 0 ? load16<RB, HINT64>(table + (int64_t)r[u] * RB + lt * 16) : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int u = 0; u < NB; ++u) acc += v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
  }
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// ---- TMA tile::gather4 ----
constexpr int G4_WARPS = 4;     // warps per CTA, each with its own ring
constexpr int G4_STAGES = 32;   // stages per warp: 4 rows each
constexpr uint32_t kPolls = 1u << 20;

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(1000u)
      : "memory");
  return ok != 0;
}

// The warp's ring: stage s holds rows idx[4 q .. 4 q + 3] of its q-th group.
// Lane 0 keeps every stage in flight; the warp waits for a stage, folds it
// into the checksum, and lane 0 refills it with the group G4_STAGES ahead.
// A wait that gives up sets *err and stops the warp after its loads land.
template <int RB>
__global__ void __launch_bounds__(G4_WARPS * 32) probe_gather4_kernel(const __grid_constant__ CUtensorMap map,
                                                                      const int32_t* __restrict__ idx, int64_t m,
                                                                      uint32_t* __restrict__ sink, int* err) {
  extern __shared__ __align__(1024) uint8_t g4_smem[];
  __shared__ __align__(8) uint64_t bars[G4_WARPS][G4_STAGES];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint8_t* ring = g4_smem + (size_t)warp * G4_STAGES * 4 * RB;
  const int64_t groups = m / 4;
  const int64_t gw = (int64_t)blockIdx.x * G4_WARPS + warp, nw = (int64_t)gridDim.x * G4_WARPS;
  // this warp's groups: gw, gw + nw, ...
  const int64_t mine = groups > gw ? (groups - gw + nw - 1) / nw : 0;
  if (lane == 0) {
    for (int s = 0; s < G4_STAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bars[warp][s])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  auto issue = [&](int64_t q) {  // group q of this warp into stage q % G4_STAGES
    const int s = (int)(q % G4_STAGES);
    const int64_t e = (gw + q * nw) * 4;
    const int r0 = __ldg(idx + e), r1 = __ldg(idx + e + 1), r2 = __ldg(idx + e + 2), r3 = __ldg(idx + e + 3);
    const uint32_t bar = saddr(&bars[warp][s]);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(4 * RB) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile::gather4.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(saddr(ring + (size_t)s * 4 * RB)),
        "l"(&map), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar)
        : "memory");
  };
  if (lane == 0)
    for (int64_t q = 0; q < mine && q < G4_STAGES; ++q) issue(q);
  uint32_t acc = 0;
  int64_t q = 0;
  for (; q < mine; ++q) {
    const int s = (int)(q % G4_STAGES);
    const uint32_t par = (uint32_t)(q / G4_STAGES) & 1u;
    bool ok = false;
    for (uint32_t i = 0; i < kPolls && !ok; ++i) ok = try_wait(saddr(&bars[warp][s]), par);
    if (!__all_sync(kFull, ok)) {
      if (lane == 0) atomicExch(err, 1);
      break;
    }
    // 4 rows of RB bytes: 16-byte pieces over the lanes
    for (int o = lane * 16; o < 4 * RB; o += 512) {
      const uint4 v = *reinterpret_cast<const uint4*>(ring + (size_t)s * 4 * RB + o);
      acc += v.x ^ v.y ^ v.z ^ v.w;
    }
    __syncwarp();
    if (lane == 0 && q + G4_STAGES < mine) issue(q + G4_STAGES);
  }
  // a warp that gave up still lets its issued loads land before the CTA exits
  if (q < mine && lane == 0) {
    for (int64_t p = q; p < mine && p < q + G4_STAGES; ++p) {
      bool ok = false;
      for (uint32_t i = 0; i < kPolls && !ok; ++i)
        ok = try_wait(saddr(&bars[warp][p % G4_STAGES]), (uint32_t)(p / G4_STAGES) & 1u);
    }
  }
  sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

}  // namespace

namespace {
template <int RB, bool H>
void launch_ldg(const void* table, const int32_t* idx, int64_t m, int grid, uint32_t* sink, cudaStream_t s) {
  probe_ldg_kernel<RB, H><<<grid, 256, 0, s>>>(static_cast<const uint8_t*>(table), idx, m, sink);
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}
}  // namespace

// Gather m rows of row_bytes (32, 64, 128 or 256) from `table` (rows x
// row_bytes, device, 16-byte aligned) at the row indices idx[0..m) (device,
// each in [0, rows)).  mode 0: plain 16-byte loads; mode 1: the same with the
// 64-byte L2 fetch hint (row_bytes <= 64); mode 2: TMA tile::gather4 (row_bytes
// 64 or 128, m a multiple of 4).  grid: CTAs (0 = a full wave).  sink: device
// uint32 scratch of at least grid x 256 entries (checksums).  Runs `reps`
// launches on `stream` and writes their mean duration in milliseconds (CUDA
// events) to *ms.  Returns 0, or a nonzero code: 1 bad argument, 2 CUDA
// error, 3 a wait of the gather4 kernel gave up.
PROBE_API int probe_gather(const void* table, int64_t rows, int32_t row_bytes, const int32_t* idx, int64_t m,
                           int32_t mode, int32_t grid, int32_t reps, void* sink, void* stream, double* ms) {
  if (!table || !idx || !sink || !ms || rows < 1 || m < 4 || reps < 1 || rows > 0x7fffffffLL) return 1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))
    return 2;
  uint32_t* sk = static_cast<uint32_t*>(sink);
  CUtensorMap map;
  int* err = nullptr;
  size_t smem = 0;
  if (mode == 2) {
    if ((row_bytes != 64 && row_bytes != 128) || m % 4) return 1;
    auto enc = encoder();
    if (!enc) return 2;
    const cuuint64_t dims[2] = {(cuuint64_t)(row_bytes / 4), (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    const cuuint32_t box[2] = {(cuuint32_t)(row_bytes / 4), 1};
    const cuuint32_t es[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT32, 2, const_cast<void*>(table), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return 2;
    smem = (size_t)G4_WARPS * G4_STAGES * 4 * row_bytes;
    cudaError_t e = row_bytes == 64
                        ? cudaFuncSetAttribute(probe_gather4_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem)
                        : cudaFuncSetAttribute(probe_gather4_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return 2;
    int occ = 0;
    e = row_bytes == 64
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_gather4_kernel<64>, G4_WARPS * 32, smem)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, probe_gather4_kernel<128>, G4_WARPS * 32, smem);
    if (e != cudaSuccess) return 2;
    if (grid <= 0) grid = sms * (occ > 0 ? occ : 1);
    if (cudaMalloc(&err, sizeof(int)) != cudaSuccess) return 2;
    cudaMemsetAsync(err, 0, sizeof(int), s);
  } else {
    if (row_bytes != 32 && row_bytes != 64 && row_bytes != 128 && row_bytes != 256) return 1;
    if (mode == 1 && row_bytes > 64) return 1;
    if (grid <= 0) grid = sms * 8;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps; ++r) {
    if (mode == 2) {
      if (row_bytes == 64)
        probe_gather4_kernel<64><<<grid, G4_WARPS * 32, smem, s>>>(map, idx, m, sk, err);
      else
        probe_gather4_kernel<128><<<grid, G4_WARPS * 32, smem, s>>>(map, idx, m, sk, err);
    } else if (mode == 1) {
      if (row_bytes == 32) launch_ldg<32, true>(table, idx, m, grid, sk, s);
      else launch_ldg<64, true>(table, idx, m, grid, sk, s);
    } else {
      switch (row_bytes) {
        case 32: launch_ldg<32, false>(table, idx, m, grid, sk, s); break;
        case 64: launch_ldg<64, false>(table, idx, m, grid, sk, s); break;
        case 128: launch_ldg<128, false>(table, idx, m, grid, sk, s); break;
        default: launch_ldg<256, false>(table, idx, m, grid, sk, s); break;
      }
    }
  }
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  float t = 0.f;
  if (e == cudaSuccess) cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  int herr = 0;
  if (err) {
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(err);
  }
  if (e != cudaSuccess) return 2;
  if (herr) return 3;
  *ms = t / reps;
  return 0;
}
