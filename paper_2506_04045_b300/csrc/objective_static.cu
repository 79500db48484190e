// Allocation-free objective: cluster_objective_static.
//
// Same arithmetic as cluster_objective (the objective-only pass and its
// float64 fold), but every piece of device scratch lives in one file-scope
// __device__ array instead of memory obtained from cudaMalloc.  It exists for
// callers that cannot allocate device memory at the point where they need
// the objective: for example a service that hands all free device memory to
// its own pool allocator at start-up (so cudaMalloc would fail or fragment
// that pool), or code on a latency-critical path where cudaMalloc/cudaFree
// would synchronise the device.
#include <cuda_runtime.h>
#include <string.h>

#include <stdint.h>

#include <mutex>

#include "pass_kernels.cuh"
#include "util.h"

namespace {

using fc::FistaState;
using fc::FoldArgs;
using fc::PassArgs;

// The largest padded cluster count (k in {2, 4, 8, 16, 32}); the partial
// pool holds 320 block partials at that size.
constexpr int kMaxKP = 32;
constexpr int kPartsAtMaxKP = 320;
constexpr int kSumParts = 1024;

// Bytes of one block's partials at padded size KP: a 2 x KP x KP float32 Gram
// slot and four float64 scalars.
__host__ __device__ constexpr size_t part_bytes(int KP) { return sizeof(float) * 2 * (size_t)KP * KP + 4 * sizeof(double); }

// Scratch layout (bytes):
//   [0, P)            partial pool: parts Gram slots (2 KP^2 float32 each),
//                     then parts x 4 float64 scalar partials
//   then              fold result     kMaxKP^2 float64
//   then              sum-of-squares partials kSumParts float64
//   then              FistaState
// A smaller k fits more block partials into the same pool (parts_cap).
constexpr size_t kPoolBytes = part_bytes(kMaxKP) * kPartsAtMaxKP;
constexpr size_t kABytes = sizeof(double) * (size_t)kMaxKP * kMaxKP;
constexpr size_t kSumBytes = sizeof(double) * (size_t)kSumParts;
constexpr size_t kStateBytes = (sizeof(FistaState) + 255) / 256 * 256;
constexpr size_t kScratchBytes = kPoolBytes + kABytes + kSumBytes + kStateBytes;  // about 2.7 MB

// Block partials the pool holds at padded size KP (320 at KP = 32, 1265 at
// KP = 16, 4837 at KP = 8): a smaller k runs with as many blocks as
// cluster_objective would.
constexpr int64_t parts_cap(int KP) { return (int64_t)(kPoolBytes / part_bytes(KP)); }

static __device__ __align__(256) unsigned char g_objective_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Per-block float64 partial sums of val^2.
__global__ void __launch_bounds__(256) static_sumsq_kernel(const float* __restrict__ val, int64_t nnz,
                                                            double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)val[e];
    s += v * v;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

template <int KP>
cluster_status run_static(const cluster_csr* S, int32_t k, const float* U, cudaStream_t s, unsigned char* base,
                          int sms, double* f) {
  using L = fc::Lay<KP>;
  int occ = 0;
  const size_t smem = fc::pass_smem_bytes<KP>(true);
  FC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fc::fista_pass_kernel<KP, false, true>, L::NT, smem));
  const int64_t n = S->n;
  int64_t parts = (int64_t)sms * (occ < 1 ? 1 : occ);
  if (parts > parts_cap(KP)) parts = parts_cap(KP);
  if (parts > (n + L::R - 1) / L::R) parts = (n + L::R - 1) / L::R;
  if (parts < 1) parts = 1;

  // Gram slots first (16-byte aligned rows), the float64 scalars after them
  float* gram_part = reinterpret_cast<float*>(base);
  double* sc_part = reinterpret_cast<double*>(base + sizeof(float) * 2 * (size_t)KP * KP * parts);
  double* A = reinterpret_cast<double*>(base + kPoolBytes);
  double* sum_part = reinterpret_cast<double*>(base + kPoolBytes + kABytes);
  FistaState* st = reinterpret_cast<FistaState*>(base + kPoolBytes + kABytes + kSumBytes);

  // ||S||_F^2: block partials in scratch, folded on the host in block order
  double hpart[kSumParts];
  double S2 = 0.0;
  if (S->nnz > 0) {
    static_sumsq_kernel<<<kSumParts, 256, 0, s>>>(S->val, S->nnz, sum_part);
    FC_CUDA(cudaGetLastError());
    FC_CUDA(cudaMemcpyAsync(hpart, sum_part, sizeof(hpart), cudaMemcpyDeviceToHost, s));
    FC_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < kSumParts; ++i) S2 += hpart[i];
  }
  // the state starts from zero on every call (the fold's block counter included)
  FistaState h;
  memset(&h, 0, sizeof(h));
  h.S2 = S2;
  h.k = k;
  FC_CUDA(cudaMemcpyAsync(st, &h, sizeof(h), cudaMemcpyHostToDevice, s));

  PassArgs a;
  memset(&a, 0, sizeof(a));
  a.row_ptr = reinterpret_cast<const int64_t*>(S->row_ptr);
  a.col = S->col;
  a.val = S->val;
  a.order = nullptr;    // rows in index order
  a.cta_pos = nullptr;  // even split of the rows over the blocks
  a.n_heavy = 0;
  a.X0 = const_cast<float*>(U);  // k == KP: U is read in place (the pass never writes in this mode)
  a.gram_part = gram_part;
  a.sc_part = sc_part;
  a.st = st;
  a.n = n;
  a.k = k;
  a.eval_sel = 0;
  fc::fista_pass_kernel<KP, false, true><<<(int)parts, L::NT, smem, s>>>(a);
  FC_CUDA(cudaGetLastError());

  FoldArgs fa;
  memset(&fa, 0, sizeof(fa));
  fa.st = st;
  fa.gram_part = gram_part;
  fa.sc_part = sc_part;
  fa.parts = (int32_t)parts;
  fa.eval = 1;
  fa.eval_init = 0;
  fa.A = A;
  fc::fold_kernel<KP><<<fc::fold_blocks<KP>(true), 256, 0, s>>>(fa);
  FC_CUDA(cudaGetLastError());
  FC_CUDA(cudaMemcpyAsync(&h, st, sizeof(h), cudaMemcpyDeviceToHost, s));
  FC_CUDA(cudaStreamSynchronize(s));
  *f = h.eval_f;
  return CLUSTER_OK;
}

}  // namespace

extern "C" cluster_status cluster_objective_static(const cluster_csr* S, int32_t k, const float* U, void* stream,
                                                   double* f) {
  fc::clear_error();
  if (!S || !U || !f) FC_EINVAL("cluster_objective_static: NULL argument");
  if (S->n < 1 || S->n > 0x7fffffffLL) FC_EINVAL("cluster_objective_static: n must be in [1, 2^31)");
  if (S->nnz < 0 || !S->row_ptr || (S->nnz > 0 && (!S->col || !S->val)))
    FC_EINVAL("cluster_objective_static: bad CSR arrays");
  if (!S->index64)
    FC_EINVAL("cluster_objective_static: row_ptr must be int64 (index64 = 1); widening it would need memory");
  if (k != 2 && k != 4 && k != 8 && k != 16 && k != 32)
    FC_EINVAL("cluster_objective_static: k must be 2, 4, 8, 16 or 32 (got %d); other k need a padded copy of U", k);
  if (reinterpret_cast<uintptr_t>(U) % (k == 2 ? 8 : 16) != 0)
    FC_EINVAL("cluster_objective_static: U must be %d-byte aligned", k == 2 ? 8 : 16);
  // the call synchronises its stream and reads partial sums on the host, which
  // a stream capture cannot record
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  FC_CUDA(cudaStreamIsCapturing((cudaStream_t)stream, &cap));
  if (cap != cudaStreamCaptureStatusNone)
    FC_EINVAL("cluster_objective_static: the stream is being captured (the call synchronises it and reads "
              "results on the host, so it cannot be part of a CUDA graph)");
  int dev = 0;
  FC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) FC_EINVAL("cluster_objective_static: device index %d out of range", dev);
  void* base = nullptr;
  {
    // one-time set-up per device: the device address of the scratch array
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_objective_scratch);
      if (e != cudaSuccess || !p) {
        fc::set_error("cluster_objective_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
        return CLUSTER_ECUDA;
      }
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }
  int sms = 0;
  FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t s = (cudaStream_t)stream;
  unsigned char* b = static_cast<unsigned char*>(base);
  switch (k) {
    case 2: return run_static<2>(S, k, U, s, b, sms, f);
    case 4: return run_static<4>(S, k, U, s, b, sms, f);
    case 8: return run_static<8>(S, k, U, s, b, sms, f);
    case 16: return run_static<16>(S, k, U, s, b, sms, f);
    default: return run_static<32>(S, k, U, s, b, sms, f);
  }
}
