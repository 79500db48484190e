// Set-up kernels: input validation, ||S||_F^2, degree ordering and the internal
// numbering, cost-balanced block ranges, padding copies, and power iteration
// for ||S||_2.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fc {

// error bits reported by the validation kernels
enum : int {
  kErrRowPtr = 1,      // row_ptr[0] != 0, decreasing, or row_ptr[n] != nnz
  kErrColRange = 2,    // column outside [0, n)
  kErrColOrder = 4,    // columns not strictly increasing within a row
  kErrNoDiag = 8,      // a row without its diagonal entry
  kErrValue = 16,      // non-finite value
  kErrAsym = 32,       // s_ij != s_ji or (j, i) missing
  kErrU0Range = 64,    // U0 entry negative or non-finite
  kErrU0Sum = 128,     // U0 row sum differs from 1 by more than 1e-5
};

static __global__ void rowptr32_to_64(const int32_t* __restrict__ in, int64_t* __restrict__ out, int64_t n1) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n1; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i];
}

static __global__ void validate_rowptr_kernel(const int64_t* __restrict__ rp, int64_t n, int64_t nnz, int* err) {
  int bits = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = rp[i];
    if (v < 0 || v > nnz) bits |= kErrRowPtr;
    if (i == 0 && v != 0) bits |= kErrRowPtr;
    if (i == n && v != nnz) bits |= kErrRowPtr;
    if (i > 0 && rp[i - 1] > v) bits |= kErrRowPtr;
  }
  if (bits) atomicOr(err, bits);
}

// Runs only after validate_rowptr_kernel found row_ptr sound, so every
// index it forms stays inside [0, nnz).
static __global__ void validate_csr_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const float* __restrict__ val, int64_t n, int need_diag, int* err) {
  int bits = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lo = rp[i], hi = rp[i + 1];
    bool diag = false;
    int64_t prev = -1;
    for (int64_t e = lo; e < hi; ++e) {
      const int64_t c = col[e];
      if (c < 0 || c >= n) bits |= kErrColRange;
      if (c <= prev) bits |= kErrColOrder;
      if (c == i) diag = true;
      if (!isfinite(val[e])) bits |= kErrValue;
      prev = c;
    }
    if (need_diag && !diag) bits |= kErrNoDiag;
  }
  if (bits) atomicOr(err, bits);
}

// s_ij must equal s_ji: look up (j, i) by binary search in row j (runs only on
// a structurally valid CSR).
static __global__ void validate_sym_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const float* __restrict__ val, int64_t n, int* err) {
  int bits = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) {
      const int64_t j = col[e];
      int64_t lo = rp[j], hi = rp[j + 1];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < i) lo = mid + 1;
        else hi = mid;
      }
      if (lo >= rp[j + 1] || col[lo] != i || val[lo] != val[e]) bits |= kErrAsym;
    }
  }
  if (bits) atomicOr(err, bits);
}

static __global__ void validate_u0_kernel(const float* __restrict__ U, int64_t n, int k, int* err) {
  int bits = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int a = 0; a < k; ++a) {
      const float v = U[i * k + a];
      if (!(v >= 0.0f) || !isfinite(v)) bits |= kErrU0Range;
      s += (double)v;
    }
    if (fabs(s - 1.0) > 1e-5) bits |= kErrU0Sum;
  }
  if (bits) atomicOr(err, bits);
}

// Per-block float64 partial sums of val^2 (folded on the host in block order).
static __global__ void __launch_bounds__(256) sumsq_kernel(const float* __restrict__ val, int64_t nnz,
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

static __global__ void degree_kernel(const int64_t* __restrict__ rp, int64_t n, uint32_t* __restrict__ deg,
                              int32_t* __restrict__ iota) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = rp[i + 1] - rp[i];
    deg[i] = d > 0xffffffffLL ? 0xffffffffu : (uint32_t)d;
    iota[i] = (int32_t)i;
  }
}

// key[p] = order[p] / chunk (the row chunk of the row at position p)
static __global__ void chunk_key_kernel(const int32_t* __restrict__ order, int64_t m, int32_t chunk,
                                        uint32_t* __restrict__ key) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < m; p += (int64_t)gridDim.x * blockDim.x)
    key[p] = (uint32_t)(order[p] / chunk);
}

// sdeg[p] = deg[order[p]]
static __global__ void gather_deg_kernel(const uint32_t* __restrict__ deg, const int32_t* __restrict__ order,
                                         int64_t n, uint32_t* __restrict__ sdeg) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    sdeg[p] = deg[order[p]];
}

static __global__ void count_above_kernel(const uint32_t* __restrict__ deg, int64_t n, uint32_t thr,
                                   unsigned long long* cnt) {
  unsigned long long c = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    c += deg[i] > thr;
  if (c) atomicAdd(cnt, c);
}

static __global__ void heavy_lo_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ order, int64_t nh,
                                int64_t* __restrict__ lo) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nh; p += (int64_t)gridDim.x * blockDim.x)
    lo[p] = rp[order[p]];
}

// cost of a position: chunk count for chunked rows, degree otherwise, plus a
// fixed per-row charge for the row-local traffic and the epilogue
static __global__ void cost_kernel(const uint32_t* __restrict__ sdeg, int64_t n, int64_t nh, uint32_t chunk,
                            int64_t row_cost, int64_t* __restrict__ cost) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t d = sdeg[p];
    cost[p] = (p < nh ? (d + chunk - 1) / chunk : d) + row_cost;
  }
}

// cta_pos[c] = first position whose inclusive cost prefix exceeds c * total / parts
static __global__ void partition_kernel(const int64_t* __restrict__ prefix, int64_t n, int parts,
                                 int64_t* __restrict__ cta_pos) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > parts) return;
  if (c == 0) {
    cta_pos[0] = 0;
    return;
  }
  if (c == parts) {
    cta_pos[parts] = n;
    return;
  }
  const int64_t total = prefix[n - 1];
  const int64_t target = (int64_t)((__int128)total * c / parts);
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (prefix[mid] <= target) lo = mid + 1;
    else hi = mid;
  }
  cta_pos[c] = lo;
}

// ---- internal numbering by decreasing degree ----
// inv[perm[p]] = p
static __global__ void inverse_perm_kernel(const int32_t* __restrict__ perm, int64_t n, int32_t* __restrict__ inv) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
    inv[perm[p]] = (int32_t)p;
}

// cnt[p] = nonzeros of the caller's row perm[p]; cnt[n] = 0 (exclusive scan -> row pointers)
static __global__ void permuted_count_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ perm,
                                             int64_t n, int64_t* __restrict__ cnt) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p <= n; p += (int64_t)gridDim.x * blockDim.x)
    cnt[p] = p < n ? rp[perm[p] + 1] - rp[perm[p]] : 0;
}

// One warp per internal row p: the caller's row perm[p], entries in their
// order, columns renamed through inv.
static __global__ void relabel_rows_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                           const float* __restrict__ val, const int32_t* __restrict__ perm,
                                           const int32_t* __restrict__ inv, const int64_t* __restrict__ rp2,
                                           int64_t n, int32_t* __restrict__ col2, float* __restrict__ val2) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * blockDim.x / 32;
  for (int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; p < n; p += warps) {
    const int64_t lo = rp[perm[p]], len = rp[perm[p] + 1] - lo, dst = rp2[p];
    for (int64_t e = lane; e < len; e += 32) {
      col2[dst + e] = inv[col[lo + e]];
      val2[dst + e] = val[lo + e];
    }
  }
}

// X[p] = U[perm[p]] zero-padded to KP (+ optional copies)
static __global__ void pad_perm_kernel(const float* __restrict__ U, const int32_t* __restrict__ perm, int64_t n,
                                       int k, int KP, float* __restrict__ X, float* __restrict__ X2,
                                       __nv_bfloat16* __restrict__ XS, __nv_bfloat16* __restrict__ XS2) {
  const int64_t tot = n * KP;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / KP;
    const int a = (int)(i % KP);
    const float v = a < k ? U[(int64_t)perm[r] * k + a] : 0.0f;
    X[i] = v;
    if (X2) X2[i] = v;
    if (XS) XS[i] = __float2bfloat16_rn(v);
    if (XS2) XS2[i] = __float2bfloat16_rn(v);
  }
}

// U[i] = X[inv[i]] without the padding
static __global__ void unpad_perm_kernel(const float* __restrict__ X, const int32_t* __restrict__ inv, int64_t n,
                                         int k, int KP, float* __restrict__ U) {
  const int64_t tot = n * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / k;
    const int a = (int)(i % k);
    U[i] = X[(int64_t)inv[r] * KP + a];
  }
}

// n x k (row-major, stride k) -> n x KP zero-padded float32 (+ optional copies)
static __global__ void pad_kernel(const float* __restrict__ U, int64_t n, int k, int KP, float* __restrict__ X,
                           float* __restrict__ X2, __nv_bfloat16* __restrict__ XS,
                           __nv_bfloat16* __restrict__ XS2) {
  const int64_t tot = n * KP;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / KP;
    const int a = (int)(i % KP);
    const float v = a < k ? U[r * k + a] : 0.0f;
    X[i] = v;
    if (X2) X2[i] = v;
    if (XS) XS[i] = __float2bfloat16_rn(v);
    if (XS2) XS2[i] = __float2bfloat16_rn(v);
  }
}

static __global__ void unpad_kernel(const float* __restrict__ X, int64_t n, int k, int KP, float* __restrict__ U) {
  const int64_t tot = n * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < tot; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / k;
    const int a = (int)(i % k);
    U[i] = X[r * KP + a];
  }
}

static __global__ void to_bf16_kernel(const float* __restrict__ in, int64_t m, __nv_bfloat16* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

// y = S x, one thread per row (set-up only)
static __global__ void spmv_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const float* __restrict__ val, const double* __restrict__ x, int64_t n,
                            double* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t e = rp[i]; e < rp[i + 1]; ++e) s += (double)val[e] * x[col[e]];
    y[i] = s;
  }
}

static __global__ void __launch_bounds__(256) dot_part_kernel(const double* __restrict__ a, const double* __restrict__ b,
                                                        int64_t n, double* __restrict__ part) {
  __shared__ double red[256];
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

static __global__ void scale_kernel(double* __restrict__ x, int64_t n, double s) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] *= s;
}

static __global__ void fill_start_kernel(double* __restrict__ x, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    // fixed, strictly positive start vector (not orthogonal to the Perron vector of a nonnegative S)
    uint64_t z = (uint64_t)i * 0x9E3779B97F4A7C15ull;
    z ^= z >> 29;
    x[i] = 1.0 + (double)(z & 0xffff) / 65536.0;
  }
}

// flag = 1 if order[p] != p for some p (the gather order is not the identity)
static __global__ void order_identity_kernel(const int32_t* order, int64_t n, int* flag) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride)
    if (order[p] != (int32_t)p) *flag = 1;
}

}  // namespace fc
