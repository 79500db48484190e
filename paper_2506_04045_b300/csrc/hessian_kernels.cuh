// Second-order check (Theorem 4.1, Eq. "hessian"): the Hessian of f at U
// applied to a direction W, in row (U = Xbar^T) notation
//
//   H[W] = -4 S W + 4 W (U^T U) + 4 U (U^T W + W^T U),
//
// plus the curvature <W, H[W]> and the slope <grad f(U), W> with
// grad f(U) = -4 (S U - U U^T U).  One product S W serves all three (S is
// symmetric, so <U, S W> = <W, S U>).  The product runs through the
// solver's gather kernel; these kernels form the three k x k Grams
// (G = U^T U, M = U^T W, N = W^T W) and the row-local combination.
#pragma once
#include "iter_common.cuh"

namespace fc {

constexpr int kHessRows = 32;    // rows per shared-memory tile of the Gram kernel
constexpr int kHessPerThr = 8;   // Gram entries per thread

// Block (blockIdx.x, blockIdx.y): rows [r0, r1) of an even split into
// gridDim.x parts, entries [blockIdx.y * 256 * 8, ...) of the 3 KP^2 entries
// of (G, M, N); float32 sums over the rows into part[x][3][KP][KP].
template <int KP>
__global__ void __launch_bounds__(256) hess_gram_kernel(const float* __restrict__ Up, const float* __restrict__ Wp,
                                                        int64_t n, float* __restrict__ part) {
  __shared__ float us[kHessRows * KP];
  __shared__ float ws[kHessRows * KP];
  constexpr int E2 = KP * KP;
  const int64_t r0 = n * blockIdx.x / gridDim.x, r1 = n * (blockIdx.x + 1) / gridDim.x;
  const int ebase = blockIdx.y * 256 * kHessPerThr;
  float acc[kHessPerThr];
  int mat[kHessPerThr], ea[kHessPerThr], eb[kHessPerThr];
#pragma unroll
  for (int j = 0; j < kHessPerThr; ++j) {
    acc[j] = 0.f;
    const int e = ebase + j * 256 + threadIdx.x;
    mat[j] = e < 3 * E2 ? e / E2 : -1;
    ea[j] = (e % E2) / KP;
    eb[j] = e % KP;
  }
  for (int64_t t0 = r0; t0 < r1; t0 += kHessRows) {
    const int rows = (int)(r1 - t0 < kHessRows ? r1 - t0 : kHessRows);
    for (int i = threadIdx.x; i < kHessRows * KP; i += 256) {
      const int r = i / KP;
      us[i] = r < rows ? Up[(t0 + r) * KP + i % KP] : 0.f;
      ws[i] = r < rows ? Wp[(t0 + r) * KP + i % KP] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kHessPerThr; ++j) {
      if (mat[j] < 0) continue;
      const float* A = mat[j] == 2 ? ws : us;  // G = U^T U, M = U^T W, N = W^T W
      const float* B = mat[j] == 0 ? us : ws;
      float s = acc[j];
      for (int r = 0; r < kHessRows; ++r) s = fmaf(A[r * KP + ea[j]], B[r * KP + eb[j]], s);
      acc[j] = s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < kHessPerThr; ++j)
    if (mat[j] >= 0) part[(size_t)blockIdx.x * 3 * E2 + ebase + j * 256 + threadIdx.x] = acc[j];
}

// out[e] = sum over parts p (in order) of part[p][e], float64.
__global__ void hess_fold_kernel(const float* __restrict__ part, int parts, int entries, double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= entries) return;
  double s = 0.0;
  for (int p = 0; p < parts; ++p) s += (double)part[(size_t)p * entries + e];
  out[e] = s;
}

// One thread per (row i, column b < KP): HW_ib = -4 z_ib + 4 (w_i G)_b + 4 (u_i B)_b
// with B = M + M^T (G, B float32 in shared memory).  Block partials (float64) of
// sum_i <w_i, z_i> and sum_i <u_i, z_i>.  HW (n x k, row-major) may be null.
template <int KP>
__global__ void __launch_bounds__(256) hess_row_kernel(const float* __restrict__ Up, const float* __restrict__ Wp,
                                                       const float* __restrict__ Z, const float* __restrict__ Gf,
                                                       const float* __restrict__ Bf, int64_t n, int k,
                                                       float* __restrict__ HW, double* __restrict__ dots) {
  extern __shared__ float gb[];  // G | B
  for (int e = threadIdx.x; e < 2 * KP * KP; e += 256) gb[e] = e < KP * KP ? Gf[e] : Bf[e - KP * KP];
  __syncthreads();
  const float* G = gb;
  const float* B = gb + KP * KP;
  double wz = 0.0, uz = 0.0;
  const int64_t total = n * KP;
  for (int64_t t = (int64_t)blockIdx.x * 256 + threadIdx.x; t < total; t += (int64_t)gridDim.x * 256) {
    const int64_t i = t / KP;
    const int b = (int)(t % KP);
    const float* w = Wp + i * KP;
    const float* u = Up + i * KP;
    float wg = 0.f, ub = 0.f;
    for (int a = 0; a < KP; ++a) {
      wg = fmaf(w[a], G[a * KP + b], wg);
      ub = fmaf(u[a], B[a * KP + b], ub);
    }
    const float z = Z[t];
    if (HW && b < k) HW[i * k + b] = 4.f * (wg + ub - z);
    wz += (double)w[b] * (double)z;
    uz += (double)u[b] * (double)z;
  }
  __shared__ double red[2][256];
  red[0][threadIdx.x] = wz;
  red[1][threadIdx.x] = uz;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      red[0][threadIdx.x] += red[0][threadIdx.x + o];
      red[1][threadIdx.x] += red[1][threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    dots[blockIdx.x * 2 + 0] = red[0][0];
    dots[blockIdx.x * 2 + 1] = red[1][0];
  }
}

}  // namespace fc
