// Row schedule of a solver context: the internal numbering of the articles
// (by decreasing degree), the processing order of the gather (hub rows first
// in degree order, then chunks of consecutive rows, degree order inside each
// chunk), the chunk table of hub rows and the cost-balanced position ranges
// of the fused pass.  Included by solver.cu only.
#pragma once
#include <cub/cub.cuh>

#include <algorithm>
#include <vector>

#include "init_kernels.cuh"
#include "solver_impl.h"
#include "util.h"

namespace fc {

// rows per chunk of the gather's processing order (see build_schedule)
#ifndef FC_ROW_CHUNK
#define FC_ROW_CHUNK 8192
#endif
static const int32_t kRowChunk = FC_ROW_CHUNK;

// perm = rows by decreasing degree (stable radix sort: deterministic)
static cluster_status degree_order(cluster_ctx* c, int32_t* perm) {
  const int64_t n = c->n;
  cudaStream_t s = c->stream;
  uint32_t *deg = nullptr, *sdeg = nullptr;
  int32_t* iota = nullptr;
  void* tmp = nullptr;
  size_t tb = 0;
  cluster_status st = CLUSTER_OK;
  cudaError_t e;
  cub::DeviceRadixSort::SortPairsDescending(nullptr, tb, deg, sdeg, iota, perm, (int)n, 0, 32, s);
  if ((e = cudaMalloc(&deg, sizeof(uint32_t) * n)) != cudaSuccess ||
      (e = cudaMalloc(&sdeg, sizeof(uint32_t) * n)) != cudaSuccess ||
      (e = cudaMalloc(&iota, sizeof(int32_t) * n)) != cudaSuccess || (e = cudaMalloc(&tmp, tb)) != cudaSuccess) {
    set_error("degree order: %s", cudaGetErrorString(e));
    st = e == cudaErrorMemoryAllocation ? CLUSTER_ENOMEM : CLUSTER_ECUDA;
  } else {
    degree_kernel<<<grid_for(n), 256, 0, s>>>(c->rp, n, deg, iota);
    if ((e = cub::DeviceRadixSort::SortPairsDescending(tmp, tb, deg, sdeg, iota, perm, (int)n, 0, 32, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess) {
      set_error("degree order: %s", cudaGetErrorString(e));
      st = CLUSTER_ECUDA;
    }
  }
  void* fr[] = {deg, sdeg, iota, tmp};
  for (void* q : fr)
    if (q) cudaFree(q);
  return st;
}

static cluster_status build_schedule(cluster_ctx* c) {
  const int64_t n = c->n;
  cudaStream_t s = c->stream;
  uint32_t *deg = nullptr, *sdeg = nullptr;
  int32_t* iota = nullptr;
  void* tmp = nullptr;
  size_t tmp_bytes = 0, tmp2 = 0;
  int64_t *cost = nullptr, *prefix = nullptr, *hlo = nullptr;
  unsigned long long* cnt = nullptr;
  cluster_status st = CLUSTER_OK;
  auto fail = [&](cudaError_t e, const char* what) {
    set_error("%s: %s", what, cudaGetErrorString(e));
    st = e == cudaErrorMemoryAllocation ? CLUSTER_ENOMEM : CLUSTER_ECUDA;
  };
  cudaError_t e;
  do {
    if ((e = cudaMalloc(&deg, sizeof(uint32_t) * n)) != cudaSuccess) { fail(e, "alloc deg"); break; }
    if ((e = cudaMalloc(&sdeg, sizeof(uint32_t) * n)) != cudaSuccess) { fail(e, "alloc sdeg"); break; }
    if ((e = cudaMalloc(&iota, sizeof(int32_t) * n)) != cudaSuccess) { fail(e, "alloc iota"); break; }
    if ((e = cudaMalloc(&c->order, sizeof(int32_t) * n)) != cudaSuccess) { fail(e, "alloc order"); break; }
    degree_kernel<<<grid_for(n), 256, 0, s>>>(c->rp, n, deg, iota);
    // rows by degree, descending (stable radix sort: deterministic)
    cub::DeviceRadixSort::SortPairsDescending(nullptr, tmp_bytes, deg, sdeg, iota, c->order, (int)n, 0, 32, s);
    if ((e = cudaMalloc(&cost, sizeof(int64_t) * n)) != cudaSuccess) { fail(e, "alloc cost"); break; }
    if ((e = cudaMalloc(&prefix, sizeof(int64_t) * n)) != cudaSuccess) { fail(e, "alloc prefix"); break; }
    cub::DeviceScan::InclusiveSum(nullptr, tmp2, cost, prefix, (int)n, s);
    if (tmp2 > tmp_bytes) tmp_bytes = tmp2;
    if ((e = cudaMalloc(&tmp, tmp_bytes)) != cudaSuccess) { fail(e, "alloc sort temp"); break; }
    if ((e = cub::DeviceRadixSort::SortPairsDescending(tmp, tmp_bytes, deg, sdeg, iota, c->order, (int)n, 0, 32,
                                                       s)) != cudaSuccess) {
      fail(e, "degree sort");
      break;
    }
    // chunked ("heavy") rows: degree above H, split into chunks of H nonzeros
    if ((e = cudaMalloc(&cnt, sizeof(unsigned long long))) != cudaSuccess) { fail(e, "alloc cnt"); break; }
    cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s);
    count_above_kernel<<<grid_for(n), 256, 0, s>>>(sdeg, n, (uint32_t)c->heavy_H, cnt);
    unsigned long long nh = 0;
    cudaMemcpyAsync(&nh, cnt, sizeof(nh), cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { fail(e, "degree schedule"); break; }
    c->n_heavy = (int64_t)nh;
    // Rows below the chunk threshold: grouped by chunks of kRowChunk
    // consecutive rows (degree order kept inside a chunk, stable sort), so
    // that rows adjacent in S, whose col/val ranges share DRAM sectors, are
    // gathered at about the same time, while the teams of a warp still get
    // rows of similar degree.
    if ((int64_t)nh < n) {
      const int64_t m = n - (int64_t)nh;
      uint32_t *key = nullptr, *key2 = nullptr;
      int32_t* ord2 = nullptr;
      void* tmp3 = nullptr;
      size_t tb = 0;
      cub::DeviceRadixSort::SortPairs(nullptr, tb, key, key2, c->order + nh, ord2, (int)m, 0, 32, s);
      if ((e = cudaMalloc(&key, sizeof(uint32_t) * m)) != cudaSuccess ||
          (e = cudaMalloc(&key2, sizeof(uint32_t) * m)) != cudaSuccess ||
          (e = cudaMalloc(&ord2, sizeof(int32_t) * m)) != cudaSuccess || (e = cudaMalloc(&tmp3, tb)) != cudaSuccess) {
        fail(e, "alloc chunk order");
      } else {
        chunk_key_kernel<<<grid_for(m), 256, 0, s>>>(c->order + nh, m, kRowChunk, key);
        if ((e = cub::DeviceRadixSort::SortPairs(tmp3, tb, key, key2, c->order + nh, ord2, (int)m, 0, 32, s)) !=
            cudaSuccess)
          fail(e, "chunk order sort");
        else
          cudaMemcpyAsync(c->order + nh, ord2, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s);
        gather_deg_kernel<<<grid_for(n), 256, 0, s>>>(deg, c->order, n, sdeg);
      }
      cudaStreamSynchronize(s);
      void* fr[] = {key, key2, ord2, tmp3};
      for (void* q : fr)
        if (q) cudaFree(q);
      if (st != CLUSTER_OK) break;
    }
    if (nh > 0) {
      std::vector<uint32_t> hdeg(nh);
      std::vector<int64_t> hlo_h(nh);
      if ((e = cudaMalloc(&hlo, sizeof(int64_t) * nh)) != cudaSuccess) { fail(e, "alloc hlo"); break; }
      heavy_lo_kernel<<<grid_for((int64_t)nh), 256, 0, s>>>(c->rp, c->order, (int64_t)nh, hlo);
      cudaMemcpyAsync(hdeg.data(), sdeg, sizeof(uint32_t) * nh, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(hlo_h.data(), hlo, sizeof(int64_t) * nh, cudaMemcpyDeviceToHost, s);
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { fail(e, "heavy rows"); break; }
      std::vector<int64_t> cptr(nh + 1), ce0, ce1;
      cptr[0] = 0;
      for (size_t p = 0; p < nh; ++p) {
        const int64_t d = hdeg[p];
        for (int64_t o = 0; o < d; o += c->heavy_H) {
          ce0.push_back(hlo_h[p] + o);
          ce1.push_back(hlo_h[p] + std::min<int64_t>(d, o + c->heavy_H));
        }
        cptr[p + 1] = (int64_t)ce0.size();
        c->heavy_nnz += d;
      }
      c->n_chunks = (int64_t)ce0.size();
      if ((e = cudaMalloc(&c->chunk_ptr, sizeof(int64_t) * (nh + 1))) != cudaSuccess) { fail(e, "alloc chunks"); break; }
      if ((e = cudaMalloc(&c->chunk_e0, sizeof(int64_t) * c->n_chunks)) != cudaSuccess) { fail(e, "alloc chunks"); break; }
      if ((e = cudaMalloc(&c->chunk_e1, sizeof(int64_t) * c->n_chunks)) != cudaSuccess) { fail(e, "alloc chunks"); break; }
      if ((e = cudaMalloc(&c->hv_part, sizeof(float) * c->n_chunks * c->KP)) != cudaSuccess) { fail(e, "alloc hv"); break; }
      cudaMemcpyAsync(c->chunk_ptr, cptr.data(), sizeof(int64_t) * (nh + 1), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(c->chunk_e0, ce0.data(), sizeof(int64_t) * c->n_chunks, cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(c->chunk_e1, ce1.data(), sizeof(int64_t) * c->n_chunks, cudaMemcpyHostToDevice, s);
      if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { fail(e, "upload chunks"); break; }
    }
    // cost-balanced position ranges, one per block
    cost_kernel<<<grid_for(n), 256, 0, s>>>(sdeg, n, c->n_heavy, (uint32_t)c->heavy_H, c->row_cost, cost);
    if ((e = cub::DeviceScan::InclusiveSum(tmp, tmp_bytes, cost, prefix, (int)n, s)) != cudaSuccess) {
      fail(e, "cost scan");
      break;
    }
    if ((e = cudaMalloc(&c->cta_pos, sizeof(int64_t) * (c->parts + 1))) != cudaSuccess) { fail(e, "alloc cta_pos"); break; }
    partition_kernel<<<(c->parts + 1 + 255) / 256, 256, 0, s>>>(prefix, n, c->parts, c->cta_pos);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { fail(e, "partition"); break; }
    if ((e = cudaGetLastError()) != cudaSuccess) { fail(e, "schedule kernels"); break; }
  } while (0);
  void* tmps[] = {deg, sdeg, iota, tmp, cost, prefix, hlo, cnt};
  for (void* p : tmps)
    if (p) cudaFree(p);
  return st;
}

// Internal numbering by decreasing degree (stable): internal row p is the
// caller's row perm[p].  The context keeps its own relabelled copy of S (row
// pointers, renamed columns, values; each row's entries in their original
// order, so every row's sum is unchanged) and frees any copy it owned before.
static cluster_status relabel_csr(cluster_ctx* c) {
  const int64_t n = c->n, nnz = c->nnz;
  cudaStream_t s = c->stream;
  FC_CUDA(cudaMalloc(&c->perm, sizeof(int32_t) * n));
  FC_CUDA(cudaMalloc(&c->inv, sizeof(int32_t) * n));
  FC_TRY(degree_order(c, c->perm));
  inverse_perm_kernel<<<grid_for(n), 256, 0, s>>>(c->perm, n, c->inv);
  int64_t *cnt = nullptr, *rp2 = nullptr;
  int32_t* col2 = nullptr;
  float* val2 = nullptr;
  void* tmp = nullptr;
  size_t tb = 0;
  cluster_status st = CLUSTER_OK;
  do {
    cudaError_t e;
    cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt, rp2, (int)(n + 1), s);
    if ((e = cudaMalloc(&cnt, sizeof(int64_t) * (n + 1))) != cudaSuccess ||
        (e = cudaMalloc(&rp2, sizeof(int64_t) * (n + 1))) != cudaSuccess ||
        (e = cudaMalloc(&col2, sizeof(int32_t) * std::max<int64_t>(1, nnz))) != cudaSuccess ||
        (e = cudaMalloc(&val2, sizeof(float) * std::max<int64_t>(1, nnz))) != cudaSuccess ||
        (e = cudaMalloc(&tmp, tb)) != cudaSuccess) {
      set_error("relabel: %s", cudaGetErrorString(e));
      st = e == cudaErrorMemoryAllocation ? CLUSTER_ENOMEM : CLUSTER_ECUDA;
      break;
    }
    permuted_count_kernel<<<grid_for(n + 1), 256, 0, s>>>(c->rp, c->perm, n, cnt);
    if ((e = cub::DeviceScan::ExclusiveSum(tmp, tb, cnt, rp2, (int)(n + 1), s)) != cudaSuccess) {
      set_error("relabel scan: %s", cudaGetErrorString(e));
      st = CLUSTER_ECUDA;
      break;
    }
    relabel_rows_kernel<<<grid_for(n * 32), 256, 0, s>>>(c->rp, c->col, c->val, c->perm, c->inv, rp2, n, col2,
                                                          val2);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) {
      set_error("relabel: %s", cudaGetErrorString(e));
      st = CLUSTER_ECUDA;
      break;
    }
  } while (0);
  if (cnt) cudaFree(cnt);
  if (tmp) cudaFree(tmp);
  if (st != CLUSTER_OK) {
    if (rp2) cudaFree(rp2);
    if (col2) cudaFree(col2);
    if (val2) cudaFree(val2);
    return st;
  }
  void* old[] = {c->rp_owned, c->col_owned, c->val_owned};
  for (void* q : old)
    if (q) cudaFree(q);
  c->rp = c->rp_owned = rp2;
  c->col = c->col_owned = col2;
  c->val = c->val_owned = val2;
  c->relabeled = true;
  return CLUSTER_OK;
}

}  // namespace fc
