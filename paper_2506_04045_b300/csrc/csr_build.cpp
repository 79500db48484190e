// Host construction of the symmetric similarity matrix from an edge list
// (Example 4.1: s_ij = 1 if article i cites or is cited by article j, plus a
// unit diagonal), generalised to weights: repeated pairs keep the largest
// weight.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <utility>
#include <vector>

#include "util.h"

extern "C" CLUSTER_API cluster_status cluster_csr_from_edges(int64_t n, int64_t m, const int64_t* src,
                                                             const int64_t* dst, const float* w,
                                                             int32_t add_unit_diag, cluster_csr* out) {
  fc::clear_error();
  if (!out) FC_EINVAL("cluster_csr_from_edges: out is NULL");
  memset(out, 0, sizeof(*out));
  if (n < 0 || m < 0) FC_EINVAL("cluster_csr_from_edges: negative size");
  if (m > 0 && (!src || !dst)) FC_EINVAL("cluster_csr_from_edges: NULL edge arrays");
  if (n > (int64_t)0x7fffffff) FC_EINVAL("cluster_csr_from_edges: n exceeds int32 column range");
  for (int64_t e = 0; e < m; ++e) {
    if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n)
      FC_EINVAL("cluster_csr_from_edges: edge %lld endpoint out of range", (long long)e);
    if (w && !std::isfinite(w[e])) FC_EINVAL("cluster_csr_from_edges: weight %lld not finite", (long long)e);
  }
  // (key = row * n + col, weight) for both directions of every edge
  std::vector<std::pair<int64_t, float>> ent;
  try {
    ent.reserve((size_t)(2 * m + (add_unit_diag ? n : 0)));
  } catch (...) {
    fc::set_error("cluster_csr_from_edges: out of host memory");
    return CLUSTER_ENOMEM;
  }
  for (int64_t e = 0; e < m; ++e) {
    const int64_t a = src[e], b = dst[e];
    const float we = w ? w[e] : 1.0f;
    if (a == b) {
      if (!add_unit_diag) ent.emplace_back(a * n + a, we);
      continue;
    }
    ent.emplace_back(a * n + b, we);
    ent.emplace_back(b * n + a, we);
  }
  if (add_unit_diag)
    for (int64_t i = 0; i < n; ++i) ent.emplace_back(i * n + i, 1.0f);
  std::sort(ent.begin(), ent.end(),
            [](const std::pair<int64_t, float>& x, const std::pair<int64_t, float>& y) { return x.first < y.first; });
  // merge equal keys with max
  size_t u = 0;
  for (size_t i = 0; i < ent.size(); ++i) {
    if (u > 0 && ent[u - 1].first == ent[i].first) {
      ent[u - 1].second = std::max(ent[u - 1].second, ent[i].second);
    } else {
      ent[u++] = ent[i];
    }
  }
  ent.resize(u);
  int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (u ? u : 1));
  float* val = (float*)malloc(sizeof(float) * (u ? u : 1));
  if (!rp || !col || !val) {
    free(rp);
    free(col);
    free(val);
    fc::set_error("cluster_csr_from_edges: out of host memory");
    return CLUSTER_ENOMEM;
  }
  memset(rp, 0, sizeof(int64_t) * (size_t)(n + 1));
  for (size_t i = 0; i < u; ++i) {
    const int64_t r = ent[i].first / n;
    col[i] = (int32_t)(ent[i].first % n);
    val[i] = ent[i].second;
    rp[r + 1] += 1;
  }
  for (int64_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  out->n = n;
  out->nnz = (int64_t)u;
  out->index64 = 1;
  out->row_ptr = rp;
  out->col = col;
  out->val = val;
  return CLUSTER_OK;
}

extern "C" CLUSTER_API void cluster_csr_free(cluster_csr* csr) {
  if (!csr) return;
  free(const_cast<void*>(csr->row_ptr));
  free(const_cast<int32_t*>(csr->col));
  free(const_cast<float*>(csr->val));
  memset(csr, 0, sizeof(*csr));
}
