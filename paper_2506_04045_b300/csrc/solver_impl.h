// Solver context (opaque to callers of cluster.h).
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/cluster.h"
#include "pass_kernels.cuh"
#include "state.h"

namespace fc {
struct StreamMaps;
}

struct cluster_ctx {
  int dev = 0;
  cudaStream_t stream = nullptr;      // caller's stream
  cudaStream_t cap_stream = nullptr;  // private stream used only to capture the graph
  cluster_options opt{};
  int64_t n = 0, nnz = 0;
  int k = 0, KP = 0;
  bool mixed = false;
  // S (int64 row pointers; col/val borrowed or owned)
  const int64_t* rp = nullptr;
  const int32_t* col = nullptr;
  const float* val = nullptr;
  int64_t* rp_owned = nullptr;
  int32_t* col_owned = nullptr;
  float* val_owned = nullptr;
  __nv_bfloat16* val16 = nullptr;
  // internal numbering (opt.relabel): internal row p is the caller's row
  // perm[p]; inv is the inverse (caller's row i -> internal row inv[i])
  bool relabeled = false;
  int32_t* perm = nullptr;
  int32_t* inv = nullptr;
  // schedule: rows by degree, cost-balanced block ranges, chunked rows
  int32_t* order = nullptr;
  int64_t* cta_pos = nullptr;
  int parts = 1;
  int heavy_grid = 1;
  int64_t heavy_H = 512;
  int64_t row_cost = 6;
  int64_t n_heavy = 0, n_chunks = 0, heavy_nnz = 0;
  int64_t* chunk_ptr = nullptr;
  int64_t* chunk_e0 = nullptr;
  int64_t* chunk_e1 = nullptr;
  float* hv_part = nullptr;
  // iterate state
  float* X[2] = {nullptr, nullptr};
  __nv_bfloat16* XS[2] = {nullptr, nullptr};
  float* Zp = nullptr;                  // fused iteration: stored product S Xbar^{n-1}
  float* Z[2] = {nullptr, nullptr};     // split iteration: S Xbar^j in Z[(j+1)&1]
  unsigned long long* work = nullptr;   // split iteration: gather kernel work counter
  bool split = true;
  int parts_upd = 1;                    // blocks (and partial slots) of the update kernel
  bool tc_update = true;                // update on tcgen05 where the kernel exists (k <= 32)
  // streaming update (tc_stream.cuh, KP = 32): one CTA per SM over 128-row
  // tiles loaded by TMA through these tensor maps of X[0..1], Z[0..1]
  bool stream_update = false;
  int stream_grid = 0;
  fc::StreamMaps* smaps = nullptr;
  int spmm_grid = 1;
  int spmm_rpu = 4;                     // rows per team per gather unit (4 or 1)
  // overlapped pass (opt.overlap): row chunk c's update runs on side_stream
  // once the gather units that cover its rows (ovl_units[c+1]) are done, while
  // the next chunks are gathered; the update blocks and partial slots are the
  // unchunked launch's (ovl_blocks), so no value changes
  static constexpr int kMaxOvl = 8;
  int ovl = 0;                          // chunks (0: one gather and one update launch)
  bool ovl_eligible = false;            // relabeled, identity gather order, n >= kOvlMinRows
  int spmm_grid_ovl = 1;                // gather grid beside one update block per SM
  int n_work = 1;                       // gather work counters in use (one per gather launch)
  int64_t ovl_units[kMaxOvl + 1] = {};
  int ovl_blocks[kMaxOvl + 1] = {};
  cudaStream_t side_stream = nullptr;
  cudaEvent_t ovl_ev[kMaxOvl + 1] = {};
  double* bpart = nullptr;            // fold block partials (fold_kernel of an iteration)
  double* A[2] = {nullptr, nullptr};  // float64 fold scratch: Gram of Xbar^n, Gram of Y^{n+1}
  float* Gy = nullptr;                 // float32 G(Y) (minus its mean) read by the next pass
  float* gram_part = nullptr;
  double* sc_part = nullptr;
  fc::FistaState* st = nullptr;
  fc::FistaState host_st{};
  // graphs of graph_chunk passes, one per parity of the first pass (the
  // gather's L2 window follows the iterate buffer it reads)
  int graph_chunk = 16;
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  int64_t pass_guess = 0;       // the device's pass counter as the host expects it
  size_t l2_window_bytes = 0;   // persisting window over the first rows of the gathered copy (0 = none)
};

namespace fc {
// Internals shared by the solver and the batched engine (solver.cu).
cluster_status init_impl(const cluster_csr* S, int32_t k, const float* U0, const cluster_options* opt, void* stream,
                         cluster_ctx* c, bool capture);
void ctx_free(cluster_ctx* c);
PassArgs make_pass_args(const cluster_ctx* c, bool eval_exact);
FoldArgs make_fold_args(const cluster_ctx* c, int eval, int eval_init);
cluster_status read_state(cluster_ctx* c);
void fill_report(const cluster_ctx* c, cluster_report* rep);
cluster_status finalize_loss(cluster_ctx* c);  // make the report's f the loss of the output iterate
// U_out (n x k, the caller's numbering) from an internal n x KP iterate
void unpad_output(const cluster_ctx* c, const float* X, float* U_out, cudaStream_t s);
int grid_for(int64_t work, int threads = 256);

// Non-owning batch over instances owned by the caller (batch.cu).
cluster_status batch_view_new(void* stream, int graph_chunk, cluster_batch** out);
cluster_status batch_view_set(cluster_batch* b, const std::vector<cluster_ctx*>& members);
cluster_status batch_view_run(cluster_batch* b, int64_t iters);  // advance and read every member's state
void batch_view_delete(cluster_batch* b);
}  // namespace fc
