// C ABI of the fuzzy-clustering solver: context set-up, the per-iteration
// launch sequence captured in CUDA graphs, reports, checkpoints and the
// standalone objective.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cub/cub.cuh>
#include <cudaTypedefs.h>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "init_kernels.cuh"
#include "pass_kernels.cuh"
#include "tc_update.cuh"
#include "tc_stream.cuh"
#include "hessian_kernels.cuh"
#include "solver_impl.h"
#include "util.h"
#include "schedule.cuh"

namespace fc {

static thread_local std::string g_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
}
void clear_error() { g_err.clear(); }

static int padded_k(int k) {
  int kp = 2;
  while (kp < k) kp <<= 1;
  return kp;
}

int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 65535LL * 8) b = 65535LL * 8;
  return (int)b;
}

// ---------------------------------------------------------------------------
// per-KP dispatch
// ---------------------------------------------------------------------------
template <int KP>
struct KPOps {
  using L = Lay<KP>;
  static int rows_per_tile() { return L::R; }
  static int fold_nb() { return fold_blocks<KP>(false); }

  template <bool MIXED, bool EVAL>
  static cudaError_t setup_pass_attr() {
    const size_t smem = pass_smem_bytes<KP>(EVAL);
    return cudaFuncSetAttribute(fista_pass_kernel<KP, MIXED, EVAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem);
  }
  static cudaError_t setup_attrs() {
    cudaError_t e;
    if ((e = setup_pass_attr<false, false>()) != cudaSuccess) return e;
    if ((e = setup_pass_attr<true, false>()) != cudaSuccess) return e;
    if ((e = setup_pass_attr<false, true>()) != cudaSuccess) return e;
    return cudaSuccess;
  }
  static int occupancy(bool mixed) {
    int occ = 0;
    const size_t smem = pass_smem_bytes<KP>(false);
    if (mixed)
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fista_pass_kernel<KP, true, false>, L::NT, smem);
    else
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fista_pass_kernel<KP, false, false>, L::NT, smem);
    return occ < 1 ? 1 : occ;
  }
  static void launch_pass(const PassArgs& a, int grid, bool mixed, cudaStream_t s, const LaunchOpt& o) {
    const size_t smem = pass_smem_bytes<KP>(false);
    launch_ex(mixed ? fista_pass_kernel<KP, true, false> : fista_pass_kernel<KP, false, false>, grid, L::NT, smem, s,
              o, a);
  }
  static void launch_eval(const PassArgs& a, int grid, cudaStream_t s) {
    fista_pass_kernel<KP, false, true><<<grid, L::NT, pass_smem_bytes<KP>(true), s>>>(a);
  }
  static void launch_heavy(const PassArgs& a, int grid, bool mixed, bool eval, cudaStream_t s, const LaunchOpt& o) {
    launch_ex(eval ? heavy_kernel<KP, false, true> : mixed ? heavy_kernel<KP, true, false> : heavy_kernel<KP, false, false>,
              grid, L::NT, 0, s, o, a);
  }
  // first gather unit whose rows all lie at positions >= r (units: chunk units
  // of hub rows, then row units of TPW * kRowsPerUnit positions from n_heavy)
  static int64_t unit_of_position(bool mixed, int64_t r, int64_t n_heavy, int64_t n_chunks) {
    const int64_t cu = mixed ? spmm_chunk_units<KP, true>(n_chunks) : spmm_chunk_units<KP, false>(n_chunks);
    const int64_t per = (int64_t)(mixed ? WLay<KP, true>::TPW : WLay<KP, false>::TPW) * kRowsPerUnit;
    const int64_t q = std::max<int64_t>(r, n_heavy) - n_heavy;
    return cu + (q + per - 1) / per;
  }
  static int64_t units(bool mixed, int64_t n, int64_t n_heavy, int64_t n_chunks, int rpu) {
    if (rpu == 1)
      return mixed ? spmm_units<KP, true, 1>(n, n_heavy, n_chunks) : spmm_units<KP, false, 1>(n, n_heavy, n_chunks);
    return mixed ? spmm_units<KP, true>(n, n_heavy, n_chunks) : spmm_units<KP, false>(n, n_heavy, n_chunks);
  }
  static int occ_spmm(bool mixed) {
    int occ = 0;
    if (mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spmm_kernel<KP, true>, L::NT, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, spmm_kernel<KP, false>, L::NT, 0);
    return occ < 1 ? 1 : occ;
  }
  // k <= 32: the tcgen05 update (tc_update.cuh) unless tc is false; otherwise
  // the warp-level one
  static int occ_update(bool mixed, bool tc) {
    int occ = 0;
    if constexpr (TcUpd<KP>::ON) {
      if (tc) {
        const void* fn = mixed ? (const void*)update_tc_kernel<KP, true> : (const void*)update_tc_kernel<KP, false>;
        return tc_blocks_per_sm(fn, L::NT, TcUpd<KP>::smem(), TcUpd<KP>::TMEM_COLS);
      }
    }
    const size_t smem = update_smem_bytes<KP>();
    if (mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, update_kernel<KP, true>, L::NT, smem);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, update_kernel<KP, false>, L::NT, smem);
    return occ < 1 ? 1 : occ;
  }
  static cudaError_t setup_update_attr() {
    if constexpr (TcUpd<KP>::ON) {
      const int smem = (int)TcUpd<KP>::smem();
      cudaError_t e = cudaFuncSetAttribute(update_tc_kernel<KP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
      e = cudaFuncSetAttribute(update_tc_kernel<KP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      if (e != cudaSuccess) return e;
    }
    const int smem = (int)update_smem_bytes<KP>();
    cudaError_t e = cudaFuncSetAttribute(update_kernel<KP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(update_kernel<KP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  }
  // o.win_bytes > 0: with a persisting L2 window (the gathered iterate's hot rows)
  // rpu: rows per team per gather unit (kRowsPerUnit or 1)
  static void launch_spmm(const PassArgs& a, int grid, bool mixed, int rpu, cudaStream_t s, const LaunchOpt& o) {
    if (rpu == 1) launch_ex(mixed ? spmm_kernel<KP, true, 1> : spmm_kernel<KP, false, 1>, grid, L::NT, 0, s, o, a);
    else launch_ex(mixed ? spmm_kernel<KP, true> : spmm_kernel<KP, false>, grid, L::NT, 0, s, o, a);
  }
  static void launch_finalize(const PassArgs& a, cudaStream_t s, const LaunchOpt& o) {
    const int64_t threads = a.n_heavy * L::T;
    int grid = (int)std::min<int64_t>((threads + 255) / 256, 4096);
    launch_ex(heavy_finalize_kernel<KP>, grid < 1 ? 1 : grid, 256, 0, s, o, a);
  }
  static void launch_update(const PassArgs& a, int grid, bool mixed, bool tc, cudaStream_t s, const LaunchOpt& o) {
    if constexpr (TcUpd<KP>::ON) {
      if (tc) {
        launch_ex(mixed ? update_tc_kernel<KP, true> : update_tc_kernel<KP, false>, grid, L::NT, TcUpd<KP>::smem(), s,
                  o, a);
        return;
      }
    }
    launch_ex(mixed ? update_kernel<KP, true> : update_kernel<KP, false>, grid, L::NT, update_smem_bytes<KP>(), s, o,
              a);
  }
  static void launch_gram0(const float* X, int64_t n, float* gp, double* sp, int grid, cudaStream_t s) {
    if constexpr (KP <= 64) gram0_kernel<KP><<<grid, 256, 0, s>>>(X, n, gp, sp);
  }
  static int occ_gram0() {
    int occ = 1;
    if constexpr (KP <= 64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gram0_kernel<KP>, 256, 0);
    return occ < 1 ? 1 : occ;
  }
  static void launch_fold(const FoldArgs& f, cudaStream_t s, const LaunchOpt& o) {
    const int nent = f.eval ? KP * KP : 2 * KP * KP;
    launch_ex(fold_kernel<KP>, (nent + fold_epb<KP>() - 1) / fold_epb<KP>(), 256, 0, s, o, f);
  }
};

#define FC_DISPATCH(KPV, CALL)                        \
  switch (KPV) {                                      \
    case 2: { using Ops = KPOps<2>; CALL; } break;    \
    case 4: { using Ops = KPOps<4>; CALL; } break;    \
    case 8: { using Ops = KPOps<8>; CALL; } break;    \
    case 16: { using Ops = KPOps<16>; CALL; } break;  \
    case 32: { using Ops = KPOps<32>; CALL; } break;  \
    case 64: { using Ops = KPOps<64>; CALL; } break;  \
    default: { using Ops = KPOps<128>; CALL; } break; \
  }

static int kp_rows_per_tile(int KP) {
  int r = 1;
  FC_DISPATCH(KP, r = Ops::rows_per_tile());
  return r;
}
static cudaError_t kp_setup_attrs(int KP) {
  cudaError_t e = cudaSuccess;
  FC_DISPATCH(KP, e = Ops::setup_attrs());
  return e;
}
static int kp_occupancy(int KP, bool mixed) {
  int o = 1;
  FC_DISPATCH(KP, o = Ops::occupancy(mixed));
  return o;
}
static void kp_launch_pass(int KP, const PassArgs& a, int grid, bool mixed, cudaStream_t s,
                           const LaunchOpt& o = LaunchOpt()) {
  FC_DISPATCH(KP, Ops::launch_pass(a, grid, mixed, s, o));
}
static void kp_launch_eval(int KP, const PassArgs& a, int grid, cudaStream_t s) {
  FC_DISPATCH(KP, Ops::launch_eval(a, grid, s));
}
static void kp_launch_heavy(int KP, const PassArgs& a, int grid, bool mixed, bool eval, cudaStream_t s,
                            const LaunchOpt& o = LaunchOpt()) {
  FC_DISPATCH(KP, Ops::launch_heavy(a, grid, mixed, eval, s, o));
}
static void kp_launch_fold(int KP, const FoldArgs& f, cudaStream_t s, const LaunchOpt& o = LaunchOpt()) {
  FC_DISPATCH(KP, Ops::launch_fold(f, s, o));
}
static int kp_fold_blocks(int KP) {
  int nb = 1;
  FC_DISPATCH(KP, nb = Ops::fold_nb());
  return nb;
}
static int kp_occ_gram0(int KP) {
  int o = 1;
  FC_DISPATCH(KP, o = Ops::occ_gram0());
  return o;
}
static void kp_launch_gram0(int KP, const float* X, int64_t n, float* gp, double* sp, int grid, cudaStream_t s) {
  FC_DISPATCH(KP, Ops::launch_gram0(X, n, gp, sp, grid, s));
}
static int64_t kp_unit_of_position(int KP, bool mixed, int64_t r, int64_t n_heavy, int64_t n_chunks) {
  int64_t u = 0;
  FC_DISPATCH(KP, u = Ops::unit_of_position(mixed, r, n_heavy, n_chunks));
  return u;
}
static int64_t kp_units(int KP, bool mixed, int64_t n, int64_t n_heavy, int64_t n_chunks, int rpu = kRowsPerUnit) {
  int64_t u = 0;
  FC_DISPATCH(KP, u = Ops::units(mixed, n, n_heavy, n_chunks, rpu));
  return u;
}
static int kp_occ_spmm(int KP, bool mixed) {
  int o = 1;
  FC_DISPATCH(KP, o = Ops::occ_spmm(mixed));
  return o;
}
static int kp_occ_update(int KP, bool mixed, bool tc) {
  int o = 1;
  FC_DISPATCH(KP, o = Ops::occ_update(mixed, tc));
  return o;
}
static cudaError_t kp_setup_update_attr(int KP) {
  cudaError_t e = cudaSuccess;
  FC_DISPATCH(KP, e = Ops::setup_update_attr());
  return e;
}
static void kp_launch_spmm(int KP, const PassArgs& a, int grid, bool mixed, cudaStream_t s,
                           const LaunchOpt& o = LaunchOpt(), int rpu = kRowsPerUnit) {
  FC_DISPATCH(KP, Ops::launch_spmm(a, grid, mixed, rpu, s, o));
}
static void kp_launch_finalize(int KP, const PassArgs& a, cudaStream_t s, const LaunchOpt& o = LaunchOpt()) {
  FC_DISPATCH(KP, Ops::launch_finalize(a, s, o));
}
static void kp_launch_update(int KP, const PassArgs& a, int grid, bool mixed, bool tc, cudaStream_t s,
                             const LaunchOpt& o = LaunchOpt()) {
  FC_DISPATCH(KP, Ops::launch_update(a, grid, mixed, tc, s, o));
}

// ---- streaming update (tc_stream.cuh) ----
static cudaError_t stream_setup_attr() {
  const void* fns[4] = {(const void*)update_stream_kernel<false, false>, (const void*)update_stream_kernel<false, true>,
                        (const void*)update_stream_kernel<true, false>, (const void*)update_stream_kernel<true, true>};
  for (const void* fn : fns) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ts::SMEM);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Tensor maps of the iterate and product buffers (n x 32 float32): boxes of
// 32 x 128 rows with 128-byte swizzle; rows at or beyond n read as zero.
static cluster_status make_stream_maps(cluster_ctx* c) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  if (!encode) {
    set_error("streaming update: the driver's cuTensorMapEncodeTiled is unavailable");
    return CLUSTER_ECUDA;
  }
  c->smaps = new (std::nothrow) StreamMaps;
  if (!c->smaps) {
    set_error("streaming update: host allocation failed");
    return CLUSTER_ENOMEM;
  }
  float* bufs[4] = {c->X[0], c->X[1], c->Z[0], c->Z[1]};
  CUtensorMap* maps[4] = {&c->smaps->X[0], &c->smaps->X[1], &c->smaps->Z[0], &c->smaps->Z[1]};
  const cuuint64_t dims[2] = {32, (cuuint64_t)c->n};
  const cuuint64_t strides[1] = {32 * sizeof(float)};
  const cuuint32_t box[2] = {32, (cuuint32_t)ts::R};
  const cuuint32_t estr[2] = {1, 1};
  for (int i = 0; i < 4; ++i) {
    const CUresult r = encode(maps[i], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, bufs[i], dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error("streaming update: cuTensorMapEncodeTiled failed (%d)", (int)r);
      return CLUSTER_ECUDA;
    }
  }
  return CLUSTER_OK;
}

// the row-local update of a split pass with the context's engine
static void launch_update_ctx(const cluster_ctx* c, const PassArgs& a, cudaStream_t s,
                              const LaunchOpt& o = LaunchOpt()) {
  if (c->stream_update) {
    const bool full = c->k == 32;
    auto fn = c->mixed ? (full ? update_stream_kernel<true, true> : update_stream_kernel<true, false>)
                       : (full ? update_stream_kernel<false, true> : update_stream_kernel<false, false>);
    launch_ex(fn, c->stream_grid, ts::NT, ts::SMEM, s, o, a, *c->smaps);
  } else {
    kp_launch_update(c->KP, a, c->parts_upd, c->mixed, c->tc_update, s, o);
  }
}

__global__ void set_limit_kernel(FistaState* st, int64_t iters) { st->limit = st->pass + iters; }

// ---------------------------------------------------------------------------
// CSR preparation shared by the solver and the standalone objective
// ---------------------------------------------------------------------------
static cluster_status prepare_rowptr(const cluster_csr* S, cudaStream_t s, const int64_t** rp_out,
                                     int64_t** owned) {
  *owned = nullptr;
  if (S->index64) {
    *rp_out = reinterpret_cast<const int64_t*>(S->row_ptr);
    return CLUSTER_OK;
  }
  int64_t* rp = nullptr;
  FC_CUDA(cudaMalloc(&rp, sizeof(int64_t) * (S->n + 1)));
  rowptr32_to_64<<<grid_for(S->n + 1), 256, 0, s>>>(reinterpret_cast<const int32_t*>(S->row_ptr), rp, S->n + 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    cudaFree(rp);
    set_error("row_ptr conversion failed: %s", cudaGetErrorString(e));
    return CLUSTER_ECUDA;
  }
  *owned = rp;
  *rp_out = rp;
  return CLUSTER_OK;
}

static cluster_status check_csr_args(const cluster_csr* S, int32_t k) {
  if (!S) FC_EINVAL("S is NULL");
  if (S->n < 1) FC_EINVAL("n must be >= 1 (got %lld)", (long long)S->n);
  if (S->n > 0x7fffffffLL) FC_EINVAL("n exceeds the int32 column range");
  if (S->nnz < 0) FC_EINVAL("nnz must be >= 0");
  if (k < 1 || k > 128) FC_EINVAL("k must be in [1, 128] (got %d)", k);
  if (!S->row_ptr) FC_EINVAL("row_ptr is NULL");
  if (S->nnz > 0 && (!S->col || !S->val)) FC_EINVAL("col/val are NULL");
  return CLUSTER_OK;
}

// ---------------------------------------------------------------------------
// context helpers
// ---------------------------------------------------------------------------
// The persisting L2 set-aside is a limit of the process's CUDA context,
// shared by all solvers: raised while at least one solver with a window
// lives, restored (and persisting lines reset) when the last one goes.
static std::mutex g_l2_mu;
static int g_l2_users = 0;
static size_t g_l2_saved = 0;

static cluster_status l2_setaside_acquire(size_t bytes) {
  std::lock_guard<std::mutex> lk(g_l2_mu);
  size_t cur = 0;
  FC_CUDA(cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize));
  if (g_l2_users == 0) g_l2_saved = cur;
  if (cur < bytes) FC_CUDA(cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, bytes));
  ++g_l2_users;
  return CLUSTER_OK;
}

static void l2_setaside_release() {
  std::lock_guard<std::mutex> lk(g_l2_mu);
  if (g_l2_users > 0 && --g_l2_users == 0) {
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_l2_saved);
  }
}

// update blocks: at least this many tiles each (see init_impl)
static const int64_t kMinTilesPerBlock = 32;
// overlapped pass: minimum rows, and update blocks per resident update block
static const int64_t kOvlMinRows = 1 << 20;
// update_engine 0 takes the streaming update for solvers of at least this many
// articles (a persistent grid of one CTA per SM needs a few tiles per CTA)
static const int64_t kStreamMinRows = 1 << 17;
static const int kOvlBlockFactor = 4;

void ctx_free(cluster_ctx* c) {
  if (!c) return;
  delete c->smaps;
  for (cudaGraphExec_t g : c->graph_exec)
    if (g) cudaGraphExecDestroy(g);
  if (c->l2_window_bytes) l2_setaside_release();
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->side_stream) cudaStreamDestroy(c->side_stream);
  for (cudaEvent_t e : c->ovl_ev)
    if (e) cudaEventDestroy(e);
  void* bufs[] = {c->rp_owned, c->col_owned, c->val_owned, c->val16, c->order, c->cta_pos, c->chunk_ptr,
                  c->chunk_e0, c->chunk_e1, c->hv_part, c->X[0], c->X[1], c->XS[0], c->XS[1], c->Zp, c->A[0],
                  c->A[1], c->Gy, c->bpart, c->gram_part, c->sc_part, c->st, c->Z[0], c->Z[1], c->work, c->perm, c->inv};
  for (void* p : bufs)
    if (p) cudaFree(p);
  delete c;
}

PassArgs make_pass_args(const cluster_ctx* c, bool eval_exact) {
  PassArgs a;
  memset(&a, 0, sizeof(a));
  a.row_ptr = c->rp;
  a.col = c->col;
  a.val = (c->mixed && !eval_exact) ? (const void*)c->val16 : (const void*)c->val;
  a.order = c->order;
  a.cta_pos = c->cta_pos;
  a.n_heavy = c->n_heavy;
  a.chunk_ptr = c->chunk_ptr;
  a.chunk_e0 = c->chunk_e0;
  a.chunk_e1 = c->chunk_e1;
  a.n_chunks = c->n_chunks;
  a.hv_part = c->hv_part;
  a.X0 = c->X[0];
  a.X1 = c->X[1];
  a.XS0 = c->XS[0];
  a.XS1 = c->XS[1];
  a.Zp = c->Zp;
  a.Z0 = c->Z[0];
  a.Z1 = c->Z[1];
  a.work = c->work;
  a.unit_lo = 0;
  a.unit_hi = -1;
  a.upd_block0 = 0;
  a.upd_parts = 0;
  a.Gy = c->Gy;
  a.gram_part = c->gram_part;
  a.sc_part = c->sc_part;
  a.st = c->st;
  a.n = c->n;
  a.k = c->k;
  a.eval_sel = 0;
  return a;
}

FoldArgs make_fold_args(const cluster_ctx* c, int eval, int eval_init) {
  FoldArgs f;
  memset(&f, 0, sizeof(f));
  f.st = c->st;
  f.gram_part = c->gram_part;
  f.sc_part = c->sc_part;
  f.parts = (!eval && c->split) ? c->parts_upd : c->parts;
  f.work = (!eval && c->split) ? c->work : nullptr;
  f.n_work = (!eval && c->split) ? c->n_work : 0;
  f.eval = eval;
  f.eval_init = eval_init;
  f.A = c->A[0];
  f.G = c->A[1];
  f.Gy = c->Gy;
  f.bpart = c->bpart;
  return f;
}

// Enqueue one iteration (heavy chunks, fused pass, fold).
// One pass; `parity` is the pass counter's parity when it runs (it selects
// the iterate buffer the gather reads and so the L2 window).
// Overlapped split pass: gather chunk ch on s (hub-row sums after the first),
// then the update of row chunk ch on the side stream, which waits only for
// the gathers so far; the caller's stream waits for the last update.
// tev (profiling, may be null): [0], [1] after the last gather, [2] after the join.
static void enqueue_split_ovl(const cluster_ctx* c, cudaStream_t s, int parity, cudaEvent_t* tev) {
  const PassArgs a = make_pass_args(c, false);
  void* win = c->mixed ? (void*)c->XS[parity & 1] : (void*)c->X[parity & 1];
  for (int ch = 0; ch < c->ovl; ++ch) {
    PassArgs g = a;
    g.unit_lo = c->ovl_units[ch];
    g.unit_hi = c->ovl_units[ch + 1];
    g.work = c->work + ch;
    if (g.unit_hi > g.unit_lo) {
      LaunchOpt o;
      o.win = win;
      o.win_bytes = c->l2_window_bytes;
      kp_launch_spmm(c->KP, g, c->spmm_grid_ovl, c->mixed, s, o);
    }
    if (ch == 0 && c->n_heavy > 0) kp_launch_finalize(c->KP, a, s);
    if (tev && ch + 1 == c->ovl) {
      cudaEventRecord(tev[0], s);
      cudaEventRecord(tev[1], s);
    }
    cudaEventRecord(c->ovl_ev[ch], s);
    cudaStreamWaitEvent(c->side_stream, c->ovl_ev[ch], 0);
    PassArgs u = a;
    u.upd_block0 = c->ovl_blocks[ch];
    u.upd_parts = c->parts_upd;
    const int nb = c->ovl_blocks[ch + 1] - c->ovl_blocks[ch];
    if (nb > 0) kp_launch_update(c->KP, u, nb, c->mixed, c->tc_update, c->side_stream);
  }
  cudaEventRecord(c->ovl_ev[c->ovl], c->side_stream);
  cudaStreamWaitEvent(s, c->ovl_ev[c->ovl], 0);
  if (tev) cudaEventRecord(tev[2], s);
}

static void enqueue_pass(const cluster_ctx* c, cudaStream_t s, int parity) {
  PassArgs a = make_pass_args(c, false);
  if (c->split && c->ovl > 0) {
    enqueue_split_ovl(c, s, parity, nullptr);
  } else if (c->split) {
    LaunchOpt g;
    g.win = c->mixed ? (void*)c->XS[parity & 1] : (void*)c->X[parity & 1];
    g.win_bytes = c->l2_window_bytes;
    kp_launch_spmm(c->KP, a, c->spmm_grid, c->mixed, s, g, c->spmm_rpu);
    if (c->n_heavy > 0) kp_launch_finalize(c->KP, a, s);
    launch_update_ctx(c, a, s);
  } else {
    if (c->n_chunks > 0) kp_launch_heavy(c->KP, a, c->heavy_grid, c->mixed, false, s);
    kp_launch_pass(c->KP, a, c->parts, c->mixed, s);
  }
  kp_launch_fold(c->KP, make_fold_args(c, 0, 0), s);
}

// Objective-only pass over iterate buffer `sel` (float32 master, float32 S).
static void enqueue_eval(const cluster_ctx* c, int sel, int init, cudaStream_t s) {
  PassArgs a = make_pass_args(c, true);
  a.eval_sel = sel;
  if (c->n_chunks > 0) kp_launch_heavy(c->KP, a, c->heavy_grid, false, true, s);
  kp_launch_eval(c->KP, a, c->parts, s);
  kp_launch_fold(c->KP, make_fold_args(c, 1, init), s);
}

cluster_status read_state(cluster_ctx* c) {
  FC_CUDA(cudaMemcpyAsync(&c->host_st, c->st, sizeof(FistaState), cudaMemcpyDeviceToHost, c->stream));
  FC_CUDA(cudaStreamSynchronize(c->stream));
  c->pass_guess = c->host_st.pass;
  return CLUSTER_OK;
}

void fill_report(const cluster_ctx* c, cluster_report* rep) {
  if (!rep) return;
  const FistaState& s = c->host_st;
  rep->iters = s.pass;
  rep->f_iter = s.f_iter;
  rep->f = s.loss_last;
  rep->trace_SU = s.trace_last;
  rep->gram_fro2 = s.gram2_last;
  rep->pg_norm = s.pg_last;
  rep->tau = s.tau;
  rep->L = s.L;
  rep->out_iter = s.out_iter;
  rep->done = s.done;
  rep->status = s.status;
}

static cluster_status power_norm(cluster_ctx* c, double* out) {
  const int64_t n = c->n;
  cudaStream_t s = c->stream;
  double *x = nullptr, *y = nullptr, *part = nullptr;
  const int nb = 256;
  std::vector<double> hp(nb);
  FC_CUDA(cudaMalloc(&x, sizeof(double) * n));
  FC_CUDA(cudaMalloc(&y, sizeof(double) * n));
  FC_CUDA(cudaMalloc(&part, sizeof(double) * nb));
  auto dot = [&](const double* a, const double* b) {
    dot_part_kernel<<<nb, 256, 0, s>>>(a, b, n, part);
    cudaMemcpyAsync(hp.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    double t = 0;
    for (double v : hp) t += v;
    return t;
  };
  fill_start_kernel<<<grid_for(n), 256, 0, s>>>(x, n);
  scale_kernel<<<grid_for(n), 256, 0, s>>>(x, n, 1.0 / std::sqrt(dot(x, x)));
  double lam = 0.0;
  for (int it = 0; it < 1000; ++it) {
    spmv_kernel<<<grid_for(n), 256, 0, s>>>(c->rp, c->col, c->val, x, n, y);
    const double nrm = std::sqrt(dot(y, y));
    if (!(nrm > 0.0)) break;
    scale_kernel<<<grid_for(n), 256, 0, s>>>(y, n, 1.0 / nrm);
    std::swap(x, y);
    const bool conv = it > 5 && std::fabs(nrm - lam) <= 1e-10 * nrm;
    lam = nrm;
    if (conv) break;
  }
  cudaError_t e = cudaGetLastError();
  cudaFree(x);
  cudaFree(y);
  cudaFree(part);
  if (e != cudaSuccess) {
    set_error("power iteration: %s", cudaGetErrorString(e));
    return CLUSTER_ECUDA;
  }
  *out = lam;
  return CLUSTER_OK;
}

static cluster_status capture_graph(cluster_ctx* c) {
  const int variants = c->l2_window_bytes ? 2 : 1;
  for (int p0 = 0; p0 < variants; ++p0) {
    cudaGraph_t g = nullptr;
    FC_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < c->graph_chunk; ++i) enqueue_pass(c, c->cap_stream, p0 + i);
    FC_CUDA(cudaStreamEndCapture(c->cap_stream, &g));
    // node priorities: the overlapped update launches come from a high-priority stream
    cudaError_t e = cudaGraphInstantiate(&c->graph_exec[p0], g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      set_error("graph instantiate: %s", cudaGetErrorString(e));
      return CLUSTER_ECUDA;
    }
  }
  return CLUSTER_OK;
}

static cluster_status validate_inputs(cluster_ctx* c, const float* U0) {
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  int* derr = nullptr;
  int herr = 0;
  FC_CUDA(cudaMalloc(&derr, sizeof(int)));
  cudaMemsetAsync(derr, 0, sizeof(int), s);
  validate_rowptr_kernel<<<grid_for(n + 1), 256, 0, s>>>(c->rp, n, c->nnz, derr);
  cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && herr == 0) {
    validate_csr_kernel<<<grid_for(n), 256, 0, s>>>(c->rp, c->col, c->val, n, 1, derr);
    validate_u0_kernel<<<grid_for(n), 256, 0, s>>>(U0, n, c->k, derr);
    cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
  }
  if (e == cudaSuccess && herr == 0 && c->opt.validate >= 2) {
    validate_sym_kernel<<<grid_for(n), 256, 0, s>>>(c->rp, c->col, c->val, n, derr);
    cudaMemcpyAsync(&herr, derr, sizeof(int), cudaMemcpyDeviceToHost, s);
    e = cudaStreamSynchronize(s);
  }
  cudaFree(derr);
  if (e != cudaSuccess) {
    set_error("validation: %s", cudaGetErrorString(e));
    return CLUSTER_ECUDA;
  }
  if (herr) {
    set_error("invalid input (flags 0x%x):%s%s%s%s%s%s%s%s", herr, (herr & kErrRowPtr) ? " row_ptr" : "",
              (herr & kErrColRange) ? " col-range" : "", (herr & kErrColOrder) ? " col-order" : "",
              (herr & kErrNoDiag) ? " missing-diagonal" : "", (herr & kErrValue) ? " nonfinite-value" : "",
              (herr & kErrAsym) ? " asymmetric" : "", (herr & kErrU0Range) ? " U0-negative-or-nonfinite" : "",
              (herr & kErrU0Sum) ? " U0-row-sum" : "");
    return CLUSTER_EINVAL;
  }
  return CLUSTER_OK;
}

static cluster_status sum_squares(const float* val, int64_t nnz, cudaStream_t s, double* out) {
  *out = 0.0;
  if (nnz <= 0) return CLUSTER_OK;
  const int nb = 1024;
  double* part = nullptr;
  std::vector<double> hp(nb);
  FC_CUDA(cudaMalloc(&part, sizeof(double) * nb));
  sumsq_kernel<<<nb, 256, 0, s>>>(val, nnz, part);
  cudaMemcpyAsync(hp.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  cudaFree(part);
  if (e != cudaSuccess) {
    set_error("sum of squares: %s", cudaGetErrorString(e));
    return CLUSTER_ECUDA;
  }
  double t = 0.0;
  for (double v : hp) t += v;
  *out = t;
  return CLUSTER_OK;
}

void unpad_output(const cluster_ctx* c, const float* X, float* U_out, cudaStream_t s) {
  if (c->relabeled) unpad_perm_kernel<<<grid_for(c->n * c->k), 256, 0, s>>>(X, c->inv, c->n, c->k, c->KP, U_out);
  else unpad_kernel<<<grid_for(c->n * c->k), 256, 0, s>>>(X, c->n, c->k, c->KP, U_out);
}

cluster_status init_impl(const cluster_csr* S, int32_t k, const float* U0, const cluster_options* optp,
                         void* stream, cluster_ctx* c, bool capture) {
  FC_TRY(check_csr_args(S, k));
  if (!U0) FC_EINVAL("U0 is NULL");
  cluster_options opt;
  if (optp) opt = *optp;
  else cluster_options_default(&opt);
  if (opt.precision != CLUSTER_FP32 && opt.precision != CLUSTER_MIXED_BF16)
    FC_EINVAL("unknown precision %d", opt.precision);
  if (opt.step_rule < 0 || opt.step_rule > 2) FC_EINVAL("unknown step rule %d", opt.step_rule);
  if (opt.stop_rule < 0 || opt.stop_rule > 3) FC_EINVAL("unknown stop rule %d", opt.stop_rule);
  if (opt.max_iter < 1) FC_EINVAL("max_iter must be >= 1");
  if (!(opt.tau >= 0.0) || !std::isfinite(opt.tau)) FC_EINVAL("tau must be finite and >= 0");
  if (opt.step_rule == CLUSTER_STEP_CONST && !(opt.tau > 0.0)) FC_EINVAL("constant step needs tau > 0");
  if (!std::isfinite(opt.tol)) FC_EINVAL("tol must be finite");
  if (opt.graph_chunk < 1) opt.graph_chunk = 16;
  c->opt = opt;
  c->stream = (cudaStream_t)stream;
  c->n = S->n;
  c->nnz = S->nnz;
  c->k = k;
  c->KP = padded_k(k);
  c->mixed = opt.precision == CLUSTER_MIXED_BF16;
  c->graph_chunk = opt.graph_chunk;
  FC_CUDA(cudaGetDevice(&c->dev));
  FC_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  cudaStream_t s = c->stream;
  const int64_t n = c->n, nnz = c->nnz;

  // CSR: int64 row pointers always; copy col/val unless borrowed
  FC_TRY(prepare_rowptr(S, s, &c->rp, &c->rp_owned));
  if (!c->rp_owned && !opt.borrow) {
    FC_CUDA(cudaMalloc(&c->rp_owned, sizeof(int64_t) * (n + 1)));
    FC_CUDA(cudaMemcpyAsync(c->rp_owned, S->row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyDeviceToDevice, s));
    c->rp = c->rp_owned;
  }
  if (opt.borrow || nnz == 0) {
    c->col = S->col;
    c->val = S->val;
  } else {
    FC_CUDA(cudaMalloc(&c->col_owned, sizeof(int32_t) * nnz));
    FC_CUDA(cudaMalloc(&c->val_owned, sizeof(float) * nnz));
    FC_CUDA(cudaMemcpyAsync(c->col_owned, S->col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToDevice, s));
    FC_CUDA(cudaMemcpyAsync(c->val_owned, S->val, sizeof(float) * nnz, cudaMemcpyDeviceToDevice, s));
    c->col = c->col_owned;
    c->val = c->val_owned;
  }
  if (opt.validate >= 1) FC_TRY(validate_inputs(c, U0));
  if (opt.relabel && n > 1) FC_TRY(relabel_csr(c));

  // ||S||_F^2 in float64, step size
  double S2 = 0.0;
  FC_TRY(sum_squares(c->val, nnz, s, &S2));
  double L = 0.0, tau = opt.tau;
  if (opt.step_rule == CLUSTER_STEP_INV_L_FROB) {
    L = 4.0 * std::sqrt(S2) + 12.0 * (double)n;
    tau = (opt.tau > 0.0 ? opt.tau : 1.0) / L;
  } else if (opt.step_rule == CLUSTER_STEP_INV_L_SPEC) {
    double nrm = 0.0;
    FC_TRY(power_norm(c, &nrm));
    L = 4.0 * nrm + 12.0 * (double)n;
    tau = (opt.tau > 0.0 ? opt.tau : 1.0) / L;
  }

  // mixed precision: bfloat16 copy of the values
  if (c->mixed && nnz > 0) {
    FC_CUDA(cudaMalloc(&c->val16, sizeof(__nv_bfloat16) * nnz));
    to_bf16_kernel<<<grid_for(nnz), 256, 0, s>>>(c->val, nnz, c->val16);
  }

  // launch geometry: one block range per resident block
  FC_CUDA(kp_setup_attrs(c->KP));
  int sms = 0;
  FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  const int occ = kp_occupancy(c->KP, c->mixed);
  const int R = kp_rows_per_tile(c->KP);
  int64_t parts = (int64_t)sms * occ;
  const int64_t tiles = (n + R - 1) / R;
  if (parts > tiles) parts = tiles;
  if (parts < 1) parts = 1;
  c->parts = (int)parts;
  c->heavy_grid = sms * occ;
  c->split = opt.fused_pass == 0;
  // tcgen05 per-block update: engine 2 (and 3 where the streaming form does
  // not apply) for k in 17..64.  Engine 0 takes the warp form wherever it does
  // not stream: its resident blocks keep more rows in flight per SM than the
  // per-block tcgen05 kernel's chain of short MMA round trips (per iteration,
  // k = 32: 47.1 vs 52.1 us at n = 20,000, 66.0 vs 78.4 us at n = 60,000;
  // k = 64 class of the batched workload: 2.9 vs 3.2 ms; the k = 32 class:
  // 1.10 vs 1.13 ms)
  c->tc_update = opt.update_engine == 2 || opt.update_engine == 3;
  // streaming update for 17 <= k <= 32 on a solo split solver without the
  // overlapped pass: engine 0 from kStreamMinRows articles, engine 3 always
  c->stream_update = c->split && capture && c->KP == 32 && !opt.overlap &&
                     (opt.update_engine == 3 || (opt.update_engine == 0 && n >= kStreamMinRows));
  if (c->split) {
    FC_CUDA(kp_setup_update_attr(c->KP));
    c->spmm_grid = sms * kp_occ_spmm(c->KP, c->mixed);
    int64_t pu = (int64_t)sms * kp_occ_update(c->KP, c->mixed, c->tc_update);
    // at least kMinTilesPerBlock tiles per update block, but not fewer blocks
    // than SMs: a batch runs every block's row range as a work item of its own
    // (setting up G(Y), writing a 2 x KP x KP partial that the fold reads back),
    // so tiny ranges cost more in set-up than in rows, while a lone small solve
    // still keeps every SM busy
    pu = std::min<int64_t>(pu, std::max<int64_t>((int64_t)sms, tiles / kMinTilesPerBlock));
    if (pu > tiles) pu = tiles;
    c->parts_upd = (int)std::max<int64_t>(1, pu);
    if (c->stream_update) {
      FC_CUDA(stream_setup_attr());
      const int64_t t128 = (n + fc::ts::R - 1) / fc::ts::R;
      c->stream_grid = (int)std::max<int64_t>(1, std::min<int64_t>(sms, t128));
      c->parts_upd = 4 * c->stream_grid;  // per CTA: two warpgroups x (high, low) partial slots
    }
  }
  // rows above H nonzeros are chunked: H is about 64 KB of gathered float32
  // data, and at most an eighth of a resident gather warp's share of the
  // nonzeros, so that in a small problem no unit (a team takes up to 4 rows
  // of a unit in turn) sets the critical path of the launch
  {
    const int64_t warps = (int64_t)(c->split ? c->spmm_grid : c->heavy_grid) * 8;
    c->heavy_H = std::max<int64_t>(64, std::min<int64_t>(16384 / c->KP, nnz / std::max<int64_t>(1, 8 * warps)));
  }
  c->row_cost = 6;
  FC_TRY(build_schedule(c));
  // An instance whose units of kRowsPerUnit rows per team leave resident warps
  // idle gathers in one-row units instead (shorter chains of dependent loads
  // per unit; same sums).  A gather launch then needs no more warps (8 a
  // block) than units: a surplus warp only draws a unit number from the shared
  // counter and stops, and at a few thousand rows those draws (one counter)
  // took longer than the gather.
  if (c->split) {
    const int64_t u4 = kp_units(c->KP, c->mixed, n, c->n_heavy, c->n_chunks);
    c->spmm_rpu = (u4 < (int64_t)c->spmm_grid * 8 && n < kOvlMinRows) ? 1 : kRowsPerUnit;
    const int64_t units = c->spmm_rpu == 1 ? kp_units(c->KP, c->mixed, n, c->n_heavy, c->n_chunks, 1) : u4;
    c->spmm_grid = (int)std::min<int64_t>(c->spmm_grid, std::max<int64_t>(1, (units + 7) / 8));
  }

  // Overlapped pass: with the internal numbering the gather order is the
  // identity, so a prefix of the gather's units is a prefix of the rows and
  // the update of a row chunk can start once that prefix is gathered.  Eligible
  // contexts use kOvlBlockFactor times more (smaller) update blocks, with or
  // without the overlap, so that both schedules sum the same partials (same
  // bits) and the last chunk's update is short.
  if (c->split && c->relabeled && n >= kOvlMinRows && !c->stream_update) {
    int* dflag = nullptr;
    int hflag = 1;
    FC_CUDA(cudaMalloc(&dflag, sizeof(int)));
    cudaError_t e = cudaMemsetAsync(dflag, 0, sizeof(int), s);
    if (e == cudaSuccess) {
      order_identity_kernel<<<grid_for(n), 256, 0, s>>>(c->order, n, dflag);
      e = cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(dflag);
    if (e != cudaSuccess) {
      set_error("order check: %s", cudaGetErrorString(e));
      return CLUSTER_ECUDA;
    }
    if (hflag == 0) {
      c->ovl_eligible = true;
      c->parts_upd = (int)std::min<int64_t>((int64_t)c->parts_upd * kOvlBlockFactor, tiles);
      if (opt.overlap) {
        c->ovl = cluster_ctx::kMaxOvl;
        c->n_work = c->ovl;
        c->spmm_grid_ovl = sms * std::max(1, kp_occ_spmm(c->KP, c->mixed) - 1);
        for (int ch = 0; ch <= c->ovl; ++ch) c->ovl_blocks[ch] = (int)((int64_t)ch * c->parts_upd / c->ovl);
        c->ovl_units[0] = 0;
        for (int ch = 1; ch < c->ovl; ++ch)
          c->ovl_units[ch] = kp_unit_of_position(c->KP, c->mixed, n * (int64_t)c->ovl_blocks[ch] / c->parts_upd,
                                                 c->n_heavy, c->n_chunks);
        c->ovl_units[c->ovl] = kp_units(c->KP, c->mixed, n, c->n_heavy, c->n_chunks);
        int prio_lo = 0, prio_hi = 0;
        FC_CUDA(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        FC_CUDA(cudaStreamCreateWithPriority(&c->side_stream, cudaStreamNonBlocking, prio_hi));
        for (int ch = 0; ch <= c->ovl; ++ch) FC_CUDA(cudaEventCreateWithFlags(&c->ovl_ev[ch], cudaEventDisableTiming));
      }
    }
  }

  // iterate buffers and reductions
  const size_t nk = (size_t)n * c->KP;
  FC_CUDA(cudaMalloc(&c->X[0], sizeof(float) * nk));
  FC_CUDA(cudaMalloc(&c->X[1], sizeof(float) * nk));
  if (c->split) {
    FC_CUDA(cudaMalloc(&c->Z[0], sizeof(float) * nk));
    FC_CUDA(cudaMalloc(&c->Z[1], sizeof(float) * nk));
    FC_CUDA(cudaMemsetAsync(c->Z[0], 0, sizeof(float) * nk, s));
    FC_CUDA(cudaMemsetAsync(c->Z[1], 0, sizeof(float) * nk, s));
    FC_CUDA(cudaMalloc(&c->work, sizeof(unsigned long long) * cluster_ctx::kMaxOvl));
    FC_CUDA(cudaMemsetAsync(c->work, 0, sizeof(unsigned long long) * cluster_ctx::kMaxOvl, s));
  } else {
    FC_CUDA(cudaMalloc(&c->Zp, sizeof(float) * nk));
    FC_CUDA(cudaMemsetAsync(c->Zp, 0, sizeof(float) * nk, s));
  }
  if (c->mixed) {
    FC_CUDA(cudaMalloc(&c->XS[0], sizeof(__nv_bfloat16) * nk));
    FC_CUDA(cudaMalloc(&c->XS[1], sizeof(__nv_bfloat16) * nk));
  }
  const size_t e2 = (size_t)c->KP * c->KP;
  FC_CUDA(cudaMalloc(&c->A[0], sizeof(double) * e2));
  FC_CUDA(cudaMalloc(&c->A[1], sizeof(double) * e2));
  FC_CUDA(cudaMalloc(&c->Gy, sizeof(float) * e2));
  FC_CUDA(cudaMalloc(&c->bpart, sizeof(double) * 2 * (size_t)kp_fold_blocks(c->KP)));
  const int slots = std::max(c->parts, c->parts_upd);
  FC_CUDA(cudaMalloc(&c->gram_part, sizeof(float) * 2 * e2 * slots));
  FC_CUDA(cudaMalloc(&c->sc_part, sizeof(double) * 4 * slots));
  FC_CUDA(cudaMalloc(&c->st, sizeof(FistaState)));
  if (c->stream_update) FC_TRY(make_stream_maps(c));

  // Xbar^0 = U0 in buffer 0; buffer 1 starts as a copy (momentum is 0 for the first two passes)
  if (c->relabeled)
    pad_perm_kernel<<<grid_for((int64_t)nk), 256, 0, s>>>(U0, c->perm, n, k, c->KP, c->X[0], c->X[1], c->XS[0],
                                                          c->XS[1]);
  else
    pad_kernel<<<grid_for((int64_t)nk), 256, 0, s>>>(U0, n, k, c->KP, c->X[0], c->X[1], c->XS[0], c->XS[1]);
  FistaState& h = c->host_st;
  memset(&h, 0, sizeof(h));
  h.S2 = S2;
  h.tau = tau;
  h.L = L;
  h.tol = opt.tol;
  h.t = 1.0;
  h.beta = 0.0;       // beta_1 = 0 (X^1 = Xbar^0)
  h.beta_next = 0.0;  // beta_2 = (t_1 - 1) / t_2 = 0
  h.max_iter = opt.max_iter;
  h.f_iter = -1;
  h.out_iter = 0;
  h.stop_rule = opt.stop_rule;
  h.accel = opt.accel ? 1 : 0;
  h.k = k;
  FC_CUDA(cudaMemcpyAsync(c->st, &h, sizeof(FistaState), cudaMemcpyHostToDevice, s));
  // Gram of Xbar^0: seeds G(Y^1) = Xbar^0^T Xbar^0 and ||Xbar^0^T Xbar^0||^2.  For
  // k <= 64 without a product with S: the first pass's product gives the trace
  // term of f(Xbar^0), and its fold the loss (f_iter stays -1 until then).
  // k = 128: one objective-only pass (also f(Xbar^0) at once).
  if (c->KP <= 64) {
    // one wave of resident blocks (at most one per partial slot, at least 32 rows each)
    const int slots = std::max(c->parts, c->parts_upd);
    const int g0 = (int)std::max<int64_t>(
        1, std::min<int64_t>({(int64_t)slots, (int64_t)sms * kp_occ_gram0(c->KP), (n + 31) / 32}));
    kp_launch_gram0(c->KP, c->X[0], n, c->gram_part, c->sc_part, g0, s);
    FoldArgs f0 = make_fold_args(c, 1, 1);
    f0.parts = g0;
    kp_launch_fold(c->KP, f0, s);
    FC_CUDA(cudaGetLastError());
    FC_TRY(read_state(c));
  } else {
    enqueue_eval(c, 0, 1, s);
    FC_CUDA(cudaGetLastError());
    FC_TRY(read_state(c));
    h = c->host_st;
    h.loss_last = h.eval_f;
    h.trace_last = h.eval_trace;
    h.gram2_last = h.eval_gram2;
    h.f_iter = 0;
    FC_CUDA(cudaMemcpyAsync(c->st, &h, sizeof(FistaState), cudaMemcpyHostToDevice, s));
    FC_CUDA(cudaStreamSynchronize(s));
  }
  c->pass_guess = 0;
  // persisting L2 window over the gathered rows of the highest-degree
  // articles (the first rows in the internal numbering): half of the
  // device's persisting maximum, which measured best at n = 70M, k = 32
  // (solo solvers only: the batched kernels take no window, and a set-aside
  // only shrinks the L2 they share)
  if (capture && c->split && c->relabeled && opt.l2_window) {
    int maxp = 0, maxw = 0;
    FC_CUDA(cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, c->dev));
    FC_CUDA(cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, c->dev));
    const size_t rowb = (size_t)c->KP * (c->mixed ? 2 : 4);
    size_t want = std::min<size_t>((size_t)maxp / 2, (size_t)maxw);
    want = std::min<size_t>(want, rowb * (size_t)n);
    if (want >= ((size_t)1 << 20)) {
      FC_TRY(l2_setaside_acquire(want));
      c->l2_window_bytes = want;
    }
  }
  if (capture) FC_TRY(capture_graph(c));
  return CLUSTER_OK;
}

cluster_status finalize_loss(cluster_ctx* c) {
  FistaState& h = c->host_st;
  if (h.f_iter == h.out_iter || h.status == 4) return CLUSTER_OK;
  enqueue_eval(c, (int)(h.out_iter & 1), 0, c->stream);
  FC_CUDA(cudaGetLastError());
  FC_TRY(read_state(c));
  FistaState& g = c->host_st;
  g.loss_last = g.eval_f;
  g.trace_last = g.eval_trace;
  g.gram2_last = g.eval_gram2;
  g.f_iter = g.out_iter;
  // keep the device copy in step so later reports agree
  FC_CUDA(cudaMemcpyAsync(&c->st->loss_last, &g.loss_last, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  FC_CUDA(cudaMemcpyAsync(&c->st->trace_last, &g.trace_last, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  FC_CUDA(cudaMemcpyAsync(&c->st->gram2_last, &g.gram2_last, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  FC_CUDA(cudaMemcpyAsync(&c->st->f_iter, &g.f_iter, sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
  FC_CUDA(cudaStreamSynchronize(c->stream));
  return CLUSTER_OK;
}

// checkpoint layout: header, FistaState, Gy (float32 KP^2), X0, X1, Z0, Z1 (split) or Zp (fused)
// [, XS0, XS1]
struct StateHeader {
  uint64_t magic;
  int64_t n;
  int32_t k, KP, mixed, pad;
};
static const uint64_t kStateMagic = 0x46434C5553543031ull;  // "FCLUST01"

static size_t state_bytes(const cluster_ctx* c) {
  const size_t e2 = (size_t)c->KP * c->KP, nk = (size_t)c->n * c->KP;
  size_t b = sizeof(StateHeader) + sizeof(FistaState) + e2 * sizeof(float) + (c->split ? 4 : 3) * nk * sizeof(float);
  if (c->mixed) b += 2 * nk * sizeof(__nv_bfloat16);
  return b;
}

// Objective-only evaluation with a temporary context: the same degree
// schedule and chunked rows as a solver, so power-law hubs stay balanced.
static cluster_status objective_impl(const cluster_csr* S, int32_t k, const float* U, void* stream, double* f,
                                     cluster_ctx* c) {
  c->stream = (cudaStream_t)stream;
  c->n = S->n;
  c->nnz = S->nnz;
  c->k = k;
  c->KP = padded_k(k);
  c->mixed = false;
  FC_CUDA(cudaGetDevice(&c->dev));
  cudaStream_t s = c->stream;
  FC_TRY(prepare_rowptr(S, s, &c->rp, &c->rp_owned));
  c->col = S->col;
  c->val = S->val;
  FC_CUDA(kp_setup_attrs(c->KP));
  int sms = 0;
  FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  const int occ = kp_occupancy(c->KP, false);
  const int R = kp_rows_per_tile(c->KP);
  int64_t parts = (int64_t)sms * occ;
  if (parts > (c->n + R - 1) / R) parts = (c->n + R - 1) / R;
  c->parts = (int)std::max<int64_t>(1, parts);
  c->heavy_grid = sms * occ;
  c->heavy_H = std::max<int64_t>(64, 16384 / c->KP);
  FC_TRY(build_schedule(c));
  const size_t e2 = (size_t)c->KP * c->KP, nk = (size_t)c->n * c->KP;
  FC_CUDA(cudaMalloc(&c->X[0], sizeof(float) * nk));
  FC_CUDA(cudaMalloc(&c->A[0], sizeof(double) * e2));
  FC_CUDA(cudaMalloc(&c->gram_part, sizeof(float) * 2 * e2 * c->parts));
  FC_CUDA(cudaMalloc(&c->sc_part, sizeof(double) * 4 * c->parts));
  FC_CUDA(cudaMalloc(&c->st, sizeof(FistaState)));
  FistaState h;
  memset(&h, 0, sizeof(h));
  h.k = k;
  FC_TRY(sum_squares(S->val, S->nnz, s, &h.S2));
  FC_CUDA(cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  pad_kernel<<<grid_for((int64_t)nk), 256, 0, s>>>(U, c->n, k, c->KP, c->X[0], nullptr, nullptr, nullptr);
  enqueue_eval(c, 0, 0, s);
  FC_CUDA(cudaGetLastError());
  FC_TRY(read_state(c));
  *f = c->host_st.eval_f;
  return CLUSTER_OK;
}

}  // namespace fc

using namespace fc;

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" void cluster_options_default(cluster_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = CLUSTER_FP32;
  opt->step_rule = CLUSTER_STEP_INV_L_FROB;
  opt->stop_rule = CLUSTER_STOP_LOSS;
  opt->accel = 1;
  opt->borrow = 0;
  opt->validate = 1;
  opt->tau = 1.0;
  opt->tol = 0.0;
  opt->max_iter = 1000;
  opt->graph_chunk = 16;
  opt->fused_pass = 0;
  opt->relabel = 1;
  opt->l2_window = 1;
  opt->update_engine = 0;
  opt->overlap = 0;
}

extern "C" const char* cluster_last_error(void) { return g_err.c_str(); }

extern "C" cluster_status cluster_init(const cluster_csr* S, int32_t k, const float* U0, const cluster_options* opt,
                                       void* stream, cluster_ctx** out) {
  clear_error();
  if (!out) FC_EINVAL("out is NULL");
  *out = nullptr;
  cluster_ctx* c = new (std::nothrow) cluster_ctx();
  if (!c) {
    set_error("out of host memory");
    return CLUSTER_ENOMEM;
  }
  cluster_status st = init_impl(S, k, U0, opt, stream, c, true);
  if (st != CLUSTER_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    ctx_free(c);
    return st;
  }
  *out = c;
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_enqueue(cluster_ctx* c, int64_t iters) {
  clear_error();
  if (!c) FC_EINVAL("ctx is NULL");
  if (iters < 0) FC_EINVAL("iters must be >= 0");
  if (iters == 0) return CLUSTER_OK;
  FC_CUDA(cudaSetDevice(c->dev));
  set_limit_kernel<<<1, 1, 0, c->stream>>>(c->st, iters);
  const int64_t reps = (iters + c->graph_chunk - 1) / c->graph_chunk;
  for (int64_t r = 0; r < reps; ++r) {
    // the graph whose window follows the buffers of the expected passes (a
    // wrong guess, e.g. after an early stop, only costs cache hits)
    const int par = c->graph_exec[1] ? (int)((c->pass_guess + r * c->graph_chunk) & 1) : 0;
    FC_CUDA(cudaGraphLaunch(c->graph_exec[par], c->stream));
  }
  c->pass_guess += iters;
  FC_CUDA(cudaGetLastError());
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_enqueue_profiled(cluster_ctx* c, int64_t iters, cluster_kernel_times* out) {
  clear_error();
  if (!c || !out) FC_EINVAL("NULL argument");
  if (iters < 1) FC_EINVAL("iters must be >= 1");
  FC_CUDA(cudaSetDevice(c->dev));
  memset(out, 0, sizeof(*out));
  cudaStream_t s = c->stream;
  std::vector<cudaEvent_t> ev((size_t)(5 * iters));
  for (auto& e : ev) FC_CUDA(cudaEventCreate(&e));
  set_limit_kernel<<<1, 1, 0, s>>>(c->st, iters);
  PassArgs a = make_pass_args(c, false);
  const FoldArgs f = make_fold_args(c, 0, 0);
  // events: [0] start, [1] after the gather (split) / chunk kernel (fused), [2] after the chunk sums (split) /
  // fused pass, [3] after the update (split), [4] after the fold
  for (int64_t i = 0; i < iters; ++i) {
    cudaEvent_t* e = &ev[(size_t)(5 * i)];
    cudaEventRecord(e[0], s);
    if (c->split && c->ovl > 0) {
      // overlapped: pass = start to the last gather (hub-row sums included),
      // update = the part of the updates after the last gather
      enqueue_split_ovl(c, s, (int)((c->pass_guess + i) & 1), &e[1]);
    } else if (c->split) {
      const int par = (int)((c->pass_guess + i) & 1);
      LaunchOpt g;
      g.win = c->mixed ? (void*)c->XS[par] : (void*)c->X[par];
      g.win_bytes = c->l2_window_bytes;
      kp_launch_spmm(c->KP, a, c->spmm_grid, c->mixed, s, g, c->spmm_rpu);
      cudaEventRecord(e[1], s);
      if (c->n_heavy > 0) kp_launch_finalize(c->KP, a, s);
      cudaEventRecord(e[2], s);
      launch_update_ctx(c, a, s);
    } else {
      if (c->n_chunks > 0) kp_launch_heavy(c->KP, a, c->heavy_grid, c->mixed, false, s);
      cudaEventRecord(e[1], s);
      kp_launch_pass(c->KP, a, c->parts, c->mixed, s);
      cudaEventRecord(e[2], s);
    }
    cudaEventRecord(e[3], s);
    kp_launch_fold(c->KP, f, s);
    cudaEventRecord(e[4], s);
  }
  c->pass_guess += iters;
  cudaError_t err = cudaStreamSynchronize(s);
  if (err == cudaSuccess) err = cudaGetLastError();
  double th = 0, tp = 0, tf = 0, tu = 0;
  float ms = 0.f;
  for (int64_t i = 0; i < iters && err == cudaSuccess; ++i) {
    cudaEvent_t* e = &ev[(size_t)(5 * i)];
    float m01, m12, m23, m34;
    cudaEventElapsedTime(&m01, e[0], e[1]);
    cudaEventElapsedTime(&m12, e[1], e[2]);
    cudaEventElapsedTime(&m23, e[2], e[3]);
    cudaEventElapsedTime(&m34, e[3], e[4]);
    if (c->split) {
      tp += m01;
      th += m12;
      tu += m23;
    } else {
      th += m01;
      tp += m12;
    }
    tf += m34;
  }
  if (err == cudaSuccess) {
    cudaEventElapsedTime(&ms, ev.front(), ev.back());
    out->total_ms = ms;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (err != cudaSuccess) {
    set_error("profiled iterations: %s", cudaGetErrorString(err));
    return CLUSTER_ECUDA;
  }
  out->pass_ms = tp / iters;
  out->heavy_ms = th / iters;
  out->fold_ms = tf / iters;
  out->update_ms = tu / iters;
  out->launches = iters;
  {
    // launches per iteration: split = gather(s) + update(s) + chunk sums (if any) + fold;
    // fused = chunk partials (if any) + pass + fold; plus the limit kernel
    int64_t per = 0;
    if (c->split && c->ovl > 0) {
      for (int ch = 0; ch < c->ovl; ++ch)
        per += (c->ovl_units[ch + 1] > c->ovl_units[ch] ? 1 : 0) + (c->ovl_blocks[ch + 1] > c->ovl_blocks[ch] ? 1 : 0);
      per += (c->n_heavy > 0 ? 1 : 0) + 1;
    } else if (c->split) {
      per = 3 + (c->n_heavy > 0 ? 1 : 0);
    } else {
      per = 2 + (c->n_chunks > 0 ? 1 : 0);
    }
    out->kernels = 1 + per * iters;
  }
  out->heavy_rows = c->n_heavy;
  out->heavy_nnz = c->heavy_nnz;
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_step(cluster_ctx* c, int64_t iters, cluster_report* rep) {
  FC_TRY(cluster_enqueue(c, iters));
  FC_TRY(read_state(c));
  fill_report(c, rep);
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_get_report(cluster_ctx* c, cluster_report* rep) {
  clear_error();
  if (!c) FC_EINVAL("ctx is NULL");
  FC_TRY(read_state(c));
  fill_report(c, rep);
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_test_hooks(cluster_ctx* c, int32_t flags) {
  clear_error();
  if (!c) FC_EINVAL("ctx is NULL");
  FC_CUDA(cudaMemcpyAsync(reinterpret_cast<char*>(c->st) + offsetof(FistaState, hooks), &flags, sizeof(flags),
                          cudaMemcpyHostToDevice, c->stream));
  FC_CUDA(cudaStreamSynchronize(c->stream));
  c->host_st.hooks = flags;
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_solve(cluster_ctx* c, cluster_report* rep) {
  clear_error();
  if (!c) FC_EINVAL("ctx is NULL");
  FC_CUDA(cudaSetDevice(c->dev));
  FC_TRY(read_state(c));
  while (!c->host_st.done) {
    const int64_t left = c->host_st.max_iter - c->host_st.pass;
    const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(left, (int64_t)c->graph_chunk * 8));
    FC_TRY(cluster_step(c, chunk, nullptr));
  }
  FC_TRY(finalize_loss(c));
  fill_report(c, rep);
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_get_U(cluster_ctx* c, float* U_out) {
  clear_error();
  if (!c || !U_out) FC_EINVAL("NULL argument");
  FC_CUDA(cudaSetDevice(c->dev));
  FC_TRY(read_state(c));
  unpad_output(c, c->X[c->host_st.out_iter & 1], U_out, c->stream);
  FC_CUDA(cudaGetLastError());
  FC_CUDA(cudaStreamSynchronize(c->stream));
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_state_size(cluster_ctx* c, size_t* bytes) {
  clear_error();
  if (!c || !bytes) FC_EINVAL("NULL argument");
  *bytes = state_bytes(c);
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_get_state(cluster_ctx* c, void* buf, size_t bytes) {
  clear_error();
  if (!c || !buf) FC_EINVAL("NULL argument");
  if (bytes < state_bytes(c)) FC_EINVAL("state buffer too small (%zu < %zu)", bytes, state_bytes(c));
  FC_CUDA(cudaSetDevice(c->dev));
  char* p = (char*)buf;
  StateHeader hd{kStateMagic, c->n, c->k, c->KP, c->mixed ? 1 : 0, (c->split ? 1 : 0) | (c->relabeled ? 2 : 0)};
  memcpy(p, &hd, sizeof(hd));
  p += sizeof(hd);
  const size_t e2 = (size_t)c->KP * c->KP, nk = (size_t)c->n * c->KP;
  struct Seg {
    const void* src;
    size_t b;
  } segs[8];
  int nseg = 0;
  segs[nseg++] = {c->st, sizeof(FistaState)};
  segs[nseg++] = {c->Gy, e2 * 4};
  segs[nseg++] = {c->X[0], nk * 4};
  segs[nseg++] = {c->X[1], nk * 4};
  if (c->split) {
    segs[nseg++] = {c->Z[0], nk * 4};
    segs[nseg++] = {c->Z[1], nk * 4};
  } else {
    segs[nseg++] = {c->Zp, nk * 4};
  }
  if (c->mixed) {
    segs[nseg++] = {c->XS[0], nk * 2};
    segs[nseg++] = {c->XS[1], nk * 2};
  }
  for (int i = 0; i < nseg; ++i) {
    FC_CUDA(cudaMemcpyAsync(p, segs[i].src, segs[i].b, cudaMemcpyDeviceToHost, c->stream));
    p += segs[i].b;
  }
  FC_CUDA(cudaStreamSynchronize(c->stream));
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_set_state(cluster_ctx* c, const void* buf, size_t bytes) {
  clear_error();
  if (!c || !buf) FC_EINVAL("NULL argument");
  if (bytes < state_bytes(c)) FC_EINVAL("state buffer too small");
  FC_CUDA(cudaSetDevice(c->dev));
  const char* p = (const char*)buf;
  StateHeader hd;
  memcpy(&hd, p, sizeof(hd));
  if (hd.magic != kStateMagic || hd.n != c->n || hd.k != c->k || hd.KP != c->KP || hd.mixed != (c->mixed ? 1 : 0) ||
      hd.pad != ((c->split ? 1 : 0) | (c->relabeled ? 2 : 0)))
    FC_EINVAL("state does not match this context (n, k, precision, iteration form or numbering differ)");
  p += sizeof(hd);
  FistaState fs;
  memcpy(&fs, p, sizeof(fs));
  fs.ticket = 0;
  const size_t e2 = (size_t)c->KP * c->KP, nk = (size_t)c->n * c->KP;
  struct Seg {
    void* dst;
    size_t b;
  } segs[8];
  int nseg = 0;
  segs[nseg++] = {c->st, sizeof(FistaState)};
  segs[nseg++] = {c->Gy, e2 * 4};
  segs[nseg++] = {c->X[0], nk * 4};
  segs[nseg++] = {c->X[1], nk * 4};
  if (c->split) {
    segs[nseg++] = {c->Z[0], nk * 4};
    segs[nseg++] = {c->Z[1], nk * 4};
  } else {
    segs[nseg++] = {c->Zp, nk * 4};
  }
  if (c->mixed) {
    segs[nseg++] = {c->XS[0], nk * 2};
    segs[nseg++] = {c->XS[1], nk * 2};
  }
  for (int i = 0; i < nseg; ++i) {
    const void* src = (i == 0) ? (const void*)&fs : (const void*)p;
    FC_CUDA(cudaMemcpyAsync(segs[i].dst, src, segs[i].b, cudaMemcpyHostToDevice, c->stream));
    p += segs[i].b;
  }
  FC_CUDA(cudaStreamSynchronize(c->stream));
  c->host_st = fs;
  c->pass_guess = fs.pass;
  return CLUSTER_OK;
}

extern "C" void cluster_destroy(cluster_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  cudaStreamSynchronize(c->stream);
  ctx_free(c);
}

// ---------------------------------------------------------------------------
// standalone objective
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// second-order check: H[W], <W, H[W]>, <grad f(U), W> from one product S W
// ---------------------------------------------------------------------------
template <int KP>
static cluster_status hess_combine(cluster_ctx* c, const float* Up, const float* Wp, float* HW, double* curvature,
                                   double* slope) {
  constexpr int E2 = KP * KP;
  cudaStream_t s = c->stream;
  const int64_t n = c->n;
  int sms = 0;
  FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  const int gparts = (int)std::max<int64_t>(1, std::min<int64_t>(2 * sms, (n + kHessRows - 1) / kHessRows));
  const int echunks = (3 * E2 + 256 * kHessPerThr - 1) / (256 * kHessPerThr);
  float* gpart = nullptr;
  double* gsum = nullptr;
  float *Gf = nullptr, *Bf = nullptr;
  double* dots = nullptr;
  const int rparts = 4 * sms;
  cluster_status st = CLUSTER_OK;
  do {
    cudaError_t e;
    if ((e = cudaMalloc(&gpart, sizeof(float) * 3 * E2 * gparts)) != cudaSuccess ||
        (e = cudaMalloc(&gsum, sizeof(double) * 3 * E2)) != cudaSuccess ||
        (e = cudaMalloc(&Gf, sizeof(float) * 2 * E2)) != cudaSuccess ||
        (e = cudaMalloc(&dots, sizeof(double) * 2 * rparts)) != cudaSuccess) {
      set_error("hessian scratch: %s", cudaGetErrorString(e));
      st = e == cudaErrorMemoryAllocation ? CLUSTER_ENOMEM : CLUSTER_ECUDA;
      break;
    }
    Bf = Gf + E2;
    hess_gram_kernel<KP><<<dim3(gparts, echunks), 256, 0, s>>>(Up, Wp, n, gpart);
    hess_fold_kernel<<<(3 * E2 + 255) / 256, 256, 0, s>>>(gpart, gparts, 3 * E2, gsum);
    std::vector<double> g(3 * E2);
    cudaMemcpyAsync(g.data(), gsum, sizeof(double) * 3 * E2, cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
      set_error("hessian Grams: %s", cudaGetErrorString(e));
      st = CLUSTER_ECUDA;
      break;
    }
    const double* G = g.data();
    const double* M = G + E2;  // U^T W
    const double* N = M + E2;  // W^T W
    std::vector<float> gb(2 * E2);
    double NG = 0.0, MM = 0.0, MMt = 0.0, MG = 0.0;
    for (int a = 0; a < KP; ++a)
      for (int b = 0; b < KP; ++b) {
        gb[a * KP + b] = (float)G[a * KP + b];
        gb[E2 + a * KP + b] = (float)(M[a * KP + b] + M[b * KP + a]);
        NG += N[a * KP + b] * G[a * KP + b];
        MM += M[a * KP + b] * M[a * KP + b];
        MMt += M[a * KP + b] * M[b * KP + a];
        MG += M[a * KP + b] * G[a * KP + b];
      }
    cudaMemcpyAsync(Gf, gb.data(), sizeof(float) * 2 * E2, cudaMemcpyHostToDevice, s);
    const int smem = (int)(sizeof(float) * 2 * E2);
    if ((e = cudaFuncSetAttribute(hess_row_kernel<KP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
        cudaSuccess) {
      set_error("hessian attributes: %s", cudaGetErrorString(e));
      st = CLUSTER_ECUDA;
      break;
    }
    hess_row_kernel<KP><<<rparts, 256, smem, s>>>(Up, Wp, c->Z[1], Gf, Bf, n, c->k, HW, dots);
    std::vector<double> d(2 * rparts);
    cudaMemcpyAsync(d.data(), dots, sizeof(double) * 2 * rparts, cudaMemcpyDeviceToHost, s);
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
      set_error("hessian rows: %s", cudaGetErrorString(e));
      st = CLUSTER_ECUDA;
      break;
    }
    double wz = 0.0, uz = 0.0;
    for (int p = 0; p < rparts; ++p) {
      wz += d[2 * p];
      uz += d[2 * p + 1];
    }
    // <W, H[W]> = -4 <W, S W> + 4 <W^T W, G> + 4 <M, M + M^T>;  <grad f, W> = -4 <U, S W> + 4 <M, G>
    if (curvature) *curvature = -4.0 * wz + 4.0 * NG + 4.0 * (MM + MMt);
    if (slope) *slope = -4.0 * uz + 4.0 * MG;
  } while (0);
  if (gpart) cudaFree(gpart);
  if (gsum) cudaFree(gsum);
  if (Gf) cudaFree(Gf);
  if (dots) cudaFree(dots);
  return st;
}

static cluster_status hessian_impl(const cluster_csr* S, int32_t k, const float* U, const float* W, void* stream,
                                   float* HW, double* curvature, double* slope, cluster_ctx* c) {
  c->stream = (cudaStream_t)stream;
  c->n = S->n;
  c->nnz = S->nnz;
  c->k = k;
  c->KP = padded_k(k);
  c->mixed = false;
  FC_CUDA(cudaGetDevice(&c->dev));
  cudaStream_t s = c->stream;
  FC_TRY(prepare_rowptr(S, s, &c->rp, &c->rp_owned));
  c->col = S->col;
  c->val = S->val;
  FC_CUDA(kp_setup_attrs(c->KP));
  int sms = 0;
  FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
  const int occ = kp_occupancy(c->KP, false);
  const int R = kp_rows_per_tile(c->KP);
  int64_t parts = (int64_t)sms * occ;
  if (parts > (c->n + R - 1) / R) parts = (c->n + R - 1) / R;
  c->parts = (int)std::max<int64_t>(1, parts);
  c->heavy_grid = sms * occ;
  c->heavy_H = std::max<int64_t>(64, 16384 / c->KP);
  FC_TRY(build_schedule(c));
  c->spmm_grid = sms * kp_occ_spmm(c->KP, false);
  const size_t nk = (size_t)c->n * c->KP;
  // X0 = W (the gathered operand), X1 = U; S W lands in Z1 (a pass-0 product)
  FC_CUDA(cudaMalloc(&c->X[0], sizeof(float) * nk));
  FC_CUDA(cudaMalloc(&c->X[1], sizeof(float) * nk));
  FC_CUDA(cudaMalloc(&c->Z[1], sizeof(float) * nk));
  FC_CUDA(cudaMalloc(&c->work, sizeof(unsigned long long)));
  FC_CUDA(cudaMemsetAsync(c->work, 0, sizeof(unsigned long long), s));
  FC_CUDA(cudaMalloc(&c->st, sizeof(FistaState)));
  FistaState h;
  memset(&h, 0, sizeof(h));
  h.k = k;
  h.limit = 1;  // one product: pass 0 of a state that is not done
  FC_CUDA(cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, s));
  pad_kernel<<<grid_for((int64_t)nk), 256, 0, s>>>(W, c->n, k, c->KP, c->X[0], nullptr, nullptr, nullptr);
  pad_kernel<<<grid_for((int64_t)nk), 256, 0, s>>>(U, c->n, k, c->KP, c->X[1], nullptr, nullptr, nullptr);
  PassArgs a = make_pass_args(c, true);
  kp_launch_spmm(c->KP, a, c->spmm_grid, false, s);
  if (c->n_heavy > 0) kp_launch_finalize(c->KP, a, s);
  FC_CUDA(cudaGetLastError());
  cluster_status st = CLUSTER_OK;
  switch (c->KP) {
    case 2: st = hess_combine<2>(c, c->X[1], c->X[0], HW, curvature, slope); break;
    case 4: st = hess_combine<4>(c, c->X[1], c->X[0], HW, curvature, slope); break;
    case 8: st = hess_combine<8>(c, c->X[1], c->X[0], HW, curvature, slope); break;
    case 16: st = hess_combine<16>(c, c->X[1], c->X[0], HW, curvature, slope); break;
    case 32: st = hess_combine<32>(c, c->X[1], c->X[0], HW, curvature, slope); break;
    case 64: st = hess_combine<64>(c, c->X[1], c->X[0], HW, curvature, slope); break;
    default: st = hess_combine<128>(c, c->X[1], c->X[0], HW, curvature, slope); break;
  }
  return st;
}

extern "C" cluster_status cluster_hessian_apply(const cluster_csr* S, int32_t k, const float* U, const float* W,
                                                void* stream, float* HW, double* curvature, double* slope) {
  clear_error();
  FC_TRY(check_csr_args(S, k));
  if (!U || !W) FC_EINVAL("NULL argument");
  cluster_ctx* c = new (std::nothrow) cluster_ctx();
  if (!c) {
    set_error("out of host memory");
    return CLUSTER_ENOMEM;
  }
  cluster_status st = hessian_impl(S, k, U, W, stream, HW, curvature, slope, c);
  cudaStreamSynchronize((cudaStream_t)stream);
  ctx_free(c);
  return st;
}

extern "C" cluster_status cluster_objective(const cluster_csr* S, int32_t k, const float* U, void* stream,
                                            double* f) {
  clear_error();
  FC_TRY(check_csr_args(S, k));
  if (!U || !f) FC_EINVAL("NULL argument");
  cluster_ctx* c = new (std::nothrow) cluster_ctx();
  if (!c) {
    set_error("out of host memory");
    return CLUSTER_ENOMEM;
  }
  cluster_status st = objective_impl(S, k, U, stream, f, c);
  cudaStreamSynchronize((cudaStream_t)stream);
  ctx_free(c);
  return st;
}
