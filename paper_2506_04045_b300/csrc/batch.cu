// Batched solves: many independent clustering instances of uneven n and k
// advanced together.  Instances are grouped into classes by padded cluster
// count and precision; per class and iteration there is one persistent
// gather launch, one chunk-sum launch, one persistent update launch and one
// fold launch covering every instance of the class.  The iteration sequence
// of all classes is captured in a CUDA graph of graph_chunk iterations.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "batch_kernels.cuh"
#include "solver_impl.h"
#include "util.h"

using namespace fc;

namespace {

struct BatchClass {
  int KP = 0;
  bool mixed = false;
  bool tc = true;            // update on tcgen05 (cluster_options.update_engine == 0)
  std::vector<int> members;  // instance indices
  // device copies of the per-instance tables
  PassArgs* d_args = nullptr;
  FoldArgs* d_folds = nullptr;
  int64_t* d_unit_base = nullptr;   // gather unit prefix sums of the current shape (one of d_ub)
  int64_t* d_ub[kGatherShapes] = {};  // per gather tile shape (rows per unit differ)
  int64_t units_s[kGatherShapes] = {};
  int shape = 0;                      // gather tile shape (BShape index)
  int64_t* d_heavy_base = nullptr;
  int32_t* d_item_inst = nullptr;
  int32_t* d_item_slot = nullptr;
  int32_t* d_parts = nullptr;
  FistaState** d_states = nullptr;
  unsigned long long* d_work = nullptr;
  int n_items = 0;
  int64_t units = 0, heavy = 0;
  int spmm_grid = 1, upd_grid = 1, fin_grid = 1;
  int occ_spmm = 1, occ_upd = 1;   // resident blocks per SM of the two persistent kernels
  int64_t gather_blocks_max = 1;   // blocks beyond this would find no gather unit
  bool tuned = false;
  double gather_ms = 0.0, update_ms = 0.0;  // autotune: the chosen shapes' best times (class alone)
  BatchMeta meta{};
};

template <int KP>
struct BOps {
  using L = Lay<KP>;
  using UpdFn = void (*)(BatchMeta);
  static bool use_tc(bool tc) { return tc && TcUpd<KP>::ON; }
  static UpdFn upd_fn(bool mixed, bool tc) {
    if constexpr (TcUpd<KP>::ON) {
      if (tc) return mixed ? batch_update_kernel<KP, true, true> : batch_update_kernel<KP, false, true>;
    }
    return mixed ? batch_update_kernel<KP, true, false> : batch_update_kernel<KP, false, false>;
  }
  static size_t upd_smem(bool tc) { return use_tc(tc) ? TcUpd<KP>::smem() : update_smem_bytes<KP>(); }
  static cudaError_t setup() {
    for (int v = 0; v < (TcUpd<KP>::ON ? 4 : 2); ++v) {
      const bool mixed = v & 1, tc = v >> 1;
      cudaError_t e = cudaFuncSetAttribute(upd_fn(mixed, tc), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)upd_smem(tc));
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  static void grids(BatchClass& bc, int sms) {
    int o1 = 0, o2 = 0;
    const size_t smem = upd_smem(bc.tc);
    if (bc.mixed) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, batch_spmm_kernel<KP, true>, L::NT, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o1, batch_spmm_kernel<KP, false>, L::NT, 0);
    if (use_tc(bc.tc)) o2 = tc_blocks_per_sm((const void*)upd_fn(bc.mixed, true), L::NT, smem, TcUpd<KP>::TMEM_COLS);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o2, upd_fn(bc.mixed, false), L::NT, smem);
    bc.occ_spmm = std::max(1, o1);
    bc.occ_upd = std::max(1, o2);
    // untuned default: a class whose units of kRowsPerUnit rows per team leave
    // resident gather warps idle takes one-row units (shape 1; shorter chains
    // of dependent loads per unit, the same sums)
    if (!bc.tuned && bc.units_s[0] < (int64_t)sms * bc.occ_spmm * L::WARPS) {
      bc.shape = 1;
      bc.units = bc.units_s[1];
      bc.d_unit_base = bc.d_ub[1];
    }
    bc.spmm_grid = sms * std::max(1, o1);
    bc.gather_blocks_max = std::max<int64_t>(1, (bc.units + L::WARPS - 1) / L::WARPS);
    bc.spmm_grid = (int)std::min<int64_t>(bc.spmm_grid, bc.gather_blocks_max);
    bc.upd_grid = std::max(1, std::min(sms * std::max(1, o2), bc.n_items));
    const int64_t fin_threads = bc.heavy * L::T;
    bc.fin_grid = (int)std::max<int64_t>(1, std::min<int64_t>((fin_threads + 255) / 256, 4096));
  }
  // the gather of shape `shape` (its own unit table)
  template <int S>
  static void spmm_s(const BatchClass& bc, int grid, cudaStream_t s) {
    BatchMeta m = bc.meta;
    m.unit_base = bc.d_ub[S];
    if (bc.mixed) batch_spmm_kernel<KP, true, S><<<grid, L::NT, 0, s>>>(m);
    else batch_spmm_kernel<KP, false, S><<<grid, L::NT, 0, s>>>(m);
  }
  static void spmm(const BatchClass& bc, int shape, int grid, cudaStream_t s) {
    static_assert(kGatherShapes == 3, "gather shapes");
    if (shape == 1) spmm_s<1>(bc, grid, s);
    else if (shape == 2) spmm_s<2>(bc, grid, s);
    else spmm_s<0>(bc, grid, s);
  }
  static void iteration(const BatchClass& bc, cudaStream_t s) {
    cudaMemsetAsync(bc.d_work, 0, 2 * sizeof(unsigned long long), s);
    spmm(bc, bc.shape, bc.spmm_grid, s);
    if (bc.heavy > 0) batch_finalize_kernel<KP><<<bc.fin_grid, 256, 0, s>>>(bc.meta);
    upd_fn(bc.mixed, bc.tc)<<<bc.upd_grid, L::NT, upd_smem(bc.tc), s>>>(bc.meta);
    batch_fold_kernel<KP><<<(int)bc.members.size() * fold_blocks<KP>(false), 256, 0, s>>>(bc.meta);
  }
  template <int S>
  static int64_t units_s(const cluster_ctx* c) {
    constexpr int R1 = BShape<KP, true, S>::RPU, R0 = BShape<KP, false, S>::RPU;
    return c->mixed ? spmm_units<KP, true, R1>(c->n, c->n_heavy, c->n_chunks)
                    : spmm_units<KP, false, R0>(c->n, c->n_heavy, c->n_chunks);
  }
  static int64_t units(const cluster_ctx* c, int shape) {
    return shape == 1 ? units_s<1>(c) : shape == 2 ? units_s<2>(c) : units_s<0>(c);
  }
  static int nb(bool mixed, int shape) {
    if (mixed) return shape == 2 ? BShape<KP, true, 2>::NB : BShape<KP, true, 0>::NB;
    return shape == 2 ? BShape<KP, false, 2>::NB : BShape<KP, false, 0>::NB;
  }
  static int rpu(int shape) { return shape == 1 ? BShape<KP, false, 1>::RPU : BShape<KP, false, 0>::RPU; }
  // one iteration with events around the two persistent kernels
  static void timed_iteration(const BatchClass& bc, int shape, int spmm_grid, int upd_grid, cudaEvent_t* ev,
                              cudaStream_t s) {
    cudaMemsetAsync(bc.d_work, 0, 2 * sizeof(unsigned long long), s);
    cudaEventRecord(ev[0], s);
    spmm(bc, shape, spmm_grid, s);
    cudaEventRecord(ev[1], s);
    if (bc.heavy > 0) batch_finalize_kernel<KP><<<bc.fin_grid, 256, 0, s>>>(bc.meta);
    cudaEventRecord(ev[2], s);
    upd_fn(bc.mixed, bc.tc)<<<upd_grid, L::NT, upd_smem(bc.tc), s>>>(bc.meta);
    cudaEventRecord(ev[3], s);
    batch_fold_kernel<KP><<<(int)bc.members.size() * fold_blocks<KP>(false), 256, 0, s>>>(bc.meta);
  }
};

#define FC_BDISPATCH(KPV, CALL)                      \
  switch (KPV) {                                     \
    case 2: { using Ops = BOps<2>; CALL; } break;    \
    case 4: { using Ops = BOps<4>; CALL; } break;    \
    case 8: { using Ops = BOps<8>; CALL; } break;    \
    case 16: { using Ops = BOps<16>; CALL; } break;  \
    case 32: { using Ops = BOps<32>; CALL; } break;  \
    case 64: { using Ops = BOps<64>; CALL; } break;  \
    default: { using Ops = BOps<128>; CALL; } break; \
  }

}  // namespace

struct cluster_batch {
  int dev = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cluster_options opt{};
  std::vector<cluster_ctx*> inst;
  std::vector<BatchClass> classes;
  FistaState** d_all_states = nullptr;
  FistaState* d_collect = nullptr;
  std::vector<FistaState> h_collect;
  int graph_chunk = 16;
  cudaGraphExec_t graph = nullptr;
  std::vector<cudaStream_t> branch;  // one capture stream per class
  std::vector<cudaEvent_t> ev;       // fork event + one join event per class
  bool owns = true;                  // destroy frees the instances too
};

// Free the per-class tables, state arrays and graph (not the instances).
static void batch_release_tables(cluster_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  for (auto& bc : b->classes) {
    void* ps[] = {bc.d_args, bc.d_folds, bc.d_ub[0], bc.d_ub[1], bc.d_ub[2], bc.d_heavy_base, bc.d_item_inst,
                  bc.d_item_slot, bc.d_parts, bc.d_states, bc.d_work};
    for (void* p : ps)
      if (p) cudaFree(p);
  }
  b->classes.clear();
  if (b->d_all_states) cudaFree(b->d_all_states);
  if (b->d_collect) cudaFree(b->d_collect);
  b->d_all_states = nullptr;
  b->d_collect = nullptr;
}

static void batch_free(cluster_batch* b) {
  if (!b) return;
  batch_release_tables(b);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  for (cudaStream_t st : b->branch) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  if (b->owns)
    for (cluster_ctx* c : b->inst) ctx_free(c);
  delete b;
}

template <typename T>
static cluster_status upload(T** dst, const std::vector<T>& src, cudaStream_t s) {
  FC_CUDA(cudaMalloc(dst, sizeof(T) * std::max<size_t>(1, src.size())));
  if (!src.empty()) FC_CUDA(cudaMemcpyAsync(*dst, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice, s));
  return CLUSTER_OK;
}

static cluster_status build_class(cluster_batch* b, BatchClass& bc, int sms) {
  cudaStream_t s = b->stream;
  std::vector<PassArgs> args;
  std::vector<FoldArgs> folds;
  std::vector<int64_t> ubase[kGatherShapes], hbase(1, 0);
  for (auto& u : ubase) u.assign(1, 0);
  std::vector<int32_t> item_inst, item_slot, parts;
  std::vector<FistaState*> states;
  for (size_t j = 0; j < bc.members.size(); ++j) {
    const cluster_ctx* c = b->inst[bc.members[j]];
    args.push_back(make_pass_args(c, false));
    FoldArgs f = make_fold_args(c, 0, 0);
    f.work = nullptr;  // the batch zeroes its own counters
    folds.push_back(f);
    for (int sh = 0; sh < kGatherShapes; ++sh) {
      int64_t u = 0;
      FC_BDISPATCH(bc.KP, u = Ops::units(c, sh));
      ubase[sh].push_back(ubase[sh].back() + u);
    }
    hbase.push_back(hbase.back() + c->n_heavy);
    parts.push_back(c->parts_upd);
    for (int sl = 0; sl < c->parts_upd; ++sl) {
      item_inst.push_back((int32_t)j);
      item_slot.push_back(sl);
    }
    states.push_back(c->st);
  }
  for (int sh = 0; sh < kGatherShapes; ++sh) bc.units_s[sh] = ubase[sh].back();
  bc.units = bc.units_s[0];
  bc.heavy = hbase.back();
  bc.n_items = (int)item_inst.size();
  FC_TRY(upload(&bc.d_args, args, s));
  FC_TRY(upload(&bc.d_folds, folds, s));
  for (int sh = 0; sh < kGatherShapes; ++sh) FC_TRY(upload(&bc.d_ub[sh], ubase[sh], s));
  bc.d_unit_base = bc.d_ub[0];
  FC_TRY(upload(&bc.d_heavy_base, hbase, s));
  FC_TRY(upload(&bc.d_item_inst, item_inst, s));
  FC_TRY(upload(&bc.d_item_slot, item_slot, s));
  FC_TRY(upload(&bc.d_parts, parts, s));
  FC_TRY(upload(&bc.d_states, states, s));
  FC_CUDA(cudaMalloc(&bc.d_work, 2 * sizeof(unsigned long long)));
  FC_CUDA(cudaMemsetAsync(bc.d_work, 0, 2 * sizeof(unsigned long long), s));
  BatchMeta& m = bc.meta;
  m.args = bc.d_args;
  m.folds = bc.d_folds;
  m.unit_base = bc.d_unit_base;
  m.heavy_base = bc.d_heavy_base;
  m.item_inst = bc.d_item_inst;
  m.item_slot = bc.d_item_slot;
  m.parts_upd = bc.d_parts;
  m.states = bc.d_states;
  m.m = (int32_t)bc.members.size();
  m.n_items = bc.n_items;
  m.work = bc.d_work;
  FC_CUDA(cudaSetDevice(b->dev));
  cudaError_t e = cudaSuccess;
  FC_BDISPATCH(bc.KP, e = Ops::setup());
  FC_CUDA(e);
  FC_BDISPATCH(bc.KP, Ops::grids(bc, sms));
  return CLUSTER_OK;
}

// Graph of graph_chunk iterations of every class.  Classes share no data, so
// each class's chain of iterations is its own branch of the graph (fork at
// the start, join at the end) and the classes' kernels overlap on the GPU.
static cluster_status capture_batch_graph(cluster_batch* b) {
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  const size_t ncls = b->classes.size();
  while (b->branch.size() < ncls) {
    cudaStream_t st = nullptr;
    FC_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    b->branch.push_back(st);
  }
  while (b->ev.size() < ncls + 1) {
    cudaEvent_t e = nullptr;
    FC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->ev.push_back(e);
  }
  cudaGraph_t g = nullptr;
  FC_CUDA(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
  FC_CUDA(cudaEventRecord(b->ev[0], b->cap_stream));
  for (size_t ci = 0; ci < ncls; ++ci) {
    const BatchClass& bc = b->classes[ci];
    FC_CUDA(cudaStreamWaitEvent(b->branch[ci], b->ev[0], 0));
    for (int i = 0; i < b->graph_chunk; ++i) FC_BDISPATCH(bc.KP, Ops::iteration(bc, b->branch[ci]));
    FC_CUDA(cudaEventRecord(b->ev[ci + 1], b->branch[ci]));
    FC_CUDA(cudaStreamWaitEvent(b->cap_stream, b->ev[ci + 1], 0));
  }
  FC_CUDA(cudaStreamEndCapture(b->cap_stream, &g));
  cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  FC_CUDA(e);
  return CLUSTER_OK;
}

// Group b->inst into classes, upload the tables and capture the graph.
static cluster_status batch_assemble(cluster_batch* b) {
  batch_release_tables(b);
  const int count = (int)b->inst.size();
  if (count == 0) return CLUSTER_OK;
  std::map<std::pair<int, int>, int> cls;
  for (int i = 0; i < count; ++i) {
    const cluster_ctx* c = b->inst[i];
    const auto key = std::make_pair(c->KP, c->mixed ? 1 : 0);
    auto it = cls.find(key);
    if (it == cls.end()) {
      BatchClass bc;
      bc.KP = c->KP;
      bc.mixed = c->mixed;
      bc.tc = c->tc_update;
      cls[key] = (int)b->classes.size();
      b->classes.push_back(bc);
      it = cls.find(key);
    }
    b->classes[it->second].members.push_back(i);
  }
  int sms = 0;
  FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev));
  for (auto& bc : b->classes) FC_TRY(build_class(b, bc, sms));
  std::vector<FistaState*> all;
  for (cluster_ctx* c : b->inst) all.push_back(c->st);
  FC_TRY(upload(&b->d_all_states, all, b->stream));
  FC_CUDA(cudaMalloc(&b->d_collect, sizeof(FistaState) * count));
  b->h_collect.resize(count);
  FC_CUDA(cudaStreamSynchronize(b->stream));
  return capture_batch_graph(b);
}

static cluster_status batch_create_impl(cluster_batch* b, int32_t count, const cluster_csr* S, const int32_t* k,
                                        const float* const* U0, const cluster_options* optp, void* stream) {
  if (count < 1) FC_EINVAL("count must be >= 1");
  if (!S || !k || !U0) FC_EINVAL("NULL argument");
  cluster_options opt;
  if (optp) opt = *optp;
  else cluster_options_default(&opt);
  if (opt.fused_pass) FC_EINVAL("batched solves use the split iteration (fused_pass must be 0)");
  if (opt.graph_chunk < 1) opt.graph_chunk = 16;
  b->opt = opt;
  b->stream = (cudaStream_t)stream;
  b->graph_chunk = opt.graph_chunk;
  FC_CUDA(cudaGetDevice(&b->dev));
  FC_CUDA(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
  for (int32_t i = 0; i < count; ++i) {
    cluster_ctx* c = new (std::nothrow) cluster_ctx();
    if (!c) {
      set_error("out of host memory");
      return CLUSTER_ENOMEM;
    }
    b->inst.push_back(c);
    cluster_status st = init_impl(&S[i], k[i], U0[i], &opt, stream, c, false);
    if (st != CLUSTER_OK) {
      set_error("instance %d: %s", i, cluster_last_error());
      return st;
    }
  }
  return batch_assemble(b);
}

extern "C" cluster_status cluster_batch_create(int32_t count, const cluster_csr* S, const int32_t* k,
                                               const float* const* U0, const cluster_options* opt, void* stream,
                                               cluster_batch** out) {
  clear_error();
  if (!out) FC_EINVAL("out is NULL");
  *out = nullptr;
  cluster_batch* b = new (std::nothrow) cluster_batch();
  if (!b) {
    set_error("out of host memory");
    return CLUSTER_ENOMEM;
  }
  cluster_status st = batch_create_impl(b, count, S, k, U0, opt, stream);
  if (st != CLUSTER_OK) {
    cudaStreamSynchronize((cudaStream_t)stream);
    batch_free(b);
    return st;
  }
  *out = b;
  return CLUSTER_OK;
}

static cluster_status batch_read(cluster_batch* b, cluster_report* reps) {
  const int m = (int)b->inst.size();
  if (m == 0) return CLUSTER_OK;
  batch_collect_kernel<<<m, 64, 0, b->stream>>>(b->d_all_states, m, b->d_collect);
  FC_CUDA(cudaGetLastError());
  FC_CUDA(cudaMemcpyAsync(b->h_collect.data(), b->d_collect, sizeof(FistaState) * m, cudaMemcpyDeviceToHost,
                          b->stream));
  FC_CUDA(cudaStreamSynchronize(b->stream));
  for (int i = 0; i < m; ++i) {
    b->inst[i]->host_st = b->h_collect[i];
    if (reps) fill_report(b->inst[i], &reps[i]);
  }
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_batch_enqueue(cluster_batch* b, int64_t iters) {
  clear_error();
  if (!b) FC_EINVAL("batch is NULL");
  if (iters < 0) FC_EINVAL("iters must be >= 0");
  if (iters == 0 || b->inst.empty()) return CLUSTER_OK;
  FC_CUDA(cudaSetDevice(b->dev));
  const int m = (int)b->inst.size();
  batch_set_limit_kernel<<<(m + 255) / 256, 256, 0, b->stream>>>(b->d_all_states, m, iters);
  const int64_t reps = (iters + b->graph_chunk - 1) / b->graph_chunk;
  for (int64_t r = 0; r < reps; ++r) FC_CUDA(cudaGraphLaunch(b->graph, b->stream));
  FC_CUDA(cudaGetLastError());
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_batch_step(cluster_batch* b, int64_t iters, cluster_report* reps) {
  FC_TRY(cluster_batch_enqueue(b, iters));
  return batch_read(b, reps);
}

extern "C" cluster_status cluster_batch_get_U(cluster_batch* b, int32_t i, float* U_out) {
  clear_error();
  if (!b || !U_out) FC_EINVAL("NULL argument");
  if (i < 0 || i >= (int32_t)b->inst.size()) FC_EINVAL("instance index %d out of range", i);
  return cluster_get_U(b->inst[i], U_out);
}

// Tile and launch shapes per class, chosen by timing.  The gather's
// candidates are its tile shapes (BShape: nonzeros per batch, rows per work
// unit) times 1..occupancy resident blocks per SM; then the update kernel's
// 1..occupancy blocks per SM with the chosen gather.  Every trial is a real
// iteration of all unfinished instances; no shape changes a value (each row is
// summed by one team in index order, update items are the instances' solo
// blocks), so tuning does not perturb the solve.  The graph is re-captured
// with the chosen shapes.
extern "C" cluster_status cluster_batch_autotune(cluster_batch* b, int32_t trials) {
  clear_error();
  if (!b) FC_EINVAL("batch is NULL");
  if (trials < 1) trials = 1;
  FC_CUDA(cudaSetDevice(b->dev));
  int sms = 0;
  FC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev));
  const int m = (int)b->inst.size();
  const int ncls = (int)b->classes.size();
  std::vector<int> ng(ncls);  // gather candidates of each class
  int max_cand = 1;
  for (int ci = 0; ci < ncls; ++ci) {
    const BatchClass& bc = b->classes[ci];
    ng[ci] = kGatherShapes * bc.occ_spmm;
    max_cand = std::max(max_cand, ng[ci] + bc.occ_upd);
  }
  auto gather_grid = [&](const BatchClass& bc, int shape, int per_sm) {
    int warps = 8;
    FC_BDISPATCH(bc.KP, warps = Ops::L::WARPS);
    const int64_t bmax = std::max<int64_t>(1, (bc.units_s[shape] + warps - 1) / warps);
    return (int)std::min<int64_t>((int64_t)sms * per_sm, bmax);
  };
  std::vector<cudaEvent_t> ev((size_t)ncls * 4);
  for (auto& e : ev) FC_CUDA(cudaEventCreate(&e));
  std::vector<int> best_s(ncls), best_u(ncls), best_sh(ncls);
  std::vector<double> best_g(ncls, 1e30), best_t(ncls, 1e30), cur(ncls, 1e30);
  for (int ci = 0; ci < ncls; ++ci) {
    best_s[ci] = b->classes[ci].spmm_grid;
    best_u[ci] = b->classes[ci].upd_grid;
    best_sh[ci] = b->classes[ci].shape;
  }
  cluster_status st = CLUSTER_OK;
  for (int cand = 0; cand < max_cand && st == CLUSTER_OK; ++cand) {
    std::fill(cur.begin(), cur.end(), 1e30);
    std::vector<int> gs(ncls), gu(ncls), sh(ncls);
    for (int ci = 0; ci < ncls; ++ci) {
      const BatchClass& bc = b->classes[ci];
      if (cand < ng[ci]) {
        sh[ci] = cand / bc.occ_spmm;
        gs[ci] = gather_grid(bc, sh[ci], cand % bc.occ_spmm + 1);
        gu[ci] = bc.upd_grid;
      } else {
        const int cu = std::min(cand - ng[ci], bc.occ_upd - 1);
        sh[ci] = best_sh[ci];
        gs[ci] = best_s[ci];
        gu[ci] = std::max(1, std::min(sms * (cu + 1), bc.n_items));
      }
    }
    for (int rep = 0; rep < trials && st == CLUSTER_OK; ++rep) {
      batch_set_limit_kernel<<<(m + 255) / 256, 256, 0, b->stream>>>(b->d_all_states, m, 1);
      for (int ci = 0; ci < ncls; ++ci) {
        BatchClass& bc = b->classes[ci];
        FC_BDISPATCH(bc.KP, Ops::timed_iteration(bc, sh[ci], gs[ci], gu[ci], &ev[(size_t)ci * 4], b->stream));
      }
      cudaError_t e = cudaStreamSynchronize(b->stream);
      if (e != cudaSuccess) {
        set_error("autotune: %s", cudaGetErrorString(e));
        st = CLUSTER_ECUDA;
        break;
      }
      for (int ci = 0; ci < ncls; ++ci) {
        float ms_s = 0.f, ms_u = 0.f;
        cudaEventElapsedTime(&ms_s, ev[(size_t)ci * 4 + 0], ev[(size_t)ci * 4 + 1]);
        cudaEventElapsedTime(&ms_u, ev[(size_t)ci * 4 + 2], ev[(size_t)ci * 4 + 3]);
        cur[ci] = std::min(cur[ci], (double)(cand < ng[ci] ? ms_s : ms_u));
      }
    }
    if (st != CLUSTER_OK) break;
    for (int ci = 0; ci < ncls; ++ci) {
      BatchClass& bc = b->classes[ci];
      if (cand < ng[ci]) {
        if (cur[ci] < best_g[ci]) {
          best_g[ci] = cur[ci];
          best_sh[ci] = sh[ci];
          best_s[ci] = gs[ci];
          bc.gather_ms = cur[ci];
        }
      } else if (cand - ng[ci] < bc.occ_upd && cur[ci] < best_t[ci]) {
        best_t[ci] = cur[ci];
        best_u[ci] = gu[ci];
        bc.update_ms = cur[ci];
      }
    }
  }
  for (auto& e : ev) cudaEventDestroy(e);
  if (st != CLUSTER_OK) return st;
  for (int ci = 0; ci < ncls; ++ci) {
    BatchClass& bc = b->classes[ci];
    bc.shape = best_sh[ci];
    bc.d_unit_base = bc.d_ub[bc.shape];
    bc.meta.unit_base = bc.d_unit_base;
    bc.units = bc.units_s[bc.shape];
    bc.spmm_grid = best_s[ci];
    bc.upd_grid = best_u[ci];
    bc.tuned = true;
  }
  FC_TRY(capture_batch_graph(b));
  return batch_read(b, nullptr);
}

// Classes and launch shapes as JSON (for reports).
extern "C" cluster_status cluster_batch_describe(cluster_batch* b, char* buf, size_t len) {
  clear_error();
  if (!b || !buf || len == 0) FC_EINVAL("NULL argument");
  std::string out = "{\"instances\": " + std::to_string(b->inst.size()) + ", \"classes\": [";
  for (size_t ci = 0; ci < b->classes.size(); ++ci) {
    const BatchClass& bc = b->classes[ci];
    int nbv = 0, rpu = 0;
    FC_BDISPATCH(bc.KP, (nbv = Ops::nb(bc.mixed, bc.shape), rpu = Ops::rpu(bc.shape)));
    char tmp[640];
    snprintf(tmp, sizeof(tmp),
             "%s{\"kp\": %d, \"mixed\": %d, \"instances\": %zu, \"gather_units\": %lld, \"chunked_rows\": %lld, "
             "\"update_items\": %d, \"gather_shape\": %d, \"gather_nonzeros_per_batch\": %d, "
             "\"gather_rows_per_unit\": %d, \"gather_blocks\": %d, \"update_blocks\": %d, \"tuned\": %d, "
             "\"gather_ms\": %.4f, \"update_ms\": %.4f}",
             ci ? ", " : "", bc.KP, bc.mixed ? 1 : 0, bc.members.size(), (long long)bc.units, (long long)bc.heavy,
             bc.n_items, bc.shape, nbv, rpu, bc.spmm_grid, bc.upd_grid, bc.tuned ? 1 : 0, bc.gather_ms, bc.update_ms);
    out += tmp;
  }
  out += "]}";
  if (out.size() + 1 > len) FC_EINVAL("buffer too small (%zu bytes needed)", out.size() + 1);
  memcpy(buf, out.c_str(), out.size() + 1);
  return CLUSTER_OK;
}

extern "C" void cluster_batch_destroy(cluster_batch* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  cudaStreamSynchronize(b->stream);
  batch_free(b);
}

// ---------------------------------------------------------------------------
// non-owning batches over instances owned by someone else (the server)
// ---------------------------------------------------------------------------
namespace fc {

cluster_status batch_view_new(void* stream, int graph_chunk, cluster_batch** out) {
  cluster_batch* b = new (std::nothrow) cluster_batch();
  if (!b) {
    set_error("out of host memory");
    return CLUSTER_ENOMEM;
  }
  b->owns = false;
  b->stream = (cudaStream_t)stream;
  b->graph_chunk = graph_chunk < 1 ? 16 : graph_chunk;
  cudaError_t e = cudaGetDevice(&b->dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete b;
    set_error("batch view: %s", cudaGetErrorString(e));
    return CLUSTER_ECUDA;
  }
  *out = b;
  return CLUSTER_OK;
}

cluster_status batch_view_set(cluster_batch* b, const std::vector<cluster_ctx*>& members) {
  b->inst = members;
  return batch_assemble(b);
}

cluster_status batch_view_run(cluster_batch* b, int64_t iters) {
  FC_TRY(cluster_batch_enqueue(b, iters));
  return batch_read(b, nullptr);
}

void batch_view_delete(cluster_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
}

}  // namespace fc
