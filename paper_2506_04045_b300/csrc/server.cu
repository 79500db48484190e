// Serving loop with continuous batching.
//
// A worker thread owns the device work.  Requests (a host CSR, k and a host
// start point) are queued by cluster_server_submit; the worker admits them in
// arrival order while their estimated device footprint fits the memory
// budget, keeps every admitted solve resident, and advances all resident
// solves together, `iters_per_tick` iterations per tick, through the batched
// segmented launches.  After each tick, solves whose stop rule fired (or that
// reached max_iter) get their final objective, are copied to the host and
// freed, and the freed memory admits queued requests.  A solve's arithmetic
// does not depend on what else is resident, so every result equals the same
// request solved alone.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "init_kernels.cuh"
#include "solver_impl.h"
#include "util.h"

using namespace fc;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  int64_t n = 0, nnz = 0;
  int32_t k = 0;
  // inputs: owned copies, or the caller's arrays (borrow_host)
  std::vector<int64_t> rp;
  std::vector<int32_t> col;
  std::vector<float> val;
  std::vector<float> U0;
  const void* b_rp = nullptr;
  int32_t b_index64 = 1;
  const int32_t* b_col = nullptr;
  const float* b_val = nullptr;
  const float* b_U0 = nullptr;
  bool borrowed = false;
  size_t host_bytes = 0;
  size_t footprint = 0;
  // device resources while resident
  int64_t* d_rp = nullptr;
  int32_t* d_col = nullptr;
  float* d_val = nullptr;
  cluster_ctx* ctx = nullptr;
  // result
  std::vector<float> U;
  cluster_report rep{};
  cluster_status status = CLUSTER_OK;
  std::string err;
  double t_submit = 0, t_admit = 0, t_done = 0;
  int state = 0;  // 0 queued, 1 resident, 2 finished
};

int padded(int k) {
  int kp = 2;
  while (kp < k) kp <<= 1;
  return kp;
}

}  // namespace

struct cluster_server {
  cluster_server_options opt{};
  int dev = 0;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> queue;
  std::vector<Request*> resident;
  std::unordered_map<uint64_t, Request*> all;
  uint64_t next_ticket = 1;
  bool stop = false;
  size_t used = 0;
  size_t queued_host = 0;
  cluster_server_stats stats{};
  double busy_t0 = 0;
};

// Device bytes a request needs while resident (CSR, iterates and stored
// products, schedule, partials) plus the transient set-up scratch.
static size_t footprint(int64_t n, int64_t nnz, int k, const cluster_options& o) {
  const size_t kp = (size_t)padded(k);
  const bool mixed = o.precision == CLUSTER_MIXED_BF16;
  size_t b = 8 * (size_t)(n + 1) + 8 * (size_t)nnz + (mixed ? 2 * (size_t)nnz : 0);
  b += (size_t)n * kp * 4 * 4 + (mixed ? (size_t)n * kp * 2 * 2 : 0);
  b += 4 * (size_t)n + 28 * (size_t)n;             // row order + set-up scratch
  b += (size_t)600 * 2 * kp * kp * 4 + 8 * kp * kp * 4;  // per-block Gram partials, fold buffers
  b += (size_t)2 << 20;
  return b;
}

static void finish(cluster_server* sv, Request* r, cluster_status st, const std::string& err) {
  r->status = st;
  r->err = err;
  r->t_done = now_s();
  r->state = 2;
  r->rp.clear();
  r->rp.shrink_to_fit();
  r->col.clear();
  r->col.shrink_to_fit();
  r->val.clear();
  r->val.shrink_to_fit();
  r->U0.clear();
  r->U0.shrink_to_fit();
  if (st == CLUSTER_OK) sv->stats.completed++;
  else sv->stats.failed++;
}

static void release_device(Request* r) {
  if (r->ctx) ctx_free(r->ctx);
  r->ctx = nullptr;
  if (r->d_rp) cudaFree(r->d_rp);
  if (r->d_col) cudaFree(r->d_col);
  if (r->d_val) cudaFree(r->d_val);
  r->d_rp = nullptr;
  r->d_col = nullptr;
  r->d_val = nullptr;
}

// Upload and initialise one admitted request on the worker's stream.
static cluster_status admit(cluster_server* sv, Request* r, cudaStream_t s) {
  if (r->borrowed) {
    // row pointers are uploaded as int64; widen an int32 array first
    if (r->b_index64) {
      r->rp.clear();
    } else {
      const int32_t* p = (const int32_t*)r->b_rp;
      r->rp.resize(r->n + 1);
      for (int64_t i = 0; i <= r->n; ++i) r->rp[i] = p[i];
    }
  }
  const int64_t* h_rp = (r->borrowed && r->b_index64) ? (const int64_t*)r->b_rp : r->rp.data();
  const int32_t* h_col = r->borrowed ? r->b_col : r->col.data();
  const float* h_val = r->borrowed ? r->b_val : r->val.data();
  const float* h_U0 = r->borrowed ? r->b_U0 : r->U0.data();
  float* d_U0 = nullptr;
  cudaError_t e = cudaMalloc(&r->d_rp, sizeof(int64_t) * (r->n + 1));
  if (e == cudaSuccess && r->nnz > 0) e = cudaMalloc(&r->d_col, sizeof(int32_t) * r->nnz);
  if (e == cudaSuccess && r->nnz > 0) e = cudaMalloc(&r->d_val, sizeof(float) * r->nnz);
  if (e == cudaSuccess) e = cudaMalloc(&d_U0, sizeof(float) * r->n * r->k);
  if (e == cudaSuccess) e = cudaMemcpyAsync(r->d_rp, h_rp, sizeof(int64_t) * (r->n + 1), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && r->nnz > 0)
    e = cudaMemcpyAsync(r->d_col, h_col, sizeof(int32_t) * r->nnz, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && r->nnz > 0)
    e = cudaMemcpyAsync(r->d_val, h_val, sizeof(float) * r->nnz, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_U0, h_U0, sizeof(float) * r->n * r->k, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    if (d_U0) cudaFree(d_U0);
    set_error("admission: %s", cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? CLUSTER_ENOMEM : CLUSTER_ECUDA;
  }
  cluster_csr S;
  memset(&S, 0, sizeof(S));
  S.n = r->n;
  S.nnz = r->nnz;
  S.index64 = 1;
  S.row_ptr = r->d_rp;
  S.col = r->d_col;
  S.val = r->d_val;
  cluster_options o = sv->opt.solve;
  o.borrow = 1;       // the request's device arrays live as long as the solve
  o.fused_pass = 0;
  r->ctx = new (std::nothrow) cluster_ctx();
  cluster_status st = r->ctx ? init_impl(&S, r->k, d_U0, &o, s, r->ctx, false) : CLUSTER_ENOMEM;
  cudaStreamSynchronize(s);
  cudaFree(d_U0);
  if (st == CLUSTER_OK && r->ctx->relabeled) {
    // the context keeps its own renumbered copy of S: the uploaded one is no
    // longer referenced (the footprint counts one copy)
    cudaFree(r->d_rp);
    cudaFree(r->d_col);
    cudaFree(r->d_val);
    r->d_rp = nullptr;
    r->d_col = nullptr;
    r->d_val = nullptr;
  }
  // the device has its own copy now
  r->rp.clear();
  r->rp.shrink_to_fit();
  r->col.clear();
  r->col.shrink_to_fit();
  r->val.clear();
  r->val.shrink_to_fit();
  r->U0.clear();
  r->U0.shrink_to_fit();
  return st;
}

// Final objective and host copy of a finished solve.
static cluster_status harvest(Request* r, cudaStream_t s) {
  cluster_ctx* c = r->ctx;
  FC_TRY(finalize_loss(c));
  fill_report(c, &r->rep);
  float* d_U = nullptr;
  FC_CUDA(cudaMalloc(&d_U, sizeof(float) * c->n * c->k));
  unpad_output(c, c->X[c->host_st.out_iter & 1], d_U, s);
  r->U.resize((size_t)c->n * c->k);
  cudaError_t e = cudaMemcpyAsync(r->U.data(), d_U, sizeof(float) * r->U.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(d_U);
  if (e != cudaSuccess) {
    set_error("copy-out: %s", cudaGetErrorString(e));
    return CLUSTER_ECUDA;
  }
  return CLUSTER_OK;
}

static void worker_main(cluster_server* sv) {
  cudaSetDevice(sv->dev);
  cudaStream_t s = nullptr;
  cluster_batch* view = nullptr;
  bool ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
            batch_view_new(s, sv->opt.solve.graph_chunk, &view) == CLUSTER_OK;
  std::vector<Request*> resident;
  for (;;) {
    std::vector<Request*> admits;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      if (!ok) {
        // no stream: fail everything that arrives
        while (!sv->queue.empty()) {
          Request* r = sv->queue.front();
          sv->queue.pop_front();
          sv->queued_host -= r->host_bytes;
          finish(sv, r, CLUSTER_ECUDA, "server could not create its CUDA stream");
        }
        sv->cv_done.notify_all();
        if (sv->stop) break;
        sv->cv_work.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
        continue;
      }
      if (sv->stop) break;
      while (!sv->queue.empty()) {
        Request* r = sv->queue.front();
        if (r->footprint > sv->opt.hbm_budget) {  // can never fit
          sv->queue.pop_front();
          sv->queued_host -= r->host_bytes;
          finish(sv, r, CLUSTER_ENOMEM, "request needs more device memory than the server budget");
          continue;
        }
        const size_t count = resident.size() + admits.size();
        if (sv->opt.max_resident > 0 && count >= (size_t)sv->opt.max_resident) break;
        if (sv->used + r->footprint > sv->opt.hbm_budget) break;
        sv->queue.pop_front();
        sv->used += r->footprint;
        sv->queued_host -= r->host_bytes;
        admits.push_back(r);
      }
      sv->cv_done.notify_all();
      if (resident.empty() && admits.empty()) {
        sv->cv_work.wait(lk, [&] { return sv->stop || !sv->queue.empty(); });
        continue;
      }
    }
    bool changed = false;
    for (Request* r : admits) {
      const double t = now_s();
      cluster_status st = admit(sv, r, s);
      std::lock_guard<std::mutex> lk(sv->mu);
      if (st != CLUSTER_OK) {
        std::string msg = cluster_last_error();
        release_device(r);
        sv->used -= r->footprint;
        finish(sv, r, st, msg);
      } else {
        r->t_admit = t;
        r->state = 1;
        resident.push_back(r);
        sv->stats.admitted++;
        changed = true;
      }
    }
    if (changed) {
      std::vector<cluster_ctx*> members;
      for (Request* r : resident) members.push_back(r->ctx);
      if (batch_view_set(view, members) != CLUSTER_OK) ok = false;
    }
    if (ok && !resident.empty()) {
      if (batch_view_run(view, sv->opt.iters_per_tick) != CLUSTER_OK) ok = false;
    }
    std::vector<Request*> keep, done;
    if (!ok) {
      std::string msg = cluster_last_error();
      std::lock_guard<std::mutex> lk(sv->mu);
      for (Request* r : resident) {
        release_device(r);
        sv->used -= r->footprint;
        finish(sv, r, CLUSTER_ECUDA, msg);
      }
      resident.clear();
      sv->cv_done.notify_all();
      continue;
    }
    for (Request* r : resident) (r->ctx->host_st.done ? done : keep).push_back(r);
    for (Request* r : done) {
      cluster_status st = harvest(r, s);
      std::string msg = st == CLUSTER_OK ? "" : cluster_last_error();
      release_device(r);
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->used -= r->footprint;
      finish(sv, r, st, msg);
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stats.ticks++;
      resident.swap(keep);
      sv->stats.resident = (int64_t)resident.size();
      sv->stats.resident_bytes = sv->used;
      sv->stats.queued = (int64_t)sv->queue.size();
      sv->cv_done.notify_all();
    }
    if (!done.empty()) {
      std::vector<cluster_ctx*> members;
      for (Request* r : resident) members.push_back(r->ctx);
      if (batch_view_set(view, members) != CLUSTER_OK) ok = false;
    }
  }
  // shutdown: drop everything still resident or queued
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (view) batch_view_set(view, {});
    for (Request* r : resident) {
      release_device(r);
      sv->used -= r->footprint;
      finish(sv, r, CLUSTER_EAGAIN, "server shut down before the solve finished");
    }
    while (!sv->queue.empty()) {
      Request* r = sv->queue.front();
      sv->queue.pop_front();
      sv->queued_host -= r->host_bytes;
      finish(sv, r, CLUSTER_EAGAIN, "server shut down before the request was admitted");
    }
    sv->cv_done.notify_all();
  }
  if (view) batch_view_delete(view);
  if (s) cudaStreamDestroy(s);
}

extern "C" void cluster_server_options_default(cluster_server_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  cluster_options_default(&o->solve);
  o->solve.stop_rule = CLUSTER_STOP_PG_REL;
  o->solve.tol = 1e-5;
  o->solve.max_iter = 5000;
  o->hbm_budget = 0;
  o->iters_per_tick = 64;
  o->max_resident = 0;
}

extern "C" cluster_status cluster_server_create(const cluster_server_options* opt, cluster_server** out) {
  clear_error();
  if (!out) FC_EINVAL("out is NULL");
  *out = nullptr;
  cluster_server_options o;
  if (opt) o = *opt;
  else cluster_server_options_default(&o);
  if (o.iters_per_tick < 1) FC_EINVAL("iters_per_tick must be >= 1");
  if (o.solve.max_iter < 1) FC_EINVAL("max_iter must be >= 1");
  if (o.solve.fused_pass) FC_EINVAL("the server uses the split iteration (fused_pass must be 0)");
  cluster_server* sv = new (std::nothrow) cluster_server();
  if (!sv) {
    set_error("out of host memory");
    return CLUSTER_ENOMEM;
  }
  cudaError_t e = cudaGetDevice(&sv->dev);
  if (e == cudaSuccess && o.hbm_budget == 0) {
    size_t free_b = 0, total_b = 0;
    e = cudaMemGetInfo(&free_b, &total_b);
    o.hbm_budget = free_b / 10 * 8;
  }
  if (e != cudaSuccess) {
    delete sv;
    set_error("server: %s", cudaGetErrorString(e));
    return CLUSTER_ECUDA;
  }
  sv->opt = o;
  sv->busy_t0 = now_s();
  try {
    sv->worker = std::thread(worker_main, sv);
  } catch (...) {
    delete sv;
    set_error("server: could not start the worker thread");
    return CLUSTER_ENOMEM;
  }
  *out = sv;
  return CLUSTER_OK;
}

extern "C" cluster_status cluster_server_submit(cluster_server* sv, const cluster_csr* S, int32_t k, const float* U0,
                                                uint64_t* ticket) {
  clear_error();
  if (!sv || !S || !U0 || !ticket) FC_EINVAL("NULL argument");
  if (S->n < 1 || S->n > 0x7fffffffLL) FC_EINVAL("n must be in [1, 2^31)");
  if (S->nnz < 0 || !S->row_ptr || (S->nnz > 0 && (!S->col || !S->val))) FC_EINVAL("bad CSR arrays");
  if (k < 1 || k > 128) FC_EINVAL("k must be in [1, 128]");
  Request* r = new (std::nothrow) Request();
  if (!r) {
    set_error("out of host memory");
    return CLUSTER_ENOMEM;
  }
  r->n = S->n;
  r->nnz = S->nnz;
  r->k = k;
  const size_t bytes = 8 * (size_t)(S->n + 1) + 8 * (size_t)S->nnz + 4 * (size_t)S->n * k;
  if (sv->opt.borrow_host) {
    r->borrowed = true;
    r->b_rp = S->row_ptr;
    r->b_index64 = S->index64;
    r->b_col = S->col;
    r->b_val = S->val;
    r->b_U0 = U0;
  } else {
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      // an empty queue always takes one request, however large
      if (sv->opt.queue_bytes_max > 0 && sv->queued_host > 0 && sv->queued_host + bytes > sv->opt.queue_bytes_max) {
        sv->stats.rejected++;
        delete r;
        set_error("queue full: %zu bytes of requests wait for admission", sv->queued_host);
        return CLUSTER_EAGAIN;
      }
    }
    try {
      r->rp.resize(S->n + 1);
      if (S->index64) {
        memcpy(r->rp.data(), S->row_ptr, sizeof(int64_t) * (S->n + 1));
      } else {
        const int32_t* p = (const int32_t*)S->row_ptr;
        for (int64_t i = 0; i <= S->n; ++i) r->rp[i] = p[i];
      }
      r->col.assign(S->col, S->col + S->nnz);
      r->val.assign(S->val, S->val + S->nnz);
      r->U0.assign(U0, U0 + S->n * k);
    } catch (...) {
      delete r;
      set_error("out of host memory");
      return CLUSTER_ENOMEM;
    }
    r->host_bytes = bytes;
  }
  r->footprint = footprint(r->n, r->nnz, k, sv->opt.solve);
  r->t_submit = now_s();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) {
      delete r;
      set_error("server is shutting down");
      return CLUSTER_EAGAIN;
    }
    sv->queued_host += r->host_bytes;
    r->ticket = sv->next_ticket++;
    sv->all[r->ticket] = r;
    sv->queue.push_back(r);
    sv->stats.submitted++;
    sv->stats.queued = (int64_t)sv->queue.size();
  }
  sv->cv_work.notify_one();
  *ticket = r->ticket;
  return CLUSTER_OK;
}

// Hand a finished request to the caller (lock held); frees it.
static cluster_status take(cluster_server* sv, Request* r, float* U_out, cluster_report* rep,
                           cluster_request_times* times) {
  cluster_status st = r->status;
  if (times) {
    times->queue_s = (r->t_admit > 0 ? r->t_admit : r->t_done) - r->t_submit;
    times->run_s = r->t_admit > 0 ? r->t_done - r->t_admit : 0.0;
    times->total_s = r->t_done - r->t_submit;
  }
  if (st == CLUSTER_OK) {
    if (U_out) memcpy(U_out, r->U.data(), sizeof(float) * r->U.size());
    if (rep) *rep = r->rep;
  } else {
    set_error("%s", r->err.c_str());
  }
  sv->all.erase(r->ticket);
  delete r;
  return st;
}

extern "C" cluster_status cluster_server_poll(cluster_server* sv, uint64_t ticket, float* U_out, cluster_report* rep,
                                              cluster_request_times* times) {
  clear_error();
  if (!sv) FC_EINVAL("server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) FC_EINVAL("unknown ticket %llu", (unsigned long long)ticket);
  if (it->second->state != 2) return CLUSTER_EAGAIN;
  return take(sv, it->second, U_out, rep, times);
}

extern "C" cluster_status cluster_server_wait(cluster_server* sv, uint64_t ticket, double timeout_s, float* U_out,
                                              cluster_report* rep, cluster_request_times* times) {
  clear_error();
  if (!sv) FC_EINVAL("server is NULL");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->all.find(ticket);
  if (it == sv->all.end()) FC_EINVAL("unknown ticket %llu", (unsigned long long)ticket);
  Request* r = it->second;
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
  if (!sv->cv_done.wait_until(lk, deadline, [&] { return r->state == 2; })) {
    set_error("request %llu still pending after %.3f s", (unsigned long long)ticket, timeout_s);
    return CLUSTER_ETIMEOUT;
  }
  return take(sv, r, U_out, rep, times);
}

extern "C" cluster_status cluster_server_get_stats(cluster_server* sv, cluster_server_stats* out) {
  clear_error();
  if (!sv || !out) FC_EINVAL("NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  *out = sv->stats;
  out->queued = (int64_t)sv->queue.size();
  out->budget_bytes = sv->opt.hbm_budget;
  out->queued_host_bytes = sv->queued_host;
  out->uptime_s = now_s() - sv->busy_t0;
  return CLUSTER_OK;
}

extern "C" void cluster_server_destroy(cluster_server* sv) {
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->worker.joinable()) sv->worker.join();
  for (auto& kv : sv->all) delete kv.second;
  delete sv;
}
