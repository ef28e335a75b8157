// The operator object behind the opaque purify_op handle: the virtual
// interface implemented per precision in api.cu, plus kernel-timing state.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/purify.h"

struct purify_op {
  virtual ~purify_op() {}
  virtual int phi(const void* x, void* y, cudaStream_t s) = 0;
  virtual int phi_adj(const void* y, void* x, cudaStream_t s) = 0;
  virtual int sara_fwd(const void* x, void* c, cudaStream_t s) = 0;
  virtual int sara_adj(const void* c, void* x, cudaStream_t s) = 0;
  virtual int solve(const void* y, const purify_params* p, void* x, purify_stats* st, cudaStream_t s) = 0;
  virtual int gram(const void* x, void* out, int mode, cudaStream_t s) = 0;
  virtual int set_blocks(const int* blocks, int R, cudaStream_t s) = 0;
  virtual int set_dictionary(unsigned mask) = 0;
  virtual int set_prior(int prior, int tv_iters) = 0;
  virtual unsigned dictionary(int* nbases) const = 0;
  // resumable solve (request server)
  virtual int begin(const void* y, const purify_params* p, cudaStream_t user) = 0;
  virtual int step_launch() = 0;
  virtual int step_check(int* done) = 0;
  virtual int end(void* x, purify_stats* st, cudaStream_t user) = 0;
  // Up to max_iters iterations of the resumable solve, then a synchronous
  // check of the device error flag; *done = 1 once the last round finished.
  virtual int run_steps(int max_iters, int* done) = 0;
  // Iteration-level batching (request server): a non-zero key groups solves
  // that can advance through one batched graph; the hooks run each solve's
  // round set-up before it and its halting read-back after it, on `s`.  The
  // caller sees the batched iteration complete (an event on `s`) before it
  // makes the next call on the solve.
  virtual uint64_t batch_key() const = 0;
  virtual int prepare_iteration(cudaStream_t s) = 0;
  virtual int finish_iteration(cudaStream_t s) = 0;
  // Solver state between iterations (checkpoint / resume).
  virtual int64_t state_bytes() const = 0;
  virtual int save_state(void* host, int64_t bytes) = 0;
  virtual int load_state(const void* host, int64_t bytes) = 0;
  virtual cudaStream_t stream() const = 0;
  // Phi then Phi^H in the solver's sorted visibility order (autotuner timing).
  virtual int sorted_pair(const void* x, void* y, void* out, cudaStream_t s) = 0;
  virtual void info(int* n, int64_t* M, int* K, int* tile, int* n_items, int* precision, int64_t* bytes) const = 0;

  // ---- kernel timing (instrumentation)
  enum Kind { KK_ROW_FWD = 0, KK_COL_FWD, KK_DEGRID, KK_GRID, KK_GRAM, KK_COL_INV, KK_ROW_INV, KK_SARA_ANA,
              KK_SARA_SYN, KK_VEC, KK_MEMSET, KK_COL_CONV, KK_ROW_FWD_H, KK_ROW_INV_H, KK_TV, KK_COUNT };
  bool prof = false;
  struct Pending { int kind; cudaEvent_t a, b; };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  double prof_ms[KK_COUNT] = {0};
  int64_t prof_n[KK_COUNT] = {0};
  cudaStream_t prof_stream = nullptr;
  int prof_kind = -1;
  cudaEvent_t ev() {
    if (!pool.empty()) {
      cudaEvent_t e = pool.back();
      pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void prof_begin(int kind, cudaStream_t s) {
    if (!prof) return;
    Pending p{kind, ev(), ev()};
    cudaEventRecord(p.a, s);
    pending.push_back(p);
  }
  void prof_end(cudaStream_t s) {
    if (!prof || pending.empty()) return;
    cudaEventRecord(pending.back().b, s);
  }
  void prof_collect() {
    for (auto& p : pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
        prof_ms[p.kind] += ms;
        prof_n[p.kind] += 1;
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
  void prof_reset() {
    prof_collect();
    for (int k = 0; k < KK_COUNT; ++k) {
      prof_ms[k] = 0;
      prof_n[k] = 0;
    }
  }
  void prof_release() {
    prof_collect();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
  }
};

namespace purify {
// Operator whose device memory all comes from `pool` (stream-ordered, never
// synchronising the device on release): the request server's operators.
// Arguments as purify_op_create_ex; `opt` may be null.
int create_pooled_op(const double* uv, int64_t M, int n, int levels, int precision, const purify_op_options* opt,
                     cudaMemPool_t pool, cudaStream_t s, purify_op** out);
// Record the detail returned by purify_last_error() on this thread.
void set_last_error(const char* msg);
// One SDMM iteration of `count` active solves of one batch key as a batched
// graph (one launch per pass over all of them), tables from `pool`.
struct BatchGraph;
int batch_graph_create(purify_op* const* ops, int count, cudaMemPool_t pool, BatchGraph** out);
int batch_graph_launch(BatchGraph* g, cudaStream_t s);
void batch_graph_destroy(BatchGraph* g);
}  // namespace purify
