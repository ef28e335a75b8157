// Request server: continuous batching of SARA-SDMM solves on one GPU.
//
// Requests (host uv, host visibilities, image side, parameters) wait in a
// FIFO queue.  A scheduling round admits queued requests while a slot is free
// and their estimated device memory fits the budget (operator creation: uv
// binning, tables; the solve's state then stays resident), then advances every
// admitted solve by one SDMM iteration (Algorithm 1), each on its operator's
// own stream so that the solves' kernels overlap on the device.  A finished
// solve's image is copied back, its memory is released and the next request
// can take its slot in the following round.  The caller drives the rounds and
// collects results; the server is not thread-safe.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <new>
#include <vector>

#include "op.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Request {
  int id = 0;
  int n = 0, levels = 0, precision = 0;
  int64_t M = 0;
  std::vector<double> uv;
  std::vector<unsigned char> y;
  purify_params P{};
  int64_t est = 0;
  purify_op* op = nullptr;
  void* y_dev = nullptr;
  void* x_dev = nullptr;
  std::vector<unsigned char> x;
  purify_stats st{};
  int status = 1;  // 1 queued/active, 0 done, < 0 error, -5 done without convergence
  double t_submit = 0, t_admit = 0, t_done = 0;
};

size_t real_bytes(int precision) { return precision == PURIFY_FP32 ? 4 : 8; }

}  // namespace

extern "C" int purify_estimate_bytes(int64_t M, int n, int dwt_levels, int precision, int64_t* bytes) {
  if (!bytes || M < 1 || n < 16 || (n & (n - 1)) || dwt_levels < 1) return PURIFY_ERR_INVALID;
  const double r = double(real_bytes(precision)), c = 2 * r;
  const double N = double(n) * n, K = 2.0 * n, KP = K + 8;
  double b = 0;
  b += M * (2 * r + 4 + 16);                 // positions, permutation, kept uv
  b += double(n) * (K / 2) * c + 2 * KP * KP * c;  // half-spectrum rows, forward grid, gridding grid
  b += 2 * 8 * (N / 4) * r + 9 * N * r;      // wavelet scratch bands, prox output
  b += 6 * N * r + 18 * N * r + 2 * M * c;   // solver vectors, z1 and weights, z3 and sorted y
  b += (M / 1024.0 + 4.0 * K * K / 256) * 16;  // work items (bound) and partial sums
  if (n <= 1024) {
    // composite operator: spectrum kept; while it is built, a 2n operator,
    // a unit-visibility vector and two K^2 buffers live for a moment
    const double n2 = 2.0 * n, N2 = n2 * n2, K2 = 2 * n2, KP2 = K2 + 8;
    b += (K / 2 + 1) * K * r;
    b += M * (2 * r + 4 + 16) + n2 * K2 * c + 2 * KP2 * KP2 * c + 2 * 8 * (N2 / 4) * r + 9 * N2 * r;
    b += M * c + K * K * (r + c);
  }
  *bytes = int64_t(b * 1.05) + (int64_t(8) << 20);
  return PURIFY_OK;
}

struct purify_server {
  int64_t budget = 0;
  int max_slots = 1;
  int64_t in_use = 0;
  int next_id = 1;
  std::deque<Request*> queue;
  std::vector<Request*> active;
  std::map<int, Request*> all;
  std::map<int, purify_op_options> opts;  // per image side (from the autotuner)

  ~purify_server() {
    for (auto& kv : all) {
      release(kv.second);
      delete kv.second;
    }
  }

  void release(Request* r) {
    if (r->op) purify_op_destroy(r->op);
    if (r->y_dev) cudaFree(r->y_dev);
    if (r->x_dev) cudaFree(r->x_dev);
    r->op = nullptr;
    r->y_dev = r->x_dev = nullptr;
  }

  void fail(Request* r, int rc) {
    r->status = rc;
    r->t_done = now_s();
    release(r);
    in_use -= r->est;
  }

  // Admission: FIFO, a free slot and the estimated memory within the budget.
  int admit() {
    while (!queue.empty() && int(active.size()) < max_slots) {
      Request* r = queue.front();
      if (in_use + r->est > budget && !active.empty()) break;  // wait for memory
      queue.pop_front();
      in_use += r->est;
      r->t_admit = now_s();
      const size_t cb = 2 * real_bytes(r->precision);
      double* uv_dev = nullptr;
      cudaError_t e = cudaMalloc(&uv_dev, r->uv.size() * sizeof(double));
      if (e == cudaSuccess) e = cudaMalloc(&r->y_dev, size_t(r->M) * cb);
      if (e == cudaSuccess) e = cudaMalloc(&r->x_dev, size_t(r->n) * r->n * real_bytes(r->precision));
      if (e == cudaSuccess)
        e = cudaMemcpy(uv_dev, r->uv.data(), r->uv.size() * sizeof(double), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(r->y_dev, r->y.data(), r->y.size(), cudaMemcpyHostToDevice);
      int rc = e == cudaSuccess ? PURIFY_OK : (e == cudaErrorMemoryAllocation ? PURIFY_ERR_NOMEM : PURIFY_ERR_CUDA);
      if (!rc) {
        auto oi = opts.find(r->n);
        rc = purify_op_create_ex(uv_dev, r->M, r->n, 2, 8, r->levels, r->precision,
                                 oi == opts.end() ? nullptr : &oi->second, nullptr, &r->op);
      }
      cudaFree(uv_dev);
      if (!rc) rc = r->op->begin(r->y_dev, &r->P, r->op->stream());
      if (rc) {
        fail(r, rc);
        continue;
      }
      active.push_back(r);
    }
    return PURIFY_OK;
  }

  // One scheduling round: admit, launch one iteration of every admitted solve
  // (each on its own stream), then check them; finished solves release their
  // memory and slot.
  int step() {
    admit();
    for (Request* r : active) {
      const int rc = r->op->step_launch();
      if (rc) r->status = rc;
    }
    std::vector<Request*> keep;
    for (Request* r : active) {
      int done = 0;
      if (r->status == 1) {
        const int rc = r->op->step_check(&done);
        if (rc) r->status = rc;
      }
      if (r->status != 1) {
        fail(r, r->status);
        continue;
      }
      if (!done) {
        keep.push_back(r);
        continue;
      }
      const size_t xb = size_t(r->n) * r->n * real_bytes(r->precision);
      int rc = r->op->end(r->x_dev, &r->st, r->op->stream());
      r->x.resize(xb);
      const int rc2 = cudaMemcpy(r->x.data(), r->x_dev, xb, cudaMemcpyDeviceToHost) == cudaSuccess ? 0 : -3;
      if (rc == PURIFY_OK || rc == PURIFY_ERR_NOT_CONVERGED) rc = rc2 ? rc2 : rc;
      r->status = rc;
      r->t_done = now_s();
      release(r);
      in_use -= r->est;
    }
    active.swap(keep);
    return PURIFY_OK;
  }
};

extern "C" {

int purify_server_create(int64_t budget_bytes, int max_slots, purify_server** out) {
  if (!out || budget_bytes <= 0 || max_slots < 1) return PURIFY_ERR_INVALID;
  purify_server* s = new (std::nothrow) purify_server();
  if (!s) return PURIFY_ERR_NOMEM;
  s->budget = budget_bytes;
  s->max_slots = max_slots;
  *out = s;
  return PURIFY_OK;
}

int purify_server_set_options(purify_server* srv, int n, const purify_op_options* opt) {
  if (!srv || !opt) return PURIFY_ERR_INVALID;
  srv->opts[n] = *opt;
  return PURIFY_OK;
}

int purify_server_destroy(purify_server* srv) {
  delete srv;
  return PURIFY_OK;
}

int purify_server_submit(purify_server* srv, const double* uv_host, const void* y_host, int64_t M, int n,
                         int dwt_levels, int precision, const purify_params* params, int* request_id) {
  if (!srv || !uv_host || !y_host || !params || !request_id || M < 1 || n < 16 || n > 2048 || (n & (n - 1)) ||
      dwt_levels < 1 || (n >> dwt_levels) < 2 || (precision != PURIFY_FP32 && precision != PURIFY_FP64))
    return PURIFY_ERR_INVALID;
  Request* r = new (std::nothrow) Request();
  if (!r) return PURIFY_ERR_NOMEM;
  r->id = srv->next_id++;
  r->n = n;
  r->levels = dwt_levels;
  r->precision = precision;
  r->M = M;
  r->uv.assign(uv_host, uv_host + 2 * M);
  const size_t yb = size_t(M) * 2 * real_bytes(precision);
  r->y.resize(yb);
  std::memcpy(r->y.data(), y_host, yb);
  r->P = *params;
  r->P.eps_blocks = nullptr;
  purify_estimate_bytes(M, n, dwt_levels, precision, &r->est);
  if (r->est > srv->budget) {
    delete r;
    return PURIFY_ERR_BUDGET;
  }
  r->t_submit = now_s();
  srv->queue.push_back(r);
  srv->all[r->id] = r;
  *request_id = r->id;
  return PURIFY_OK;
}

int purify_server_step(purify_server* srv, int* n_active, int* n_queued) {
  if (!srv) return PURIFY_ERR_INVALID;
  const int rc = srv->step();
  if (n_active) *n_active = int(srv->active.size());
  if (n_queued) *n_queued = int(srv->queue.size());
  return rc;
}

int purify_server_result(purify_server* srv, int request_id, void* x_host, purify_stats* stats, double* latency_s,
                         double* queue_s) {
  if (!srv) return PURIFY_ERR_INVALID;
  auto it = srv->all.find(request_id);
  if (it == srv->all.end()) return PURIFY_ERR_INVALID;
  Request* r = it->second;
  if (r->status == 1) return 0;
  if (r->status < 0 && r->status != PURIFY_ERR_NOT_CONVERGED) return r->status;
  if (x_host) std::memcpy(x_host, r->x.data(), r->x.size());
  if (stats) *stats = r->st;
  if (latency_s) *latency_s = r->t_done - r->t_submit;
  if (queue_s) *queue_s = r->t_admit - r->t_submit;
  return 1;
}

}  // extern "C"
