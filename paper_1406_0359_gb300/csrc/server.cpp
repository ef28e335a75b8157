// Request server: continuous batching of SARA-SDMM solves on one GPU.
//
// Requests (host uv, host visibilities, image side, parameters) wait in a
// FIFO queue.  Each scheduling call admits queued requests while a slot is
// free and their estimated device memory fits the budget (operator creation:
// uv binning, tables; the solve's state then stays resident), and keeps every
// admitted solve moving one SDMM iteration (Algorithm 1) at a time on its
// operator's own stream, so that the solves' kernels overlap on the device.
// A solve whose iteration has completed (its event has fired) gets its
// halting test and its next iteration at once; one whose iteration is still
// running is left alone, so a large image never holds back a small one.  A
// finished solve's image is copied back, its memory returns to the pool and
// the next request can take its slot.
//
// Iteration-level batching (off by default): solves that share a batch key
// (image side, precision, CG steps, dictionary; the convolution form of the
// CG operator) and are between iterations advance together -- one SDMM
// iteration of all of them is one batched graph (each pass one launch over
// the group, see purify_batch_solve) on the group's own stream, cached for
// as long as the group's membership stays the same.  A ready solve whose key
// has a group in flight waits for it and joins at the next iteration.  On
// GB300 the solves' own streams already keep the device full for images of
// 128^2 and up (16-64 concurrent solves ran 3-20 % faster per iteration that
// way than in batched groups), so batching stays opt-in.
//
// Device memory of admitted solves (operators, state, staging of uv and y)
// comes from one stream-ordered memory pool of the server that keeps up to
// the budget mapped: admitting and releasing solves never calls cudaMalloc or
// cudaFree, which would synchronise the whole device.  Host inputs reach the
// device through a pinned staging buffer on the server's admission stream.
//
// The caller drives the server (purify_server_step) and collects results;
// the server is not thread-safe.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
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
  void* x_dev = nullptr;
  cudaEvent_t ev = nullptr;  // end of the iteration in flight
  bool inflight = false;
  bool grouped = false;      // the iteration in flight is a batched group's
  uint64_t gkey = 0;         // and that group's key
  std::vector<unsigned char> x;
  purify_stats st{};
  int status = 1;  // 1 queued/active, 0 done, < 0 error, -5 done without convergence
  double t_submit = 0, t_admit = 0, t_done = 0;
};

size_t real_bytes(int precision) { return precision == PURIFY_FP32 ? 4 : 8; }

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return PURIFY_OK;
  return e == cudaErrorMemoryAllocation ? PURIFY_ERR_NOMEM : PURIFY_ERR_CUDA;
}

// Index of the first non-finite value among n, or -1.
template <typename T> int64_t first_nonfinite(const T* v, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) return i;
  return -1;
}

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
  b += (M / 256.0 + 4.0 * K * K / 256) * 16;  // work items (bound, chunks of >= 256) and partial sums
  b += M * (16 + c) + N * r;                 // the server's staging of uv and y, the result image
  if (n <= 1024) {
    // composite operator: spectrum kept; while it is built, a 2n operator,
    // a unit-visibility vector and two K^2 buffers live for a moment
    const double n2 = 2.0 * n, N2 = n2 * n2, K2 = 2 * n2, KP2 = K2 + 8;
    b += (K / 2 + 1) * K * r + n * (K / 2) * c + N * r;  // and the CG start's A x_hat with its half spectra
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
  int device = 0;
  cudaMemPool_t pool = nullptr;
  cudaStream_t adm = nullptr;  // admission copies and operator set-up
  void* pin = nullptr;         // pinned staging of one request's uv and y
  size_t pin_bytes = 0;
  std::deque<Request*> queue;
  std::vector<Request*> active;
  // batched groups by key: the members of the iteration in flight or last
  // launched, their cached graph, its stream and completion event (groups of
  // different keys run side by side)
  struct Group {
    std::vector<int> ids;
    std::vector<Request*> members;
    purify::BatchGraph* graph = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    bool inflight = false;
  };
  std::map<uint64_t, Group> groups;
  bool batching = false;
  int64_t n_batched = 0, n_solo = 0;  // solve-iterations launched each way
  std::map<int, Request*> all;
  std::map<int, purify_op_options> opts;  // per image side (from the autotuner)

  int init(int64_t budget_bytes, int slots) {
    budget = budget_bytes;
    max_slots = slots;
    if (cudaGetDevice(&device) != cudaSuccess) return PURIFY_ERR_CUDA;
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaError_t e = cudaMemPoolCreate(&pool, &props);
    if (e == cudaSuccess) {
      uint64_t keep = uint64_t(budget);
      e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&adm, cudaStreamNonBlocking);
    return cuda_status(e);
  }

  ~purify_server() {
    for (auto& kv : groups)
      if (kv.second.stream) cudaStreamSynchronize(kv.second.stream);
    for (auto& kv : groups) {
      purify::batch_graph_destroy(kv.second.graph);
      if (kv.second.ev) cudaEventDestroy(kv.second.ev);
      if (kv.second.stream) cudaStreamDestroy(kv.second.stream);
    }
    for (auto& kv : all) {
      release(kv.second);
      delete kv.second;
    }
    if (adm) cudaStreamSynchronize(adm);
    if (adm) cudaStreamDestroy(adm);
    if (pin) cudaFreeHost(pin);
    if (pool) cudaMemPoolDestroy(pool);
  }

  // Return a solve's memory to the pool (its streams are idle afterwards).
  void release(Request* r) {
    if (r->op) {
      cudaStreamSynchronize(r->op->stream());
      if (r->x_dev) cudaFreeAsync(r->x_dev, r->op->stream());
      purify_op_destroy(r->op);
    }
    if (r->ev) cudaEventDestroy(r->ev);
    r->op = nullptr;
    r->x_dev = nullptr;
    r->ev = nullptr;
    r->inflight = false;
  }

  void finish(Request* r, int status) {
    r->status = status;
    r->t_done = now_s();
    release(r);
    in_use -= r->est;
  }

  int stage(size_t bytes) {
    if (bytes <= pin_bytes) return PURIFY_OK;
    if (pin) {
      cudaStreamSynchronize(adm);
      cudaFreeHost(pin);
      pin = nullptr;
      pin_bytes = 0;
    }
    if (cudaMallocHost(&pin, bytes) != cudaSuccess) return PURIFY_ERR_NOMEM;
    pin_bytes = bytes;
    return PURIFY_OK;
  }

  // Set up one admitted request: stage uv and y, build its operator from the
  // pool, start its solve.  uv and y copies return to the pool once the
  // solve has taken its own copy of y.
  int setup(Request* r) {
    const size_t uvb = r->uv.size() * sizeof(double), yb = r->y.size();
    int rc = stage(uvb + yb);
    if (rc) return rc;
    unsigned char* h = static_cast<unsigned char*>(pin);
    cudaError_t e = cudaStreamSynchronize(adm);  // the staging buffer is free again
    if (e != cudaSuccess) return cuda_status(e);
    std::memcpy(h, r->uv.data(), uvb);
    std::memcpy(h + uvb, r->y.data(), yb);
    void *uv_dev = nullptr, *y_dev = nullptr;
    e = cudaMallocFromPoolAsync(&uv_dev, uvb, pool, adm);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&y_dev, yb, pool, adm);
    if (e == cudaSuccess)
      e = cudaMallocFromPoolAsync(&r->x_dev, size_t(r->n) * r->n * real_bytes(r->precision), pool, adm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(uv_dev, h, uvb, cudaMemcpyHostToDevice, adm);
    if (e == cudaSuccess) e = cudaMemcpyAsync(y_dev, h + uvb, yb, cudaMemcpyHostToDevice, adm);
    rc = cuda_status(e);
    if (!rc) {
      auto oi = opts.find(r->n);
      rc = purify::create_pooled_op(static_cast<const double*>(uv_dev), r->M, r->n, r->levels, r->precision,
                                    oi == opts.end() ? nullptr : &oi->second, pool, adm, &r->op);
    }
    if (!rc) rc = r->op->begin(y_dev, &r->P, adm);  // returns once y is gathered into the solve's state
    if (!rc) rc = cuda_status(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
    if (uv_dev) cudaFreeAsync(uv_dev, adm);
    if (y_dev) cudaFreeAsync(y_dev, adm);
    return rc;
  }

  // Admission: FIFO, a free slot and the estimated memory within the budget.
  void admit() {
    while (!queue.empty() && int(active.size()) < max_slots) {
      Request* r = queue.front();
      if (in_use + r->est > budget && !active.empty()) break;  // wait for memory
      queue.pop_front();
      in_use += r->est;
      r->t_admit = now_s();
      const int rc = setup(r);
      if (rc) {
        finish(r, rc);
        continue;
      }
      active.push_back(r);
    }
  }

  // A finished solve: its image to host memory, its memory back to the pool.
  void complete(Request* r) {
    cudaStream_t s = r->op->stream();
    int rc = r->op->end(r->x_dev, &r->st, s);
    const size_t xb = size_t(r->n) * r->n * real_bytes(r->precision);
    r->x.resize(xb);
    cudaError_t e = cudaMemcpyAsync(r->x.data(), r->x_dev, xb, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if ((rc == PURIFY_OK || rc == PURIFY_ERR_NOT_CONVERGED) && e != cudaSuccess) rc = cuda_status(e);
    finish(r, rc);
  }

  // A solve whose iteration has completed: its halting test, then completion
  // or (when it continues) nothing -- its next launch comes with the others.
  void settle(Request* r, cudaError_t q) {
    r->inflight = false;
    r->grouped = false;
    if (r->status != 1) return;  // cancelled meanwhile
    int done = 0;
    const int rc = q == cudaSuccess ? r->op->step_check(&done) : cuda_status(q);
    if (rc) finish(r, rc);
    else if (done) complete(r);
  }

  void launch_solo(Request* r) {
    ++n_solo;
    int rc = r->op->step_launch();
    if (!rc) rc = cuda_status(cudaEventRecord(r->ev, r->op->stream()));
    if (rc) {
      finish(r, rc);
      return;
    }
    r->inflight = true;
  }

  // One batched iteration of `list` (one key, at least two solves).
  void launch_group(uint64_t key, std::vector<Request*>& list) {
    std::sort(list.begin(), list.end(), [](const Request* a, const Request* b) { return a->id < b->id; });
    Group& g = groups[key];
    if (!g.stream && cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess) g.stream = nullptr;
    if (!g.ev && cudaEventCreateWithFlags(&g.ev, cudaEventDisableTiming) != cudaSuccess) g.ev = nullptr;
    if (!g.stream || !g.ev) {  // cannot batch: each on its own
      for (Request* r : list) launch_solo(r);
      return;
    }
    std::vector<Request*> ok;
    for (Request* r : list) {  // round set-ups (on the group's stream)
      const int rc = r->op->prepare_iteration(g.stream);
      if (rc) finish(r, rc);
      else ok.push_back(r);
    }
    if (ok.size() < 2) {
      for (Request* r : ok) launch_solo(r);
      return;
    }
    std::vector<int> ids;
    for (Request* r : ok) ids.push_back(r->id);
    if (g.graph && g.ids != ids) {
      purify::batch_graph_destroy(g.graph);
      g.graph = nullptr;
    }
    if (!g.graph) {
      std::vector<purify_op*> ops;
      for (Request* r : ok) ops.push_back(r->op);
      if (purify::batch_graph_create(ops.data(), int(ops.size()), pool, &g.graph)) g.graph = nullptr;
    }
    if (!g.graph || purify::batch_graph_launch(g.graph, g.stream)) {  // cannot batch: each on its own
      for (Request* r : ok) launch_solo(r);
      return;
    }
    g.ids = ids;
    g.members = ok;
    n_batched += int64_t(ok.size());
    for (Request* r : ok) {
      const int rc = r->op->finish_iteration(g.stream);
      r->inflight = true;
      r->grouped = true;
      r->gkey = key;
      if (rc) r->status = rc;  // reported when the group settles
    }
    cudaEventRecord(g.ev, g.stream);
    g.inflight = true;
  }

  // One scheduling pass: admit; settle every solve whose iteration in flight
  // has completed (a batched group all at once); then launch the next
  // iteration of every solve between iterations -- together with the others
  // of its batch key when batching is on, else on its own stream.
  int step() {
    admit();
    for (auto& kv : groups) {
      Group& g = kv.second;
      if (!g.inflight) continue;
      const cudaError_t q = cudaEventQuery(g.ev);
      if (q == cudaErrorNotReady) continue;
      g.inflight = false;
      for (Request* r : g.members) {
        if (r->status < 0 && r->status != 1 && r->op) {  // a hook failed at launch
          finish(r, r->status);
          continue;
        }
        settle(r, q);
      }
    }
    for (Request* r : active) {
      if (!r->inflight || r->grouped || r->status != 1) continue;
      const cudaError_t q = cudaEventQuery(r->ev);
      if (q != cudaErrorNotReady) settle(r, q);
    }
    active.erase(std::remove_if(active.begin(), active.end(), [](const Request* r) { return r->status != 1; }),
                 active.end());
    std::map<uint64_t, std::vector<Request*>> ready;
    for (Request* r : active) {
      if (r->inflight) continue;
      const uint64_t key = batching ? r->op->batch_key() : 0;
      if (key) {
        auto gi = groups.find(key);
        if (gi != groups.end() && gi->second.inflight) continue;  // join the group at its next iteration
      }
      ready[key].push_back(r);
    }
    for (auto& kv : ready) {
      if (kv.first && kv.second.size() >= 2) {
        launch_group(kv.first, kv.second);
      } else {
        for (Request* r : kv.second) launch_solo(r);
      }
    }
    active.erase(std::remove_if(active.begin(), active.end(), [](const Request* r) { return r->status != 1; }),
                 active.end());
    return PURIFY_OK;
  }

  int cancel(int id) {
    auto it = all.find(id);
    if (it == all.end()) return PURIFY_ERR_INVALID;
    Request* r = it->second;
    if (r->status != 1) return PURIFY_ERR_INVALID;  // already finished
    auto q = std::find(queue.begin(), queue.end(), r);
    if (q != queue.end()) {
      queue.erase(q);
      r->status = PURIFY_ERR_CANCELLED;
      r->t_done = now_s();
      return PURIFY_OK;
    }
    auto a = std::find(active.begin(), active.end(), r);
    if (a == active.end()) return PURIFY_ERR_INVALID;
    active.erase(a);
    if (r->grouped) cudaStreamSynchronize(groups[r->gkey].stream);  // its iteration runs in a batched group
    finish(r, PURIFY_ERR_CANCELLED);  // waits for the iteration in flight, then releases
    return PURIFY_OK;
  }
};

extern "C" {

int purify_server_create(int64_t budget_bytes, int max_slots, purify_server** out) {
  if (!out || budget_bytes <= 0 || max_slots < 1) return PURIFY_ERR_INVALID;
  purify_server* s = new (std::nothrow) purify_server();
  if (!s) return PURIFY_ERR_NOMEM;
  const int rc = s->init(budget_bytes, max_slots);
  if (rc) {
    delete s;
    return rc;
  }
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
  // inputs are checked here, before they can reach the device
  int64_t bad = first_nonfinite(uv_host, 2 * M);
  const char* what = "uv";
  if (bad < 0) {
    bad = precision == PURIFY_FP32 ? first_nonfinite(static_cast<const float*>(y_host), 2 * M)
                                   : first_nonfinite(static_cast<const double*>(y_host), 2 * M);
    what = "y";
  }
  if (bad >= 0) {
    char buf[128];
    std::snprintf(buf, sizeof(buf), "purify_server_submit: %s holds a non-finite value (visibility %lld)", what,
                  static_cast<long long>(bad / 2));
    purify::set_last_error(buf);
    return PURIFY_ERR_INVALID;
  }
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

int purify_server_set_batching(purify_server* srv, int enable) {
  if (!srv) return PURIFY_ERR_INVALID;
  srv->batching = enable != 0;
  return PURIFY_OK;
}

int purify_server_counts(purify_server* srv, int64_t* batched, int64_t* solo) {
  if (!srv) return PURIFY_ERR_INVALID;
  if (batched) *batched = srv->n_batched;
  if (solo) *solo = srv->n_solo;
  return PURIFY_OK;
}

int purify_server_cancel(purify_server* srv, int request_id) {
  if (!srv) return PURIFY_ERR_INVALID;
  return srv->cancel(request_id);
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
