// C-ABI of libpurify_gb300 (include/purify.h): operator set-up, the operator
// pairs Phi / Phi^H and Psi^H / Psi, and the SDMM solver with the SARA
// reweighting loop (Section 2.2, Section 3 Algorithm 1) driven from the host,
// all compute in this library's kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <map>
#include <mutex>
#include <initializer_list>
#include <new>
#include <vector>

#include "../../include/purify.h"
#include "host_math.h"
#include "internal.h"
#include "solver_kernels.h"

#include "op.h"

#define PROF(kind, stream, stmt) \
  do {                           \
    prof_begin(kind, stream);    \
    stmt;                        \
    prof_end(stream);            \
  } while (0)

namespace purify {

cudaMemPool_t library_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
      cudaMemPoolProps props;
      std::memset(&props, 0, sizeof(props));
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      cudaMemPool_t np = nullptr;
      if (cudaMemPoolCreate(&np, &props) == cudaSuccess) {
        uint64_t keep = kSetupPoolKeep;
        cudaMemPoolSetAttribute(np, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = np;
      } else {
        cudaGetLastError();  // fall back to the device's default pool
        if (cudaDeviceGetDefaultMemPool(&np, dev) != cudaSuccess) return nullptr;
        pools[dev] = np;
      }
    }
    pool = pools[dev];
  }
  return pool;
}

cudaError_t setup_alloc(void** p, size_t bytes, cudaStream_t s) {
  cudaMemPool_t pool = library_pool();
  if (!pool) return cudaMallocAsync(p, bytes, s);
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

thread_local char g_last_error[256] = "";
void set_last_error(const char* msg) { std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

void note_error(const char* what, int line, const char* detail) {
  char buf[256];
  std::snprintf(buf, sizeof(buf), "%s (api.cu:%d): %s", what, line, detail);
  set_last_error(buf);
}

int map_err(cudaError_t e, int line = 0) {
  if (e == cudaSuccess) return PURIFY_OK;
  note_error("CUDA call failed", line, cudaGetErrorName(e));
  if (e == cudaErrorMemoryAllocation) return PURIFY_ERR_NOMEM;
  return PURIFY_ERR_CUDA;
}

#define CK(call)                                          \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return map_err(e_, __LINE__);  \
  } while (0)

// Kernel attributes (dynamic shared-memory limits) are per device, so they
// are set once per device and precision, not per operator.
template <typename T> cudaError_t configure_once() {
  static std::mutex mu;
  static uint64_t done = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  const uint64_t bit = dev < 64 ? (uint64_t(1) << dev) : 0;
  if (bit && (done & bit)) return cudaSuccess;
  e = configure_fft<T>();
  if (e == cudaSuccess) e = configure_nufft<T>();
  if (e == cudaSuccess) e = configure_sara<T>();
  if (e == cudaSuccess) done |= bit;
  return e;
}

// Pinned host mirrors of the device scalars (kNumScalars doubles each, for the
// asynchronous copies of the resumable solver), carved from 64 KB pinned
// pages: creating an operator does not pay a pinned allocation.
class PinnedSlots {
 public:
  static constexpr size_t kSlot = 32;  // doubles per slot (>= kNumScalars)
  double* get() {
    std::lock_guard<std::mutex> lk(mu_);
    if (free_.empty()) {
      void* page = nullptr;
      if (cudaMallocHost(&page, 65536) != cudaSuccess) return nullptr;
      pages_.push_back(page);
      for (size_t k = 0; k < 65536 / (kSlot * sizeof(double)); ++k)
        free_.push_back(static_cast<double*>(page) + k * kSlot);
    }
    double* p = free_.back();
    free_.pop_back();
    return p;
  }
  void put(double* p) {
    std::lock_guard<std::mutex> lk(mu_);
    free_.push_back(p);
  }

 private:
  std::mutex mu_;
  std::vector<void*> pages_;  // kept for the life of the process
  std::vector<double*> free_;
};
static_assert(PinnedSlots::kSlot >= size_t(kNumScalars), "slot holds the scalars");
PinnedSlots& pinned_slots() {
  static PinnedSlots* p = new PinnedSlots();
  return *p;
}

template <typename T> class OpImpl : public purify_op {
  typedef typename cplx_t<T>::type C;

 public:
  Geometry g{};
  int levels = 0, chunk = 0, n_items = 0;
  Pos<T>* pos = nullptr;
  int* perm = nullptr;
  WorkItem* items = nullptr;
  T* deapod = nullptr;
  C* tw = nullptr;
  C* gridA = nullptr;
  C* gridP = nullptr;
  C* gridQ = nullptr;
  CUtensorMap tmap;
  KbPoly<T> kb;
  SaraPlan<T> sara{};
  double* partials = nullptr;
  double* cg_part = nullptr;        // CG partial sums (row pass, CG update)
  unsigned int* tickets = nullptr;  // last-block tickets: CG reductions (0, 1), ball scalars (2)
  double* fin_part = nullptr;       // per-CTA partials of the ball-scalar merge (2 x kFinCtas)
  static constexpr int kCgPart = 4096;
  double* sc = nullptr;
  double* h_sc = nullptr;
  int* err = nullptr;
  // solver state
  T *xh = nullptr, *xs = nullptr, *r = nullptr, *p = nullptr, *Ap = nullptr;
  T *z1 = nullptr, *z2 = nullptr, *w = nullptr;
  C *z3 = nullptr, *ys = nullptr;
  // composite operator by convolution (Section 3: precompute Phi^H Phi)
  double* uv_keep = nullptr;  // device copy of uv, for the PSF set-up
  T* khat = nullptr;          // real PSF half spectrum, launch_col_conv_h layout
  T* axh = nullptr;           // (nu^2 Re Phi^H Phi + 2I) x_hat, for the next CG start
  C* gridA2 = nullptr;        // half-spectrum rows of that product (beside the ball block's gridA)
  bool toep = false;          // current normal-operator mode
  bool own_pending = false;   // work may be in flight on the own stream (begin, a solo iteration)
  // visibility blocks (Eq. 4-5)
  int nblocks = 1;
  std::vector<int64_t> block_sizes;
  double* eps_dev = nullptr;    // nu-independent radii eps_b (R)
  double* scale_dev = nullptr;  // projection scale per block (R)
  // prior of the f_1 block: 0 the l1 analysis prior over the dictionary
  // (SARA and its sub-dictionaries), 1 TV (Section 4's TV / RWTV)
  int prior = 0;
  int tv_iters = 20;
  T* tvq = nullptr;  // the TV prox's dual: two buffers of 2N
  int64_t bytes = 0;
  std::vector<void*> allocs;
  // Set-up (light) operator: buffers from the set-up pool on this stream, the
  // only stream that uses them; released in stream order.
  cudaStream_t pool_stream = nullptr;
  bool items_pooled = false;  // items from the set-up pool (refined operator)
  cudaMemPool_t lib_pool = nullptr;  // the library's per-device pool (plain operators)
  // Operator of the request server: every allocation comes from the server's
  // stream-ordered pool on the operator's own stream and goes back to it in
  // stream order, so creating and releasing solves never synchronises the
  // device (cudaMalloc / cudaFree would stall the solves running beside).
  cudaMemPool_t mem_pool = nullptr;
  cudaStream_t own = nullptr;  // solver stream (capturable, non-blocking)
  cudaStream_t aux = nullptr;  // second branch of an SDMM iteration (ball block)
  cudaStream_t aux2 = nullptr;  // zeroing of the gridding accumulator beside the ball block's first passes
  cudaStream_t aux3 = nullptr;  // the A x_hat passes for the next CG start (lowest priority)
  cudaEvent_t ev_axf = nullptr, ev_axj = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr, ev_join = nullptr;
  cudaEvent_t ev_zfork = nullptr, ev_zjoin = nullptr;
  double* bpart = nullptr;     // ball-block partials (2 per work item), apart from the l1 block's
  int bpart_cap = 0;
  CUtensorMap* tmap_dev = nullptr;  // device copy of tmap (batched degridding reads it there)

  // ---- recording of one SDMM iteration for the batched solver: with `rec`
  // set, the pass helpers append their launch arguments instead of
  // launching (branch 1 = the ball block's stream).
  enum RecKind { R_RF, R_CC, R_RI, R_CF, R_CI, R_DG, R_GR, R_B1, R_ZERO, R_AXPY, R_FIN, R_SARA, R_FORK, R_JOIN };
  struct PassRec {
    int kind = 0, branch = 0;
    RowFwdArgs<T> rf{};
    ColConvArgs<T> cc{};
    RowInvArgs<T> ri{};
    ColFwdArgs<T> cf{};
    ColInvArgs<T> ci{};
    DegridArgs<T> dg{};
    GridArgs<T> gr{};
    Ball1Args b1{};
    ZeroArgs z{};
    AxpyArgs<T> ax{};
    FinArgs fin{};
    SaraBatchInst<T> sara{};
  };
  std::vector<PassRec>* rec = nullptr;
  PassRec& record(int kind, cudaStream_t s) {
    rec->emplace_back();
    rec->back().kind = kind;
    rec->back().branch = (s == aux && aux != own) ? 1 : 0;
    return rec->back();
  }

  int partials_cap = 0;
  int size_partials() {
    const int np = std::max({2 * n_items, row_inv_blocks(g), sara_partials_capacity(g.n, levels),
                             vec_blocks(9 * N()), tv_partials(g.n), 1});
    if (2 * n_items > bpart_cap) {
      double* bnew = nullptr;
      const int rc = alloc(&bnew, size_t(std::max(2 * n_items, 1)));
      if (rc) return rc;
      bpart = bnew;
      bpart_cap = std::max(2 * n_items, 1);
    }
    if (np <= partials_cap) return PURIFY_OK;
    double* pnew = nullptr;
    const int rc = alloc(&pnew, np);
    if (rc) return rc;
    partials = pnew;
    partials_cap = np;
    return PURIFY_OK;
  }

  // Re-bin the visibilities by (block, tile, cell) for R data blocks.
  int set_blocks(const int* blocks, int R, cudaStream_t s) override {
    if (R < 1 || R > 64 || (R > 1 && !blocks)) return PURIFY_ERR_INVALID;
    std::vector<int> hb;
    std::vector<int64_t> sizes(R, 0);
    if (R > 1) {
      hb.resize(size_t(g.M));
      CK(cudaMemcpyAsync(hb.data(), blocks, hb.size() * sizeof(int), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      for (int b : hb) {
        if (b < 0 || b >= R) {
          note_error("purify_op_set_blocks", __LINE__, "block index out of range");
          return PURIFY_ERR_INVALID;
        }
        sizes[b] += 1;
      }
    } else {
      sizes[0] = g.M;
    }
    WorkItem* new_items = nullptr;
    int new_n = 0;
    const int rc =
        build_bins<T>(uv_keep, g.M, g, chunk, pos, perm, &new_items, &new_n, s, blocks, R, mem_pool ? mem_pool : lib_pool);
    if (rc) {
      note_error("uv binning failed", __LINE__, cudaGetErrorName(cudaGetLastError()));
      return rc;
    }
    CK(cudaStreamSynchronize(own));
    free_items();
    items = new_items;
    n_items = new_n;
    nblocks = R;
    ++struct_gen;
    block_sizes = sizes;
    return size_partials();
  }

  void free_items() {
    if (!items) return;
    if (items_pooled) cudaFreeAsync(items, pool_stream);
    else if (mem_pool || lib_pool) cudaFreeAsync(items, own);
    else cudaFree(items);
    items = nullptr;
  }

  ~OpImpl() override {
    run_release();
    if (gcache) cudaGraphExecDestroy(gcache);
    prof_release();
    if (own) cudaStreamSynchronize(own);
    if (aux) cudaStreamSynchronize(aux);
    free_items();
    if (pool_stream) {  // set-up operator: every use was on pool_stream
      for (void* a : allocs) cudaFreeAsync(a, pool_stream);
    } else if (mem_pool || lib_pool) {  // both streams are idle
      for (void* a : allocs) cudaFreeAsync(a, own);
    } else {
      for (void* a : allocs) cudaFree(a);
    }
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (ev_zfork) cudaEventDestroy(ev_zfork);
    if (ev_zjoin) cudaEventDestroy(ev_zjoin);
    if (aux2) cudaStreamSynchronize(aux2);
    if (aux2) cudaStreamDestroy(aux2);
    if (aux3) cudaStreamSynchronize(aux3);
    if (aux3) cudaStreamDestroy(aux3);
    if (ev_axf) cudaEventDestroy(ev_axf);
    if (ev_axj) cudaEventDestroy(ev_axj);
    if (own) cudaStreamDestroy(own);
    if (aux) cudaStreamDestroy(aux);
    if (h_sc) pinned_slots().put(h_sc);
  }

  template <typename U> int alloc(U** ptr, size_t count) {
    void* a = nullptr;
    const size_t b = count * sizeof(U) > 0 ? count * sizeof(U) : 16;
    if (pool_stream) {
      CK(setup_alloc(&a, b, pool_stream));
    } else if (mem_pool || lib_pool) {
      // complete before return, so that any stream may use it
      CK(cudaMallocFromPoolAsync(&a, b, mem_pool ? mem_pool : lib_pool, own));
      CK(cudaStreamSynchronize(own));
    } else {
      CK(cudaMalloc(&a, b));
    }
    allocs.push_back(a);
    bytes += int64_t(b);
    ++struct_gen;
    *ptr = static_cast<U*>(a);
    return PURIFY_OK;
  }

  size_t N() const { return size_t(g.n) * g.n; }
  // coefficients of the f_1 block: the dictionary's, or one per pixel for TV
  size_t D() const { return prior == 1 ? N() : size_t(sara.nbases) * N(); }

  int set_prior(int pr, int iters) override {
    if (run.active) {
      note_error("purify_op_set_prior", __LINE__, "a solve is in progress on this operator");
      return PURIFY_ERR_INVALID;
    }
    if ((pr != 0 && pr != 1) || (pr == 1 && (iters < 1 || iters > 100000))) {
      note_error("purify_op_set_prior", __LINE__, "prior must be 0 (l1 analysis) or 1 (TV, 1 <= tv_iters <= 1e5)");
      return PURIFY_ERR_INVALID;
    }
    prior = pr;
    if (pr == 1) tv_iters = iters;
    ++struct_gen;
    return PURIFY_OK;
  }

  // Dictionary of the l1 block: the SARA bases in `mask` (bit 0 Dirac, bit K DbK).
  int set_dictionary(unsigned mask) override {
    if (run.active) {
      note_error("purify_op_set_dictionary", __LINE__, "a solve is in progress on this operator");
      return PURIFY_ERR_INVALID;
    }
    SaraPlan<T> p = sara;
    if (sara_select(p, mask) < 0) {
      note_error("purify_op_set_dictionary", __LINE__, "mask must be a non-empty subset of bits 0..8");
      return PURIFY_ERR_INVALID;
    }
    sara = p;
    ++struct_gen;
    return PURIFY_OK;
  }
  unsigned dictionary(int* nbases) const override {
    unsigned m = sara.dirac ? 1u : 0u;
    for (int z = 0; z < sara.nf; ++z) m |= 2u << sara.fid[z];
    if (nbases) *nbases = sara.nbases;
    return m;
  }
  size_t grid_bytes() const { return size_t(g.KP) * g.KP * sizeof(C); }

  // light: gridding-only operator (Phi^H; no forward grid, no uv copy), as
  // the PSF set-up of the convolution form needs.
  bool light = false;
  // refine: light operator on the grid of twice the resolution of `refine`
  // (tile 8 there, 16 here), reusing its binning (items, order) instead of
  // sorting the visibilities again.
  int create(const double* uv, int64_t M, int n, int L, cudaStream_t s, int tile = 0, int chunk_opt = 0,
             bool light_only = false, const OpImpl* refine = nullptr, cudaMemPool_t pool = nullptr) {
    light = light_only || refine;
    mem_pool = light ? nullptr : pool;
    if (light) pool_stream = s;
    // An operator's own memory comes from the library's per-device pool,
    // which keeps released memory mapped (up to kSetupPoolKeep), so that the
    // next operator's creation reuses it instead of mapping new memory, and
    // destroying an operator does not synchronise the device (cudaFree would).
    if (!light && !mem_pool) lib_pool = library_pool();
    g.n = n;
    g.K = 2 * n;
    g.KP = g.K + kJ;
    g.pad_lo = kJ / 2 - 1;
    g.TB = tile > 0 ? tile : 8;
    if (g.TB > g.K) g.TB = g.K;
    g.ntile1d = g.K / g.TB;
    g.M = M;
    levels = L;
    // default work-item length by M (what purify_autotune usually picks:
    // many short items for small M, fewer long ones for large M)
    chunk = chunk_opt > 0 ? chunk_opt : (M < (int64_t(1) << 20) ? 256 : M >= (int64_t(1) << 21) ? 2048 : 1024);
    if (!light) {  // a set-up operator runs only on the caller's stream
      // the ball block is the longer branch of an iteration: its kernels'
      // CTAs go first when several branches have work waiting, then the
      // l1 / positivity blocks (own stream), then the A x_hat passes
      int lo = 0, hi = 0;
      CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      CK(cudaStreamCreateWithPriority(&own, cudaStreamNonBlocking, (lo + hi) / 2));
      CK(cudaStreamCreateWithPriority(&aux, cudaStreamNonBlocking, hi));
      CK(cudaStreamCreateWithPriority(&aux3, cudaStreamNonBlocking, lo));
      CK(cudaEventCreateWithFlags(&ev_axf, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ev_axj, cudaEventDisableTiming));
      CK(cudaStreamCreateWithFlags(&aux2, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&ev_zfork, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ev_zjoin, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
    }
    CK(configure_once<T>());
    // tables: deapodisation, twiddles, kernel polynomial, filters (host, double)
    const double beta = kb_beta(kJ, 2.0);
    std::vector<double> hd;
    kb_deapod_table(n, g.K, kJ, beta, hd);
    std::vector<T> hs(hd.begin(), hd.end());
    std::vector<C> htw(g.K);
    for (int m = 0; m < g.K; ++m) {
      const double a = -2.0 * M_PI * double(m) / g.K;
      htw[m].x = T(std::cos(a));
      htw[m].y = T(std::sin(a));
    }
    constexpr int D = KbDeg<T>::value;
    const std::vector<double>& coef = kb_poly_cached(kJ, beta, D);
    for (int a = 0; a < kJ; ++a)
      for (int d = 0; d <= D; ++d) kb.c[a][d] = T(coef[size_t(a) * (D + 1) + d]);
    std::memset(&sara.f, 0, sizeof(sara.f));
    for (int k = 1; k <= kMaxDb; ++k) {
      const std::vector<double>& h = daubechies_lowpass_cached(k);
      const int F = 2 * k;
      for (int m = 0; m < F; ++m) {
        sara.f.h[k - 1][m] = T(h[m]);
        sara.f.g[k - 1][m] = T(((m & 1) ? -1.0 : 1.0) * h[F - 1 - m]);
      }
    }
    int rc;
    if ((rc = alloc(&deapod, n))) return rc;
    if ((rc = alloc(&tw, g.K))) return rc;
    if ((rc = alloc(&pos, M))) return rc;
    if (!light) {
      if ((rc = alloc(&uv_keep, 2 * size_t(M)))) return rc;
      CK(cudaMemcpyAsync(uv_keep, uv, 2 * size_t(M) * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    if (!refine && (rc = alloc(&perm, M))) return rc;
    if ((rc = alloc(&gridA, size_t(n) * (g.K / 2)))) return rc;  // half-spectrum rows
    if (!light && (rc = alloc(&gridP, size_t(g.KP) * g.KP))) return rc;
    if ((rc = alloc(&gridQ, size_t(g.KP) * g.KP))) return rc;
    if ((rc = alloc(&sc, kNumScalars))) return rc;
    if ((rc = alloc(&err, 2))) return rc;  // [0] timed-out wait, [1] non-finite input
    sara.n = n;
    sara.levels = L;
    sara_select(sara, kSaraAll);
    h_sc = pinned_slots().get();
    if (!h_sc) {
      note_error("pinned host memory", __LINE__, "no pinned slot for the device scalars");
      return PURIFY_ERR_NOMEM;
    }
    CK(cudaMemcpyAsync(deapod, hs.data(), n * sizeof(T), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(tw, htw.data(), g.K * sizeof(C), cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(err, 0, 2 * sizeof(int), s));
    CK(cudaMemsetAsync(sc, 0, kNumScalars * sizeof(double), s));
    if (!light) launch_check_finite<double>(uv, 2 * size_t(M), err + 1, s);
    if (!light) CK(cudaMemsetAsync(gridP, 0, grid_bytes(), s));
    if (refine) {
      n_items = refine->n_items;
      CK(setup_alloc(&items, size_t(n_items > 0 ? n_items : 1) * sizeof(WorkItem), s));
      items_pooled = true;
      CK(cudaMemcpyAsync(items, refine->items, size_t(n_items) * sizeof(WorkItem), cudaMemcpyDeviceToDevice, s));
      launch_encode_x2<T>(refine->uv_keep, refine->perm, M, refine->g.K, g.TB, pos, s);
    } else {
      rc = build_bins<T>(uv, M, g, chunk, pos, perm, &items, &n_items, s, nullptr, 1, mem_pool ? mem_pool : lib_pool);
    }
    if (rc) {
      note_error("uv binning failed", __LINE__, cudaGetErrorName(cudaGetLastError()));
      return rc;
    }
    block_sizes.assign(1, M);
    if ((rc = size_partials())) return rc;
    if ((rc = alloc(&eps_dev, 64)) || (rc = alloc(&scale_dev, 64))) return rc;
    if ((rc = alloc(&cg_part, 5 * kCgPart))) return rc;
    if ((rc = alloc(&tickets, 4))) return rc;
    if ((rc = alloc(&fin_part, 2 * kFinCtas))) return rc;
    CK(cudaMemsetAsync(tickets, 0, 4 * sizeof(unsigned int), s));
    if (light) return check(s, false);  // its user synchronises s
    // TMA descriptor of the padded forward grid, 8-byte elements
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
      note_error("cuTensorMapEncodeTiled unavailable", __LINE__, "driver entry point not found");
      return PURIFY_ERR_CUDA;
    }
    const int cw = int(sizeof(C) / 8);
    const int PW = g.TB + kJ;
    cuuint64_t dims[2] = {cuuint64_t(g.KP) * cw, cuuint64_t(g.KP)};
    cuuint64_t strides[1] = {cuuint64_t(g.KP) * sizeof(C)};
    cuuint32_t box[2] = {cuuint32_t((PW + 2) * cw), cuuint32_t(PW)};  // PW rows of PW + 2 (bank spread)
    cuuint32_t estr[2] = {1, 1};
    CUresult cr = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, gridP, dims, strides, box, estr,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) {
      char buf[64];
      std::snprintf(buf, sizeof(buf), "CUresult %d", int(cr));
      note_error("cuTensorMapEncodeTiled failed", __LINE__, buf);
      return PURIFY_ERR_CUDA;
    }
    if ((rc = alloc(&tmap_dev, 1))) return rc;
    CK(cudaMemcpyAsync(tmap_dev, &tmap, sizeof(CUtensorMap), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    if ((rc = take_input_flag("purify_op_create", "uv holds a non-finite coordinate"))) return rc;
    return PURIFY_OK;
  }

  // Read and clear the non-finite-input flag (stream already synchronised).
  int take_input_flag(const char* who, const char* what) {
    int h = 0;
    CK(cudaMemcpy(&h, err + 1, sizeof(int), cudaMemcpyDeviceToHost));
    if (!h) return PURIFY_OK;
    CK(cudaMemset(err + 1, 0, sizeof(int)));
    note_error(who, __LINE__, what);
    return PURIFY_ERR_INVALID;
  }

  void info(int* n, int64_t* M, int* K, int* tile, int* ni, int* prec, int64_t* b) const override {
    if (n) *n = g.n;
    if (M) *M = g.M;
    if (K) *K = g.K;
    if (tile) *tile = g.TB;
    if (ni) *ni = n_items;
    if (prec) *prec = sizeof(T) == 4 ? PURIFY_FP32 : PURIFY_FP64;
    if (b) *b = bytes;
  }

  // ---- operator building blocks (enqueue only)
  // F Z S in real form (the image is real): row pairs to half spectra, then
  // the half-spectrum columns to the full padded grid with their mirrors.
  void fwd_grid(const RowPro<T>& pro, cudaStream_t s) {
    if (rec) {
      record(R_RF, s).rf = RowFwdArgs<T>{g, pro, deapod, gridA, tw, row_pass_nseq(g)};
      record(R_CF, s).cf = ColFwdArgs<T>{g, gridA, gridP, tw, col_pass_width<T>()};
      return;
    }
    PROF(KK_ROW_FWD, s, launch_row_fwd_h<T>(g, pro, deapod, gridA, tw, s));
    PROF(KK_COL_FWD, s, launch_col_fwd_h<T>(g, gridA, gridP, tw, s));
  }
  void zero_q(cudaStream_t s) {
    if (rec) {
      record(R_ZERO, s).z = ZeroArgs{gridQ, grid_bytes()};
      return;
    }
    PROF(KK_MEMSET, s, cudaMemsetAsync(gridQ, 0, grid_bytes(), s));
  }
  // Re F^H of the gridded accumulator: the half-spectrum columns of its
  // Hermitian part (the row pass follows in row_ep / normal_back).
  void col_inv(cudaStream_t s) {
    if (rec) {
      record(R_CI, s).ci = ColInvArgs<T>{g, gridQ, gridA, tw, col_pass_width<T>()};
      return;
    }
    PROF(KK_COL_INV, s, launch_col_inv_h<T>(g, gridQ, gridA, tw, s));
  }
  void degrid(const DegridEp<C>& ep, cudaStream_t s) {
    if (rec) {
      record(R_DG, s).dg = DegridArgs<T>{g, tmap_dev, items, n_items, pos, perm, ep, err};
      return;
    }
    PROF(KK_DEGRID, s, launch_degrid<T>(g, tmap, items, n_items, pos, perm, kb, ep, err, s));
  }
  void grid(const GridPro<C>& pro, cudaStream_t s) {
    if (rec) {
      record(R_GR, s).gr = GridArgs<T>{g, items, n_items, pos, perm, pro, gridQ};
      return;
    }
    PROF(KK_GRID, s, launch_grid<T>(g, items, n_items, pos, perm, kb, pro, gridQ, s));
  }
  void fin(const double* pa, int na, int op, double arg, cudaStream_t s) {
    if (rec) {
      record(R_FIN, s).fin = FinArgs{pa, na, op, arg, sc};
      return;
    }
    PROF(KK_VEC, s, launch_finalize<T>(pa, na, op, arg, sc, s));
  }
  RowPro<T> plain(const T* x) const {
    RowPro<T> pro{};
    pro.mode = PRO_PLAIN;
    pro.x = x;
    return pro;
  }
  // Re(Phi^H Phi) up to the row epilogue: forward passes, gram, inverse column pass.
  void gram_front(const RowPro<T>& pro, cudaStream_t s) {
    fwd_grid(pro, s);
    zero_q(s);
    PROF(KK_GRAM, s, launch_gram<T>(g, tmap, items, n_items, pos, kb, gridQ, err, s));
    col_inv(s);
  }
  int row_ep(const RowEp<T>& ep_in, cudaStream_t s) {
    RowEp<T> ep = ep_in;
    if (!ep.err) ep.err = err;
    if (rec) {
      record(R_RI, s).ri = RowInvArgs<T>{g, gridA, deapod, ep, tw, row_pass_nseq(g), row_inv_blocks(g)};
      return row_inv_blocks(g);
    }
    int np = 0;
    PROF(KK_ROW_INV, s, np = launch_row_inv_h<T>(g, gridA, deapod, ep, tw, s));
    return np;
  }

  // Set-up of the convolution form of Re(Phi^H Phi): the PSF
  // k(d) = sum_m exp(i k_m . d) over offsets d in [-n, n)^2 is Re Phi^H of
  // all-ones visibilities on a 2n x 2n image (same uv), and its spectrum on
  // the 2n grid is stored once.  Needs 2n <= 2048.
  int ensure_toeplitz(cudaStream_t s) {
    if (khat) return PURIFY_OK;
    if (2 * g.n > 2048) {
      note_error("convolution normal operator", __LINE__, "needs n <= 1024");
      return PURIFY_ERR_INVALID;
    }
    int rc;
    T* khat_l = nullptr;
    if ((rc = alloc(&khat_l, size_t(g.K / 2 + 1) * g.K))) return rc;
    if ((rc = alloc(&axh, N())) || (rc = alloc(&gridA2, size_t(g.n) * (g.K / 2)))) return rc;
    // The spectrum is built on s and not waited for here: its temporaries
    // return to the pool in stream order, and the caller's next work on s
    // comes after it.
    {
      OpImpl<T> big;
      const bool reuse = g.TB == 8;  // this binning serves the 2n operator (tiles 16 on its grid)
      rc = reuse ? big.create(uv_keep, g.M, 2 * g.n, 1, s, 16, chunk, true, this)
                 : big.create(uv_keep, g.M, 2 * g.n, 1, s, 0, 0, true);
      if (rc) return rc;
      C* y1 = nullptr;
      T* psf = nullptr;
      C* X = nullptr;
      // temporaries from the set-up pool
      cudaError_t e = setup_alloc(&y1, size_t(g.M) * sizeof(C), s);
      if (e == cudaSuccess) e = setup_alloc(&psf, size_t(g.K) * g.K * sizeof(T), s);
      if (e == cudaSuccess) e = setup_alloc(&X, size_t(g.K) * g.K * sizeof(C), s);
      if (e == cudaSuccess) {
        C one;
        one.x = T(1);
        one.y = T(0);
        launch_fill<C>(y1, size_t(g.M), one, s);
      }
      if (e == cudaSuccess) rc = big.adjoint_sorted(y1, psf, s);
      if (e == cudaSuccess && rc == 0) build_psf_spectrum<T>(psf, g.n, khat_l, X, tw, s);
      for (void* t : {static_cast<void*>(y1), static_cast<void*>(psf), static_cast<void*>(X)})
        if (t) cudaFreeAsync(t, s);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) return map_err(e, __LINE__);
      if (rc) return rc;
    }
    khat = khat_l;
    return PURIFY_OK;
  }

  // Front half of Re(Phi^H Phi) x: up to the half-spectrum rows in gridA, by the
  // NUFFT (G^H G per application) or by the precomputed convolution.
  // (The convolution form may run in the half-spectrum buffer `B` instead,
  // beside a pass of Phi or Phi^H in gridA.)
  void normal_front(const RowPro<T>& pro, cudaStream_t s, C* B = nullptr) {
    if (!B) B = gridA;
    if (rec) {  // the batched solver takes the convolution form only
      record(R_RF, s).rf = RowFwdArgs<T>{g, pro, nullptr, B, tw, row_pass_nseq(g)};
      record(R_CC, s).cc = ColConvArgs<T>{g, B, khat, khat + size_t(g.K / 2) * g.K, tw, col_pass_width<T>()};
      return;
    }
    if (toep) {
      PROF(KK_ROW_FWD_H, s, launch_row_fwd_h<T>(g, pro, nullptr, B, tw, s));
      PROF(KK_COL_CONV, s, launch_col_conv_h<T>(g, B, khat, tw, s));
    } else {
      gram_front(pro, s);
    }
  }
  int normal_back(const RowEp<T>& ep_in, cudaStream_t s, C* B = nullptr) {
    RowEp<T> ep = ep_in;
    if (!ep.err) ep.err = err;
    if (!B) B = gridA;
    if (rec) {
      record(R_RI, s).ri = RowInvArgs<T>{g, B, nullptr, ep, tw, row_pass_nseq(g), row_inv_blocks(g)};
      return row_inv_blocks(g);
    }
    int np = 0;
    if (toep) PROF(KK_ROW_INV_H, s, np = launch_row_inv_h<T>(g, B, nullptr, ep, tw, s));
    else PROF(KK_ROW_INV, s, np = launch_row_inv_h<T>(g, gridA, deapod, ep, tw, s));
    return np;
  }

  // out = (nu2 Re Phi^H Phi + 2I) x
  void normal_apply_qx(const T* x, T* out, double nu2, cudaStream_t s, C* B = nullptr) {
    normal_front(plain(x), s, B);
    RowEp<T> ep{};
    ep.mode = EP_QX;
    ep.out = out;
    ep.p = x;
    ep.nu2 = nu2;
    normal_back(ep, s, B);
  }

  int gram(const void* x, void* out, int mode, cudaStream_t s) override {
    if (mode != 0 && mode != 1) return PURIFY_ERR_INVALID;
    if (mode == 1) {
      const int rc = ensure_toeplitz(s);
      if (rc) return rc;
    }
    toep = mode == 1;
    normal_front(plain(static_cast<const T*>(x)), s);
    RowEp<T> ep{};
    ep.mode = EP_STORE;
    ep.out = static_cast<T*>(out);
    normal_back(ep, s);
    return check(s, false);
  }

  int check(cudaStream_t s, bool sync) {
    CK(cudaGetLastError());
    if (sync) {
      CK(cudaStreamSynchronize(s));
      int h = 0;
      CK(cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost));
      if (h) {
        cudaMemset(err, 0, sizeof(int));
        note_error("bounded device wait", __LINE__, "a TMA or bulk-copy wait gave up");
        return PURIFY_ERR_TIMEOUT;
      }
    }
    return PURIFY_OK;
  }

  // ---- public operators
  int phi(const void* x, void* y, cudaStream_t s) override {
    fwd_grid(plain(static_cast<const T*>(x)), s);
    DegridEp<C> ep{};
    ep.mode = DG_STORE_PERM;
    ep.y = static_cast<C*>(y);
    degrid(ep, s);
    return check(s, false);
  }

  int phi_adj(const void* y, void* x, cudaStream_t s) override {
    zero_q(s);
    GridPro<C> pro{};
    pro.mode = GP_PERM;
    pro.y = static_cast<const C*>(y);
    grid(pro, s);
    col_inv(s);
    RowEp<T> ep{};
    ep.mode = EP_STORE;
    ep.out = static_cast<T*>(x);
    row_ep(ep, s);
    return check(s, false);
  }

  // Re Phi^H y for y in the operator's sorted visibility order.
  int adjoint_sorted(const C* y, T* x, cudaStream_t s) {
    zero_q(s);
    GridPro<C> pro{};
    pro.mode = GP_SORTED;
    pro.y = y;
    grid(pro, s);
    col_inv(s);
    RowEp<T> ep{};
    ep.mode = EP_STORE;
    ep.out = x;
    row_ep(ep, s);
    return check(s, false);
  }

  // SARA scratch (bands and prox output), allocated on first use: an operator
  // used only for Phi / Phi^H (e.g. the PSF set-up) never needs it.
  int ensure_sara() {
    if (sara.cs) return PURIFY_OK;
    int rc;
    if ((rc = alloc(&sara.s0, 8 * N() / 4)) || (rc = alloc(&sara.s1, 8 * N() / 4)) || (rc = alloc(&sara.cs, 9 * N())))
      return rc;
    return PURIFY_OK;
  }

  int sara_fwd(const void* x, void* c, cudaStream_t s) override {
    if (const int rc = ensure_sara()) return rc;
    PROF(KK_SARA_ANA, s, sara_analysis<T>(sara, static_cast<const T*>(x), static_cast<T*>(c), s));
    return check(s, false);
  }
  int sara_adj(const void* c, void* x, cudaStream_t s) override {
    if (const int rc = ensure_sara()) return rc;
    PROF(KK_SARA_SYN, s, sara_synthesis<T>(sara, static_cast<const T*>(c), static_cast<T*>(x), s));
    return check(s, false);
  }

  // ---- solver
  int ensure_solver() {
    if (xh) return PURIFY_OK;
    int rc;
    if ((rc = ensure_sara())) return rc;
    const size_t n2 = N();
    if ((rc = alloc(&xh, n2)) || (rc = alloc(&xs, n2)) || (rc = alloc(&r, n2)) || (rc = alloc(&p, n2)) ||
        (rc = alloc(&Ap, n2)) || (rc = alloc(&z1, 9 * n2)) || (rc = alloc(&z2, n2)) || (rc = alloc(&w, 9 * n2)) ||
        (rc = alloc(&z3, size_t(g.M))) || (rc = alloc(&ys, size_t(g.M))))
      return rc;
    return PURIFY_OK;
  }
  int ensure_tv() {
    if (tvq) return PURIFY_OK;
    return alloc(&tvq, 4 * N());
  }

  int read_scalars(cudaStream_t s) {
    CK(cudaMemcpyAsync(h_sc, sc, kNumScalars * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return PURIFY_OK;
  }

  // ||Phi||^2 by power iteration on Re(Phi^H Phi) from the all-ones image / n.
  int power_norm_sq(int iters, double* lam, cudaStream_t s) {
    launch_fill<T>(p, N(), T(1.0 / g.n), s);
    for (int it = 0; it < iters; ++it) {
      RowPro<T> pro{};
      if (it == 0) {
        pro = plain(p);
      } else {
        pro.mode = PRO_SCALE;
        pro.x = Ap;
        pro.scalars = sc;
        pro.idx = S_INVNORM;
      }
      normal_front(pro, s);
      RowEp<T> ep{};
      ep.mode = EP_POWER;
      ep.out = Ap;
      ep.partials = partials;
      const int np = normal_back(ep, s);
      fin(partials, np, FIN_NORM, 0.0, s);
    }
    int rc = check(s, true);
    if (rc) return rc;
    if ((rc = read_scalars(s))) return rc;
    *lam = h_sc[S_LAMBDA];
    return PURIFY_OK;
  }

  // 1e-3 ||Psi^H (nu^2 Re Phi^H y)||_inf with y the sorted visibilities
  // (Psi^H = I for the TV prior).
  int default_gamma(double nu, double* gamma, cudaStream_t s) {
    zero_q(s);
    GridPro<C> pro{};
    pro.mode = GP_SORTED;
    pro.y = ys;
    grid(pro, s);
    col_inv(s);
    RowEp<T> ep{};
    ep.mode = EP_STORE;
    ep.out = Ap;
    row_ep(ep, s);
    const T* coef = Ap;  // TV: the back-projection itself (L_1 = I)
    if (prior == 0) {
      sara_analysis<T>(sara, Ap, z1, s);
      coef = z1;
    }
    const int np = launch_reduce<T>(coef, D(), RED_MAXABS, sc, partials, s);
    launch_max_partials(partials, np, sc, s);
    int rc = check(s, true);
    if (rc) return rc;
    if ((rc = read_scalars(s))) return rc;
    *gamma = 1e-3 * nu * nu * h_sc[S_MAXABS];
    return PURIFY_OK;
  }

  // Population standard deviation of Psi^H x_hat (reweighting delta_1), or
  // of the gradient magnitudes |grad x_hat| for the TV prior.
  int coef_std(double* out, cudaStream_t s) {
    if (prior == 1) tv_magnitude<T>(xh, z1, g.n, s);
    else sara_analysis<T>(sara, xh, z1, s);
    const size_t D = this->D();
    int np = launch_reduce<T>(z1, D, RED_SUM, sc, partials, s);
    launch_finalize<T>(partials, np, FIN_MEAN, double(D), sc, s);
    np = launch_reduce<T>(z1, D, RED_VAR, sc, partials, s);
    launch_finalize<T>(partials, np, FIN_VAR, double(D), sc, s);
    int rc = check(s, true);
    if (rc) return rc;
    if ((rc = read_scalars(s))) return rc;
    *out = h_sc[S_STD];
    return PURIFY_OK;
  }

  // One SDMM iteration (Algorithm 1, steps 5-10), enqueue only.
  void iteration(double nu, double gamma, double eps, int cg_iters, cudaStream_t s) {
    const double nu2 = nu * nu;
    const size_t n2 = N();
    // step 5: x_hat = (Phi^H Phi + 2I)^-1 sum_i x_i by CG, warm-started at x_hat.
    // The scalars stay on the device and need no launches of their own: the
    // last block of the inverse row pass sets <r,r> (initial residual), or
    // alpha and beta (CG step, from five inner products of the step's vectors);
    // the forward row pass of the next step applies x += alpha p,
    // r -= alpha Ap, p = r + beta p on the fly.  With the convolution form the
    // initial residual b - A x_hat needs no operator pass here: A x_hat was
    // formed at the end of the previous iteration beside the ball block (or by
    // the round set-up), and the first forward row pass takes r = p = b - A x_hat.
    if (!toep) {
      normal_front(plain(xh), s);
      RowEp<T> ep{};
      ep.mode = EP_CG_R0;
      ep.out = r;
      ep.out2 = p;
      ep.p = xh;
      ep.b = xs;
      ep.nu2 = nu2;
      ep.partials = cg_part;
      ep.pstride = kCgPart;
      ep.scalars = sc;
      ep.ticket = tickets;
      normal_back(ep, s);
    }
    for (int it = 0; it < cg_iters; ++it) {
      RowPro<T> pro = plain(p);
      if (it == 0 && toep) {
        pro.mode = PRO_CG_START;
        pro.x = xs;
        pro.ap = axh;
        pro.p = p;
        pro.r = r;
      } else if (it > 0) {
        pro.mode = PRO_CG_STEP;
        pro.p = p;
        pro.r = r;
        pro.xu = xh;
        pro.ap = Ap;
        pro.scalars = sc;
      }
      normal_front(pro, s);
      RowEp<T> ep{};
      ep.mode = EP_CG_AP;
      ep.out = Ap;
      ep.p = p;
      ep.r = r;
      ep.nu2 = nu2;
      ep.partials = cg_part;
      ep.pstride = kCgPart;
      ep.scalars = sc;
      ep.ticket = tickets + 1;
      normal_back(ep, s);
    }
    if (cg_iters > 0) {  // last step: x += alpha p
      if (rec) record(R_AXPY, s).ax = AxpyArgs<T>{xh, p, sc, S_ALPHA, n2};
      else PROF(KK_VEC, s, launch_axpy<T>(xh, p, sc, S_ALPHA, n2, s));
    }
    // The three proximal blocks (steps 6-8) are independent until their sum:
    // the ball block's degridding, projection and gridding run on the second
    // stream beside the l1 and positivity blocks, and the join feeds its last
    // pass, which adds nu Re Phi^H (2 r_3 - v_3) to x_1 + x_2.
    // (With kernel timing enabled both branches stay on one stream, so that
    // every kernel's time is its own.)
    cudaStream_t b3 = prof ? s : aux;
    if (rec) {
      record(R_FORK, s);
    } else if (b3 != s) {
      cudaEventRecord(ev_fork, s);
      cudaStreamWaitEvent(b3, ev_fork, 0);
    }
    // block 3 (data fidelity): v = nu Phi x_hat + z_3, project on the ball.
    // The gridding accumulator is zeroed on a third stream meanwhile (nothing
    // before the gridding pass touches it).
    const bool zpar = !rec && b3 != s;
    if (zpar && toep) {  // A x_hat for the next CG start on its own, lowest-priority stream
      cudaEventRecord(ev_axf, s);
      cudaStreamWaitEvent(aux3, ev_axf, 0);
      normal_apply_qx(xh, axh, nu2, aux3, gridA2);
      cudaEventRecord(ev_axj, aux3);
    }
    if (zpar) {
      cudaEventRecord(ev_zfork, b3);
      cudaStreamWaitEvent(aux2, ev_zfork, 0);
      zero_q(aux2);
      cudaEventRecord(ev_zjoin, aux2);
    }
    fwd_grid(plain(xh), b3);
    DegridEp<C> dep{};
    dep.mode = DG_BALL;
    dep.z = z3;
    dep.ys = ys;
    dep.nu = nu;
    dep.part0 = bpart;
    dep.part1 = bpart + n_items;
    degrid(dep, b3);
    if (rec)
      record(R_B1, b3).b1 = Ball1Args{bpart, bpart + n_items, n_items, nu, eps_dev, scale_dev, sc, fin_part, tickets + 2};
    else
      PROF(KK_VEC, b3, launch_finalize_blocks<T>(bpart, bpart + n_items, reinterpret_cast<const int*>(items), n_items,
                                                  nblocks, nu, eps_dev, scale_dev, sc, fin_part, tickets + 2, b3));
    if (zpar) cudaStreamWaitEvent(b3, ev_zjoin, 0);
    else zero_q(b3);
    GridPro<C> gp{};
    gp.mode = GP_BALL;
    gp.z = z3;
    gp.ys = ys;
    gp.nu = nu;
    gp.scalars = sc;
    gp.scale_idx = S_BALLSCALE;
    gp.block_scale = scale_dev;
    grid(gp, b3);
    col_inv(b3);
    if (!rec && b3 != s) cudaEventRecord(ev_join, b3);
    if (prior == 1) {
      // block 1 (weighted TV, L_1 = I) with block 2 (positivity) in its
      // epilogue: xs = x_1 + x_2
      TvBlock<T> tb{};
      tb.n = g.n;
      tb.iters = tv_iters;
      tb.gamma = gamma;
      tb.xh = xh;
      tb.z1 = z1;
      tb.z2 = z2;
      tb.w = w;
      tb.v = sara.cs;
      tb.qa = tvq;
      tb.qb = tvq + 2 * n2;
      tb.xs = xs;
      tb.partials = partials;
      int npo = 0;
      PROF(KK_TV, s, npo = tv_block<T>(tb, s));
      fin(partials, npo, FIN_OBJ, 0.0, s);
    } else if (rec) {
      record(R_SARA, s).sara = SaraBatchInst<T>{&sara, xh, z1, w, gamma, partials, z2, xs};
      fin(partials, sara_prox_partials<T>(sara), FIN_OBJ, 0.0, s);
    } else {
      // block 1 (l1 on Psi^H x_hat) fused into the analysis, block 2 (positivity)
      // fused into the synthesis: xs = x_1 + x_2
      L1Block<T> b1{};
      b1.z1 = z1;
      b1.w = w;
      b1.gamma = gamma;
      b1.partials = partials;
      int npo = 0;
      PROF(KK_SARA_ANA, s, npo = sara_analysis_prox<T>(sara, xh, b1, s));
      fin(partials, npo, FIN_OBJ, 0.0, s);
      PROF(KK_SARA_SYN, s, sara_synthesis_pos<T>(sara, xh, z2, xs, s));
    }
    // A x_hat for the next iteration's CG start (on the lowest-priority
    // stream when the branches run side by side), in its own half-spectrum buffer
    if (toep && !zpar) normal_apply_qx(xh, axh, nu2, s, gridA2);
    if (toep && zpar) cudaStreamWaitEvent(s, ev_axj, 0);
    // join: xs += nu Re Phi^H (2 r_3 - v_3) (the batched record joins here too,
    // so that its l1 and positivity blocks also run beside the ball block)
    if (rec) record(R_JOIN, s);
    else if (b3 != s) cudaStreamWaitEvent(s, ev_join, 0);
    RowEp<T> ep{};
    ep.mode = EP_XS_ADD;
    ep.out = xs;
    ep.b = xs;
    ep.nu = nu;
    row_ep(ep, s);
  }

  // ---- resumable solve: begin, then (launch one iteration, check) pairs, then
  // end.  The blocking purify_sdmm_solve and the request server share it.
  // Everything runs on the operator's own stream (the caller's stream may be
  // the legacy default stream, which cannot be captured into a graph),
  // ordered after the caller's prior work and before its later work by events.
  struct Run {
    purify_params P{};
    std::vector<double> eps_b;
    double nu = 0, gamma = 0, decay = 0.1, delta1 = 0, prev = -1;
    int round = 0, t = 0, total = 0, converged = 0;
    bool active = false, round_ready = false;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr, ev_sc = nullptr;
  } run;

  void run_release() {
    if (run.e0) cudaEventDestroy(run.e0);
    if (run.e1) cudaEventDestroy(run.e1);
    if (run.ev_sc) cudaEventDestroy(run.ev_sc);
    run.gexec = nullptr;
    run.e0 = run.e1 = run.ev_sc = nullptr;
    run.active = false;
  }

  int begin(const void* y, const purify_params* P, cudaStream_t user) override {
    if (!(P->eps > 0) || P->t_max < 1 || P->cg_iters < 1 || P->n_reweight < 0 || P->xi < 0 ||
        (P->nu <= 0 && P->power_iters < 1))
      return PURIFY_ERR_INVALID;
    if (run.active) run_release();
    int rc = ensure_solver();
    if (!rc && prior == 1) rc = ensure_tv();
    if (rc) return rc;
    cudaStream_t s = own;
    CK(cudaEventRecord(ev_in, user));
    CK(cudaStreamWaitEvent(s, ev_in, 0));
    run = Run();
    run.P = *P;
    run.P.eps_blocks = nullptr;
    CK(cudaEventCreate(&run.e0));
    CK(cudaEventCreate(&run.e1));
    CK(cudaEventCreateWithFlags(&run.ev_sc, cudaEventDisableTiming));
    CK(cudaEventRecord(run.e0, s));
    const size_t n2 = N(), M = size_t(g.M);
    run.eps_b.resize(nblocks);
    for (int b = 0; b < nblocks; ++b)
      run.eps_b[b] = (nblocks > 1 && P->eps_blocks) ? P->eps_blocks[b]
                                                     : P->eps * std::sqrt(double(block_sizes[b]) / double(g.M));
    for (double e : run.eps_b)
      if (!(e > 0)) return PURIFY_ERR_INVALID;
    CK(cudaMemcpyAsync(eps_dev, run.eps_b.data(), nblocks * sizeof(double), cudaMemcpyHostToDevice, s));
    const int gmode = P->gram < 0 ? (g.n <= 1024 ? 1 : 0) : P->gram;
    if (gmode == 1 && (rc = ensure_toeplitz(s))) return rc;
    toep = gmode == 1;
    launch_gather<C>(static_cast<const C*>(y), perm, M, ys, s);
    launch_check_finite<T>(reinterpret_cast<const T*>(ys), 2 * M, err + 1, s);
    run.nu = P->nu;
    run.gamma = P->gamma;
    run.decay = P->delta_decay > 0 ? P->delta_decay : 0.1;
    // With nu and gamma given, the iteration graph is captured while the
    // device still runs the set-up above (the PSF spectrum, the gather).
    const bool early = run.nu > 0 && run.gamma > 0;
    if (early && (rc = capture_iteration(s))) return rc;
    CK(cudaStreamSynchronize(s));
    if ((rc = take_input_flag("purify_sdmm_solve", "y holds a non-finite visibility"))) return rc;
    if (!(run.nu > 0)) {
      double lam = 0;
      if ((rc = power_norm_sq(P->power_iters, &lam, s))) return rc;
      run.nu = lam > 0 ? 1.0 / std::sqrt(lam) : 1.0;
    }
    if (!(run.gamma > 0)) {
      if ((rc = default_gamma(run.nu, &run.gamma, s))) return rc;
      if (!(run.gamma > 0)) run.gamma = 1e-12;
    }
    if (!early && (rc = capture_iteration(s))) return rc;
    launch_fill<T>(w, D(), T(1), s);
    CK(cudaMemsetAsync(xh, 0, n2 * sizeof(T), s));
    CK(cudaMemsetAsync(sc + S_CG0, 0, 5 * sizeof(double), s));  // the CG's accumulators start at zero
    run.active = true;
    own_pending = true;
    return check(s, false);
  }

  // One SDMM iteration captured as a CUDA graph (when the parameters ask for
  // replay), with the current nu and gamma baked into its kernel arguments.
  // The graph stays with the operator: a later solve with the same scalars,
  // CG steps and pass structure (no buffer allocated, re-binned or
  // re-planned since: struct_gen) replays it without capturing again.
  struct GraphKey {
    double nu, gamma, eps;
    int cg, toep, prior, tv_iters, nblocks;
    unsigned dict;
    uint64_t gen;
    bool operator==(const GraphKey& o) const {
      return nu == o.nu && gamma == o.gamma && eps == o.eps && cg == o.cg && toep == o.toep && prior == o.prior &&
             tv_iters == o.tv_iters && nblocks == o.nblocks && dict == o.dict && gen == o.gen;
    }
  };
  cudaGraphExec_t gcache = nullptr;
  GraphKey gkey{};
  uint64_t struct_gen = 0;
  int capture_iteration(cudaStream_t s) {
    run.gexec = nullptr;
    if (!run.P.use_graph || prof) return PURIFY_OK;
    const GraphKey k{run.nu,   run.gamma, run.P.eps, run.P.cg_iters, toep ? 1 : 0, prior, tv_iters,
                     nblocks,  dictionary(nullptr), struct_gen};
    if (gcache && k == gkey) {
      run.gexec = gcache;
      return PURIFY_OK;
    }
    if (gcache) {
      cudaGraphExecDestroy(gcache);
      gcache = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    iteration(run.nu, run.gamma, run.P.eps, run.P.cg_iters, s);
    cudaError_t ce = cudaStreamEndCapture(s, &graph);
    if (ce != cudaSuccess) return map_err(ce, __LINE__);
    ce = cudaGraphInstantiate(&gcache, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      gcache = nullptr;
      return map_err(ce, __LINE__);
    }
    gkey = k;
    run.gexec = gcache;
    return PURIFY_OK;
  }

  // ---- iteration-level batching in the request server: the solves of one
  // key (image side, precision, CG steps, dictionary) advance together
  // through a batched graph; these hooks do each solve's part around it.
  uint64_t batch_key() const override {
    if (!run.active || !toep || prior != 0 || nblocks != 1 || g.n < 64 || g.n > 1024 || prof) return 0;
    return uint64_t(g.n) | (uint64_t(sizeof(T) == 4 ? 1 : 2) << 12) | (uint64_t(run.P.cg_iters) << 16) |
           (uint64_t(dictionary(nullptr)) << 32);
  }
  int prepare_iteration(cudaStream_t s) override {
    if (!run.active) return PURIFY_ERR_INVALID;
    if (own_pending) {  // work begin() or a solo iteration left on the own stream comes first
      CK(cudaEventRecord(ev_in, own));
      CK(cudaStreamWaitEvent(s, ev_in, 0));
      own_pending = false;
    }
    return run.round_ready ? PURIFY_OK : start_round(s);
  }
  int finish_iteration(cudaStream_t s) override {
    if (!run.active) return PURIFY_ERR_INVALID;
    if (run.P.xi > 0) {
      CK(cudaMemcpyAsync(h_sc, sc, kNumScalars * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(run.ev_sc, s));
    }
    return PURIFY_OK;
  }

  int run_steps(int max_iters, int* done) override {
    *done = 0;
    if (!run.active || max_iters < 0) return PURIFY_ERR_INVALID;
    int rc = PURIFY_OK;
    for (int k = 0; k < max_iters && !*done && !rc; ++k) {
      rc = step_launch();
      if (!rc) rc = step_check(done);
    }
    if (!rc) rc = check(own, true);
    return rc;
  }

  // ---- checkpoint: the state an SDMM iteration carries to the next
  // (Algorithm 1: x_hat, sum_i x_i and the duals z_1, z_2, z_3), the SARA
  // weights of the round and the loop counters.  CG vectors restart from
  // x_hat every iteration and are not state.
  struct StateHeader {
    uint32_t magic, version;
    int32_t precision, n;
    int64_t M;
    int32_t nbases, nblocks, round, t, total, converged, round_ready, prior;
    double nu, gamma, delta1, prev;
  };
  static constexpr uint32_t kStateMagic = 0x4D445350u;  // "PSDM"
  int64_t state_bytes() const override {
    const size_t tv = prior == 1 ? 2 * N() : 0;  // the TV prox's warm-started dual
    return int64_t(sizeof(StateHeader)) + int64_t((3 * N() + 2 * D() + 2 * size_t(g.M) + tv) * sizeof(T));
  }
  // (device array, element count) pairs in checkpoint order; returns their number.
  int state_arrays(T* (&a)[7], size_t (&len)[7]) const {
    T* arr[7] = {xh, xs, z1, z2, w, reinterpret_cast<T*>(z3), tvq};
    const size_t l[7] = {N(), N(), D(), N(), D(), 2 * size_t(g.M), 2 * N()};
    for (int k = 0; k < 7; ++k) {
      a[k] = arr[k];
      len[k] = l[k];
    }
    return prior == 1 ? 7 : 6;
  }
  int save_state(void* host, int64_t bytes) override {
    if (!run.active || !host || bytes < state_bytes()) return PURIFY_ERR_INVALID;
    CK(cudaStreamSynchronize(own));
    StateHeader h{};
    h.magic = kStateMagic;
    h.version = 1;
    h.precision = sizeof(T) == 4 ? PURIFY_FP32 : PURIFY_FP64;
    h.n = g.n;
    h.M = g.M;
    h.nbases = sara.nbases;
    h.nblocks = nblocks;
    h.round = run.round;
    h.t = run.t;
    h.total = run.total;
    h.converged = run.converged;
    h.round_ready = run.round_ready ? 1 : 0;
    h.prior = prior;
    h.nu = run.nu;
    h.gamma = run.gamma;
    h.delta1 = run.delta1;
    h.prev = run.prev;
    unsigned char* dst = static_cast<unsigned char*>(host);
    std::memcpy(dst, &h, sizeof(h));
    dst += sizeof(h);
    T* a[7];
    size_t len[7];
    const int na = state_arrays(a, len);
    for (int k = 0; k < na; ++k) {
      CK(cudaMemcpy(dst, a[k], len[k] * sizeof(T), cudaMemcpyDeviceToHost));
      dst += len[k] * sizeof(T);
    }
    return PURIFY_OK;
  }
  int load_state(const void* host, int64_t bytes) override {
    if (!run.active || !host || bytes < state_bytes()) return PURIFY_ERR_INVALID;
    StateHeader h;
    std::memcpy(&h, host, sizeof(h));
    if (h.magic != kStateMagic || h.version != 1 || h.precision != (sizeof(T) == 4 ? PURIFY_FP32 : PURIFY_FP64) ||
        h.n != g.n || h.M != g.M || h.nbases != sara.nbases || h.nblocks != nblocks || h.prior != prior ||
        h.round > run.P.n_reweight) {
      note_error("purify_solve_load", __LINE__, "checkpoint does not match this operator or solve");
      return PURIFY_ERR_INVALID;
    }
    CK(cudaStreamSynchronize(own));
    const unsigned char* src = static_cast<const unsigned char*>(host) + sizeof(h);
    T* a[7];
    size_t len[7];
    const int na = state_arrays(a, len);
    for (int k = 0; k < na; ++k) {
      CK(cudaMemcpy(a[k], src, len[k] * sizeof(T), cudaMemcpyHostToDevice));
      src += len[k] * sizeof(T);
    }
    run.round = h.round;
    run.t = h.t;
    run.total = h.total;
    run.converged = h.converged;
    run.round_ready = h.round_ready != 0;
    run.delta1 = h.delta1;
    run.prev = h.prev;
    if (h.nu != run.nu || h.gamma != run.gamma) {
      run.nu = h.nu;
      run.gamma = h.gamma;
      int rc = capture_iteration(own);
      if (rc) return rc;
    }
    // the CG start's A x_hat is not state: it is formed again from x_hat by
    // the same passes as in the iteration
    if (toep && run.round_ready) normal_apply_qx(xh, axh, run.nu * run.nu, own);
    return check(own, true);
  }

  // Round set-up (Algorithm 1 steps 1-3; SARA weights from the previous round).
  int start_round(cudaStream_t s) {
    const size_t n2 = N(), M = size_t(g.M);
    const purify_params& P = run.P;
    int rc;
    if (run.round > 0) {
      if (run.round == 1) {
        if (P.delta0 > 0) {
          run.delta1 = P.delta0;
        } else if ((rc = coef_std(&run.delta1, s))) {
          return rc;
        }
        if (!(run.delta1 > 0)) run.delta1 = 1.0;
      }
      const double dmin = P.delta_min > 0 ? P.delta_min : 1e-4 * run.delta1;
      const double delta = std::max(std::pow(run.decay, run.round - 1) * run.delta1, dmin);
      if (prior == 1) tv_magnitude<T>(xh, w, g.n, s);  // RWTV: delta / (delta + |grad x_hat|)
      else sara_analysis<T>(sara, xh, w, s);
      launch_reweight<T>(w, D(), delta, s);
    }
    cudaMemsetAsync(z1, 0, D() * sizeof(T), s);
    if (prior == 1) cudaMemsetAsync(tvq, 0, 2 * n2 * sizeof(T), s);
    cudaMemsetAsync(z2, 0, n2 * sizeof(T), s);
    cudaMemsetAsync(z3, 0, M * sizeof(C), s);
    if (run.round > 0 && P.warm_start) {
      // steps 1-3 with x_hat^(0) = previous solution: sum_i x_i = (Phi^H Phi + 2I) x_hat^(0)
      normal_apply_qx(xh, xs, run.nu * run.nu, s);
      if (toep) cudaMemcpyAsync(axh, xs, n2 * sizeof(T), cudaMemcpyDeviceToDevice, s);  // the CG start's A x_hat
    } else {
      cudaMemsetAsync(xh, 0, n2 * sizeof(T), s);
      cudaMemsetAsync(xs, 0, n2 * sizeof(T), s);
      if (toep) cudaMemsetAsync(axh, 0, n2 * sizeof(T), s);
    }
    run.t = 0;
    run.prev = -1.0;
    run.converged = 0;
    run.round_ready = true;
    return check(s, false);
  }

  // Enqueue one SDMM iteration (after the round set-up when a round starts).
  int step_launch() override {
    if (!run.active) return PURIFY_ERR_INVALID;
    cudaStream_t s = own;
    int rc;
    own_pending = true;
    if (!run.round_ready && (rc = start_round(s))) return rc;
    if (run.gexec) {
      CK(cudaGraphLaunch(run.gexec, s));
    } else {
      iteration(run.nu, run.gamma, run.P.eps, run.P.cg_iters, s);
    }
    if (run.P.xi > 0) {
      CK(cudaMemcpyAsync(h_sc, sc, kNumScalars * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaEventRecord(run.ev_sc, s));
    }
    return check(s, false);
  }

  // After the launched iteration: the halting test (Section 3) and the round
  // bookkeeping; *done = 1 when the last round has finished.
  int step_check(int* done) override {
    *done = 0;
    if (!run.active) return PURIFY_ERR_INVALID;
    ++run.t;
    ++run.total;
    if (run.P.xi > 0) {
      CK(cudaEventSynchronize(run.ev_sc));
      const double f = h_sc[S_OBJ], feas = h_sc[S_FEAS];
      if (run.prev >= 0 && std::fabs(f - run.prev) / std::max(run.prev, 1e-300) < run.P.xi && feas <= 1 + 1e-3)
        run.converged = 1;
      run.prev = f;
    }
    if (run.converged || run.t >= run.P.t_max) {
      if (run.round >= run.P.n_reweight) {
        *done = 1;
      } else {
        ++run.round;
        run.round_ready = false;
      }
    }
    return PURIFY_OK;
  }

  int end(void* x_out, purify_stats* st, cudaStream_t user) override {
    if (!run.active) return PURIFY_ERR_INVALID;
    cudaStream_t s = own;
    int rc = PURIFY_OK;
    const size_t n2 = N();
    cudaError_t e = cudaMemcpyAsync(x_out, xh, n2 * sizeof(T), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaEventRecord(run.e1, s);
    if (e != cudaSuccess) rc = map_err(e, __LINE__);
    if (!rc) rc = check(s, true);
    if (!rc) rc = read_scalars(s);
    prof_collect();
    float ms = 0.f;
    if (!rc) cudaEventElapsedTime(&ms, run.e0, run.e1);
    if (!rc && st) {
      st->iterations = run.total;
      st->rounds = run.round + 1;
      st->converged = run.converged;
      st->objective = h_sc[S_OBJ];
      st->residual = h_sc[S_RESID];
      st->nu = run.nu;
      st->gamma = run.gamma;
      st->elapsed_ms = ms;
    }
    const bool not_conv = run.P.xi > 0 && !run.converged;
    if (!rc && !(std::isfinite(h_sc[S_OBJ]) && std::isfinite(h_sc[S_RESID]))) {
      note_error("purify_sdmm_solve", __LINE__, "objective or residual is not finite");
      rc = PURIFY_ERR_NONFINITE;
    }
    run_release();
    cudaEventRecord(ev_out, s);
    cudaStreamWaitEvent(user, ev_out, 0);
    if (rc) return rc;
    return not_conv ? PURIFY_ERR_NOT_CONVERGED : PURIFY_OK;
  }

  int solve(const void* y, const purify_params* P, void* x_out, purify_stats* st, cudaStream_t user) override {
    int rc = begin(y, P, user);
    int done = 0;
    while (!rc && !done) {
      rc = step_launch();
      if (!rc) rc = step_check(&done);
    }
    if (rc) {
      if (run.active) run_release();
      cudaEventRecord(ev_out, own);
      cudaStreamWaitEvent(user, ev_out, 0);
      return rc;
    }
    return end(x_out, st, user);
  }

  cudaStream_t stream() const override { return own; }

  int sorted_pair(const void* x, void* y, void* out, cudaStream_t s) override {
    fwd_grid(plain(static_cast<const T*>(x)), s);
    DegridEp<C> ep{};
    ep.mode = DG_STORE_SORTED;
    ep.y = static_cast<C*>(y);
    degrid(ep, s);
    zero_q(s);
    GridPro<C> pro{};
    pro.mode = GP_SORTED;
    pro.y = static_cast<const C*>(y);
    grid(pro, s);
    col_inv(s);
    RowEp<T> rep{};
    rep.mode = EP_STORE;
    rep.out = static_cast<T*>(out);
    row_ep(rep, s);
    return check(s, false);
  }
};

// ---------------------------------------------------------------------------
// Batched solver: many independent SARA-SDMM instances (different images, uv
// coverages and visibility counts) advanced together.  Instances are grouped
// by image side; for each group every pass of an SDMM iteration -- the CG
// passes, the ball block, the SARA blocks, the vector steps -- is ONE launch
// over all of the group's instances, its arguments read from a device table
// (one entry per instance, recorded from each instance's own iteration so
// that the batched passes are exactly the single-instance ones).  One SDMM
// iteration of the whole batch is one captured CUDA graph whose groups run
// as parallel branches.
template <typename T> class BatchImpl {
  typedef typename OpImpl<T>::PassRec Rec;

 public:
  struct Group {
    std::vector<int> idx;              // instances (indices into ops)
    std::vector<int> kinds, branches;  // the recorded pass sequence
    std::vector<size_t> off;           // offset of each pass's table in the group's buffer
    void* dev = nullptr;
    SaraBatch<T>* sara = nullptr;
    int max_items = 0, max_tb = 8;
    size_t max_q = 0;
    cudaStream_t main = nullptr, aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, done = nullptr;
  };
  std::vector<OpImpl<T>*> ops;
  std::vector<Group> groups;
  cudaMemPool_t pool = nullptr;  // tables from this pool (the request server's) when set
  cudaStream_t bs = nullptr;
  cudaEvent_t ev0 = nullptr;
  cudaGraphExec_t gexec = nullptr;

  ~BatchImpl() {
    if (bs) cudaStreamSynchronize(bs);
    if (gexec) cudaGraphExecDestroy(gexec);
    for (Group& gr : groups) {
      if (gr.dev) {
        if (pool) cudaFreeAsync(gr.dev, bs);
        else cudaFree(gr.dev);
      }
      sara_batch_destroy(gr.sara);
      const cudaEvent_t evs[3] = {gr.fork, gr.join, gr.done};
      for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
      if (gr.main) cudaStreamDestroy(gr.main);
      if (gr.aux) cudaStreamDestroy(gr.aux);
    }
    if (ev0) cudaEventDestroy(ev0);
    if (bs) cudaStreamSynchronize(bs);
    if (bs) cudaStreamDestroy(bs);
  }

  // Record every instance's iteration, group by image side, upload the tables.
  int build() {
    CK(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&ev0, cudaEventDisableTiming));
    std::vector<std::vector<Rec>> recs(ops.size());
    for (size_t i = 0; i < ops.size(); ++i) {
      OpImpl<T>* o = ops[i];
      o->rec = &recs[i];
      o->iteration(o->run.nu, o->run.gamma, o->run.P.eps, o->run.P.cg_iters, o->own);
      o->rec = nullptr;
    }
    std::map<int, int> gid;
    for (size_t i = 0; i < ops.size(); ++i) {
      auto it = gid.find(ops[i]->g.n);
      if (it == gid.end()) {
        gid[ops[i]->g.n] = int(groups.size());
        groups.emplace_back();
        it = gid.find(ops[i]->g.n);
      }
      groups[it->second].idx.push_back(int(i));
    }
    for (Group& gr : groups) {
      const std::vector<Rec>& r0 = recs[gr.idx[0]];
      for (const Rec& r : r0) {
        gr.kinds.push_back(r.kind);
        gr.branches.push_back(r.branch);
      }
      for (int i : gr.idx) {
        if (recs[i].size() != r0.size()) return invalid("instances of one image side differ in their passes");
        for (size_t k = 0; k < r0.size(); ++k)
          if (recs[i][k].kind != r0[k].kind) return invalid("instances of one image side differ in their passes");
        gr.max_items = std::max(gr.max_items, ops[i]->n_items);
        gr.max_tb = std::max(gr.max_tb, ops[i]->g.TB);
        gr.max_q = std::max(gr.max_q, ops[i]->grid_bytes());
      }
      // tables: one entry per instance for every pass with arguments
      const int cnt = int(gr.idx.size());
      size_t total = 0;
      for (int kind : gr.kinds) {
        gr.off.push_back(total);
        total += (entry_bytes(kind) * cnt + 255) & ~size_t(255);
      }
      std::vector<unsigned char> host(total > 0 ? total : 1);
      std::vector<SaraBatchInst<T>> sara_in;
      for (size_t k = 0; k < gr.kinds.size(); ++k)
        for (int j = 0; j < cnt; ++j) {
          const Rec& r = recs[gr.idx[j]][k];
          unsigned char* d = host.data() + gr.off[k] + entry_bytes(r.kind) * j;
          switch (r.kind) {
            case OpImpl<T>::R_RF: std::memcpy(d, &r.rf, sizeof(r.rf)); break;
            case OpImpl<T>::R_CC: std::memcpy(d, &r.cc, sizeof(r.cc)); break;
            case OpImpl<T>::R_RI: std::memcpy(d, &r.ri, sizeof(r.ri)); break;
            case OpImpl<T>::R_CF: std::memcpy(d, &r.cf, sizeof(r.cf)); break;
            case OpImpl<T>::R_CI: std::memcpy(d, &r.ci, sizeof(r.ci)); break;
            case OpImpl<T>::R_DG: std::memcpy(d, &r.dg, sizeof(r.dg)); break;
            case OpImpl<T>::R_GR: std::memcpy(d, &r.gr, sizeof(r.gr)); break;
            case OpImpl<T>::R_B1: std::memcpy(d, &r.b1, sizeof(r.b1)); break;
            case OpImpl<T>::R_ZERO: std::memcpy(d, &r.z, sizeof(r.z)); break;
            case OpImpl<T>::R_AXPY: std::memcpy(d, &r.ax, sizeof(r.ax)); break;
            case OpImpl<T>::R_FIN: std::memcpy(d, &r.fin, sizeof(r.fin)); break;
            case OpImpl<T>::R_SARA: sara_in.push_back(r.sara); break;
            default: break;
          }
        }
      if (pool) {
        CK(cudaMallocFromPoolAsync(&gr.dev, host.size(), pool, bs));
        CK(cudaMemcpyAsync(gr.dev, host.data(), host.size(), cudaMemcpyHostToDevice, bs));
        CK(cudaStreamSynchronize(bs));
      } else {
        CK(cudaMalloc(&gr.dev, host.size()));
        CK(cudaMemcpy(gr.dev, host.data(), host.size(), cudaMemcpyHostToDevice));
      }
      if (!sara_in.empty()) {
        int np = 0;
        const int rc = sara_batch_create<T>(sara_in, &gr.sara, &np, pool, bs);
        if (rc) return rc;
      }
      CK(cudaStreamCreateWithFlags(&gr.main, cudaStreamNonBlocking));
      int lo = 0, hi = 0;
      CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
      CK(cudaStreamCreateWithPriority(&gr.aux, cudaStreamNonBlocking, hi));  // the ball block's branch first
      CK(cudaEventCreateWithFlags(&gr.fork, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&gr.join, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&gr.done, cudaEventDisableTiming));
    }
    return capture();
  }

  static size_t entry_bytes(int kind) {
    switch (kind) {
      case OpImpl<T>::R_RF: return sizeof(RowFwdArgs<T>);
      case OpImpl<T>::R_CC: return sizeof(ColConvArgs<T>);
      case OpImpl<T>::R_RI: return sizeof(RowInvArgs<T>);
      case OpImpl<T>::R_CF: return sizeof(ColFwdArgs<T>);
      case OpImpl<T>::R_CI: return sizeof(ColInvArgs<T>);
      case OpImpl<T>::R_DG: return sizeof(DegridArgs<T>);
      case OpImpl<T>::R_GR: return sizeof(GridArgs<T>);
      case OpImpl<T>::R_B1: return sizeof(Ball1Args);
      case OpImpl<T>::R_ZERO: return sizeof(ZeroArgs);
      case OpImpl<T>::R_AXPY: return sizeof(AxpyArgs<T>);
      case OpImpl<T>::R_FIN: return sizeof(FinArgs);
      default: return 0;
    }
  }

  int invalid(const char* why) {
    note_error("purify_batch_solve", __LINE__, why);
    return PURIFY_ERR_INVALID;
  }

  // One SDMM iteration of every instance as one graph: per group, the
  // recorded passes as batched launches on the group's main stream, the ball
  // block between the fork and the join on its second stream.
  int capture() {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(bs, cudaStreamCaptureModeThreadLocal));
    cudaEventRecord(ev0, bs);
    for (Group& gr : groups) {
      cudaStreamWaitEvent(gr.main, ev0, 0);
      const int cnt = int(gr.idx.size());
      const Geometry& g = ops[gr.idx[0]]->g;
      const size_t N = size_t(g.n) * g.n;
      unsigned char* d = static_cast<unsigned char*>(gr.dev);
      for (size_t k = 0; k < gr.kinds.size(); ++k) {
        cudaStream_t s = gr.branches[k] ? gr.aux : gr.main;
        const void* tab = d + gr.off[k];
        switch (gr.kinds[k]) {
          case OpImpl<T>::R_RF: launch_row_fwd_h_batch<T>(g, static_cast<const RowFwdArgs<T>*>(tab), cnt, s); break;
          case OpImpl<T>::R_CC: launch_col_conv_h_batch<T>(g, static_cast<const ColConvArgs<T>*>(tab), cnt, s); break;
          case OpImpl<T>::R_RI: launch_row_inv_h_batch<T>(g, static_cast<const RowInvArgs<T>*>(tab), cnt, s); break;
          case OpImpl<T>::R_CF: launch_col_fwd_h_batch<T>(g, static_cast<const ColFwdArgs<T>*>(tab), cnt, s); break;
          case OpImpl<T>::R_CI: launch_col_inv_h_batch<T>(g, static_cast<const ColInvArgs<T>*>(tab), cnt, s); break;
          case OpImpl<T>::R_DG:
            launch_degrid_batch<T>(static_cast<const DegridArgs<T>*>(tab), cnt, gr.max_items, gr.max_tb,
                                   ops[gr.idx[0]]->kb, s);
            break;
          case OpImpl<T>::R_GR:
            launch_grid_batch<T>(static_cast<const GridArgs<T>*>(tab), cnt, gr.max_items, gr.max_tb,
                                 ops[gr.idx[0]]->kb, s);
            break;
          case OpImpl<T>::R_B1: launch_finalize_ball1_batch<T>(static_cast<const Ball1Args*>(tab), cnt, s); break;
          case OpImpl<T>::R_ZERO: launch_zero_batch(static_cast<const ZeroArgs*>(tab), cnt, gr.max_q, s); break;
          case OpImpl<T>::R_AXPY: launch_axpy_batch<T>(static_cast<const AxpyArgs<T>*>(tab), cnt, N, s); break;
          case OpImpl<T>::R_FIN: launch_finalize_batch<T>(static_cast<const FinArgs*>(tab), cnt, s); break;
          case OpImpl<T>::R_SARA: sara_batch_launch<T>(gr.sara, s); break;
          case OpImpl<T>::R_FORK:
            cudaEventRecord(gr.fork, gr.main);
            cudaStreamWaitEvent(gr.aux, gr.fork, 0);
            break;
          case OpImpl<T>::R_JOIN:
            cudaEventRecord(gr.join, gr.aux);
            cudaStreamWaitEvent(gr.main, gr.join, 0);
            break;
          default: break;
        }
      }
      cudaEventRecord(gr.done, gr.main);
      cudaStreamWaitEvent(bs, gr.done, 0);
    }
    cudaError_t ce = cudaStreamEndCapture(bs, &graph);
    if (ce != cudaSuccess) return map_err(ce, __LINE__);
    ce = cudaGraphInstantiate(&gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) return map_err(ce, __LINE__);
    return PURIFY_OK;
  }
};

template <typename T> int batch_graph_build(purify_op* const* ops, int count, cudaMemPool_t pool, void** out) {
  BatchImpl<T>* b = new (std::nothrow) BatchImpl<T>();
  if (!b) return PURIFY_ERR_NOMEM;
  b->pool = pool;
  for (int i = 0; i < count; ++i) {
    OpImpl<T>* o = dynamic_cast<OpImpl<T>*>(ops[i]);
    if (!o) {
      delete b;
      return PURIFY_ERR_INVALID;
    }
    b->ops.push_back(o);
  }
  const int rc = b->build();
  if (rc) {
    delete b;
    return rc;
  }
  *out = b;
  return PURIFY_OK;
}

// purify_batch_solve: begin every instance (nu, gamma, round 0 on its own
// stream), record and capture the batched iteration, then run the rounds in
// lock step -- the round set-ups per instance, the iterations as graph
// replays -- and end every instance.
template <typename T>
int batch_solve(int count, purify_op* const* ops_in, const void* const* y, const purify_params* params,
                void* const* x_out, purify_stats* stats, cudaStream_t user) {
  BatchImpl<T> b;
  for (int i = 0; i < count; ++i) {
    OpImpl<T>* o = dynamic_cast<OpImpl<T>*>(ops_in[i]);
    if (!o || !y[i] || !x_out[i]) return PURIFY_ERR_INVALID;
    const purify_params& P = params[i];
    const purify_params& P0 = params[0];
    if (P.xi != 0.0 || P.t_max != P0.t_max || P.cg_iters != P0.cg_iters || P.n_reweight != P0.n_reweight ||
        o->nblocks != 1 || o->prior != 0 || o->g.n < 64 || o->g.n > 1024 || P.gram == 0) {
      note_error("purify_batch_solve", __LINE__,
                 "instances need xi = 0, equal t_max, cg_iters and n_reweight, one visibility block, the l1 prior, "
                 "64 <= n <= 1024 and the convolution form of the CG operator");
      return PURIFY_ERR_INVALID;
    }
    for (int j = 0; j < i; ++j)
      if (ops_in[j] == ops_in[i]) return PURIFY_ERR_INVALID;
    b.ops.push_back(o);
  }
  // every instance's set-up (its CG operator, nu, gamma, state) on its own stream
  for (int i = 0; i < count; ++i) {
    purify_params P = params[i];
    P.use_graph = 0;
    P.gram = 1;
    const int rc = b.ops[i]->begin(y[i], &P, user);
    if (rc) {
      for (int j = 0; j <= i; ++j) b.ops[j]->run_release();
      return rc;
    }
  }
  int rc = b.build();
  cudaStream_t bs = b.bs;
  if (!rc) {
    for (OpImpl<T>* o : b.ops) {
      cudaEventRecord(o->ev_out, o->own);
      cudaStreamWaitEvent(bs, o->ev_out, 0);
    }
  }
  bool done = rc != 0;
  while (!done && !rc) {
    for (OpImpl<T>* o : b.ops)
      if (!rc && !o->run.round_ready) rc = o->start_round(bs);
    if (rc) break;
    cudaError_t e = cudaGraphLaunch(b.gexec, bs);
    if (e != cudaSuccess) rc = map_err(e, __LINE__);
    int all = 1;
    for (OpImpl<T>* o : b.ops) {
      int d = 0;
      if (!rc) rc = o->step_check(&d);
      all &= d;
    }
    done = all != 0;
  }
  if (!rc) {
    cudaError_t e = cudaStreamSynchronize(bs);
    if (e != cudaSuccess) rc = map_err(e, __LINE__);
  }
  int first = rc;
  for (int i = 0; i < count; ++i) {
    OpImpl<T>* o = b.ops[i];
    if (rc) {
      o->run_release();
      continue;
    }
    const int r = o->end(x_out[i], stats ? &stats[i] : nullptr, user);
    if (r && !first) first = r;
  }
  return first;
}

}  // namespace

// The request server's batched iteration over solves of one key.
struct BatchGraph {
  int prec = 0;
  void* impl = nullptr;
};

int batch_graph_create(purify_op* const* ops, int count, cudaMemPool_t pool, BatchGraph** out) {
  if (!ops || count < 1 || !out) return PURIFY_ERR_INVALID;
  int prec = 0;
  ops[0]->info(nullptr, nullptr, nullptr, nullptr, nullptr, &prec, nullptr);
  BatchGraph* g = new (std::nothrow) BatchGraph();
  if (!g) return PURIFY_ERR_NOMEM;
  g->prec = prec;
  const int rc = prec == PURIFY_FP32 ? batch_graph_build<float>(ops, count, pool, &g->impl)
                                     : batch_graph_build<double>(ops, count, pool, &g->impl);
  if (rc) {
    delete g;
    return rc;
  }
  *out = g;
  return PURIFY_OK;
}

int batch_graph_launch(BatchGraph* g, cudaStream_t s) {
  cudaGraphExec_t ge = g->prec == PURIFY_FP32 ? static_cast<BatchImpl<float>*>(g->impl)->gexec
                                              : static_cast<BatchImpl<double>*>(g->impl)->gexec;
  const cudaError_t e = cudaGraphLaunch(ge, s);
  return e == cudaSuccess ? PURIFY_OK : map_err(e, __LINE__);
}

void batch_graph_destroy(BatchGraph* g) {
  if (!g) return;
  if (g->prec == PURIFY_FP32) delete static_cast<BatchImpl<float>*>(g->impl);
  else delete static_cast<BatchImpl<double>*>(g->impl);
  delete g;
}

int create_pooled_op(const double* uv, int64_t M, int n, int levels, int precision, const purify_op_options* opt,
                     cudaMemPool_t pool, cudaStream_t s, purify_op** out) {
  const int tile = opt ? opt->tile : 0, chunk = opt ? opt->chunk : 0;
  if (!uv || !out || !pool || M < 1 || M >= (int64_t(1) << 31) || n < 16 || n > 2048 || (n & (n - 1)) ||
      levels < 1 || (n >> levels) < 2 || (tile != 0 && tile != 8 && tile != 16) || tile > 2 * n ||
      (chunk != 0 && (chunk < 64 || chunk > 8192)) || (precision != PURIFY_FP32 && precision != PURIFY_FP64))
    return PURIFY_ERR_INVALID;
  purify_op* op = nullptr;
  int rc;
  if (precision == PURIFY_FP32) {
    OpImpl<float>* o = new (std::nothrow) OpImpl<float>();
    if (!o) return PURIFY_ERR_NOMEM;
    rc = o->create(uv, M, n, levels, s, tile, chunk, false, nullptr, pool);
    op = o;
  } else {
    OpImpl<double>* o = new (std::nothrow) OpImpl<double>();
    if (!o) return PURIFY_ERR_NOMEM;
    rc = o->create(uv, M, n, levels, s, tile, chunk, false, nullptr, pool);
    op = o;
  }
  if (rc) {
    delete op;
    return rc;
  }
  *out = op;
  return PURIFY_OK;
}

}  // namespace purify

using purify::OpImpl;

extern "C" {

int purify_op_create(const double* uv, int64_t M, int n, int oversample, int J, int dwt_levels, int precision,
                     void* stream, purify_op** out) {
  if (!uv || !out || M < 1 || M >= (int64_t(1) << 31) || n < 16 || n > 2048 || (n & (n - 1)) ||
      oversample != 2 || J != purify::kJ || dwt_levels < 1 || (n >> dwt_levels) < 2 ||
      (precision != PURIFY_FP32 && precision != PURIFY_FP64))
    return PURIFY_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  purify_op* op = nullptr;
  int rc;
  if (precision == PURIFY_FP32) {
    OpImpl<float>* o = new (std::nothrow) OpImpl<float>();
    if (!o) return PURIFY_ERR_NOMEM;
    rc = o->create(uv, M, n, dwt_levels, s);
    op = o;
  } else {
    OpImpl<double>* o = new (std::nothrow) OpImpl<double>();
    if (!o) return PURIFY_ERR_NOMEM;
    rc = o->create(uv, M, n, dwt_levels, s);
    op = o;
  }
  if (rc) {
    delete op;
    return rc;
  }
  *out = op;
  return PURIFY_OK;
}

int purify_op_create_ex(const double* uv, int64_t M, int n, int oversample, int J, int dwt_levels, int precision,
                        const purify_op_options* opt, void* stream, purify_op** out) {
  const int tile = opt ? opt->tile : 0, chunk = opt ? opt->chunk : 0;
  if (tile != 0 && tile != 8 && tile != 16) return PURIFY_ERR_INVALID;
  if (tile > 2 * n || (chunk != 0 && (chunk < 64 || chunk > 8192))) return PURIFY_ERR_INVALID;
  if (!uv || !out || M < 1 || M >= (int64_t(1) << 31) || n < 16 || n > 2048 || (n & (n - 1)) ||
      oversample != 2 || J != purify::kJ || dwt_levels < 1 || (n >> dwt_levels) < 2 ||
      (precision != PURIFY_FP32 && precision != PURIFY_FP64))
    return PURIFY_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  purify_op* op = nullptr;
  int rc;
  if (precision == PURIFY_FP32) {
    OpImpl<float>* o = new (std::nothrow) OpImpl<float>();
    if (!o) return PURIFY_ERR_NOMEM;
    rc = o->create(uv, M, n, dwt_levels, s, tile, chunk);
    op = o;
  } else {
    OpImpl<double>* o = new (std::nothrow) OpImpl<double>();
    if (!o) return PURIFY_ERR_NOMEM;
    rc = o->create(uv, M, n, dwt_levels, s, tile, chunk);
    op = o;
  }
  if (rc) {
    delete op;
    return rc;
  }
  *out = op;
  return PURIFY_OK;
}

int purify_autotune(const double* uv, int64_t M, int n, int dwt_levels, int precision, int reps, void* stream,
                    purify_op_options* best, double* best_ms) {
  if (!best || reps < 1) return PURIFY_ERR_INVALID;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t rb = precision == PURIFY_FP32 ? 4 : 8;
  void* x = nullptr;
  void* y = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&x, size_t(n) * n * rb);
  if (e == cudaSuccess) e = cudaMalloc(&y, size_t(M) * 2 * rb);
  if (e == cudaSuccess) e = cudaMemset(x, 0, size_t(n) * n * rb);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int rc = e == cudaSuccess ? PURIFY_OK : PURIFY_ERR_CUDA;
  double best_t = 1e300;
  purify_op_options bo{16, 1024};
  struct Timed { purify_op_options o; double ms; };
  std::vector<Timed> times;
  const int tiles[2] = {8, 16};
  const int chunks[4] = {256, 512, 1024, 2048};
  for (int ti = 0; ti < 2 && !rc; ++ti) {
    if (tiles[ti] > 2 * n) continue;
    for (int ci = 0; ci < 4 && !rc; ++ci) {
      purify_op_options o{tiles[ti], chunks[ci]};
      purify_op* op = nullptr;
      int r = purify_op_create_ex(uv, M, n, 2, 8, dwt_levels, precision, &o, stream, &op);
      if (r) {
        if (r == PURIFY_ERR_NOMEM) continue;
        rc = r;
        break;
      }
      r = op->sorted_pair(x, y, x, s);
      cudaEventRecord(e0, s);
      for (int k = 0; k < reps && !r; ++k) r = op->sorted_pair(x, y, x, s);
      cudaEventRecord(e1, s);
      float ms = 0.f;
      if (!r && cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        times.push_back({o, double(ms) / reps});
      delete op;
      if (r) rc = r;
    }
  }
  cudaFree(x);
  cudaFree(y);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (rc) return rc;
  // fastest pair; among candidates within 2% of it (timing noise), the one
  // with the largest chunk (fewer work items, fewer flushes and atomics)
  const Timed* pick = nullptr;
  for (const Timed& c : times)
    if (!pick || c.ms < pick->ms) pick = &c;
  if (pick) {
    const double lim = 1.02 * pick->ms;
    for (const Timed& c : times)
      if (c.ms <= lim && (c.o.chunk > pick->o.chunk || (c.o.chunk == pick->o.chunk && c.ms < pick->ms))) pick = &c;
    bo = pick->o;
    best_t = pick->ms;
  }
  *best = bo;
  if (best_ms) *best_ms = best_t;
  return PURIFY_OK;
}

int purify_op_destroy(purify_op* op) {
  delete op;
  return PURIFY_OK;
}

int purify_op_info(const purify_op* op, int* n, int64_t* M, int* K, int* tile, int* n_items, int* precision,
                   int64_t* device_bytes) {
  if (!op) return PURIFY_ERR_INVALID;
  op->info(n, M, K, tile, n_items, precision, device_bytes);
  return PURIFY_OK;
}

int purify_phi(purify_op* op, const void* x, void* y, void* stream) {
  if (!op || !x || !y) return PURIFY_ERR_INVALID;
  return op->phi(x, y, static_cast<cudaStream_t>(stream));
}

int purify_phi_adj(purify_op* op, const void* y, void* x, void* stream) {
  if (!op || !x || !y) return PURIFY_ERR_INVALID;
  return op->phi_adj(y, x, static_cast<cudaStream_t>(stream));
}

int purify_sara_fwd(purify_op* op, const void* x, void* c, void* stream) {
  if (!op || !x || !c) return PURIFY_ERR_INVALID;
  return op->sara_fwd(x, c, static_cast<cudaStream_t>(stream));
}

int purify_sara_adj(purify_op* op, const void* c, void* x, void* stream) {
  if (!op || !x || !c) return PURIFY_ERR_INVALID;
  return op->sara_adj(c, x, static_cast<cudaStream_t>(stream));
}

int purify_op_set_blocks(purify_op* op, const int* block_ids, int R, void* stream) {
  if (!op) return PURIFY_ERR_INVALID;
  return op->set_blocks(block_ids, R, static_cast<cudaStream_t>(stream));
}

int purify_op_set_dictionary(purify_op* op, unsigned mask) {
  if (!op) return PURIFY_ERR_INVALID;
  return op->set_dictionary(mask);
}

int purify_op_dictionary(const purify_op* op, unsigned* mask, int* n_bases) {
  if (!op || !mask) return PURIFY_ERR_INVALID;
  *mask = op->dictionary(n_bases);
  return PURIFY_OK;
}

int purify_op_set_prior(purify_op* op, int prior, int tv_iters) {
  if (!op) return PURIFY_ERR_INVALID;
  return op->set_prior(prior, tv_iters);
}

int purify_gram(purify_op* op, const void* x, void* out, int mode, void* stream) {
  if (!op || !x || !out) return PURIFY_ERR_INVALID;
  return op->gram(x, out, mode, static_cast<cudaStream_t>(stream));
}

int purify_profile(purify_op* op, int enable) {
  if (!op) return PURIFY_ERR_INVALID;
  op->prof_reset();
  op->prof = enable != 0;
  return PURIFY_OK;
}

int purify_profile_read(purify_op* op, int kind, double* total_ms, int64_t* launches) {
  if (!op || kind < 0 || kind >= PURIFY_NUM_KERNEL_KINDS) return PURIFY_ERR_INVALID;
  op->prof_collect();
  if (total_ms) *total_ms = op->prof_ms[kind];
  if (launches) *launches = op->prof_n[kind];
  return PURIFY_OK;
}

const char* purify_kernel_name(int kind) {
  static const char* names[] = {"row_fwd", "col_fwd", "degrid", "grid", "gram", "col_inv",
                                "row_inv", "sara_analysis", "sara_synthesis", "vector", "memset", "col_conv",
                                "row_fwd_h", "row_inv_h", "tv"};
  if (kind < 0 || kind >= PURIFY_NUM_KERNEL_KINDS) return "unknown";
  return names[kind];
}

void purify_default_params(purify_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->eps = 0.0;
  p->gamma = 0.0;
  p->nu = 0.0;
  p->t_max = 200;
  p->cg_iters = 10;
  p->xi = 0.0;
  p->n_reweight = 0;
  p->delta0 = 0.0;
  p->delta_min = 0.0;
  p->delta_decay = 0.1;
  p->warm_start = 1;
  p->power_iters = 30;
  p->use_graph = 1;
  p->gram = -1;
}

int purify_sdmm_solve(purify_op* op, const void* y, const purify_params* params, void* x_out, purify_stats* stats,
                      void* stream) {
  if (!op || !y || !params || !x_out) return PURIFY_ERR_INVALID;
  return op->solve(y, params, x_out, stats, static_cast<cudaStream_t>(stream));
}

int purify_batch_solve(int count, purify_op* const* ops, const void* const* y, const purify_params* params,
                       void* const* x_out, purify_stats* stats, void* stream) {
  if (count < 1 || !ops || !y || !params || !x_out) return PURIFY_ERR_INVALID;
  int prec = -1;
  for (int i = 0; i < count; ++i) {
    if (!ops[i]) return PURIFY_ERR_INVALID;
    int p = 0;
    ops[i]->info(nullptr, nullptr, nullptr, nullptr, nullptr, &p, nullptr);
    if (prec >= 0 && p != prec) return PURIFY_ERR_INVALID;
    prec = p;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (prec == PURIFY_FP32) return purify::batch_solve<float>(count, ops, y, params, x_out, stats, s);
  return purify::batch_solve<double>(count, ops, y, params, x_out, stats, s);
}

int purify_solve_begin(purify_op* op, const void* y, const purify_params* params, void* stream) {
  if (!op || !y || !params) return PURIFY_ERR_INVALID;
  return op->begin(y, params, static_cast<cudaStream_t>(stream));
}

int purify_solve_step(purify_op* op, int max_iters, int* done) {
  if (!op || !done) return PURIFY_ERR_INVALID;
  return op->run_steps(max_iters, done);
}

int purify_solve_end(purify_op* op, void* x_out, purify_stats* stats, void* stream) {
  if (!op || !x_out) return PURIFY_ERR_INVALID;
  return op->end(x_out, stats, static_cast<cudaStream_t>(stream));
}

int purify_solve_state_bytes(const purify_op* op, int64_t* bytes) {
  if (!op || !bytes) return PURIFY_ERR_INVALID;
  *bytes = op->state_bytes();
  return PURIFY_OK;
}

int purify_solve_save(purify_op* op, void* host, int64_t bytes) {
  if (!op) return PURIFY_ERR_INVALID;
  return op->save_state(host, bytes);
}

int purify_solve_load(purify_op* op, const void* host, int64_t bytes) {
  if (!op) return PURIFY_ERR_INVALID;
  return op->load_state(host, bytes);
}

int purify_set_wait_limit(uint32_t spins) {
  const uint32_t s = spins ? spins : purify::kSpinLimit;
  cudaError_t e = purify::set_wait_spins_fft(s);
  if (e == cudaSuccess) e = purify::set_wait_spins_nufft(s);
  if (e == cudaSuccess) e = purify::set_wait_spins_solver(s);
  return purify::map_err(e, __LINE__);
}

int purify_wait_selftest(int deliver, void* stream) {
  int timed_out = 0;
  const cudaError_t e = purify::wait_selftest(deliver, static_cast<cudaStream_t>(stream), &timed_out);
  if (e != cudaSuccess) return purify::map_err(e, __LINE__);
  if (timed_out) {
    purify::set_last_error("purify_wait_selftest: the bounded wait gave up (nothing was delivered)");
    return PURIFY_ERR_TIMEOUT;
  }
  return PURIFY_OK;
}

const char* purify_last_error(void) { return purify::g_last_error; }

const char* purify_strerror(int status) {
  switch (status) {
    case PURIFY_OK: return "ok";
    case PURIFY_ERR_INVALID: return "invalid argument";
    case PURIFY_ERR_NOMEM: return "device allocation failed";
    case PURIFY_ERR_CUDA: return "CUDA runtime error";
    case PURIFY_ERR_TIMEOUT: return "bounded device wait timed out";
    case PURIFY_ERR_NOT_CONVERGED: return "halting rule not met within t_max";
    case PURIFY_ERR_BUDGET: return "device memory budget exceeded";
    case PURIFY_ERR_CANCELLED: return "request cancelled";
    case PURIFY_ERR_NONFINITE: return "solve produced non-finite values";
    default: return "unknown status";
  }
}

}  // extern "C"
