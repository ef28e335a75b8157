// Small vector kernels of the SDMM solver (Algorithm 1) and the SARA
// reweighting: the last CG update, deterministic finalisation of device
// scalars from compensated per-block partials (the l2-ball scales, the
// objective, norms), visibility permutation and the reweighting rule.
#include "solver_kernels.h"

namespace purify {

namespace {
constexpr int kT = 256;
constexpr int kFinT = 1024;  // the single-block merge of the per-item partials

// 16-byte vectors of the CG update.
template <typename T> struct Vec16;
template <> struct Vec16<float> { typedef float4 type; static constexpr int W = 4; };
template <> struct Vec16<double> { typedef double2 type; static constexpr int W = 2; };

// x += sc[idx] p on 16-byte vectors (N / W of them, both arrays 16-byte aligned).
template <typename T, typename Src>
__global__ void __launch_bounds__(kT) k_axpy(Src src) {
  typedef typename Vec16<T>::type V;
  decltype(auto) args = src.get();
  T* __restrict__ x = args.x;
  const T* __restrict__ p = args.p;
  const double* __restrict__ sc = args.sc;
  const int idx = args.idx;
  const size_t N = args.N;
  constexpr int W = Vec16<T>::W;
  const T a = T(sc[idx]);
  V* xv = reinterpret_cast<V*>(x);
  const V* pv = reinterpret_cast<const V*>(p);
  for (size_t i = size_t(blockIdx.x) * kT + threadIdx.x; i < N / W; i += size_t(gridDim.x) * kT) {
    V xs = xv[i];
    const V ps = pv[i];
    T* xe = reinterpret_cast<T*>(&xs);
    const T* pe = reinterpret_cast<const T*>(&ps);
#pragma unroll
    for (int k = 0; k < W; ++k) xe[k] = fma(a, pe[k], xe[k]);
    xv[i] = xs;
  }
}

// One block: merge the compensated partials (Acc<T>) in a fixed order, then
// apply `op` (FinOp) in FP64.
template <typename T, typename Src>
__global__ void __launch_bounds__(kT) k_finalize(Src src) {
  __shared__ double red[32];
  decltype(auto) args = src.get();
  const double* __restrict__ pa = args.pa;
  const int na = args.na, op = args.op;
  const double arg = args.arg;
  double* __restrict__ sc = args.sc;
  const double a = merge_array<kT>(reinterpret_cast<const Acc<T>*>(pa), na, red).value();
  if (threadIdx.x != 0) return;
  switch (op) {
    case FIN_OBJ:
      sc[S_OBJ] = a;
      break;
    case FIN_NORM: {
      const double l = sqrt(a);
      sc[S_LAMBDA] = l;
      sc[S_INVNORM] = l > 0.0 ? 1.0 / l : 0.0;
    } break;
    case FIN_MEAN:  // arg = element count
      sc[S_MEAN] = a / arg;
      break;
    case FIN_VAR:
      sc[S_STD] = sqrt(a / arg);
      break;
    default:
      break;
  }
}

// Per-block l2-ball scalars (Eq. 5): for every visibility block b, ||v - nu y||
// and ||Phi x - y|| over the work items of that block (fixed order, from the
// items' compensated partials), the projection scale
// min(1, nu eps_b / ||v - nu y||_b), the total residual and the worst
// feasibility ratio max_b ||y_b - Phi_b x|| / eps_b.
template <typename T>
__global__ void __launch_bounds__(kFinT) k_finalize_blocks(const double* __restrict__ part0,
                                                           const double* __restrict__ part1,
                                                           const int* __restrict__ item_block, int n_items, int R,
                                                           double nu, const double* __restrict__ eps_b,
                                                           double* __restrict__ scale_b, double* __restrict__ sc) {
  __shared__ double red[2 * 32];  // one Acc<T> per warp
  const Acc<T>* p0 = reinterpret_cast<const Acc<T>*>(part0);
  const Acc<T>* p1 = reinterpret_cast<const Acc<T>*>(part1);
  double tot1 = 0.0, worst = 0.0;
  constexpr int U = 8;  // loads in flight per thread and array
  for (int b = 0; b < R; ++b) {
    Acc<T> a, c;
    int i = threadIdx.x;
    for (; i + (U - 1) * kFinT < n_items; i += U * kFinT) {
      Acc<T> x[U], y[U];
      bool in[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = i + u * kFinT;
        in[u] = R == 1 || item_block[4 * j] == b;  // WorkItem::pad
        x[u] = p0[j];
        y[u] = p1[j];
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (in[u]) {
          acc_merge(a, x[u]);
          acc_merge(c, y[u]);
        }
    }
    for (; i < n_items; i += kFinT) {
      if (R == 1 || item_block[4 * i] == b) {
        acc_merge(a, p0[i]);
        acc_merge(c, p1[i]);
      }
    }
    const double av = block_merge<kFinT>(a, red).value();
    const double cv = block_merge<kFinT>(c, red).value();
    if (threadIdx.x == 0) {
      const double s = sqrt(av), rad = nu * eps_b[b];
      scale_b[b] = s <= rad ? 1.0 : rad / s;
      tot1 += cv;
      const double ratio = sqrt(cv) / eps_b[b];
      worst = ratio > worst ? ratio : worst;
    }
  }
  if (threadIdx.x == 0) {
    sc[S_RESID] = sqrt(tot1);
    sc[S_FEAS] = worst;
    sc[S_BALLSCALE] = scale_b[0];
  }
}

// The same scalars for one visibility block (R = 1) in two levels: kFinCtas
// CTAs each merge a contiguous slice of the items' partials (fixed order),
// the last CTA to finish (ticket) merges the CTAs' partials in index order.
template <typename T, typename Src>
__global__ void __launch_bounds__(kT) k_finalize_ball1(Src src) {
  __shared__ double red[32];
  decltype(auto) args = src.get();
  const double* __restrict__ part0 = args.part0;
  const double* __restrict__ part1 = args.part1;
  const int n_items = args.n_items;
  const double nu = args.nu;
  const double* __restrict__ eps_b = args.eps_b;
  double* __restrict__ scale_b = args.scale_b;
  double* __restrict__ sc = args.sc;
  double* __restrict__ cpart = args.cpart;
  unsigned int* __restrict__ ticket = args.ticket;
  const Acc<T>* p0 = reinterpret_cast<const Acc<T>*>(part0);
  const Acc<T>* p1 = reinterpret_cast<const Acc<T>*>(part1);
  Acc<T>* c0 = reinterpret_cast<Acc<T>*>(cpart);
  Acc<T>* c1 = c0 + gridDim.x;
  const int per = (n_items + int(gridDim.x) - 1) / int(gridDim.x);
  const int lo = int(blockIdx.x) * per, hi = min(n_items, lo + per);
  constexpr int U = 4;
  Acc<T> a, c;
  int i = lo + int(threadIdx.x);
  for (; i + (U - 1) * kT < hi; i += U * kT) {
    Acc<T> x[U], y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      x[u] = p0[i + u * kT];
      y[u] = p1[i + u * kT];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      acc_merge(a, x[u]);
      acc_merge(c, y[u]);
    }
  }
  for (; i < hi; i += kT) {
    acc_merge(a, p0[i]);
    acc_merge(c, p1[i]);
  }
  a = block_merge<kT>(a, red);
  c = block_merge<kT>(c, red);
  if (threadIdx.x == 0) {
    c0[blockIdx.x] = a;
    c1[blockIdx.x] = c;
  }
  if (!last_block_done(ticket, gridDim.x)) return;
  const double av = merge_array<kT>(c0, int(gridDim.x), red).value();
  const double cv = merge_array<kT>(c1, int(gridDim.x), red).value();
  if (threadIdx.x == 0) {
    const double s = sqrt(av), rad = nu * eps_b[0];
    scale_b[0] = s <= rad ? 1.0 : rad / s;
    sc[S_RESID] = sqrt(cv);
    sc[S_FEAS] = sqrt(cv) / eps_b[0];
    sc[S_BALLSCALE] = scale_b[0];
  }
}

// Per-block partials of a reduction over v: compensated sums (RED_SUM, RED_VAR
// about sc[S_MEAN], RED_SQ) stored as Acc<T>; RED_MAXABS stores the block
// maximum as a double.
template <typename T>
__global__ void __launch_bounds__(kT) k_sum_partials(const T* __restrict__ v, size_t N, int op,
                                                     const double* __restrict__ sc, double* __restrict__ partials) {
  __shared__ double red[32];
  if (op == RED_MAXABS) {
    double m = 0.0;
    for (size_t i = size_t(blockIdx.x) * kT + threadIdx.x; i < N; i += size_t(gridDim.x) * kT)
      m = fmax(m, fabs(double(v[i])));
    m = block_max<kT>(m, red);
    if (threadIdx.x == 0) partials[blockIdx.x] = m;
    return;
  }
  Acc<T> part;
  const T mean = op == RED_VAR ? T(sc[S_MEAN]) : T(0);
  for (size_t i = size_t(blockIdx.x) * kT + threadIdx.x; i < N; i += size_t(gridDim.x) * kT) {
    const T x = v[i];
    if (op == RED_SUM) {
      part.add(x);
    } else if (op == RED_VAR) {
      const T d = x - mean;
      part.add_prod(d, d);
    } else {
      part.add_prod(x, x);
    }
  }
  const Acc<T> t = block_merge<kT>(part, red);
  if (threadIdx.x == 0) reinterpret_cast<Acc<T>*>(partials)[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kT) k_max_partials(const double* __restrict__ p, int np, double* __restrict__ sc) {
  __shared__ double red[32];
  double m = 0.0;
  for (int i = threadIdx.x; i < np; i += kT) m = fmax(m, p[i]);
  m = block_max<kT>(m, red);
  if (threadIdx.x == 0) sc[S_MAXABS] = m;
}

template <typename T>
__global__ void k_reweight(T* __restrict__ w, size_t N, double delta) {
  for (size_t i = size_t(blockIdx.x) * kT + threadIdx.x; i < N; i += size_t(gridDim.x) * kT)
    w[i] = T(delta / (delta + fabs(double(w[i]))));
}

template <typename T>
__global__ void k_fill(T* __restrict__ v, size_t N, T val) {
  for (size_t i = size_t(blockIdx.x) * kT + threadIdx.x; i < N; i += size_t(gridDim.x) * kT) v[i] = val;
}

template <typename T>
__global__ void k_scale(T* __restrict__ v, size_t N, const double* __restrict__ sc, int idx, double mul) {
  const T s = T(sc[idx] * mul);
  for (size_t i = size_t(blockIdx.x) * kT + threadIdx.x; i < N; i += size_t(gridDim.x) * kT) v[i] *= s;
}

// Zero `bytes` (a multiple of 16) of one instance's buffer.
__global__ void __launch_bounds__(kT) k_zero(ArgTab<ZeroArgs> src) {
  const ZeroArgs a = src.get();
  uint4* p = static_cast<uint4*>(a.p);
  const size_t n = a.bytes / 16;
  for (size_t i = size_t(blockIdx.x) * kT + threadIdx.x; i < n; i += size_t(gridDim.x) * kT) p[i] = make_uint4(0, 0, 0, 0);
}

template <typename T>
__global__ void k_check_finite(const T* __restrict__ v, size_t N, int* __restrict__ flag) {
  bool bad = false;
  for (size_t i = size_t(blockIdx.x) * kT + threadIdx.x; i < N; i += size_t(gridDim.x) * kT)
    bad |= !isfinite(v[i]);
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicExch(flag, 1);
}

// Self-test of the bounded mbarrier wait: thread 0 arms the barrier for 16
// bytes; with deliver set a bulk copy brings them, otherwise nothing is ever
// sent and the wait runs out of its budget (no copy is in flight, so there
// is nothing to drain).  The outcome goes to the module's flag.
static __device__ int g_selftest_flag;
static __device__ __align__(16) unsigned char g_selftest_src[16];
__global__ void k_wait_selftest(int deliver) {
  __shared__ __align__(16) unsigned char dst[16];
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    g_selftest_flag = DEV_OK;
    mbar_init(&bar, 1);
    fence_barrier_init();
    mbar_arrive_expect_tx(&bar, 16u);
    if (deliver) bulk_load(dst, g_selftest_src, 16u, &bar);
  }
  __syncthreads();
  mbar_wait_bounded(&bar, 0, &g_selftest_flag, deliver != 0);
}

template <typename C>
__global__ void k_gather(const C* __restrict__ src, const int* __restrict__ perm, size_t M, C* __restrict__ dst) {
  for (size_t i = size_t(blockIdx.x) * kT + threadIdx.x; i < M; i += size_t(gridDim.x) * kT) dst[i] = src[perm[i]];
}

inline int nblk(size_t N) {
  size_t b = (N + kT - 1) / kT;
  if (b > 4096) b = 4096;
  return int(b > 0 ? b : 1);
}
}  // namespace

int vec_blocks(size_t N) { return nblk(N); }

template <typename T> void launch_axpy(T* x, const T* p, const double* sc, int idx, size_t N, cudaStream_t s) {
  // one 16-byte vector per thread; N and the pointers are multiples of 16
  // bytes (n x n images, n >= 16; cudaMalloc'd arrays)
  k_axpy<T><<<nblk((N + 3) / 4), kT, 0, s>>>(ArgVal<AxpyArgs<T>>{AxpyArgs<T>{x, p, sc, idx, N}});
}
template <typename T> void launch_axpy_batch(const AxpyArgs<T>* tab, int count, size_t N, cudaStream_t s) {
  k_axpy<T><<<dim3(nblk((N + 3) / 4), count), kT, 0, s>>>(ArgTab<AxpyArgs<T>>{tab});
}
template <typename T> void launch_finalize_batch(const FinArgs* tab, int count, cudaStream_t s) {
  k_finalize<T><<<dim3(1, count), kT, 0, s>>>(ArgTab<FinArgs>{tab});
}
template <typename T> void launch_finalize_ball1_batch(const Ball1Args* tab, int count, cudaStream_t s) {
  k_finalize_ball1<T><<<dim3(kFinCtas, count), kT, 0, s>>>(ArgTab<Ball1Args>{tab});
}
void launch_zero_batch(const ZeroArgs* tab, int count, size_t max_bytes, cudaStream_t s) {
  size_t b = (max_bytes / 16 + kT - 1) / kT;
  if (b > 2048) b = 2048;
  k_zero<<<dim3(unsigned(b > 0 ? b : 1), count), kT, 0, s>>>(ArgTab<ZeroArgs>{tab});
}

template <typename T> void launch_finalize(const double* pa, int na, int op, double arg, double* sc, cudaStream_t s) {
  k_finalize<T><<<1, kT, 0, s>>>(ArgVal<FinArgs>{FinArgs{pa, na, op, arg, sc}});
}

template <typename T>
int launch_reduce(const T* v, size_t N, int op, const double* sc, double* partials, cudaStream_t s) {
  const int b = nblk(N);
  k_sum_partials<T><<<b, kT, 0, s>>>(v, N, op, sc, partials);
  return b;
}

template <typename T>
void launch_finalize_blocks(const double* part0, const double* part1, const int* items_as_int, int n_items, int R,
                            double nu, const double* eps_b, double* scale_b, double* sc, double* cpart,
                            unsigned int* ticket, cudaStream_t s) {
  if (R == 1 && cpart && ticket) {
    int nb = (n_items + 4 * kT - 1) / (4 * kT);
    nb = nb < 1 ? 1 : (nb > kFinCtas ? kFinCtas : nb);
    k_finalize_ball1<T><<<nb, kT, 0, s>>>(
        ArgVal<Ball1Args>{Ball1Args{part0, part1, n_items, nu, eps_b, scale_b, sc, cpart, ticket}});
  } else {
    k_finalize_blocks<T><<<1, kFinT, 0, s>>>(part0, part1, items_as_int + 3, n_items, R, nu, eps_b, scale_b, sc);
  }
}

void launch_max_partials(const double* p, int np, double* sc, cudaStream_t s) {
  k_max_partials<<<1, kT, 0, s>>>(p, np, sc);
}

template <typename T> void launch_reweight(T* w, size_t N, double delta, cudaStream_t s) {
  k_reweight<T><<<nblk(N), kT, 0, s>>>(w, N, delta);
}
template <typename T> void launch_fill(T* v, size_t N, T val, cudaStream_t s) {
  k_fill<T><<<nblk(N), kT, 0, s>>>(v, N, val);
}
template <typename T> void launch_scale(T* v, size_t N, const double* sc, int idx, double mul, cudaStream_t s) {
  k_scale<T><<<nblk(N), kT, 0, s>>>(v, N, sc, idx, mul);
}
template <typename C> void launch_gather(const C* src, const int* perm, size_t M, C* dst, cudaStream_t s) {
  k_gather<C><<<nblk(M), kT, 0, s>>>(src, perm, M, dst);
}
template <typename T> void launch_check_finite(const T* v, size_t n, int* flag, cudaStream_t s) {
  k_check_finite<T><<<nblk(n), kT, 0, s>>>(v, n, flag);
}
template void launch_check_finite<float>(const float*, size_t, int*, cudaStream_t);
template void launch_check_finite<double>(const double*, size_t, int*, cudaStream_t);

cudaError_t set_wait_spins_solver(uint32_t spins) { return set_module_wait_spins(spins); }

cudaError_t wait_selftest(int deliver, cudaStream_t s, int* timed_out) {
  k_wait_selftest<<<1, 32, 0, s>>>(deliver);
  cudaError_t e = cudaGetLastError();
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyFromSymbolAsync(&h, g_selftest_flag, sizeof(int), 0, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) *timed_out = h != DEV_OK;
  return e;
}

#define INST(T)                                                                                       \
  template void launch_axpy<T>(T*, const T*, const double*, int, size_t, cudaStream_t);                \
  template void launch_axpy_batch<T>(const AxpyArgs<T>*, int, size_t, cudaStream_t);                   \
  template void launch_finalize_batch<T>(const FinArgs*, int, cudaStream_t);                            \
  template void launch_finalize_ball1_batch<T>(const Ball1Args*, int, cudaStream_t);                    \
  template void launch_finalize<T>(const double*, int, int, double, double*, cudaStream_t);             \
  template void launch_finalize_blocks<T>(const double*, const double*, const int*, int, int, double,           \
                                          const double*, double*, double*, double*, unsigned int*,             \
                                          cudaStream_t);                                                       \
  template int launch_reduce<T>(const T*, size_t, int, const double*, double*, cudaStream_t);           \
  template void launch_reweight<T>(T*, size_t, double, cudaStream_t);                                   \
  template void launch_fill<T>(T*, size_t, T, cudaStream_t);                                            \
  template void launch_scale<T>(T*, size_t, const double*, int, double, cudaStream_t);
INST(float)
INST(double)
#undef INST
template void launch_fill<float2>(float2*, size_t, float2, cudaStream_t);
template void launch_fill<double2>(double2*, size_t, double2, cudaStream_t);
template void launch_gather<float2>(const float2*, const int*, size_t, float2*, cudaStream_t);
template void launch_gather<double2>(const double2*, const int*, size_t, double2*, cudaStream_t);

}  // namespace purify
