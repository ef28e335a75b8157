// Shared device helpers for the GB300 SARA-SDMM kernels: complex arithmetic,
// FP64 block reductions, bounded mbarrier waits and TMA copies (sm_103a).
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#define PD __device__ __forceinline__

namespace purify {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { typedef float2 type; };
template <> struct cplx_t<double> { typedef double2 type; };

template <typename C> PD C cz() { C r; r.x = 0; r.y = 0; return r; }
template <typename C, typename T> PD C cmk(T a, T b) { C r; r.x = a; r.y = b; return r; }
template <typename C> PD C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> PD C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> PD C cmul(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename C, typename T> PD C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
template <typename C> PD C cmul_i(C a) { C r; r.x = -a.y; r.y = a.x; return r; }  // i * a

// Device error flag values (first writer wins).
enum : int { DEV_OK = 0, DEV_TIMEOUT = 1 };

// Bounded spin budget for mbarrier waits: far beyond any TMA latency, short
// enough that a lost transaction surfaces as an error instead of a hang.
constexpr uint32_t kSpinLimit = 1u << 24;
// The first-phase budget (before a wait is reported as timed out) is a
// device variable of each compiled module, kSpinLimit unless the host lowers
// it (purify_set_wait_limit); the drain phase that follows a timeout, which
// lets copies still in flight land before the CTA exits, always keeps the
// full kSpinLimit.
static __device__ uint32_t g_wait_spins = kSpinLimit;
// Host side: set this module's first-phase budget on the current device.
static inline cudaError_t set_module_wait_spins(uint32_t spins) {
  return cudaMemcpyToSymbol(g_wait_spins, &spins, sizeof(spins));
}

PD void set_error(int* err, int code) {
  if (err) atomicCAS(err, DEV_OK, code);
}

// Raise a kernel's dynamic shared-memory limit to what the device allows
// next to the kernel's static shared memory (host).
template <typename K> inline cudaError_t raise_smem_limit(K kernel) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes a;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - int(a.sharedSizeBytes));
  return e;
}

// ---------------------------------------------------------------- reductions
// Per-thread partial sums (inner products, norms, objective terms).  On the
// FP32 path a Kahan-compensated FP32 sum, each product split exactly into its
// rounded value and an FMA-recovered error that joins the compensation; the
// pair goes to FP64 once per thread, and everything across threads is summed
// in FP64.  GB300 runs FP64 arithmetic at a small fraction of its FP32 rate,
// so converting every element to double would dominate these kernels.
template <typename T> struct Acc;
template <> struct Acc<float> {
  float s = 0.f, c = 0.f;  // the sum is s - c
  PD void add(float a) {
    const float y = a - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  PD void add_prod(float a, float b) {
    const float p = a * b;
    add(p);
    c -= fmaf(a, b, -p);
  }
  PD double value() const { return double(s) - double(c); }
};
template <> struct Acc<double> {
  double s = 0.0;
  PD void add(double a) { s += a; }
  PD void add_prod(double a, double b) { s = fma(a, b, s); }
  PD double value() const { return s; }
};

PD double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
PD double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// Merging of compensated partials.  Per-block partial sums are stored as
// Acc<T> (8 bytes, in double-sized slots) and merged in the same compensated
// FP32 form, so the only FP64 arithmetic of a reduction is the final value:
// the FP64 units of GB300 are few, and chains of dependent FP64 adds in every
// block's tail would cost microseconds.
PD void acc_merge(Acc<float>& a, const Acc<float>& b) {
  a.c += b.c;
  a.add(b.s);
}
PD void acc_merge(Acc<double>& a, const Acc<double>& b) { a.s += b.s; }
PD void warp_merge(Acc<float>& a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Acc<float> b;
    b.s = __shfl_down_sync(0xffffffffu, a.s, o);
    b.c = __shfl_down_sync(0xffffffffu, a.c, o);
    acc_merge(a, b);
  }
}
PD void warp_merge(Acc<double>& a) { a.s = warp_sum(a.s); }
// Block merge; result valid in thread 0.  sh: NT/32 double-sized slots.
template <int NT, typename T> __device__ Acc<T> block_merge(Acc<T> a, double* sh) {
  Acc<T>* st = reinterpret_cast<Acc<T>*>(sh);
  warp_merge(a);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) st[w] = a;
  __syncthreads();
  if (w == 0) {
    a = lane < NT / 32 ? st[lane] : Acc<T>();
    warp_merge(a);
  }
  __syncthreads();
  return a;
}
// Merge of n stored partials by one block of NT threads; result in thread 0.
// Each thread merges p[tid], p[tid + NT], ... in that order; the loads are
// issued eight at a time so that their latencies overlap.
template <int NT, typename T> __device__ Acc<T> merge_array(const Acc<T>* p, int n, double* sh) {
  constexpr int U = 8;
  Acc<T> a;
  int i = threadIdx.x;
  for (; i + (U - 1) * NT < n; i += U * NT) {
    Acc<T> v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) v[u] = p[i + u * NT];
#pragma unroll
    for (int u = 0; u < U; ++u) acc_merge(a, v[u]);
  }
  for (; i < n; i += NT) acc_merge(a, p[i]);
  return block_merge<NT>(a, sh);
}
template <int NT> __device__ double block_max(double v, double* sh) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (w == 0) {
    r = (lane < NT / 32) ? sh[lane] : 0.0;
    r = warp_max(r);
  }
  __syncthreads();
  return r;
}

// Last-block reduction: every block has written partials[blockIdx.x]; the
// block that finishes last (atomic ticket, no waiting) returns true in all
// its threads, after which it may read all partials.  It resets the ticket.
__device__ __forceinline__ bool last_block_done(unsigned int* ticket,
                                                unsigned int count = gridDim.x * gridDim.y * gridDim.z) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == count - 1);
    if (last) *ticket = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// As last_block_done, for blocks whose global results for the last block
// were all written by thread 0 (only thread 0 fences before the ticket);
// `count` blocks take part (one instance's blocks of a batched launch).
__device__ __forceinline__ bool last_block_done_t0(unsigned int* ticket, unsigned int count) {
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned int t = atomicAdd(ticket, 1u);
    last = (t == count - 1);
    if (last) *ticket = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Kernel arguments: by value for one operator (ArgVal, kernel parameter
// space), or from a device table for a batch of independent instances of the
// same size (ArgTab: instance blockIdx.y, every instance the same grid).
template <typename A> struct ArgVal {
  static constexpr bool kTable = false;
  A a;
  PD const A& get() const { return a; }
  PD const A& get_at(int) const { return a; }
  PD int inst() const { return 0; }
};
template <typename A> struct ArgTab {
  static constexpr bool kTable = true;
  const A* t;
  PD A get() const { return t[blockIdx.y]; }
  PD A get_at(int i) const { return t[i]; }
  PD int inst() const { return int(blockIdx.y); }
};


// ---------------------------------------------------------------- mbarrier + TMA
PD uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

PD void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
PD void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
PD void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
PD bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
// Wait for `phase` of `bar` with a bounded spin; on timeout flag the error,
// keep waiting (bounded again, unless drain is false because nothing is in
// flight) so the copy in flight lands before the CTA can exit, and return
// false.
PD bool mbar_wait_bounded(uint64_t* bar, uint32_t phase, int* err, bool drain = true) {
  const uint32_t lim = g_wait_spins;
  for (uint32_t i = 0; i < lim; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  set_error(err, DEV_TIMEOUT);
  if (drain)
    for (uint32_t i = 0; i < kSpinLimit; ++i)
      if (mbar_try_wait(bar, phase)) break;
  return false;
}
// Untiled bulk copy global -> shared: both addresses 16-byte aligned, bytes a
// multiple of 16; completion counted on `bar`.
PD void bulk_load(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(smem_dst)),
               "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Before the first TMA use of a tensor map that lives in global memory
// (written there by a host copy): order the generic-proxy write before the
// tensor-map proxy's read.
PD void tensormap_acquire(const CUtensorMap* map) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(map) : "memory");
}
PD void tma_load_2d(void* smem_dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(smem_dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

}  // namespace purify
