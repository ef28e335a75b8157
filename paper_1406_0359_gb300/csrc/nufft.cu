// Kaiser-Bessel interpolation G of Phi = G F Z S (Section 4) and its adjoint
// G^H, over uv-sorted visibility tiles.
//
// Visibilities are binned once per operator into TB x TB tiles of the K x K
// oversampled grid (stable LSD radix sort on the tile id) and cut into work
// items of at most `chunk` visibilities.  One CTA runs one work item:
//   degrid: the tile's (TB+J)^2 grid patch is staged in shared memory by one
//           TMA tile load (the grid carries a periodic J-wide halo, so the
//           patch is contiguous); every thread then gathers its visibilities'
//           J x J taps from shared memory.
//   grid:   every thread scatters its visibilities' J x J taps into a
//           shared-memory patch accumulator with shared atomics; the patch is
//           flushed to the padded global grid with one vector atomic per
//           non-zero cell.
//   gram:   both at once for the CG operator Phi^H Phi: y_m is formed from the
//           staged patch and scattered straight back with the same weights.
// Kernel weights come from a per-tap polynomial in the fractional offset
// (Chebyshev fit of the Kaiser-Bessel kernel, computed on the host).
#include <cstdio>

#include "internal.h"

namespace purify {

namespace {

constexpr int kThreads = 256;

PD void decode(const Pos<float>& p, int& cu, float& fu, int& cv, float& fv) {
  const float sc = 1.0f / 16777216.0f;
  cu = int(p.u >> 24);
  cv = int(p.v >> 24);
  fu = float(p.u & 0xFFFFFFu) * sc;
  fv = float(p.v & 0xFFFFFFu) * sc;
}
PD void decode(const Pos<double>& p, int& cu, double& fu, int& cv, double& fv) {
  const double a = floor(p.u), b = floor(p.v);
  cu = int(a);
  cv = int(b);
  fu = p.u - a;
  fv = p.v - b;
}

template <typename T> PD void kb_eval(const KbPoly<T>& kb, T f, T (&w)[kJ]) {
  constexpr int D = KbDeg<T>::value;
  const T x = T(2) * f - T(1);
#pragma unroll
  for (int a = 0; a < kJ; ++a) {
    T acc = kb.c[a][D];
#pragma unroll
    for (int d = D - 1; d >= 0; --d) acc = fma(acc, x, kb.c[a][d]);
    w[a] = acc;
  }
}

template <typename C> PD void atomic_add_global(C* p, C v);
template <> PD void atomic_add_global<float2>(float2* p, float2 v) { atomicAdd(p, v); }
template <> PD void atomic_add_global<double2>(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// Stage the work item's grid patch by TMA; returns false on a timed-out wait.
template <typename C>
PD bool stage_patch(C* patch, uint64_t* bar, const CUtensorMap* map, int tu, int tv, int TB, int PW, int* err) {
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, uint32_t(PW * PW * sizeof(C)));
    const int cw = int(sizeof(C) / 8);
    tma_load_2d(patch, map, tv * TB * cw, tu * TB, bar);
  }
  // every thread waits (bounded); the CTA leaves together if any wait gave up
  const bool ok = mbar_wait_bounded(bar, 0, err);
  return __syncthreads_and(ok) != 0;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_degrid(Geometry g, const __grid_constant__ CUtensorMap map,
                                                     const WorkItem* __restrict__ items,
                                                     const Pos<T>* __restrict__ pos, const int* __restrict__ perm,
                                                     KbPoly<T> kb, DegridEp<typename cplx_t<T>::type> ep, int* err) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ double red[32];
  C* patch = reinterpret_cast<C*>(sm_raw);
  const WorkItem it = items[blockIdx.x];
  const int tu = it.tile / g.ntile1d, tv = it.tile - tu * g.ntile1d;
  const int PW = g.TB + kJ;
  if (!stage_patch(patch, &bar, &map, tu, tv, g.TB, PW, err)) return;
  double p0 = 0.0, p1 = 0.0;
  for (int i = it.begin + threadIdx.x; i < it.end; i += kThreads) {
    int cu, cv;
    T fu, fv;
    decode(pos[i], cu, fu, cv, fv);
    T wu[kJ], wv[kJ];
    kb_eval(kb, fu, wu);
    kb_eval(kb, fv, wv);
    T ax = 0, ay = 0;
#pragma unroll
    for (int a = 0; a < kJ; ++a) {
      const C* row = patch + (cu + a) * PW + cv;
      T hx = 0, hy = 0;
#pragma unroll
      for (int b = 0; b < kJ; ++b) {
        const C gv = row[b];
        hx = fma(wv[b], gv.x, hx);
        hy = fma(wv[b], gv.y, hy);
      }
      ax = fma(wu[a], hx, ax);
      ay = fma(wu[a], hy, ay);
    }
    if (ep.mode == DG_STORE_PERM) {
      ep.y[perm[i]] = cmk<C>(ax, ay);
    } else if (ep.mode == DG_STORE_SORTED) {
      ep.y[i] = cmk<C>(ax, ay);
    } else {  // DG_BALL
      const C z = ep.z[i], yv = ep.ys[i];
      const T nu = T(ep.nu);
      const C v = cmk<C>(fma(nu, ax, z.x), fma(nu, ay, z.y));
      ep.z[i] = v;
      const double dx = double(v.x) - ep.nu * double(yv.x), dy = double(v.y) - ep.nu * double(yv.y);
      p0 += dx * dx + dy * dy;
      const double ex = double(ax) - double(yv.x), ey = double(ay) - double(yv.y);
      p1 += ex * ex + ey * ey;
    }
  }
  if (ep.mode == DG_BALL) {
    const double s0 = block_sum<kThreads>(p0, red);
    const double s1 = block_sum<kThreads>(p1, red);
    if (threadIdx.x == 0) {
      ep.part0[blockIdx.x] = s0;
      ep.part1[blockIdx.x] = s1;
    }
  }
}

template <typename C>
PD void flush_patch(const C* acc, C* Q, int tu, int tv, int TB, int PW, int KP) {
  for (int e = threadIdx.x; e < PW * PW; e += kThreads) {
    const C v = acc[e];
    if (v.x != 0 || v.y != 0) {
      const int r = e / PW, c = e - r * PW;
      atomic_add_global(Q + size_t(tu * TB + r) * KP + (tv * TB + c), v);
    }
  }
}

template <typename T>
PD void scatter_taps(typename cplx_t<T>::type* acc, int PW, int cu, int cv, const T (&wu)[kJ], const T (&wv)[kJ],
                     T ux, T uy) {
#pragma unroll
  for (int a = 0; a < kJ; ++a) {
    typename cplx_t<T>::type* row = acc + (cu + a) * PW + cv;
    const T sx = wu[a] * ux, sy = wu[a] * uy;
#pragma unroll
    for (int b = 0; b < kJ; ++b) {
      atomicAdd(&row[b].x, wv[b] * sx);
      atomicAdd(&row[b].y, wv[b] * sy);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_grid(Geometry g, const WorkItem* __restrict__ items,
                                                   const Pos<T>* __restrict__ pos, const int* __restrict__ perm,
                                                   KbPoly<T> kb, GridPro<typename cplx_t<T>::type> pro,
                                                   typename cplx_t<T>::type* __restrict__ Q) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  C* acc = reinterpret_cast<C*>(sm_raw);
  const WorkItem it = items[blockIdx.x];
  const int tu = it.tile / g.ntile1d, tv = it.tile - tu * g.ntile1d;
  const int PW = g.TB + kJ;
  for (int e = threadIdx.x; e < PW * PW; e += kThreads) acc[e] = cz<C>();
  __syncthreads();
  T scale = 0;
  if (pro.mode == GP_BALL) scale = T(pro.scalars[pro.scale_idx]);
  for (int i = it.begin + threadIdx.x; i < it.end; i += kThreads) {
    C u;
    if (pro.mode == GP_PERM) {
      u = pro.y[perm[i]];
    } else if (pro.mode == GP_SORTED) {
      u = pro.y[i];
    } else {  // GP_BALL
      const C v = pro.z[i], yv = pro.ys[i];
      const T nu = T(pro.nu);
      const T cx = nu * yv.x, cy = nu * yv.y;
      const T rx = fma(v.x - cx, scale, cx), ry = fma(v.y - cy, scale, cy);
      pro.z[i] = cmk<C>(v.x - rx, v.y - ry);
      u = cmk<C>(T(2) * rx - v.x, T(2) * ry - v.y);
    }
    int cu, cv;
    T fu, fv;
    decode(pos[i], cu, fu, cv, fv);
    T wu[kJ], wv[kJ];
    kb_eval(kb, fu, wu);
    kb_eval(kb, fv, wv);
    scatter_taps<T>(acc, PW, cu, cv, wu, wv, u.x, u.y);
  }
  __syncthreads();
  flush_patch(acc, Q, tu, tv, g.TB, PW, g.KP);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_gram(Geometry g, const __grid_constant__ CUtensorMap map,
                                                   const WorkItem* __restrict__ items,
                                                   const Pos<T>* __restrict__ pos, KbPoly<T> kb,
                                                   typename cplx_t<T>::type* __restrict__ Q, int* err) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  __shared__ __align__(8) uint64_t bar;
  const WorkItem it = items[blockIdx.x];
  const int tu = it.tile / g.ntile1d, tv = it.tile - tu * g.ntile1d;
  const int PW = g.TB + kJ;
  C* patch = reinterpret_cast<C*>(sm_raw);
  C* acc = patch + PW * PW;
  for (int e = threadIdx.x; e < PW * PW; e += kThreads) acc[e] = cz<C>();
  if (!stage_patch(patch, &bar, &map, tu, tv, g.TB, PW, err)) return;
  for (int i = it.begin + threadIdx.x; i < it.end; i += kThreads) {
    int cu, cv;
    T fu, fv;
    decode(pos[i], cu, fu, cv, fv);
    T wu[kJ], wv[kJ];
    kb_eval(kb, fu, wu);
    kb_eval(kb, fv, wv);
    T ax = 0, ay = 0;
#pragma unroll
    for (int a = 0; a < kJ; ++a) {
      const C* row = patch + (cu + a) * PW + cv;
      T hx = 0, hy = 0;
#pragma unroll
      for (int b = 0; b < kJ; ++b) {
        const C gv = row[b];
        hx = fma(wv[b], gv.x, hx);
        hy = fma(wv[b], gv.y, hy);
      }
      ax = fma(wu[a], hx, ax);
      ay = fma(wu[a], hy, ay);
    }
    scatter_taps<T>(acc, PW, cu, cv, wu, wv, ax, ay);
  }
  __syncthreads();
  flush_patch(acc, Q, tu, tv, g.TB, PW, g.KP);
}

// ----------------------------------------------------------------- binning
// Grid coordinate of a uv sample on the K-periodic grid, in [0, K).
PD double grid_coord(double u, int K) {
  double t = u * (double(K) / (2.0 * 3.14159265358979323846));
  t -= double(K) * floor(t / double(K));
  if (t >= double(K)) t -= double(K);
  if (t < 0.0) t = 0.0;
  return t;
}

__global__ void k_bin_keys(const double* __restrict__ uv, int64_t M, int K, int TB, int ntile1d,
                           uint32_t* __restrict__ keys, int* __restrict__ vals) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const double tu = grid_coord(uv[2 * m], K), tv = grid_coord(uv[2 * m + 1], K);
  const int cu = min(int(tu), K - 1), cv = min(int(tv), K - 1);
  keys[m] = uint32_t((cu / TB) * ntile1d + (cv / TB));
  vals[m] = int(m);
}

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

__global__ void __launch_bounds__(kSortThreads) k_radix_hist(const uint32_t* __restrict__ keys, int64_t M, int shift,
                                                             int nblocks, int* __restrict__ hist) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  for (int k = 0; k < kSortItems; ++k) {
    const int64_t i = base + int64_t(k) * kSortThreads + threadIdx.x;
    if (i < M) atomicAdd(&h[(keys[i] >> shift) & 255u], 1);
  }
  __syncthreads();
  hist[int64_t(threadIdx.x) * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of a[0..L) in place by one 1024-thread block; total -> *total.
__global__ void __launch_bounds__(1024) k_scan(int* __restrict__ a, int64_t L, int* __restrict__ total) {
  __shared__ int sums[1024];
  const int64_t per = (L + 1023) / 1024;
  const int64_t lo = int64_t(threadIdx.x) * per;
  const int64_t hi = lo + per < L ? lo + per : L;
  int s = 0;
  for (int64_t i = lo; i < hi; ++i) s += a[i];
  sums[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int v = threadIdx.x >= off ? sums[threadIdx.x - off] : 0;
    __syncthreads();
    sums[threadIdx.x] += v;
    __syncthreads();
  }
  int run = threadIdx.x > 0 ? sums[threadIdx.x - 1] : 0;
  for (int64_t i = lo; i < hi; ++i) {
    const int v = a[i];
    a[i] = run;
    run += v;
  }
  if (threadIdx.x == 1023 && total) *total = sums[1023];
}

__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(const uint32_t* __restrict__ kin,
                                                                const int* __restrict__ vin, int64_t M, int shift,
                                                                int nblocks, const int* __restrict__ offs,
                                                                uint32_t* __restrict__ kout, int* __restrict__ vout) {
  constexpr int NW = kSortThreads / 32;
  __shared__ int running[256];
  __shared__ int wcount[NW][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  running[threadIdx.x] = offs[int64_t(threadIdx.x) * nblocks + blockIdx.x];
  for (int k = 0; k < NW; ++k) wcount[k][threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = int64_t(blockIdx.x) * kSortTile;
  const unsigned lt = (1u << lane) - 1u;
  for (int round = 0; round < kSortItems; ++round) {
    const int64_t i = base + int64_t(round) * kSortThreads + threadIdx.x;
    const bool valid = i < M;
    uint32_t key = 0;
    int val = 0;
    int d = 256;  // sentinel digit for the ragged tail
    if (valid) {
      key = kin[i];
      val = vin[i];
      d = int((key >> shift) & 255u);
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & lt);
    if (valid && rank == 0) wcount[w][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      int pos = running[d] + rank;
      for (int k = 0; k < w; ++k) pos += wcount[k][d];
      kout[pos] = key;
      vout[pos] = val;
    }
    __syncthreads();
    int add = 0;
    for (int k = 0; k < NW; ++k) {
      add += wcount[k][threadIdx.x];
      wcount[k][threadIdx.x] = 0;
    }
    running[threadIdx.x] += add;
    __syncthreads();
  }
}

__global__ void k_tile_bounds(const uint32_t* __restrict__ keys, int64_t M, int* __restrict__ start,
                              int* __restrict__ end) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const uint32_t k = keys[i];
  if (i == 0 || keys[i - 1] != k) start[k] = int(i);
  if (i == M - 1 || keys[i + 1] != k) end[k] = int(i + 1);
}

__global__ void k_chunk_counts(const int* __restrict__ start, const int* __restrict__ end, int ntiles, int chunk,
                               int* __restrict__ cnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const int c = end[t] - start[t];
  cnt[t] = (c + chunk - 1) / chunk;
}

__global__ void k_fill_items(const int* __restrict__ start, const int* __restrict__ end,
                             const int* __restrict__ off, int ntiles, int chunk, WorkItem* __restrict__ items) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const int s = start[t], e = end[t];
  int o = off[t];
  for (int b = s; b < e; b += chunk, ++o) {
    WorkItem w;
    w.tile = t;
    w.begin = b;
    w.end = min(e, b + chunk);
    w.pad = 0;
    items[o] = w;
  }
}

template <typename T>
__global__ void k_encode(const double* __restrict__ uv, const int* __restrict__ perm, int64_t M, int K, int TB,
                         Pos<T>* __restrict__ pos);
template <>
__global__ void k_encode<float>(const double* __restrict__ uv, const int* __restrict__ perm, int64_t M, int K, int TB,
                                Pos<float>* __restrict__ pos) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t m = perm[i];
  const double t[2] = {grid_coord(uv[2 * m], K), grid_coord(uv[2 * m + 1], K)};
  uint32_t e[2];
  for (int a = 0; a < 2; ++a) {
    const int cell = min(int(t[a]), K - 1);
    double f = t[a] - double(cell);
    uint32_t q = uint32_t(f * 16777216.0);
    if (q > 0xFFFFFFu) q = 0xFFFFFFu;
    e[a] = (uint32_t(cell % TB) << 24) | q;
  }
  Pos<float> p;
  p.u = e[0];
  p.v = e[1];
  pos[i] = p;
}
template <>
__global__ void k_encode<double>(const double* __restrict__ uv, const int* __restrict__ perm, int64_t M, int K, int TB,
                                 Pos<double>* __restrict__ pos) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t m = perm[i];
  const double tu = grid_coord(uv[2 * m], K), tv = grid_coord(uv[2 * m + 1], K);
  const int cu = min(int(tu), K - 1), cv = min(int(tv), K - 1);
  Pos<double> p;
  p.u = tu - double((cu / TB) * TB);
  p.v = tv - double((cv / TB) * TB);
  pos[i] = p;
}

template <typename T> inline size_t patch_bytes(const Geometry& g) {
  const size_t PW = size_t(g.TB + kJ);
  return PW * PW * sizeof(typename cplx_t<T>::type);
}

}  // namespace

template <typename T> cudaError_t configure_nufft() {
  const int mx = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_degrid<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_grid<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gram<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return e;
}
template cudaError_t configure_nufft<float>();
template cudaError_t configure_nufft<double>();

template <typename T>
void launch_degrid(const Geometry& g, const CUtensorMap& map, const WorkItem* items, int n_items, const Pos<T>* pos,
                   const int* perm, const KbPoly<T>& kb, const DegridEp<typename cplx_t<T>::type>& ep, int* err,
                   cudaStream_t s) {
  if (n_items <= 0) return;
  const size_t sm = patch_bytes<T>(g);
  k_degrid<T><<<n_items, kThreads, sm, s>>>(g, map, items, pos, perm, kb, ep, err);
}

template <typename T>
void launch_grid(const Geometry& g, const WorkItem* items, int n_items, const Pos<T>* pos, const int* perm,
                 const KbPoly<T>& kb, const GridPro<typename cplx_t<T>::type>& pro, typename cplx_t<T>::type* Q,
                 cudaStream_t s) {
  if (n_items <= 0) return;
  const size_t sm = patch_bytes<T>(g);
  k_grid<T><<<n_items, kThreads, sm, s>>>(g, items, pos, perm, kb, pro, Q);
}

template <typename T>
void launch_gram(const Geometry& g, const CUtensorMap& map, const WorkItem* items, int n_items, const Pos<T>* pos,
                 const KbPoly<T>& kb, typename cplx_t<T>::type* Q, int* err, cudaStream_t s) {
  if (n_items <= 0) return;
  const size_t sm = 2 * patch_bytes<T>(g);
  k_gram<T><<<n_items, kThreads, sm, s>>>(g, map, items, pos, kb, Q, err);
}

template <typename T>
int build_bins(const double* uv, int64_t M, const Geometry& g, int chunk, Pos<T>* pos, int* perm,
               WorkItem** items_out, int* n_items_out, cudaStream_t s) {
  const int ntiles = g.ntile1d * g.ntile1d;
  int bits = 0;
  while ((1 << bits) < ntiles) ++bits;
  const int passes = (bits + 7) / 8;
  const int nblocks = int((M + kSortTile - 1) / kSortTile);
  uint32_t *k0 = nullptr, *k1 = nullptr;
  int *v1 = nullptr, *hist = nullptr, *tstart = nullptr, *tend = nullptr, *cnt = nullptr, *total = nullptr;
  WorkItem* items = nullptr;
  int rc = 0;
  int h_total = 0;
  auto fail = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == 0) rc = (e == cudaErrorMemoryAllocation) ? -2 : -3;
  };
  fail(cudaMalloc(&k0, M * sizeof(uint32_t)));
  fail(cudaMalloc(&k1, M * sizeof(uint32_t)));
  fail(cudaMalloc(&v1, M * sizeof(int)));
  fail(cudaMalloc(&hist, size_t(256) * nblocks * sizeof(int)));
  fail(cudaMalloc(&tstart, size_t(ntiles) * sizeof(int)));
  fail(cudaMalloc(&tend, size_t(ntiles) * sizeof(int)));
  fail(cudaMalloc(&cnt, size_t(ntiles) * sizeof(int)));
  fail(cudaMalloc(&total, sizeof(int)));
  if (rc == 0) {
    const int tb = 256;
    k_bin_keys<<<int((M + tb - 1) / tb), tb, 0, s>>>(uv, M, g.K, g.TB, g.ntile1d, k0, perm);
    uint32_t* kin = k0;
    uint32_t* kout = k1;
    int* vin = perm;
    int* vout = v1;
    for (int p = 0; p < passes; ++p) {
      k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(kin, M, 8 * p, nblocks, hist);
      k_scan<<<1, 1024, 0, s>>>(hist, int64_t(256) * nblocks, nullptr);
      k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(kin, vin, M, 8 * p, nblocks, hist, kout, vout);
      std::swap(kin, kout);
      std::swap(vin, vout);
    }
    if (vin != perm) fail(cudaMemcpyAsync(perm, vin, M * sizeof(int), cudaMemcpyDeviceToDevice, s));
    fail(cudaMemsetAsync(tstart, 0, size_t(ntiles) * sizeof(int), s));
    fail(cudaMemsetAsync(tend, 0, size_t(ntiles) * sizeof(int), s));
    k_tile_bounds<<<int((M + tb - 1) / tb), tb, 0, s>>>(kin, M, tstart, tend);
    k_chunk_counts<<<(ntiles + tb - 1) / tb, tb, 0, s>>>(tstart, tend, ntiles, chunk, cnt);
    k_scan<<<1, 1024, 0, s>>>(cnt, ntiles, total);
    fail(cudaMemcpyAsync(&h_total, total, sizeof(int), cudaMemcpyDeviceToHost, s));
    fail(cudaStreamSynchronize(s));
    fail(cudaGetLastError());
  }
  if (rc == 0) {
    fail(cudaMalloc(&items, size_t(h_total > 0 ? h_total : 1) * sizeof(WorkItem)));
    if (rc == 0) {
      const int tb = 256;
      k_fill_items<<<(ntiles + tb - 1) / tb, tb, 0, s>>>(tstart, tend, cnt, ntiles, chunk, items);
      k_encode<T><<<int((M + tb - 1) / tb), tb, 0, s>>>(uv, perm, M, g.K, g.TB, pos);
      fail(cudaStreamSynchronize(s));
      fail(cudaGetLastError());
    }
  }
  cudaFree(k0);
  cudaFree(k1);
  cudaFree(v1);
  cudaFree(hist);
  cudaFree(tstart);
  cudaFree(tend);
  cudaFree(cnt);
  cudaFree(total);
  if (rc != 0) {
    cudaFree(items);
    return rc;
  }
  *items_out = items;
  *n_items_out = h_total;
  return 0;
}

#define INST(T)                                                                                              \
  template void launch_degrid<T>(const Geometry&, const CUtensorMap&, const WorkItem*, int, const Pos<T>*,      \
                                 const int*, const KbPoly<T>&, const DegridEp<cplx_t<T>::type>&, int*,          \
                                 cudaStream_t);                                                                \
  template void launch_grid<T>(const Geometry&, const WorkItem*, int, const Pos<T>*, const int*,                \
                               const KbPoly<T>&, const GridPro<cplx_t<T>::type>&, cplx_t<T>::type*,             \
                               cudaStream_t);                                                                  \
  template void launch_gram<T>(const Geometry&, const CUtensorMap&, const WorkItem*, int, const Pos<T>*,        \
                               const KbPoly<T>&, cplx_t<T>::type*, int*, cudaStream_t);                         \
  template int build_bins<T>(const double*, int64_t, const Geometry&, int, Pos<T>*, int*, WorkItem**, int*,     \
                             cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace purify
