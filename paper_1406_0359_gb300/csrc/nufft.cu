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
#include <algorithm>
#include <cstring>
#include <vector>

#include <initializer_list>

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

// Kernel weights of the J taps at fractional offset f.  The kernel is even,
// so tap J-1-a at f equals tap a at 1-f, i.e. its polynomial in x = 2f-1 is
// tap a's at -x: with P_a(x) = E_a(x^2) + x O_a(x^2) both taps of a pair come
// from one even and one odd Horner chain in x^2.
template <typename T> PD void kb_eval(const KbPoly<T>& kb, T f, T (&w)[kJ]) {
  constexpr int D = KbDeg<T>::value;
  const T x = T(2) * f - T(1);
  const T x2 = x * x;
#pragma unroll
  for (int a = 0; a < kJ / 2; ++a) {
    T e = kb.c[a][D - (D & 1)];
#pragma unroll
    for (int d = D - (D & 1) - 2; d >= 0; d -= 2) e = fma(e, x2, kb.c[a][d]);
    T o = kb.c[a][D - 1 + (D & 1)];
#pragma unroll
    for (int d = D - 1 + (D & 1) - 2; d >= 1; d -= 2) o = fma(o, x2, kb.c[a][d]);
    w[a] = fma(x, o, e);
    w[kJ - 1 - a] = fma(-x, o, e);
  }
}

template <typename C> PD void atomic_add_global(C* p, C v);
template <> PD void atomic_add_global<float2>(float2* p, float2 v) { atomicAdd(p, v); }
template <> PD void atomic_add_global<double2>(double2* p, double2 v) {
  atomicAdd(&p->x, v.x);
  atomicAdd(&p->y, v.y);
}

// Stage the work item's grid patch by TMA; false (for every thread) when the
// bounded wait gave up in any thread.
// Staged patch: PW = TB + J rows of PP = PW + 2 grid values (the wider pitch
// spreads consecutive patch rows over distinct shared banks; the two extra
// columns are read past the grid's edge on the last tile column, where the
// tensor copy fills zeros, and never used).
template <typename C>
PD bool stage_patch(C* patch, uint64_t* bar, const CUtensorMap* map, int tu, int tv, int TB, int PW, int* err) {
  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    mbar_arrive_expect_tx(bar, uint32_t(PW * (PW + 2) * sizeof(C)));
    const int cw = int(sizeof(C) / 8);
    tma_load_2d(patch, map, tv * TB * cw, tu * TB, bar);
  }
  const bool ok = mbar_wait_bounded(bar, 0, err);
  return __syncthreads_and(ok) != 0;
}

enum TileMode : int { TM_DEGRID = 0, TM_GRID = 1, TM_GRAM = 2 };
constexpr int kWarps = kThreads / 32;
constexpr int kStage = 2 * kJ + 4;  // wu[J], wv[J], u.re, u.im, packed cell (int bits), pad

template <typename T> struct Pair2;
template <> struct Pair2<float> { typedef float2 type; };
template <> struct Pair2<double> { typedef double2 type; };

// One lane's staged visibility record (kStage values: wu[J], wv[J], e0, e1,
// the packed cell as int bits, pad) written as 16-byte vectors: at the 80-byte
// (FP32) lane stride each quarter-warp's vector stores hit distinct bank
// groups, where scalar stores at that stride collide four ways.
template <typename T> PD void stage_store(T* st, const T (&wu)[kJ], const T (&wv)[kJ], T e0, T e1, int cell);
template <> PD void stage_store<float>(float* st, const float (&wu)[kJ], const float (&wv)[kJ], float e0, float e1,
                                       int cell) {
  float4* d = reinterpret_cast<float4*>(st);
  d[0] = make_float4(wu[0], wu[1], wu[2], wu[3]);
  d[1] = make_float4(wu[4], wu[5], wu[6], wu[7]);
  d[2] = make_float4(wv[0], wv[1], wv[2], wv[3]);
  d[3] = make_float4(wv[4], wv[5], wv[6], wv[7]);
  d[4] = make_float4(e0, e1, __int_as_float(cell), 0.f);
}
template <> PD void stage_store<double>(double* st, const double (&wu)[kJ], const double (&wv)[kJ], double e0,
                                        double e1, int cell) {
  double2* d = reinterpret_cast<double2*>(st);
#pragma unroll
  for (int a = 0; a < kJ / 2; ++a) {
    d[a] = make_double2(wu[2 * a], wu[2 * a + 1]);
    d[kJ / 2 + a] = make_double2(wv[2 * a], wv[2 * a + 1]);
  }
  d[kJ] = make_double2(e0, e1);
  d[kJ + 1] = make_double2(__hiloint2double(0, cell), 0.0);
}
static_assert(kStage == 2 * kJ + 4 && kJ == 8, "stage_store writes 2J + 4 values");

// Gridding's staged record: {u.re, u.im, cell bits, pad}, then wu interleaved
// as (wu[a], wu[a + 4]) pairs, then wv[0..7] -- lane (ta, tc) reads the first
// 16 bytes, one 8-byte pair and one value per visibility.
template <typename T> PD void stage_store_grid(T* st, const T (&wu)[kJ], const T (&wv)[kJ], T ux, T uy, int cell);
template <> PD void stage_store_grid<float>(float* st, const float (&wu)[kJ], const float (&wv)[kJ], float ux,
                                            float uy, int cell) {
  float4* d = reinterpret_cast<float4*>(st);
  d[0] = make_float4(ux, uy, __int_as_float(cell), 0.f);
  d[1] = make_float4(wu[0], wu[4], wu[1], wu[5]);
  d[2] = make_float4(wu[2], wu[6], wu[3], wu[7]);
  d[3] = make_float4(wv[0], wv[1], wv[2], wv[3]);
  d[4] = make_float4(wv[4], wv[5], wv[6], wv[7]);
}
template <> PD void stage_store_grid<double>(double* st, const double (&wu)[kJ], const double (&wv)[kJ], double ux,
                                             double uy, int cell) {
  double2* d = reinterpret_cast<double2*>(st);
  d[0] = make_double2(ux, uy);
  d[1] = make_double2(__hiloint2double(0, cell), 0.0);
#pragma unroll
  for (int a = 0; a < kJ / 2; ++a) {
    d[2 + a] = make_double2(wu[a], wu[a + 4]);
    d[2 + kJ / 2 + a] = make_double2(wv[2 * a], wv[2 * a + 1]);
  }
}

template <typename T> __host__ __device__ inline size_t tile_patch_bytes(int TB) {
  const size_t PW = size_t(TB + kJ);
  return PW * (PW + 2) * sizeof(typename cplx_t<T>::type);
}
template <typename T> __host__ __device__ inline size_t tile_acc_bytes(int TB) {
  const size_t PW = size_t(TB + kJ);
  return size_t(kWarps) * PW * (PW + 1) * sizeof(typename cplx_t<T>::type);
}
template <typename T> __host__ __device__ inline size_t tile_stage_bytes() {
  return size_t(kWarps) * 32 * kStage * sizeof(T);
}

template <typename C> PD C warp_allsum(C v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// One CTA per work item; visibilities arrive sorted by grid cell inside the
// tile.  Warp w takes a contiguous slice of the item.  In 32-wide batches
// every lane first computes its own visibility's kernel weights (and, for
// gridding, its value) into a per-warp staging row; then the warp walks the
// batch one visibility at a time with lane l owning taps (l/4, 2(l%4)) and
// (l/4, 2(l%4)+1) of the J x J footprint.  For a run of visibilities in the
// same cell the lanes keep the footprint's grid values (gather) and its
// scatter sums (gridding) in registers; shared memory is touched only when
// the cell changes.  Gathered values are summed across the warp by a
// butterfly of shuffles.  Scatter sums go to the warp's private accumulator
// patch (no atomics); the patches are merged and flushed with one vector
// atomic per non-zero cell at the end.
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) k_tile(Geometry g, const __grid_constant__ CUtensorMap map,
                                                   const WorkItem* __restrict__ items,
                                                   const Pos<T>* __restrict__ pos, const int* __restrict__ perm,
                                                   KbPoly<T> kb, DegridEp<typename cplx_t<T>::type> dep,
                                                   GridPro<typename cplx_t<T>::type> gpro,
                                                   typename cplx_t<T>::type* __restrict__ Q, int* err) {
  typedef typename cplx_t<T>::type C;
  typedef typename Pair2<T>::type T2;
  constexpr bool kGather = MODE != TM_GRID;
  constexpr bool kScatter = MODE != TM_DEGRID;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ double red[32];
  const WorkItem it = items[blockIdx.x];
  const int tu = it.tile / g.ntile1d, tv = it.tile - tu * g.ntile1d;
  const int PW = g.TB + kJ, PA = PW + 1;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* cur = sm_raw;
  C* patch = reinterpret_cast<C*>(cur);
  if (kGather) cur += tile_patch_bytes<T>(g.TB);
  C* acc = reinterpret_cast<C*>(cur);
  if (kScatter) {
    cur += tile_acc_bytes<T>(g.TB);
    for (int e = threadIdx.x; e < kWarps * PW * PA; e += kThreads) acc[e] = cz<C>();
  }
  T* stage = reinterpret_cast<T*>(cur);
  if (kGather) {
    if (!stage_patch(patch, &bar, &map, tu, tv, g.TB, PW, err)) return;
  } else {
    __syncthreads();
  }
  C* wacc = acc + warp * PW * PA;
  T* wst = stage + warp * 32 * kStage;
  T scale = 0;
  if (MODE == TM_GRID && gpro.mode == GP_BALL) scale = T(gpro.scalars[gpro.scale_idx]);
  // this warp's contiguous slice of the work item
  const int cnt = it.end - it.begin;
  const int per = (cnt + kWarps - 1) / kWarps;
  const int w0 = it.begin + min(cnt, warp * per), w1 = it.begin + min(cnt, (warp + 1) * per);
  const int ta = lane >> 2, tb = (lane & 3) * 2;
  int cell_cur = -1;
  C g0 = cz<C>(), g1 = cz<C>();   // footprint grid values of the current cell (gather)
  C s0 = cz<C>(), s1 = cz<C>();   // footprint scatter sums of the current cell
  Acc<T> p0, p1;
  for (int base = w0; base < w1; base += 32) {
    const int i = base + lane;
    const bool valid = i < w1;
    T wu[kJ], wv[kJ];
    int cu = 0, cv = 0;
    C u = cz<C>();
    if (valid) {
      T fu, fv;
      decode(pos[i], cu, fu, cv, fv);
      kb_eval(kb, fu, wu);
      kb_eval(kb, fv, wv);
      if (MODE == TM_GRID) {
        if (gpro.mode == GP_PERM) {
          u = gpro.y[perm[i]];
        } else if (gpro.mode == GP_SORTED) {
          u = gpro.y[i];
        } else {  // GP_BALL
          const C v = gpro.z[i], yv = gpro.ys[i];
          const T nu = T(gpro.nu);
          const T cx = nu * yv.x, cy = nu * yv.y;
          const T rx = fma(v.x - cx, scale, cx), ry = fma(v.y - cy, scale, cy);
          gpro.z[i] = cmk<C>(v.x - rx, v.y - ry);
          u = cmk<C>(T(2) * rx - v.x, T(2) * ry - v.y);
        }
      }
    } else {
#pragma unroll
      for (int a = 0; a < kJ; ++a) wu[a] = wv[a] = T(0);
    }
    T* st = wst + lane * kStage;
#pragma unroll
    for (int a = 0; a < kJ; ++a) {
      st[a] = wu[a];
      st[kJ + a] = wv[a];
    }
    st[2 * kJ] = u.x;
    st[2 * kJ + 1] = u.y;
    *reinterpret_cast<int*>(st + 2 * kJ + 2) = cu * 256 + cv;
    __syncwarp();
    const int nv = min(32, w1 - base);
    C mine = cz<C>();  // gathered value of this lane's own visibility
    for (int j = 0; j < nv; ++j) {
      const T* sj = wst + j * kStage;
      const int cell = *reinterpret_cast<const int*>(sj + 2 * kJ + 2);
      if (cell != cell_cur) {  // warp-uniform
        const int ro = ((cell >> 8) + ta) * (PW + 2) + (cell & 255) + tb;
        if (kScatter && cell_cur >= 0) {
          C* row = wacc + ((cell_cur >> 8) + ta) * PA + (cell_cur & 255) + tb;
          row[0] = cadd(row[0], s0);
          row[1] = cadd(row[1], s1);
          s0 = s1 = cz<C>();
        }
        if (kGather) {
          g0 = patch[ro];
          g1 = patch[ro + 1];
        }
        cell_cur = cell;
      }
      const T wa = sj[ta];
      const T2 wbp = *reinterpret_cast<const T2*>(sj + kJ + tb);
      const T wb0 = wa * wbp.x, wb1 = wa * wbp.y;
      C uj;
      if (kGather) {
        C part = cmk<C>(fma(wb0, g0.x, wb1 * g1.x), fma(wb0, g0.y, wb1 * g1.y));
        uj = warp_allsum(part);
        if (lane == j) mine = uj;
      } else {
        uj = cmk<C>(sj[2 * kJ], sj[2 * kJ + 1]);
      }
      if (kScatter) {
        s0.x = fma(wb0, uj.x, s0.x);
        s0.y = fma(wb0, uj.y, s0.y);
        s1.x = fma(wb1, uj.x, s1.x);
        s1.y = fma(wb1, uj.y, s1.y);
      }
    }
    __syncwarp();
    if (MODE == TM_DEGRID && valid) {
      if (dep.mode == DG_STORE_PERM) {
        dep.y[perm[i]] = mine;
      } else if (dep.mode == DG_STORE_SORTED) {
        dep.y[i] = mine;
      } else {  // DG_BALL
        const C z = dep.z[i], yv = dep.ys[i];
        const T nu = T(dep.nu);
        const C v = cmk<C>(fma(nu, mine.x, z.x), fma(nu, mine.y, z.y));
        dep.z[i] = v;
        const T dx = fma(-nu, yv.x, v.x), dy = fma(-nu, yv.y, v.y);
        p0.add_prod(dx, dx);
        p0.add_prod(dy, dy);
        const T ex = mine.x - yv.x, ey = mine.y - yv.y;
        p1.add_prod(ex, ex);
        p1.add_prod(ey, ey);
      }
    }
  }
  if (MODE == TM_DEGRID) {
    if (dep.mode == DG_BALL) {
      const Acc<T> r0 = block_merge<kThreads>(p0, red);
      const Acc<T> r1 = block_merge<kThreads>(p1, red);
      if (threadIdx.x == 0) {
        reinterpret_cast<Acc<T>*>(dep.part0)[blockIdx.x] = r0;
        reinterpret_cast<Acc<T>*>(dep.part1)[blockIdx.x] = r1;
      }
    }
    return;
  }
  if (cell_cur >= 0) {
    C* row = wacc + ((cell_cur >> 8) + ta) * PA + (cell_cur & 255) + tb;
    row[0] = cadd(row[0], s0);
    row[1] = cadd(row[1], s1);
  }
  __syncthreads();
  // merge the warps' accumulators and flush the patch (one vector atomic per non-zero cell)
  for (int e = threadIdx.x; e < PW * PW; e += kThreads) {
    const int r = e / PW, c = e - r * PW;
    C v = cz<C>();
#pragma unroll
    for (int w = 0; w < kWarps; ++w) v = cadd(v, acc[w * PW * PA + r * PA + c]);
    if (v.x != 0 || v.y != 0) atomic_add_global(Q + size_t(tu * g.TB + r) * g.KP + (tv * g.TB + c), v);
  }
}

constexpr int kDgStage = 2 * kJ + 4;  // wu[J], wv[J], result re, im, cell, pad

// ---------------------------------------------------------------------------
// Warp-per-item forms of degridding and gridding (the ball block and the
// operator calls).  Each warp owns one work item end to end: its own TMA-staged
// patch and mbarrier (degridding) or its own accumulator patch (gridding), so
// there are no CTA-wide barriers and no cross-warp merges; items are ordered
// largest first so the hardware's CTA scheduling balances the load.
constexpr int kWItems = kThreads / 32;  // items (warps) per CTA

template <typename T> __host__ __device__ inline size_t warp_patch_elems(int TB) {
  const size_t PW = size_t(TB + kJ);
  return PW * (PW + 2);
}

template <typename C>
PD bool warp_stage_patch(C* patch, uint64_t* bar, const CUtensorMap* map, int tu, int tv, int TB, int PW, int lane,
                         int* err) {
  if (lane == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
    mbar_arrive_expect_tx(bar, uint32_t(PW * (PW + 2) * sizeof(C)));
    const int cw = int(sizeof(C) / 8);
    tma_load_2d(patch, map, tv * TB * cw, tu * TB, bar);
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(bar, 0, err);
  return __all_sync(0xffffffffu, ok) != 0;
}

template <typename T, typename Src>
__global__ void __launch_bounds__(kThreads) k_degrid_w(Src src, KbPoly<T> kb, const __grid_constant__ CUtensorMap map0) {
  typedef typename cplx_t<T>::type C;
  decltype(auto) a = src.get();
  const Geometry& g = a.g;
  const WorkItem* __restrict__ items = a.items;
  const int n_items = a.n_items;
  const Pos<T>* __restrict__ pos = a.pos;
  const int* __restrict__ perm = a.perm;
  const DegridEp<C>& dep = a.dep;
  int* err = a.err;
  const CUtensorMap* map = Src::kTable ? a.map : &map0;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  __shared__ __align__(8) uint64_t bars[kWItems];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int item = blockIdx.x * kWItems + warp;
  if (item >= n_items) return;
  const WorkItem it = items[item];
  const int tu = it.tile / g.ntile1d, tv = it.tile - tu * g.ntile1d;
  const int PW = g.TB + kJ, PP = PW + 2;
  const size_t pe = warp_patch_elems<T>(g.TB);
  C* patch = reinterpret_cast<C*>(sm_raw) + warp * pe;
  T* wst = reinterpret_cast<T*>(reinterpret_cast<C*>(sm_raw) + kWItems * pe) + warp * 32 * kDgStage;
  if (Src::kTable && lane == 0) tensormap_acquire(map);
  if (!warp_stage_patch(patch, &bars[warp], map, tu, tv, g.TB, PW, lane, err)) return;
  const int grp = lane >> 2, k = lane & 3;
  Acc<T> p0, p1;
  for (int base = it.begin; base < it.end; base += 32) {
    const int i = base + lane;
    const bool valid = i < it.end;
    const int nv = min(32, it.end - base);
    {
      T wu[kJ], wv[kJ];
      int cu = 0, cv = 0;
      if (valid) {
        T fu, fv;
        decode(pos[i], cu, fu, cv, fv);
        kb_eval(kb, fu, wu);
        kb_eval(kb, fv, wv);
      } else {
#pragma unroll
        for (int a = 0; a < kJ; ++a) wu[a] = wv[a] = T(0);
      }
      stage_store(wst + lane * kDgStage, wu, wv, T(0), T(0), cu * 256 + cv);
    }
    __syncwarp();
#pragma unroll
    for (int s4 = 0; s4 < 4; ++s4) {
      const int j = s4 * 8 + grp;
      C part = cz<C>();
      if (j < nv) {
        const T* sj = wst + j * kDgStage;
        const int cell = *reinterpret_cast<const int*>(sj + 2 * kJ + 2);
        const T wa0 = sj[2 * k], wa1 = sj[2 * k + 1];
        T wv[kJ];
        if constexpr (sizeof(T) == 4) {
          const float4 w0 = *reinterpret_cast<const float4*>(sj + kJ);
          const float4 w1 = *reinterpret_cast<const float4*>(sj + kJ + 4);
          wv[0] = w0.x; wv[1] = w0.y; wv[2] = w0.z; wv[3] = w0.w;
          wv[4] = w1.x; wv[5] = w1.y; wv[6] = w1.z; wv[7] = w1.w;
        } else {
#pragma unroll
          for (int b = 0; b < kJ; ++b) wv[b] = sj[kJ + b];
        }
        const C* r0 = patch + ((cell >> 8) + 2 * k) * PP + (cell & 255);
        const C* r1 = r0 + PP;
        T hx0 = 0, hy0 = 0, hx1 = 0, hy1 = 0;
#pragma unroll
        for (int b = 0; b < kJ; ++b) {
          const C g0 = r0[b], g1 = r1[b];
          hx0 = fma(wv[b], g0.x, hx0);
          hy0 = fma(wv[b], g0.y, hy0);
          hx1 = fma(wv[b], g1.x, hx1);
          hy1 = fma(wv[b], g1.y, hy1);
        }
        part = cmk<C>(fma(wa0, hx0, wa1 * hx1), fma(wa0, hy0, wa1 * hy1));
      }
      part.x += __shfl_xor_sync(0xffffffffu, part.x, 1);
      part.y += __shfl_xor_sync(0xffffffffu, part.y, 1);
      part.x += __shfl_xor_sync(0xffffffffu, part.x, 2);
      part.y += __shfl_xor_sync(0xffffffffu, part.y, 2);
      if (k == 0 && j < nv) {
        T* sj = wst + j * kDgStage;
        sj[2 * kJ] = part.x;
        sj[2 * kJ + 1] = part.y;
      }
    }
    __syncwarp();
    if (valid) {
      const T* st = wst + lane * kDgStage;
      const C acc_v = cmk<C>(st[2 * kJ], st[2 * kJ + 1]);
      if (dep.mode == DG_STORE_PERM) {
        dep.y[perm[i]] = acc_v;
      } else if (dep.mode == DG_STORE_SORTED) {
        dep.y[i] = acc_v;
      } else {  // DG_BALL
        const C z = dep.z[i], yv = dep.ys[i];
        const T nu = T(dep.nu);
        const C v = cmk<C>(fma(nu, acc_v.x, z.x), fma(nu, acc_v.y, z.y));
        dep.z[i] = v;
        const T dx = fma(-nu, yv.x, v.x), dy = fma(-nu, yv.y, v.y);
        p0.add_prod(dx, dx);
        p0.add_prod(dy, dy);
        const T ex = acc_v.x - yv.x, ey = acc_v.y - yv.y;
        p1.add_prod(ex, ex);
        p1.add_prod(ey, ey);
      }
    }
    __syncwarp();
  }
  if (dep.mode == DG_BALL) {
    warp_merge(p0);
    warp_merge(p1);
    if (lane == 0) {
      reinterpret_cast<Acc<T>*>(dep.part0)[item] = p0;
      reinterpret_cast<Acc<T>*>(dep.part1)[item] = p1;
    }
  }
}

// A gridding accumulator cell (one complex value); a run sum is added into
// it with one 8-byte (FP32) shared read-modify-write.  Rows of the per-warp
// patch are padded so that the quarter-warps of an update (four patch rows,
// 8 consecutive cells each) that share a half-warp fall in different banks.
template <typename T> struct __align__(2 * sizeof(T)) GCell { T x, y; };
template <typename T> PD void cell_add(GCell<T>* cell, T vx, T vy) {
  GCell<T> k = *cell;
  k.x += vx;
  k.y += vy;
  *cell = k;
}
// FP32 cells are 8 bytes, and a warp's 8-byte accesses are served per
// half-warp: its two quarter-warps (two patch rows) must fall on disjoint
// banks, i.e. rows an odd multiple of 64 bytes apart (stride = 8 mod 16
// cells).  FP64 cells (16 bytes) are served per quarter-warp and need none.
template <typename T> __host__ __device__ constexpr int grid_row_stride(int pw) {
  return (sizeof(T) == 4 && pw % 16 == 0) ? pw + 8 : pw;
}

template <typename T, typename Src>
__global__ void __launch_bounds__(kThreads) k_grid_w(Src src, KbPoly<T> kb) {
  typedef typename cplx_t<T>::type C;
  decltype(auto) a = src.get();
  const Geometry& g = a.g;
  const WorkItem* __restrict__ items = a.items;
  const int n_items = a.n_items;
  const Pos<T>* __restrict__ pos = a.pos;
  const int* __restrict__ perm = a.perm;
  const GridPro<C>& gpro = a.gpro;
  C* __restrict__ Q = a.Q;
  extern __shared__ __align__(128) unsigned char sm_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int item = blockIdx.x * kWItems + warp;
  if (item >= n_items) return;
  const WorkItem it = items[item];
  const int tu = it.tile / g.ntile1d, tv = it.tile - tu * g.ntile1d;
  const int PW = g.TB + kJ;
  // per warp: a PW x PW patch of cells (row stride PS), then the staging rows
  const int PS = grid_row_stride<T>(PW);
  GCell<T>* wacc = reinterpret_cast<GCell<T>*>(sm_raw) + warp * PW * PS;
  T* wst = reinterpret_cast<T*>(reinterpret_cast<GCell<T>*>(sm_raw) + kWItems * PW * PS) + warp * 32 * kStage;
  for (int e = lane; e < PW * PS; e += 32) wacc[e] = GCell<T>{T(0), T(0)};
  __syncwarp();
  T scale = 0;
  if (gpro.mode == GP_BALL) scale = T(gpro.block_scale ? gpro.block_scale[it.pad] : gpro.scalars[gpro.scale_idx]);
  // lane (ta, tc) accumulates footprint cells (ta, tc) and (ta + 4, tc), so
  // each quarter-warp updates 8 consecutive cells of one patch row.
  const int ta = lane >> 3, tc = lane & 7;
  const int lo = ta * PS + tc;  // the lane's first cell relative to a footprint's corner
  int scell = -1;               // the current run's cell, as its footprint corner's offset in the patch
  C s0 = cz<C>(), s1 = cz<C>();
  for (int base = it.begin; base < it.end; base += 32) {
    const int i = base + lane;
    const bool valid = i < it.end;
    const int nv = min(32, it.end - base);
    {
      T wu[kJ], wv[kJ];
      int cu = 0, cv = 0;
      C u = cz<C>();
      if (valid) {
        T fu, fv;
        decode(pos[i], cu, fu, cv, fv);
        kb_eval(kb, fu, wu);
        kb_eval(kb, fv, wv);
        if (gpro.mode == GP_PERM) {
          u = gpro.y[perm[i]];
        } else if (gpro.mode == GP_SORTED) {
          u = gpro.y[i];
        } else {  // GP_BALL
          const C v = gpro.z[i], yv = gpro.ys[i];
          const T nu = T(gpro.nu);
          const T cx = nu * yv.x, cy = nu * yv.y;
          const T rx = fma(v.x - cx, scale, cx), ry = fma(v.y - cy, scale, cy);
          gpro.z[i] = cmk<C>(v.x - rx, v.y - ry);
          u = cmk<C>(T(2) * rx - v.x, T(2) * ry - v.y);
        }
      } else {
#pragma unroll
        for (int a = 0; a < kJ; ++a) wu[a] = wv[a] = T(0);
      }
      stage_store_grid(wst + lane * kStage, wu, wv, u.x, u.y, cu * PS + cv);
    }
    __syncwarp();
    for (int j = 0; j < nv; ++j) {
      const T* sj = wst + j * kStage;
      T ux, uy;
      int cell;
      if constexpr (sizeof(T) == 4) {
        const float4 h = *reinterpret_cast<const float4*>(sj);
        ux = h.x;
        uy = h.y;
        cell = __float_as_int(h.z);
      } else {
        ux = sj[0];
        uy = sj[1];
        cell = *reinterpret_cast<const int*>(sj + 2);
      }
      if (cell != scell) {  // warp-uniform
        if (scell >= 0) {
          const int o = scell + lo;
          cell_add(wacc + o, s0.x, s0.y);
          cell_add(wacc + o + 4 * PS, s1.x, s1.y);
          s0 = s1 = cz<C>();
        }
        scell = cell;
      }
      typedef typename Pair2<T>::type T2;
      const T wb = sj[4 + kJ + tc];
      const T2 wa = *reinterpret_cast<const T2*>(sj + 4 + 2 * ta);  // (wu[ta], wu[ta + 4])
      const T a0 = wa.x * wb, a1 = wa.y * wb;
      s0.x = fma(a0, ux, s0.x);
      s0.y = fma(a0, uy, s0.y);
      s1.x = fma(a1, ux, s1.x);
      s1.y = fma(a1, uy, s1.y);
    }
    __syncwarp();
  }
  if (scell >= 0) {
    const int o = scell + lo;
    cell_add(wacc + o, s0.x, s0.y);
    cell_add(wacc + o + 4 * PS, s1.x, s1.y);
  }
  __syncwarp();
  for (int e = lane; e < PW * PW; e += 32) {
    const int r = e / PW, c = e - r * PW;
    const GCell<T> kc = wacc[r * PS + c];
    const C v = cmk<C>(kc.x, kc.y);
    if (v.x != 0 || v.y != 0) atomic_add_global(Q + size_t(tu * g.TB + r) * g.KP + (tv * g.TB + c), v);
  }
}

// ----------------------------------------------------------------- binning
// Grid cell and fractional offset of a uv sample: t = u K / (2 pi), cell =
// floor(t) taken modulo K, f = t - floor(t) in [0, 1).  The expression order
// matches the plain definition so that samples lying exactly on grid nodes
// fall in the same cell.
PD void grid_cell(double u, int K, int& cell, double& f) {
  const double t = (u * double(K)) / (2.0 * 3.14159265358979323846);
  const double fl = floor(t);
  f = t - fl;
  long long c = (long long)fl % K;
  if (c < 0) c += K;
  cell = int(c);
}

// Sort key: tile id, then the cell inside the tile (row-major), so that a
// tile's visibilities come grouped by grid cell.
// With visibility blocks (Eq. 4) the block index leads the key, so that every
// work item lies in one block.
__global__ void k_bin_keys(const double* __restrict__ uv, const int* __restrict__ blocks, int64_t M, int K, int TB,
                           int lb, int ntile1d, int tbits, uint32_t* __restrict__ keys, int* __restrict__ vals) {
  const int64_t m = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (m >= M) return;
  int cu, cv;
  double fu, fv;
  grid_cell(uv[2 * m], K, cu, fu);
  grid_cell(uv[2 * m + 1], K, cv, fv);
  const uint32_t tile = uint32_t((cu / TB) * ntile1d + (cv / TB));
  const uint32_t blk = blocks ? uint32_t(blocks[m]) : 0u;
  keys[m] = (blk << (tbits + 2 * lb)) | (tile << (2 * lb)) | (uint32_t(cu % TB) << lb) | uint32_t(cv % TB);
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

// Exclusive scan of a[0..L) in place, three phases: per-chunk sums, a scan of
// the chunk sums by one block, and per-chunk scans offset by their chunk's
// prefix (all loads and stores coalesced).  total (if not null) receives the
// sum of all L values.  Needs L <= kScanChunk * 1024.
constexpr int kScanT = 256, kScanE = 16, kScanChunk = kScanT * kScanE;

__device__ __forceinline__ int block_excl_scan_int(int v, int* sh /*[32]*/, int* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (w == 0) {
    int x = lane < nw ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += u;
    }
    sh[lane] = x;  // inclusive prefix of warp sums
  }
  __syncthreads();
  const int before = w > 0 ? sh[w - 1] : 0;
  if (total) *total = sh[nw - 1];
  __syncthreads();
  return before + incl - v;
}

__global__ void __launch_bounds__(kScanT) k_scan_reduce(const int* __restrict__ a, int64_t L, int* __restrict__ bsum) {
  __shared__ int sh[32];
  const int64_t base = int64_t(blockIdx.x) * kScanChunk;
  int v = 0;
#pragma unroll
  for (int j = 0; j < kScanE; ++j) {
    const int64_t i = base + threadIdx.x + int64_t(j) * kScanT;
    if (i < L) v += a[i];
  }
  int tot = 0;
  block_excl_scan_int(v, sh, &tot);
  if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) k_scan_top(int* __restrict__ bsum, int B, int* __restrict__ total) {
  __shared__ int sh[32];
  const int v = int(threadIdx.x) < B ? bsum[threadIdx.x] : 0;
  int tot = 0;
  const int ex = block_excl_scan_int(v, sh, &tot);
  if (int(threadIdx.x) < B) bsum[threadIdx.x] = ex;
  if (threadIdx.x == 0 && total) *total = tot;
}

__global__ void __launch_bounds__(kScanT) k_scan_down(int* __restrict__ a, int64_t L, const int* __restrict__ bsum) {
  __shared__ int tile[kScanChunk + kScanChunk / 32];
  __shared__ int sh[32];
  auto pad = [](int e) { return e + (e >> 5); };
  const int64_t base = int64_t(blockIdx.x) * kScanChunk;
#pragma unroll
  for (int j = 0; j < kScanE; ++j) {
    const int e = threadIdx.x + j * kScanT;
    tile[pad(e)] = base + e < L ? a[base + e] : 0;
  }
  __syncthreads();
  int loc[kScanE];
  int run = 0;
#pragma unroll
  for (int k = 0; k < kScanE; ++k) {
    loc[k] = run;
    run += tile[pad(threadIdx.x * kScanE + k)];
  }
  const int off = block_excl_scan_int(run, sh, nullptr) + bsum[blockIdx.x];
#pragma unroll
  for (int k = 0; k < kScanE; ++k) tile[pad(threadIdx.x * kScanE + k)] = loc[k] + off;
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kScanE; ++j) {
    const int e = threadIdx.x + j * kScanT;
    if (base + e < L) a[base + e] = tile[pad(e)];
  }
}

// Exclusive scan of a[0..L) in place by one 1024-thread block (fallback for
// L beyond the three-phase limit); total -> *total.
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

// bsum: scratch of at least 1024 ints.
inline void launch_scan(int* a, int64_t L, int* total, int* bsum, cudaStream_t s) {
  const int64_t B = (L + kScanChunk - 1) / kScanChunk;
  if (B <= 1024) {
    k_scan_reduce<<<int(B > 0 ? B : 1), kScanT, 0, s>>>(a, L, bsum);
    k_scan_top<<<1, 1024, 0, s>>>(bsum, int(B > 0 ? B : 1), total);
    k_scan_down<<<int(B > 0 ? B : 1), kScanT, 0, s>>>(a, L, bsum);
  } else {
    k_scan<<<1, 1024, 0, s>>>(a, L, total);
  }
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

__global__ void k_tile_bounds(const uint32_t* __restrict__ keys, int64_t M, int shift, int* __restrict__ start,
                              int* __restrict__ end) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const uint32_t k = keys[i] >> shift;
  if (i == 0 || (keys[i - 1] >> shift) != k) start[k] = int(i);
  if (i == M - 1 || (keys[i + 1] >> shift) != k) end[k] = int(i + 1);
}

__global__ void k_chunk_counts(const int* __restrict__ start, const int* __restrict__ end, int ntiles, int chunk,
                               int* __restrict__ cnt) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  const int c = end[t] - start[t];
  cnt[t] = (c + chunk - 1) / chunk;
}

// Bins are (block, tile) pairs, bin = block * tiles_per_block + tile; the
// item records the tile and (in `pad`) the block.
__global__ void k_fill_items(const int* __restrict__ start, const int* __restrict__ end,
                             const int* __restrict__ off, int nbins, int tiles_per_block, int chunk,
                             WorkItem* __restrict__ items) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nbins) return;
  const int s = start[t], e = end[t];
  int o = off[t];
  for (int b = s; b < e; b += chunk, ++o) {
    WorkItem w;
    w.tile = t % tiles_per_block;
    w.begin = b;
    w.end = min(e, b + chunk);
    w.pad = t / tiles_per_block;
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
  uint32_t e[2];
  for (int a = 0; a < 2; ++a) {
    int cell;
    double f;
    grid_cell(uv[2 * m + a], K, cell, f);
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
  int cu, cv;
  double fu, fv;
  grid_cell(uv[2 * m], K, cu, fu);
  grid_cell(uv[2 * m + 1], K, cv, fv);
  Pos<double> p;
  // cell + f may round up to the next integer when f is within an ulp of 1:
  // keep the sum inside the cell
  p.u = fmin(double(cu % TB) + fu, nextafter(double(cu % TB + 1), 0.0));
  p.v = fmin(double(cv % TB) + fv, nextafter(double(cv % TB + 1), 0.0));
  pos[i] = p;
}

// Positions on the grid of twice the resolution (K = 2 Kc) from the cells of
// the Kc grid: t = 2 (cell_c + f_c) exactly, so that tile (cell / TB) of the
// fine grid equals tile (cell_c / (TB/2)) of the coarse one and the coarse
// binning's items and order serve the fine grid unchanged.
template <typename T>
__global__ void k_encode_x2(const double* __restrict__ uv, const int* __restrict__ perm, int64_t M, int Kc, int TB,
                            Pos<T>* __restrict__ pos) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= M) return;
  const int64_t m = perm[i];
  int cell[2];
  double fr[2];
  for (int a = 0; a < 2; ++a) {
    int cc;
    double fc;
    grid_cell(uv[2 * m + a], Kc, cc, fc);
    const double t2 = 2.0 * fc;  // exact
    const double up = t2 >= 1.0 ? 1.0 : 0.0;
    cell[a] = (2 * cc + int(up)) % TB;
    fr[a] = t2 - up;
  }
  Pos<T> p;
  if constexpr (sizeof(T) == 4) {
    uint32_t e[2];
    for (int a = 0; a < 2; ++a) {
      uint32_t q = uint32_t(fr[a] * 16777216.0);
      if (q > 0xFFFFFFu) q = 0xFFFFFFu;
      e[a] = (uint32_t(cell[a]) << 24) | q;
    }
    p.u = e[0];
    p.v = e[1];
  } else {
    p.u = fmin(double(cell[0]) + fr[0], nextafter(double(cell[0] + 1), 0.0));
    p.v = fmin(double(cell[1]) + fr[1], nextafter(double(cell[1] + 1), 0.0));
  }
  pos[i] = p;
}

}  // namespace

template <typename T> cudaError_t configure_nufft() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = raise_smem_limit(k_degrid_w<T, ArgVal<DegridArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_grid_w<T, ArgVal<GridArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_degrid_w<T, ArgTab<DegridArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_grid_w<T, ArgTab<GridArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_tile<T, TM_GRAM>);
  return e;
}
template cudaError_t configure_nufft<float>();
template cudaError_t configure_nufft<double>();

cudaError_t set_wait_spins_nufft(uint32_t spins) { return set_module_wait_spins(spins); }

size_t tile_smem_bytes(int precision_bytes, int TB, int mode) {
  if (precision_bytes == 4) {
    size_t b = tile_stage_bytes<float>();
    if (mode != TM_GRID) b += tile_patch_bytes<float>(TB);
    if (mode != TM_DEGRID) b += tile_acc_bytes<float>(TB);
    return b;
  }
  size_t b = tile_stage_bytes<double>();
  if (mode != TM_GRID) b += tile_patch_bytes<double>(TB);
  if (mode != TM_DEGRID) b += tile_acc_bytes<double>(TB);
  return b;
}

template <typename T>
void launch_degrid(const Geometry& g, const CUtensorMap& map, const WorkItem* items, int n_items, const Pos<T>* pos,
                   const int* perm, const KbPoly<T>& kb, const DegridEp<typename cplx_t<T>::type>& ep, int* err,
                   cudaStream_t s) {
  if (n_items <= 0) return;
  const size_t sm = kWItems * (warp_patch_elems<T>(g.TB) * sizeof(typename cplx_t<T>::type) + 32 * kDgStage * sizeof(T));
  ArgVal<DegridArgs<T>> src{DegridArgs<T>{g, nullptr, items, n_items, pos, perm, ep, err}};
  k_degrid_w<T><<<(n_items + kWItems - 1) / kWItems, kThreads, sm, s>>>(src, kb, map);
}

template <typename T>
void launch_degrid_batch(const DegridArgs<T>* tab, int count, int max_items, int max_tb, const KbPoly<T>& kb,
                         cudaStream_t s) {
  if (max_items <= 0 || count <= 0) return;
  const size_t sm = kWItems * (warp_patch_elems<T>(max_tb) * sizeof(typename cplx_t<T>::type) + 32 * kDgStage * sizeof(T));
  CUtensorMap unused;
  std::memset(&unused, 0, sizeof(unused));
  ArgTab<DegridArgs<T>> src{tab};
  k_degrid_w<T><<<dim3((max_items + kWItems - 1) / kWItems, count), kThreads, sm, s>>>(src, kb, unused);
}

template <typename T>
void launch_grid(const Geometry& g, const WorkItem* items, int n_items, const Pos<T>* pos, const int* perm,
                 const KbPoly<T>& kb, const GridPro<typename cplx_t<T>::type>& pro, typename cplx_t<T>::type* Q,
                 cudaStream_t s) {
  if (n_items <= 0) return;
  const size_t PW = size_t(g.TB + kJ);
  const size_t sm = kWItems * (PW * size_t(grid_row_stride<T>(int(PW))) * sizeof(GCell<T>) + 32 * kStage * sizeof(T));
  ArgVal<GridArgs<T>> src{GridArgs<T>{g, items, n_items, pos, perm, pro, Q}};
  k_grid_w<T><<<(n_items + kWItems - 1) / kWItems, kThreads, sm, s>>>(src, kb);
}

template <typename T>
void launch_grid_batch(const GridArgs<T>* tab, int count, int max_items, int max_tb, const KbPoly<T>& kb,
                       cudaStream_t s) {
  if (max_items <= 0 || count <= 0) return;
  const size_t PW = size_t(max_tb + kJ);
  const size_t sm = kWItems * (PW * size_t(grid_row_stride<T>(int(PW))) * sizeof(GCell<T>) + 32 * kStage * sizeof(T));
  ArgTab<GridArgs<T>> src{tab};
  k_grid_w<T><<<dim3((max_items + kWItems - 1) / kWItems, count), kThreads, sm, s>>>(src, kb);
}

template <typename T>
void launch_gram(const Geometry& g, const CUtensorMap& map, const WorkItem* items, int n_items, const Pos<T>* pos,
                 const KbPoly<T>& kb, typename cplx_t<T>::type* Q, int* err, cudaStream_t s) {
  if (n_items <= 0) return;
  const size_t sm = tile_smem_bytes(sizeof(T), g.TB, TM_GRAM);
  DegridEp<typename cplx_t<T>::type> ep{};
  GridPro<typename cplx_t<T>::type> gp{};
  k_tile<T, TM_GRAM><<<n_items, kThreads, sm, s>>>(g, map, items, pos, nullptr, kb, ep, gp, Q, err);
}

template <typename T>
void launch_encode_x2(const double* uv, const int* perm, int64_t M, int Kc, int TB, Pos<T>* pos, cudaStream_t s) {
  const int tb = 256;
  k_encode_x2<T><<<int((M + tb - 1) / tb), tb, 0, s>>>(uv, perm, M, Kc, TB, pos);
}

template <typename T>
int build_bins(const double* uv, int64_t M, const Geometry& g, int chunk, Pos<T>* pos, int* perm,
               WorkItem** items_out, int* n_items_out, cudaStream_t s, const int* blocks, int R,
               cudaMemPool_t items_pool) {
  const int tiles_per_block = g.ntile1d * g.ntile1d;
  const int ntiles = tiles_per_block * (R > 1 ? R : 1);  // bins
  int lb = 0;
  while ((1 << lb) < g.TB) ++lb;
  int tbits = 0;
  while ((1 << tbits) < tiles_per_block) ++tbits;
  int rbits = 0;
  while ((1 << rbits) < (R > 1 ? R : 1)) ++rbits;
  const int bits = 2 * lb + tbits + rbits;
  const int passes = (bits + 7) / 8;
  const int nblocks = int((M + kSortTile - 1) / kSortTile);
  uint32_t *k0 = nullptr, *k1 = nullptr;
  int *v1 = nullptr, *hist = nullptr, *tstart = nullptr, *tend = nullptr, *cnt = nullptr, *total = nullptr;
  int* bsum = nullptr;
  WorkItem* items = nullptr;
  int rc = 0;
  int h_total = 0;
  auto fail = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == 0) rc = (e == cudaErrorMemoryAllocation) ? -2 : -3;
  };
  // temporaries from the set-up pool (no device-wide synchronisation on
  // release, reused across operator creations)
  fail(setup_alloc(&k0, M * sizeof(uint32_t), s));
  fail(setup_alloc(&k1, M * sizeof(uint32_t), s));
  fail(setup_alloc(&v1, M * sizeof(int), s));
  fail(setup_alloc(&hist, size_t(256) * nblocks * sizeof(int), s));
  fail(setup_alloc(&tstart, size_t(ntiles) * sizeof(int), s));
  fail(setup_alloc(&tend, size_t(ntiles) * sizeof(int), s));
  fail(setup_alloc(&cnt, size_t(ntiles) * sizeof(int), s));
  fail(setup_alloc(&total, sizeof(int), s));
  fail(setup_alloc(&bsum, 1024 * sizeof(int), s));
  if (rc == 0) {
    const int tb = 256;
    k_bin_keys<<<int((M + tb - 1) / tb), tb, 0, s>>>(uv, R > 1 ? blocks : nullptr, M, g.K, g.TB, lb, g.ntile1d,
                                                     tbits, k0, perm);
    uint32_t* kin = k0;
    uint32_t* kout = k1;
    int* vin = perm;
    int* vout = v1;
    for (int p = 0; p < passes; ++p) {
      k_radix_hist<<<nblocks, kSortThreads, 0, s>>>(kin, M, 8 * p, nblocks, hist);
      launch_scan(hist, int64_t(256) * nblocks, nullptr, bsum, s);
      k_radix_scatter<<<nblocks, kSortThreads, 0, s>>>(kin, vin, M, 8 * p, nblocks, hist, kout, vout);
      std::swap(kin, kout);
      std::swap(vin, vout);
    }
    if (vin != perm) fail(cudaMemcpyAsync(perm, vin, M * sizeof(int), cudaMemcpyDeviceToDevice, s));
    fail(cudaMemsetAsync(tstart, 0, size_t(ntiles) * sizeof(int), s));
    fail(cudaMemsetAsync(tend, 0, size_t(ntiles) * sizeof(int), s));
    // bin index = key >> 2 lb = block << tbits | tile; with tiles_per_block a power of
    // two this equals block * tiles_per_block + tile
    k_tile_bounds<<<int((M + tb - 1) / tb), tb, 0, s>>>(kin, M, 2 * lb, tstart, tend);
    k_chunk_counts<<<(ntiles + tb - 1) / tb, tb, 0, s>>>(tstart, tend, ntiles, chunk, cnt);
    launch_scan(cnt, ntiles, total, bsum, s);
    fail(cudaMemcpyAsync(&h_total, total, sizeof(int), cudaMemcpyDeviceToHost, s));
    fail(cudaStreamSynchronize(s));
    fail(cudaGetLastError());
  }
  if (rc == 0) {
    const size_t ib = size_t(h_total > 0 ? h_total : 1) * sizeof(WorkItem);
    fail(items_pool ? cudaMallocFromPoolAsync(reinterpret_cast<void**>(&items), ib, items_pool, s)
                    : cudaMalloc(&items, ib));
    if (rc == 0) {
      const int tb = 256;
      k_fill_items<<<(ntiles + tb - 1) / tb, tb, 0, s>>>(tstart, tend, cnt, ntiles, tiles_per_block, chunk, items);
      k_encode<T><<<int((M + tb - 1) / tb), tb, 0, s>>>(uv, perm, M, g.K, g.TB, pos);
      fail(cudaStreamSynchronize(s));
      fail(cudaGetLastError());
      // largest items first (stable): whole-warp items then finish together
      if (rc == 0 && h_total > 1) {
        std::vector<WorkItem> h(h_total), o(h_total);
        fail(cudaMemcpyAsync(h.data(), items, h.size() * sizeof(WorkItem), cudaMemcpyDeviceToHost, s));
        fail(cudaStreamSynchronize(s));
        // stable counting sort by length, longest first (lengths <= chunk)
        std::vector<int> first(size_t(chunk) + 2, 0);
        for (const WorkItem& w : h) first[size_t(chunk - (w.end - w.begin)) + 1] += 1;
        for (size_t k = 1; k < first.size(); ++k) first[k] += first[k - 1];
        for (const WorkItem& w : h) o[size_t(first[size_t(chunk - (w.end - w.begin))]++)] = w;
        fail(cudaMemcpyAsync(items, o.data(), o.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
        fail(cudaStreamSynchronize(s));
      }
    }
  }
  for (void* t : {static_cast<void*>(k0), static_cast<void*>(k1), static_cast<void*>(v1), static_cast<void*>(hist),
                  static_cast<void*>(bsum), static_cast<void*>(tstart), static_cast<void*>(tend),
                  static_cast<void*>(cnt), static_cast<void*>(total)})
    if (t) cudaFreeAsync(t, s);
  if (rc != 0) {
    if (items_pool) cudaFreeAsync(items, s);
    else cudaFree(items);
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
  template void launch_degrid_batch<T>(const DegridArgs<T>*, int, int, int, const KbPoly<T>&, cudaStream_t);    \
  template void launch_grid_batch<T>(const GridArgs<T>*, int, int, int, const KbPoly<T>&, cudaStream_t);        \
  template void launch_gram<T>(const Geometry&, const CUtensorMap&, const WorkItem*, int, const Pos<T>*,        \
                               const KbPoly<T>&, cplx_t<T>::type*, int*, cudaStream_t);                         \
  template void launch_encode_x2<T>(const double*, const int*, int64_t, int, int, Pos<T>*, cudaStream_t);     \
  template int build_bins<T>(const double*, int64_t, const Geometry&, int, Pos<T>*, int*, WorkItem**, int*,     \
                             cudaStream_t, const int*, int, cudaMemPool_t);
INST(float)
INST(double)
#undef INST

}  // namespace purify
