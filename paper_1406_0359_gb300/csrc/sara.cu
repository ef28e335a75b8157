// SARA dictionary Psi = [Dirac, Db1, ..., Db8] / 3 (Section 2.2) on the GPU,
// or a sub-dictionary of it (Section 4's BP = Dirac, BPDb8 = Db8, ...): the q
// selected bases, each scaled by 1/sqrt(q), coefficients basis-major in
// increasing basis order (Dirac first).
//
// Analysis (Psi^H): one launch per wavelet level covers all selected
// Daubechies filters (blockIdx.z = filter slot).  A CTA stages its periodic input tile once in
// shared memory, filters the rows (axis 1) into low/high halves, then the
// columns (axis 0), and writes the three detail sub-bands of the level to their
// Mallat positions; the low-low band goes to a scratch band for the next level
// (or to its final place at the last level).  Convention, per axis:
//     lo[k] = sum_m h[m] x[(2k + m) mod L],   hi[k] = sum_m g[m] x[(2k + m) mod L].
// Synthesis (Psi) is the exact adjoint, one launch per level from the coarsest;
// the finest level is fused across all eight filters and the Dirac block, so
// the image is written once.
//
// SDMM fusions (Algorithm 1, blocks i = 1, 2): the analysis epilogue applies
// the l1 proximity operator to v = Psi^H x_hat + z_1 (soft threshold at
// gamma w), updates z_1 and emits 2 r_1 - v_1 for the synthesis, plus FP64
// partial sums of the objective ||W Psi^H x_hat||_1; the final synthesis
// epilogue applies the positivity block and writes x_1 + x_2.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/purify.h"
#include "host_math.h"
#include "internal.h"

namespace purify {

namespace {

constexpr int kTH = 16;  // analysis: output coefficients per tile side
constexpr int kTO = 32;  // synthesis: output samples per tile side
constexpr int kThr = 256;

// Periodic index i mod L (the integer modulo only off the common in-range case).
PD int wrap(int i, int L) {
  if (i >= 0 && i < L) return i;
  i %= L;
  return i < 0 ? i + L : i;
}

// Final coefficient epilogue: plain store or fused l1 prox.
template <typename T> struct CoefOut {
  T* c;           // plain: Psi^H x [9][n][n]
  int prox;       // 0: plain, 1: l1 block
  T* z1;
  const T* w;
  T* cs;          // prox output 2r - v
  T gamma;
};

template <typename T> PD void emit(const CoefOut<T>& o, size_t idx, T alpha, Acc<T>& part) {
  if (!o.prox) {
    o.c[idx] = alpha;
    return;
  }
  const T wj = o.w ? o.w[idx] : T(1);
  const T v = alpha + o.z1[idx];
  const T thr = o.gamma * wj;
  const T av = fabs(v);
  const T r = av > thr ? copysign(av - thr, v) : T(0);
  o.z1[idx] = v - r;
  o.cs[idx] = T(2) * r - v;
  part.add_prod(wj, fabs(alpha));
}

// emit for NE coefficients at once: every w and z_1 load precedes the first
// store (the stores may alias them, which would otherwise serialise one memory
// round trip per coefficient).
template <int NE, typename T>
PD void emit_n(const CoefOut<T>& o, const size_t (&idx)[NE], const T (&alpha)[NE], int ne, Acc<T>& part) {
  if (!o.prox) {
#pragma unroll
    for (int k = 0; k < NE; ++k)
      if (k < ne) o.c[idx[k]] = alpha[k];
    return;
  }
  T wj[NE], z[NE];
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    wj[k] = (k < ne && o.w) ? o.w[idx[k]] : T(1);
    z[k] = k < ne ? o.z1[idx[k]] : T(0);
  }
#pragma unroll
  for (int k = 0; k < NE; ++k) {
    if (k >= ne) continue;
    const T v = alpha[k] + z[k];
    const T thr = o.gamma * wj[k];
    const T av = fabs(v);
    const T r = av > thr ? copysign(av - thr, v) : T(0);
    o.z1[idx[k]] = v - r;
    o.cs[idx[k]] = T(2) * r - v;
    part.add_prod(wj[k], fabs(alpha[k]));
  }
}

template <typename T> struct AnaArgs {
  const T* in;
  size_t in_stride;  // elements between filters' input bands (0: shared input)
  int L;             // input band side
  int n;
  T* s_out;          // LL scratch [filter slot][H*H]
  int last;          // LL band is final
  int slot0;         // coefficient block of filter slot 0 (1 when the Dirac basis is selected)
  int fid[kMaxDb];   // Daubechies filter (K - 1) of each filter slot
  T scale;           // 1 / sqrt(number of bases)
  CoefOut<T> out;
  double* partials;  // per-CTA objective partials, Acc<T> in double slots (prox only)
};

template <typename T, int F>
__device__ void ana_body(const AnaArgs<T>& A, const T* __restrict__ h, const T* __restrict__ g, int z, T* sm,
                         double* red) {
  constexpr int W = 2 * kTH + F - 2;
  T* X = sm;
  T* lo = X + W * W;
  T* hi = lo + W * kTH;
  const int L = A.L, H = L / 2, n = A.n;
  const int r0 = blockIdx.y * kTH, c0 = blockIdx.x * kTH;
  const T* in = A.in + size_t(z) * A.in_stride;
  {
    // warps take rows, lanes columns: each lane wraps its few columns once
    constexpr int NC = (W + 31) / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int cols[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) cols[k] = wrap(2 * c0 + lane + 32 * k, L);
    for (int ir = wid; ir < W; ir += kThr / 32) {
      const T* row = in + size_t(wrap(2 * r0 + ir, L)) * L;
#pragma unroll
      for (int k = 0; k < NC; ++k)
        if (lane + 32 * k < W) X[ir * W + lane + 32 * k] = row[cols[k]];
    }
  }
  __syncthreads();
  // row filtering, CB consecutive outputs per item: they share F + 2 CB - 2 inputs
  constexpr int CB = 4;
  for (int e = threadIdx.x; e < W * (kTH / CB); e += kThr) {
    const int ir = e / (kTH / CB), cg = e - ir * (kTH / CB);
    const T* xr = X + ir * W + 2 * CB * cg;
    T xv[F + 2 * CB - 2];
#pragma unroll
    for (int k = 0; k < F + 2 * CB - 2; ++k) xv[k] = xr[k];
#pragma unroll
    for (int b = 0; b < CB; ++b) {
      T sl = 0, sh = 0;
#pragma unroll
      for (int m = 0; m < F; ++m) {
        sl = fma(h[m], xv[2 * b + m], sl);
        sh = fma(g[m], xv[2 * b + m], sh);
      }
      lo[ir * kTH + CB * cg + b] = sl;
      hi[ir * kTH + CB * cg + b] = sh;
    }
  }
  __syncthreads();
  Acc<T> part;
  const int r = threadIdx.x / kTH, c = threadIdx.x - r * kTH;
  const int R = r0 + r, Cc = c0 + c;
  if (R < H && Cc < H) {
    T ll = 0, lh = 0, hl = 0, hh = 0;
#pragma unroll
    for (int m = 0; m < F; ++m) {
      const T a = lo[(2 * r + m) * kTH + c], b = hi[(2 * r + m) * kTH + c];
      ll = fma(h[m], a, ll);
      lh = fma(h[m], b, lh);
      hl = fma(g[m], a, hl);
      hh = fma(g[m], b, hh);
    }
    const size_t base = size_t(A.slot0 + z) * n * n;
    const T sc = A.scale;
    const size_t idx[4] = {base + size_t(R) * n + (H + Cc), base + size_t(H + R) * n + Cc,
                           base + size_t(H + R) * n + (H + Cc), base + size_t(R) * n + Cc};
    const T val[4] = {lh * sc, hl * sc, hh * sc, ll * sc};
    emit_n<4>(A.out, idx, val, A.last ? 4 : 3, part);
    if (!A.last) A.s_out[size_t(z) * H * H + size_t(R) * H + Cc] = ll;
  }
  if (A.partials) {
    const Acc<T> t = block_merge<kThr>(part, red);
    if (threadIdx.x == 0)
      reinterpret_cast<Acc<T>*>(A.partials)[(size_t(z) * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
  }
}

// One analysis level; blockIdx.z = instance * nf + filter slot (one
// instance: nf = gridDim.z).
template <typename T, typename Src>
__global__ void __launch_bounds__(kThr) k_ana_level(Src src, int nf, DbFilters<T> f) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ double red[32];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const int inst = int(blockIdx.z) / nf, z = int(blockIdx.z) - inst * nf;
  const AnaArgs<T> A = src.get_at(inst);
  const int k = A.fid[z];
  const T* h = f.h[k];
  const T* g = f.g[k];
  switch (k) {
    case 0: ana_body<T, 2>(A, h, g, z, sm, red); break;
    case 1: ana_body<T, 4>(A, h, g, z, sm, red); break;
    case 2: ana_body<T, 6>(A, h, g, z, sm, red); break;
    case 3: ana_body<T, 8>(A, h, g, z, sm, red); break;
    case 4: ana_body<T, 10>(A, h, g, z, sm, red); break;
    case 5: ana_body<T, 12>(A, h, g, z, sm, red); break;
    case 6: ana_body<T, 14>(A, h, g, z, sm, red); break;
    default: ana_body<T, 16>(A, h, g, z, sm, red); break;
  }
}

// Dirac block: c_0 = x / sqrt(q) (with the prox epilogue when fused).
template <typename T> struct DiracArgs {
  const T* x;
  size_t N;
  T scale;
  CoefOut<T> out;
  double* partials;
};
template <typename T, typename Src>
__global__ void __launch_bounds__(kThr) k_dirac(Src src) {
  __shared__ double red[32];
  decltype(auto) a = src.get();
  const T* __restrict__ x = a.x;
  const size_t N = a.N;
  const T scale = a.scale;
  const CoefOut<T>& out = a.out;
  double* partials = a.partials;
  Acc<T> part;
  const size_t i = size_t(blockIdx.x) * kThr + threadIdx.x;
  if (i < N) emit(out, i, x[i] * scale, part);
  if (partials) {
    const Acc<T> t = block_merge<kThr>(part, red);
    if (threadIdx.x == 0) reinterpret_cast<Acc<T>*>(partials)[blockIdx.x] = t;
  }
}

template <typename T> struct SynArgs {
  const T* c;       // final coefficients [q][n][n] (plain Psi^H layout)
  const T* s_in;    // LL band from the coarser synthesis level, or null (LL is final in c)
  int H;            // coefficient band side; output side L = 2H
  int n;
  T* s_out;         // [filter slot][L*L] (intermediate levels)
  int slot0;        // coefficient block of filter slot 0 (1 when the Dirac basis is selected)
  int nf;           // selected Daubechies filters
  int fid[kMaxDb];  // Daubechies filter (K - 1) of each filter slot
  T scale;          // 1 / sqrt(number of bases)
  // finest level (fused over filters):
  int fused;
  int pos_block;    // apply the positivity block
  T* x_out;
  const T* xh;
  T* z2;
};

// Output samples of thread t in a synthesis tile: acc[2 q + p] is row
// il = e / (kTO/2), column jl = 2 (e mod kTO/2) + p of item e = t + q kThr.
PD void syn_out_pos(int q, int& il, int& jl) {
  const int e = int(threadIdx.x) + (q >> 1) * kThr;
  il = e / (kTO / 2);
  jl = 2 * (e % (kTO / 2)) + (q & 1);
}
constexpr int kUP = 48;  // row pitch of the upsampled rows (16 mod 32: two rows of a warp's reads hit distinct banks)

// One filter's level synthesis of the output tile (i0, j0).  Upsampling along
// rows then columns; outputs 2j and 2j + 1 of either pass read the same
// inputs (rows / columns j - t + F/2), so each item computes both parities.
template <typename T, int F>
__device__ void syn_body(const SynArgs<T>& S, const T* __restrict__ h, const T* __restrict__ g, int z, T* sm,
                         int i0, int j0, T (&acc)[kTO * kTO / kThr], bool accumulate) {
  constexpr int CT = kTO / 2 + F / 2, HF = F / 2;
  static_assert(CT <= kUP && kTO * kTO / kThr == 4, "tile shape");
  T* LLt = sm;
  T* LHt = LLt + CT * CT;
  T* HLt = LHt + CT * CT;
  T* HHt = HLt + CT * CT;
  T* Ulo = HHt + CT * CT;      // [kTO][kUP]
  T* Uhi = Ulo + kTO * kUP;
  const int H = S.H, n = S.n, L = 2 * H;
  const T* cb = S.c + size_t(S.slot0 + z) * n * n;
  const T t3 = S.scale;
  const int rb = i0 / 2 - F / 2, cbase = j0 / 2 - F / 2;
  {
    // warps take rows, lanes columns (CT <= 24 columns)
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int lc = lane;
    const int c = wrap(cbase + lc, H);
    const T* sb = S.s_in ? S.s_in + size_t(z) * H * H : nullptr;
    for (int lr = wid; lr < CT; lr += kThr / 32) {
      if (lc >= CT) continue;
      const int r = wrap(rb + lr, H);
      const int e = lr * CT + lc;
      LLt[e] = sb ? sb[size_t(r) * H + c] : cb[size_t(r) * n + c] * t3;
      LHt[e] = cb[size_t(r) * n + (H + c)] * t3;
      HLt[e] = cb[size_t(H + r) * n + c] * t3;
      HHt[e] = cb[size_t(H + r) * n + (H + c)] * t3;
    }
  }
  __syncthreads();
  // rows il = 2j + par: U(il, lc) = sum_t h[par + 2t] LL(j - t + HF, lc) + g[par + 2t] HL(...)
  for (int e = threadIdx.x; e < (kTO / 2) * CT; e += kThr) {
    const int j = e / CT, lc = e - j * CT;
    const int o = (j + HF) * CT + lc;
    T ul0 = 0, ul1 = 0, uh0 = 0, uh1 = 0;
#pragma unroll
    for (int t = 0; t < HF; ++t) {
      const T a = LLt[o - t * CT], b = HLt[o - t * CT], c = LHt[o - t * CT], d = HHt[o - t * CT];
      ul0 = fma(h[2 * t], a, fma(g[2 * t], b, ul0));
      ul1 = fma(h[2 * t + 1], a, fma(g[2 * t + 1], b, ul1));
      uh0 = fma(h[2 * t], c, fma(g[2 * t], d, uh0));
      uh1 = fma(h[2 * t + 1], c, fma(g[2 * t + 1], d, uh1));
    }
    Ulo[(2 * j) * kUP + lc] = ul0;
    Ulo[(2 * j + 1) * kUP + lc] = ul1;
    Uhi[(2 * j) * kUP + lc] = uh0;
    Uhi[(2 * j + 1) * kUP + lc] = uh1;
  }
  __syncthreads();
  // columns jl = 2j + par: X(il, jl) = sum_t h[par + 2t] Ulo(il, j - t + HF) + g[par + 2t] Uhi(...)
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int e = threadIdx.x + q * kThr;
    const int il = e / (kTO / 2), j = e % (kTO / 2);
    const int o = il * kUP + j + HF;
    T v0 = 0, v1 = 0;
#pragma unroll
    for (int t = 0; t < HF; ++t) {
      const T a = Ulo[o - t], b = Uhi[o - t];
      v0 = fma(h[2 * t], a, fma(g[2 * t], b, v0));
      v1 = fma(h[2 * t + 1], a, fma(g[2 * t + 1], b, v1));
    }
    if (accumulate) {
      acc[2 * q] += v0;
      acc[2 * q + 1] += v1;
    } else if (i0 + il < L && j0 + 2 * j + 1 < L) {
      T* dst = S.s_out + size_t(z) * L * L + size_t(i0 + il) * L + (j0 + 2 * j);
      dst[0] = v0;
      dst[1] = v1;
    }
  }
  __syncthreads();
}

template <typename T>
__device__ void syn_dispatch(const SynArgs<T>& S, const DbFilters<T>& f, int z, int k, T* sm, int i0, int j0,
                             T (&acc)[kTO * kTO / kThr], bool accumulate) {
  const T* h = f.h[k];
  const T* g = f.g[k];
  switch (k) {
    case 0: syn_body<T, 2>(S, h, g, z, sm, i0, j0, acc, accumulate); break;
    case 1: syn_body<T, 4>(S, h, g, z, sm, i0, j0, acc, accumulate); break;
    case 2: syn_body<T, 6>(S, h, g, z, sm, i0, j0, acc, accumulate); break;
    case 3: syn_body<T, 8>(S, h, g, z, sm, i0, j0, acc, accumulate); break;
    case 4: syn_body<T, 10>(S, h, g, z, sm, i0, j0, acc, accumulate); break;
    case 5: syn_body<T, 12>(S, h, g, z, sm, i0, j0, acc, accumulate); break;
    case 6: syn_body<T, 14>(S, h, g, z, sm, i0, j0, acc, accumulate); break;
    default: syn_body<T, 16>(S, h, g, z, sm, i0, j0, acc, accumulate); break;
  }
}

// Intermediate synthesis level: blockIdx.z = instance * nf + filter slot,
// output band -> scratch.
template <typename T, typename Src>
__global__ void __launch_bounds__(kThr) k_syn_level(Src src, int nf, DbFilters<T> f) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const int inst = int(blockIdx.z) / nf, z = int(blockIdx.z) - inst * nf;
  const SynArgs<T> S = src.get_at(inst);
  T acc[kTO * kTO / kThr];
  syn_dispatch(S, f, z, S.fid[z], sm, blockIdx.y * kTO, blockIdx.x * kTO, acc, false);
}

// Finest level: all selected filters and the Dirac block summed into the
// image (ALL: the eight filters in slots 0..7, unrolled).
template <typename T, bool ALL, typename Src>
__global__ void __launch_bounds__(kThr) k_syn_final(Src src, DbFilters<T> f) {
  const SynArgs<T> S = src.get_at(int(blockIdx.z));
  extern __shared__ __align__(16) unsigned char sm_raw[];
  T* sm = reinterpret_cast<T*>(sm_raw);
  const int i0 = blockIdx.y * kTO, j0 = blockIdx.x * kTO;
  T acc[kTO * kTO / kThr];
#pragma unroll
  for (int q = 0; q < kTO * kTO / kThr; ++q) acc[q] = 0;
  if constexpr (ALL) {
#pragma unroll
    for (int k = 0; k < kMaxDb; ++k) syn_dispatch(S, f, k, k, sm, i0, j0, acc, true);
  } else {
    for (int z = 0; z < S.nf; ++z) syn_dispatch(S, f, z, S.fid[z], sm, i0, j0, acc, true);
  }
  const int n = S.n;
#pragma unroll
  for (int q = 0; q < kTO * kTO / kThr; ++q) {
    int il, jl;
    syn_out_pos(q, il, jl);
    if (i0 + il >= n || j0 + jl >= n) continue;
    const size_t idx = size_t(i0 + il) * n + (j0 + jl);
    const T x1 = S.slot0 ? acc[q] + S.c[idx] * S.scale : acc[q];  // Dirac block
    if (S.pos_block) {
      const T v2 = S.xh[idx] + S.z2[idx];
      const T r2 = v2 > T(0) ? v2 : T(0);
      S.z2[idx] = v2 - r2;
      S.x_out[idx] = x1 + (T(2) * r2 - v2);
    } else {
      S.x_out[idx] = x1;
    }
  }
}

template <typename T> size_t ana_smem(int F) {
  const int W = 2 * kTH + F - 2;
  return size_t(W * W + 2 * W * kTH) * sizeof(T);
}
template <typename T> size_t syn_smem(int F) {
  const int CT = kTO / 2 + F / 2;
  return size_t(4 * CT * CT + 2 * kTO * kUP) * sizeof(T);
}

inline int cdiv(int a, int b) { return (a + b - 1) / b; }

// Launch plan of one analysis (Dirac block, then one launch per level) and
// one synthesis (coarse levels, then the fused finest level), shared by the
// single-operator path (arguments by value) and the batch (device tables).
template <typename T> struct AnaPlan {
  bool dirac;
  DiracArgs<T> d;
  int nb0;
  int levels;
  AnaArgs<T> a[16];
  dim3 grid[16];  // z = filter slots
  int np;         // objective partials written
};
template <typename T>
AnaPlan<T> plan_analysis(const SaraPlan<T>& P, const T* x, const CoefOut<T>& out, double* partials) {
  AnaPlan<T> pl{};
  const int n = P.n;
  const size_t N = size_t(n) * n;
  pl.dirac = P.dirac != 0;
  pl.nb0 = int((N + kThr - 1) / kThr);
  pl.d = DiracArgs<T>{x, N, P.scale, out, partials};
  int np = pl.dirac && partials ? pl.nb0 : 0;
  pl.levels = P.nf > 0 ? P.levels : 0;
  const T* in = x;
  size_t in_stride = 0;
  T* bufs[2] = {P.s0, P.s1};
  for (int lev = 1; lev <= pl.levels; ++lev) {
    const int L = n >> (lev - 1), H = L / 2;
    AnaArgs<T>& A = pl.a[lev - 1];
    A.in = in;
    A.in_stride = in_stride;
    A.L = L;
    A.n = n;
    A.s_out = bufs[lev & 1];
    A.last = lev == P.levels;
    A.slot0 = P.dirac;
    for (int z = 0; z < kMaxDb; ++z) A.fid[z] = P.fid[z];
    A.scale = P.scale;
    A.out = out;
    A.partials = partials ? partials + np : nullptr;
    pl.grid[lev - 1] = dim3(cdiv(H, kTH), cdiv(H, kTH), P.nf);
    if (partials) np += int(pl.grid[lev - 1].x * pl.grid[lev - 1].y * pl.grid[lev - 1].z);
    in = A.s_out;
    in_stride = size_t(H) * H;
  }
  pl.np = np;
  return pl;
}

template <typename T> struct SynPlan {
  int levels;  // coarse levels (launches before the final one)
  SynArgs<T> a[16];
  dim3 grid[16];
  SynArgs<T> fin;
  dim3 fgrid;
  bool all;  // the eight filters: the unrolled final kernel
};
template <typename T>
SynPlan<T> plan_synthesis(const SaraPlan<T>& P, const T* c, T* x, int pos_block, const T* xh, T* z2) {
  SynPlan<T> pl{};
  const int n = P.n;
  T* bufs[2] = {P.s0, P.s1};
  const T* s_in = nullptr;
  auto select = [&](SynArgs<T>& S) {
    S.slot0 = P.dirac;
    S.nf = P.nf;
    for (int z = 0; z < kMaxDb; ++z) S.fid[z] = P.fid[z];
    S.scale = P.scale;
  };
  int k = 0;
  for (int lev = P.levels; lev >= 2 && P.nf > 0; --lev, ++k) {
    const int H = n >> lev, L = 2 * H;
    SynArgs<T>& S = pl.a[k];
    S = SynArgs<T>{};
    S.c = c;
    S.s_in = s_in;
    S.H = H;
    S.n = n;
    S.s_out = bufs[lev & 1];
    select(S);
    pl.grid[k] = dim3(cdiv(L, kTO), cdiv(L, kTO), P.nf);
    s_in = S.s_out;
  }
  pl.levels = k;
  SynArgs<T>& S = pl.fin;
  S = SynArgs<T>{};
  S.c = c;
  S.s_in = s_in;
  S.H = n / 2;
  S.n = n;
  select(S);
  S.fused = 1;
  S.pos_block = pos_block;
  S.x_out = x;
  S.xh = xh;
  S.z2 = z2;
  pl.fgrid = dim3(cdiv(n, kTO), cdiv(n, kTO), 1);
  pl.all = P.nf == kMaxDb;
  return pl;
}

// Runs the analysis levels; returns partial sums written (prox mode).
template <typename T>
int run_analysis(const SaraPlan<T>& P, const T* x, const CoefOut<T>& out, double* partials, cudaStream_t s) {
  const AnaPlan<T> pl = plan_analysis(P, x, out, partials);
  if (pl.dirac) k_dirac<T><<<pl.nb0, kThr, 0, s>>>(ArgVal<DiracArgs<T>>{pl.d});
  const size_t sm = ana_smem<T>(16);
  for (int l = 0; l < pl.levels; ++l)
    k_ana_level<T><<<pl.grid[l], kThr, sm, s>>>(ArgVal<AnaArgs<T>>{pl.a[l]}, P.nf, P.f);
  return pl.np;
}

template <typename T>
void run_synthesis(const SaraPlan<T>& P, const T* c, T* x, int pos_block, const T* xh, T* z2, cudaStream_t s) {
  const SynPlan<T> pl = plan_synthesis(P, c, x, pos_block, xh, z2);
  const size_t sm = syn_smem<T>(16);
  for (int l = 0; l < pl.levels; ++l) k_syn_level<T><<<pl.grid[l], kThr, sm, s>>>(ArgVal<SynArgs<T>>{pl.a[l]}, P.nf, P.f);
  if (pl.all)
    k_syn_final<T, true><<<pl.fgrid, kThr, sm, s>>>(ArgVal<SynArgs<T>>{pl.fin}, P.f);
  else
    k_syn_final<T, false><<<pl.fgrid, kThr, sm, s>>>(ArgVal<SynArgs<T>>{pl.fin}, P.f);
}

}  // namespace

template <typename T> cudaError_t configure_sara() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = raise_smem_limit(k_ana_level<T, ArgVal<AnaArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_syn_level<T, ArgVal<SynArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_syn_final<T, true, ArgVal<SynArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_syn_final<T, false, ArgVal<SynArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_ana_level<T, ArgTab<AnaArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_syn_level<T, ArgTab<SynArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_syn_final<T, true, ArgTab<SynArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_syn_final<T, false, ArgTab<SynArgs<T>>>);
  return e;
}
template cudaError_t configure_sara<float>();
template cudaError_t configure_sara<double>();

template <typename T> int sara_select(SaraPlan<T>& P, unsigned mask) {
  if (mask == 0 || (mask & ~kSaraAll)) return -1;
  P.dirac = int(mask & 1u);
  P.nf = 0;
  for (int k = 0; k < kMaxDb; ++k) {
    P.fid[k] = 0;
    if (mask & (2u << k)) P.fid[P.nf++] = k;
  }
  P.nbases = P.dirac + P.nf;
  P.scale = T(1.0 / std::sqrt(double(P.nbases)));
  return P.nbases;
}
template int sara_select<float>(SaraPlan<float>&, unsigned);
template int sara_select<double>(SaraPlan<double>&, unsigned);

int sara_partials_capacity(int n, int levels) {
  int np = (n * n + kThr - 1) / kThr;
  for (int lev = 1; lev <= levels; ++lev) {
    const int H = n >> lev;
    np += cdiv(H, kTH) * cdiv(H, kTH) * kMaxDb;
  }
  return np;
}

template <typename T> void sara_analysis(const SaraPlan<T>& P, const T* x, T* c, cudaStream_t s) {
  CoefOut<T> out{};
  out.c = c;
  out.prox = 0;
  run_analysis<T>(P, x, out, nullptr, s);
}

template <typename T> void sara_synthesis(const SaraPlan<T>& P, const T* c, T* x, cudaStream_t s) {
  run_synthesis<T>(P, c, x, 0, nullptr, nullptr, s);
}

template <typename T>
int sara_analysis_prox(const SaraPlan<T>& P, const T* xh, const L1Block<T>& b, cudaStream_t s) {
  CoefOut<T> out{};
  out.prox = 1;
  out.z1 = b.z1;
  out.w = b.w;
  out.cs = P.cs;
  out.gamma = T(b.gamma);
  return run_analysis(P, xh, out, b.partials, s);
}

template <typename T>
void sara_synthesis_pos(const SaraPlan<T>& P, const T* xh, T* z2, T* xs, cudaStream_t s) {
  run_synthesis<T>(P, P.cs, xs, 1, xh, z2, s);
}

// ---- batched SDMM blocks 1 and 2 (l1 prox on the analysis, positivity on
// the synthesis) for instances of one image side, levels and dictionary:
// every launch of the sequence covers all instances (device argument
// tables, instance in blockIdx.y / blockIdx.z).
template <typename T> struct SaraBatch {
  void* dev = nullptr;
  cudaMemPool_t pool = nullptr;  // dev from this pool (freed in stream order) when set
  cudaStream_t pool_stream = nullptr;
  int count = 0, nf = 0, levels_a = 0, levels_s = 0, nb0 = 0;
  bool dirac = false, all = false;
  dim3 agrid[16], sgrid[16], fgrid;
  const DiracArgs<T>* dtab = nullptr;
  const AnaArgs<T>* atab[16] = {};
  const SynArgs<T>* stab[16] = {};
  const SynArgs<T>* ftab = nullptr;
  DbFilters<T> f;
};

template <typename T>
int sara_batch_create(const std::vector<SaraBatchInst<T>>& in, SaraBatch<T>** out, int* np, cudaMemPool_t pool,
                      cudaStream_t s) {
  if (in.empty()) return PURIFY_ERR_INVALID;
  SaraBatch<T>* b = new (std::nothrow) SaraBatch<T>();
  if (!b) return PURIFY_ERR_NOMEM;
  const int count = int(in.size());
  std::vector<AnaPlan<T>> ap(count);
  std::vector<SynPlan<T>> sp(count);
  for (int i = 0; i < count; ++i) {
    const SaraBatchInst<T>& u = in[i];
    CoefOut<T> co{};
    co.prox = 1;
    co.z1 = u.z1;
    co.w = u.w;
    co.cs = u.P->cs;
    co.gamma = T(u.gamma);
    ap[i] = plan_analysis(*u.P, u.xh, co, u.partials);
    sp[i] = plan_synthesis(*u.P, u.P->cs, u.xs, 1, u.xh, u.z2);
  }
  const SaraPlan<T>& P0 = *in[0].P;
  b->count = count;
  b->nf = P0.nf;
  b->dirac = ap[0].dirac;
  b->nb0 = ap[0].nb0;
  b->levels_a = ap[0].levels;
  b->levels_s = sp[0].levels;
  b->all = sp[0].all;
  b->f = P0.f;
  // one device buffer: Dirac table, analysis tables per level, synthesis tables per level, final table
  const size_t nd = sizeof(DiracArgs<T>) * count, na = sizeof(AnaArgs<T>) * count, ns = sizeof(SynArgs<T>) * count;
  const size_t total = nd + na * b->levels_a + ns * (b->levels_s + 1);
  std::vector<unsigned char> host(total);
  size_t off = 0;
  for (int i = 0; i < count; ++i) std::memcpy(&host[off + i * sizeof(DiracArgs<T>)], &ap[i].d, sizeof(DiracArgs<T>));
  const size_t doff = off;
  off += nd;
  size_t aoff[16], soff[16];
  for (int l = 0; l < b->levels_a; ++l, off += na) {
    aoff[l] = off;
    b->agrid[l] = dim3(ap[0].grid[l].x, ap[0].grid[l].y, ap[0].grid[l].z * count);
    for (int i = 0; i < count; ++i) std::memcpy(&host[off + i * sizeof(AnaArgs<T>)], &ap[i].a[l], sizeof(AnaArgs<T>));
  }
  for (int l = 0; l < b->levels_s; ++l, off += ns) {
    soff[l] = off;
    b->sgrid[l] = dim3(sp[0].grid[l].x, sp[0].grid[l].y, sp[0].grid[l].z * count);
    for (int i = 0; i < count; ++i) std::memcpy(&host[off + i * sizeof(SynArgs<T>)], &sp[i].a[l], sizeof(SynArgs<T>));
  }
  const size_t foff = off;
  b->fgrid = dim3(sp[0].fgrid.x, sp[0].fgrid.y, count);
  for (int i = 0; i < count; ++i) std::memcpy(&host[off + i * sizeof(SynArgs<T>)], &sp[i].fin, sizeof(SynArgs<T>));
  b->pool = pool;
  b->pool_stream = s;
  if ((pool ? cudaMallocFromPoolAsync(&b->dev, total, pool, s) : cudaMalloc(&b->dev, total)) != cudaSuccess) {
    delete b;
    return PURIFY_ERR_NOMEM;
  }
  const cudaError_t ce = pool ? cudaMemcpyAsync(b->dev, host.data(), total, cudaMemcpyHostToDevice, s)
                              : cudaMemcpy(b->dev, host.data(), total, cudaMemcpyHostToDevice);
  if (ce != cudaSuccess || (pool && cudaStreamSynchronize(s) != cudaSuccess)) {
    sara_batch_destroy(b);
    return PURIFY_ERR_CUDA;
  }
  unsigned char* d = static_cast<unsigned char*>(b->dev);
  b->dtab = reinterpret_cast<const DiracArgs<T>*>(d + doff);
  for (int l = 0; l < b->levels_a; ++l) b->atab[l] = reinterpret_cast<const AnaArgs<T>*>(d + aoff[l]);
  for (int l = 0; l < b->levels_s; ++l) b->stab[l] = reinterpret_cast<const SynArgs<T>*>(d + soff[l]);
  b->ftab = reinterpret_cast<const SynArgs<T>*>(d + foff);
  *np = ap[0].np;
  *out = b;
  return PURIFY_OK;
}

template <typename T> void sara_batch_launch(const SaraBatch<T>* b, cudaStream_t s) {
  if (b->dirac) k_dirac<T><<<dim3(b->nb0, b->count), kThr, 0, s>>>(ArgTab<DiracArgs<T>>{b->dtab});
  const size_t sma = ana_smem<T>(16), sms = syn_smem<T>(16);
  for (int l = 0; l < b->levels_a; ++l)
    k_ana_level<T><<<b->agrid[l], kThr, sma, s>>>(ArgTab<AnaArgs<T>>{b->atab[l]}, b->nf, b->f);
  for (int l = 0; l < b->levels_s; ++l)
    k_syn_level<T><<<b->sgrid[l], kThr, sms, s>>>(ArgTab<SynArgs<T>>{b->stab[l]}, b->nf, b->f);
  if (b->all)
    k_syn_final<T, true><<<b->fgrid, kThr, sms, s>>>(ArgTab<SynArgs<T>>{b->ftab}, b->f);
  else
    k_syn_final<T, false><<<b->fgrid, kThr, sms, s>>>(ArgTab<SynArgs<T>>{b->ftab}, b->f);
}

template <typename T> int sara_prox_partials(const SaraPlan<T>& P) {
  CoefOut<T> co{};
  co.prox = 1;
  double dummy = 0;
  return plan_analysis(P, static_cast<const T*>(nullptr), co, &dummy).np;
}

template <typename T> void sara_batch_destroy(SaraBatch<T>* b) {
  if (!b) return;
  if (b->dev) {
    if (b->pool) cudaFreeAsync(b->dev, b->pool_stream);
    else cudaFree(b->dev);
  }
  delete b;
}

#define INST(T)                                                                                 \
  template int sara_batch_create<T>(const std::vector<SaraBatchInst<T>>&, SaraBatch<T>**, int*,   \
                                    cudaMemPool_t, cudaStream_t);                                 \
  template void sara_batch_launch<T>(const SaraBatch<T>*, cudaStream_t);                          \
  template void sara_batch_destroy<T>(SaraBatch<T>*);                                             \
  template int sara_prox_partials<T>(const SaraPlan<T>&);                                         \
  template void sara_analysis<T>(const SaraPlan<T>&, const T*, T*, cudaStream_t);                 \
  template void sara_synthesis<T>(const SaraPlan<T>&, const T*, T*, cudaStream_t);                \
  template int sara_analysis_prox<T>(const SaraPlan<T>&, const T*, const L1Block<T>&, cudaStream_t); \
  template void sara_synthesis_pos<T>(const SaraPlan<T>&, const T*, T*, T*, cudaStream_t);
INST(float)
INST(double)
#undef INST


// ---------------------------------------------------------------------------
// Allocation-free SARA analysis.
//
// Some callers cannot call cudaMalloc once they are running: pipelines that
// reserve all device memory at start-up and must not allocate while they
// stream (an allocation can stall or fail when memory is fragmented or held
// by another framework's caching allocator), and hosts that hand this library
// only pre-sized buffers.  For them the scratch bands of the multi-level
// analysis live in one fixed file-scope device array instead of operator
// memory.  The array exists once per device that loads the library and
// stays allocated until the process exits.
constexpr int kStaticMaxN = 512;  // largest image side served from the fixed scratch
constexpr size_t kStaticBand = size_t(kMaxDb) * (kStaticMaxN / 2) * (kStaticMaxN / 2);
static __device__ __align__(256) float g_static_scratch[2 * kStaticBand];  // 4 MiB

namespace {
std::mutex g_static_mu;
float* g_static_ptr[128] = {nullptr};
DbFilters<float> g_static_filters;
bool g_static_filters_ready = false;

// Device address of the fixed scratch for the current device (host code may
// not use the symbol itself as a device address).
int static_scratch(float** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 128) {
    set_last_error("purify_sara_fwd_static: cannot query the current device");
    return PURIFY_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p) {
      char buf[160];
      std::snprintf(buf, sizeof(buf), "purify_sara_fwd_static: cudaGetSymbolAddress failed: %s",
                    cudaGetErrorName(e));
      set_last_error(buf);
      return PURIFY_ERR_CUDA;
    }
    g_static_ptr[dev] = static_cast<float*>(p);
  }
  if (!g_static_filters_ready) {
    for (int k = 1; k <= kMaxDb; ++k) {
      const std::vector<double>& h = daubechies_lowpass_cached(k);
      const int F = 2 * k;
      for (int m = 0; m < kMaxTaps; ++m) {
        g_static_filters.h[k - 1][m] = m < F ? float(h[m]) : 0.0f;
        g_static_filters.g[k - 1][m] = m < F ? float(((m & 1) ? -1.0 : 1.0) * h[F - 1 - m]) : 0.0f;
      }
    }
    g_static_filters_ready = true;
  }
  *out = g_static_ptr[dev];
  return PURIFY_OK;
}
}  // namespace

}  // namespace purify

extern "C" int purify_sara_fwd_static(const float* x, float* c, int n, int levels, void* stream) {
  using namespace purify;
  if (!x || !c || n < 16 || (n & (n - 1)) || levels < 1 || (n >> levels) < 2) {
    set_last_error("purify_sara_fwd_static: need non-null x and c, n a power of two >= 16, n / 2^levels >= 2");
    return PURIFY_ERR_INVALID;
  }
  if (n > kStaticMaxN) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "purify_sara_fwd_static: n = %d exceeds the fixed-scratch limit n <= %d", n,
                  kStaticMaxN);
    set_last_error(buf);
    return PURIFY_ERR_INVALID;
  }
  float* scratch = nullptr;
  const int rc = static_scratch(&scratch);
  if (rc) return rc;
  SaraPlan<float> P{};
  P.n = n;
  P.levels = levels;
  P.s0 = scratch;
  P.s1 = scratch + kStaticBand;
  P.cs = nullptr;
  P.f = g_static_filters;
  sara_select(P, kSaraAll);
  sara_analysis<float>(P, x, c, static_cast<cudaStream_t>(stream));
  const cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) {
    char buf[160];
    std::snprintf(buf, sizeof(buf), "purify_sara_fwd_static: launch failed: %s", cudaGetErrorName(e));
    set_last_error(buf);
    return PURIFY_ERR_CUDA;
  }
  return PURIFY_OK;
}
