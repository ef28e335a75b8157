// Oversampled 2D FFT passes of the NUFFT (operator F of Phi = G F Z S, Section 4).
//
// Each length-K transform (K = 2n, a power of two) is a Stockham sequence of
// register radix-16 stages (one radix-8/4/2 stage last when log2 K is not a
// multiple of 4).  A thread always holds the 16 elements t + m K/16 of its
// sequence: the first stage reads them straight from global memory, the last
// writes its outputs straight to global memory, and the stages in between
// exchange through shared memory (padded every 16 elements against bank
// conflicts) -- two shared round trips for K = 2048.
//
// Forward (Phi):   row pass over the n non-zero image rows, fused with the
//                  deapodisation S and zero-padding Z (only the n non-zero
//                  inputs are read); column pass over all K columns, reading
//                  only the n non-zero rows and writing the padded grid (with
//                  its periodic J-wide halo) that degridding stages by TMA.
// Adjoint (Phi^H): column pass reading the padded gridding accumulator, folding
//                  its halo back onto the torus, writing only the n rows the
//                  crop Z^T keeps; row pass fused with the crop, the
//                  deapodisation and the solver epilogues.
#include "internal.h"

namespace purify {

namespace {

template <typename C> PD C cneg(C a) { a.x = -a.x; a.y = -a.y; return a; }

template <typename C> PD void dft2(C& a, C& b) {
  const C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

// X_k = sum_r a_r exp(dir 2 pi i r k / 4), dir = -1 forward, +1 inverse
template <typename C> PD void dft4(C& a0, C& a1, C& a2, C& a3, int dir) {
  const C s02 = cadd(a0, a2), d02 = csub(a0, a2);
  const C s13 = cadd(a1, a3), d13 = csub(a1, a3);
  C j13 = cmul_i(d13);
  if (dir < 0) j13 = cneg(j13);
  a0 = cadd(s02, s13);
  a2 = csub(s02, s13);
  a1 = cadd(d02, j13);
  a3 = csub(d02, j13);
}

// exp(dir 2 pi i m / 16) for the fixed m used by the radix-16/8 butterflies
template <typename C> PD C w16(int m, int dir) {
  typedef decltype(C().x) T;
  const T c1 = T(0.92387953251128675613), s1 = T(0.38268343236508977173);
  const T h = T(0.70710678118654752440);
  T re = 1, im = 0;
  switch (m) {
    case 1: re = c1; im = s1; break;
    case 2: re = h; im = h; break;
    case 3: re = s1; im = c1; break;
    case 4: re = 0; im = 1; break;
    case 6: re = -h; im = h; break;
    case 9: re = -c1; im = -s1; break;
    default: break;
  }
  return cmk<C>(re, dir < 0 ? -im : im);
}

// In-register DFT of a[o], a[o+st], ..., R points (Cooley-Tukey, natural order out).
template <int R, typename C> struct Dft;
template <typename C> struct Dft<2, C> {
  static PD void run(C* a, int o, int st, int) { dft2(a[o], a[o + st]); }
};
template <typename C> struct Dft<4, C> {
  static PD void run(C* a, int o, int st, int dir) { dft4(a[o], a[o + st], a[o + 2 * st], a[o + 3 * st], dir); }
};
template <typename C> struct Dft<8, C> {
  // 8 = 2 x 4: 2-point DFTs on (n2, n2+4), twiddle W8^(n2 k1), 4-point DFTs over n2
  static PD void run(C* a, int o, int st, int dir) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2) dft2(a[o + n2 * st], a[o + (n2 + 4) * st]);
    a[o + 5 * st] = cmul(a[o + 5 * st], w16<C>(2, dir));
    a[o + 6 * st] = cmul(a[o + 6 * st], w16<C>(4, dir));
    a[o + 7 * st] = cmul(a[o + 7 * st], w16<C>(6, dir));
    dft4(a[o], a[o + st], a[o + 2 * st], a[o + 3 * st], dir);
    dft4(a[o + 4 * st], a[o + 5 * st], a[o + 6 * st], a[o + 7 * st], dir);
    C t[8];  // X[k1 + 2 k2] = a[4 k1 + k2]
#pragma unroll
    for (int k1 = 0; k1 < 2; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) t[k1 + 2 * k2] = a[o + (k1 * 4 + k2) * st];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[o + k * st] = t[k];
  }
};
template <typename C> struct Dft<16, C> {
  // 16 = 4 x 4: 4-point DFTs on (n2, n2+4, n2+8, n2+12), twiddle W16^(n2 k1), 4-point DFTs
  static PD void run(C* a, int o, int st, int dir) {
#pragma unroll
    for (int n2 = 0; n2 < 4; ++n2)
      dft4(a[o + n2 * st], a[o + (n2 + 4) * st], a[o + (n2 + 8) * st], a[o + (n2 + 12) * st], dir);
#pragma unroll
    for (int n2 = 1; n2 < 4; ++n2)
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1)
        a[o + (n2 + 4 * k1) * st] = cmul(a[o + (n2 + 4 * k1) * st], w16<C>(n2 * k1, dir));
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
      dft4(a[o + 4 * k1 * st], a[o + (4 * k1 + 1) * st], a[o + (4 * k1 + 2) * st], a[o + (4 * k1 + 3) * st], dir);
    C t[16];  // X[k1 + 4 k2] = a[4 k1 + k2]
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
      for (int k2 = 0; k2 < 4; ++k2) t[k1 + 4 * k2] = a[o + (4 * k1 + k2) * st];
#pragma unroll
    for (int k = 0; k < 16; ++k) a[o + k * st] = t[k];
  }
};

PD int sidx(int e) { return e + (e >> 4); }  // padded shared index

// Compile-time plan of a length-2^LOGN transform: radix-16 stages, then one
// radix-2^(LOGN mod 4) stage; T = N/16 threads per sequence.
template <int LOGN> struct Plan {
  static constexpr int N = 1 << LOGN;
  static constexpr int T = N / 16;
  static constexpr int NST = (LOGN + 3) / 4;
  __host__ __device__ static constexpr int radix(int st) { return (st + 1 < NST || LOGN % 4 == 0) ? 16 : (1 << (LOGN % 4)); }
};

// One Stockham stage on the registers: v[m] holds element t + m T of the
// stage input.  Thread t owns butterflies j = t + q T (q < 16/R); input r of
// butterfly j is element j + r N/R, i.e. register q + r 16/R.  After the
// twiddles and the DFT, register q + r 16/R is output (j - k) R + k + r Ns
// with k = j mod Ns; sink(position, value) receives every output.
template <int R, int N, int T, typename C, typename Sink>
PD void stage(C (&v)[16], int t, int Ns, const C* __restrict__ tw, int dir, Sink sink) {
  constexpr int Q = 16 / R;
  const int tstride = N / (Ns * R);
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = t + q * T;
    const int k = j & (Ns - 1);
    if (k) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = tw[r * k * tstride];
        if (dir > 0) w.y = -w.y;
        v[q + r * Q] = cmul(v[q + r * Q], w);
      }
    }
    Dft<R, C>::run(v, q, Q, dir);
  }
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int j = t + q * T;
    const int k = j & (Ns - 1);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) sink(base + r * Ns, v[q + r * Q]);
  }
}

// Shared buffers hold element q of a sequence at s[sidx(q) * ss]: ss = 1 for
// one sequence per buffer (rows), ss = cw for cw interleaved columns, so that
// the lanes that read 32 contiguous bytes of cw columns from global memory
// also touch contiguous shared words.
template <int LOGN, int ST, typename C, typename Store>
PD void run_stages(C (&v)[16], int t, int Ns, C* s, int ss, const C* tw, int dir, Store store) {
  typedef Plan<LOGN> P;
  constexpr int R = P::radix(ST);
  if constexpr (ST + 1 == P::NST) {
    stage<R, P::N, P::T>(v, t, Ns, tw, dir, store);
  } else {
    stage<R, P::N, P::T>(v, t, Ns, tw, dir, [&](int q, C x) { s[sidx(q) * ss] = x; });
    __syncthreads();
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = s[sidx(t + m * P::T) * ss];
    __syncthreads();
    run_stages<LOGN, ST + 1>(v, t, Ns * R, s, ss, tw, dir, store);
  }
}

// All stages of one sequence: load(m) supplies input element t + m T,
// store(q, value) receives output q.
template <int LOGN, typename C, typename Load, typename Store>
PD void fft_seq(int t, C* s, int ss, const C* tw, int dir, Load load, Store store) {
  C v[16];
#pragma unroll
  for (int m = 0; m < 16; ++m) v[m] = load(m);
  run_stages<LOGN, 0>(v, t, 1, s, ss, tw, dir, store);
}

constexpr int kRowCta = 256;

inline int row_nseq(const Geometry& g) {
  int s = kRowCta / (g.K / 16);
  if (s < 1) s = 1;
  if (s > g.n) s = g.n;
  return s;
}
template <typename T> inline int col_width() { return 32 / int(sizeof(typename cplx_t<T>::type)); }
__host__ __device__ inline size_t padded(int N) { return size_t(N) + size_t(N) / 16 + 1; }

// ----------------------------------------------------------------- kernels
template <typename T, int LOGN> struct ColThreads {
  static constexpr int value = (32 / int(sizeof(typename cplx_t<T>::type))) * ((1 << LOGN) / 16);
};

template <typename T, int LOGN>
__global__ void __launch_bounds__(kRowCta) k_row_fwd(Geometry g, RowPro<T> pro, const T* __restrict__ deapod,
                                                  typename cplx_t<T>::type* __restrict__ A,
                                                  const typename cplx_t<T>::type* __restrict__ tw, int nseq) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int K = g.K, n = g.n, half = n / 2;
  const int seq = threadIdx.x / Plan<LOGN>::T, t = threadIdx.x - seq * Plan<LOGN>::T;
  const int i1 = blockIdx.x * nseq + seq;
  C* s = reinterpret_cast<C*>(sm_raw) + seq * padded(K);
  const T s1 = deapod[i1];
  const T beta = pro.mode == PRO_CG_P ? T(pro.scalars[pro.idx]) : T(0);
  const T scl = pro.mode == PRO_SCALE ? T(pro.scalars[pro.idx]) : T(1);
  auto load = [&](int m) -> C {
    const int q = t + m * Plan<LOGN>::T;            // grid column
    const int i2 = (q + half) & (K - 1);  // image column when q is a padded position
    if (i2 >= n) return cz<C>();
    const size_t idx = size_t(i1) * n + i2;
    T v;
    if (pro.mode == PRO_CG_P) {
      v = pro.r[idx] + beta * pro.p[idx];
      pro.p[idx] = v;
    } else {
      v = pro.x[idx] * scl;
    }
    return cmk<C>(v * s1 * deapod[i2], T(0));
  };
  C* out = A + size_t(i1) * K;
  auto store = [&](int q, C v) { out[q] = v; };
  fft_seq<LOGN>(t, s, 1, tw, -1, load, store);
}

template <typename T, int LOGN>
__global__ void __launch_bounds__(ColThreads<T, LOGN>::value, ColThreads<T, LOGN>::value <= 512 ? 2 : 1) k_col_fwd(Geometry g, const typename cplx_t<T>::type* __restrict__ A,
                                                  typename cplx_t<T>::type* __restrict__ Pg,
                                                  const typename cplx_t<T>::type* __restrict__ tw, int cw) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int K = g.K, n = g.n, half = n / 2, pl = g.pad_lo, KP = g.KP;
  const int cc = threadIdx.x % cw, t = threadIdx.x / cw;
  const int c = blockIdx.x * cw + cc;
  C* s = reinterpret_cast<C*>(sm_raw) + cc;  // cw interleaved columns
  auto load = [&](int m) -> C {
    const int q = t + m * Plan<LOGN>::T;  // grid row
    const int i1 = (q + half) & (K - 1);
    return i1 < n ? A[size_t(i1) * K + c] : cz<C>();
  };
  const int jhi = kJ - pl;  // grid indices < jhi repeat past the end
  int cols[2] = {c + pl, -1};
  if (c >= K - pl) cols[1] = c + pl - K;
  else if (c < jhi) cols[1] = c + pl + K;
  auto store = [&](int q, C v) {
    int rows[2] = {q + pl, -1};
    if (q >= K - pl) rows[1] = q + pl - K;
    else if (q < jhi) rows[1] = q + pl + K;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
        if (rows[a] >= 0 && cols[b] >= 0) Pg[size_t(rows[a]) * KP + cols[b]] = v;
  };
  fft_seq<LOGN>(t, s, cw, tw, -1, load, store);
}

template <typename T, int LOGN>
__global__ void __launch_bounds__(ColThreads<T, LOGN>::value, ColThreads<T, LOGN>::value <= 512 ? 2 : 1) k_col_inv(Geometry g, const typename cplx_t<T>::type* __restrict__ Q,
                                                  typename cplx_t<T>::type* __restrict__ A,
                                                  const typename cplx_t<T>::type* __restrict__ tw, int cw) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int K = g.K, n = g.n, half = n / 2, pl = g.pad_lo, KP = g.KP;
  const int cc = threadIdx.x % cw, t = threadIdx.x / cw;
  const int c = blockIdx.x * cw + cc;
  C* s = reinterpret_cast<C*>(sm_raw) + cc;  // cw interleaved columns
  const int jhi = kJ - pl;
  int cols[2] = {c + pl, -1};
  if (c >= K - pl) cols[1] = c + pl - K;
  else if (c < jhi) cols[1] = c + pl + K;
  auto load = [&](int m) -> C {
    const int q = t + m * Plan<LOGN>::T;
    int rows[2] = {q + pl, -1};
    if (q >= K - pl) rows[1] = q + pl - K;
    else if (q < jhi) rows[1] = q + pl + K;
    C v = cz<C>();
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
        if (rows[a] >= 0 && cols[b] >= 0) v = cadd(v, Q[size_t(rows[a]) * KP + cols[b]]);
    return v;
  };
  auto store = [&](int q, C v) {
    const int i1 = (q + half) & (K - 1);
    if (i1 < n) A[size_t(i1) * K + c] = v;
  };
  fft_seq<LOGN>(t, s, cw, tw, +1, load, store);
}

template <typename T, int LOGN>
__global__ void __launch_bounds__(kRowCta) k_row_inv(Geometry g, const typename cplx_t<T>::type* __restrict__ A,
                                                  const T* __restrict__ deapod, RowEp<T> ep,
                                                  const typename cplx_t<T>::type* __restrict__ tw, int nseq) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ double red[32];
  const int K = g.K, n = g.n, half = n / 2;
  const int seq = threadIdx.x / Plan<LOGN>::T, t = threadIdx.x - seq * Plan<LOGN>::T;
  const int i1 = blockIdx.x * nseq + seq;
  C* s = reinterpret_cast<C*>(sm_raw) + seq * padded(K);
  const C* in = A + size_t(i1) * K;
  auto load = [&](int m) -> C { return in[t + m * Plan<LOGN>::T]; };
  const T s1 = deapod[i1];
  double part = 0.0;
  auto store = [&](int q, C v) {
    const int i2 = (q + half) & (K - 1);
    if (i2 >= n) return;
    const size_t idx = size_t(i1) * n + i2;
    const T val = v.x * s1 * deapod[i2];
    switch (ep.mode) {
      case EP_CG_AP: {
        const T pv = ep.p[idx];
        const T o = T(ep.nu2) * val + T(2) * pv;
        ep.out[idx] = o;
        part += double(pv) * double(o);
      } break;
      case EP_CG_R0: {
        const T o = ep.b[idx] - (T(ep.nu2) * val + T(2) * ep.p[idx]);
        ep.out[idx] = o;
        ep.out2[idx] = o;
        part += double(o) * double(o);
      } break;
      case EP_POWER:
        ep.out[idx] = val;
        part += double(val) * double(val);
        break;
      case EP_XS_ADD:
        ep.out[idx] = ep.b[idx] + T(ep.nu) * val;
        break;
      case EP_QX:
        ep.out[idx] = T(ep.nu2) * val + T(2) * ep.p[idx];
        break;
      default:
        ep.out[idx] = val;
    }
  };
  fft_seq<LOGN>(t, s, 1, tw, +1, load, store);
  if (ep.partials) {
    part = warp_sum(part);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int k = 0; k < int((blockDim.x + 31) >> 5); ++k) tot += red[k];
      ep.partials[blockIdx.x] = tot;
    }
    if (ep.ticket && last_block_done(ep.ticket)) {
      const double sum = block_sum_array(ep.partials, int(gridDim.x), red);
      if (threadIdx.x == 0) {
        if (ep.mode == EP_CG_R0) {
          ep.scalars[0] = sum;  // <r, r>
        } else if (ep.mode == EP_CG_AP) {
          ep.scalars[1] = sum > 0.0 ? ep.scalars[0] / sum : 0.0;  // alpha = <r, r> / <p, Ap>
        }
      }
    }
  }
}

// Composite operator by convolution (Section 3: precompute Phi^H Phi).  One
// CTA takes cw columns of the n compact rows (after the row FFT): forward
// column FFT, multiply by the precomputed real spectrum of the PSF
// (layout [column block][row][cw]), inverse column FFT, and keep the n rows
// the crop retains -- the transform of the column never leaves the SM.
template <typename T, int LOGN>
__global__ void __launch_bounds__(ColThreads<T, LOGN>::value, ColThreads<T, LOGN>::value <= 512 ? 2 : 1)
    k_col_conv(Geometry g, typename cplx_t<T>::type* __restrict__ A, const T* __restrict__ khat,
               const typename cplx_t<T>::type* __restrict__ tw, int cw) {
  typedef typename cplx_t<T>::type C;
  constexpr int TT = Plan<LOGN>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int K = g.K, n = g.n, half = n / 2;
  const int cc = threadIdx.x % cw, t = threadIdx.x / cw;
  const int c = blockIdx.x * cw + cc;
  C* s = reinterpret_cast<C*>(sm_raw) + cc;  // cw interleaved columns
  auto load = [&](int m) -> C {
    const int q = t + m * TT;
    const int i1 = (q + half) & (K - 1);
    return i1 < n ? A[size_t(i1) * K + c] : cz<C>();
  };
  auto to_smem = [&](int q, C v) { s[sidx(q) * cw] = v; };
  fft_seq<LOGN>(t, s, cw, tw, -1, load, to_smem);
  __syncthreads();
  C v[16];
  const T* kc = khat + (size_t(blockIdx.x) * K) * cw + cc;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int q = t + m * TT;
    v[m] = cscale(s[sidx(q) * cw], kc[size_t(q) * cw]);
  }
  __syncthreads();
  auto store = [&](int q, C x) {
    const int i1 = (q + half) & (K - 1);
    if (i1 < n) A[size_t(i1) * K + c] = x;
  };
  run_stages<LOGN, 0>(v, t, 1, s, cw, tw, +1, store);
}

// Plain in-place transforms of a K x K complex array (set-up of the PSF spectrum).
template <typename T, int LOGN>
__global__ void __launch_bounds__(kRowCta) k_rows_plain(typename cplx_t<T>::type* __restrict__ X,
                                                        const typename cplx_t<T>::type* __restrict__ tw, int nseq,
                                                        int dir) {
  typedef typename cplx_t<T>::type C;
  constexpr int TT = Plan<LOGN>::T, K = Plan<LOGN>::N;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int seq = threadIdx.x / TT, t = threadIdx.x - seq * TT;
  C* row = X + size_t(blockIdx.x * nseq + seq) * K;
  C* s = reinterpret_cast<C*>(sm_raw) + seq * padded(K);
  auto load = [&](int m) -> C { return row[t + m * TT]; };
  C out[16];
  int qs[16];
  int cnt = 0;
  auto store = [&](int q, C v) { out[cnt] = v; qs[cnt] = q; ++cnt; };
  fft_seq<LOGN>(t, s, 1, tw, dir, load, store);
  __syncthreads();
#pragma unroll
  for (int m = 0; m < 16; ++m) row[qs[m]] = out[m];
}

template <typename T, int LOGN>
__global__ void __launch_bounds__(ColThreads<T, LOGN>::value) k_cols_plain(typename cplx_t<T>::type* __restrict__ X,
                                                                         const typename cplx_t<T>::type* __restrict__ tw,
                                                                         int cw, int dir) {
  typedef typename cplx_t<T>::type C;
  constexpr int TT = Plan<LOGN>::T, K = Plan<LOGN>::N;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int cc = threadIdx.x % cw, t = threadIdx.x / cw;
  const int c = blockIdx.x * cw + cc;
  C* s = reinterpret_cast<C*>(sm_raw) + cc;  // cw interleaved columns
  auto load = [&](int m) -> C { return X[size_t(t + m * TT) * K + c]; };
  C out[16];
  int qs[16];
  int cnt = 0;
  auto store = [&](int q, C v) { out[cnt] = v; qs[cnt] = q; ++cnt; };
  fft_seq<LOGN>(t, s, cw, tw, dir, load, store);
  __syncthreads();
#pragma unroll
  for (int m = 0; m < 16; ++m) X[size_t(qs[m]) * K + c] = out[m];
}

}  // namespace

int row_inv_blocks(const Geometry& g) { return g.n / row_nseq(g); }

#define PURIFY_LOGN_SWITCH(K, BODY)     \
  switch (K) {                          \
    case 32: { constexpr int L = 5; BODY; } break;   \
    case 64: { constexpr int L = 6; BODY; } break;   \
    case 128: { constexpr int L = 7; BODY; } break;  \
    case 256: { constexpr int L = 8; BODY; } break;  \
    case 512: { constexpr int L = 9; BODY; } break;  \
    case 1024: { constexpr int L = 10; BODY; } break; \
    case 2048: { constexpr int L = 11; BODY; } break; \
    default: { constexpr int L = 12; BODY; } break;  \
  }

template <typename T, int L> cudaError_t configure_one() {
  cudaError_t e = raise_smem_limit(k_row_fwd<T, L>);
  if (e == cudaSuccess) e = raise_smem_limit(k_row_inv<T, L>);
  if (e == cudaSuccess) e = raise_smem_limit(k_col_fwd<T, L>);
  if (e == cudaSuccess) e = raise_smem_limit(k_col_inv<T, L>);
  if (e == cudaSuccess) e = raise_smem_limit(k_col_conv<T, L>);
  if (e == cudaSuccess) e = raise_smem_limit(k_rows_plain<T, L>);
  if (e == cudaSuccess) e = raise_smem_limit(k_cols_plain<T, L>);
  return e;
}

template <typename T> cudaError_t configure_fft() {
  cudaError_t e = cudaSuccess;
  for (int K = 32; K <= 4096 && e == cudaSuccess; K *= 2) {
    PURIFY_LOGN_SWITCH(K, e = (configure_one<T, L>()));
  }
  return e;
}
template cudaError_t configure_fft<float>();
template cudaError_t configure_fft<double>();

template <typename T>
void launch_row_fwd(const Geometry& g, const RowPro<T>& pro, const T* deapod, typename cplx_t<T>::type* A,
                    const typename cplx_t<T>::type* tw, cudaStream_t s) {
  typedef typename cplx_t<T>::type C;
  const int nseq = row_nseq(g);
  const size_t sm = nseq * padded(g.K) * sizeof(C);
  PURIFY_LOGN_SWITCH(g.K, (k_row_fwd<T, L><<<g.n / nseq, nseq * Plan<L>::T, sm, s>>>(g, pro, deapod, A, tw, nseq)));
}

template <typename T>
void launch_col_fwd(const Geometry& g, const typename cplx_t<T>::type* A, typename cplx_t<T>::type* Pg,
                    const typename cplx_t<T>::type* tw, cudaStream_t s) {
  typedef typename cplx_t<T>::type C;
  const int cw = col_width<T>();
  const size_t sm = cw * padded(g.K) * sizeof(C);
  PURIFY_LOGN_SWITCH(g.K, (k_col_fwd<T, L><<<g.K / cw, cw * Plan<L>::T, sm, s>>>(g, A, Pg, tw, cw)));
}

template <typename T>
void launch_col_inv(const Geometry& g, const typename cplx_t<T>::type* Q, typename cplx_t<T>::type* A,
                    const typename cplx_t<T>::type* tw, cudaStream_t s) {
  typedef typename cplx_t<T>::type C;
  const int cw = col_width<T>();
  const size_t sm = cw * padded(g.K) * sizeof(C);
  PURIFY_LOGN_SWITCH(g.K, (k_col_inv<T, L><<<g.K / cw, cw * Plan<L>::T, sm, s>>>(g, Q, A, tw, cw)));
}

template <typename T>
int launch_row_inv(const Geometry& g, const typename cplx_t<T>::type* A, const T* deapod, const RowEp<T>& ep,
                   const typename cplx_t<T>::type* tw, cudaStream_t s) {
  typedef typename cplx_t<T>::type C;
  const int nseq = row_nseq(g);
  const size_t sm = nseq * padded(g.K) * sizeof(C);
  PURIFY_LOGN_SWITCH(g.K, (k_row_inv<T, L><<<g.n / nseq, nseq * Plan<L>::T, sm, s>>>(g, A, deapod, ep, tw, nseq)));
  return g.n / nseq;
}

template <typename T>
__global__ void k_embed_psf(const T* __restrict__ psf, int n, typename cplx_t<T>::type* __restrict__ X) {
  typedef typename cplx_t<T>::type C;
  const int K = 2 * n;
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= size_t(K) * K) return;
  const int q1 = int(idx / K), q2 = int(idx % K);
  // kernel offset d = q - K for q >= n; the PSF image holds offsets [-n, n)
  const int i1 = (q1 + n) & (K - 1), i2 = (q2 + n) & (K - 1);
  X[idx] = cmk<C>(psf[size_t(i1) * K + i2], T(0));
}

template <typename T>
__global__ void k_spectrum_layout(const typename cplx_t<T>::type* __restrict__ X, int K, int cw, double scale,
                                  T* __restrict__ khat) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= size_t(K) * K) return;
  const int q = int(idx / K), c = int(idx % K);
  khat[(size_t(c / cw) * K + q) * cw + (c % cw)] = T(double(X[idx].x) * scale);
}

template <typename T>
void build_psf_spectrum(const T* psf, int n, T* khat, typename cplx_t<T>::type* X, const typename cplx_t<T>::type* tw,
                        cudaStream_t s) {
  const int K = 2 * n;
  const size_t tot = size_t(K) * K;
  const int tb = 256;
  k_embed_psf<T><<<int((tot + tb - 1) / tb), tb, 0, s>>>(psf, n, X);
  launch_fft2_plain<T>(K, X, tw, -1, s);
  k_spectrum_layout<T><<<int((tot + tb - 1) / tb), tb, 0, s>>>(X, K, col_width<T>(), 1.0 / (double(K) * K), khat);
}

template <typename T>
void launch_col_conv(const Geometry& g, typename cplx_t<T>::type* A, const T* khat,
                     const typename cplx_t<T>::type* tw, cudaStream_t s) {
  typedef typename cplx_t<T>::type C;
  const int cw = col_width<T>();
  const size_t sm = cw * padded(g.K) * sizeof(C);
  PURIFY_LOGN_SWITCH(g.K, (k_col_conv<T, L><<<g.K / cw, cw * Plan<L>::T, sm, s>>>(g, A, khat, tw, cw)));
}

template <typename T>
void launch_fft2_plain(int K, typename cplx_t<T>::type* X, const typename cplx_t<T>::type* tw, int dir,
                       cudaStream_t s) {
  typedef typename cplx_t<T>::type C;
  const int cw = col_width<T>();
  int nseq = kRowCta / (K / 16);
  if (nseq < 1) nseq = 1;
  if (nseq > K) nseq = K;
  const size_t smr = nseq * padded(K) * sizeof(C);
  const size_t smc = cw * padded(K) * sizeof(C);
  PURIFY_LOGN_SWITCH(K, (k_rows_plain<T, L><<<K / nseq, nseq * Plan<L>::T, smr, s>>>(X, tw, nseq, dir)));
  PURIFY_LOGN_SWITCH(K, (k_cols_plain<T, L><<<K / cw, cw * Plan<L>::T, smc, s>>>(X, tw, cw, dir)));
}

#define INST(T)                                                                                              \
  template void launch_row_fwd<T>(const Geometry&, const RowPro<T>&, const T*, cplx_t<T>::type*,                \
                                  const cplx_t<T>::type*, cudaStream_t);                                        \
  template void launch_col_fwd<T>(const Geometry&, const cplx_t<T>::type*, cplx_t<T>::type*,                   \
                                  const cplx_t<T>::type*, cudaStream_t);                                        \
  template void launch_col_inv<T>(const Geometry&, const cplx_t<T>::type*, cplx_t<T>::type*,                   \
                                  const cplx_t<T>::type*, cudaStream_t);                                        \
  template int launch_row_inv<T>(const Geometry&, const cplx_t<T>::type*, const T*, const RowEp<T>&,            \
                                 const cplx_t<T>::type*, cudaStream_t);                                        \
  template void launch_col_conv<T>(const Geometry&, cplx_t<T>::type*, const T*, const cplx_t<T>::type*,         \
                                   cudaStream_t);                                                              \
  template void launch_fft2_plain<T>(int, cplx_t<T>::type*, const cplx_t<T>::type*, int, cudaStream_t);     \
  template void build_psf_spectrum<T>(const T*, int, T*, cplx_t<T>::type*, const cplx_t<T>::type*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace purify
