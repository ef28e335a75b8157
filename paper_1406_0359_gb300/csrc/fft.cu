// Oversampled 2D FFT passes of the NUFFT (operator F of Phi = G F Z S, Section 4)
// as shared-memory Stockham transforms: one radix-8 stage when log2 K is odd,
// then radix-4 stages, each butterfly held in registers between two barriers.
//
// Forward (Phi):   row pass over the n non-zero image rows, fused with the
//                  deapodisation S and zero-padding Z; column pass over all K
//                  columns, writing the padded grid (periodic J-wide halo) that
//                  the degridding kernels stage by TMA.
// Adjoint (Phi^H): column pass reading the padded gridding accumulator and
//                  folding its halo back onto the torus, keeping only the n rows
//                  the crop Z^T retains; row pass fused with the crop, the
//                  deapodisation and the solver epilogues.
#include "internal.h"

namespace purify {

namespace {

template <typename C> PD void dft4(C (&a)[4], int dir) {
  // X_k = sum_r a_r exp(dir * 2 pi i r k / 4), dir = -1 forward, +1 inverse
  const C s02 = cadd(a[0], a[2]), d02 = csub(a[0], a[2]);
  const C s13 = cadd(a[1], a[3]), d13 = csub(a[1], a[3]);
  C j13 = cmul_i(d13);
  if (dir < 0) { j13.x = -j13.x; j13.y = -j13.y; }
  a[0] = cadd(s02, s13);
  a[2] = csub(s02, s13);
  a[1] = cadd(d02, j13);
  a[3] = csub(d02, j13);
}

template <typename C> PD void dft8(C (&a)[8], int dir) {
  typedef decltype(a[0].x) T;
  C e[4] = {a[0], a[2], a[4], a[6]};
  C o[4] = {a[1], a[3], a[5], a[7]};
  dft4(e, dir);
  dft4(o, dir);
  const T h = T(0.70710678118654752440084436210485);
  const T sg = dir < 0 ? T(-1) : T(1);
  C w1 = cmk<C>(h, sg * h), w3 = cmk<C>(-h, sg * h);
  C t1 = cmul(o[1], w1);
  C t2 = cmul_i(o[2]);
  if (dir < 0) { t2.x = -t2.x; t2.y = -t2.y; }
  C t3 = cmul(o[3], w3);
  a[0] = cadd(e[0], o[0]);
  a[4] = csub(e[0], o[0]);
  a[1] = cadd(e[1], t1);
  a[5] = csub(e[1], t1);
  a[2] = cadd(e[2], t2);
  a[6] = csub(e[2], t2);
  a[3] = cadd(e[3], t3);
  a[7] = csub(e[3], t3);
}

template <int R, typename C> PD void dftR(C (&a)[R], int dir);
template <> PD void dftR<4, float2>(float2 (&a)[4], int dir) { dft4(a, dir); }
template <> PD void dftR<4, double2>(double2 (&a)[4], int dir) { dft4(a, dir); }
template <> PD void dftR<8, float2>(float2 (&a)[8], int dir) { dft8(a, dir); }
template <> PD void dftR<8, double2>(double2 (&a)[8], int dir) { dft8(a, dir); }

// One Stockham radix-R stage over nseq sequences of length N (pitch apart),
// sub-transform length Ns.  Every thread holds at most MAXB butterflies.
template <int R, int MAXB, typename C>
__device__ void fft_stage(C* s, int N, int Ns, int nseq, int pitch, const C* __restrict__ tw, int dir) {
  const int nbs = N / R;
  const int nb = nseq * nbs;
  const int tstride = N / (Ns * R);
  C a[MAXB][R];
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    const int j = threadIdx.x + b * blockDim.x;
    if (j < nb) {
      const int seq = j / nbs, jj = j - seq * nbs;
      const int k = jj & (Ns - 1);
      const C* src = s + seq * pitch + jj;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        C v = src[r * nbs];
        if (r > 0 && k > 0) {
          C t = tw[r * k * tstride];
          if (dir > 0) t.y = -t.y;
          v = cmul(v, t);
        }
        a[b][r] = v;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    const int j = threadIdx.x + b * blockDim.x;
    if (j < nb) {
      const int seq = j / nbs, jj = j - seq * nbs;
      const int k = jj & (Ns - 1);
      dftR<R>(a[b], dir);
      C* dst = s + seq * pitch + (jj - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * Ns] = a[b][r];
    }
  }
  __syncthreads();
}

constexpr int kMaxB = 8;

template <typename C>
__device__ void fft_smem(C* s, int N, int logN, int nseq, int pitch, const C* __restrict__ tw, int dir) {
  int Ns = 1;
  if (logN & 1) {
    fft_stage<8, kMaxB / 2>(s, N, 1, nseq, pitch, tw, dir);
    Ns = 8;
  }
  while (Ns < N) {
    fft_stage<4, kMaxB>(s, N, Ns, nseq, pitch, tw, dir);
    Ns *= 4;
  }
}

constexpr int kRowThreads = 128;

inline int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}
inline int row_nseq(const Geometry& g) {
  int s = 512 / g.K;
  if (s < 1) s = 1;
  if (s > 4) s = 4;
  return s;
}
template <typename T> inline int col_width() { return 32 / int(sizeof(typename cplx_t<T>::type)); }
inline int col_threads(int cw, int K) {
  int t = cw * K / 4 / kMaxB;
  if (t < 128) t = 128;
  if (t > 1024) t = 1024;
  return t;
}

// ----------------------------------------------------------------- kernels
template <typename T>
__global__ void __launch_bounds__(kRowThreads) k_row_fwd(Geometry g, RowPro<T> pro, const T* __restrict__ deapod,
                                                          typename cplx_t<T>::type* __restrict__ A,
                                                          const typename cplx_t<T>::type* __restrict__ tw, int nseq,
                                                          int logK) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* s = reinterpret_cast<C*>(sm_raw);
  const int K = g.K, n = g.n, half = n / 2;
  const int row0 = blockIdx.x * nseq;
  for (int e = threadIdx.x; e < nseq * K; e += blockDim.x) s[e] = cz<C>();
  __syncthreads();
  for (int e = threadIdx.x; e < nseq * n; e += blockDim.x) {
    const int r = e / n, i2 = e - r * n, i1 = row0 + r;
    const size_t idx = size_t(i1) * n + i2;
    T v;
    if (pro.mode == PRO_CG_P) {
      const T beta = T(pro.scalars[pro.idx]);
      v = pro.r[idx] + beta * pro.p[idx];
      pro.p[idx] = v;
    } else if (pro.mode == PRO_SCALE) {
      v = pro.x[idx] * T(pro.scalars[pro.idx]);
    } else {
      v = pro.x[idx];
    }
    const int q2 = (i2 - half) & (K - 1);
    s[r * K + q2] = cmk<C>(v * deapod[i1] * deapod[i2], T(0));
  }
  __syncthreads();
  fft_smem(s, K, logK, nseq, K, tw, -1);
  for (int e = threadIdx.x; e < nseq * K; e += blockDim.x) A[size_t(row0) * K + e] = s[e];
}

template <typename T>
__global__ void k_col_fwd(Geometry g, const typename cplx_t<T>::type* __restrict__ A,
                          typename cplx_t<T>::type* __restrict__ P, const typename cplx_t<T>::type* __restrict__ tw,
                          int cw, int logK) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* s = reinterpret_cast<C*>(sm_raw);
  const int K = g.K, n = g.n, half = n / 2, pl = g.pad_lo, KP = g.KP;
  const int pitch = K + 1;
  const int c0 = blockIdx.x * cw;
  for (int e = threadIdx.x; e < cw * pitch; e += blockDim.x) s[e] = cz<C>();
  __syncthreads();
  for (int e = threadIdx.x; e < n * cw; e += blockDim.x) {
    const int i1 = e / cw, cc = e - i1 * cw;
    const int q1 = (i1 - half) & (K - 1);
    s[cc * pitch + q1] = A[size_t(i1) * K + c0 + cc];
  }
  __syncthreads();
  fft_smem(s, K, logK, cw, pitch, tw, -1);
  const int jhi = kJ - pl;  // grid indices < jhi are repeated past the end
  for (int e = threadIdx.x; e < K * cw; e += blockDim.x) {
    const int q = e / cw, cc = e - q * cw, c = c0 + cc;
    const C v = s[cc * pitch + q];
    int rows[2] = {q + pl, -1}, cols[2] = {c + pl, -1};
    if (q >= K - pl) rows[1] = q + pl - K;
    else if (q < jhi) rows[1] = q + pl + K;
    if (c >= K - pl) cols[1] = c + pl - K;
    else if (c < jhi) cols[1] = c + pl + K;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
        if (rows[a] >= 0 && cols[b] >= 0) P[size_t(rows[a]) * KP + cols[b]] = v;
  }
}

template <typename T>
__global__ void k_col_inv(Geometry g, const typename cplx_t<T>::type* __restrict__ Q,
                          typename cplx_t<T>::type* __restrict__ A, const typename cplx_t<T>::type* __restrict__ tw,
                          int cw, int logK) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C* s = reinterpret_cast<C*>(sm_raw);
  const int K = g.K, n = g.n, half = n / 2, pl = g.pad_lo, KP = g.KP;
  const int pitch = K + 1;
  const int c0 = blockIdx.x * cw;
  const int jhi = kJ - pl;
  for (int e = threadIdx.x; e < K * cw; e += blockDim.x) {
    const int q = e / cw, cc = e - q * cw, c = c0 + cc;
    int rows[2] = {q + pl, -1}, cols[2] = {c + pl, -1};
    if (q >= K - pl) rows[1] = q + pl - K;
    else if (q < jhi) rows[1] = q + pl + K;
    if (c >= K - pl) cols[1] = c + pl - K;
    else if (c < jhi) cols[1] = c + pl + K;
    C v = cz<C>();
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
        if (rows[a] >= 0 && cols[b] >= 0) v = cadd(v, Q[size_t(rows[a]) * KP + cols[b]]);
    s[cc * pitch + q] = v;
  }
  __syncthreads();
  fft_smem(s, K, logK, cw, pitch, tw, +1);
  for (int e = threadIdx.x; e < n * cw; e += blockDim.x) {
    const int i1 = e / cw, cc = e - i1 * cw;
    const int q1 = (i1 - half) & (K - 1);
    A[size_t(i1) * K + c0 + cc] = s[cc * pitch + q1];
  }
}

template <typename T>
__global__ void __launch_bounds__(kRowThreads) k_row_inv(Geometry g, const typename cplx_t<T>::type* __restrict__ A,
                                                          const T* __restrict__ deapod, RowEp<T> ep,
                                                          const typename cplx_t<T>::type* __restrict__ tw, int nseq,
                                                          int logK) {
  typedef typename cplx_t<T>::type C;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ double red[32];
  C* s = reinterpret_cast<C*>(sm_raw);
  const int K = g.K, n = g.n, half = n / 2;
  const int row0 = blockIdx.x * nseq;
  for (int e = threadIdx.x; e < nseq * K; e += blockDim.x) s[e] = A[size_t(row0) * K + e];
  __syncthreads();
  fft_smem(s, K, logK, nseq, K, tw, +1);
  double part = 0.0;
  for (int e = threadIdx.x; e < nseq * n; e += blockDim.x) {
    const int r = e / n, i2 = e - r * n, i1 = row0 + r;
    const size_t idx = size_t(i1) * n + i2;
    const int q2 = (i2 - half) & (K - 1);
    const T val = s[r * K + q2].x * deapod[i1] * deapod[i2];
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
  }
  if (ep.partials) {
    const double t = block_sum<kRowThreads>(part, red);
    if (threadIdx.x == 0) ep.partials[blockIdx.x] = t;
  }
}

}  // namespace

int row_inv_blocks(const Geometry& g) { return g.n / row_nseq(g); }

template <typename T> cudaError_t configure_fft() {
  const int mx = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(k_row_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_row_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_fwd<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_col_inv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return e;
}
template cudaError_t configure_fft<float>();
template cudaError_t configure_fft<double>();

template <typename T>
void launch_row_fwd(const Geometry& g, const RowPro<T>& pro, const T* deapod, typename cplx_t<T>::type* A,
                    const typename cplx_t<T>::type* tw, cudaStream_t s) {
  typedef typename cplx_t<T>::type C;
  const int nseq = row_nseq(g);
  const size_t sm = size_t(nseq) * g.K * sizeof(C);
  k_row_fwd<T><<<g.n / nseq, kRowThreads, sm, s>>>(g, pro, deapod, A, tw, nseq, ilog2(g.K));
}

template <typename T>
void launch_col_fwd(const Geometry& g, const typename cplx_t<T>::type* A, typename cplx_t<T>::type* P,
                    const typename cplx_t<T>::type* tw, cudaStream_t s) {
  typedef typename cplx_t<T>::type C;
  const int cw = col_width<T>();
  const size_t sm = size_t(cw) * (g.K + 1) * sizeof(C);
  k_col_fwd<T><<<g.K / cw, col_threads(cw, g.K), sm, s>>>(g, A, P, tw, cw, ilog2(g.K));
}

template <typename T>
void launch_col_inv(const Geometry& g, const typename cplx_t<T>::type* Q, typename cplx_t<T>::type* A,
                    const typename cplx_t<T>::type* tw, cudaStream_t s) {
  typedef typename cplx_t<T>::type C;
  const int cw = col_width<T>();
  const size_t sm = size_t(cw) * (g.K + 1) * sizeof(C);
  k_col_inv<T><<<g.K / cw, col_threads(cw, g.K), sm, s>>>(g, Q, A, tw, cw, ilog2(g.K));
}

template <typename T>
int launch_row_inv(const Geometry& g, const typename cplx_t<T>::type* A, const T* deapod, const RowEp<T>& ep,
                   const typename cplx_t<T>::type* tw, cudaStream_t s) {
  typedef typename cplx_t<T>::type C;
  const int nseq = row_nseq(g);
  const size_t sm = size_t(nseq) * g.K * sizeof(C);
  k_row_inv<T><<<g.n / nseq, kRowThreads, sm, s>>>(g, A, deapod, ep, tw, nseq, ilog2(g.K));
  return g.n / nseq;
}

#define INST(T)                                                                                              \
  template void launch_row_fwd<T>(const Geometry&, const RowPro<T>&, const T*, cplx_t<T>::type*,                \
                                  const cplx_t<T>::type*, cudaStream_t);                                        \
  template void launch_col_fwd<T>(const Geometry&, const cplx_t<T>::type*, cplx_t<T>::type*,                   \
                                  const cplx_t<T>::type*, cudaStream_t);                                        \
  template void launch_col_inv<T>(const Geometry&, const cplx_t<T>::type*, cplx_t<T>::type*,                   \
                                  const cplx_t<T>::type*, cudaStream_t);                                        \
  template int launch_row_inv<T>(const Geometry&, const cplx_t<T>::type*, const T*, const RowEp<T>&,            \
                                 const cplx_t<T>::type*, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace purify
