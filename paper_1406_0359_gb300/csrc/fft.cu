// Oversampled 2D FFT passes of the NUFFT (operator F of Phi = G F Z S, Section 4).
//
// Each length-K transform (K = 2n, a power of two) is a Stockham sequence of
// register radix-E stages (E = 8 or 16; one smaller stage last when log2 K
// is not a multiple of log2 E).  A thread always holds the E elements
// t + m K/E of its sequence: the first stage reads them straight from global
// memory, the last writes its outputs straight to global memory, and the
// stages in between exchange through shared memory (padded every 16
// elements against bank conflicts).
//
// The image is real, so every pass works in real form: two image rows a, b
// travel as one complex row x_a + i x_b, and only the half spectra (columns
// 0..K/2 of the row transforms) are kept, n x K/2 complex values.
// Forward (Phi):   row pass over the n non-zero image rows (pairs), fused with
//                  the deapodisation S and zero-padding Z; column pass over
//                  the K/2 half-spectrum columns, writing each grid column
//                  and its conjugate mirror into the padded grid (with its
//                  periodic J-wide halo) that degridding stages by TMA.
// Adjoint (Phi^H): column pass reading the padded gridding accumulator,
//                  folding its halo back onto the torus and taking its
//                  Hermitian part (Re of the image is all Phi^H keeps),
//                  writing only the n rows the crop Z^T keeps; row pass
//                  fused with the crop, the deapodisation and the solver
//                  epilogues.
#include "internal.h"
#include "solver_kernels.h"

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

// Compile-time plan of a length-2^LOGN transform with E (8 or 16) elements
// per thread: radix-E stages, then one radix-2^r stage for the remaining r
// bits; T = N/E threads per sequence.
template <int LOGN, int E = 16> struct Plan {
  static_assert(E == 8 || E == 16, "8 or 16 elements per thread");
  static constexpr int LE = E == 16 ? 4 : 3;
  static constexpr int N = 1 << LOGN;
  static constexpr int T = N / E;
  static constexpr int NST = (LOGN + LE - 1) / LE;
  __host__ __device__ static constexpr int radix(int st) {
    return st + 1 < NST ? E : (1 << (LOGN - LE * (NST - 1)));
  }
};

// One Stockham stage on the registers: v[m] holds element t + m T of the
// stage input.  Thread t owns butterflies j = t + q T (q < E/R); input r of
// butterfly j is element j + r N/R, i.e. register q + r E/R.  After the
// twiddles and the DFT, register q + r E/R is output (j - k) R + k + r Ns
// with k = j mod Ns; sink(position, value) receives every output.
template <int R, int N, int T, int E, typename C, typename Sink>
PD void stage(C (&v)[E], int t, int Ns, const C* __restrict__ tw, int dir, Sink sink) {
  constexpr int Q = E / R;
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
template <int LOGN, int ST, int E, typename C, typename Store>
PD void run_stages(C (&v)[E], int t, int Ns, C* s, int ss, const C* tw, int dir, Store store) {
  typedef Plan<LOGN, E> P;
  constexpr int R = P::radix(ST);
  if constexpr (ST + 1 == P::NST) {
    stage<R, P::N, P::T, E>(v, t, Ns, tw, dir, store);
  } else {
    stage<R, P::N, P::T, E>(v, t, Ns, tw, dir, [&](int q, C x) { s[sidx(q) * ss] = x; });
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) v[m] = s[sidx(t + m * P::T) * ss];
    __syncthreads();
    run_stages<LOGN, ST + 1, E>(v, t, Ns * R, s, ss, tw, dir, store);
  }
}

// All stages of one sequence: load(m) supplies input element t + m T,
// store(q, value) receives output q.
template <int LOGN, int E = 16, typename C, typename Load, typename Store>
PD void fft_seq(int t, C* s, int ss, const C* tw, int dir, Load load, Store store) {
  C v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = load(m);
  run_stages<LOGN, 0, E>(v, t, 1, s, ss, tw, dir, store);
}

// Output position of the cnt-th value a thread's final stage hands to its
// sink: the final radix-R stage has Ns = K/R and butterflies j = t + q T < Ns,
// so its outputs come in the order (q, r) at t + q T + r K/R.
template <int LOGN, int E = 16> PD int last_pos(int t, int cnt) {
  typedef Plan<LOGN, E> P;
  constexpr int R = P::radix(P::NST - 1);
  return t + (cnt / R) * P::T + (cnt % R) * (P::N / R);
}

constexpr int kRowCta = 256;
constexpr int kRowE = 8;  // elements per thread in the real-form row passes
// ... unless a row of K / 8 threads would not fit one CTA (K = 4096): 16 there.
template <int LOGN> constexpr int row_e() { return (1 << LOGN) / kRowE <= kRowCta ? kRowE : 16; }
inline int row_e_host(int K) { return K / kRowE <= kRowCta ? kRowE : 16; }

// Column passes read kColBytes contiguous bytes of each row: col_width
// interleaved columns per CTA.
constexpr int kColBytes = 32;
template <typename T> inline int col_width() { return kColBytes / int(sizeof(typename cplx_t<T>::type)); }
__host__ __device__ inline size_t padded(int N) { return size_t(N) + size_t(N) / 16 + 1; }

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Row-pass epilogues (see RowEpMode): per output, its operands (EpOpd, from
// the rows staged in shared memory) and the stores and partial sums of the
// mode.
template <typename T> struct EpOpd { T a, b; };
template <typename T> struct EpAcc { Acc<T> a[5]; };
template <int MODE, typename T>
PD void row_ep_store(const RowEp<T>& ep, size_t idx, T val, EpOpd<T> opd, EpAcc<T>& part) {
  if constexpr (MODE == EP_CG_AP) {
    // A thread's 16 terms are summed by plain FMAs (their rounding errors are
    // independent across the ~10^5 threads and average out); the per-thread
    // sums are then merged compensated.
    const T o = T(ep.nu2) * val + T(2) * opd.a;  // (A p)_i
    ep.out[idx] = o;
    part.a[0].s = fma(opd.a, o, part.a[0].s);
    part.a[1].s = fma(opd.b, o, part.a[1].s);
    part.a[2].s = fma(o, o, part.a[2].s);
    part.a[3].s = fma(opd.b, opd.a, part.a[3].s);
    part.a[4].s = fma(opd.b, opd.b, part.a[4].s);
  } else if constexpr (MODE == EP_CG_R0) {
    const T o = opd.a - T(ep.nu2) * val;
    ep.out[idx] = o;
    ep.out2[idx] = o;
    part.a[0].add_prod(o, o);
  } else if constexpr (MODE == EP_POWER) {
    ep.out[idx] = val;
    part.a[0].add_prod(val, val);
  } else if constexpr (MODE == EP_XS_ADD) {
    ep.out[idx] = opd.a + T(ep.nu) * val;
  } else if constexpr (MODE == EP_QX) {
    ep.out[idx] = T(ep.nu2) * val + T(2) * opd.a;
  } else {
    ep.out[idx] = val;
  }
}
// Image column of the m-th output of thread t of an inverse row pass (grid
// column q maps to image column (q + K/4) mod K, kept when < n = K/2).
template <int LOGN, int E = 16> PD int ep_col(int t, int m) {
  constexpr int K = 1 << LOGN;
  return (last_pos<LOGN, E>(t, m) + K / 4) & (K - 1);
}

// Register slot m of the j-th of the E/2 grid columns of a thread that hold
// image pixels: with K = 2n, grid column q = t + m K/E holds image column
// i2 = (q + K/4) mod K, inside the image for m < E/4 and m >= 3E/4 only.
template <int E> PD constexpr int kept_slot(int j) { return j < E / 4 ? j : j + E / 2; }

// Forward row prologue (see RowProMode) of image rows row0[r] at the E/2
// kept grid columns of thread t.  All loads precede the CG step's stores.
template <int LOGN, int NR, int E, typename T>
PD void row_prologue(const RowPro<T>& pro, const size_t (&row0)[NR], int t, T (&val)[NR][E / 2], int (&i2)[E / 2]) {
  constexpr int K = 1 << LOGN, TT = K / E;
#pragma unroll
  for (int j = 0; j < E / 2; ++j) i2[j] = (t + kept_slot<E>(j) * TT + K / 4) & (K - 1);
  if (pro.mode == PRO_CG_STEP) {
    // x += alpha p, r -= alpha Ap, p = r + beta p (alpha, beta of the previous step)
    const T alpha = T(pro.scalars[S_ALPHA]), beta = T(pro.scalars[S_BETA]);
    T xv[NR][E / 2], rv[NR][E / 2], av[NR][E / 2];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < E / 2; ++j) {
        const size_t idx = row0[r] + i2[j];
        xv[r][j] = pro.xu[idx];
        rv[r][j] = pro.r[idx];
        val[r][j] = pro.p[idx];
        av[r][j] = pro.ap[idx];
      }
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < E / 2; ++j) {
        const size_t idx = row0[r] + i2[j];
        const T pv = val[r][j];
        const T rn = fma(-alpha, av[r][j], rv[r][j]);
        pro.xu[idx] = fma(alpha, pv, xv[r][j]);
        pro.r[idx] = rn;
        val[r][j] = fma(beta, pv, rn);
        pro.p[idx] = val[r][j];
      }
  } else if (pro.mode == PRO_CG_START) {
    // r = b - A x_hat, p = r (b in pro.x, A x_hat in pro.ap)
    T bv[NR][E / 2], av[NR][E / 2];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < E / 2; ++j) {
        const size_t idx = row0[r] + i2[j];
        bv[r][j] = pro.x[idx];
        av[r][j] = pro.ap[idx];
      }
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < E / 2; ++j) {
        const size_t idx = row0[r] + i2[j];
        val[r][j] = bv[r][j] - av[r][j];
        pro.r[idx] = val[r][j];
        pro.p[idx] = val[r][j];
      }
  } else {
    const T scl = pro.mode == PRO_SCALE ? T(pro.scalars[pro.idx]) : T(1);
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < E / 2; ++j) val[r][j] = pro.x[row0[r] + i2[j]] * scl;
  }
}

// Per-CTA partials of the epilogue sums (ep.partials + k * ep.pstride for the
// k-th sum); the last CTA finalises the CG scalars in FP64:
//   EP_CG_R0: <r, r>.
//   EP_CG_AP: from <p,Ap>, <r,Ap>, <Ap,Ap>, <r,p> and <r,r> of this step's
//             vectors: the exact line search alpha = <r,p> / <p,Ap> (equal to
//             <r,r> / <p,Ap> in exact arithmetic); the next residual norm by
//             ||r - alpha Ap||^2 = <r,r> - 2 alpha <r,Ap> + alpha^2 <Ap,Ap>
//             (clamped at 0); beta = ||r_new||^2 / <r,r>.
template <typename T>
PD void row_ep_finish(const RowEp<T>& ep, EpAcc<T> part, double* red /*[5*32]*/, int bid, int nblocks) {
  if (!ep.partials) return;
  const int nsum = ep.mode == EP_CG_AP ? 5 : 1;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = int((blockDim.x + 31) >> 5);
  Acc<T>* st = reinterpret_cast<Acc<T>*>(red);
  Acc<T>* P = reinterpret_cast<Acc<T>*>(ep.partials);
  for (int k = 0; k < nsum; ++k) {
    warp_merge(part.a[k]);
    if (lane == 0) st[k * 32 + w] = part.a[k];
  }
  __syncthreads();
  // CG step: the CTA's five sums go straight into FP64 accumulators (atomic
  // adds as the CTAs finish), so that the last CTA only reads five values
  const bool acc64 = ep.mode == EP_CG_AP && ep.ticket;
  if (w == 0) {
    for (int k = 0; k < nsum; ++k) {
      Acc<T> b = lane < nw ? st[k * 32 + lane] : Acc<T>();
      warp_merge(b);
      if (lane == 0) {
        if (acc64) atomicAdd(ep.scalars + S_CG0 + k, b.value());
        else P[size_t(k) * ep.pstride + bid] = b;
      }
    }
  }
  if (!ep.ticket || !last_block_done_t0(ep.ticket, unsigned(nblocks))) return;
  if (acc64) {
    if (threadIdx.x != 0) return;
    double sum[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      sum[k] = __ldcg(ep.scalars + S_CG0 + k);
      ep.scalars[S_CG0 + k] = 0.0;  // ready for the next step
    }
    double* sc = ep.scalars;
    const double rr = sum[4];
    const double alpha = sum[0] > 0.0 ? sum[3] / sum[0] : 0.0;
    double rr_new = rr - 2.0 * alpha * sum[1] + alpha * alpha * sum[2];
    if (rr_new < 0.0) rr_new = 0.0;
    sc[S_PAP] = sum[0];
    sc[S_ALPHA] = alpha;
    sc[S_BETA] = rr > 0.0 ? rr_new / rr : 0.0;
    sc[S_RR] = rr_new;
    return;
  }
  // last block: merge all blocks' partials (fixed order), FP64 only at the end
  EpAcc<T> tot;
  int i = threadIdx.x;
  for (; i + int(blockDim.x) < nblocks; i += 2 * blockDim.x) {  // two CTAs' partials in flight
    Acc<T> v[2][5];
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (k < nsum) {
        v[0][k] = P[size_t(k) * ep.pstride + i];
        v[1][k] = P[size_t(k) * ep.pstride + i + blockDim.x];
      }
#pragma unroll
    for (int k = 0; k < 5; ++k)
      if (k < nsum) {
        acc_merge(tot.a[k], v[0][k]);
        acc_merge(tot.a[k], v[1][k]);
      }
  }
  for (; i < nblocks; i += blockDim.x)
    for (int k = 0; k < nsum; ++k) acc_merge(tot.a[k], P[size_t(k) * ep.pstride + i]);
  for (int k = 0; k < nsum; ++k) {
    warp_merge(tot.a[k]);
    if (lane == 0) st[k * 32 + w] = tot.a[k];
  }
  __syncthreads();
  if (w != 0) return;
  double sum[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (int k = 0; k < nsum; ++k) {
    Acc<T> b = lane < nw ? st[k * 32 + lane] : Acc<T>();
    warp_merge(b);
    sum[k] = b.value();
  }
  if (lane != 0) return;
  double* sc = ep.scalars;
  if (ep.mode == EP_CG_R0) {
    sc[S_RR] = sum[0];
  } else if (ep.mode == EP_CG_AP) {
    const double rr = sum[4];
    const double alpha = sum[0] > 0.0 ? sum[3] / sum[0] : 0.0;
    double rr_new = rr - 2.0 * alpha * sum[1] + alpha * alpha * sum[2];
    if (rr_new < 0.0) rr_new = 0.0;
    sc[S_PAP] = sum[0];
    sc[S_ALPHA] = alpha;
    sc[S_BETA] = rr > 0.0 ? rr_new / rr : 0.0;
    sc[S_RR] = rr_new;
  }
}

// Operand arrays an epilogue reads (staged in shared memory by the real-form
// inverse row pass): CG_AP p, r; CG_R0 b, p; QX p; XS_ADD b.
template <typename T> PD int ep_staged(const RowEp<T>& ep, const T** src) {
  switch (ep.mode) {
    case EP_CG_AP: src[0] = ep.p; src[1] = ep.r; return 2;
    case EP_CG_R0: src[0] = ep.b; src[1] = ep.p; return 2;
    case EP_QX: src[0] = ep.p; return 1;
    case EP_XS_ADD: src[0] = ep.b; return 1;
    default: return 0;
  }
}
// Epilogue of both rows of a real-form sequence with the operands in shared
// memory (ops[k][row][n]).
template <int LOGN, int MODE, int E, typename T>
PD EpAcc<T> row_ep_staged_mode(const RowEp<T>& ep, const T (&val)[2][E], int t, const size_t (&row0)[2],
                               const T* ops) {
  constexpr int n = (1 << LOGN) / 2;
  EpAcc<T> part;
#pragma unroll
  for (int m = 0; m < E; ++m) {
    const int i2 = ep_col<LOGN, E>(t, m);
    if (i2 < n) {
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const T o0 = ops[r * n + i2], o1 = ops[(2 + r) * n + i2];
        EpOpd<T> opd{T(0), T(0)};
        if constexpr (MODE == EP_CG_AP) opd = EpOpd<T>{o0, o1};
        else if constexpr (MODE == EP_CG_R0) opd.a = o0 - T(2) * o1;
        else if constexpr (MODE == EP_QX || MODE == EP_XS_ADD) opd.a = o0;
        row_ep_store<MODE>(ep, row0[r] + i2, val[r][m], opd, part);
      }
    }
  }
  return part;
}
template <int LOGN, int E, typename T>
PD EpAcc<T> row_ep_staged(const RowEp<T>& ep, const T (&val)[2][E], int t, const size_t (&row0)[2], const T* ops) {
  switch (ep.mode) {
    case EP_CG_AP: return row_ep_staged_mode<LOGN, EP_CG_AP>(ep, val, t, row0, ops);
    case EP_CG_R0: return row_ep_staged_mode<LOGN, EP_CG_R0>(ep, val, t, row0, ops);
    case EP_POWER: return row_ep_staged_mode<LOGN, EP_POWER>(ep, val, t, row0, ops);
    case EP_XS_ADD: return row_ep_staged_mode<LOGN, EP_XS_ADD>(ep, val, t, row0, ops);
    case EP_QX: return row_ep_staged_mode<LOGN, EP_QX>(ep, val, t, row0, ops);
    default: return row_ep_staged_mode<LOGN, EP_STORE>(ep, val, t, row0, ops);
  }
}

// ----------------------------------------------------------------- kernels
template <typename T, int LOGN> struct ColThreads {
  static constexpr int value = (kColBytes / int(sizeof(typename cplx_t<T>::type))) * ((1 << LOGN) / 16);
};

// Composite operator by convolution (Section 3: precompute Phi^H Phi), in its
// real form.  The image is real and the PSF spectrum real and even, so only
// the half spectrum k2 in [0, K/2] of each image row is carried: two rows a, b
// travel as one complex row z = x_a + i x_b, whose transform Z separates as
// X_a(k) = (Z(k) + conj Z(-k)) / 2 and X_b(k) = (Z(k) - conj Z(-k)) / (2i).
// A half-spectrum row holds K/2 complex values; its entry 0 carries the two
// real ones, X(0) + i X(K/2).  Half-spectrum rows are stored n x K/2 in A.

// Forward row pass of the real form: rows 2 pr and 2 pr + 1 of the prologue's
// image, zero-padded to K columns, to their half spectra.
template <typename T, int LOGN, int E, typename Src>
__global__ void __launch_bounds__(kRowCta) k_row_fwd_h(Src src) {
  typedef typename cplx_t<T>::type C;
  decltype(auto) a = src.get();
  const Geometry& g = a.g;
  const RowPro<T>& pro = a.pro;
  const T* __restrict__ deapod = a.deapod;
  C* __restrict__ B = a.B;
  const C* __restrict__ tw = a.tw;
  const int nseq = a.nseq;
  constexpr int TT = Plan<LOGN, E>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int K = g.K, n = g.n, H = K / 2;
  const int seq = threadIdx.x / TT, t = threadIdx.x - seq * TT;
  const int ia = 2 * (blockIdx.x * nseq + seq), ib = ia + 1;
  C* s = reinterpret_cast<C*>(sm_raw) + seq * padded(K);
  const size_t row0[2] = {size_t(ia) * n, size_t(ib) * n};
  T val[2][E / 2];
  int i2[E / 2];
  row_prologue<LOGN, 2, E>(pro, row0, t, val, i2);
  C v[E];
#pragma unroll
  for (int m = 0; m < E; ++m) v[m] = cz<C>();
  if (deapod) {  // S: deapodisation of both rows (the Phi form; the convolution form has none)
    const T da = deapod[ia], db = deapod[ib];
#pragma unroll
    for (int j = 0; j < E / 2; ++j) {
      const T dc = deapod[i2[j]];
      v[kept_slot<E>(j)] = cmk<C>(val[0][j] * da * dc, val[1][j] * db * dc);
    }
  } else {
#pragma unroll
    for (int j = 0; j < E / 2; ++j) v[kept_slot<E>(j)] = cmk<C>(val[0][j], val[1][j]);
  }
  auto to_smem = [&](int q, C x) { s[sidx(q)] = x; };
  run_stages<LOGN, 0, E>(v, t, 1, s, 1, tw, -1, to_smem);
  __syncthreads();
  C* oa = B + size_t(ia) * H;
  C* ob = oa + H;
#pragma unroll
  for (int m = 0; m < E / 2; ++m) {
    const int k = t + m * TT;
    const C zk = s[sidx(k)];
    if (k == 0) {
      const C zh = s[sidx(H)];
      oa[0] = cmk<C>(zk.x, zh.x);
      ob[0] = cmk<C>(zk.y, zh.y);
    } else {
      const C zm = s[sidx(K - k)];  // Z(-k)
      oa[k] = cmk<C>(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
      ob[k] = cmk<C>(T(0.5) * (zk.y + zm.y), T(0.5) * (zm.x - zk.x));
    }
  }
}

// Column pass of the real form: cw half-spectrum columns per CTA, forward
// FFT over the K rows (n non-zero), multiply by the PSF spectrum, inverse FFT,
// keep the n rows the crop retains.  Column 0 holds two real-row columns,
// c0 = X(., 0) + i X(., K/2): its transform P splits into the even part
// (P(q) + conj P(-q)) / 2 (column 0's) and (P(q) - conj P(-q)) / 2 (i times
// column K/2's), each multiplied by its own spectrum column.
// One CTA per SM and the full register file per thread: the radix-16
// stages then run spill-free, which measured faster (22.6 against 24.8 us per
// launch at K = 2048) than two spilling CTAs per SM, despite the second wave.
template <typename T, int LOGN, typename Src>
__global__ void __launch_bounds__(ColThreads<T, LOGN>::value, 1)
    k_col_conv_h(Src src) {
  typedef typename cplx_t<T>::type C;
  decltype(auto) a = src.get();
  const Geometry& g = a.g;
  C* __restrict__ B = a.B;
  const T* __restrict__ khat = a.khat;
  const T* __restrict__ knyq = a.knyq;
  const C* __restrict__ tw = a.tw;
  const int cw = a.cw;
  constexpr int TT = Plan<LOGN>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int K = g.K, n = g.n, half = n / 2, H = K / 2;
  const int cc = threadIdx.x % cw, t = threadIdx.x / cw;
  const int c = blockIdx.x * cw + cc;
  C* s = reinterpret_cast<C*>(sm_raw) + cc;  // cw interleaved columns
  auto load = [&](int m) -> C {
    const int i1 = (t + m * TT + half) & (K - 1);
    return i1 < n ? B[size_t(i1) * H + c] : cz<C>();
  };
  auto to_smem = [&](int q, C v) { s[sidx(q) * cw] = v; };
  fft_seq<LOGN>(t, s, cw, tw, -1, load, to_smem);
  __syncthreads();
  if (blockIdx.x == 0) {
    // column 0 (this CTA's first): the pairs (q, -q), q = 0..K/2, in place,
    // spread over all the CTA's threads with their spectrum values loaded
    // first; ev(-q) = conj ev(q), od(-q) = -conj od(q)
    C* s0 = reinterpret_cast<C*>(sm_raw);
    const int nt = blockDim.x;
    for (int q0 = 0; q0 <= H; q0 += 4 * nt) {
      T h0[4], hn[4], h0m[4], hnm[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * nt + int(threadIdx.x), qm = (K - q) & (K - 1);
        if (q <= H) {
          h0[u] = khat[size_t(q) * cw];
          hn[u] = knyq[q];
          h0m[u] = khat[size_t(qm) * cw];
          hnm[u] = knyq[qm];
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * nt + int(threadIdx.x), qm = (K - q) & (K - 1);
        if (q <= H) {
          const C P = s0[sidx(q) * cw], Pm = s0[sidx(qm) * cw];
          const T evx = T(0.5) * (P.x + Pm.x), evy = T(0.5) * (P.y - Pm.y);
          const T odx = T(0.5) * (P.x - Pm.x), ody = T(0.5) * (P.y + Pm.y);
          s0[sidx(q) * cw] = cmk<C>(h0[u] * evx + hn[u] * odx, h0[u] * evy + hn[u] * ody);
          if (qm != q) s0[sidx(qm) * cw] = cmk<C>(h0m[u] * evx - hnm[u] * odx, hnm[u] * ody - h0m[u] * evy);
        }
      }
    }
  }
  __syncthreads();
  C v[16];
  const T* kc = khat + (size_t(blockIdx.x) * K) * cw + cc;
#pragma unroll
  for (int m = 0; m < 16; ++m) {
    const int q = t + m * TT;
    v[m] = cscale(s[sidx(q) * cw], c ? kc[size_t(q) * cw] : T(1));
  }
  __syncthreads();
  auto store = [&](int q, C x) {
    const int i1 = (q + half) & (K - 1);
    if (i1 < n) B[size_t(i1) * H + c] = x;
  };
  run_stages<LOGN, 0>(v, t, 1, s, cw, tw, +1, store);
}

// Inverse row pass of the real form: the half spectra of rows a = 2 pr and
// b = 2 pr + 1 rebuilt into Z = Y_a + i Y_b over all K frequencies
// (Y(K - k) = conj Y(k)), one inverse FFT, Re -> row a, Im -> row b, crop and
// row epilogue.
template <typename T, int LOGN, int E, typename Src>
__global__ void __launch_bounds__(kRowCta, 2) k_row_inv_h(Src src) {
  typedef typename cplx_t<T>::type C;
  decltype(auto) a = src.get();
  const Geometry& g = a.g;
  const C* __restrict__ B = a.B;
  const T* __restrict__ deapod = a.deapod;
  const RowEp<T>& ep = a.ep;
  const C* __restrict__ tw = a.tw;
  const int nseq = a.nseq;
  constexpr int TT = Plan<LOGN, E>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  __shared__ double red[5 * 32];
  __shared__ __align__(8) uint64_t bar;
  const int K = g.K, n = g.n, H = K / 2;
  const int seq = threadIdx.x / TT, t = threadIdx.x - seq * TT;
  const int ia = 2 * (blockIdx.x * nseq + seq), ib = ia + 1;
  C* s = reinterpret_cast<C*>(sm_raw) + seq * padded(K);
  // The epilogue's operand rows (ops[seq][k][row][n]) arrive by bulk copies
  // while the transform runs.
  T* ops_all = reinterpret_cast<T*>(sm_raw + align16(nseq * padded(K) * sizeof(C)));
  const T* opd[2] = {nullptr, nullptr};
  const int nop = ep_staged(ep, opd);
  if (nop > 0 && threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
    const uint32_t row_bytes = uint32_t(n * sizeof(T));
    mbar_arrive_expect_tx(&bar, uint32_t(nseq * nop * 2) * row_bytes);
    for (int q = 0; q < nseq; ++q) {
      const int r0 = 2 * (blockIdx.x * nseq + q);
      for (int k = 0; k < nop; ++k)
        for (int r = 0; r < 2; ++r)
          bulk_load(ops_all + ((size_t(q) * 2 + k) * 2 + r) * n, opd[k] + size_t(r0 + r) * n, row_bytes, &bar);
    }
  }
  __syncthreads();
  const C* ba = B + size_t(ia) * H;
  const C* bb = ba + H;
  // frequency q = t + m K/E: entry q for m < E/2, entry K - q (entry 0 for
  // q = K/2) above; thread 0 unpacks entry 0 into Y(0) and Y(K/2)
  auto load = [&](int m) -> C {
    const int q = t + m * TT;
    const int e = m < E / 2 ? q : ((K - q) & (H - 1));
    const C a = ba[e], b = bb[e];
    if (t == 0 && (m == 0 || m == E / 2)) return m == 0 ? cmk<C>(a.x, b.x) : cmk<C>(a.y, b.y);
    return m < E / 2 ? cmk<C>(a.x - b.y, a.y + b.x) : cmk<C>(a.x + b.y, b.x - a.y);
  };
  T val[2][E];
  int cnt = 0;
  auto stash = [&](int, C v) {  // sink order, see last_pos
    val[0][cnt] = v.x;
    val[1][cnt] = v.y;
    ++cnt;
  };
  fft_seq<LOGN, E>(t, s, 1, tw, +1, load, stash);
  if (deapod) {  // S^T after the crop (the Phi^H form)
    const T da = deapod[ia], db = deapod[ib];
#pragma unroll
    for (int m = 0; m < E; ++m) {
      const int i2 = ep_col<LOGN, E>(t, m);
      if (i2 < n) {
        const T dc = deapod[i2];
        val[0][m] *= da * dc;
        val[1][m] *= db * dc;
      }
    }
  }
  const size_t row0[2] = {size_t(ia) * n, size_t(ib) * n};
  bool ok = true;
  if (nop > 0) ok = mbar_wait_bounded(&bar, 0, ep.err);
  EpAcc<T> part;
  if (ok) part = row_ep_staged<LOGN>(ep, val, t, row0, ops_all + size_t(seq) * 4 * n);
  row_ep_finish(ep, part, red, int(blockIdx.x), a.nblocks);
}

// Real-form column passes of Phi and Phi^H on the padded grid (K + J per side,
// periodic halo of J cells).  Grid cell (q, c) sits at padded row/column
// q + pad_lo and also, near the edges, at its periodic image.
PD int halo_images(int q, int K, int pl, int (&at)[2]) {
  const int jhi = kJ - pl;  // grid indices < jhi repeat past the end
  at[0] = q + pl;
  at[1] = q >= K - pl ? q + pl - K : (q < jhi ? q + pl + K : -1);
  return at[1] >= 0 ? 2 : 1;
}

// Phi: cw half-spectrum columns c per CTA.  For the image rows' half spectra
// X(., c), c < K/2, the column FFT gives grid column c, and column K - c is
// its conjugate mirror, G(q, K - c) = conj G(-q, c) (a real image).  Column 0
// carries X(., 0) + i X(., K/2): its transform P gives grid column 0 as
// (P(q) + conj P(-q)) / 2 and column K/2 as -i (P(q) - conj P(-q)) / 2.
// One CTA per SM, spill-free (measured 22.3 against 24.6 us at K = 2048 for
// two spilling CTAs per SM; the adjoint pass below measured slower that way,
// 39.4 against 36.4 us, and keeps two).
template <typename T, int LOGN, typename Src>
__global__ void __launch_bounds__(ColThreads<T, LOGN>::value, 1)
    k_col_fwd_h(Src src) {
  typedef typename cplx_t<T>::type C;
  decltype(auto) a = src.get();
  const Geometry& g = a.g;
  const C* __restrict__ B = a.B;
  C* __restrict__ Pg = a.Pg;
  const C* __restrict__ tw = a.tw;
  const int cw = a.cw;
  constexpr int TT = Plan<LOGN>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int K = g.K, n = g.n, half = n / 2, H = K / 2, pl = g.pad_lo, KP = g.KP;
  const int cc = threadIdx.x % cw, t = threadIdx.x / cw;
  const int c = blockIdx.x * cw + cc;
  C* s = reinterpret_cast<C*>(sm_raw) + cc;
  auto load = [&](int m) -> C {
    const int i1 = (t + m * TT + half) & (K - 1);
    return i1 < n ? B[size_t(i1) * H + c] : cz<C>();
  };
  auto to_smem = [&](int q, C v) { s[sidx(q) * cw] = v; };
  fft_seq<LOGN>(t, s, cw, tw, -1, load, to_smem);
  __syncthreads();
  auto put = [&](int q, int col, C v) {
    int rows[2], cols[2];
    const int nr = halo_images(q, K, pl, rows), nc = halo_images(col, K, pl, cols);
    for (int a = 0; a < nr; ++a)
      for (int b = 0; b < nc; ++b) Pg[size_t(rows[a]) * KP + cols[b]] = v;
  };
#pragma unroll 4
  for (int m = 0; m < 16; ++m) {
    const int q = t + m * TT, qm = (K - q) & (K - 1);
    const C P = s[sidx(q) * cw];
    if (c != 0) {
      put(q, c, P);
      put(qm, K - c, cmk<C>(P.x, -P.y));
    } else {
      const C Pm = s[sidx(qm) * cw];
      put(q, 0, cmk<C>(T(0.5) * (P.x + Pm.x), T(0.5) * (P.y - Pm.y)));
      // -i (P - conj Pm) / 2
      put(q, H, cmk<C>(T(0.5) * (P.y + Pm.y), T(0.5) * (Pm.x - P.x)));
    }
  }
}

// Phi^H: Re of the inverse transform of the gridded accumulator Q is the
// inverse transform of its Hermitian part Qh(q, c) = (Q(q, c) + conj Q(-q, -c)) / 2,
// so only columns c <= K/2 are transformed: cw half-spectrum columns per
// CTA (halo folded on load), inverse column FFT, the n cropped rows into the
// half-spectrum rows B; column 0 packs the two Hermitian columns 0 and K/2 as
// Qh(., 0) + i Qh(., K/2), whose transforms are real.
template <typename T, int LOGN, typename Src>
__global__ void __launch_bounds__(ColThreads<T, LOGN>::value, ColThreads<T, LOGN>::value <= 512 ? 2 : 1)
    k_col_inv_h(Src src) {
  typedef typename cplx_t<T>::type C;
  decltype(auto) a = src.get();
  const Geometry& g = a.g;
  const C* __restrict__ Q = a.Q;
  C* __restrict__ B = a.B;
  const C* __restrict__ tw = a.tw;
  const int cw = a.cw;
  constexpr int TT = Plan<LOGN>::T;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  const int K = g.K, n = g.n, half = n / 2, H = K / 2, pl = g.pad_lo, KP = g.KP;
  const int cc = threadIdx.x % cw, t = threadIdx.x / cw;
  const int c = blockIdx.x * cw + cc;
  C* s = reinterpret_cast<C*>(sm_raw) + cc;
  auto fold = [&](int q, int col) -> C {
    int rows[2], cols[2];
    const int nr = halo_images(q, K, pl, rows), nc = halo_images(col, K, pl, cols);
    C v = cz<C>();
    for (int a = 0; a < nr; ++a)
      for (int b = 0; b < nc; ++b) v = cadd(v, Q[size_t(rows[a]) * KP + cols[b]]);
    return v;
  };
  auto load = [&](int m) -> C {
    const int q = t + m * TT, qm = (K - q) & (K - 1);
    if (c != 0) {
      const C a = fold(q, c), b = fold(qm, K - c);
      return cmk<C>(T(0.5) * (a.x + b.x), T(0.5) * (a.y - b.y));
    }
    const C a0 = fold(q, 0), b0 = fold(qm, 0), aH = fold(q, H), bH = fold(qm, H);
    const C h0 = cmk<C>(T(0.5) * (a0.x + b0.x), T(0.5) * (a0.y - b0.y));
    const C hH = cmk<C>(T(0.5) * (aH.x + bH.x), T(0.5) * (aH.y - bH.y));
    return cmk<C>(h0.x - hH.y, h0.y + hH.x);  // h0 + i hH
  };
  auto store = [&](int q, C v) {
    const int i1 = (q + half) & (K - 1);
    if (i1 < n) B[size_t(i1) * H + c] = v;
  };
  fft_seq<LOGN>(t, s, cw, tw, +1, load, store);
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


// Row pairs per CTA of the real-form row passes (E elements per thread).
inline int row_pair_nseq(const Geometry& g, int E) {
  int s = kRowCta / (g.K / E);
  if (s < 1) s = 1;
  if (s > g.n / 2) s = g.n / 2;
  return s;
}

// CTAs of one inverse row pass (its epilogue's partial sums).
int row_inv_blocks(const Geometry& g) { return g.n / 2 / row_pair_nseq(g, row_e_host(g.K)); }
int row_pass_nseq(const Geometry& g) { return row_pair_nseq(g, row_e_host(g.K)); }
template <typename T> int col_pass_width() { return col_width<T>(); }
template int col_pass_width<float>();
template int col_pass_width<double>();

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

// Grid sides of the batched passes (image sides 64..1024).
#define PURIFY_LOGN_SWITCH_BATCH(K, BODY)                 \
  switch (K) {                                            \
    case 128: { constexpr int L = 7; BODY; } break;       \
    case 256: { constexpr int L = 8; BODY; } break;       \
    case 512: { constexpr int L = 9; BODY; } break;       \
    case 1024: { constexpr int L = 10; BODY; } break;     \
    case 2048: { constexpr int L = 11; BODY; } break;     \
    default: break;                                       \
  }

template <typename T, int L> cudaError_t configure_one() {
  cudaError_t e = raise_smem_limit(k_row_fwd_h<T, L, row_e<L>(), ArgVal<RowFwdArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_col_conv_h<T, L, ArgVal<ColConvArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_col_fwd_h<T, L, ArgVal<ColFwdArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_col_inv_h<T, L, ArgVal<ColInvArgs<T>>>);
  if (e == cudaSuccess) e = raise_smem_limit(k_row_inv_h<T, L, row_e<L>(), ArgVal<RowInvArgs<T>>>);
  if constexpr (L >= 7 && L <= 11) {
    if (e == cudaSuccess) e = raise_smem_limit(k_row_fwd_h<T, L, row_e<L>(), ArgTab<RowFwdArgs<T>>>);
    if (e == cudaSuccess) e = raise_smem_limit(k_col_conv_h<T, L, ArgTab<ColConvArgs<T>>>);
    if (e == cudaSuccess) e = raise_smem_limit(k_col_fwd_h<T, L, ArgTab<ColFwdArgs<T>>>);
    if (e == cudaSuccess) e = raise_smem_limit(k_col_inv_h<T, L, ArgTab<ColInvArgs<T>>>);
    if (e == cudaSuccess) e = raise_smem_limit(k_row_inv_h<T, L, row_e<L>(), ArgTab<RowInvArgs<T>>>);
  }
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

cudaError_t set_wait_spins_fft(uint32_t spins) { return set_module_wait_spins(spins); }

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

// Real part of the spectrum, columns [0, K/2) in launch_col_conv_h's layout
// [column block][row][cw], column K/2 after them.
template <typename T>
__global__ void k_spectrum_layout(const typename cplx_t<T>::type* __restrict__ X, int K, int cw, double scale,
                                  T* __restrict__ khat) {
  const size_t idx = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= size_t(K) * K) return;
  const int q = int(idx / K), c = int(idx % K), H = K / 2;
  const T v = T(double(X[idx].x) * scale);
  if (c < H) khat[(size_t(c / cw) * K + q) * cw + (c % cw)] = v;
  else if (c == H) khat[size_t(H) * K + q] = v;
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

// Launch shapes of the real-form passes for grid side K (image side n = K/2).
inline int row_pass_ctas(const Geometry& g) { return g.n / 2 / row_pair_nseq(g, row_e_host(g.K)); }
template <typename T> inline size_t row_fwd_smem(const Geometry& g) {
  return row_pair_nseq(g, row_e_host(g.K)) * padded(g.K) * sizeof(typename cplx_t<T>::type);
}
template <typename T> inline size_t row_inv_smem(const Geometry& g) {
  const int nseq = row_pair_nseq(g, row_e_host(g.K));
  return align16(nseq * padded(g.K) * sizeof(typename cplx_t<T>::type)) + size_t(nseq) * 4 * g.n * sizeof(T);
}
template <typename T> inline size_t col_smem(const Geometry& g) {
  return col_width<T>() * padded(g.K) * sizeof(typename cplx_t<T>::type);
}

template <typename T>
void launch_row_fwd_h(const Geometry& g, const RowPro<T>& pro, const T* deapod, typename cplx_t<T>::type* B,
                      const typename cplx_t<T>::type* tw, cudaStream_t s) {
  const int nseq = row_pair_nseq(g, row_e_host(g.K));
  ArgVal<RowFwdArgs<T>> src{RowFwdArgs<T>{g, pro, deapod, B, tw, nseq}};
  PURIFY_LOGN_SWITCH(g.K, (k_row_fwd_h<T, L, row_e<L>()><<<row_pass_ctas(g), nseq * Plan<L, row_e<L>()>::T,
                                                           row_fwd_smem<T>(g), s>>>(src)));
}

template <typename T>
void launch_col_conv_h(const Geometry& g, typename cplx_t<T>::type* B, const T* khat,
                       const typename cplx_t<T>::type* tw, cudaStream_t s) {
  const int cw = col_width<T>();
  ArgVal<ColConvArgs<T>> src{ColConvArgs<T>{g, B, khat, khat + size_t(g.K / 2) * g.K, tw, cw}};
  PURIFY_LOGN_SWITCH(g.K, (k_col_conv_h<T, L><<<g.K / 2 / cw, cw * Plan<L>::T, col_smem<T>(g), s>>>(src)));
}

template <typename T>
void launch_col_fwd_h(const Geometry& g, const typename cplx_t<T>::type* B, typename cplx_t<T>::type* Pg,
                      const typename cplx_t<T>::type* tw, cudaStream_t s) {
  const int cw = col_width<T>();
  ArgVal<ColFwdArgs<T>> src{ColFwdArgs<T>{g, B, Pg, tw, cw}};
  PURIFY_LOGN_SWITCH(g.K, (k_col_fwd_h<T, L><<<g.K / 2 / cw, cw * Plan<L>::T, col_smem<T>(g), s>>>(src)));
}

template <typename T>
void launch_col_inv_h(const Geometry& g, const typename cplx_t<T>::type* Q, typename cplx_t<T>::type* B,
                      const typename cplx_t<T>::type* tw, cudaStream_t s) {
  const int cw = col_width<T>();
  ArgVal<ColInvArgs<T>> src{ColInvArgs<T>{g, Q, B, tw, cw}};
  PURIFY_LOGN_SWITCH(g.K, (k_col_inv_h<T, L><<<g.K / 2 / cw, cw * Plan<L>::T, col_smem<T>(g), s>>>(src)));
}

template <typename T>
int launch_row_inv_h(const Geometry& g, const typename cplx_t<T>::type* B, const T* deapod, const RowEp<T>& ep,
                     const typename cplx_t<T>::type* tw, cudaStream_t s) {
  const int nseq = row_pair_nseq(g, row_e_host(g.K));
  const int nb = row_pass_ctas(g);
  ArgVal<RowInvArgs<T>> src{RowInvArgs<T>{g, B, deapod, ep, tw, nseq, nb}};
  PURIFY_LOGN_SWITCH(g.K, (k_row_inv_h<T, L, row_e<L>()><<<nb, nseq * Plan<L, row_e<L>()>::T, row_inv_smem<T>(g),
                                                           s>>>(src)));
  return nb;
}

// Batched passes: `count` instances of one grid side (g gives the shared
// shape), arguments in a device table, instance = blockIdx.y.
template <typename T>
void launch_row_fwd_h_batch(const Geometry& g, const RowFwdArgs<T>* tab, int count, cudaStream_t s) {
  const int nseq = row_pair_nseq(g, row_e_host(g.K));
  ArgTab<RowFwdArgs<T>> src{tab};
  PURIFY_LOGN_SWITCH_BATCH(g.K, (k_row_fwd_h<T, L, row_e<L>()><<<dim3(row_pass_ctas(g), count),
                                                           nseq * Plan<L, row_e<L>()>::T, row_fwd_smem<T>(g), s>>>(src)));
}
template <typename T>
void launch_col_conv_h_batch(const Geometry& g, const ColConvArgs<T>* tab, int count, cudaStream_t s) {
  const int cw = col_width<T>();
  ArgTab<ColConvArgs<T>> src{tab};
  PURIFY_LOGN_SWITCH_BATCH(g.K, (k_col_conv_h<T, L><<<dim3(g.K / 2 / cw, count), cw * Plan<L>::T, col_smem<T>(g), s>>>(src)));
}
template <typename T>
void launch_col_fwd_h_batch(const Geometry& g, const ColFwdArgs<T>* tab, int count, cudaStream_t s) {
  const int cw = col_width<T>();
  ArgTab<ColFwdArgs<T>> src{tab};
  PURIFY_LOGN_SWITCH_BATCH(g.K, (k_col_fwd_h<T, L><<<dim3(g.K / 2 / cw, count), cw * Plan<L>::T, col_smem<T>(g), s>>>(src)));
}
template <typename T>
void launch_col_inv_h_batch(const Geometry& g, const ColInvArgs<T>* tab, int count, cudaStream_t s) {
  const int cw = col_width<T>();
  ArgTab<ColInvArgs<T>> src{tab};
  PURIFY_LOGN_SWITCH_BATCH(g.K, (k_col_inv_h<T, L><<<dim3(g.K / 2 / cw, count), cw * Plan<L>::T, col_smem<T>(g), s>>>(src)));
}
template <typename T>
void launch_row_inv_h_batch(const Geometry& g, const RowInvArgs<T>* tab, int count, cudaStream_t s) {
  const int nseq = row_pair_nseq(g, row_e_host(g.K));
  ArgTab<RowInvArgs<T>> src{tab};
  PURIFY_LOGN_SWITCH_BATCH(g.K, (k_row_inv_h<T, L, row_e<L>()><<<dim3(row_pass_ctas(g), count),
                                                           nseq * Plan<L, row_e<L>()>::T, row_inv_smem<T>(g), s>>>(src)));
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
  template void launch_row_fwd_h<T>(const Geometry&, const RowPro<T>&, const T*, cplx_t<T>::type*,             \
                                    const cplx_t<T>::type*, cudaStream_t);                                     \
  template void launch_col_conv_h<T>(const Geometry&, cplx_t<T>::type*, const T*, const cplx_t<T>::type*,       \
                                     cudaStream_t);                                                            \
  template int launch_row_inv_h<T>(const Geometry&, const cplx_t<T>::type*, const T*, const RowEp<T>&,          \
                                   const cplx_t<T>::type*, cudaStream_t);                                      \
  template void launch_fft2_plain<T>(int, cplx_t<T>::type*, const cplx_t<T>::type*, int, cudaStream_t);     \
  template void launch_col_fwd_h<T>(const Geometry&, const cplx_t<T>::type*, cplx_t<T>::type*,                \
                                    const cplx_t<T>::type*, cudaStream_t);                                     \
  template void launch_col_inv_h<T>(const Geometry&, const cplx_t<T>::type*, cplx_t<T>::type*,                \
                                    const cplx_t<T>::type*, cudaStream_t);                                     \
  template void build_psf_spectrum<T>(const T*, int, T*, cplx_t<T>::type*, const cplx_t<T>::type*, cudaStream_t); \
  template void launch_row_fwd_h_batch<T>(const Geometry&, const RowFwdArgs<T>*, int, cudaStream_t);         \
  template void launch_col_conv_h_batch<T>(const Geometry&, const ColConvArgs<T>*, int, cudaStream_t);       \
  template void launch_col_fwd_h_batch<T>(const Geometry&, const ColFwdArgs<T>*, int, cudaStream_t);         \
  template void launch_col_inv_h_batch<T>(const Geometry&, const ColInvArgs<T>*, int, cudaStream_t);         \
  template void launch_row_inv_h_batch<T>(const Geometry&, const RowInvArgs<T>*, int, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace purify
