// Total-variation prior (Section 4's TV and RWTV) inside SDMM (Algorithm 1).
//
// The l1 block f_1 = gamma ||W Psi^H .||_1 is replaced by f_1 = gamma TV_w
// with L_1 = I, so the composite operator stays nu^2 Phi^H Phi + 2I.  TV_w is
// the weighted isotropic total variation with forward differences and a zero
// difference past the last row / column:
//     (grad x)_1[i, j] = x[i+1, j] - x[i, j] (0 on the last row),
//     (grad x)_2[i, j] = x[i, j+1] - x[i, j] (0 on the last column),
//     TV_w(x) = sum_ij w_ij |(grad x)[i, j]|,
// and div = -grad^T.  Its proximity operator (Eq. 7) is taken through the
// dual: prox(v) = v + div q with q minimising |v + div q|^2 / 2 over
// |q_ij| <= gamma w_ij, by projected-gradient steps
//     q <- P(q + tau grad(v + div q)),  tau = 1/8,
// a fixed number per SDMM iteration, warm-started from the previous
// iteration's q (zero at the start of each round).  Each step is one launch
// (every pixel's update needs its neighbours' previous q), ping-ponging
// between two dual buffers; the epilogue forms r_1 = v + div q, updates z_1,
// applies the positivity block (f_2, L_2 = I) and writes x_1 + x_2, with the
// objective's partial sums TV_w(x_hat).
#include "internal.h"
#include "solver_kernels.h"

namespace purify {

namespace {

constexpr int kTvT = 256;

// d = v + div q at (i, j) (q1 plane first, then q2; n x n each).
template <typename T> PD T dval(const T* __restrict__ v, const T* __restrict__ q, int n, int i, int j) {
  const size_t N = size_t(n) * n, k = size_t(i) * n + j;
  const T* q1 = q;
  const T* q2 = q + N;
  T d = v[k];
  if (i < n - 1) d += q1[k];
  if (i > 0) d -= q1[k - n];
  if (j < n - 1) d += q2[k];
  if (j > 0) d -= q2[k - 1];
  return d;
}

// One projected-gradient step of the dual: qo = P(qi + tau grad(v + div qi)),
// P the pixelwise projection onto |q_ij| <= gamma w_ij.
template <typename T>
__global__ void __launch_bounds__(kTvT) k_tv_dual_step(const T* __restrict__ v, const T* __restrict__ w, T gamma,
                                                       const T* __restrict__ qi, T* __restrict__ qo, int n) {
  const size_t N = size_t(n) * n;
  const size_t k = size_t(blockIdx.x) * kTvT + threadIdx.x;
  if (k >= N) return;
  const int i = int(k / n), j = int(k - size_t(i) * n);
  const T d = dval(v, qi, n, i, j);
  const T g1 = i < n - 1 ? dval(v, qi, n, i + 1, j) - d : T(0);
  const T g2 = j < n - 1 ? dval(v, qi, n, i, j + 1) - d : T(0);
  const T tau = T(0.125);
  T a = fma(tau, g1, qi[k]), b = fma(tau, g2, qi[k + N]);
  const T bound = gamma * (w ? w[k] : T(1));
  const T m = sqrt(a * a + b * b);
  if (m > bound) {
    const T s = bound / m;
    a *= s;
    b *= s;
  }
  qo[k] = a;
  qo[k + N] = b;
}

// v_1 = x_hat + z_1 (the TV block's input).
template <typename T>
__global__ void __launch_bounds__(kTvT) k_tv_input(const T* __restrict__ xh, const T* __restrict__ z1,
                                                   T* __restrict__ v, size_t N) {
  const size_t k = size_t(blockIdx.x) * kTvT + threadIdx.x;
  if (k < N) v[k] = xh[k] + z1[k];
}

// Epilogue: r_1 = v + div q, z_1 = v - r_1, x_1 = 2 r_1 - v; positivity block
// v_2 = x_hat + z_2, r_2 = max(v_2, 0), z_2 = v_2 - r_2; xs = x_1 + 2 r_2 - v_2;
// per-CTA partials of TV_w(x_hat).  With qcopy set the final dual is also
// written back to the buffer the next iteration starts from.
template <typename T>
__global__ void __launch_bounds__(kTvT) k_tv_epilogue(const T* __restrict__ v, const T* __restrict__ q,
                                                      T* __restrict__ qcopy, const T* __restrict__ xh,
                                                      const T* __restrict__ w, T* __restrict__ z1,
                                                      T* __restrict__ z2, T* __restrict__ xs, double* partials,
                                                      int n) {
  __shared__ double red[32];
  const size_t N = size_t(n) * n;
  const size_t k = size_t(blockIdx.x) * kTvT + threadIdx.x;
  Acc<T> part;
  if (k < N) {
    const int i = int(k / n), j = int(k - size_t(i) * n);
    const T vk = v[k];
    const T r1 = dval(v, q, n, i, j);
    z1[k] = vk - r1;
    const T v2 = xh[k] + z2[k];
    const T r2 = v2 > T(0) ? v2 : T(0);
    z2[k] = v2 - r2;
    xs[k] = (T(2) * r1 - vk) + (T(2) * r2 - v2);
    if (qcopy) {
      qcopy[k] = q[k];
      qcopy[k + N] = q[k + N];
    }
    const T x0 = xh[k];
    const T g1 = i < n - 1 ? xh[k + n] - x0 : T(0);
    const T g2 = j < n - 1 ? xh[k + 1] - x0 : T(0);
    part.add(sqrt(g1 * g1 + g2 * g2) * (w ? w[k] : T(1)));
  }
  if (partials) {
    const Acc<T> t = block_merge<kTvT>(part, red);
    if (threadIdx.x == 0) reinterpret_cast<Acc<T>*>(partials)[blockIdx.x] = t;
  }
}

// |grad x| per pixel (RWTV weights and their delta).
template <typename T>
__global__ void __launch_bounds__(kTvT) k_tv_magnitude(const T* __restrict__ x, T* __restrict__ out, int n) {
  const size_t N = size_t(n) * n;
  const size_t k = size_t(blockIdx.x) * kTvT + threadIdx.x;
  if (k >= N) return;
  const int i = int(k / n), j = int(k - size_t(i) * n);
  const T x0 = x[k];
  const T g1 = i < n - 1 ? x[k + n] - x0 : T(0);
  const T g2 = j < n - 1 ? x[k + 1] - x0 : T(0);
  out[k] = sqrt(g1 * g1 + g2 * g2);
}

inline int tv_blocks(int n) { return int((size_t(n) * n + kTvT - 1) / kTvT); }

}  // namespace

int tv_partials(int n) { return tv_blocks(n); }

template <typename T>
int tv_block(const TvBlock<T>& b, cudaStream_t s) {
  const int n = b.n, nb = tv_blocks(n);
  const size_t N = size_t(n) * n;
  k_tv_input<T><<<nb, kTvT, 0, s>>>(b.xh, b.z1, b.v, N);
  const T* qi = b.qa;
  T* qo = b.qb;
  for (int it = 0; it < b.iters; ++it) {
    k_tv_dual_step<T><<<nb, kTvT, 0, s>>>(b.v, b.w, T(b.gamma), qi, qo, n);
    const T* t = qo;
    qo = const_cast<T*>(qi);
    qi = t;
  }
  // after an odd number of steps the dual sits in qb: copy it back to qa
  T* qcopy = (b.iters & 1) ? b.qa : nullptr;
  k_tv_epilogue<T><<<nb, kTvT, 0, s>>>(b.v, qi, qcopy, b.xh, b.w, b.z1, b.z2, b.xs, b.partials, n);
  return nb;
}

template <typename T> void tv_magnitude(const T* x, T* out, int n, cudaStream_t s) {
  k_tv_magnitude<T><<<tv_blocks(n), kTvT, 0, s>>>(x, out, n);
}

template int tv_block<float>(const TvBlock<float>&, cudaStream_t);
template int tv_block<double>(const TvBlock<double>&, cudaStream_t);
template void tv_magnitude<float>(const float*, float*, int, cudaStream_t);
template void tv_magnitude<double>(const double*, double*, int, cudaStream_t);

}  // namespace purify
