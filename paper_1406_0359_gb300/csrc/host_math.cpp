// Host-side tables for the CUDA path (see host_math.h).
#include "host_math.h"

#include <cmath>
#include <complex>
#include <map>
#include <mutex>
#include <stdexcept>
#include <tuple>

namespace purify {

double bessel_i0(double z) {
  const double q = 0.25 * z * z;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 500; ++k) {
    term *= q / (double(k) * double(k));
    sum += term;
    if (term <= 1e-18 * sum) break;
  }
  return sum;
}

double kb_beta(int J, double alpha) {
  const double a = (J / alpha) * (alpha - 0.5);
  return M_PI * std::sqrt(a * a - 0.8);
}

double kb_value(double s, int J, double beta) {
  const double r = 2.0 * s / J;
  const double arg = 1.0 - r * r;
  if (arg < 0.0) return 0.0;
  return bessel_i0(beta * std::sqrt(arg)) / bessel_i0(beta);
}

double kb_fourier(double xi, int J, double beta) {
  // J/I0(beta) * sinh(r)/r with r^2 = beta^2 - (pi J xi)^2 (sin form past the branch point)
  const double t = M_PI * J * xi;
  const double d = beta * beta - t * t;
  double v;
  if (d > 1e-12) {
    const double r = std::sqrt(d);
    v = std::sinh(r) / r;
  } else if (d < -1e-12) {
    const double r = std::sqrt(-d);
    v = std::sin(r) / r;
  } else {
    v = 1.0;
  }
  return v * J / bessel_i0(beta);
}

double kb_poly_fit(int J, double beta, int deg, std::vector<double>& coef) {
  const int nc = deg + 1;
  coef.assign(size_t(J) * nc, 0.0);
  std::vector<double> nodes(nc), vals(nc), cheb(nc);
  for (int i = 0; i < nc; ++i) nodes[i] = std::cos(M_PI * (i + 0.5) / nc);
  double maxerr = 0.0;
  for (int a = 0; a < J; ++a) {
    const double off = J / 2.0 - 1.0 - a;  // s = f + off, f = (x + 1)/2
    for (int i = 0; i < nc; ++i) vals[i] = kb_value(0.5 * (nodes[i] + 1.0) + off, J, beta);
    // Chebyshev coefficients c_k = (2 - [k==0]) / nc * sum_i vals_i T_k(node_i)
    for (int k = 0; k < nc; ++k) {
      double s = 0.0;
      for (int i = 0; i < nc; ++i) s += vals[i] * std::cos(k * M_PI * (i + 0.5) / nc);
      cheb[k] = s * (k == 0 ? 1.0 : 2.0) / nc;
    }
    // convert sum c_k T_k(x) to monomials with the recurrence T_{k+1} = 2x T_k - T_{k-1}
    std::vector<double> tkm1(nc, 0.0), tk(nc, 0.0), mono(nc, 0.0);
    tkm1[0] = 1.0;  // T0
    if (nc > 1) tk[1] = 1.0;  // T1
    for (int d = 0; d < nc; ++d) mono[d] += cheb[0] * tkm1[d];
    if (nc > 1)
      for (int d = 0; d < nc; ++d) mono[d] += cheb[1] * tk[d];
    for (int k = 2; k < nc; ++k) {
      std::vector<double> tn(nc, 0.0);
      for (int d = 0; d < nc; ++d) {
        if (d > 0) tn[d] += 2.0 * tk[d - 1];
        tn[d] -= tkm1[d];
      }
      for (int d = 0; d < nc; ++d) mono[d] += cheb[k] * tn[d];
      tkm1.swap(tk);
      tk.swap(tn);
    }
    for (int d = 0; d < nc; ++d) coef[size_t(a) * nc + d] = mono[d];
    for (int t = 0; t <= 1000; ++t) {
      const double f = t / 1000.0 * (1.0 - 1e-12);
      const double x = 2.0 * f - 1.0;
      double p = 0.0;
      for (int d = nc - 1; d >= 0; --d) p = p * x + mono[d];
      maxerr = std::max(maxerr, std::fabs(p - kb_value(f + off, J, beta)));
    }
  }
  return maxerr;
}

namespace {
typedef std::complex<double> cd;

// All roots of sum_k c[k] y^k (c[deg] != 0) by Durand-Kerner iteration,
// polished by Newton steps on the original polynomial.
std::vector<cd> poly_roots(const std::vector<double>& c) {
  const int deg = int(c.size()) - 1;
  std::vector<cd> r(deg);
  if (deg <= 0) return r;
  const cd seed(0.4, 0.9);
  for (int i = 0; i < deg; ++i) r[i] = std::pow(seed, i);
  auto eval = [&](cd y) {
    cd p = c[deg];
    for (int k = deg - 1; k >= 0; --k) p = p * y + c[k];
    return p;
  };
  auto deriv = [&](cd y) {
    cd p = double(deg) * c[deg];
    for (int k = deg - 1; k >= 1; --k) p = p * y + double(k) * c[k];
    return p;
  };
  for (int it = 0; it < 2000; ++it) {
    double moved = 0.0;
    for (int i = 0; i < deg; ++i) {
      cd den = c[deg];
      for (int j = 0; j < deg; ++j)
        if (j != i) den *= (r[i] - r[j]);
      const cd step = eval(r[i]) / den;
      r[i] -= step;
      moved = std::max(moved, std::abs(step));
    }
    if (moved < 1e-15) break;
  }
  for (int i = 0; i < deg; ++i)
    for (int k = 0; k < 3; ++k) {
      const cd d = deriv(r[i]);
      if (std::abs(d) > 0) r[i] -= eval(r[i]) / d;
    }
  return r;
}
}  // namespace

std::vector<double> daubechies_lowpass(int K) {
  if (K < 1) throw std::invalid_argument("K >= 1");
  // |H|^2 = 2 cos^2K(w/2) P(sin^2(w/2)),  P(y) = sum_{k<K} binom(K-1+k, k) y^k
  std::vector<double> p(K);
  double b = 1.0;
  for (int k = 0; k < K; ++k) {
    p[k] = b;  // binom(K-1+k, k)
    b = b * double(K + k) / double(k + 1);
  }
  std::vector<cd> h(1, cd(1.0, 0.0));
  auto mul = [&](cd c0, cd c1) {  // h <- h * (c0 + c1 z^-1)
    std::vector<cd> out(h.size() + 1, cd(0.0, 0.0));
    for (size_t i = 0; i < h.size(); ++i) {
      out[i] += h[i] * c0;
      out[i + 1] += h[i] * c1;
    }
    h.swap(out);
  };
  for (int k = 0; k < K; ++k) mul(1.0, 1.0);
  if (K > 1) {
    for (const cd& y : poly_roots(p)) {
      // y = (2 - z - 1/z)/4  <=>  z^2 - (2 - 4y) z + 1 = 0; keep |z| < 1
      const cd bb = 2.0 - 4.0 * y;
      const cd disc = std::sqrt(bb * bb - 4.0);
      cd z = 0.5 * (bb + disc);
      if (std::abs(z) >= 1.0) z = 0.5 * (bb - disc);
      mul(1.0, -z);
    }
  }
  std::vector<double> out(h.size());
  double s = 0.0;
  for (size_t i = 0; i < h.size(); ++i) {
    out[i] = h[i].real();
    s += out[i];
  }
  for (double& v : out) v *= std::sqrt(2.0) / s;
  return out;
}

namespace {
std::mutex g_table_mutex;
}  // namespace

const std::vector<double>& kb_poly_cached(int J, double beta, int deg) {
  static std::map<std::tuple<int, double, int>, std::vector<double>> cache;
  std::lock_guard<std::mutex> lock(g_table_mutex);
  auto it = cache.find(std::make_tuple(J, beta, deg));
  if (it == cache.end()) {
    std::vector<double> coef;
    kb_poly_fit(J, beta, deg, coef);
    it = cache.emplace(std::make_tuple(J, beta, deg), std::move(coef)).first;
  }
  return it->second;
}

const std::vector<double>& daubechies_lowpass_cached(int K) {
  static std::map<int, std::vector<double>> cache;
  std::lock_guard<std::mutex> lock(g_table_mutex);
  auto it = cache.find(K);
  if (it == cache.end()) it = cache.emplace(K, daubechies_lowpass(K)).first;
  return it->second;
}

void kb_deapod_table(int n, int K, int J, double beta, std::vector<double>& out) {
  const double scale = J / bessel_i0(beta);
  out.resize(size_t(n));
  for (int i = 0; i < n; ++i) {
    const double t = M_PI * J * double(i - n / 2) / K;
    const double d = beta * beta - t * t;
    double v;
    if (d > 1e-12) {
      const double r = std::sqrt(d);
      v = std::sinh(r) / r;
    } else if (d < -1e-12) {
      const double r = std::sqrt(-d);
      v = std::sin(r) / r;
    } else {
      v = 1.0;
    }
    out[size_t(i)] = 1.0 / (v * scale);
  }
}

}  // namespace purify
