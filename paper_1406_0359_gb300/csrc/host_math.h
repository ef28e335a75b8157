// Host-side tables for the CUDA path: Kaiser-Bessel kernel, its Fourier
// transform for deapodisation, the piecewise-polynomial kernel used by the
// FP32 kernels, and the Daubechies filters.  Computed in double on the host;
// the kernel polynomial and the filters once per process.
#pragma once
#include <vector>

namespace purify {

// Modified Bessel I0 from its power series sum_k (z^2/4)^k / (k!)^2.
double bessel_i0(double z);
// Beatty et al. (2005) Kaiser-Bessel shape for support J, oversampling alpha.
double kb_beta(int J, double alpha);
// Kernel value kb(s) = I0(beta sqrt(1 - (2s/J)^2)) / I0(beta), |s| <= J/2.
double kb_value(double s, int J, double beta);
// Continuous Fourier transform of kb at xi cycles per grid cell.
double kb_fourier(double xi, int J, double beta);

// Piecewise polynomial for the J taps: for tap a and fraction f in [0, 1),
// kb(f + J/2 - 1 - a) ~= sum_d coef[a*(deg+1) + d] * x^d, x = 2f - 1.
// Chebyshev interpolation in double, converted to monomials.  Returns the
// max abs error over a dense check grid.
double kb_poly_fit(int J, double beta, int deg, std::vector<double>& coef);

// DbK low-pass analysis filter (length 2K) by spectral factorisation with
// the minimum-phase root choice, normalised to sum sqrt(2).
std::vector<double> daubechies_lowpass(int K);

// The two tables above computed once per process and kept (thread-safe).
const std::vector<double>& kb_poly_cached(int J, double beta, int deg);
const std::vector<double>& daubechies_lowpass_cached(int K);

// Deapodisation weights 1 / kb_fourier((i - n/2) / K), i < n, with I0(beta)
// evaluated once.
void kb_deapod_table(int n, int K, int J, double beta, std::vector<double>& out);

}  // namespace purify
