// Prints the CUDA path's host-side tables (computed by the library's own
// host code) as JSON, for tests/test_host_tables.py to compare with the
// oracle: the Kaiser-Bessel shape, deapodisation weights, the per-tap kernel
// polynomials and the Daubechies filters.
#include <cstdio>
#include <vector>

#include "../paper_1406_0359_gb300/csrc/host_math.h"

using namespace purify;

static void print_vec(const char* name, const std::vector<double>& v, bool last = false) {
  std::printf("\"%s\": [", name);
  for (size_t i = 0; i < v.size(); ++i) std::printf("%s%.17g", i ? ", " : "", v[i]);
  std::printf("]%s\n", last ? "" : ",");
}

int main() {
  const int J = 8;
  const double beta = kb_beta(J, 2.0);
  std::printf("{\"beta\": %.17g,\n", beta);
  std::vector<double> d;
  kb_deapod_table(64, 128, J, beta, d);
  print_vec("deapod_64_128", d);
  print_vec("poly10", kb_poly_cached(J, beta, 10));
  print_vec("poly16", kb_poly_cached(J, beta, 16));
  for (int k = 1; k <= 8; ++k) {
    char name[16];
    std::snprintf(name, sizeof(name), "db%d", k);
    print_vec(name, daubechies_lowpass_cached(k), k == 8);
  }
  std::printf("}\n");
  return 0;
}
