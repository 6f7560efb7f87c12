// Host-side constants of the analyzer: the integer DCT matrix and the energy weights.
//
// Section 2, item (2) of the paper: the analyzer's DCT is an integer encoder routine.
// The matrix is the round-cosine integer DCT with row 0 equal to 64; the weights are the
// exponential DCT-energy weights of the block texture energy (Section 2, E).
#include <cmath>

#include "vca_internal.h"

namespace vca {

void make_dct_matrix(int N, int8_t* out) {
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < N; ++k) {
    const double alpha = k == 0 ? std::sqrt(1.0 / N) : std::sqrt(2.0 / N);
    for (int n = 0; n < N; ++n) {
      const double c = 64.0 * std::sqrt((double)N) * alpha * std::cos(pi * (2 * n + 1) * k / (2.0 * N));
      out[k * N + n] = (int8_t)std::lround(c);  // lround rounds half away from zero
    }
  }
}

void make_energy_weights(int N, float* out) {
  for (int u = 0; u < N; ++u) {
    for (int v = 0; v < N; ++v) {
      const double r = (double)(u + 1) * (v + 1) / ((double)N * N);
      out[u * N + v] = (float)std::exp(std::fabs(r * r - 1.0));
    }
  }
  out[0] = 0.0f;  // the DC coefficient carries no texture
}

void transform_shifts(int N, int B, int* s1, int* s2) {
  int l = 0;
  while ((1 << l) < N) ++l;
  *s1 = l + B - 9;
  *s2 = l + 6;
}

}  // namespace vca
