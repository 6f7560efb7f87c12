// Host-side constants of the analyzer: the integer DCT matrix and the energy weights.
//
// Section 2, item (2) of the paper: the analyzer's DCT is an integer encoder routine.
// The matrix is the round-cosine integer DCT with row 0 equal to 64; the weights are the
// exponential DCT-energy weights of the block texture energy (Section 2, E).
#include <cmath>
#include <cstdio>
#include <cstdlib>

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

void make_energy_weights_rect(int Nv, int Nh, float* out) {
  for (int u = 0; u < Nv; ++u) {
    for (int v = 0; v < Nh; ++v) {
      const double r = (double)(u + 1) * (v + 1) / ((double)Nv * Nh);
      out[u * Nh + v] = (float)std::exp(std::fabs(r * r - 1.0));
    }
  }
  out[0] = 0.0f;  // the DC coefficient carries no texture
}

void make_energy_weights(int N, float* out) { make_energy_weights_rect(N, N, out); }

void transform_shifts(int N, int B, int* s1, int* s2) {
  int l = 0;
  while ((1 << l) < N) ++l;
  *s1 = l + B - 9;
  *s2 = l + 6;
}

bool check_dct_matrix(int N, int B, const int8_t* m, char* why, size_t why_len) {
  auto say = [&](const char* fmt, int a, int b, int c) {
    if (why && why_len) snprintf(why, why_len, fmt, a, b, c);
    return false;
  };
  if (N != 4 && N != 8 && N != 16 && N != 32) return say("matrix size %d is not 4, 8, 16 or 32", N, 0, 0);
  if (m[0] != 64) return say("entry (0, 0) is %d, not 64", m[0], 0, 0);
  // The even/odd structure of the DCT at every level L = N, N/2, ..., 2: the level-L matrix is
  // made of rows 0, N/L, 2N/L, ... of m on their first L columns; its row k is even about the
  // middle for even k and odd for odd k.  (Row 0 is then 64 everywhere, and every other row sums
  // to 0.)
  for (int L = N; L >= 2; L /= 2) {
    const int S = N / L;
    for (int k = 0; k < L; ++k) {
      const int8_t* row = m + (size_t)k * S * N;
      for (int n = 0; n < L / 2; ++n) {
        const int a = row[n], b = row[L - 1 - n];
        if ((k % 2 == 0 && a != b) || (k % 2 == 1 && a != -b))
          return say("row %d breaks the DCT symmetry at column %d (level %d)", k * S, n, L);
      }
    }
  }
  // Stage 1 must keep T in 16 bits for samples of up to 10 bits (the tensor-core form splits it
  // into two bytes): max_k sum_n |m[k][n]| (2^B - 1), rounded and shifted by s1, below 2^15.
  if (B <= 10) {
    int s1, s2;
    transform_shifts(N, B, &s1, &s2);
    long long most = 0;
    for (int k = 0; k < N; ++k) {
      long long sum = 0;
      for (int n = 0; n < N; ++n) sum += std::llabs((long long)m[k * N + n]);
      if (sum > most) most = sum;
    }
    const long long t = (most * ((1ll << B) - 1) + (1ll << (s1 - 1))) >> s1;
    if (t > 32767) return say("row sums of |m| reach T = %d for %d-bit samples (limit 32767)", (int)t, B, 0);
  }
  return true;
}

}  // namespace vca
