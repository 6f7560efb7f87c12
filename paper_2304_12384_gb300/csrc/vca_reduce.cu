// Frame reduction of the analyzer (Section 2 of the paper: the seven per-frame features).
//
// One CTA per frame sums the per-block values in FP64 in a fixed order (thread i takes
// blocks i, i + 256, ...; then a fixed shared-memory tree), so the features are
// deterministic:
//   E_P = sum_k H_{P,k} / (C N_P^2), L_P = sum_k L_{P,k} / C,
//   h_t = sum_k |H_{Y,k,t} - H_{Y,k,t-1}| / (C w^2), and h = 0 without a previous frame.
// The CTA of the last frame also writes that frame's luma energies as the next call's
// previous-frame state (into a buffer distinct from the one read here).
#include "vca_internal.h"

namespace vca {
namespace {

constexpr int kThreads = 256;
constexpr int kSums = 7;  // H_Y, L_Y, H_U, L_U, H_V, L_V, |dH_Y|

struct ReduceArgs {
  const float* blockvals;
  const float* prevH_in;
  float* prevH_out;
  double* feats;
  int64_t C;
  int nframes;
  int has_prev;
  double normY, normC;  // C w^2 and C (w/2)^2
};

__global__ void __launch_bounds__(kThreads) reduce_kernel(const ReduceArgs a) {
  __shared__ double part[kSums][kThreads];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  const int64_t C = a.C;
  const float* bv = a.blockvals + (int64_t)f * N_ROWS * C;
  const float* prev = f > 0 ? a.blockvals + (int64_t)(f - 1) * N_ROWS * C + ROW_H_Y * C : a.prevH_in;
  const bool has_prev = f > 0 || a.has_prev;

  double s[kSums] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t k = tid; k < C; k += kThreads) {
#pragma unroll
    for (int r = 0; r < N_ROWS; ++r) s[r] += (double)bv[r * C + k];
    if (has_prev) s[6] += fabs((double)bv[ROW_H_Y * C + k] - (double)prev[k]);
  }
#pragma unroll
  for (int r = 0; r < kSums; ++r) part[r][tid] = s[r];
  __syncthreads();
  for (int half = kThreads / 2; half > 0; half >>= 1) {
    if (tid < half) {
#pragma unroll
      for (int r = 0; r < kSums; ++r) part[r][tid] += part[r][tid + half];
    }
    __syncthreads();
  }
  if (tid == 0) {
    double* out = a.feats + (int64_t)f * FEAT_STRIDE;
    const double Cd = (double)C;
    out[0] = part[ROW_H_Y][0] / a.normY;  // E_Y
    out[1] = part[6][0] / a.normY;        // h
    out[2] = part[ROW_L_Y][0] / Cd;       // L_Y
    out[3] = part[ROW_H_U][0] / a.normC;  // E_U
    out[4] = part[ROW_H_V][0] / a.normC;  // E_V
    out[5] = part[ROW_L_U][0] / Cd;       // L_U
    out[6] = part[ROW_L_V][0] / Cd;       // L_V
    out[7] = 0.0;
  }
  if (f == a.nframes - 1) {
    for (int64_t k = tid; k < C; k += kThreads) a.prevH_out[k] = bv[ROW_H_Y * C + k];
  }
}

}  // namespace

cudaError_t launch_reduce(const Geometry& g, int nframes, const float* blockvals, const float* prevH_in,
                          int has_prev, float* prevH_out, double* feats, cudaStream_t s, int64_t* launches) {
  if (nframes <= 0) return cudaSuccess;
  ReduceArgs a{};
  a.blockvals = blockvals;
  a.prevH_in = prevH_in;
  a.prevH_out = prevH_out;
  a.feats = feats;
  a.C = g.C;
  a.nframes = nframes;
  a.has_prev = has_prev;
  a.normY = (double)g.C * g.w * g.w;
  a.normC = (double)g.C * g.nc * g.nc;
  reduce_kernel<<<nframes, kThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) ++*launches;
  return e;
}

}  // namespace vca
