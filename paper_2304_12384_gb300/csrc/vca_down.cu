// Downsample reading of the low-pass option (Section 2 item (3) of the paper: the features
// "evaluated on the video spatially downsampled by a factor of two"): every plane of every frame
// is halved in each direction, out[i][j] = (p[2i][2j] + p[2i][2j+1] + p[2i+1][2j] + p[2i+1][2j+1]
// + 2) >> 2, a plane of odd height or width repeating its last row or column; the analysis then
// runs on the halved planes with half-size blocks.
#include "vca_internal.h"

namespace vca {
namespace {

constexpr int kThreads = 256;
constexpr int kOut = 4;  // output samples per thread

template <typename Pix>
__global__ void __launch_bounds__(kThreads) down_kernel(const DownArgs a) {
  const DownPlane& P = a.p[blockIdx.y];
  const int groups = (P.wd + kOut - 1) / kOut;
  const int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  if (idx >= (int64_t)groups * P.hd) return;
  const int i = (int)(idx / groups);
  const int j0 = (int)(idx - (int64_t)i * groups) * kOut;
  const uint8_t* src = P.src + (int64_t)blockIdx.z * P.src_fstride;
  uint8_t* dst = P.dst + (int64_t)blockIdx.z * P.dst_fstride;
  const Pix* r0 = reinterpret_cast<const Pix*>(src + (int64_t)min(2 * i, P.h - 1) * P.src_pitch);
  const Pix* r1 = reinterpret_cast<const Pix*>(src + (int64_t)min(2 * i + 1, P.h - 1) * P.src_pitch);
  Pix* out = reinterpret_cast<Pix*>(dst + (int64_t)i * P.dst_pitch);
#pragma unroll
  for (int t = 0; t < kOut; ++t) {
    const int j = j0 + t;
    if (j >= P.wd) break;
    const int c0 = min(2 * j, P.w - 1), c1 = min(2 * j + 1, P.w - 1);
    const unsigned s = (unsigned)r0[c0] + (unsigned)r0[c1] + (unsigned)r1[c0] + (unsigned)r1[c1];
    out[j] = (Pix)((s + 2) >> 2);
  }
}

}  // namespace

cudaError_t launch_downsample(const DownArgs& a, int nframes, int bps, cudaStream_t s) {
  if (nframes <= 0) return cudaSuccess;
  int64_t most = 0;
  for (int p = 0; p < 3; ++p) {
    const int64_t n = (int64_t)((a.p[p].wd + kOut - 1) / kOut) * a.p[p].hd;
    if (n > most) most = n;
  }
  const dim3 grid((unsigned)((most + kThreads - 1) / kThreads), 3, (unsigned)nframes);
  if (bps == 1)
    down_kernel<uint8_t><<<grid, kThreads, 0, s>>>(a);
  else
    down_kernel<uint16_t><<<grid, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace vca
