// Plain CUDA-core form of the analyzer's per-block work (Section 2 of the paper): one launch for
// the luma plane and one for both chroma planes of a batch of frames, each CTA running the block
// routine of vca_plain.cuh on BPC consecutive blocks.
#include <cstdint>

#include "vca_plain.cuh"

namespace vca {
namespace {

template <int NV, int NH, bool LP, typename Pix, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) plain_kernel(const PlainArgs p) {
  __shared__ PlainSmem<NV, NH, LP, WARPS> sh;
  plain_blocks<NV, NH, LP, Pix, WARPS>(p, blockIdx.y, blockIdx.z, blockIdx.x, sh);
}

template <int NV, int NH, int WARPS>
cudaError_t launch_planes(const PlainArgs& a, int nplanes, int nframes, bool lp, int bps, cudaStream_t s) {
  constexpr int BPC = WARPS * (32 / NV);
  dim3 grid((unsigned)((a.C + BPC - 1) / BPC), nplanes, nframes);
  dim3 block(WARPS * 32);
  if (lp) {
    if (bps == 1) plain_kernel<NV, NH, true, uint8_t, WARPS><<<grid, block, 0, s>>>(a);
    else plain_kernel<NV, NH, true, uint16_t, WARPS><<<grid, block, 0, s>>>(a);
  } else {
    if (bps == 1) plain_kernel<NV, NH, false, uint8_t, WARPS><<<grid, block, 0, s>>>(a);
    else plain_kernel<NV, NH, false, uint16_t, WARPS><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// Blocks of NV rows and NH columns: square (NV = NH in {32, 16, 8, 4}) or the 4:2:2 chroma
// shapes (NV = 2 NH, NV in {32, 16, 8}).
template <int WARPS>
cudaError_t launch_nw(int NV, int NH, const PlainArgs& a, int nplanes, int nframes, bool lp, int bps,
                      cudaStream_t s) {
  if (NV == NH) {
    switch (NV) {
      case 32: return launch_planes<32, 32, WARPS>(a, nplanes, nframes, lp, bps, s);
      case 16: return launch_planes<16, 16, WARPS>(a, nplanes, nframes, lp, bps, s);
      case 8: return launch_planes<8, 8, WARPS>(a, nplanes, nframes, lp, bps, s);
      case 4: return launch_planes<4, 4, WARPS>(a, nplanes, nframes, lp, bps, s);
      default: return cudaErrorInvalidValue;
    }
  }
  if (NV == 2 * NH) {
    switch (NV) {
      case 32: return launch_planes<32, 16, WARPS>(a, nplanes, nframes, lp, bps, s);
      case 16: return launch_planes<16, 8, WARPS>(a, nplanes, nframes, lp, bps, s);
      case 8: return launch_planes<8, 4, WARPS>(a, nplanes, nframes, lp, bps, s);
      default: return cudaErrorInvalidValue;
    }
  }
  return cudaErrorInvalidValue;
}

// warps per CTA: 2, 4 (the default) or 8
cudaError_t launch_n(int NV, int NH, const PlainArgs& a, int nplanes, int nframes, bool lp, int bps,
                     cudaStream_t s, int warps) {
  switch (warps) {
    case 2: return launch_nw<2>(NV, NH, a, nplanes, nframes, lp, bps, s);
    case 4: return launch_nw<4>(NV, NH, a, nplanes, nframes, lp, bps, s);
    case 8: return launch_nw<8>(NV, NH, a, nplanes, nframes, lp, bps, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_plain(const Geometry& g, const FramePlanes& fp, int nframes, const DeviceTables& t,
                         float* blockvals, int16_t* const zdump[3], cudaStream_t s, int64_t* launches, int warps) {
  if (nframes <= 0) return cudaSuccess;
  PlainArgs a{};
  a.nbx = g.nbx;
  a.C = g.C;
  a.out_fstride = (int64_t)N_ROWS * g.C;

  // Luma.
  a.base[0] = fp.y;
  a.base[1] = nullptr;
  a.pitch = fp.pitch_y;
  a.fstride = fp.fstride_y;
  a.width = g.W;
  a.height = g.H;
  a.s1 = g.s1y;
  a.s2 = g.s2y;
  a.M = t.M_y;
  a.M2 = t.M_y;
  a.W = t.W_y;
  a.outH[0] = blockvals + ROW_H_Y * g.C;
  a.outL[0] = blockvals + ROW_L_Y * g.C;
  a.outH[1] = a.outL[1] = nullptr;
  a.zdump[0] = zdump ? zdump[0] : nullptr;
  a.zdump[1] = nullptr;
  cudaError_t e = launch_n(g.w, g.w, a, 1, nframes, g.low_pass, g.bps, s, warps);
  if (e != cudaSuccess) return e;
  ++*launches;

  // Chroma: U and V in one launch (grid.y selects the plane).
  a.base[0] = fp.u;
  a.base[1] = fp.v;
  a.pitch = fp.pitch_uv;
  a.fstride = fp.fstride_uv;
  a.width = g.cw;
  a.height = g.ch;
  a.s1 = g.s1c;
  a.s2 = g.s2c;
  a.M = t.M_c;
  a.M2 = t.M_cv;
  a.W = t.W_c;
  a.outH[0] = blockvals + ROW_H_U * g.C;
  a.outL[0] = blockvals + ROW_L_U * g.C;
  a.outH[1] = blockvals + ROW_H_V * g.C;
  a.outL[1] = blockvals + ROW_L_V * g.C;
  a.zdump[0] = zdump ? zdump[1] : nullptr;
  a.zdump[1] = zdump ? zdump[2] : nullptr;
  e = launch_n(g.ncv, g.nc, a, 2, nframes, g.low_pass, g.bps, s, warps);
  if (e != cudaSuccess) return e;
  ++*launches;
  return cudaSuccess;
}

}  // namespace vca
