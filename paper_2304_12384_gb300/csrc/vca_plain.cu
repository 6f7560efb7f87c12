// Plain CUDA-core form of the analyzer's per-block work (Section 2 of the paper: blockwise
// integer DCT, texture energy H and brightness L of every Y, U and V block).
//
// One warp owns 32/N blocks.  Stage 1: lane (j, r) keeps row r of block j in registers
// and produces T[r][k] = (sum_c x[r][c] M[k][c] + 2^(s1-1)) >> s1; stage 2: lane (j, v)
// keeps column v of T in registers and produces Z[u][v] = (sum_r M[u][r] T[r][v] +
// 2^(s2-1)) >> s2, accumulating H_v = sum_u w(u,v) |Z[u][v]| in increasing u with FMA.
// The block energy is then the xor-butterfly sum of H_v over the NK lanes of the block
// (offsets NK/2 .. 1), the same order the tensor-core form uses, so both forms give
// bit-identical H.
#include <cstdint>

#include "vca_internal.h"

namespace vca {
namespace {

constexpr int kWarps = 4;

struct PlainArgs {
  const uint8_t* base[2];  // plane of frame 0, per plane in this launch
  int64_t pitch;           // bytes between rows
  int64_t fstride;         // bytes between frames
  int width, height;       // plane size in samples
  int nbx;
  int64_t C;
  int s1, s2;
  const int8_t* M;         // N x N
  const float* W;          // N x N, W[0] = 0
  float* outH[2];
  float* outL[2];
  int64_t out_fstride;     // floats between frames of block values
  int16_t* zdump[2];       // optional coefficient dump (frame 0 only)
};

// Loads N samples of one block row, repeating the last sample of the plane past its edge.
template <int N, typename Pix>
__device__ __forceinline__ void load_row(const Pix* row, int x0, int width, int (&x)[N]) {
  constexpr int kBytes = N * (int)sizeof(Pix);
  if (x0 + N <= width && (kBytes % 16) == 0) {
    uint32_t words[kBytes / 4];
#pragma unroll
    for (int i = 0; i < kBytes / 16; ++i) {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(row + x0) + i);
      words[4 * i + 0] = q.x;
      words[4 * i + 1] = q.y;
      words[4 * i + 2] = q.z;
      words[4 * i + 3] = q.w;
    }
#pragma unroll
    for (int c = 0; c < N; ++c) {
      if (sizeof(Pix) == 1) {
        x[c] = (words[c / 4] >> (8 * (c % 4))) & 0xff;
      } else {
        x[c] = (words[c / 2] >> (16 * (c % 2))) & 0xffff;
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < N; ++c) x[c] = row[min(x0 + c, width - 1)];
  }
}

template <int N, bool LP, typename Pix>
__global__ void __launch_bounds__(kWarps * 32) plain_kernel(const PlainArgs p) {
  constexpr int NK = LP ? N / 2 : N;
  constexpr int BPW = 32 / N;
  constexpr int BPC = kWarps * BPW;
  __shared__ __align__(16) int sM[N][N];
  __shared__ float sW[NK][NK];
  __shared__ int sT[kWarps][BPW][N][NK + 1];

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  for (int i = tid; i < N * N; i += kWarps * 32) sM[i / N][i % N] = p.M[i];
  for (int i = tid; i < NK * NK; i += kWarps * 32) sW[i / NK][i % NK] = p.W[(i / NK) * N + (i % NK)];
  __syncthreads();

  const int plane = blockIdx.y;
  const int f = blockIdx.z;
  const int j = lane / N;
  const int r = lane % N;
  const int64_t k = (int64_t)blockIdx.x * BPC + warp * BPW + j;
  const bool valid = k < p.C;
  const int bx = valid ? (int)(k % p.nbx) : 0;
  const int by = valid ? (int)(k / p.nbx) : 0;
  const uint8_t* base = p.base[plane] + (int64_t)f * p.fstride;
  const int off1 = 1 << (p.s1 - 1);
  const int off2 = 1 << (p.s2 - 1);

  if (valid) {
    int x[N];
    const int yy = min(by * N + r, p.height - 1);
    load_row<N, Pix>(reinterpret_cast<const Pix*>(base + (int64_t)yy * p.pitch), bx * N, p.width, x);
#pragma unroll 2
    for (int kk = 0; kk < NK; ++kk) {
      int acc = 0;
#pragma unroll
      for (int c = 0; c < N; c += 4) {
        const int4 m = *reinterpret_cast<const int4*>(&sM[kk][c]);
        acc += m.x * x[c] + m.y * x[c + 1] + m.z * x[c + 2] + m.w * x[c + 3];
      }
      sT[warp][j][r][kk] = (acc + off1) >> p.s1;
    }
  }
  __syncwarp();

  float H = 0.0f;
  int z00 = 0;
  const int v = r;
  if (valid && v < NK) {
    int t[N];
#pragma unroll
    for (int rr = 0; rr < N; ++rr) t[rr] = sT[warp][j][rr][v];
    int16_t* zd = p.zdump[plane] && f == 0 ? p.zdump[plane] + k * NK * NK : nullptr;
#pragma unroll 2
    for (int u = 0; u < NK; ++u) {
      int acc = 0;
#pragma unroll
      for (int c = 0; c < N; c += 4) {
        const int4 m = *reinterpret_cast<const int4*>(&sM[u][c]);
        acc += m.x * t[c] + m.y * t[c + 1] + m.z * t[c + 2] + m.w * t[c + 3];
      }
      const int z = (acc + off2) >> p.s2;
      if (u == 0) z00 = z;
      if (zd) zd[u * NK + v] = (int16_t)z;
      H = fmaf(fabsf((float)z), sW[u][v], H);
    }
  }
#pragma unroll
  for (int o = NK / 2; o > 0; o >>= 1) H += __shfl_xor_sync(0xffffffffu, H, o);
  if (valid && v == 0) {
    p.outH[plane][f * p.out_fstride + k] = H;
    p.outL[plane][f * p.out_fstride + k] = __fsqrt_rn((float)z00);
  }
}

template <int N>
cudaError_t launch_planes(const PlainArgs& a, int nplanes, int nframes, bool lp, int bps, cudaStream_t s) {
  constexpr int BPC = kWarps * (32 / N);
  dim3 grid((unsigned)((a.C + BPC - 1) / BPC), nplanes, nframes);
  dim3 block(kWarps * 32);
  if (lp) {
    if (bps == 1) plain_kernel<N, true, uint8_t><<<grid, block, 0, s>>>(a);
    else plain_kernel<N, true, uint16_t><<<grid, block, 0, s>>>(a);
  } else {
    if (bps == 1) plain_kernel<N, false, uint8_t><<<grid, block, 0, s>>>(a);
    else plain_kernel<N, false, uint16_t><<<grid, block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_n(int N, const PlainArgs& a, int nplanes, int nframes, bool lp, int bps, cudaStream_t s) {
  switch (N) {
    case 32: return launch_planes<32>(a, nplanes, nframes, lp, bps, s);
    case 16: return launch_planes<16>(a, nplanes, nframes, lp, bps, s);
    case 8: return launch_planes<8>(a, nplanes, nframes, lp, bps, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_plain(const Geometry& g, const FramePlanes& fp, int nframes, const DeviceTables& t,
                         float* blockvals, int16_t* const zdump[3], cudaStream_t s, int64_t* launches) {
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
  a.W = t.W_y;
  a.outH[0] = blockvals + ROW_H_Y * g.C;
  a.outL[0] = blockvals + ROW_L_Y * g.C;
  a.outH[1] = a.outL[1] = nullptr;
  a.zdump[0] = zdump ? zdump[0] : nullptr;
  a.zdump[1] = nullptr;
  cudaError_t e = launch_n(g.w, a, 1, nframes, g.low_pass, g.bps, s);
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
  a.W = t.W_c;
  a.outH[0] = blockvals + ROW_H_U * g.C;
  a.outL[0] = blockvals + ROW_L_U * g.C;
  a.outH[1] = blockvals + ROW_H_V * g.C;
  a.outL[1] = blockvals + ROW_L_V * g.C;
  a.zdump[0] = zdump ? zdump[1] : nullptr;
  a.zdump[1] = zdump ? zdump[2] : nullptr;
  e = launch_n(g.nc, a, 2, nframes, g.low_pass, g.bps, s);
  if (e != cudaSuccess) return e;
  ++*launches;
  return cudaSuccess;
}

}  // namespace vca
