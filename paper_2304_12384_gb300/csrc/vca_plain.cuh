// The plain CUDA-core block routine (Section 2 of the paper: blockwise integer DCT, texture energy
// H and brightness L of every Y, U and V block), shared by the single-analyzer kernel and the
// batched multi-stream kernel.
//
// One warp owns 32/N blocks.  Stage 1: lane (j, r) keeps row r of block j in registers
// and produces T[r][k] = (sum_c x[r][c] M[k][c] + 2^(s1-1)) >> s1; stage 2: lane (j, v)
// keeps column v of T in registers and produces Z[u][v] = (sum_r M[u][r] T[r][v] +
// 2^(s2-1)) >> s2, accumulating H_v = sum_u w(u,v) |Z[u][v]| in increasing u with FMA.
// 4:2:2 chroma blocks are rectangular (w rows of w/2 samples): the rows take the (w/2)-point
// matrix and the columns the w-point one, each stage with the shift of its own length.
// Both sums use the even/odd butterfly (Butterfly below), which equals the matrix form exactly.
// The block energy is then the xor-butterfly sum of H_v over the NK lanes of the block
// (offsets NK/2 .. 1), the same order the tensor-core form uses, so both forms give
// bit-identical H.
#pragma once

#include <cstdint>

#include "vca_internal.h"

namespace vca {

constexpr int kWarps = 4;

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

// y[k] = sum_n M_N[k][n] x[n] for k < NK (N a power of two), by even/odd decomposition: with
// e[n] = x[n] + x[N-1-n] and o[n] = x[n] - x[N-1-n] (n < N/2), the even outputs are the
// N/2-point transform of e (the even rows of M_N are M_{N/2} on the first N/2 columns) and the
// odd outputs apply the odd rows of M_N, first N/2 columns, to o; M_1 = [64].  M points at the
// full matrix in shared memory (LD ints per row); at recursion step S, row k of the current
// matrix is row k * S of the full one.  Integer arithmetic, so the result equals the matrix form
// exactly.
template <int N, int NK, int S, int LD>
struct Butterfly {
  static __device__ __forceinline__ void run(const int (&x)[N], int (&y)[NK], const int* M) {
    constexpr int H = N / 2;
    constexpr int NKE = (NK + 1) / 2;
    int e[H], o[H];
#pragma unroll
    for (int n = 0; n < H; ++n) {
      e[n] = x[n] + x[N - 1 - n];
      o[n] = x[n] - x[N - 1 - n];
    }
    int ye[NKE];
    Butterfly<H, NKE, 2 * S, LD>::run(e, ye, M);
#pragma unroll
    for (int k = 0; 2 * k < NK; ++k) y[2 * k] = ye[k];
#pragma unroll
    for (int k = 1; k < NK; k += 2) {
      const int* row = M + k * S * LD;
      int acc = 0;
      if (H >= 4) {
#pragma unroll
        for (int n = 0; n < H; n += 4) {
          const int4 m = *reinterpret_cast<const int4*>(row + n);
          acc += m.x * o[n] + m.y * o[n + 1] + m.z * o[n + 2] + m.w * o[n + 3];
        }
      } else {
#pragma unroll
        for (int n = 0; n < H; ++n) acc += row[n] * o[n];
      }
      y[k] = acc;
    }
  }
};

template <int NK, int S, int LD>
struct Butterfly<1, NK, S, LD> {
  static __device__ __forceinline__ void run(const int (&x)[1], int (&y)[NK], const int*) { y[0] = 64 * x[0]; }
};

// Shared memory of one CTA of the block routine (WARPS warps) for blocks of NV rows and NH columns:
// the row matrix (NH x NH), the column matrix when the blocks are not square (NV x NV), the weights
// of the kept coefficients and each warp's stage-1 output.
template <int NV, int NH, bool LP, int WARPS = kWarps>
struct PlainSmem {
  static constexpr int NKV = LP ? NV / 2 : NV;
  static constexpr int NKH = LP ? NH / 2 : NH;
  static constexpr int BPW = 32 / NV;
  static constexpr int NM2 = NV != NH ? NV : 1;
  __align__(16) int M[NH][NH];
  __align__(16) int M2[NM2][NM2];
  float W[NKV][NKH];
  int T[WARPS][BPW][NV][NKH + 1];
};

// Blocks chunk * BPC .. chunk * BPC + BPC - 1 of plane `plane` of frame f (one CTA of WARPS
// warps, BPC = WARPS * 32/NV; the warp owns 32/NV blocks).  Stage 1: lane (j, r) keeps row r of
// block j (NH samples) in registers and produces T[r][k] with the NH-point matrix; stage 2: lane
// (j, v) keeps column v of T (NV values) and produces Z[u][v] with the NV-point matrix,
// accumulating H_v.  Square blocks (NV = NH) use one matrix for both stages.
template <int NV, int NH, bool LP, typename Pix, int WARPS = kWarps>
__device__ __forceinline__ void plain_blocks(const PlainArgs& p, int plane, int f, int64_t chunk,
                                             PlainSmem<NV, NH, LP, WARPS>& sh) {
  constexpr int NKV = LP ? NV / 2 : NV;
  constexpr int NKH = LP ? NH / 2 : NH;
  constexpr int BPW = 32 / NV;
  constexpr int BPC = WARPS * BPW;
  auto& sT = sh.T;

  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  for (int i = tid; i < NH * NH; i += WARPS * 32) sh.M[i / NH][i % NH] = p.M[i];
  if constexpr (NV != NH)
    for (int i = tid; i < NV * NV; i += WARPS * 32) sh.M2[i / NV][i % NV] = p.M2[i];
  for (int i = tid; i < NKV * NKH; i += WARPS * 32) sh.W[i / NKH][i % NKH] = p.W[(i / NKH) * NH + (i % NKH)];
  __syncthreads();
  const int* m1 = &sh.M[0][0];
  const int* m2;
  if constexpr (NV != NH) m2 = &sh.M2[0][0];
  else m2 = m1;

  const int j = lane / NV;
  const int r = lane % NV;
  const int64_t k = chunk * BPC + warp * BPW + j;
  const bool valid = k < p.C;
  const int bx = valid ? (int)(k % p.nbx) : 0;
  const int by = valid ? (int)(k / p.nbx) : 0;
  const uint8_t* base = p.base[plane] + (int64_t)f * p.fstride;
  const int off1 = 1 << (p.s1 - 1);
  const int off2 = 1 << (p.s2 - 1);

  if (valid) {
    int x[NH];
    const int yy = min(by * NV + r, p.height - 1);
    load_row<NH, Pix>(reinterpret_cast<const Pix*>(base + (int64_t)yy * p.pitch), bx * NH, p.width, x);
    int y[NKH];
    Butterfly<NH, NKH, 1, NH>::run(x, y, m1);
#pragma unroll
    for (int kk = 0; kk < NKH; ++kk) sT[warp][j][r][kk] = (y[kk] + off1) >> p.s1;
  }
  __syncwarp();

  float H = 0.0f;
  int z00 = 0;
  const int v = r;
  if (valid && v < NKH) {
    int t[NV];
#pragma unroll
    for (int rr = 0; rr < NV; ++rr) t[rr] = sT[warp][j][rr][v];
    int16_t* zd = p.zdump[plane] && f == 0 ? p.zdump[plane] + k * NKV * NKH : nullptr;
    int zr[NKV];
    Butterfly<NV, NKV, 1, NV>::run(t, zr, m2);
#pragma unroll
    for (int u = 0; u < NKV; ++u) {
      const int z = (zr[u] + off2) >> p.s2;
      if (u == 0) z00 = z;
      if (zd) zd[u * NKH + v] = (int16_t)z;
      H = fmaf(fabsf((float)z), sh.W[u][v], H);
    }
  }
#pragma unroll
  for (int o = NKH / 2; o > 0; o >>= 1) H += __shfl_xor_sync(0xffffffffu, H, o);
  if (valid && v == 0) {
    p.outH[plane][f * p.out_fstride + k] = H;
    p.outL[plane][f * p.out_fstride + k] = __fsqrt_rn((float)z00);
  }
}


}  // namespace vca
