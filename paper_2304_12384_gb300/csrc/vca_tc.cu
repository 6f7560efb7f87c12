// Tensor-core form of the analyzer's per-block work (Section 2 of the paper: integer DCT of
// every Y, U, V block, texture energy H and brightness L; Section 2 item (3): low-pass).
//
// Persistent kernel, one CTA per SM, warp-specialised:
//   warp 0   TMA producer: one 128x128 luma + two 64x64 chroma tiles per work item into a
//            4-stage ring (128-byte / 64-byte swizzled);
//   warp 1   TMEM owner and MMA issuer (tcgen05.mma kind::f16, FP32 accumulate);
//   warps 2-5 workers, one per TMEM lane quarter.
//
// A "job" is 128 stage-2 rows: 8 (low-pass) or 4 luma 32x32 blocks, or 16 / 8 chroma 16x16
// blocks.  Per job, through 4 TMEM slots and 2 shared-memory slots:
//   convert   raw u8 row -> fp16 (1024 + x, one PRMT per two samples) written to TMEM as the
//             A operand; accumulators pre-set with the rounding offsets and magic constants;
//   stage 1   T' = X M^T + c  (A from TMEM, M from shared memory), exact integers in FP32;
//   epilogue1 T = floor(T'/2^s1) by one round-down FMA whose magic constant leaves
//             U = T + 32768 in the low 16 bits and 0x64 in byte 2, so two PRMTs give the
//             fp16 pairs (1024 + U_lo8, 1024 + U_hi8); stored MN-major (128-byte swizzle)
//             as the stage-2 A operand -- the row/column transpose is the layout;
//   stage 2   S_hi, S_lo = M T_hi, M T_lo (A MN-major from shared memory);
//   epilogue2 Z = floor((256 S_hi + S_lo + 2^(s2-1)) / 2^s2) by two round-down FMAs, then
//             H_v = sum_u w(u,v) |Z| in increasing u and an xor tree over v.
// Every partial sum is an integer below 2^24 in magnitude (or in [2^23, 2^24) for the
// pre-offset accumulators), so the FP32 tensor-core accumulation is exact and Z is
// bit-identical to the integer definition; H uses the same FP32 order as the CUDA-core form.
//
// Every wait is bounded (about two seconds); on timeout the kernel raises a flag in *err,
// stops, waits for its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstring>
#include <mutex>

#include "vca_internal.h"
#include "vca_ptx.cuh"

namespace vca {
namespace {

using namespace ptx;

constexpr int kStages = 4;
constexpr int kRawY = 128 * 128;
constexpr int kRawC = 64 * 64;
constexpr int kStageBytes = kRawY + 2 * kRawC;
constexpr int kA2Bytes = 8192;  // one operand (hi or lo) of one job: 128 rows x 32 K x fp16
constexpr int OFF_RAW = 0;
constexpr int OFF_A2 = kStages * kStageBytes;
constexpr int OFF_BL = OFF_A2 + 2 * 2 * kA2Bytes;
constexpr int OFF_BC = OFF_BL + 2048;
constexpr int OFF_BAR = OFF_BC + 512;
constexpr int OFF_MISC = OFF_BAR + 32 * 8;
constexpr int kSmemBytes = OFF_MISC + 64 + 1024;  // + slack to align the base to 1024

// barrier indices
constexpr int B_RAW_FULL = 0, B_RAW_EMPTY = 4, B_A1 = 8, B_D1 = 12, B_A2 = 16, B_D2 = 18, B_DRAIN = 22;

constexpr int kThreads = 192;
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitNs = 2000000000ull;

// FP32 magic constants (see the file comment).
constexpr float kT1 = 14974976.0f;  // 2^23 + 0x640000 + 0x8000
constexpr float kK1 = 12582912.0f;  // 1.5 * 2^23
constexpr uint32_t kSel6464 = 0x64646464u;

struct TcParams {
  int W, H, cw, ch;
  int nbx, nby;
  int tiles_x, tiles_y;
  int nframes;
  int total_items;
  int64_t C;
  int64_t out_fstride;
  float* blockvals;
  int16_t* zdump[3];
  const int8_t* M_y;
  const int8_t* M_c;
  const float* W_y;
  const float* W_c;
  int* err;
};

template <int Nb, bool LP>
struct PC {
  static constexpr int NK = LP ? Nb / 2 : Nb;     // coefficients kept per dimension
  static constexpr int N1 = NK < 16 ? 16 : NK;    // MMA N of both stages
  static constexpr int BPG1 = 128 / Nb;           // blocks per stage-1 group (128 rows)
  static constexpr int BPG2 = 128 / NK;           // blocks per job (128 stage-2 rows)
  static constexpr int G = BPG2 / BPG1;           // stage-1 groups per job
  static constexpr int JOBS = 16 / BPG2;          // jobs of this plane per tile
  static constexpr int KS = Nb / 16;              // K = 16 steps
  static constexpr int A1COLS = Nb / 2;           // TMEM columns of one group's A operand
};

template <bool LP>
struct Jobs {
  using L = PC<32, LP>;
  using Cc = PC<16, LP>;
  static constexpr int PER_TILE = L::JOBS + 2 * Cc::JOBS;
};

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

struct Ctl {
  uint64_t* bars;
  volatile int* abort;
  int* err;
};

// Bounded wait: false on timeout (flag raised) or when another role aborted.
__device__ bool wait_bar(const Ctl& c, int idx, uint32_t parity, int code, bool ignore_abort = false) {
  uint64_t t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(&c.bars[idx], parity)) return true;
    if ((i & 63) == 63) {
      if (!ignore_abort && *c.abort) return false;
      const uint64_t t = now_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > kWaitNs) {
        *c.abort = 1;
        atomicOr(c.err, code);
        return false;
      }
    }
  }
}

// Stage-1 operand conversion for one stage-1 group: this thread's row of 2 * A1COLS samples.
template <int Nb>
__device__ __forceinline__ void load_row_fp16(const uint8_t* raw, int y, int x, int w_rem, uint32_t (&out)[Nb / 2]) {
  constexpr int kRow = Nb == 32 ? 128 : 64;  // raw tile row pitch in bytes
  uint32_t words[Nb / 4];
  const uint32_t base = smem_u32(raw);
  if (x + Nb <= w_rem) {
#pragma unroll
    for (int c = 0; c < Nb / 16; ++c) {
      const int chunk = (x >> 4) + c;
      const int sw = Nb == 32 ? (chunk ^ (y & 7)) : (chunk ^ ((y >> 1) & 3));
      const uint4 q = lds128(base + y * kRow + (sw << 4));
      words[4 * c + 0] = q.x;
      words[4 * c + 1] = q.y;
      words[4 * c + 2] = q.z;
      words[4 * c + 3] = q.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < Nb / 4; ++i) words[i] = 0;
#pragma unroll
    for (int c = 0; c < Nb; ++c) {
      const int xx = min(x + c, w_rem - 1);
      const int chunk = xx >> 4;
      const int sw = Nb == 32 ? (chunk ^ (y & 7)) : (chunk ^ ((y >> 1) & 3));
      const uint32_t b = lds_u8(base + y * kRow + (sw << 4) + (xx & 15));
      words[c >> 2] |= b << (8 * (c & 3));
    }
  }
#pragma unroll
  for (int i = 0; i < Nb / 4; ++i) {
    out[2 * i] = prmt(words[i], kSel6464, 0x5140);
    out[2 * i + 1] = prmt(words[i], kSel6464, 0x5342);
  }
}

template <int N>
__device__ __forceinline__ void fill_cols(uint32_t taddr, float first, float rest) {
  uint32_t v[N];
  v[0] = __float_as_uint(first);
#pragma unroll
  for (int i = 1; i < N; ++i) v[i] = __float_as_uint(rest);
  tmem_st<N>(taddr, v);
}

struct JobRef {
  int plane;  // 0 Y, 1 U, 2 V
  int jp;     // job index within the plane's tile
  int item;   // work item (frame, tile)
  int slot;   // TMEM slot
};

template <bool LP>
__device__ __forceinline__ JobRef job_ref(int it, int cta, int grid) {
  constexpr int JPT = Jobs<LP>::PER_TILE;
  constexpr int JL = PC<32, LP>::JOBS;
  constexpr int JC = PC<16, LP>::JOBS;
  JobRef r;
  const int t = it / JPT;
  const int j = it - t * JPT;
  r.item = cta + t * grid;
  if (j < JL) {
    r.plane = 0;
    r.jp = j;
  } else if (j < JL + JC) {
    r.plane = 1;
    r.jp = j - JL;
  } else {
    r.plane = 2;
    r.jp = j - JL - JC;
  }
  r.slot = it & 3;
  return r;
}

// ---- worker phases ----------------------------------------------------------

template <int Nb, bool LP>
__device__ void convert_job(const TcParams& p, const uint8_t* raw_plane, int jp, int tile_x, int tile_y, int plane_w,
                            int plane_h, uint32_t tslot, int q, int lane, float c0, float c, float hi0, float lo) {
  using P = PC<Nb, LP>;
  const uint32_t lanebase = (uint32_t)(32 * q) << 16;
  const int l = 32 * q + lane;
  const int bg = l / Nb;
  const int r = l % Nb;
  const int h_rem = plane_h - tile_y * 4 * Nb;
  const int w_rem = plane_w - tile_x * 4 * Nb;
#pragma unroll
  for (int g = 0; g < P::G; ++g) {
    const int idx = jp * P::BPG2 + g * P::BPG1 + bg;
    int y = (idx >> 2) * Nb + r;
    if (y >= h_rem) y = h_rem - 1;
    const int x = (idx & 3) * Nb;
    uint32_t a[Nb / 2];
    load_row_fp16<Nb>(raw_plane, y, x, w_rem, a);
    tmem_st<Nb / 2>(tslot + lanebase + g * P::A1COLS, a);
    fill_cols<P::N1>(tslot + lanebase + 32 + g * P::N1, c0, c);
  }
  fill_cols<P::N1>(tslot + lanebase + 64, hi0, kK1);
  fill_cols<P::N1>(tslot + lanebase + 96, lo, lo);
}

template <int Nb, bool LP>
__device__ void epilogue1(uint32_t tslot, uint32_t a2hi, uint32_t a2lo, int q, int lane, float s1inv) {
  using P = PC<Nb, LP>;
  constexpr int NK = P::NK;
  const uint32_t lanebase = (uint32_t)(32 * q) << 16;
  const int l = 32 * q + lane;
  const int bg = l / Nb;
  const int r = l % Nb;
#pragma unroll
  for (int g = 0; g < P::G; ++g) {
    uint32_t acc[NK];
    tmem_ld<NK>(tslot + lanebase + 32 + g * P::N1, acc);
    tmem_wait_ld();
    uint32_t hi[NK / 2], lo[NK / 2];
#pragma unroll
    for (int k = 0; k < NK; k += 2) {
      const uint32_t za = __float_as_uint(__fmaf_rd(__uint_as_float(acc[k]), s1inv, kT1));
      const uint32_t zb = __float_as_uint(__fmaf_rd(__uint_as_float(acc[k + 1]), s1inv, kT1));
      lo[k / 2] = prmt(za, zb, 0x6420);
      hi[k / 2] = prmt(za, zb, 0x6521);
    }
    const int m0 = (g * P::BPG1 + bg) * NK;
    const uint32_t rowoff = (uint32_t)((r >> 3) * 2048 + (r & 7) * 128);
#pragma unroll
    for (int c = 0; c < NK / 8; ++c) {
      const int m = m0 + 8 * c;
      const uint32_t off = rowoff + (uint32_t)((m >> 6) * 1024) + (uint32_t)(((((m & 63) >> 3) ^ (r & 7))) << 4);
      sts128(a2hi + off, hi[4 * c], hi[4 * c + 1], hi[4 * c + 2], hi[4 * c + 3]);
      sts128(a2lo + off, lo[4 * c], lo[4 * c + 1], lo[4 * c + 2], lo[4 * c + 3]);
    }
  }
}

template <int Nb, bool LP, bool DUMP>
__device__ void epilogue2(const TcParams& p, uint32_t tslot, int plane, int jp, int f, int tile_x, int tile_y, int q,
                          int lane, const float (&wts)[PC<Nb, LP>::NK], float einv, float c2) {
  using P = PC<Nb, LP>;
  constexpr int NK = P::NK;
  const uint32_t lanebase = (uint32_t)(32 * q) << 16;
  uint32_t hi[NK], lo[NK];
  tmem_ld<NK>(tslot + lanebase + 64, hi);
  tmem_ld<NK>(tslot + lanebase + 96, lo);
  tmem_wait_ld();
  const int m = 32 * q + lane;
  const int b2 = m / NK;
  const int v = m % NK;
  const int idx = jp * P::BPG2 + b2;
  const int bx = tile_x * 4 + (idx & 3);
  const int by = tile_y * 4 + (idx >> 2);
  const bool valid = bx < p.nbx && by < p.nby;
  const int64_t k = (int64_t)by * p.nbx + bx;
  int16_t* zd = nullptr;
  if (DUMP) zd = (valid && f == 0) ? p.zdump[plane] + k * NK * NK : nullptr;
  float H = 0.0f, z00 = 0.0f;
#pragma unroll
  for (int u = 0; u < NK; ++u) {
    const float w = __fmaf_rd(__uint_as_float(lo[u]), 0.00390625f, __uint_as_float(hi[u]));
    const float z = __fmaf_rd(w, einv, c2) - kK1;
    if (u == 0) z00 = z;
    if (DUMP && zd) zd[u * NK + v] = (int16_t)z;
    H = fmaf(fabsf(z), wts[u], H);
  }
#pragma unroll
  for (int o = NK / 2; o > 0; o >>= 1) H += __shfl_xor_sync(0xffffffffu, H, o);
  if (valid && v == 0) {
    float* out = p.blockvals + (int64_t)f * p.out_fstride;
    out[(2 * plane) * p.C + k] = H;
    out[(2 * plane + 1) * p.C + k] = __fsqrt_rn(z00);
  }
}

// ---- the kernel --------------------------------------------------------------

template <bool LP, bool DUMP>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(const __grid_constant__ CUtensorMap mapY, const __grid_constant__ CUtensorMap mapU,
              const __grid_constant__ CUtensorMap mapV, const TcParams p) {
  using L = PC<32, LP>;
  using Cc = PC<16, LP>;
  constexpr int JPT = Jobs<LP>::PER_TILE;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = (uint64_t*)(sm + OFF_BAR);
  uint32_t* tmem_slot = (uint32_t*)(sm + OFF_MISC);
  volatile int* abort_flag = (volatile int*)(sm + OFF_MISC + 4);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int cta = blockIdx.x;
  const int grid = gridDim.x;
  const int n_items = cta < p.total_items ? (p.total_items - cta + grid - 1) / grid : 0;
  const int n_jobs = n_items * JPT;
  const int tiles_per_frame = p.tiles_x * p.tiles_y;
  Ctl ctl{bars, abort_flag, p.err};

  // Constant B operands (the integer DCT matrices as fp16), K-major without swizzle:
  // element (n, k) at (n/8)*SBO + (k/8)*128 + (n%8)*16 + (k%8)*2.
  for (int i = tid; i < L::N1 * 32; i += kThreads) {
    const int n = i >> 5, kk = i & 31;
    const __half h = __float2half_rn((float)p.M_y[n * 32 + kk]);
    *(__half*)(sm + OFF_BL + (n >> 3) * 512 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) = h;
  }
  for (int i = tid; i < 16 * 16; i += kThreads) {
    const int n = i >> 4, kk = i & 15;
    const __half h = __float2half_rn((float)p.M_c[n * 16 + kk]);
    *(__half*)(sm + OFF_BC + (n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) = h;
  }
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(&bars[B_RAW_FULL + i], 1);
      mbar_init(&bars[B_RAW_EMPTY + i], 4);
    }
    for (int i = 0; i < 4; ++i) {
      mbar_init(&bars[B_A1 + i], 4);
      mbar_init(&bars[B_D1 + i], 1);
      mbar_init(&bars[B_D2 + i], 1);
    }
    for (int i = 0; i < 2; ++i) mbar_init(&bars[B_A2 + i], 4);
    mbar_init(&bars[B_DRAIN], 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0) {
    prefetch_tensormap(&mapY);
    prefetch_tensormap(&mapU);
    prefetch_tensormap(&mapV);
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, kTmemCols);
    tmem_relinquish();
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t sbase = smem_u32(sm);

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      int issued = 0;
      for (int t = 0; t < n_items; ++t) {
        const int stage = t % kStages;
        if (t >= kStages && !wait_bar(ctl, B_RAW_EMPTY + stage, ((t / kStages) - 1) & 1, 1)) break;
        const int item = cta + t * grid;
        const int f = item / tiles_per_frame;
        const int ti = item - f * tiles_per_frame;
        const int tx = ti % p.tiles_x, ty = ti / p.tiles_x;
        uint8_t* dst = sm + OFF_RAW + stage * kStageBytes;
        mbar_arrive_expect_tx(&bars[B_RAW_FULL + stage], kStageBytes);
        tma_load_3d(dst, &mapY, tx * 128, ty * 128, f, &bars[B_RAW_FULL + stage]);
        tma_load_3d(dst + kRawY, &mapU, tx * 64, ty * 64, f, &bars[B_RAW_FULL + stage]);
        tma_load_3d(dst + kRawY + kRawC, &mapV, tx * 64, ty * 64, f, &bars[B_RAW_FULL + stage]);
        ++issued;
      }
      if (*abort_flag) {
        // Let every copy this CTA issued land before the CTA's shared memory goes away.
        for (int t = (issued > kStages ? issued - kStages : 0); t < issued; ++t)
          wait_bar(ctl, B_RAW_FULL + (t % kStages), (t / kStages) & 1, 1, true);
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t bl = sbase + OFF_BL, bc = sbase + OFF_BC;
      constexpr uint32_t idL = idesc_f16(128, L::N1, 0, 0), idC = idesc_f16(128, Cc::N1, 0, 0);
      constexpr uint32_t id2L = idesc_f16(128, L::N1, 1, 0), id2C = idesc_f16(128, Cc::N1, 1, 0);
      auto stage2 = [&](int pj) -> bool {
        const JobRef jr = job_ref<LP>(pj, cta, grid);
        const int a2 = pj & 1;
        if (!wait_bar(ctl, B_A2 + a2, (pj >> 1) & 1, 2)) return false;
        tc_fence_after();
        const uint32_t d = tmem + jr.slot * 128;
        const uint32_t ahi = sbase + OFF_A2 + a2 * 2 * kA2Bytes, alo = ahi + kA2Bytes;
        if (jr.plane == 0) {
#pragma unroll
          for (int ks = 0; ks < L::KS; ++ks) {
            const uint64_t b = smem_desc(bl + ks * 256, 128, 512, 0);
            mma_ss(d + 64, smem_desc(ahi + ks * 4096, 1024, 2048, 2), b, id2L, 1);
            mma_ss(d + 96, smem_desc(alo + ks * 4096, 1024, 2048, 2), b, id2L, 1);
          }
        } else {
          const uint64_t b = smem_desc(bc, 128, 256, 0);
          mma_ss(d + 64, smem_desc(ahi, 1024, 2048, 2), b, id2C, 1);
          mma_ss(d + 96, smem_desc(alo, 1024, 2048, 2), b, id2C, 1);
        }
        mma_commit(&bars[B_D2 + jr.slot]);
        return true;
      };
      bool ok = true;
      for (int it = 0; it < n_jobs && ok; ++it) {
        const JobRef jr = job_ref<LP>(it, cta, grid);
        if (!wait_bar(ctl, B_A1 + jr.slot, (it >> 2) & 1, 2)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + jr.slot * 128;
        if (jr.plane == 0) {
#pragma unroll
          for (int g = 0; g < L::G; ++g)
#pragma unroll
            for (int ks = 0; ks < L::KS; ++ks)
              mma_ts(d + 32 + g * L::N1, d + g * L::A1COLS + ks * 8, smem_desc(bl + ks * 256, 128, 512, 0), idL, 1);
        } else {
#pragma unroll
          for (int g = 0; g < Cc::G; ++g)
            mma_ts(d + 32 + g * Cc::N1, d + g * Cc::A1COLS, smem_desc(bc, 128, 256, 0), idC, 1);
        }
        mma_commit(&bars[B_D1 + jr.slot]);
        if (it >= 1) ok = stage2(it - 1);
      }
      if (ok && n_jobs > 0) ok = stage2(n_jobs - 1);
      if (!ok) {
        mma_commit(&bars[B_DRAIN]);
        wait_bar(ctl, B_DRAIN, 0, 2, true);
      }
    }
  } else {
    // ---------------- workers ----------------
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    float wL[L::NK], wC[Cc::NK];
#pragma unroll
    for (int u = 0; u < L::NK; ++u) wL[u] = p.W_y[u * 32 + (lane % L::NK)];
#pragma unroll
    for (int u = 0; u < Cc::NK; ++u) wC[u] = p.W_c[u * 16 + (lane % Cc::NK)];
    // Luma (N = 32, 8-bit): s1 = 4, s2 = 11; chroma (N = 16): s1 = 3, s2 = 10.
    const float c0L = 8.0f - 2097152.0f, cL = 8.0f, c0C = 4.0f - 1048576.0f, cC = 4.0f;
    const float hi0L = kK1 - 2367488.0f, hi0C = kK1 - 1183744.0f;
    const float loL = 1024.0f, loC = 512.0f;
    const float c2L = kK1 - kK1 / 8.0f, c2C = kK1 - kK1 / 4.0f;
    bool ok = true;
    for (int it = 0; it < n_jobs + 2 && ok; ++it) {
      if (it < n_jobs) {
        const JobRef jr = job_ref<LP>(it, cta, grid);
        const int t = it / JPT;
        const int j = it - t * JPT;
        const int stage = t % kStages;
        if (j == 0 && !wait_bar(ctl, B_RAW_FULL + stage, (t / kStages) & 1, 4)) {
          ok = false;
          break;
        }
        const int f = jr.item / tiles_per_frame;
        const int ti = jr.item - f * tiles_per_frame;
        const int tx = ti % p.tiles_x, ty = ti / p.tiles_x;
        const uint8_t* raw = sm + OFF_RAW + stage * kStageBytes;
        const uint32_t ts = tmem + jr.slot * 128;
        if (jr.plane == 0)
          convert_job<32, LP>(p, raw, jr.jp, tx, ty, p.W, p.H, ts, q, lane, c0L, cL, hi0L, loL);
        else
          convert_job<16, LP>(p, raw + kRawY + (jr.plane - 1) * kRawC, jr.jp, tx, ty, p.cw, p.ch, ts, q, lane, c0C,
                              cC, hi0C, loC);
        tmem_wait_st();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&bars[B_A1 + jr.slot]);
          if (j == JPT - 1) mbar_arrive(&bars[B_RAW_EMPTY + stage]);
        }
      }
      if (it >= 1 && it - 1 < n_jobs) {
        const int pj = it - 1;
        const JobRef jr = job_ref<LP>(pj, cta, grid);
        if (!wait_bar(ctl, B_D1 + jr.slot, (pj >> 2) & 1, 4)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t ahi = sbase + OFF_A2 + (pj & 1) * 2 * kA2Bytes, alo = ahi + kA2Bytes;
        const uint32_t ts = tmem + jr.slot * 128;
        if (jr.plane == 0)
          epilogue1<32, LP>(ts, ahi, alo, q, lane, 0.0625f);
        else
          epilogue1<16, LP>(ts, ahi, alo, q, lane, 0.125f);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bars[B_A2 + (pj & 1)]);
      }
      if (it >= 2) {
        const int pj = it - 2;
        const JobRef jr = job_ref<LP>(pj, cta, grid);
        if (!wait_bar(ctl, B_D2 + jr.slot, (pj >> 2) & 1, 4)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const int f = jr.item / tiles_per_frame;
        const int ti = jr.item - f * tiles_per_frame;
        const int tx = ti % p.tiles_x, ty = ti / p.tiles_x;
        const uint32_t ts = tmem + jr.slot * 128;
        if (jr.plane == 0)
          epilogue2<32, LP, DUMP>(p, ts, 0, jr.jp, f, tx, ty, q, lane, wL, 0.125f, c2L);
        else
          epilogue2<16, LP, DUMP>(p, ts, jr.plane, jr.jp, f, tx, ty, q, lane, wC, 0.25f, c2C);
        tc_fence_before();
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// ---- host side -------------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

cudaError_t make_map(CUtensorMap* m, const void* base, int w, int h, int64_t pitch, int64_t fstride, int nframes,
                     int box, CUtensorMapSwizzle sw) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (nframes == 1 || fstride <= 0) fstride = ((pitch * h + 15) / 16) * 16;
  cuuint64_t dims[3] = {(cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)nframes};
  cuuint64_t strides[2] = {(cuuint64_t)pitch, (cuuint64_t)fstride};
  cuuint32_t boxd[3] = {(cuuint32_t)box, (cuuint32_t)box, 1};
  cuuint32_t es[3] = {1, 1, 1};
  CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void*>(base), dims, strides, boxd, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <bool LP, bool DUMP>
cudaError_t launch_inst(const CUtensorMap& my, const CUtensorMap& mu, const CUtensorMap& mv, const TcParams& p,
                        int grid, cudaStream_t s) {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(tc_kernel<LP, DUMP>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
  });
  if (attr != cudaSuccess) return attr;
  tc_kernel<LP, DUMP><<<grid, kThreads, kSmemBytes, s>>>(my, mu, mv, p);
  return cudaGetLastError();
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

bool tc_supported(const Geometry& g) { return g.B == 8 && g.w == 32 && encode_fn() != nullptr; }

cudaError_t launch_tc(const Geometry& g, const FramePlanes& fp, int nframes, const DeviceTables& t, float* blockvals,
                      int16_t* const zdump[3], int* err, cudaStream_t s, int64_t* launches) {
  if (!tc_supported(g)) return cudaErrorNotSupported;
  if (nframes <= 0) return cudaSuccess;
  CUtensorMap my, mu, mv;
  cudaError_t e = make_map(&my, fp.y, g.W, g.H, fp.pitch_y, fp.fstride_y, nframes, 128, CU_TENSOR_MAP_SWIZZLE_128B);
  if (e == cudaSuccess)
    e = make_map(&mu, fp.u, g.cw, g.ch, fp.pitch_uv, fp.fstride_uv, nframes, 64, CU_TENSOR_MAP_SWIZZLE_64B);
  if (e == cudaSuccess)
    e = make_map(&mv, fp.v, g.cw, g.ch, fp.pitch_uv, fp.fstride_uv, nframes, 64, CU_TENSOR_MAP_SWIZZLE_64B);
  if (e != cudaSuccess) return e;
  TcParams p{};
  p.W = g.W;
  p.H = g.H;
  p.cw = g.cw;
  p.ch = g.ch;
  p.nbx = g.nbx;
  p.nby = g.nby;
  p.tiles_x = (g.nbx + 3) / 4;
  p.tiles_y = (g.nby + 3) / 4;
  p.nframes = nframes;
  p.total_items = p.tiles_x * p.tiles_y * nframes;
  p.C = g.C;
  p.out_fstride = (int64_t)N_ROWS * g.C;
  p.blockvals = blockvals;
  for (int i = 0; i < 3; ++i) p.zdump[i] = zdump ? zdump[i] : nullptr;
  p.M_y = t.M_y;
  p.M_c = t.M_c;
  p.W_y = t.W_y;
  p.W_c = t.W_c;
  p.err = err;
  const int grid = p.total_items < sm_count() ? p.total_items : sm_count();
  const bool dump = zdump != nullptr;
  if (g.low_pass)
    e = dump ? launch_inst<true, true>(my, mu, mv, p, grid, s) : launch_inst<true, false>(my, mu, mv, p, grid, s);
  else
    e = dump ? launch_inst<false, true>(my, mu, mv, p, grid, s) : launch_inst<false, false>(my, mu, mv, p, grid, s);
  if (e == cudaSuccess) ++*launches;
  return e;
}

}  // namespace vca
