// Tensor-core form of the analyzer's per-block work (Section 2 of the paper: integer DCT of
// every Y, U, V block, texture energy H and brightness L; Section 2 item (3): low-pass).
//
// Persistent kernel, one CTA of 28 warps per SM, specialised by warpgroup:
//   warpgroup 0   warp 0: TMA producer (one 128x128 luma + two 64x64 chroma tiles per work item
//                 into a 5-stage ring, 128-byte / 64-byte swizzled; 10-bit samples as 16-bit
//                 words: two 64-sample luma boxes, 3 stages); warp 1: TMEM owner and
//                 stage-1 MMA issuer; warp 2: stage-2 MMA issuer (tcgen05.mma kind::f16, FP32
//                 accumulate), so neither stage waits on the other's epilogue;
//   warpgroups 1, 6  convert (luma jobs, chroma jobs): raw samples -> stage-1 A operand in TMEM;
//   warpgroups 2, 3  epilogue 1 (luma jobs, chroma jobs): stage-1 accumulators -> stage-2 A
//                 operand in shared memory;
//   warpgroups 4, 5  epilogue 2 (luma jobs, chroma jobs): stage-2 accumulators -> block
//                 energies and brightness.
// Each warpgroup has one warp per TMEM lane quarter.  Jobs flow through 8 TMEM slots (64 columns
// each) and, per plane type, 2 shared-memory operand slots; every slot has a full and a free
// mbarrier, so the roles run concurrently on different jobs.
//
// A "job" is 128 stage-2 rows: 8 (low-pass) or 4 luma 32x32 blocks, or 16 / 8 chroma 16x16
// blocks.  Per job:
//   convert   raw row -> fp16 (1024 + x: one PRMT per two 8-bit samples, one AND-OR per two
//             10-bit samples) written to TMEM as the A operand;
//   stage 1   D1 = c + X M^T (A from TMEM, M from shared memory), exact integers in FP32; the
//             presets c_k (the rounding offset 2^(s1-1), minus the 1024 * 64 * N encoding bias
//             on the DC row) enter as one more MMA from constant shared-memory operands;
//   epilogue1 T = floor(D1/2^s1) by one round-down FMA whose magic constant leaves
//             U = T + 32768 in the low 16 bits and 0x64 in byte 2, so two PRMTs give the
//             fp16 pairs (1024 + U_lo8, 1024 + U_hi8); stored MN-major (128-byte swizzle)
//             as the stage-2 A operand -- the row/column transpose is the layout;
//   stage 2   S_hi, S_lo = M T_hi, M T_lo (A MN-major from shared memory), the accumulators
//             pre-set by epilogue 1 to the magic constants of epilogue 2;
//   epilogue2 Z = floor((256 S_hi + S_lo + 2^(s2-1)) / 2^s2) by two round-down FMAs, then
//             H_v = sum_u w(u,v) |Z| in increasing u and an xor tree over v.
// Every partial sum is an integer below 2^24 in magnitude (or in [2^23, 2^24) for the
// pre-offset accumulators), so the FP32 tensor-core accumulation is exact and Z is
// bit-identical to the integer definition; H uses the same FP32 order as the CUDA-core form.
//
// A launch covers one analyzer's frames (its geometry in the kernel parameters) or, for a batched
// tick, one frame of each of up to 64 analyzers of one sample size (a member table and their
// tensor maps, also in the kernel parameters, read through the constant cache).
//
// Every wait is bounded (about two seconds); on timeout the kernel raises a flag in *err,
// stops, waits for its own copies and MMAs, frees TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <cstring>
#include <mutex>
#include <new>

#include "vca_internal.h"
#include "vca_ptx.cuh"

namespace vca {
namespace {

using namespace ptx;

constexpr int kMaxStages = 5;  // raw tile ring (barrier indices are laid out for the longest)
constexpr int kA2L = 8192;      // one stage-2 operand (hi or lo) of one luma job: 128 rows x 32 K x fp16
constexpr int kA2C = 4096;      // of one chroma job: 128 rows x 16 K x fp16
constexpr int OFF_RAW = 0;
constexpr int kBars = 80;
constexpr int kA2Slots = 4;     // 0-1 luma jobs, 2-3 chroma jobs
constexpr int kMaxMembers = kMaxBatchMembers;

// One analyzer ("member") of a launch: its work items, geometry, outputs and stage-1 constants.
// A single analyzer's launch has one member with all its frames; a batched tick has one member
// per channel with one frame each.  Items are numbered member by member, frame-major tiles.
struct TcMember {
  int item_base;                   // first item of this member
  int tiles_x, tiles_per_frame;
  float inv_tiles_x, inv_tiles_per_frame;
  int W, H, cw, ch, nbx, nby;
  int64_t C, out_fstride;
  float* blockvals;
};

// Stage-1 shift s1 = log2 N + B - 9 of a plane type; the bit depth follows from the sample size
// (8-bit samples in bytes, 10-bit in 16-bit words).
template <int Nb>
__host__ __device__ constexpr int s1_of(int bps) {
  return (Nb == 32 ? 5 : 4) + (bps == 1 ? 8 : 10) - 9;
}
static_assert(sizeof(TcMember) % 8 == 0, "member table entries are copied as words");


// Shared-memory layout for BPS bytes per sample.  8-bit: a 128x128 luma tile (128-byte rows,
// 128-byte swizzle) and two 64x64 chroma tiles (64-byte rows and swizzle), 5 stages.  10-bit
// (16-bit words): the luma tile as two 64-sample-wide boxes side by side (128-byte rows each,
// 128-byte swizzle) and 64x64 chroma tiles with 128-byte rows and swizzle, 3 stages.
template <int BPS>
struct SmemLay {
  static_assert(BPS == 1 || BPS == 2, "one sample size per launch");
  static constexpr int kStages = BPS == 1 ? 5 : 3;
  static constexpr int kRawY = 128 * 128 * BPS;
  static constexpr int kRawC = 64 * 64 * BPS;
  static constexpr int kStageBytes = kRawY + 2 * kRawC;
  static constexpr int OFF_A2 = kStages * kStageBytes;   // luma: 2 slots x (hi, lo)
  static constexpr int OFF_A2C = OFF_A2 + 2 * 2 * kA2L;  // chroma: 2 slots x (hi, lo)
  static constexpr int OFF_BL = OFF_A2C + 2 * 2 * kA2C;
  static constexpr int OFF_BC = OFF_BL + 2048;
  static constexpr int OFF_ONE = OFF_BC + 512;    // preset operand U (128 x 16)
  static constexpr int OFF_KL = OFF_ONE + 4096;   // stage-1 preset operand K, luma (G N1 x 16)
  static constexpr int OFF_KC = OFF_KL + 1024;    // and chroma
  static constexpr int OFF_BAR = OFF_KC + 1024;
  static constexpr int OFF_MISC = OFF_BAR + kBars * 8;
  static constexpr int kSmemBytes = OFF_MISC + 64 + 1024;  // + slack to align the base to 1024
  static_assert(kStages <= kMaxStages && OFF_A2 % 1024 == 0 && kSmemBytes <= 232448, "layout");
};

// TMEM layout: 8 job slots of 64 columns, each holding the stage-1 operand A1 at [0, 32), the
// stage-1 accumulators D1 at [32, 64), and then the stage-2 accumulators D2 over [0, 32)
// (low-pass) or [0, 64) (all coefficients) once stage 1 has consumed A1 and epilogue 1 has read
// D1 into registers.
constexpr int kSlots = 8;
constexpr int kSlotCols = 64;
constexpr int kD1Off = 32;

// barrier indices
__host__ __device__ constexpr int b_raw_full(int s) { return s; }
__host__ __device__ constexpr int b_raw_empty(int s) { return kMaxStages + s; }
__host__ __device__ constexpr int b_slot_free(int s) { return 2 * kMaxStages + s; }
__host__ __device__ constexpr int b_d1(int s) { return 2 * kMaxStages + kSlots + s; }
__host__ __device__ constexpr int b_d2(int s) { return 2 * kMaxStages + 2 * kSlots + s; }
__host__ __device__ constexpr int b_a1_full(int s) { return 2 * kMaxStages + 3 * kSlots + s; }
__host__ __device__ constexpr int b_a2_full(int s) { return 2 * kMaxStages + 4 * kSlots + s; }
__host__ __device__ constexpr int b_a2_free(int s) { return 2 * kMaxStages + 4 * kSlots + kA2Slots + s; }
__host__ __device__ constexpr int b_drain(int i) { return 2 * kMaxStages + 4 * kSlots + 2 * kA2Slots + i; }
static_assert(b_drain(1) < kBars, "barrier area");

constexpr int kThreads = 896;
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kWaitNs = 2000000000ull;

// FP32 magic constants (see the file comment).
constexpr float kT1 = 14974976.0f;  // 2^23 + 0x640000 + 0x8000
constexpr float kK1 = 12582912.0f;  // 1.5 * 2^23
constexpr uint32_t kSel6464 = 0x64646464u;

// Kernel parameters of a launch over up to MAXM members: one analyzer's frames (MAXM = 1) or one
// frame of each channel of a batched tick (MAXM = kMaxMembers; about 29 KB, within the 32,764
// bytes a kernel may take).  The member table and the tensor maps live in parameter space, read
// through the constant cache; a batched tick graph rewrites them per tick.
template <int MAXM>
struct TcParamsT {
  int16_t* zdump[3];
  const int8_t* M_y;
  const int8_t* M_c;
  const float* W_y;
  const float* W_c;
  int* err;
  int n_members, total_items;
  TcMember mem[MAXM];
  CUtensorMap maps[3 * MAXM];  // Y, U, V of each member
};
using TcParams = TcParamsT<1>;
using TcBatchParams = TcParamsT<kMaxMembers>;
static_assert(sizeof(TcBatchParams) <= 32764, "kernel parameter space");

template <int Nb, bool LP>
struct PC {
  static constexpr int NK = LP ? Nb / 2 : Nb;     // coefficients kept per dimension
  static constexpr int N1 = NK < 16 ? 16 : NK;    // MMA N of both stages
  static constexpr int BPG1 = 128 / Nb;           // blocks per stage-1 group (128 rows)
  static constexpr int BPG2 = 128 / NK;           // blocks per job (128 stage-2 rows)
  static constexpr int G = BPG2 / BPG1;           // stage-1 groups per job
  static constexpr int JOBS = 16 / BPG2;          // jobs of this plane per tile
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
__device__ __noinline__ bool wait_bar_slow(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                          int code, bool ignore_abort, bool sleep) {
  const uint64_t t0 = now_ns();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (sleep ? mbar_try_wait_sleep(bar, parity) : mbar_try_wait(bar, parity)) return true;
    if (!ignore_abort && *abort_flag) return false;
    if (now_ns() - t0 > kWaitNs) {
      *abort_flag = 1;
      atomicOr(err, code);
      return false;
    }
  }
}

// Bounded wait on barrier idx.  Roles on the critical path spin; the producer (sleep = true) lets
// its thread sleep in hardware between polls.
__device__ __forceinline__ bool wait_bar(const Ctl& c, int idx, uint32_t parity, int code, bool ignore_abort = false,
                                         bool sleep = false) {
  uint64_t* bar = c.bars + idx;
  if (mbar_try_wait(bar, parity)) return true;
  return wait_bar_slow(bar, parity, c.abort, c.err, code, ignore_abort, sleep);
}

// Byte offset of sample xx of row y of the raw tile of this plane type.
template <int Nb, int BPS>
__device__ __forceinline__ uint32_t raw_offset(int y, int xx) {
  if (BPS == 1) {
    const int chunk = xx >> 4;
    const int sw = Nb == 32 ? (chunk ^ (y & 7)) : (chunk ^ ((y >> 1) & 3));
    return (uint32_t)(y * (Nb == 32 ? 128 : 64) + (sw << 4) + (xx & 15));
  }
  // 16-bit samples: 64-sample boxes with 128-byte rows and 128-byte swizzle; luma has two.
  const int box = Nb == 32 ? (xx >> 6) : 0;
  const int cx = xx & 63;
  const int chunk = cx >> 3;
  return (uint32_t)(box * (Nb == 32 ? 128 : 64) * 128 + y * 128 + ((chunk ^ (y & 7)) << 4) + (cx & 7) * 2);
}

// Stage-1 operand conversion: 16 samples of this thread's row starting at column x (of the raw
// tile, edge columns repeated past w_rem) -> 8 words of fp16 pairs (1024 + sample) in out.
// 8-bit samples become fp16 0x6400 | x by one PRMT per two samples; 10-bit samples (below 1024)
// by one AND-OR per two.
template <int Nb, int BPS>
__device__ __forceinline__ void convert_16(uint32_t base, int y, int x, int w_rem, uint32_t* out) {
  static_assert(BPS == 1 || BPS == 2, "one sample size");
  if (BPS == 1) {
    uint32_t words[4];
    if (x + 16 <= w_rem) {
      const uint4 q = lds128(base + raw_offset<Nb, 1>(y, x));
      words[0] = q.x;
      words[1] = q.y;
      words[2] = q.z;
      words[3] = q.w;
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) words[i] = 0;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const uint32_t b = lds_u8(base + raw_offset<Nb, 1>(y, min(x + c, w_rem - 1)));
        words[c >> 2] |= b << (8 * (c & 3));
      }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      out[2 * i] = prmt(words[i], kSel6464, 0x5140);
      out[2 * i + 1] = prmt(words[i], kSel6464, 0x5342);
    }
  } else {
    uint32_t words[8];
    if (x + 16 <= w_rem) {
      const uint4 q0 = lds128(base + raw_offset<Nb, 2>(y, x));
      const uint4 q1 = lds128(base + raw_offset<Nb, 2>(y, x + 8));
      words[0] = q0.x;
      words[1] = q0.y;
      words[2] = q0.z;
      words[3] = q0.w;
      words[4] = q1.x;
      words[5] = q1.y;
      words[6] = q1.z;
      words[7] = q1.w;
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) words[i] = 0;
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const uint32_t v = lds_u16(base + raw_offset<Nb, 2>(y, min(x + c, w_rem - 1)));
        words[c >> 1] |= v << (16 * (c & 1));
      }
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = (words[i] & 0x03FF03FFu) | 0x64006400u;
  }
}

template <int N>
__device__ __forceinline__ void fill_cols(uint32_t taddr, float first, float rest) {
  tmem_fill<N>(taddr, __float_as_uint(first), __float_as_uint(rest));
}

// Block coordinates of one job for the epilogue that writes its results.
struct JobCtx {
  int plane;  // 0 Y, 1 U, 2 V
  int jp;     // job index within the plane's tile
  int f;      // frame
  int tx, ty; // tile position (units of 4 blocks)
};

template <bool LP>
__device__ __forceinline__ void plane_of(int j, int& plane, int& jp) {
  constexpr int JL = PC<32, LP>::JOBS;
  constexpr int JC = PC<16, LP>::JOBS;
  if (j < JL) {
    plane = 0;
    jp = j;
  } else if (j < JL + JC) {
    plane = 1;
    jp = j - JL;
  } else {
    plane = 2;
    jp = j - JL - JC;
  }
}

// Stage-2 operand slot of job j and its use count: each plane type cycles through its own two
// slots, so every slot's full / free barriers see one in-order stream of jobs (a barrier is never
// waited on more than one phase ahead of its current phase).
template <bool LP>
__device__ __forceinline__ void a2_slot_of(int j, int& slot, int& use) {
  constexpr int JPT = Jobs<LP>::PER_TILE;
  constexpr int JL = PC<32, LP>::JOBS;
  const int t = j / JPT, r = j - t * JPT;
  if (r < JL) {
    const int idx = t * JL + r;
    slot = idx & 1;
    use = idx >> 1;
  } else {
    const int idx = t * (JPT - JL) + (r - JL);
    slot = 2 + (idx & 1);
    use = idx >> 1;
  }
}

// Shared-memory address of the stage-2 operand (hi; lo follows at +kA2L / +kA2C).
template <int BPS>
__device__ __forceinline__ uint32_t a2_addr(uint32_t sbase, int a2) {
  using SL = SmemLay<BPS>;
  return a2 < 2 ? sbase + SL::OFF_A2 + a2 * 2 * kA2L : sbase + SL::OFF_A2C + (a2 - 2) * 2 * kA2C;
}

// ---- worker phases ----------------------------------------------------------

// Writes the job's stage-1 A operand at ta1.
template <int Nb, bool LP, int BPS>
__device__ __forceinline__ void convert_job(const uint8_t* raw_plane, int jp, int h_rem, int w_rem, uint32_t ta1,
                                            int q, int lane) {
  using P = PC<Nb, LP>;
  // The job's groups occupy G * A1COLS consecutive columns, stored 16 at a time (8 if fewer).
  constexpr int COLS = P::G * P::A1COLS;
  constexpr int ST = COLS < 16 ? COLS : 16;
  const int l = 32 * q + lane;
  const int bg = l / Nb;
  const int r = l % Nb;
  uint32_t out[ST];
#pragma unroll
  for (int g = 0; g < P::G; ++g) {
    const int idx = jp * P::BPG2 + g * P::BPG1 + bg;
    int y = (idx >> 2) * Nb + r;
    if (y >= h_rem) y = h_rem - 1;
    const int x = (idx & 3) * Nb;
#pragma unroll
    for (int c = 0; c < Nb / 16; ++c) {
      const int col = g * P::A1COLS + 8 * c;  // first column of these 16 samples
      convert_16<Nb, BPS>(smem_u32(raw_plane), y, x + 16 * c, w_rem, out + col % ST);
      if ((col + 8) % ST == 0) tmem_st<ST>(ta1 + col + 8 - ST, out);
    }
  }
}

// Reads D1 (stage-1 accumulators at td1 + g*N1), writes the stage-2 operand to shared memory, and
// pre-sets the stage-2 accumulators at td2 (hi) and td2 + N1 (lo), which may overlap D1.
template <int Nb, bool LP>
__device__ __forceinline__ void epilogue1(uint32_t td1, uint32_t td2, uint32_t a2hi, uint32_t a2lo, int q, int lane,
                                          float s1inv, float hi0, float lo) {
  using P = PC<Nb, LP>;
  constexpr int NK = P::NK;
  const int l = 32 * q + lane;
  const int bg = l / Nb;
  const int r = l % Nb;
  // D1 is read 16 columns at a time (bounds register use).  The stage-2 hi presets at [0, N1)
  // never overlap D1 (at column kD1Off = 32); the lo presets at [N1, 2 N1) do when N1 = 32 (all
  // coefficients, luma), so they are written after every column of D1 has been read.
  constexpr int CH = NK < 16 ? NK : 16;
  constexpr bool kLoOverD1 = 2 * P::N1 > kD1Off;
  fill_cols<P::N1>(td2, hi0, kK1);
  if (!kLoOverD1) fill_cols<P::N1>(td2 + P::N1, lo, lo);
  const uint32_t rowoff = (uint32_t)((r >> 3) * 2048 + (r & 7) * 128);
#pragma unroll
  for (int g = 0; g < P::G; ++g) {
#pragma unroll
    for (int h0 = 0; h0 < NK; h0 += CH) {
      uint32_t acc[CH];
      tmem_ld<CH>(td1 + g * P::N1 + h0, acc);
      tmem_wait_ld();
      uint32_t hi[CH / 2], lw[CH / 2];
#pragma unroll
      for (int k = 0; k < CH; k += 2) {
        // D1 already holds T' = c_k + sum (the accumulators were pre-set), an exact integer.
        const uint32_t za = __float_as_uint(__fmaf_rd(__uint_as_float(acc[k]), s1inv, kT1));
        const uint32_t zb = __float_as_uint(__fmaf_rd(__uint_as_float(acc[k + 1]), s1inv, kT1));
        lw[k / 2] = prmt(za, zb, 0x6420);
        hi[k / 2] = prmt(za, zb, 0x6521);
      }
      const int m0 = (g * P::BPG1 + bg) * NK + h0;
#pragma unroll
      for (int cc = 0; cc < CH / 8; ++cc) {
        const int m = m0 + 8 * cc;
        const uint32_t off = rowoff + (uint32_t)((m >> 6) * 1024) + (uint32_t)(((((m & 63) >> 3) ^ (r & 7))) << 4);
        sts128(a2hi + off, hi[4 * cc], hi[4 * cc + 1], hi[4 * cc + 2], hi[4 * cc + 3]);
        sts128(a2lo + off, lw[4 * cc], lw[4 * cc + 1], lw[4 * cc + 2], lw[4 * cc + 3]);
      }
    }
  }
  if (kLoOverD1) fill_cols<P::N1>(td2 + P::N1, lo, lo);
}

template <int Nb, bool LP, bool DUMP>
__device__ __forceinline__ void epilogue2(int16_t* const* zdump, const TcMember& M, uint32_t td2, const JobCtx& jc,
                                          int q, int lane,
                                          const float (&wts)[PC<Nb, LP>::NK], float einv, float c2,
                                          uint64_t* slot_free) {
  using P = PC<Nb, LP>;
  constexpr int NK = P::NK;
  constexpr int HALF = NK > 16 ? 8 : NK;  // columns loaded at a time (bounds register use)
  const int m = 32 * q + lane;
  const int b2 = m / NK;
  const int v = m % NK;
  const int idx = jc.jp * P::BPG2 + b2;
  const int bx = jc.tx * 4 + (idx & 3);
  const int by = jc.ty * 4 + (idx >> 2);
  const bool valid = bx < M.nbx && by < M.nby;
  const int64_t k = (int64_t)by * M.nbx + bx;
  int16_t* zd = nullptr;
  if (DUMP) zd = (valid && jc.f == 0) ? zdump[jc.plane] + k * NK * NK : nullptr;
  float H = 0.0f, z00 = 0.0f;
#pragma unroll
  for (int h0 = 0; h0 < NK; h0 += HALF) {
    uint32_t hi[HALF], lo[HALF];
    tmem_ld<HALF>(td2 + h0, hi);
    tmem_ld<HALF>(td2 + P::N1 + h0, lo);
    tmem_wait_ld();
    if (h0 + HALF == NK) {  // every accumulator of the slot is in registers: hand the slot back
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(slot_free);
    }
#pragma unroll
    for (int uu = 0; uu < HALF; ++uu) {
      const int u = h0 + uu;
      const float w = __fmaf_rd(__uint_as_float(lo[uu]), 0.00390625f, __uint_as_float(hi[uu]));
      const float z = __fmaf_rd(w, einv, c2) - kK1;
      if (u == 0) z00 = z;
      if (DUMP && zd) zd[u * NK + v] = (int16_t)z;
      H = fmaf(fabsf(z), wts[u], H);
    }
  }
#pragma unroll
  for (int o = NK / 2; o > 0; o >>= 1) H += __shfl_xor_sync(0xffffffffu, H, o);
  if (valid && v == 0) {
    float* out = M.blockvals + (int64_t)jc.f * M.out_fstride + (2 * jc.plane) * M.C + k;
    out[0] = H;
    out[M.C] = __fsqrt_rn(z00);
  }
}

// Tile bookkeeping of a role's current tile.
struct TileInfo {
  int f, tx, ty, stage, t, m;  // frame, tile position, ring stage, CTA-local tile number, member
};

// a / b for 0 <= a < 2^24, b >= 1, from a float estimate that is off by at most one.
__device__ __forceinline__ int div_small(int a, int b, float binv) {
  int qt = __float2int_rz((float)a * binv);
  const int r = a - qt * b;
  qt += (r >= b) - (r < 0);
  return qt;
}

// The members of a launch as the roles see them.  A single analyzer's launch reads its one member
// from the kernel parameters (fields become constant-bank operands); a batched launch reads the
// member table that the CTA copied into shared memory.
struct OneMember {
  const TcMember& m0;
  __device__ __forceinline__ int member_of(int) const { return 0; }
  __device__ __forceinline__ const TcMember& operator[](int) const { return m0; }
};

struct MemberTable {
  const TcMember* mem;
  int n;
  mutable int cur;  // member of the last item asked for
  // The member that work item `item` belongs to: the last one whose first item is <= item.  Each
  // thread asks for its CTA's items in increasing order, so the search moves forward only.
  __device__ __forceinline__ int member_of(int item) const {
    while (cur + 1 < n && mem[cur + 1].item_base <= item) ++cur;
    return cur;
  }
  __device__ __forceinline__ const TcMember& operator[](int i) const { return mem[i]; }
};

template <bool BATCH>
struct MemberView;
template <>
struct MemberView<false> {
  using T = OneMember;
};
template <>
struct MemberView<true> {
  using T = MemberTable;
};

template <class MS>
__device__ __forceinline__ TileInfo tile_info(const MS& ms, int t, int item0, int step, int stages = kMaxStages) {
  TileInfo ti;
  const int item = item0 + t * step;
  const int m = ms.member_of(item);
  const TcMember& M = ms[m];
  const int local = item - M.item_base;
  ti.m = m;
  ti.t = t;
  ti.f = div_small(local, M.tiles_per_frame, M.inv_tiles_per_frame);
  const int r = local - ti.f * M.tiles_per_frame;
  ti.ty = div_small(r, M.tiles_x, M.inv_tiles_x);
  ti.tx = r - ti.ty * M.tiles_x;
  ti.stage = t % stages;
  return ti;
}

// ---- role loops (one instantiation per plane type) -------------------------------
//
// Jobs are numbered jj = t * JPT + r (tile t of this CTA, r < JPT): luma jobs first, then U,
// then V.  Job jj lives in TMEM slot jj % kSlots; each role visits only its plane type's jobs.

template <int Nb, bool LP>
__device__ __forceinline__ void plane_jobs(int& r0, int& r1) {
  constexpr int JL = PC<32, LP>::JOBS;
  r0 = Nb == 32 ? 0 : JL;
  r1 = Nb == 32 ? JL : Jobs<LP>::PER_TILE;
}

// Convert: raw samples of the tile -> stage-1 A operand in TMEM (and the D1 presets).
template <int Nb, bool LP, int BPS, class MS>
__device__ void convert_loop(const MS& ms, const Ctl& ctl, uint8_t* sm, uint32_t tq, int n_items, int item0,
                             int step, int q, int lane) {
  using SL = SmemLay<BPS>;
  constexpr int JPT = Jobs<LP>::PER_TILE;
  constexpr int T = 4 * Nb;  // tile edge of this plane in samples
  int r0, r1;
  plane_jobs<Nb, LP>(r0, r1);
  const int per_tile = r1 - r0;
  TileInfo ti{};
  int h_rem = 0, w_rem = 0;
  const int n = n_items * per_tile;
  for (int k = 0, t = 0, r = r0; k < n; ++k) {
    if (r == r0) {
      ti = tile_info(ms, t, item0, step, SL::kStages);
      const TcMember& M = ms[ti.m];
      h_rem = (Nb == 32 ? M.H : M.ch) - ti.ty * T;
      w_rem = (Nb == 32 ? M.W : M.cw) - ti.tx * T;
      if (!wait_bar(ctl, b_raw_full(ti.stage), (t / SL::kStages) & 1, 4)) return;
    }
    const int jj = t * JPT + r;
    int plane, jp;
    plane_of<LP>(r, plane, jp);
    const int slot = jj % kSlots;
    if (jj >= kSlots && !wait_bar(ctl, b_slot_free(slot), ((jj / kSlots) - 1) & 1, 4)) return;
    tc_fence_after();
    // Plane offsets within the stage follow the member's sample size (the stage fits the largest).
    const uint8_t* raw =
        sm + OFF_RAW + ti.stage * SL::kStageBytes + (plane == 0 ? 0 : SL::kRawY + (plane - 1) * SL::kRawC);
    const uint32_t ta = tq + slot * kSlotCols;
    convert_job<Nb, LP, BPS>(raw, jp, h_rem, w_rem, ta, q, lane);
    tmem_wait_st();
    tc_fence_before();
    __syncwarp();
    const bool last = r == r1 - 1;
    if (lane == 0) {
      mbar_arrive(&ctl.bars[b_a1_full(slot)]);
      if (last) mbar_arrive(&ctl.bars[b_raw_empty(ti.stage)]);
    }
    if (last) {
      r = r0;
      ++t;
    } else {
      ++r;
    }
  }
}

// Epilogue 1: T = floor(T'/2^s1) into the stage-2 operand (hi and lo bytes as fp16, MN-major;
// s1 = log2 N + B - 9), and the stage-2 accumulators pre-set: hi starts at K1 - 1156 * 64 * N for
// u = 0 (the 1024 + byte encoding of both halves and the +128 offset of the hi byte) and K1
// otherwise, lo at 2^(s2-1) (luma N = 32: s2 = 11; chroma N = 16: s2 = 10).  Each plane type
// cycles through its own two stage-2 operand slots, so every slot's full / free barriers see one
// in-order stream of jobs.
template <int Nb, bool LP, int BPS, class MS>
__device__ void epi1_loop(const MS& ms, const Ctl& ctl, uint32_t sbase, uint32_t tq, int n_items, int item0,
                          int step, int q, int lane) {
  using SL = SmemLay<BPS>;
  constexpr int JPT = Jobs<LP>::PER_TILE;
  const float s1inv = __int_as_float((127 - s1_of<Nb>(BPS)) << 23);  // 2^-s1
  const float hi0 = Nb == 32 ? kK1 - 2367488.0f : kK1 - 1183744.0f;
  const float lo = Nb == 32 ? 1024.0f : 512.0f;
  const uint32_t lo_off = Nb == 32 ? kA2L : kA2C;
  const uint32_t a2base = Nb == 32 ? sbase + SL::OFF_A2 : sbase + SL::OFF_A2C;
  const int a2first = Nb == 32 ? 0 : 2;
  int r0, r1;
  plane_jobs<Nb, LP>(r0, r1);
  const int n = n_items * (r1 - r0);
  for (int use = 0, t = 0, r = r0; use < n; ++use) {  // use: jobs of this plane type so far
    const int jj = t * JPT + r;
    const int slot = jj % kSlots;
    const int a2 = use & 1;
    if (!wait_bar(ctl, b_d1(slot), (jj / kSlots) & 1, 4, false, true)) return;
    if (use >= 2 && !wait_bar(ctl, b_a2_free(a2first + a2), ((use >> 1) - 1) & 1, 4, false, true)) return;
    tc_fence_after();
    const uint32_t ahi = a2base + a2 * 2 * lo_off;
    const uint32_t td = tq + slot * kSlotCols;
    epilogue1<Nb, LP>(td + kD1Off, td, ahi, ahi + lo_off, q, lane, s1inv, hi0, lo);
    tmem_wait_st();
    fence_proxy_async_smem();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ctl.bars[b_a2_full(a2first + a2)]);
    if (++r == r1) {
      r = r0;
      ++t;
    }
  }
}

// Epilogue 2: Z, the block energy H and brightness L, for every job of one plane type.
template <int Nb, bool LP, bool DUMP, class PP, class MS>
__device__ void epi2_loop(const PP& p, const MS& ms, const Ctl& ctl, uint32_t tq, int n_items, int item0,
                          int step, int q, int lane) {
  using P = PC<Nb, LP>;
  constexpr int JPT = Jobs<LP>::PER_TILE;
  const float* Wt = Nb == 32 ? p.W_y : p.W_c;
  float w[P::NK];
#pragma unroll
  for (int u = 0; u < P::NK; ++u) w[u] = Wt[u * Nb + (lane % P::NK)];
  const float einv = Nb == 32 ? 0.125f : 0.25f;
  const float c2 = Nb == 32 ? kK1 - kK1 / 8.0f : kK1 - kK1 / 4.0f;
  int r0, r1;
  plane_jobs<Nb, LP>(r0, r1);
  const int n = n_items * (r1 - r0);
  JobCtx jc{};
  int m = 0;
  for (int k = 0, t = 0, r = r0; k < n; ++k) {
    if (r == r0) {
      const TileInfo ti = tile_info(ms, t, item0, step);
      jc.f = ti.f;
      jc.tx = ti.tx;
      jc.ty = ti.ty;
      m = ti.m;
    }
    const int jj = t * JPT + r;
    const int slot = jj % kSlots;
    plane_of<LP>(r, jc.plane, jc.jp);
    if (!wait_bar(ctl, b_d2(slot), (jj / kSlots) & 1, 4, false, true)) return;
    tc_fence_after();
    epilogue2<Nb, LP, DUMP>(p.zdump, ms[m], tq + slot * kSlotCols, jc, q, lane, w, einv, c2,
                            &ctl.bars[b_slot_free(slot)]);
    if (++r == r1) {
      r = r0;
      ++t;
    }
  }
}

template <bool LP, bool DUMP, int BPS, bool BATCH>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(const __grid_constant__ TcParamsT<BATCH ? kMaxMembers : 1> p) {
  using L = PC<32, LP>;
  using Cc = PC<16, LP>;
  constexpr int JPT = Jobs<LP>::PER_TILE;
  static_assert(kSlots % JPT == 0, "a TMEM slot must always hold the same plane type");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  using SL = SmemLay<BPS>;
  uint64_t* bars = (uint64_t*)(sm + SL::OFF_BAR);
  uint32_t* tmem_slot = (uint32_t*)(sm + SL::OFF_MISC);
  volatile int* abort_flag = (volatile int*)(sm + SL::OFF_MISC + 4);
  const int tid = threadIdx.x;
  const int warp = tid >> 5;
  const int lane = tid & 31;
  const int role = warp >> 2;  // warpgroup
  const int q = warp & 3;      // TMEM lane quarter of this warp
  const int cta = blockIdx.x;
  const int grid = gridDim.x;
  const int total_items = p.total_items;
  // This CTA's items: item0, item0 + step, ...  A single analyzer's CTAs take every grid-th item
  // (neighbouring CTAs read neighbouring tiles); a batched launch gives each CTA one contiguous
  // run, so that a CTA meets few members (and few tensor maps).
  int item0, step, n_items;
  if (BATCH) {
    item0 = (int)((int64_t)cta * total_items / grid);
    n_items = (int)((int64_t)(cta + 1) * total_items / grid) - item0;
    step = 1;
  } else {
    item0 = cta;
    n_items = cta < total_items ? (total_items - cta + grid - 1) / grid : 0;
    step = grid;
  }
  const int n_jobs = n_items * JPT;
  Ctl ctl{bars, abort_flag, p.err};

  using MS = typename MemberView<BATCH>::T;
  MS ms = [&] {
    if constexpr (BATCH)
      return MemberTable{p.mem, p.n_members, 0};
    else
      return OneMember{p.mem[0]};
  }();

  // Constant B operands (the integer DCT matrices as fp16), K-major without swizzle:
  // element (n, k) at (n/8)*SBO + (k/8)*128 + (n%8)*16 + (k%8)*2.
  for (int i = tid; i < L::N1 * 32; i += kThreads) {
    const int n = i >> 5, kk = i & 31;
    const __half h = __float2half_rn((float)p.M_y[n * 32 + kk]);
    *(__half*)(sm + SL::OFF_BL + (n >> 3) * 512 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) = h;
  }
  for (int i = tid; i < 16 * 16; i += kThreads) {
    const int n = i >> 4, kk = i & 15;
    const __half h = __float2half_rn((float)p.M_c[n * 16 + kk]);
    *(__half*)(sm + SL::OFF_BC + (n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) = h;
  }
  // Stage-1 presets, applied by one more MMA per job ahead of the data: D1 = U x K^T with N = G N1
  // (the job's groups side by side).  Every row of U is (1024, 1, 0, ...), so column n of D1
  // starts at 1024 a_n + b_n for row n of K = (a_n, b_n, 0, ...): 2^(s1-1), the rounding offset
  // of T, minus 1024 * 64 * N in each group's DC column (the bias of the 1024 + x sample
  // encoding), split as a = -(multiple of 8 below 2^11) and b = P - 1024 a (|b| < 2^13, a multiple
  // of 8), both exact in fp16.
  for (int i = tid; i < 128 * 16; i += kThreads) {
    const int m = i >> 4, kk = i & 15;
    const float v = kk == 0 ? 1024.0f : kk == 1 ? 1.0f : 0.0f;
    *(__half*)(sm + SL::OFF_ONE + (m >> 3) * 256 + (kk >> 3) * 128 + (m & 7) * 16 + (kk & 7) * 2) = __float2half_rn(v);
  }
  for (int i = tid; i < 2 * 32 * 16; i += kThreads) {
    const int kk = i & 15, n = (i >> 4) & 31;
    const bool luma = i < 32 * 16;
    const int N = luma ? 32 : 16, N1 = luma ? L::N1 : Cc::N1, G = luma ? L::G : Cc::G;
    if (n >= G * N1) continue;
    const int P = (1 << (s1_of<32>(BPS) - (luma ? 1 : 2))) - (n % N1 == 0 ? 1024 * 64 * N : 0);
    const int a = P >= 0 ? (P >> 10) & ~7 : -(((-P) >> 10) & ~7);
    const float v = kk == 0 ? (float)a : kk == 1 ? (float)(P - a * 1024) : 0.0f;
    *(__half*)(sm + (luma ? SL::OFF_KL : SL::OFF_KC) + (n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) =
        __float2half_rn(v);
  }
  if (tid == 0) {
    for (int i = 0; i < kBars; ++i) mbar_init(&bars[i], 1);
    for (int i = 0; i < SL::kStages; ++i) mbar_init(&bars[b_raw_empty(i)], 8);  // both convert warpgroups
    for (int i = 0; i < kSlots; ++i) mbar_init(&bars[b_slot_free(i)], 4);
    for (int i = 0; i < kSlots; ++i) mbar_init(&bars[b_a1_full(i)], 4);
    for (int i = 0; i < kA2Slots; ++i) mbar_init(&bars[b_a2_full(i)], 4);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0 && lane == 0 && !BATCH) {
    prefetch_tensormap(&p.maps[0]);
    prefetch_tensormap(&p.maps[1]);
    prefetch_tensormap(&p.maps[2]);
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
  const uint32_t lanebase = (uint32_t)(32 * q) << 16;

  if (role == 0) {
    if (warp == 0 && lane == 0) {
      // ---------------- TMA producer: tiles in order into the ring ----------------
      int issued = 0;
      for (int t = 0; t < n_items; ++t) {
        const int stage = t % SL::kStages;
        if (t >= SL::kStages && !wait_bar(ctl, b_raw_empty(stage), ((t / SL::kStages) - 1) & 1, 1, false, true))
          break;
        const TileInfo ti = tile_info(ms, t, item0, step, SL::kStages);
        const CUtensorMap* mm = &p.maps[3 * ti.m];
        uint8_t* dst = sm + OFF_RAW + stage * SL::kStageBytes;
        uint64_t* full = &bars[b_raw_full(stage)];
        mbar_arrive_expect_tx(full, SL::kStageBytes);
        if (BPS == 1) {
          tma_load_3d(dst, mm, ti.tx * 128, ti.ty * 128, ti.f, full);
        } else {  // 16-bit luma: the tile is two 64-sample boxes side by side
          tma_load_3d(dst, mm, ti.tx * 128, ti.ty * 128, ti.f, full);
          tma_load_3d(dst + 128 * 64 * 2, mm, ti.tx * 128 + 64, ti.ty * 128, ti.f, full);
        }
        tma_load_3d(dst + SL::kRawY, mm + 1, ti.tx * 64, ti.ty * 64, ti.f, full);
        tma_load_3d(dst + SL::kRawY + SL::kRawC, mm + 2, ti.tx * 64, ti.ty * 64, ti.f, full);
        ++issued;
      }
      if (*abort_flag) {
        // Let every copy this CTA issued land before the CTA's shared memory goes away.
        for (int t = (issued > SL::kStages ? issued - SL::kStages : 0); t < issued; ++t)
          wait_bar(ctl, b_raw_full(t % SL::kStages), (t / SL::kStages) & 1, 1, true);
      }
    } else if (warp == 1 && lane == 0) {
      // ---------------- stage-1 MMA issuer: D1 = U x K^T (presets), then D1 += A1 (TMEM) x M^T ----------------
      const uint32_t bl = sbase + SL::OFF_BL, bc = sbase + SL::OFF_BC;
      const uint64_t du = smem_desc(sbase + SL::OFF_ONE, 128, 256, 0);
      const uint64_t dkl = smem_desc(sbase + SL::OFF_KL, 128, 256, 0), dkc = smem_desc(sbase + SL::OFF_KC, 128, 256, 0);
      constexpr uint32_t idPL = idesc_f16(128, L::G * L::N1, 0, 0), idPC = idesc_f16(128, Cc::G * Cc::N1, 0, 0);
      constexpr uint32_t idL = idesc_f16(128, L::N1, 0, 0), idC = idesc_f16(128, Cc::N1, 0, 0);
      bool ok = true;
      for (int j = 0; j < n_jobs; ++j) {
        int plane, jp;
        plane_of<LP>(j % JPT, plane, jp);
        const int slot = j % kSlots;
        if (!wait_bar(ctl, b_a1_full(slot), (j / kSlots) & 1, 2)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t a = tmem + slot * kSlotCols;
        const uint32_t d = a + kD1Off;
        if (plane == 0) {
          mma_ss(d, du, dkl, idPL, 0);  // presets of the job's groups
          // K-step outer: consecutive MMAs write different accumulators.
#pragma unroll
          for (int ks = 0; ks < 2; ++ks)
#pragma unroll
            for (int gg = 0; gg < L::G; ++gg)
              mma_ts(d + gg * L::N1, a + gg * L::A1COLS + ks * 8, smem_desc(bl + ks * 256, 128, 512, 0), idL, 1);
        } else {
          mma_ss(d, du, dkc, idPC, 0);
#pragma unroll
          for (int gg = 0; gg < Cc::G; ++gg)
            mma_ts(d + gg * Cc::N1, a + gg * Cc::A1COLS, smem_desc(bc, 128, 256, 0), idC, 1);
        }
        mma_commit(&bars[b_d1(slot)]);
      }
      if (!ok) {
        mma_commit(&bars[b_drain(0)]);
        wait_bar(ctl, b_drain(0), 0, 2, true);
      }
    } else if (warp == 2 && lane == 0) {
      // ---------------- stage-2 MMA issuer: D2 += A2 (smem, MN-major) x M^T, hi and lo (D2 pre-set by epilogue 1) ----------------
      const uint32_t bl = sbase + SL::OFF_BL, bc = sbase + SL::OFF_BC;
      constexpr uint32_t id2L = idesc_f16(128, L::N1, 1, 0), id2C = idesc_f16(128, Cc::N1, 1, 0);
      bool ok = true;
      for (int j = 0; j < n_jobs; ++j) {
        int plane, jp;
        plane_of<LP>(j % JPT, plane, jp);
        int a2, use;
        a2_slot_of<LP>(j, a2, use);
        if (!wait_bar(ctl, b_a2_full(a2), use & 1, 2)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem + (j % kSlots) * kSlotCols;
        const uint32_t ahi = a2_addr<BPS>(sbase, a2);
        if (plane == 0) {
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint64_t b = smem_desc(bl + ks * 256, 128, 512, 0);
            mma_ss(d, smem_desc(ahi + ks * 4096, 1024, 2048, 2), b, id2L, 1);
            mma_ss(d + L::N1, smem_desc(ahi + kA2L + ks * 4096, 1024, 2048, 2), b, id2L, 1);
          }
        } else {
          const uint64_t b = smem_desc(bc, 128, 256, 0);
          mma_ss(d, smem_desc(ahi, 1024, 2048, 2), b, id2C, 1);
          mma_ss(d + Cc::N1, smem_desc(ahi + kA2C, 1024, 2048, 2), b, id2C, 1);
        }
        mma_commit(&bars[b_d2(j % kSlots)]);
        mma_commit(&bars[b_a2_free(a2)]);
      }
      if (!ok) {
        mma_commit(&bars[b_drain(1)]);
        wait_bar(ctl, b_drain(1), 0, 2, true);
      }
    }
  } else if (role == 1) {
    convert_loop<32, LP, BPS>(ms, ctl, sm, tmem + lanebase, n_items, item0, step, q, lane);
  } else if (role == 6) {
    convert_loop<16, LP, BPS>(ms, ctl, sm, tmem + lanebase, n_items, item0, step, q, lane);
  } else if (role == 2) {
    epi1_loop<32, LP, BPS>(ms, ctl, sbase, tmem + lanebase, n_items, item0, step, q, lane);
  } else if (role == 3) {
    epi1_loop<16, LP, BPS>(ms, ctl, sbase, tmem + lanebase, n_items, item0, step, q, lane);
  } else if (role == 4) {
    epi2_loop<32, LP, DUMP>(p, ms, ctl, tmem + lanebase, n_items, item0, step, q, lane);
  } else {
    epi2_loop<16, LP, DUMP>(p, ms, ctl, tmem + lanebase, n_items, item0, step, q, lane);
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
                     int box_w, int box_h, int bps, CUtensorMapSwizzle sw) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  if (nframes == 1 || fstride <= 0) fstride = ((pitch * h + 15) / 16) * 16;
  cuuint64_t dims[3] = {(cuuint64_t)w, (cuuint64_t)h, (cuuint64_t)nframes};
  cuuint64_t strides[2] = {(cuuint64_t)pitch, (cuuint64_t)fstride};
  cuuint32_t boxd[3] = {(cuuint32_t)box_w, (cuuint32_t)box_h, 1};
  cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = bps == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
  CUresult r = enc(m, dt, 3, const_cast<void*>(base), dims, strides, boxd, es,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Raises the instance's dynamic shared-memory limit (once per process).
template <bool LP, bool DUMP, int BPS, bool BATCH>
cudaError_t prepare_inst() {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(tc_kernel<LP, DUMP, BPS, BATCH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SmemLay<BPS>::kSmemBytes);
  });
  return attr;
}

// grid 0: only prepare the instance.
template <bool LP, bool DUMP, int BPS, bool BATCH>
cudaError_t launch_inst(const TcParamsT<BATCH ? kMaxMembers : 1>& p, int grid, cudaStream_t s) {
  const cudaError_t attr = prepare_inst<LP, DUMP, BPS, BATCH>();
  if (attr != cudaSuccess) return attr;
  if (grid <= 0) return cudaSuccess;
  tc_kernel<LP, DUMP, BPS, BATCH><<<grid, kThreads, SmemLay<BPS>::kSmemBytes, s>>>(p);
  return cudaGetLastError();
}

// A single analyzer's launch (bps 1 or 2).
cudaError_t launch_single(const TcParams& p, int grid, bool low_pass, bool dump, int bps, cudaStream_t s) {
  if (bps == 1) {
    if (low_pass)
      return dump ? launch_inst<true, true, 1, false>(p, grid, s) : launch_inst<true, false, 1, false>(p, grid, s);
    return dump ? launch_inst<false, true, 1, false>(p, grid, s) : launch_inst<false, false, 1, false>(p, grid, s);
  }
  if (low_pass)
    return dump ? launch_inst<true, true, 2, false>(p, grid, s) : launch_inst<true, false, 2, false>(p, grid, s);
  return dump ? launch_inst<false, true, 2, false>(p, grid, s) : launch_inst<false, false, 2, false>(p, grid, s);
}

// A batched launch of members of one sample size (bps 1 or 2).
cudaError_t launch_batched(const TcBatchParams& p, int grid, bool low_pass, int bps, cudaStream_t s) {
  if (bps == 1)
    return low_pass ? launch_inst<true, false, 1, true>(p, grid, s) : launch_inst<false, false, 1, true>(p, grid, s);
  return low_pass ? launch_inst<true, false, 2, true>(p, grid, s) : launch_inst<false, false, 2, true>(p, grid, s);
}

// One member's entry: geometry, outputs and stage-1 constants; returns its number of items.
int fill_member(TcMember& m, const Geometry& g, int item_base, int nframes, float* blockvals) {
  m = TcMember{};
  m.item_base = item_base;
  m.tiles_x = (g.nbx + 3) / 4;
  m.tiles_per_frame = m.tiles_x * ((g.nby + 3) / 4);
  m.inv_tiles_x = 1.0f / (float)m.tiles_x;
  m.inv_tiles_per_frame = 1.0f / (float)m.tiles_per_frame;
  m.W = g.W;
  m.H = g.H;
  m.cw = g.cw;
  m.ch = g.ch;
  m.nbx = g.nbx;
  m.nby = g.nby;
  m.C = g.C;
  m.out_fstride = (int64_t)N_ROWS * g.C;
  m.blockvals = blockvals;
  return m.tiles_per_frame * nframes;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

}  // namespace

bool tc_supported(const Geometry& g) {
  return (g.B == 8 || g.B == 10) && g.w == 32 && g.nc == 16 && g.s1y == s1_of<32>(g.bps) &&
         g.s1c == s1_of<16>(g.bps) && encode_fn() != nullptr;
}

struct TcMapCache {
  static constexpr int kEntries = 8;
  struct Entry {
    const void *y, *u, *v;
    int64_t pitch_y, pitch_uv;
    CUtensorMap m[3];
  };
  Entry e[kEntries];
  int n = 0, next = 0;  // entries in use; the one replaced next (oldest first)
};

TcMapCache* tc_map_cache_new() { return new (std::nothrow) TcMapCache(); }

void tc_map_cache_free(TcMapCache* c) { delete c; }

int tc_batch_max_members() { return kMaxMembers; }

size_t tc_batch_params_bytes() { return sizeof(TcBatchParams); }

cudaError_t tc_batch_fill(void* params, const TcBatchFrame* frames, int n, const DeviceTables& t, int* err) {
  if (n < 0 || n > kMaxMembers) return cudaErrorInvalidValue;
  TcBatchParams& p = *static_cast<TcBatchParams*>(params);
  p.zdump[0] = p.zdump[1] = p.zdump[2] = nullptr;
  p.M_y = t.M_y;
  p.M_c = t.M_c;
  p.W_y = t.W_y;
  p.W_c = t.W_c;
  p.err = err;
  int items = 0;
  for (int i = 0; i < n; ++i) {
    const Geometry& g = *frames[i].g;
    const FramePlanes& fp = frames[i].fp;
    if (!tc_supported(g) || g.bps != frames[0].g->bps) return cudaErrorInvalidValue;
    items += fill_member(p.mem[i], g, items, 1, frames[i].blockvals);
    TcMapCache* c = frames[i].maps;
    const TcMapCache::Entry* hit = nullptr;
    for (int j = 0; c && j < c->n && !hit; ++j) {
      const TcMapCache::Entry& x = c->e[j];
      if (x.y == fp.y && x.u == fp.u && x.v == fp.v && x.pitch_y == fp.pitch_y && x.pitch_uv == fp.pitch_uv) hit = &x;
    }
    if (hit) {
      std::memcpy(&p.maps[3 * i], hit->m, sizeof hit->m);
      continue;
    }
    const CUtensorMapSwizzle swc = g.bps == 1 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    cudaError_t e = make_map(&p.maps[3 * i], fp.y, g.W, g.H, fp.pitch_y, 0, 1, g.bps == 1 ? 128 : 64, 128, g.bps,
                             CU_TENSOR_MAP_SWIZZLE_128B);
    if (e == cudaSuccess) e = make_map(&p.maps[3 * i + 1], fp.u, g.cw, g.ch, fp.pitch_uv, 0, 1, 64, 64, g.bps, swc);
    if (e == cudaSuccess) e = make_map(&p.maps[3 * i + 2], fp.v, g.cw, g.ch, fp.pitch_uv, 0, 1, 64, 64, g.bps, swc);
    if (e != cudaSuccess) return e;
    if (c) {
      TcMapCache::Entry& x = c->e[c->next];
      x.y = fp.y;
      x.u = fp.u;
      x.v = fp.v;
      x.pitch_y = fp.pitch_y;
      x.pitch_uv = fp.pitch_uv;
      std::memcpy(x.m, &p.maps[3 * i], sizeof x.m);
      c->next = (c->next + 1) % TcMapCache::kEntries;
      if (c->n < TcMapCache::kEntries) ++c->n;
    }
  }
  p.n_members = n;
  p.total_items = items;
  return cudaSuccess;
}

int tc_batch_items(const void* params) { return static_cast<const TcBatchParams*>(params)->total_items; }

cudaError_t tc_batch_prepare(int bps, bool low_pass) {
  if (bps != 1 && bps != 2) return cudaErrorInvalidValue;
  static TcBatchParams unused{};
  return launch_batched(unused, 0, low_pass, bps, nullptr);
}

cudaError_t launch_tc_batch(const void* params, int bps, bool low_pass, cudaStream_t s) {
  if (bps != 1 && bps != 2) return cudaErrorInvalidValue;
  // The number of items is known from the parameters; CTAs beyond it find no work.
  return launch_batched(*static_cast<const TcBatchParams*>(params), sm_count(), low_pass, bps, s);
}

const void* tc_batch_kernel(int bps, bool low_pass) {
  if (bps == 1)
    return low_pass ? (const void*)tc_kernel<true, false, 1, true> : (const void*)tc_kernel<false, false, 1, true>;
  return low_pass ? (const void*)tc_kernel<true, false, 2, true> : (const void*)tc_kernel<false, false, 2, true>;
}

cudaError_t launch_tc(const Geometry& g, const FramePlanes& fp, int nframes, const DeviceTables& t, float* blockvals,
                      int16_t* const zdump[3], int* err, cudaStream_t s, int64_t* launches) {
  if (!tc_supported(g)) return cudaErrorNotSupported;
  if (nframes <= 0) return cudaSuccess;
  // 8-bit: 128x128 luma boxes (128-byte swizzle), 64x64 chroma boxes (64-byte swizzle); 16-bit:
  // 64x128 luma boxes (two per tile) and 64x64 chroma boxes, all 128-byte rows and swizzle.
  const int bps = g.bps;
  const CUtensorMapSwizzle swc = bps == 1 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  CUtensorMap my, mu, mv;
  cudaError_t e = make_map(&my, fp.y, g.W, g.H, fp.pitch_y, fp.fstride_y, nframes, bps == 1 ? 128 : 64, 128, bps,
                           CU_TENSOR_MAP_SWIZZLE_128B);
  if (e == cudaSuccess) e = make_map(&mu, fp.u, g.cw, g.ch, fp.pitch_uv, fp.fstride_uv, nframes, 64, 64, bps, swc);
  if (e == cudaSuccess) e = make_map(&mv, fp.v, g.cw, g.ch, fp.pitch_uv, fp.fstride_uv, nframes, 64, 64, bps, swc);
  if (e != cudaSuccess) return e;
  TcParams p{};
  p.n_members = 1;
  p.total_items = fill_member(p.mem[0], g, 0, nframes, blockvals);
  p.maps[0] = my;
  p.maps[1] = mu;
  p.maps[2] = mv;
  for (int i = 0; i < 3; ++i) p.zdump[i] = zdump ? zdump[i] : nullptr;
  p.M_y = t.M_y;
  p.M_c = t.M_c;
  p.W_y = t.W_y;
  p.W_c = t.W_c;
  p.err = err;
  const int grid = p.total_items < sm_count() ? p.total_items : sm_count();
  e = launch_single(p, grid, g.low_pass, zdump != nullptr, bps, s);
  if (e == cudaSuccess) ++*launches;
  return e;
}

}  // namespace vca
