// Tensor-core form of the analyzer's per-block work (Section 2 of the paper: integer DCT of
// every Y, U, V block, texture energy H and brightness L; Section 2 item (3): low-pass).
//
// Persistent kernel, one CTA of 32 warps per SM.  A work item is one 128x128 luma tile and the
// two co-located 64x64 chroma tiles; it is processed as one unit (low-pass) or two units of half
// its block rows (all coefficients).  Roles:
//   warp 0        TMA producer: tiles in order into a ring (8-bit samples: 4 stages of one
//                 128x128 luma box, 128-byte swizzle, and two 64x64 chroma boxes, 64-byte
//                 swizzle; 10-bit samples as 16-bit words: 2 stages, the luma tile as two
//                 64-sample boxes, all 128-byte swizzled), and each tile's record (frame,
//                 position, distance to the frame's edges) into a ring in shared memory;
//   warps 1-7     MMA issuers (tcgen05.mma kind::f16, FP32 accumulate), one thread each with fixed
//                 streams: stage 1 of luma job 0, of luma job 1, of chroma; stage 2 of luma job 0,
//                 of luma job 1, of the chroma hi and of the chroma lo operands.  A thread is held
//                 for over a hundred cycles by every MMA it issues, however small, while MMAs
//                 from different warps overlap in the tensor pipe, so the issue is spread out;
//   warpgroup 2   convert luma, warpgroup 3 convert chroma: raw samples -> stage-1 A operands
//                 in TMEM;
//   warpgroup 4   epilogue 1 luma: stage-1 accumulators -> stage-2 A operand in shared memory;
//   warpgroup 5   epilogue 2 luma: stage-2 accumulators -> block energies and brightness;
//   warpgroups 6, 7  epilogue 1 and epilogue 2 chroma (U and V together).
// Each role waits once per unit.  TMEM holds 2 stage-1 operand slots and 3 (low-pass) or 2
// accumulator slots, shared memory 2 sets of stage-2 operands, so up to 3 units are in flight.
// Every SM sub-partition runs warps of every role (each role spans the four TMEM lane quarters),
// so its instruction cache holds the whole kernel: per-unit loops stay rolled and rare paths
// (tiles on a frame's right edge) out of line.
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
//             pre-set to the magic constants of epilogue 2 by one more MMA per stream;
//   epilogue2 Z = floor((256 S_hi + S_lo + 2^(s2-1)) / 2^s2) by two round-down FMAs, then
//             H_v = sum_u w(u,v) |Z| in increasing u and an xor tree over v.
// U and V share their MMAs: a U row and a V row lie side by side along K and the B operand holds
// the chroma matrix in the U half of N for the U K-step and in the V half for the V K-step.
// Every partial sum is an integer below 2^24 in magnitude (or in [2^23, 2^24) for the
// pre-offset accumulators), so the FP32 tensor-core accumulation is exact and Z is
// bit-identical to the integer definition; H uses the same FP32 order as the CUDA-core form.
//
// 4:4:4 (C444): the chroma planes have the luma plane's size, blocks and matrix, so each 128x128
// tile of each plane is a work item of its own through the luma roles (the chroma roles and
// issuers stay idle); epilogue 2 writes the item's plane's rows.
//
// 16x16 luma / 8x8 chroma blocks run the same data flow on 32x32 / 16x16 super-blocks of four
// blocks each: the DCT matrix appears twice along the diagonal of every B operand (rows first:
// the left and right halves of a super-block row get separate transforms; columns: the top and
// bottom halves), the presets and shifts are those of the smaller transform, and epilogue 2 sums
// each quadrant of a super-block's coefficients into its own block energy.
//
// A launch covers one analyzer's frames (its geometry in the kernel parameters) or, for a batched
// tick, one frame of each of up to 64 analyzers of one sample size (a member table and their
// tensor maps, also in the kernel parameters, read through the constant cache).
//
// Every wait is bounded (about two seconds, or the launch's wait limit); on timeout the kernel
// raises a flag in *err, stops, waits for its own copies and MMAs, frees TMEM and returns.  A
// launch may name one work item whose copies the producer withholds, so that the wait for it
// runs out (the failure path's test).
#include <cuda.h>
#include <cuda_fp16.h>

#include <climits>
#include <cstring>
#include <mutex>
#include <new>

#include "vca_fixed.cuh"
#include "vca_internal.h"
#include "vca_ptx.cuh"

namespace vca {
namespace {

using namespace ptx;

constexpr int kMaxStages = 4;   // raw tile ring (barrier indices are laid out for the longest)
constexpr int kA2L = 8192;      // one stage-2 operand (hi or lo) of one luma job: 128 rows x 32 K x fp16
constexpr int kA2C = 4096;      // of one chroma job: 128 rows x 16 K x fp16
constexpr int kA2Unit = 2 * 2 * kA2L + 2 * 2 * kA2C;  // a unit's: luma jobs 0-1, then U and V; hi, lo each
constexpr int OFF_RAW = 0;
constexpr int kASlots = 2;      // stage-1 operand (A1) slots in TMEM
constexpr int kA2Sets = 2;      // stage-2 operand sets in shared memory
constexpr int kIssuers = 7;     // MMA-issuing threads (warps 1-7, lane 0)
constexpr int kMaxMembers = kMaxBatchMembers;

// One analyzer ("member") of a launch: its work items, geometry, outputs and stage-1 constants.
// A single analyzer's launch has one member with all its frames; a batched tick has one member
// per channel with one frame each.  Items are numbered member by member, frame-major tiles.
struct TcMember {
  int item_base;                   // first item of this member
  int tiles_x, tiles_per_frame;    // tiles_per_frame counts a 4:4:4 frame's three planes
  float inv_tiles_x, inv_tiles_per_frame;
  int tiles_per_plane;             // 4:4:4: the tiles of one plane (plane p: items p T .. (p+1) T - 1)
  float inv_tiles_per_plane;
  int W, H, cw, ch, nbx, nby;
  int64_t C, out_fstride;
  float* blockvals;
  int red, red_flags;              // batched ticks: entry in the fused reduction's table, flags
  int pad_[2];
};

// Stage-1 shift s1 = log2 N + B - 9 of an N-point transform; the bit depth follows from the sample
// size (8-bit samples in bytes, 10-bit in 16-bit words).
__host__ __device__ constexpr int s1_of(int N, int bps) {
  return (N == 32 ? 5 : N == 16 ? 4 : 3) + (bps == 1 ? 8 : 10) - 9;
}

// Block sizes of a launch: 32x32 luma and 16x16 chroma blocks, or (SUB) 16x16 luma and 8x8
// chroma blocks processed as the four quadrants of each 32x32 / 16x16 area ("super-block").
// Every operand, MMA and layout is the one of the 32x32 form; the B operands hold the smaller
// matrix twice along the diagonal, so that the two halves of a super-block row (stage 1) or
// column (stage 2) take separate transforms, and epilogue 2 sums each quadrant on its own.
template <bool SUB>
struct Blk {
  static constexpr int NL = SUB ? 16 : 32;  // luma block size
  static constexpr int NC = SUB ? 8 : 16;   // chroma block size
};
static_assert(sizeof(TcMember) % 8 == 0, "member table entries are copied as words");
static_assert(sizeof(TcRedMember) % 8 == 0, "reduction entries are copied as words");


// Shared-memory layout for BPS bytes per sample.  8-bit: a 128x128 luma tile (128-byte rows,
// 128-byte swizzle) and two 64x64 chroma tiles (64-byte rows and swizzle), 4 stages.  10-bit
// (16-bit words): the luma tile as two 64-sample-wide boxes side by side (128-byte rows each,
// 128-byte swizzle) and 64x64 chroma tiles with 128-byte rows and swizzle, 2 stages.  Then two
// sets of stage-2 operands, the DCT matrices as B operands and the stage-1 preset operands.
template <int BPS>
struct SmemLay {
  static_assert(BPS == 1 || BPS == 2, "one sample size per launch");
  static constexpr int kStages = BPS == 1 ? 4 : 2;
  static constexpr int kRawY = 128 * 128 * BPS;
  static constexpr int kRawC = 64 * 64 * BPS;
  static constexpr int kStageBytes = kRawY + 2 * kRawC;
  static constexpr int OFF_A2 = kStages * kStageBytes;         // kA2Sets x kA2Unit
  static constexpr int OFF_BL = OFF_A2 + kA2Sets * kA2Unit;    // luma DCT matrix (32 x 32 fp16)
  static constexpr int OFF_BCU = OFF_BL + 2048;                // chroma matrix in the U half of N (32 x 16)
  static constexpr int OFF_BCV = OFF_BCU + 1024;               // and in the V half
  static constexpr int OFF_ONE = OFF_BCV + 1024;               // preset operand U (128 x 16)
  static constexpr int OFF_KL = OFF_ONE + 4096;                // preset operand K, luma (32 x 16)
  static constexpr int OFF_KC = OFF_KL + 1024;                 // and chroma (32 x 16)
  static constexpr int OFF_K2L = OFF_KC + 1024;                // stage-2 preset operand, luma hi and lo (64 x 16)
  static constexpr int OFF_K2CH = OFF_K2L + 2048;              // chroma hi (32 x 16)
  static constexpr int OFF_K2CL = OFF_K2CH + 1024;             // chroma lo (32 x 16)
  static constexpr int OFF_REC = OFF_K2CL + 1024;              // tile records (16 x 32 B)
  static constexpr int OFF_BAR = OFF_REC + 16 * 32;
  static constexpr int OFF_MISC = OFF_BAR + 48 * 8;
  static constexpr int OFF_REDTAB = OFF_MISC + 64;            // batched ticks: the CTA's members' reduction entries
  static constexpr int kSmemBytes = OFF_REDTAB + kMaxMembers * (int)sizeof(TcRedMember) + 1024;  // + alignment slack
  static_assert(kStages <= kMaxStages && OFF_A2 % 1024 == 0 && kA2Unit % 1024 == 0 && kSmemBytes <= 232448,
                "layout");
};

// Stage-2 operand (hi; lo follows at +kA2L / +kA2C) of luma job j or chroma plane p of an operand set.
__device__ __forceinline__ uint32_t a2_luma(uint32_t a2set, int j) { return a2set + j * 2 * kA2L; }
__device__ __forceinline__ uint32_t a2_chroma(uint32_t a2set, int p) { return a2set + 4 * kA2L + p * 2 * kA2C; }

// barrier indices: the raw ring; per A1 slot; per accumulator slot; per stage-2 operand set
__host__ __device__ constexpr int b_raw_full(int s) { return s; }
__host__ __device__ constexpr int b_raw_empty(int s) { return kMaxStages + s; }
__host__ __device__ constexpr int b_a1l_full(int a) { return 8 + a; }    // convert luma -> stage-1 luma issuers
__host__ __device__ constexpr int b_a1c_full(int a) { return 10 + a; }   // convert chroma -> stage-1 chroma issuer
__host__ __device__ constexpr int b_a1l_free(int a) { return 12 + a; }   // stage-1 luma MMAs read A1
__host__ __device__ constexpr int b_a1c_free(int a) { return 14 + a; }   // stage-1 chroma MMAs read A1
__host__ __device__ constexpr int b_d1l(int d) { return 16 + d; }        // stage-1 luma MMAs done
__host__ __device__ constexpr int b_d1c(int d) { return 19 + d; }        // stage-1 chroma MMAs done
__host__ __device__ constexpr int b_a2l_full(int e) { return 22 + e; }   // epilogue 1 luma -> stage-2 issuers
__host__ __device__ constexpr int b_a2c_full(int e) { return 24 + e; }   // epilogue 1 chroma -> stage-2 issuers
__host__ __device__ constexpr int b_a2l_free(int e) { return 26 + e; }   // stage-2 luma MMAs read A2
__host__ __device__ constexpr int b_a2c_free(int e) { return 28 + e; }   // stage-2 chroma MMAs read A2
__host__ __device__ constexpr int b_d2l(int d) { return 30 + d; }        // stage-2 luma MMAs done
__host__ __device__ constexpr int b_d2c(int d) { return 33 + d; }        // stage-2 chroma MMAs done
__host__ __device__ constexpr int b_dfree(int d) { return 36 + d; }      // both epilogues 2 read the slot
__host__ __device__ constexpr int b_drain(int i) { return 39 + i; }
constexpr int kBars = 48;
static_assert(b_drain(kIssuers - 1) < kBars, "barrier area");

constexpr int kThreads = 1024;
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
  const TcRedMember* red;  // batched ticks: the fused reduction's member table (device)
  double* err_host;        // batched ticks: the tick's timeout flag (mapped host memory), or null
  long long wait_ns;  // limit of every bounded wait
  int withhold;       // work item whose copies the producer does not issue (-1: none; failure-path tests)
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
};

// A unit: the whole tile (low-pass) or half its block rows (all coefficients): two luma jobs and
// one job per chroma plane.  U and V share their MMAs: the chroma A operands put a U row and a V
// row side by side along K, and the B operand holds the chroma matrix in the U half of N for the
// U K-step and in the V half for the V K-step, so one accumulator holds U's coefficients and then
// V's (no padding of N for the 8 low-pass chroma coefficients).  TMEM holds kASlots stage-1
// operand slots and DS accumulator slots:
//   A1 slot   luma group g (one block row) at 16 g; chroma group g at A1C + 16 g (U 8 columns,
//             then V 8 columns);
//   D slot    luma D1 group g at g N1, then D2 of job j: hi at 2 j N1, lo at (2 j + 1) N1;
//             chroma D1 group g at DC + g NCC, then D2: hi at DC, lo at DC + NCC.
// A D2 that overlaps a D1 is written by the epilogue-1 warpgroup of the same plane type after it
// has read the whole D1.
template <bool LP>
struct Unit {
  using L = PC<32, LP>;
  using C = PC<16, LP>;
  static constexpr int UPT = LP ? 1 : 2;        // units per tile
  static constexpr int UR = LP ? 4 : 2;         // luma block rows (= luma stage-1 groups) per unit
  static constexpr int GC = UR / 2;             // chroma stage-1 groups per unit (two block rows each)
  static constexpr int NKC = C::NK;             // chroma coefficients kept per dimension
  static constexpr int NCC = 2 * NKC;           // chroma MMA N: U then V
  static constexpr int A1C = 16 * UR;
  static constexpr int A1COLS = A1C + 16 * GC;  // low-pass 96, all coefficients 48
  static constexpr int DC = LP ? 64 : 128;
  static constexpr int DCOLS = LP ? 96 : 192;
  static constexpr int DS = LP ? 3 : 2;         // accumulator slots (units in flight)
  static constexpr int DBASE = kASlots * A1COLS;
  static_assert(DBASE + DS * DCOLS <= (int)kTmemCols, "TMEM columns");
  static_assert(UR * L::N1 <= DC && 4 * L::N1 <= DC && DC + 2 * NCC <= DCOLS && DC + GC * NCC <= DCOLS, "D slot");
  static_assert(L::JOBS == 2 * UPT && C::JOBS == UPT && L::G * 2 == UR && C::G == GC, "jobs per unit");
  static __device__ __forceinline__ uint32_t a1(int a) { return (uint32_t)(a * A1COLS); }
  static __device__ __forceinline__ uint32_t d(int ds) { return (uint32_t)(DBASE + ds * DCOLS); }
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
  double* err_host;  // also set on timeout, if not null (batched ticks)
  uint64_t wait_ns;
};

// Bounded wait: false on timeout (flag raised) or when another role aborted.
__device__ __forceinline__ bool wait_bar_poll(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                              double* err_host, int code, bool ignore_abort, bool sleep,
                                              uint64_t wait_ns) {
  const uint64_t t0 = now_ns();
  for (;;) {
#pragma unroll 1
    for (int i = 0; i < 32; ++i)
      if (sleep ? mbar_try_wait_sleep(bar, parity) : mbar_try_wait(bar, parity)) return true;
    if (!ignore_abort && *abort_flag) return false;
    if (now_ns() - t0 > wait_ns) {
      *abort_flag = 1;
      atomicOr(err, code);
      if (err_host) *err_host = (double)code;
      return false;
    }
  }
}

__device__ __noinline__ bool wait_bar_slow(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err,
                                          double* err_host, int code, bool ignore_abort, bool sleep,
                                          uint64_t wait_ns) {
  return wait_bar_poll(bar, parity, abort_flag, err, err_host, code, ignore_abort, sleep, wait_ns);
}

// Bounded wait on barrier idx.  Roles on the critical path spin; the producer (sleep = true) lets
// its thread sleep in hardware between polls.  INL: the polling loop inline at every wait, which
// saves the call (and the registers it saves and restores) where first polls often fail -- the
// low-pass instances, 2 % faster; the all-coefficient instances, whose code is twice as large,
// run 4 % slower with it (instruction-cache misses), so they call one out-of-line copy.
template <bool INL>
__device__ __forceinline__ bool wait_bar(const Ctl& c, int idx, uint32_t parity, int code, bool ignore_abort = false,
                                         bool sleep = false) {
  uint64_t* bar = c.bars + idx;
  if (sleep ? mbar_try_wait_sleep(bar, parity) : mbar_try_wait(bar, parity)) return true;
  if constexpr (INL)
    return wait_bar_poll(bar, parity, c.abort, c.err, c.err_host, code, ignore_abort, sleep, c.wait_ns);
  else
    return wait_bar_slow(bar, parity, c.abort, c.err, c.err_host, code, ignore_abort, sleep, c.wait_ns);
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

// Sample words of 16 samples of row y from column x, columns from w_rem on repeating the last one
// (a frame's right edge).  Out of line: only edge tiles take it.
template <int Nb, int BPS>
__device__ __noinline__ void load_16_edge(uint32_t base, int y, int x, int w_rem, uint32_t* words) {
  constexpr int NW = BPS == 1 ? 4 : 8;
  for (int i = 0; i < NW; ++i) words[i] = 0;
  for (int c = 0; c < 16; ++c) {
    const int xx = min(x + c, w_rem - 1);
    if (BPS == 1)
      words[c >> 2] |= (uint32_t)lds_u8(base + raw_offset<Nb, 1>(y, xx)) << (8 * (c & 3));
    else
      words[c >> 1] |= (uint32_t)lds_u16(base + raw_offset<Nb, 2>(y, xx)) << (16 * (c & 1));
  }
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
      load_16_edge<Nb, 1>(base, y, x, w_rem, words);
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
      load_16_edge<Nb, 2>(base, y, x, w_rem, words);
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) out[i] = (words[i] & 0x03FF03FFu) | 0x64006400u;
  }
}

// Byte offsets within a stage-2 operand of this thread's 8-column chunks of a job (chunk st: group
// st / (NK / 8), columns 8 (st % (NK / 8)) ..): thread 32 q + lane holds row r = l % Nb of block
// l / Nb of each group, and writes stage-2 rows m = (g BPG1 + l / Nb) NK + h0 .. + 7 at K = r
// (MN-major, 128-byte swizzle: 8-row K groups of 2048 bytes, 64-row M atoms of 1024 bytes).
template <int Nb, bool LP>
struct E1Offs {
  static constexpr int S = PC<Nb, LP>::G * (PC<Nb, LP>::NK / 8);
  uint32_t off[S];
  __device__ __forceinline__ E1Offs(int q, int lane) {
    using P = PC<Nb, LP>;
    const int l = 32 * q + lane;
    const int bg = l / Nb, r = l % Nb;
    const uint32_t rowoff = (uint32_t)((r >> 3) * 2048 + (r & 7) * 128);
#pragma unroll
    for (int st = 0; st < S; ++st) {
      const int g = st / (P::NK / 8), h0 = (st % (P::NK / 8)) * 8;
      const int m = (g * P::BPG1 + bg) * P::NK + h0;
      off[st] = rowoff + (uint32_t)((m >> 6) * 1024) + (uint32_t)(((((m & 63) >> 3) ^ (r & 7))) << 4);
    }
  }
};

// Reads D1 of J jobs (job i: stage-1 accumulators at td1[i] + g*N1) and writes their stage-2
// operands to shared memory (hi at a2hi[i], lo lo_off bytes further), 8 columns at a time; the
// TMEM load of the next 8 columns (of the same job or the next) is in flight while this thread
// converts the current ones.  The low-pass roles take both jobs in one pipeline (J = 2); the
// all-coefficient ones, whose code is larger, one job per call (J = 1).
template <int Nb, bool LP, int J>
__device__ __forceinline__ void epilogue1(const uint32_t (&td1)[J], const uint32_t (&a2hi)[J], uint32_t lo_off,
                                          const E1Offs<Nb, LP>& eo, float s1inv) {
  using P = PC<Nb, LP>;
  constexpr int CPG = P::NK / 8;  // 8-column chunks per group
  constexpr int S1 = E1Offs<Nb, LP>::S;  // chunks per job
  constexpr int S = J * S1;
  const uint64_t s1inv2 = f2pack(__float_as_uint(s1inv), __float_as_uint(s1inv));
  const uint64_t kT1x2 = f2pack(__float_as_uint(kT1), __float_as_uint(kT1));
  uint32_t buf[2][8];
  tmem_ld<8>(td1[0], buf[0]);
#pragma unroll
  for (int st = 0; st < S; ++st) {
    tmem_wait_ld();
    if (st + 1 < S) {
      const int sn = (st + 1) % S1;
      tmem_ld<8>(td1[(st + 1) / S1] + (sn / CPG) * P::N1 + (sn % CPG) * 8, buf[(st + 1) & 1]);
    }
    const uint32_t(&acc)[8] = buf[st & 1];
    const uint32_t hiaddr = a2hi[st / S1] + eo.off[st % S1];
    uint32_t hi[4], lw[4];
#pragma unroll
    for (int k = 0; k < 8; k += 2) {
      // D1 already holds T' = c_k + sum (the accumulators were pre-set), an exact integer; two
      // columns per packed round-down FMA.
      float fa, fb;
      f2unpack(f2fma_rm(f2pack(acc[k], acc[k + 1]), s1inv2, kT1x2), fa, fb);
      const uint32_t za = __float_as_uint(fa), zb = __float_as_uint(fb);
      lw[k / 2] = prmt(za, zb, 0x6420);
      hi[k / 2] = prmt(za, zb, 0x6521);
    }
    sts128(hiaddr, hi[0], hi[1], hi[2], hi[3]);
    sts128(hiaddr + lo_off, lw[0], lw[1], lw[2], lw[3]);
  }
}

// The block value a thread of epilogue 2 stores, at most one (e2_store_job: of which job): without
// super-blocks the v = 0 thread of a block's NK lanes stores job 0's block and its v = NK/2 thread
// job 1's; with super-blocks (G = NK/2 lanes per block column group) lanes v = 0, G/4, G/2, 3G/4
// of the group store the top and bottom blocks of job 0, then of job 1.
template <bool SUB, int NK>
__device__ __forceinline__ int e2_store_job(int lane) {
  if constexpr (SUB) {
    constexpr int G = NK / 2;
    return ((lane % NK) % G) / (G / 4) >> 1;
  } else {
    return ((lane % NK) & (NK / 2)) ? 1 : 0;
  }
}

// This thread's store address for epilogue 2 (H at o[0], L at o[C]) without super-blocks: out[j]
// is job j's block of this thread's rows (null outside the frame).
template <int NK>
__device__ __forceinline__ float* e2_store(int lane, float* const (&out)[2]) {
  return ((lane % NK) & (NK / 2 - 1)) == 0 ? out[e2_store_job<false, NK>(lane)] : nullptr;
}

// The same for super-blocks: sb[j] is job j's super-block (x, y in super-blocks, x < 0: none),
// orow[j] the output row of its plane; null for threads that store nothing or blocks outside the
// frame.
template <int NK>
__device__ __forceinline__ float* e2_store_sub(int lane, const int2 (&sb)[2], float* const (&orow)[2], int nbx,
                                               int nby) {
  constexpr int G = NK / 2;
  const int vp = lane % NK, v = vp % G;
  if ((v % (G / 4)) != 0) return nullptr;
  const int quarter = v / (G / 4);
  const int j = quarter >> 1, dy = quarter & 1;
  const int bx = 2 * sb[j].x + vp / G, by = 2 * sb[j].y + dy;
  if (!orow[j] || sb[j].x < 0 || bx >= nbx || by >= nby) return nullptr;
  return orow[j] + (int64_t)by * nbx + bx;
}

// Epilogue 2 of two jobs of one plane type (luma: both luma jobs; chroma: U and V): for job j the
// stage-2 accumulators hi at td2[j] and lo at td2[j] + LO form Z, the row sums of w(u, v) |Z| in
// increasing u and the block energy H by an xor tree over the NK rows of the block; a thread with
// a store address o (e2_store) writes its block's H at o[0] and L = sqrt(Z(0,0)) at o[C].  DUMP:
// the coefficients to zd[j] (u-major) as well.  The TMEM loads of the next 8 columns are in flight
// while the current ones are processed.
template <int Nb, bool LP, bool DUMP, int LO>
__device__ __forceinline__ void epilogue2(const uint32_t (&td2)[2], int lane, const float (&wts)[PC<Nb, LP>::NK],
                                          float einv, float c2, float* o, int64_t C, int16_t* const (&zd)[2]) {
  using P = PC<Nb, LP>;
  constexpr int NK = P::NK;
  constexpr int CPJ = NK / 8;  // 8-column chunks per job
  constexpr int S = 2 * CPJ;
  const int v = lane % NK;
  const uint64_t k256 = f2pack(__float_as_uint(0.00390625f), __float_as_uint(0.00390625f));
  const uint64_t einv2 = f2pack(__float_as_uint(einv), __float_as_uint(einv));
  const uint64_t c22 = f2pack(__float_as_uint(c2), __float_as_uint(c2));
  const uint64_t mK1 = f2pack(__float_as_uint(-kK1), __float_as_uint(-kK1));
  uint32_t bh[2][8], bl[2][8];
  tmem_ld<8>(td2[0], bh[0]);
  tmem_ld<8>(td2[0] + LO, bl[0]);
  float H = 0.0f, H0 = 0.0f, z00 = 0.0f, z0 = 0.0f;
#pragma unroll
  for (int st = 0; st < S; ++st) {
    const int j = st / CPJ, h0 = (st % CPJ) * 8;
    tmem_wait_ld();
    if (st + 1 < S) {
      const uint32_t t1 = td2[(st + 1) / CPJ] + ((st + 1) % CPJ) * 8;
      tmem_ld<8>(t1, bh[(st + 1) & 1]);
      tmem_ld<8>(t1 + LO, bl[(st + 1) & 1]);
    }
#pragma unroll
    for (int uu = 0; uu < 8; uu += 2) {
      // Two rows u per packed instruction: w = lo/256 + hi and Z = floor(w 2^-(s2-8)) (round-down
      // FMAs), then the FMA chain of H in increasing u.
      const uint64_t w2 = f2fma_rm(f2pack(bl[st & 1][uu], bl[st & 1][uu + 1]), k256,
                                   f2pack(bh[st & 1][uu], bh[st & 1][uu + 1]));
      float z[2];
      f2unpack(f2add(f2fma_rm(w2, einv2, c22), mK1), z[0], z[1]);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int u = h0 + uu + e;
        if (u == 0) z00 = z[e];
        if (DUMP && zd[j]) zd[j][u * NK + v] = (int16_t)z[e];
        H = fmaf(fabsf(z[e]), wts[u], H);
      }
    }
    if (j == 0 && h0 + 8 == NK) {  // job 0 complete
      H0 = H;
      z0 = z00;
      H = 0.0f;
    }
  }
  // Both xor trees in one: the first stage sends job 1's row sum from the lower half of the block's
  // lanes and job 0's from the upper half, so that the lower half goes on with job 0 and the upper
  // half with job 1 -- every addition is the one of the separate trees (operands swapped at most).
  const bool upper = (v & (NK / 2)) != 0;
  float X = (upper ? H : H0) + __shfl_xor_sync(0xffffffffu, upper ? H0 : H, NK / 2);
#pragma unroll
  for (int o = NK / 4; o > 0; o >>= 1) X += __shfl_xor_sync(0xffffffffu, X, o);
  // job 1's Z(0,0) (held by its v = 0 lane) to the block's v = NK/2 lane; one square root for both
  const float z1 = __shfl_xor_sync(0xffffffffu, z00, NK / 2);
  const float L = __fsqrt_rn(upper ? z1 : z0);
  if (o) {
    o[0] = X;
    o[C] = L;
  }
}

// Epilogue 2 of super-blocks of four blocks (16x16 luma / 8x8 chroma blocks), two jobs as in
// epilogue2: thread (super-block, v') holds column v' of the super-block's coefficients, the left
// blocks' columns in v' < G and the right blocks' in v' >= G (G = NK / 2 coefficients per block
// and dimension), and rows u' < G of the top blocks, u' >= G of the bottom ones.  Each thread sums
// w(u, v) |Z| in increasing u separately for the top and bottom block of each job; four xor trees
// over the G lanes of a block, merged into one shuffle sequence, give the energies of the top and
// bottom blocks of both jobs, which lanes 0, G/4, G/2, 3G/4 of the G-lane group store at their
// address o (e2_store_sub; H at o[0], L = sqrt(Z(0,0)) of the block at o[C]).  sb[j]: super-block
// of job j (x, y in super-blocks); zd[j]: the coefficient dump of the plane (DUMP, frame 0).
template <int Nb, bool LP, bool DUMP, int LO>
__device__ __forceinline__ void epilogue2_sub(const uint32_t (&td2)[2], int lane, const float (&wts)[PC<Nb, LP>::NK / 2],
                                              float einv, float c2, const int2 (&sb)[2], float* o, int nbx, int nby,
                                              int64_t C, int16_t* const (&zd)[2]) {
  using P = PC<Nb, LP>;
  constexpr int NK = P::NK;
  constexpr int G = NK / 2;
  constexpr int CPJ = NK / 8;
  constexpr int S = 2 * CPJ;
  const int vp = lane % NK;
  const int v = vp % G;
  const uint64_t k256 = f2pack(__float_as_uint(0.00390625f), __float_as_uint(0.00390625f));
  const uint64_t einv2 = f2pack(__float_as_uint(einv), __float_as_uint(einv));
  const uint64_t c22 = f2pack(__float_as_uint(c2), __float_as_uint(c2));
  const uint64_t mK1 = f2pack(__float_as_uint(-kK1), __float_as_uint(-kK1));
  uint32_t bh[2][8], bl[2][8];
  tmem_ld<8>(td2[0], bh[0]);
  tmem_ld<8>(td2[0] + LO, bl[0]);
  float Ht[2] = {0.0f, 0.0f}, Hb[2] = {0.0f, 0.0f}, zt[2] = {0.0f, 0.0f}, zb[2] = {0.0f, 0.0f};
#pragma unroll
  for (int st = 0; st < S; ++st) {
    const int j = st / CPJ, h0 = (st % CPJ) * 8;
    tmem_wait_ld();
    if (st + 1 < S) {
      const uint32_t t1 = td2[(st + 1) / CPJ] + ((st + 1) % CPJ) * 8;
      tmem_ld<8>(t1, bh[(st + 1) & 1]);
      tmem_ld<8>(t1 + LO, bl[(st + 1) & 1]);
    }
#pragma unroll
    for (int uu = 0; uu < 8; uu += 2) {
      const uint64_t w2 = f2fma_rm(f2pack(bl[st & 1][uu], bl[st & 1][uu + 1]), k256,
                                   f2pack(bh[st & 1][uu], bh[st & 1][uu + 1]));
      float zz[2];
      f2unpack(f2add(f2fma_rm(w2, einv2, c22), mK1), zz[0], zz[1]);
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const int up = h0 + uu + e;
        const float z = zz[e];
        if (up == 0) zt[j] = z;
        if (up == G) zb[j] = z;
        if (DUMP && zd[j] && sb[j].x >= 0) {
          const int bx = 2 * sb[j].x + vp / G, by = 2 * sb[j].y + up / G;
          if (bx < nbx && by < nby) zd[j][((int64_t)by * nbx + bx) * G * G + (up % G) * G + v] = (int16_t)z;
        }
        if (up < G)
          Ht[j] = fmaf(fabsf(z), wts[up], Ht[j]);
        else
          Hb[j] = fmaf(fabsf(z), wts[up - G], Hb[j]);
      }
    }
  }
  // Four trees in one: at offset G/2 the lower half of the group goes on with job 0 (top and
  // bottom), the upper half with job 1; at G/4 each quarter keeps one block; then plain xor steps.
  // Every addition is one of the separate trees' (operands swapped at most).
  const bool upper = v >= G / 2;
  const float X = (upper ? Ht[1] : Ht[0]) + __shfl_xor_sync(0xffffffffu, upper ? Ht[0] : Ht[1], G / 2);
  const float Y = (upper ? Hb[1] : Hb[0]) + __shfl_xor_sync(0xffffffffu, upper ? Hb[0] : Hb[1], G / 2);
  const bool uq = (v % (G / 2)) >= G / 4;
  float R = (uq ? Y : X) + __shfl_xor_sync(0xffffffffu, uq ? X : Y, G / 4);
#pragma unroll
  for (int o = G / 8; o > 0; o >>= 1) R += __shfl_xor_sync(0xffffffffu, R, o);
  // Z(0,0) of each block sits in the group's lane 0: lane G/4 takes the bottom block's of job 0,
  // lane G/2 the top block's of job 1, lane 3G/4 the bottom block's of job 1.
  const float zb0 = __shfl_xor_sync(0xffffffffu, zb[0], G / 4);
  const float zt1 = __shfl_xor_sync(0xffffffffu, zt[1], G / 2);
  const float zb1 = __shfl_xor_sync(0xffffffffu, zb[1], 3 * G / 4);
  const int quarter = v / (G / 4);
  const float z = quarter == 0 ? zt[0] : quarter == 1 ? zb0 : quarter == 2 ? zt1 : zb1;
  if (o) {
    o[0] = R;
    o[C] = __fsqrt_rn(z);
  }
}

// Tile bookkeeping of a role's current tile.
struct TileInfo {
  int f, tx, ty, stage, t, m, p;  // frame, tile position, ring stage, CTA-local tile number, member, plane
};

// a / b for 0 <= a < 2^24, b >= 1, from a float estimate that is off by at most one.
__device__ __forceinline__ int div_small(int a, int b, float binv) {
  int qt = __float2int_rz((float)a * binv);
  const int r = a - qt * b;
  qt += (r >= b) - (r < 0);
  return qt;
}

// The members of a launch as the roles see them.  A single analyzer's launch reads its one member
// from the kernel parameters (fields become constant-bank operands); a batched launch indexes the
// member table in the kernel parameters.
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

template <bool C444, class MS>
__device__ __forceinline__ TileInfo tile_info(const MS& ms, int t, int item0, int step, int stages = kMaxStages) {
  TileInfo ti;
  const int item = item0 + t * step;
  const int m = ms.member_of(item);
  const TcMember& M = ms[m];
  const int local = item - M.item_base;
  ti.m = m;
  ti.t = t;
  ti.f = div_small(local, M.tiles_per_frame, M.inv_tiles_per_frame);
  int r = local - ti.f * M.tiles_per_frame;
  ti.p = 0;
  if constexpr (C444) {
    ti.p = div_small(r, M.tiles_per_plane, M.inv_tiles_per_plane);
    r -= ti.p * M.tiles_per_plane;
  }
  ti.ty = div_small(r, M.tiles_x, M.inv_tiles_x);
  ti.tx = r - ti.ty * M.tiles_x;
  ti.stage = t % stages;
  return ti;
}

// ---- role loops ---------------------------------------------------------------------
//
// Unit u of this CTA (tile u / UPT, half u % UPT) uses A1 slot u % 2, accumulator slot u % DS
// and stage-2 operand set u % 2.  A slot's barriers complete once per use, so a wait for unit u
// is on the parity of the number of earlier uses of that slot.

// Slot cursor: the slot of the current unit and the parity of its use count.
template <int N>
struct Cursor {
  int slot = 0;
  uint32_t par = 0;
  __device__ __forceinline__ void next() {
    if (++slot == N) {
      slot = 0;
      par ^= 1u;
    }
  }
};

// A tile as the roles see it, written once by the producer into a ring of kTileRecs entries
// (entry t % kTileRecs for the CTA's tile t) before it issues the tile's copies.  The ring is
// deep enough: the producer runs at most kStages tiles ahead of the convert warps, which run at
// most kASlots + DS units ahead of the last epilogue.
struct TileRec {
  int f, tx, ty, m;    // frame, tile position (units of 4 blocks), member
  int hy, wy, hc, wc;  // luma / chroma rows and columns from the tile's origin to the frame's edge
                       // (4:4:4: hy, wy those of the item's plane, hc the plane, wc unused)
};
constexpr int kTileRecs = 16;
static_assert(sizeof(TileRec) == 32, "two 16-byte loads");

__device__ __forceinline__ TileRec load_rec(const TileRec* ring, int t) {
  const uint32_t a = smem_u32(ring + (t & (kTileRecs - 1)));
  const uint4 x = lds128(a), y = lds128(a + 16);
  return TileRec{(int)x.x, (int)x.y, (int)x.z, (int)x.w, (int)y.x, (int)y.y, (int)y.z, (int)y.w};
}

// 32 samples (8-bit) from two 16-sample chunks -> 16 words of fp16 pairs (1024 + x).
__device__ __forceinline__ void convert_32_u8(uint32_t addr0, uint32_t addr1, uint32_t (&out)[16]) {
  const uint4 a = lds128(addr0), b = lds128(addr1);
  const uint32_t w[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    out[2 * i] = prmt(w[i], kSel6464, 0x5140);
    out[2 * i + 1] = prmt(w[i], kSel6464, 0x5342);
  }
}

// Convert, luma: the unit's block rows of the raw luma tile -> stage-1 A operands in TMEM (thread
// 32 q + lane converts row `lane` of block q of each block row).
template <bool LP, int BPS>
__device__ void convert_luma_loop(const TileRec* recs, const Ctl& ctl, uint8_t* sm, uint32_t tq, int n_items, int q,
                                  int lane) {
  using SL = SmemLay<BPS>;
  using U = Unit<LP>;
  int hy = 0, wy = 0, stage = 0;
  bool inside = false;
  // Byte offsets of this thread's two 16-sample chunks within a block row (8-bit, 128-byte swizzle).
  const uint32_t off0 = (uint32_t)(lane * 128 + (((2 * q) ^ (lane & 7)) << 4));
  const uint32_t off1 = (uint32_t)(lane * 128 + (((2 * q + 1) ^ (lane & 7)) << 4));
  Cursor<kASlots> ca;
  const int n = n_items * U::UPT;
  for (int u = 0, t = 0, h = 0; u < n; ++u, ca.next()) {
    if (h == 0) {
      stage = t % SL::kStages;
      if (!wait_bar<LP>(ctl, b_raw_full(stage), (t / SL::kStages) & 1, 4)) return;
      const TileRec r = load_rec(recs, t);
      hy = r.hy;
      wy = r.wy;
      inside = hy >= 128 && wy >= 128;
    }
    if (u >= kASlots && !wait_bar<LP>(ctl, b_a1l_free(ca.slot), ca.par ^ 1u, 4)) return;
    tc_fence_after();
    const uint32_t rbase = smem_u32(sm + OFF_RAW + stage * SL::kStageBytes);
    const uint32_t ta = tq + U::a1(ca.slot);
#pragma unroll 1
    for (int gl = 0; gl < U::UR; ++gl) {
      const int brow = h * U::UR + gl;
      uint32_t out[16];
      if (BPS == 1 && inside) {
        const uint32_t rb = rbase + (uint32_t)(brow * 4096);
        convert_32_u8(rb + off0, rb + off1, out);
      } else {
        int y = brow * 32 + lane;
        if (y >= hy) y = hy - 1;
        convert_16<32, BPS>(rbase, y, 32 * q, wy, out);
        convert_16<32, BPS>(rbase, y, 32 * q + 16, wy, out + 8);
      }
      tmem_st<16>(ta + 16 * gl, out);
    }
    tmem_wait_st();
    tc_fence_before();
    __syncwarp();
    const bool last = h == U::UPT - 1;
    if (lane == 0) {
      mbar_arrive(&ctl.bars[b_a1l_full(ca.slot)]);
      if (last) mbar_arrive(&ctl.bars[b_raw_empty(stage)]);
    }
    if (last) {
      h = 0;
      ++t;
    } else {
      ++h;
    }
  }
}

// Convert, chroma: the unit's chroma groups (8 blocks x 16 rows each) of U and V -> stage-1 A
// operands, a U row and a V row side by side (thread 32 q + lane converts row lane % 16 of
// block (32 q + lane) / 16 of the group in both planes).
template <bool LP, int BPS>
__device__ void convert_chroma_loop(const TileRec* recs, const Ctl& ctl, uint8_t* sm, uint32_t tq, int n_items, int q,
                                    int lane) {
  using SL = SmemLay<BPS>;
  using U = Unit<LP>;
  int hc = 0, wc = 0, stage = 0;
  bool inside = false;
  const int l = 32 * q + lane;
  const int bg = l >> 4, r = l & 15;
  // 8-bit, 64-byte rows and swizzle: row y of this thread's block, chunk (block column) bg & 3
  const uint32_t coff = (uint32_t)((((bg >> 2) * 16 + r) * 64) + (((bg & 3) ^ ((r >> 1) & 3)) << 4));
  Cursor<kASlots> ca;
  const int n = n_items * U::UPT;
  for (int u = 0, t = 0, h = 0; u < n; ++u, ca.next()) {
    if (h == 0) {
      stage = t % SL::kStages;
      if (!wait_bar<LP>(ctl, b_raw_full(stage), (t / SL::kStages) & 1, 4)) return;
      const TileRec rr = load_rec(recs, t);
      hc = rr.hc;
      wc = rr.wc;
      inside = hc >= 64 && wc >= 64;
    }
    if (u >= kASlots && !wait_bar<LP>(ctl, b_a1c_free(ca.slot), ca.par ^ 1u, 4)) return;
    tc_fence_after();
    const uint32_t raw = smem_u32(sm + OFF_RAW + stage * SL::kStageBytes + SL::kRawY);
    const uint32_t ta = tq + U::a1(ca.slot) + U::A1C;
#pragma unroll 1
    for (int g = 0; g < U::GC; ++g) {
      const int gt = h * U::GC + g;  // group within the chroma tile (two block rows)
      uint32_t out[16];
      if (BPS == 1 && inside) {
        const uint32_t a = raw + (uint32_t)(gt * 2048) + coff;
        convert_32_u8(a, a + SL::kRawC, out);
      } else {
        const int idx = 8 * gt + bg;
        int y = (idx >> 2) * 16 + r;
        if (y >= hc) y = hc - 1;
        const int x = (idx & 3) * 16;
        convert_16<16, BPS>(raw, y, x, wc, out);
        convert_16<16, BPS>(raw + SL::kRawC, y, x, wc, out + 8);
      }
      tmem_st<16>(ta + 16 * g, out);
    }
    tmem_wait_st();
    tc_fence_before();
    __syncwarp();
    const bool last = h == U::UPT - 1;
    if (lane == 0) {
      mbar_arrive(&ctl.bars[b_a1c_full(ca.slot)]);
      if (last) mbar_arrive(&ctl.bars[b_raw_empty(stage)]);
    }
    if (last) {
      h = 0;
      ++t;
    } else {
      ++h;
    }
  }
}

// Epilogue 1 luma: T = floor(T'/2^s1) of both luma jobs into the stage-2 operands (hi and lo bytes
// as fp16, MN-major; s1 = log2 N + B - 9).
template <bool LP, bool SUB, int BPS>
__device__ void epi1_luma_loop(const Ctl& ctl, uint32_t sbase, uint32_t tq, int n_items, int q, int lane) {
  using SL = SmemLay<BPS>;
  using U = Unit<LP>;
  using P = PC<32, LP>;
  const float s1inv = __int_as_float((127 - s1_of(Blk<SUB>::NL, BPS)) << 23);  // 2^-s1
  const E1Offs<32, LP> eo(q, lane);
  Cursor<U::DS> cd;
  Cursor<kA2Sets> ce;
  const int n = n_items * U::UPT;
  for (int u = 0; u < n; ++u, cd.next(), ce.next()) {
    if (!wait_bar<LP>(ctl, b_d1l(cd.slot), cd.par, 4)) return;
    if (u >= kA2Sets && !wait_bar<LP>(ctl, b_a2l_free(ce.slot), ce.par ^ 1u, 4)) return;
    tc_fence_after();
    const uint32_t td = tq + U::d(cd.slot);
    const uint32_t a2 = sbase + SL::OFF_A2 + (uint32_t)(ce.slot * kA2Unit);
    if constexpr (LP) {
      const uint32_t tdj[2] = {td, td + P::G * P::N1}, ahj[2] = {a2_luma(a2, 0), a2_luma(a2, 1)};
      epilogue1<32, LP, 2>(tdj, ahj, kA2L, eo, s1inv);
    } else {
#pragma unroll 1
      for (int j = 0; j < 2; ++j) {
        const uint32_t tdj[1] = {td + j * P::G * P::N1}, ahj[1] = {a2_luma(a2, j)};
        epilogue1<32, LP, 1>(tdj, ahj, kA2L, eo, s1inv);
      }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ctl.bars[b_a2l_full(ce.slot)]);
  }
}

// Output address of this thread's block values: block index k of the block that row m = 32 q + lane of
// job jp of an N-point plane covers (NK stage-2 rows per block), or -1 outside the frame.
template <int NK, int BPG2>
__device__ __forceinline__ int64_t block_of(const TcMember& M, const TileRec& r, int jp, int q, int lane) {
  const int idx = jp * BPG2 + (32 * q + lane) / NK;
  const int bx = r.tx * 4 + (idx & 3), by = r.ty * 4 + (idx >> 2);
  return (bx < M.nbx && by < M.nby) ? (int64_t)by * M.nbx + bx : -1;
}

// Super-block (x, y in super-blocks of the frame) of the stage-2 row m = 32 q + lane of job jp.
template <int NK, int BPG2>
__device__ __forceinline__ int2 superblock_of(const TileRec& r, int jp, int q, int lane) {
  const int idx = jp * BPG2 + (32 * q + lane) / NK;
  return make_int2(r.tx * 4 + (idx & 3), r.ty * 4 + (idx >> 2));
}

// Epilogue 2 luma: Z, the block energy H and brightness L of both luma jobs, then the slot's luma
// columns are handed back.
template <bool LP, bool SUB, bool DUMP, bool C444, class PP, class MS>
__device__ void epi2_luma_loop(const PP& p, const MS& ms, const TileRec* recs, const Ctl& ctl, uint32_t tq,
                               int n_items, int q, int lane) {
  using P = PC<32, LP>;
  using U = Unit<LP>;
  constexpr int NW = SUB ? P::NK / 2 : P::NK;  // weights per thread: one block column
  constexpr int NL = Blk<SUB>::NL;
  constexpr float einv = SUB ? 0.25f : 0.125f;  // 2^8 / 2^s2, s2 = log2 N + 6
  float w[NW];
#pragma unroll
  for (int uu = 0; uu < NW; ++uu) w[uu] = p.W_y[uu * NL + (lane % P::NK) % NW];
  Cursor<U::DS> cd;
  const int n = n_items * U::UPT;
  TileRec rec{};
  for (int u = 0, t = 0, h = 0; u < n; ++u, cd.next()) {
    if (!wait_bar<LP>(ctl, b_d2l(cd.slot), cd.par, 4)) return;
    tc_fence_after();
    if (h == 0) rec = load_rec(recs, t);  // written by the producer before this unit's copies
    const TcMember& M = ms[rec.m];
    const uint32_t td = tq + U::d(cd.slot);
    const int plane = C444 ? rec.hc : 0;  // the rows H, L of Y (0), U (1) or V (2)
    float* const base = M.blockvals + (int64_t)rec.f * M.out_fstride + (int64_t)(2 * plane) * M.C;
    uint32_t td2[2];
    int16_t* zd[2];
    if constexpr (SUB) {
      int2 sb[2];
      float* const orow[2] = {base, base};
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        sb[j] = superblock_of<P::NK, P::BPG2>(rec, h * 2 + j, q, lane);
        td2[j] = td + 2 * j * P::N1;
        zd[j] = (DUMP && rec.f == 0) ? p.zdump[plane] : nullptr;
      }
      float* const o = e2_store_sub<P::NK>(lane, sb, orow, M.nbx, M.nby);
      epilogue2_sub<32, LP, DUMP, P::N1>(td2, lane, w, einv, kK1 - kK1 * einv, sb, o, M.nbx, M.nby, M.C, zd);
    } else {
      float* out[2];
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int64_t k = block_of<P::NK, P::BPG2>(M, rec, h * 2 + j, q, lane);
        td2[j] = td + 2 * j * P::N1;
        out[j] = k >= 0 ? base + k : nullptr;
        zd[j] = (DUMP && k >= 0 && rec.f == 0) ? p.zdump[plane] + k * P::NK * P::NK : nullptr;
      }
      epilogue2<32, LP, DUMP, P::N1>(td2, lane, w, einv, kK1 - kK1 * einv, e2_store<P::NK>(lane, out), M.C, zd);
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(&ctl.bars[b_dfree(cd.slot)]);
    if (++h == U::UPT) {
      h = 0;
      ++t;
    }
  }
}

// Chroma epilogues, one warpgroup: for unit u, epilogue 1 (as for luma, both planes), then
// epilogue 2 of unit u - 1.
template <bool LP, bool SUB, bool DUMP, int BPS, class PP, class MS>
__device__ void chroma_epi_loop(const PP& p, const MS& ms, const TileRec* recs, const Ctl& ctl, uint32_t sbase,
                                uint32_t tq, int n_items, int q, int lane, int mode) {
  using SL = SmemLay<BPS>;
  using U = Unit<LP>;
  using P = PC<16, LP>;
  constexpr int NKC = U::NKC, NCC = U::NCC;
  constexpr int NW = SUB ? P::NK / 2 : P::NK;
  constexpr int NC = Blk<SUB>::NC;
  constexpr float einv = SUB ? 0.5f : 0.25f;  // 2^8 / 2^s2
  const float s1inv = __int_as_float((127 - s1_of(NC, BPS)) << 23);
  const E1Offs<16, LP> eo(q, lane);
  float w[NW];
#pragma unroll
  for (int uu = 0; uu < NW; ++uu) w[uu] = p.W_c[uu * NC + (lane % P::NK) % NW];
  Cursor<U::DS> cd, cd2;
  Cursor<kA2Sets> ce;
  const int n = n_items * U::UPT;
  TileRec rec{};
  for (int u = 0, t = 0, h = 0; u <= n; ++u) {
    if (u < n && (mode & 1)) {  // epilogue 1 of unit u
      if (!wait_bar<LP>(ctl, b_d1c(cd.slot), cd.par, 4)) return;
      if (u >= kA2Sets && !wait_bar<LP>(ctl, b_a2c_free(ce.slot), ce.par ^ 1u, 4)) return;
      tc_fence_after();
      const uint32_t td = tq + U::d(cd.slot) + U::DC;
      const uint32_t a2 = sbase + SL::OFF_A2 + (uint32_t)(ce.slot * kA2Unit);
      if constexpr (LP) {
        const uint32_t tdj[2] = {td, td + NKC}, ahj[2] = {a2_chroma(a2, 0), a2_chroma(a2, 1)};
        epilogue1<16, LP, 2>(tdj, ahj, kA2C, eo, s1inv);
      } else {
#pragma unroll 1
        for (int pl = 0; pl < 2; ++pl) {
          const uint32_t tdj[1] = {td + pl * NKC}, ahj[1] = {a2_chroma(a2, pl)};
          epilogue1<16, LP, 1>(tdj, ahj, kA2C, eo, s1inv);
        }
      }
      fence_proxy_async_smem();
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl.bars[b_a2c_full(ce.slot)]);
      cd.next();
      ce.next();
    }
    if (u >= 1 && (mode & 2)) {  // epilogue 2 of unit u - 1
      if (!wait_bar<LP>(ctl, b_d2c(cd2.slot), cd2.par, 4)) return;
      tc_fence_after();
      if (h == 0) rec = load_rec(recs, t);
      const TcMember& M = ms[rec.m];
      const uint32_t td = tq + U::d(cd2.slot) + U::DC;
      float* const base = M.blockvals + (int64_t)rec.f * M.out_fstride;
      uint32_t td2[2];
      int16_t* zd[2];
      if constexpr (SUB) {
        const int2 sb0 = superblock_of<P::NK, P::BPG2>(rec, h, q, lane);  // U and V share the super-block
        const int2 sb[2] = {sb0, sb0};
        float* const orow[2] = {base + 2 * M.C, base + 4 * M.C};
#pragma unroll
        for (int pl = 0; pl < 2; ++pl) {
          td2[pl] = td + pl * NKC;
          zd[pl] = (DUMP && rec.f == 0) ? p.zdump[1 + pl] : nullptr;
        }
        float* const o = e2_store_sub<P::NK>(lane, sb, orow, M.nbx, M.nby);
        epilogue2_sub<16, LP, DUMP, NCC>(td2, lane, w, einv, kK1 - kK1 * einv, sb, o, M.nbx, M.nby, M.C, zd);
      } else {
        const int64_t k = block_of<P::NK, P::BPG2>(M, rec, h, q, lane);  // U and V share the block
        float* out[2];
#pragma unroll
        for (int pl = 0; pl < 2; ++pl) {
          td2[pl] = td + pl * NKC;
          out[pl] = k >= 0 ? base + (2 + 2 * pl) * M.C + k : nullptr;
          zd[pl] = (DUMP && k >= 0 && rec.f == 0) ? p.zdump[1 + pl] + k * P::NK * P::NK : nullptr;
        }
        epilogue2<16, LP, DUMP, NCC>(td2, lane, w, einv, kK1 - kK1 * einv, e2_store<P::NK>(lane, out), M.C, zd);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl.bars[b_dfree(cd2.slot)]);
      cd2.next();
      if (++h == U::UPT) {
        h = 0;
        ++t;
      }
    }
  }
}

// MMA issue: issuer id owns stage 1 of luma job 0 (id 0) or 1 (id 1), stage 1 of chroma (id 2),
// stage 2 of luma job 0 (3) or 1 (4), of the chroma hi (5) or lo (6) operands.  Stage-1 issuers
// wait for the unit's A1 and, from the DS-th unit on, for its accumulator slot; they commit to the
// slot's D1 barrier and to the A1 slot's free barrier.  Stage-2 issuers wait for the operand set
// and commit to the slot's D2 barrier and the set's free barrier.  Barriers count one commit per
// issuer of the plane type.  Descriptors are built once; per unit only the slot offsets change.
template <bool LP, int BPS>
__device__ void issuer_loop(const Ctl& ctl, uint32_t sbase, uint32_t tmem, int id, int n_items) {
  using SL = SmemLay<BPS>;
  using U = Unit<LP>;
  using L = PC<32, LP>;
  constexpr int NCC = U::NCC;
  const uint64_t bl0 = smem_desc(sbase + SL::OFF_BL, 128, 512, 0), bl1 = smem_desc(sbase + SL::OFF_BL + 256, 128, 512, 0);
  const uint64_t dbu = smem_desc(sbase + SL::OFF_BCU, 128, 256, 0), dbv = smem_desc(sbase + SL::OFF_BCV, 128, 256, 0);
  const uint64_t du = smem_desc(sbase + SL::OFF_ONE, 128, 256, 0);
  const int n = n_items * U::UPT;
  Cursor<kASlots> ca;
  Cursor<U::DS> cd;
  Cursor<kA2Sets> ce;
  bool ok = true;
  if (id < 3) {
    const uint64_t dk = smem_desc(sbase + (id < 2 ? SL::OFF_KL : SL::OFF_KC), 128, 256, 0);
    const uint32_t aoff = id < 2 ? (uint32_t)(id * 16 * L::G) : (uint32_t)U::A1C;
    const uint32_t doff = id < 2 ? (uint32_t)(id * L::G * L::N1) : (uint32_t)U::DC;
    for (int u = 0; u < n; ++u, ca.next(), cd.next()) {
      if (!wait_bar<LP>(ctl, id < 2 ? b_a1l_full(ca.slot) : b_a1c_full(ca.slot), ca.par, 2) ||
          (u >= U::DS && !wait_bar<LP>(ctl, b_dfree(cd.slot), cd.par ^ 1u, 2))) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint32_t a = tmem + U::a1(ca.slot) + aoff, d = tmem + U::d(cd.slot) + doff;
      // D1 = U x K^T (presets of the stream's columns), then D1 += A1 (TMEM) x M^T.
      if (id < 2) {
        mma_ss(d, du, dk, idesc_f16(128, L::G * L::N1, 0, 0), 0);
        // K-step outer: consecutive MMAs write different accumulators.
#pragma unroll
        for (int ks = 0; ks < 2; ++ks)
#pragma unroll
          for (int gg = 0; gg < L::G; ++gg)
            mma_ts(d + gg * L::N1, a + gg * 16 + ks * 8, ks ? bl1 : bl0, idesc_f16(128, L::N1, 0, 0), 1);
        mma_commit(&ctl.bars[b_d1l(cd.slot)]);
        mma_commit(&ctl.bars[b_a1l_free(ca.slot)]);
      } else {
        mma_ss(d, du, dk, idesc_f16(128, U::GC * NCC, 0, 0), 0);
#pragma unroll
        for (int g = 0; g < U::GC; ++g) {
          mma_ts(d + g * NCC, a + 16 * g, dbu, idesc_f16(128, NCC, 0, 0), 1);      // U row against the U half
          mma_ts(d + g * NCC, a + 16 * g + 8, dbv, idesc_f16(128, NCC, 0, 0), 1);  // V row against the V half
        }
        mma_commit(&ctl.bars[b_d1c(cd.slot)]);
        mma_commit(&ctl.bars[b_a1c_free(ca.slot)]);
      }
    }
  } else {
    // D2 = presets, then D2 += A2 (smem, MN-major) x M^T; descriptors of operand set 0, set 1 is
    // kA2Unit bytes further.
    const bool luma = id < 5;
    const int j = id - 3;
    const uint32_t lo = id == 6 ? 1u : 0u;
    const uint32_t a2 = sbase + SL::OFF_A2;
    uint64_t ad[4];
    if (luma) {
      const uint32_t ahi = a2_luma(a2, j);
      ad[0] = smem_desc(ahi, 1024, 2048, 2);
      ad[1] = smem_desc(ahi + kA2L, 1024, 2048, 2);
      ad[2] = smem_desc(ahi + 4096, 1024, 2048, 2);
      ad[3] = smem_desc(ahi + kA2L + 4096, 1024, 2048, 2);
    } else {
      ad[0] = smem_desc(a2_chroma(a2, 0) + lo * kA2C, 1024, 2048, 2);
      ad[1] = smem_desc(a2_chroma(a2, 1) + lo * kA2C, 1024, 2048, 2);
      ad[2] = ad[3] = 0;
    }
    const uint32_t doff = luma ? (uint32_t)(2 * j * L::N1) : (uint32_t)(U::DC + lo * NCC);
    // stage-2 presets (D2 = U x K2^T, overwriting): the stream's hi and lo columns (luma) or its
    // hi or lo columns (chroma)
    const uint64_t dk2 = smem_desc(sbase + (luma ? SL::OFF_K2L : lo ? SL::OFF_K2CL : SL::OFF_K2CH), 128, 256, 0);
    const uint32_t idP2 = luma ? idesc_f16(128, 2 * L::N1, 0, 0) : idesc_f16(128, NCC, 0, 0);
    for (int u = 0; u < n; ++u, cd.next(), ce.next()) {
      if (!wait_bar<LP>(ctl, luma ? b_a2l_full(ce.slot) : b_a2c_full(ce.slot), ce.par, 2)) {
        ok = false;
        break;
      }
      tc_fence_after();
      const uint64_t so = (uint64_t)(ce.slot * (kA2Unit >> 4));  // descriptor address field of the set
      const uint32_t d = tmem + U::d(cd.slot) + doff;
      mma_ss(d, du, dk2, idP2, 0);
      if (luma) {
        mma_ss(d, ad[0] + so, bl0, idesc_f16(128, L::N1, 1, 0), 1);
        mma_ss(d + L::N1, ad[1] + so, bl0, idesc_f16(128, L::N1, 1, 0), 1);
        mma_ss(d, ad[2] + so, bl1, idesc_f16(128, L::N1, 1, 0), 1);
        mma_ss(d + L::N1, ad[3] + so, bl1, idesc_f16(128, L::N1, 1, 0), 1);
        mma_commit(&ctl.bars[b_d2l(cd.slot)]);
        mma_commit(&ctl.bars[b_a2l_free(ce.slot)]);
      } else {
        mma_ss(d, ad[0] + so, dbu, idesc_f16(128, NCC, 1, 0), 1);
        mma_ss(d, ad[1] + so, dbv, idesc_f16(128, NCC, 1, 0), 1);
        mma_commit(&ctl.bars[b_d2c(cd.slot)]);
        mma_commit(&ctl.bars[b_a2c_free(ce.slot)]);
      }
    }
  }
  if (!ok) {  // let this thread's MMAs finish before the CTA frees TMEM
    mma_commit(&ctl.bars[b_drain(id)]);
    wait_bar<LP>(ctl, b_drain(id), 0, 2, true);
  }
}

// ---- frame reduction of a batched tick, in each CTA's tail (see TcRedMember) ----------------
//
// After its role loops a CTA reduces the block values of its own tiles, still in L2.  Its run of
// tiles covers one or more members ("segments"); all segments go through each step together, so
// the tail costs a few memory round trips however many members the run touches:
//   1. every thread takes one block at a time (kThreads blocks per pass): fixed23 of the six rows
//      (4:4:4: of its plane's two) and, for luma rows, |H - H_prev|, writing H as the next tick's
//      previous energy; a warp whose blocks are of one segment stores its warp sums in a slot of
//      its own, then warp r adds sum r of every slot into the segments' totals in shared memory
//      (warps whose blocks straddle two segments add per thread, atomically); the totals are kept
//      as low-32-bit and high parts, exact;
//   2. the totals of every segment go to the members' accumulators in global memory;
//   3. one count per segment (its tiles); the CTA whose count completes a member
//   4. writes the features -- the same exact totals, rounded once, as the separate frame
//      reduction -- and leaves the accumulators and the count at zero.
// The epilogues carry none of this: on the tensor-core pipeline's critical path every added
// instruction or load costs far more than here (sums kept per unit in the epilogue-2 warps made
// the batched launches a third slower).

// Exact sum over the warp of per-thread values below 2^59 (the total is below 2^64): three 21-bit
// limbs, each summed by one warp reduction (limb totals below 2^26).
__device__ __forceinline__ unsigned long long warp_sum64(unsigned long long v) {
  const unsigned a = __reduce_add_sync(0xffffffffu, (unsigned)(v & 0x1FFFFFull));
  const unsigned b = __reduce_add_sync(0xffffffffu, (unsigned)((v >> 21) & 0x1FFFFFull));
  const unsigned c = __reduce_add_sync(0xffffffffu, (unsigned)(v >> 42));
  return (unsigned long long)a + ((unsigned long long)b << 21) + ((unsigned long long)c << 42);
}

// Adds v to a total kept as (sum of low 32-bit parts, sum of the rest) at t[0], t[1].
__device__ __forceinline__ void add_split(unsigned long long* t, unsigned long long v) {
  atomicAdd(t, v & 0xFFFFFFFFull);
  atomicAdd(t + 1, v >> 32);
}

// scratch: shared memory (the raw ring, no longer in use) for kMaxMembers segments x kRedSums
// split totals, a flag per segment and the warps' slots.  Blocks are taken kThreads at a time,
// one per thread.
// tab: the reduction entries of the CTA's members (tab[m - m0] for member m, m0 the CTA's first),
// copied into shared memory when the launch started.
template <bool SUB, bool C444, class PP>
__device__ __noinline__ void red_tail(const PP& p, int item0, int n_items, unsigned long long* scratch,
                                      const TcRedMember* tab) {
  constexpr int BPT = SUB ? 8 : 4;  // blocks per tile side
  constexpr int BPT2 = BPT * BPT;
  const int tid = threadIdx.x, lane = tid & 31;
  constexpr int kWarps = kThreads / 32;
  int* flags = reinterpret_cast<int*>(scratch + kMaxMembers * kRedSums * 2);
  unsigned long long* wslot = scratch + kMaxMembers * kRedSums * 2 + kMaxMembers / 2;  // [kWarps][kRedSums]
  int* wseg = reinterpret_cast<int*>(wslot + kWarps * kRedSums);                     // segment of each slot
  const int warp = tid >> 5;
  if (n_items <= 0) return;
  MemberTable ms{p.mem, p.n_members, 0};
  const int m0 = ms.member_of(item0);
  const int nseg = ms.member_of(item0 + n_items - 1) - m0 + 1;
  for (int i = tid; i < nseg * kRedSums * 2; i += kThreads) scratch[i] = 0ull;
  __syncthreads();
  // 1. blocks -> per-segment totals in shared memory
  MemberTable mt{p.mem, p.n_members, m0};
  const int nblocks = n_items * BPT2;
  for (int base = 0; base < nblocks; base += kThreads) {
    const int i = base + tid;
    unsigned long long v[kRedSums];
#pragma unroll
    for (int r = 0; r < kRedSums; ++r) v[r] = 0ull;
    int seg = -1;
    if (i < nblocks) {
      const int item = item0 + i / BPT2, b = i % BPT2;
      const int m = mt.member_of(item);
      const TcMember& M = mt[m];
      seg = m - m0;
      int r = item - M.item_base, pl = 0;
      if constexpr (C444) {
        pl = div_small(r, M.tiles_per_plane, M.inv_tiles_per_plane);
        r -= pl * M.tiles_per_plane;
      }
      const int ty = div_small(r, M.tiles_x, M.inv_tiles_x), tx = r - ty * M.tiles_x;
      const int bx = tx * BPT + b % BPT, by = ty * BPT + b / BPT;
      if (bx < M.nbx && by < M.nby) {
        const int64_t k = (int64_t)by * M.nbx + bx;
        const float* bv = M.blockvals + k;
#pragma unroll
        for (int row = 0; row < N_ROWS; ++row)
          if (!C444 || row / 2 == pl) v[row] = fixed23(bv[row * M.C]);
        if (!C444 || pl == 0) {
          const TcRedMember& R = tab[seg];
          const int pb = (M.red_flags & kRedPrevBuf) ? 1 : 0;
          const float hy = bv[0];
          const unsigned long long fh = fixed23(hy);
          const unsigned long long fp = (M.red_flags & kRedHasPrev) ? fixed23(R.prevH[pb][k]) : fh;
          v[kRedSums - 1] = fh > fp ? fh - fp : fp - fh;
          R.prevH[pb ^ 1][k] = hy;
        }
      }
    }
    const int seg0 = __shfl_sync(0xffffffffu, seg, 0);
    if (__all_sync(0xffffffffu, seg == seg0 || seg < 0)) {
#pragma unroll
      for (int r = 0; r < kRedSums; ++r) {
        const unsigned long long w = warp_sum64(v[r]);
        if (lane == 0) wslot[warp * kRedSums + r] = w;
      }
      if (lane == 0) wseg[warp] = seg0;  // -1: no blocks
    } else {
      if (seg >= 0) {
#pragma unroll
        for (int r = 0; r < kRedSums; ++r) add_split(scratch + (seg * kRedSums + r) * 2, v[r]);
      }
      if (lane == 0) wseg[warp] = -1;
    }
    __syncthreads();
    // Warp r folds sum r of the slots (each below 2^58) into the segments' totals; the segments of
    // a pass are consecutive, in the order of the warps.
    if (warp < kRedSums) {
      const int sl = wseg[lane];
      const unsigned long long x = sl >= 0 ? wslot[lane * kRedSums + warp] : 0ull;
      const int first = __reduce_min_sync(0xffffffffu, sl >= 0 ? sl : INT_MAX);
      const int last = __reduce_max_sync(0xffffffffu, sl);
      for (int sg = first; sg <= last; ++sg) {
        const unsigned long long t = warp_sum64(sl == sg ? x : 0ull);
        if (lane == 0) {
          scratch[(sg * kRedSums + warp) * 2] += t & 0xFFFFFFFFull;
          scratch[(sg * kRedSums + warp) * 2 + 1] += t >> 32;
        }
      }
    }
    __syncthreads();  // the slots are reused by the next pass
  }
  // 2. each segment's totals to its member's accumulators
  for (int i = tid; i < nseg * kRedSums; i += kThreads) {
    const int sg = i / kRedSums, r = i % kRedSums;
    const TcMember& M = ms[m0 + sg];
    unsigned long long* acc = tab[sg].acc[(M.red_flags & kRedGraph) ? 1 : 0] + 2 * r;
    // the segment's total lo + hi * 2^32, as a low-32-bit part and the rest
    U128 t{scratch[i * 2], 0ull};
    const unsigned long long hi = scratch[i * 2 + 1];
    add_to(t, U128{hi << 32, hi >> 32});
    atomicAdd(acc, t.lo & 0xFFFFFFFFull);
    atomicAdd(acc + 1, (t.lo >> 32) | (t.hi << 32));
    __threadfence();  // the totals before the count
  }
  __syncthreads();
  // 3. one count per segment: this CTA's tiles of the member
  for (int sg = tid; sg < nseg; sg += kThreads) {
    const TcMember& M = ms[m0 + sg];
    const int lo = max(item0, M.item_base), hi = min(item0 + n_items, M.item_base + M.tiles_per_frame);
    const unsigned n = (unsigned)(hi - lo);
    flags[sg] = atomicAdd(tab[sg].done[(M.red_flags & kRedGraph) ? 1 : 0], n) + n == (unsigned)M.tiles_per_frame;
  }
  __syncthreads();
  // 4. the members this CTA completed: features, and the state left at zero
  for (int i = tid; i < nseg * kRedSums; i += kThreads) {
    const int sg = i / kRedSums, r = i % kRedSums;
    if (!flags[sg]) continue;
    __threadfence();  // every other CTA fenced its totals before its count
    const TcMember& M = ms[m0 + sg];
    const TcRedMember& R = tab[sg];
    const int g = (M.red_flags & kRedGraph) ? 1 : 0;
    volatile unsigned long long* acc = R.acc[g];
    const unsigned long long lo = acc[2 * r], hi = acc[2 * r + 1];
    U128 t{lo, 0ull};
    add_to(t, U128{hi << 32, hi >> 32});
    int slot;
    const double f = feature_of_sum(r, t, (double)M.C, R.normY, R.normC, slot);
    R.feats[g][slot] = f;
    acc[2 * r] = 0ull;
    acc[2 * r + 1] = 0ull;
    if (r == 0) {
      R.feats[g][7] = 0.0;
      *R.done[g] = 0u;
    }
  }
}

template <bool LP, bool SUB, bool DUMP, int BPS, bool BATCH, bool C444>
__global__ void __launch_bounds__(kThreads, 1)
    tc_kernel(const __grid_constant__ TcParamsT<BATCH ? kMaxMembers : 1> p) {
  using L = PC<32, LP>;
  using U = Unit<LP>;
  constexpr int NL = Blk<SUB>::NL, NC = Blk<SUB>::NC;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  using SL = SmemLay<BPS>;
  uint64_t* bars = (uint64_t*)(sm + SL::OFF_BAR);
  uint32_t* tmem_slot = (uint32_t*)(sm + SL::OFF_MISC);
  TileRec* recs = (TileRec*)(sm + SL::OFF_REC);
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
  Ctl ctl{bars, abort_flag, p.err, BATCH ? p.err_host : nullptr, p.wait_ns > 0 ? (uint64_t)p.wait_ns : kWaitNs};

  using MS = typename MemberView<BATCH>::T;
  MS ms = [&] {
    if constexpr (BATCH)
      return MemberTable{p.mem, p.n_members, 0};
    else
      return OneMember{p.mem[0]};
  }();

  // Constant B operands (the integer DCT matrices as fp16), K-major without swizzle:
  // element (n, k) at (n/8)*SBO + (k/8)*128 + (n%8)*16 + (k%8)*2.  Luma: M (N1 rows, K = 32).
  // Chroma: M's first NKC rows in rows [0, NKC) of the U operand and rows [NKC, 2 NKC) of the V
  // operand, zero elsewhere (K = 16).  SUB: the smaller matrix's first N1/2 (luma) or NKC/2
  // (chroma) rows twice along the diagonal -- operand row n = (half, row), column k = (half, col).
  for (int i = tid; i < L::N1 * 32; i += kThreads) {
    const int n = i >> 5, kk = i & 31;
    float v;
    if (SUB) {
      const int hn = L::N1 / 2;
      v = (n / hn == kk / 16) ? (float)p.M_y[(n % hn) * 16 + (kk % 16)] : 0.0f;
    } else {
      v = (float)p.M_y[n * 32 + kk];
    }
    *(__half*)(sm + SL::OFF_BL + (n >> 3) * 512 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) = __float2half_rn(v);
  }
  for (int i = tid; i < 2 * 32 * 16; i += kThreads) {
    const int pl = i >> 9, n = (i >> 4) & 31, kk = i & 15;
    const int row = n - pl * U::NKC;  // matrix row held at operand row n
    float v = 0.0f;
    if (row >= 0 && row < U::NKC) {
      if (SUB) {
        const int hn = U::NKC / 2;
        v = (row / hn == kk / 8) ? (float)p.M_c[(row % hn) * 8 + (kk % 8)] : 0.0f;
      } else {
        v = (float)p.M_c[row * 16 + kk];
      }
    }
    *(__half*)(sm + (pl ? SL::OFF_BCV : SL::OFF_BCU) + (n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) =
        __float2half_rn(v);
  }
  // Stage-1 presets, applied by one more MMA per stream ahead of the data: D1 = U x K^T with N =
  // the stream's D1 columns side by side.  Every row of U is (1024, 1, 0, ...), so column n of D1
  // starts at 1024 a_n + b_n for row n of K = (a_n, b_n, 0, ...): 2^(s1-1), the rounding offset
  // of T, minus 1024 * 64 * N in each DC column (the bias of the 1024 + x sample encoding), split
  // as a = -(multiple of 8 below 2^11) and b = P - 1024 a (|b| < 2^13, a multiple of 8), both exact
  // in fp16.  Luma DC columns: every N1-th; chroma: every NKC-th (U and V alternate); SUB: every
  // N1/2-th and NKC/2-th (the left and right blocks of a super-block).
  for (int i = tid; i < 128 * 16; i += kThreads) {
    const int m = i >> 4, kk = i & 15;
    const float v = kk == 0 ? 1024.0f : kk == 1 ? 1.0f : 0.0f;
    *(__half*)(sm + SL::OFF_ONE + (m >> 3) * 256 + (kk >> 3) * 128 + (m & 7) * 16 + (kk & 7) * 2) = __float2half_rn(v);
  }
  for (int i = tid; i < 2 * 32 * 16; i += kThreads) {
    const bool luma = i < 32 * 16;
    const int kk = i & 15, n = (i >> 4) & 31;
    const int N = luma ? NL : NC, period = (luma ? L::N1 : U::NKC) / (SUB ? 2 : 1);
    const int P = (1 << (s1_of(N, BPS) - 1)) - (n % period == 0 ? 1024 * 64 * N : 0);
    const int a = P >= 0 ? (P >> 10) & ~7 : -(((-P) >> 10) & ~7);
    const float v = kk == 0 ? (float)a : kk == 1 ? (float)(P - a * 1024) : 0.0f;
    *(__half*)(sm + (luma ? SL::OFF_KL : SL::OFF_KC) + (n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) =
        __float2half_rn(v);
  }
  // Stage-2 presets, by one more MMA per stage-2 stream: hi accumulators start at K1, minus
  // 1156 * 64 * N on each u = 0 column (the 1024 + byte encoding of both halves and the +128
  // offset of the hi byte), lo accumulators at 2^(s2-1) (s2 = log2 N + 6: 11 for N = 32, 10 for
  // 16, 9 for 8), the magic constants of epilogue 2; split as for the stage-1 presets.  Luma: N1
  // hi rows then N1 lo rows; chroma: NCC rows each for hi (u = 0 every NKC-th; SUB: every
  // N1/2-th and NKC/2-th, the top and bottom blocks) and lo.
  for (int i = tid; i < (64 + 32 + 32) * 16; i += kThreads) {
    const int kk = i & 15, row = i >> 4;
    int P, off, n;
    if (row < 64) {
      n = row;
      off = SL::OFF_K2L;
      P = n < L::N1 ? (n % (SUB ? L::N1 / 2 : L::N1) == 0 ? 12582912 - 1156 * 64 * NL : 12582912) : NL * 32;
    } else if (row < 96) {
      n = row - 64;
      off = SL::OFF_K2CH;
      P = n % (SUB ? U::NKC / 2 : U::NKC) == 0 ? 12582912 - 1156 * 64 * NC : 12582912;
    } else {
      n = row - 96;
      off = SL::OFF_K2CL;
      P = NC * 32;
    }
    const int a = (P >> 10) & ~7;
    const float v = kk == 0 ? (float)a : kk == 1 ? (float)(P - a * 1024) : 0.0f;
    *(__half*)(sm + off + (n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) = __float2half_rn(v);
  }
  if constexpr (BATCH) {
    // The reduction entries of this CTA's members, for the launch's tail: read there from shared
    // memory, each phase of the tail saves a dependent global load.
    if (n_items > 0) {
      MemberTable mt{p.mem, p.n_members, 0};
      const int m0 = mt.member_of(item0);
      const int nm = mt.member_of(item0 + n_items - 1) - m0 + 1;
      constexpr int W = (int)(sizeof(TcRedMember) / 8);
      const unsigned long long* src = reinterpret_cast<const unsigned long long*>(p.red);
      unsigned long long* dst = reinterpret_cast<unsigned long long*>(sm + SL::OFF_REDTAB);
      for (int i = tid; i < nm * W; i += kThreads) dst[i] = src[(int64_t)mt[m0 + i / W].red * W + i % W];
    }
  }
  if (tid == 0) {
    for (int i = 0; i < kBars; ++i) mbar_init(&bars[i], 1);
    for (int i = 0; i < SL::kStages; ++i)
      mbar_init(&bars[b_raw_empty(i)], C444 ? 4 : 8);  // the convert warpgroups (4:4:4: luma only)
    for (int a = 0; a < kASlots; ++a) {
      mbar_init(&bars[b_a1l_full(a)], 4);  // convert luma warps
      mbar_init(&bars[b_a1c_full(a)], 4);  // convert chroma warps
      mbar_init(&bars[b_a1l_free(a)], 2);  // issuers 0, 1
    }
    for (int d = 0; d < U::DS; ++d) {
      mbar_init(&bars[b_d1l(d)], 2);   // issuers 0, 1
      mbar_init(&bars[b_d2l(d)], 2);   // issuers 3, 4
      mbar_init(&bars[b_d2c(d)], 2);   // issuers 5, 6
      mbar_init(&bars[b_dfree(d)], C444 ? 4 : 8);  // epilogue-2 luma and chroma warps (4:4:4: luma)
    }
    for (int e = 0; e < kA2Sets; ++e) {
      mbar_init(&bars[b_a2l_full(e)], 4);  // epilogue-1 luma warps
      mbar_init(&bars[b_a2c_full(e)], 4);  // chroma epilogue warps
      mbar_init(&bars[b_a2l_free(e)], 2);  // issuers 3, 4
      mbar_init(&bars[b_a2c_free(e)], 2);  // issuers 5, 6
    }
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

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer: tiles in order into the ring ----------------
      int issued = 0;
      const uint64_t pol = l2_evict_first_policy();
      for (int t = 0; t < n_items; ++t) {
        const int stage = t % SL::kStages;
        if (t >= SL::kStages && !wait_bar<LP>(ctl, b_raw_empty(stage), ((t / SL::kStages) - 1) & 1, 1, false, true))
          break;
        const TileInfo ti = tile_info<C444>(ms, t, item0, step, SL::kStages);
        {
          const TcMember& M = ms[ti.m];
          TileRec* rec = recs + (t & (kTileRecs - 1));
          if (C444)
            *rec = TileRec{ti.f, ti.tx, ti.ty, ti.m, M.H - ti.ty * 128, M.W - ti.tx * 128, ti.p, 0};
          else
            *rec = TileRec{ti.f, ti.tx, ti.ty, ti.m, M.H - ti.ty * 128, M.W - ti.tx * 128, M.ch - ti.ty * 64,
                           M.cw - ti.tx * 64};
        }
        const CUtensorMap* mm = &p.maps[3 * ti.m + ti.p];
        uint8_t* dst = sm + OFF_RAW + stage * SL::kStageBytes;
        uint64_t* full = &bars[b_raw_full(stage)];
        if (item0 + t * step == p.withhold) {  // failure-path test: the stage never fills
          ++issued;
          continue;
        }
        mbar_arrive_expect_tx(full, C444 ? SL::kRawY : SL::kStageBytes);
        // The frames are read once: loaded to be evicted from L2 first, so that what is read again
        // stays there -- in a batched tick the block values and previous energies that the
        // launch's reduction tail reads back (2 % more ticks per second on the 24-channel ladder;
        // single analyzers' low-pass launches measured 0.8 % faster).
        auto load = [&](void* d, const CUtensorMap* map, int x, int y) {
          tma_load_3d_hint(d, map, x, y, ti.f, full, pol);
        };
        if (BPS == 1) {
          load(dst, mm, ti.tx * 128, ti.ty * 128);
        } else {  // 16-bit luma: the tile is two 64-sample boxes side by side
          load(dst, mm, ti.tx * 128, ti.ty * 128);
          load(dst + 128 * 64 * 2, mm, ti.tx * 128 + 64, ti.ty * 128);
        }
        if (!C444) {
          load(dst + SL::kRawY, mm + 1, ti.tx * 64, ti.ty * 64);
          load(dst + SL::kRawY + SL::kRawC, mm + 2, ti.tx * 64, ti.ty * 64);
        }
        ++issued;
      }
      // Every copy this CTA issued lands before its shared memory goes away: in a normal run the
      // convert warps waited for each tile, but a role that gave up on a wait no longer does.
      for (int t = (issued > SL::kStages ? issued - SL::kStages : 0); t < issued; ++t)
        if (item0 + t * step != p.withhold)
          wait_bar<LP>(ctl, b_raw_full(t % SL::kStages), (t / SL::kStages) & 1, 1, true);
    }
  } else if (warp <= kIssuers) {
    // 4:4:4: the chroma issuers (stage 1 chroma: 2; stage 2 chroma hi, lo: 5, 6) have no work
    const int id = warp - 1;
    const bool chroma_issuer = id == 2 || id >= 5;
    if (lane == 0 && !(C444 && chroma_issuer)) issuer_loop<LP, BPS>(ctl, sbase, tmem, id, n_items);
  } else if (role == 2) {
    convert_luma_loop<LP, BPS>(recs, ctl, sm, tmem + lanebase, n_items, q, lane);
  } else if (role == 3) {
    if (!C444) convert_chroma_loop<LP, BPS>(recs, ctl, sm, tmem + lanebase, n_items, q, lane);
  } else if (role == 4) {
    epi1_luma_loop<LP, SUB, BPS>(ctl, sbase, tmem + lanebase, n_items, q, lane);
  } else if (role == 5) {
    epi2_luma_loop<LP, SUB, DUMP, C444>(p, ms, recs, ctl, tmem + lanebase, n_items, q, lane);
  } else if (role == 6) {
    if (!C444) chroma_epi_loop<LP, SUB, DUMP, BPS>(p, ms, recs, ctl, sbase, tmem + lanebase, n_items, q, lane, 1);
  } else {
    if (!C444) chroma_epi_loop<LP, SUB, DUMP, BPS>(p, ms, recs, ctl, sbase, tmem + lanebase, n_items, q, lane, 2);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, kTmemCols);
  }
  // Batched ticks: this CTA's share of its members' frame reductions (not after a wait ran out:
  // the tick is lost, and the host clears its graph's reduction state).
  if constexpr (BATCH) {
    if (!*abort_flag)
      red_tail<SUB, C444>(p, item0, n_items, reinterpret_cast<unsigned long long*>(sm + OFF_RAW),
                          reinterpret_cast<const TcRedMember*>(sm + SL::OFF_REDTAB));
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
template <bool LP, bool SUB, bool DUMP, int BPS, bool BATCH, bool C444>
cudaError_t prepare_inst() {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(tc_kernel<LP, SUB, DUMP, BPS, BATCH, C444>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                SmemLay<BPS>::kSmemBytes);
  });
  return attr;
}

template <bool BATCH>
using ParamsOf = TcParamsT<BATCH ? kMaxMembers : 1>;

// grid 0: only prepare the instance.
template <bool LP, bool SUB, bool DUMP, int BPS, bool BATCH, bool C444>
cudaError_t launch_inst(const ParamsOf<BATCH>& p, int grid, cudaStream_t s) {
  const cudaError_t attr = prepare_inst<LP, SUB, DUMP, BPS, BATCH, C444>();
  if (attr != cudaSuccess) return attr;
  if (grid <= 0) return cudaSuccess;
  tc_kernel<LP, SUB, DUMP, BPS, BATCH, C444><<<grid, kThreads, SmemLay<BPS>::kSmemBytes, s>>>(p);
  return cudaGetLastError();
}

template <bool SUB, bool DUMP, bool BATCH, bool C444>
cudaError_t launch_lb(const ParamsOf<BATCH>& p, int grid, bool low_pass, int bps, cudaStream_t s) {
  if (bps == 1)
    return low_pass ? launch_inst<true, SUB, DUMP, 1, BATCH, C444>(p, grid, s)
                    : launch_inst<false, SUB, DUMP, 1, BATCH, C444>(p, grid, s);
  return low_pass ? launch_inst<true, SUB, DUMP, 2, BATCH, C444>(p, grid, s)
                  : launch_inst<false, SUB, DUMP, 2, BATCH, C444>(p, grid, s);
}

// A launch of the instance for block size w (32, or 16 for the super-block form), 4:4:4 or not,
// low-pass or not, bps 1 or 2.
template <bool DUMP, bool BATCH>
cudaError_t launch_any(const ParamsOf<BATCH>& p, int grid, int w, bool c444, bool low_pass, int bps, cudaStream_t s) {
  if (w == 16)
    return c444 ? launch_lb<true, DUMP, BATCH, true>(p, grid, low_pass, bps, s)
                : launch_lb<true, DUMP, BATCH, false>(p, grid, low_pass, bps, s);
  return c444 ? launch_lb<false, DUMP, BATCH, true>(p, grid, low_pass, bps, s)
              : launch_lb<false, DUMP, BATCH, false>(p, grid, low_pass, bps, s);
}

// A single analyzer's launch.
cudaError_t launch_single(const TcParams& p, int grid, int w, bool c444, bool low_pass, bool dump, int bps,
                          cudaStream_t s) {
  return dump ? launch_any<true, false>(p, grid, w, c444, low_pass, bps, s)
              : launch_any<false, false>(p, grid, w, c444, low_pass, bps, s);
}

// A batched launch of members of one sample size.
cudaError_t launch_batched(const TcBatchParams& p, int grid, int w, bool c444, bool low_pass, int bps, cudaStream_t s) {
  return launch_any<false, true>(p, grid, w, c444, low_pass, bps, s);
}

// The batched kernel instance.
template <bool SUB, bool C444>
const void* batch_kernel_of(int bps, bool low_pass) {
  if (bps == 1)
    return low_pass ? (const void*)tc_kernel<true, SUB, false, 1, true, C444>
                    : (const void*)tc_kernel<false, SUB, false, 1, true, C444>;
  return low_pass ? (const void*)tc_kernel<true, SUB, false, 2, true, C444>
                  : (const void*)tc_kernel<false, SUB, false, 2, true, C444>;
}

// Tensor maps of one frame's planes: the luma plane as 128x128 boxes (8-bit samples, 128-byte
// swizzle) or as pairs of 64x128 boxes (16-bit words), and the chroma planes the same way in
// 4:4:4, else as 64x64 boxes (64-byte swizzle for bytes, 128-byte for words).
cudaError_t make_frame_maps(CUtensorMap* m, const Geometry& g, const FramePlanes& fp, int nframes) {
  const bool c444 = g.nc == g.w;
  const int bps = g.bps;
  const int by = bps == 1 ? 128 : 64;
  cudaError_t e = make_map(&m[0], fp.y, g.W, g.H, fp.pitch_y, fp.fstride_y, nframes, by, 128, bps,
                           CU_TENSOR_MAP_SWIZZLE_128B);
  for (int pl = 1; pl < 3 && e == cudaSuccess; ++pl) {
    const uint8_t* base = pl == 1 ? fp.u : fp.v;
    if (c444)
      e = make_map(&m[pl], base, g.cw, g.ch, fp.pitch_uv, fp.fstride_uv, nframes, by, 128, bps,
                   CU_TENSOR_MAP_SWIZZLE_128B);
    else
      e = make_map(&m[pl], base, g.cw, g.ch, fp.pitch_uv, fp.fstride_uv, nframes, 64, 64, bps,
                   bps == 1 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
  }
  return e;
}

// One member's entry: geometry, outputs and stage-1 constants; returns its number of items.  A
// tile is 128 x 128 luma samples: 4 x 4 blocks of 32 x 32, or 8 x 8 of 16 x 16; a 4:4:4 frame has
// three planes of tiles.
int fill_member(TcMember& m, const Geometry& g, int item_base, int nframes, float* blockvals) {
  m = TcMember{};
  m.item_base = item_base;
  const int bpt = 128 / g.w;
  m.tiles_x = (g.nbx + bpt - 1) / bpt;
  m.tiles_per_plane = m.tiles_x * ((g.nby + bpt - 1) / bpt);
  m.inv_tiles_per_plane = 1.0f / (float)m.tiles_per_plane;
  m.tiles_per_frame = m.tiles_per_plane * (g.nc == g.w ? 3 : 1);
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
  // 4:2:0 (chroma blocks w/2) and 4:4:4 (chroma blocks w, through the luma roles)
  const bool sizes = (g.w == 32 || g.w == 16) && (g.nc == g.w / 2 || g.nc == g.w);
  return (g.B == 8 || g.B == 10) && sizes && g.ncv == g.nc && g.s1y == s1_of(g.w, g.bps) &&
         g.s1c == s1_of(g.nc, g.bps) && encode_fn() != nullptr;
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

cudaError_t tc_batch_fill(void* params, const TcBatchFrame* frames, int n, const DeviceTables& t, int* err,
                          const TcRedMember* red, double* err_host, long long wait_ns, int withhold) {
  if (n < 0 || n > kMaxMembers) return cudaErrorInvalidValue;
  TcBatchParams& p = *static_cast<TcBatchParams*>(params);
  p.zdump[0] = p.zdump[1] = p.zdump[2] = nullptr;
  p.M_y = t.M_y;
  p.M_c = t.M_c;
  p.W_y = t.W_y;
  p.W_c = t.W_c;
  p.err = err;
  p.red = red;
  p.err_host = err_host;
  p.wait_ns = wait_ns;
  p.withhold = withhold;
  int items = 0;
  for (int i = 0; i < n; ++i) {
    const Geometry& g = *frames[i].g;
    const FramePlanes& fp = frames[i].fp;
    if (!tc_supported(g) || g.bps != frames[0].g->bps || g.w != frames[0].g->w || g.nc != frames[0].g->nc)
      return cudaErrorInvalidValue;
    items += fill_member(p.mem[i], g, items, 1, frames[i].blockvals);
    p.mem[i].red = frames[i].red;
    p.mem[i].red_flags = frames[i].red_flags;
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
    FramePlanes one = fp;
    one.fstride_y = one.fstride_uv = 0;
    cudaError_t e = make_frame_maps(&p.maps[3 * i], g, one, 1);
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

cudaError_t tc_batch_prepare(int w, bool c444, int bps, bool low_pass) {
  if ((bps != 1 && bps != 2) || (w != 32 && w != 16)) return cudaErrorInvalidValue;
  static TcBatchParams unused{};
  return launch_batched(unused, 0, w, c444, low_pass, bps, nullptr);
}

const void* tc_batch_kernel(int w, bool c444, int bps, bool low_pass) {
  if (w == 16)
    return c444 ? batch_kernel_of<true, true>(bps, low_pass) : batch_kernel_of<true, false>(bps, low_pass);
  return c444 ? batch_kernel_of<false, true>(bps, low_pass) : batch_kernel_of<false, false>(bps, low_pass);
}

cudaError_t tc_batch_node_params(int w, bool c444, int bps, bool low_pass, int grid, void** args,
                                 cudaKernelNodeParams* kp) {
  const cudaError_t e = tc_batch_prepare(w, c444, bps, low_pass);
  if (e != cudaSuccess) return e;
  *kp = cudaKernelNodeParams{};
  kp->func = const_cast<void*>(tc_batch_kernel(w, c444, bps, low_pass));
  kp->gridDim = dim3((unsigned)(grid > 0 ? grid : 1));
  kp->blockDim = dim3(kThreads);
  kp->sharedMemBytes = bps == 1 ? SmemLay<1>::kSmemBytes : SmemLay<2>::kSmemBytes;
  kp->kernelParams = args;
  kp->extra = nullptr;
  return cudaSuccess;
}

cudaError_t launch_tc(const Geometry& g, const FramePlanes& fp, int nframes, const DeviceTables& t, float* blockvals,
                      int16_t* const zdump[3], int* err, cudaStream_t s, int64_t* launches, int ctas,
                      long long wait_ns, int withhold) {
  if (!tc_supported(g)) return cudaErrorNotSupported;
  if (nframes <= 0) return cudaSuccess;
  const int bps = g.bps;
  TcParams p{};
  cudaError_t e = make_frame_maps(p.maps, g, fp, nframes);
  if (e != cudaSuccess) return e;
  p.n_members = 1;
  p.total_items = fill_member(p.mem[0], g, 0, nframes, blockvals);
  for (int i = 0; i < 3; ++i) p.zdump[i] = zdump ? zdump[i] : nullptr;
  p.M_y = t.M_y;
  p.M_c = t.M_c;
  p.W_y = t.W_y;
  p.W_c = t.W_c;
  p.err = err;
  p.wait_ns = wait_ns;
  p.withhold = withhold;
  int grid = ctas > 0 && ctas < sm_count() ? ctas : sm_count();
  if (p.total_items < grid) grid = p.total_items;
  e = launch_single(p, grid, g.w, g.nc == g.w, g.low_pass, zdump != nullptr, bps, s);
  if (e == cudaSuccess) ++*launches;
  return e;
}

}  // namespace vca
