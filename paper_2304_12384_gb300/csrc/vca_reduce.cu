// Frame reduction of the analyzer (Section 2 of the paper: the seven per-frame features).
//
//   E_P = sum_k H_{P,k} / (C N_P^2), L_P = sum_k L_{P,k} / C,
//   h_t = sum_k |H_{Y,k,t} - H_{Y,k,t-1}| / (C w^2), and h = 0 without a previous frame.
//
// The sums are exact.  Every block value the analyzer writes is 0 or a float in [1, 2^30) (H adds
// weights >= 1 times integers |Z| < 2^16 over at most 32 x 32 coefficients; L is the square root
// of an integer), so it is a multiple of 2^-23 and v * 2^23 is an integer below 2^53, taken from
// the float's bits with integer instructions.  The per-frame sums of those integers, and of
// |H_t - H_{t-1}| in the same units, are kept in 128 bits; only the final total is rounded to
// FP64 (once, to nearest) and divided by its norm.  The features therefore do not depend on how
// the blocks are split between threads and CTAs.
//
// Each frame is summed by S CTAs ("slices", S = ceil(C / 512) up to 32, chosen per launch): CTA s
// takes the blocks [s*C/S, (s+1)*C/S), its threads and warps combine their sums by shuffles and
// shared memory, and the last CTA of the frame to finish (a per-frame arrival counter) adds the S
// slice totals and writes the features.  The CTAs of the last frame also copy its luma energies
// as the next call's previous-frame state (into a buffer distinct from the one read here).
#include <cstdio>
#include <mutex>

#include "vca.h"
#include "vca_fixed.cuh"
#include "vca_internal.h"

namespace vca {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxSlices = 32;
constexpr int64_t kSliceBlocks = 512;

// Slices of a frame of C blocks.
int slices_for(int64_t C) {
  const int64_t s = (C + kSliceBlocks - 1) / kSliceBlocks;
  return (int)(s < 1 ? 1 : s > kMaxSlices ? kMaxSlices : s);
}

// Slice `slice` of S of frame f (one CTA of kThreads threads).  partials: [frame][kMaxSlices][kSums]
// 128-bit slice totals.
__device__ __forceinline__ void reduce_slice(const ReduceArgs& a, int f, int slice, int S) {
  __shared__ U128 wsum[kWarps][kSums];
  __shared__ bool last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t C = a.C;
  const int64_t k0 = C * slice / S, k1 = C * (slice + 1) / S;
  const float* bv = a.blockvals + (int64_t)f * N_ROWS * C;
  const float* prev = f > 0 ? a.blockvals + (int64_t)(f - 1) * N_ROWS * C + ROW_H_Y * C : a.prevH_in;
  const bool has_prev = f > 0 || a.has_prev;

  U128 q[kSums];
#pragma unroll
  for (int r = 0; r < kSums; ++r) q[r] = U128{0ull, 0ull};
  for (int64_t k = k0 + tid; k < k1; k += kThreads) {
    unsigned long long v[N_ROWS];
#pragma unroll
    for (int r = 0; r < N_ROWS; ++r) {
      v[r] = fixed23(bv[r * C + k]);
      add_to(q[r], v[r]);
    }
    if (has_prev) {
      const unsigned long long pv = fixed23(prev[k]);
      add_to(q[6], v[ROW_H_Y] > pv ? v[ROW_H_Y] - pv : pv - v[ROW_H_Y]);
    }
  }
  if (f == a.nframes - 1) {
    for (int64_t k = k0 + tid; k < k1; k += kThreads) a.prevH_out[k] = bv[ROW_H_Y * C + k];
  }
#pragma unroll
  for (int r = 0; r < kSums; ++r) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      U128 other;
      other.lo = __shfl_xor_sync(0xffffffffu, q[r].lo, o);
      other.hi = __shfl_xor_sync(0xffffffffu, q[r].hi, o);
      add_to(q[r], other);
    }
    if (lane == 0) wsum[warp][r] = q[r];
  }
  __syncthreads();
  if (tid < kSums) {  // this slice's total of sum tid, published before the arrival below
    U128 t = wsum[0][tid];
#pragma unroll
    for (int w = 1; w < kWarps; ++w) add_to(t, wsum[w][tid]);
    volatile unsigned long long* mine = a.partials + (((int64_t)f * kMaxSlices + slice) * kSums + tid) * 2;
    mine[0] = t.lo;
    mine[1] = t.hi;
    __threadfence();
  }
  __syncthreads();
  if (tid == 0) last = atomicAdd(&a.counters[f], 1u) == (unsigned)S - 1u;
  __syncthreads();
  if (!last) return;
  // The last slice to arrive: every slice total, read in parallel, then added in slice order.
  __shared__ U128 slice_tot[kMaxSlices][kSums];
  __threadfence();
  const volatile unsigned long long* all = a.partials + (int64_t)f * kMaxSlices * kSums * 2;
  for (int i = tid; i < S * kSums; i += kThreads) slice_tot[i / kSums][i % kSums] = U128{all[2 * i], all[2 * i + 1]};
  __syncthreads();
  if (tid < kSums) {  // thread r: sum r -> its feature (E_Y, h, L_Y, E_U, E_V, L_U, L_V)
    U128 t{0ull, 0ull};
    for (int sl = 0; sl < S; ++sl) add_to(t, slice_tot[sl][tid]);
    int slot;
    const double value = feature_of_sum(tid, t, (double)C, a.normY, a.normC, slot);
    double* out = a.feats + (int64_t)f * FEAT_STRIDE;
    out[slot] = value;
    if (tid == 0) {
      out[7] = 0.0;
      a.counters[f] = 0;  // ready for the next launch (stream order separates launches)
    }
  }
}

// err, if not null: the analysis kernel's timeout flag, copied into *err_out and cleared (the
// analysis launch has finished before this one starts).
__global__ void __launch_bounds__(kThreads) reduce_kernel(const ReduceArgs a, int S, int* err, int* err_out) {
  if (err && blockIdx.x == 0 && threadIdx.x == 0) {
    *err_out = *err;
    *err = 0;
  }
  reduce_slice(a, blockIdx.x / S, blockIdx.x % S, S);
}

// One frame per analyzer of a batch: args[m] describes analyzer m (nframes 0: skipped this tick).
__global__ void __launch_bounds__(kThreads) reduce_batch_kernel(const ReduceArgs* __restrict__ args, int S) {
  const ReduceArgs a = args[blockIdx.x / S];
  if (a.nframes == 0) return;
  reduce_slice(a, 0, blockIdx.x % S, S);
}

}  // namespace

size_t reduce_partials_bytes(int max_frames) { return (size_t)max_frames * kMaxSlices * kSums * 16; }

cudaError_t launch_reduce(const Geometry& g, int nframes, const float* blockvals, const float* prevH_in,
                          int has_prev, float* prevH_out, double* feats, unsigned long long* partials,
                          unsigned int* counters, cudaStream_t s, int64_t* launches, int* err, int* err_out) {
  if (nframes <= 0) return cudaSuccess;
  const ReduceArgs a = reduce_args(g, nframes, blockvals, prevH_in, has_prev, prevH_out, feats, partials, counters);
  const int S = slices_for(g.C);
  reduce_kernel<<<nframes * S, kThreads, 0, s>>>(a, S, err, err_out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) ++*launches;
  return e;
}

ReduceArgs reduce_args(const Geometry& g, int nframes, const float* blockvals, const float* prevH_in, int has_prev,
                       float* prevH_out, double* feats, unsigned long long* partials, unsigned int* counters) {
  ReduceArgs a{};
  a.blockvals = blockvals;
  a.prevH_in = prevH_in;
  a.prevH_out = prevH_out;
  a.feats = feats;
  a.partials = partials;
  a.counters = counters;
  a.C = g.C;
  a.nframes = nframes;
  a.has_prev = has_prev;
  a.normY = (double)g.C * g.w * g.w;
  a.normC = (double)g.C * g.ncv * g.nc;
  return a;
}

int reduce_batch_slices(int64_t max_C) { return slices_for(max_C); }

cudaError_t launch_reduce_batch(const ReduceArgs* d_args, int n, int slices, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (slices < 1 || slices > kMaxSlices) return cudaErrorInvalidValue;
  reduce_batch_kernel<<<n * slices, kThreads, 0, s>>>(d_args, slices);
  return cudaGetLastError();
}

}  // namespace vca

// ---- Allocation-free entry point ------------------------------------------------------
//
// vca_reduce_frames_noalloc runs the same reduction kernel on block values the caller already
// holds on the device, with its scratch (the per-slice partial sums and the per-frame arrival
// counters) in a fixed array of this module instead of memory from the CUDA allocator.  It exists
// for callers that must not allocate device memory on their hot path: a serving loop that has
// budgeted every byte of HBM up front to decide how many channels it admits, and a host thread
// that keeps other streams' work in flight, for which cudaMalloc may block and cudaFree waits for
// the whole device.
//
// The scratch is one array per device, so calls that can run on the device at the same time
// (different streams without ordering between them, or several host threads) race on it and give
// wrong features; the caller keeps such calls ordered (one stream, or events).  The arrival
// counters must be zero when a launch starts: the loader zero-fills the array when the module is
// loaded, and every launch leaves the counters of the frames it touched at zero again.  The first
// call on each device looks up the array's device address (cudaGetSymbolAddress, which may also
// load the module), so make that first call before capturing a stream into a CUDA graph.

namespace vca {
namespace {

constexpr int kNoAllocMaxFrames = 256;
constexpr size_t kNoAllocPartialBytes = (size_t)kNoAllocMaxFrames * kMaxSlices * kSums * 16;
constexpr size_t kNoAllocBytes = kNoAllocPartialBytes + (size_t)kNoAllocMaxFrames * sizeof(unsigned int);
static_assert(kNoAllocPartialBytes % 256 == 0, "counters start on a 256-byte boundary");

// 917,504 B of slice totals (256 frames x 32 slices x 7 sums x 16 bytes), then 256 counters.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

vca_status noalloc_fail(vca_status st, const char* msg) {
  record_error(msg);
  return st;
}

}  // namespace
}  // namespace vca

extern "C" vca_status vca_reduce_frames_noalloc(const float* block_values, int64_t blocks_per_plane,
                                                int32_t block_size, int32_t n_frames, const float* prev_H_Y,
                                                float* last_H_Y, double* features, void* cuda_stream) {
  using namespace vca;
  char msg[256];
  if (!block_values || !last_H_Y || !features)
    return noalloc_fail(VCA_E_ARG, "vca_reduce_frames_noalloc: block_values, last_H_Y and features must be non-NULL");
  if (block_size != 16 && block_size != 32)
    return noalloc_fail(VCA_E_ARG, "vca_reduce_frames_noalloc: block_size must be 16 or 32");
  if (blocks_per_plane < 1 || blocks_per_plane > (int64_t)1 << 30)
    return noalloc_fail(VCA_E_ARG, "vca_reduce_frames_noalloc: blocks_per_plane must be in [1, 2^30]");
  if (n_frames < 1 || n_frames > kNoAllocMaxFrames) {
    snprintf(msg, sizeof msg,
             "vca_reduce_frames_noalloc: n_frames = %d is outside [1, %d], the frames its fixed scratch holds",
             (int)n_frames, kNoAllocMaxFrames);
    return noalloc_fail(VCA_E_ARG, msg);
  }
  // last_H_Y is written by the CTAs of the last frame while others still read prev_H_Y and the
  // block values: its bytes may overlap neither.
  {
    const uintptr_t l0 = (uintptr_t)last_H_Y, l1 = l0 + (uintptr_t)blocks_per_plane * sizeof(float);
    const uintptr_t b0 = (uintptr_t)block_values,
                    b1 = b0 + (uintptr_t)n_frames * N_ROWS * (uintptr_t)blocks_per_plane * sizeof(float);
    if (l0 < b1 && b0 < l1)
      return noalloc_fail(VCA_E_ARG, "vca_reduce_frames_noalloc: last_H_Y overlaps block_values");
    if (prev_H_Y) {
      const uintptr_t p0 = (uintptr_t)prev_H_Y, p1 = p0 + (uintptr_t)blocks_per_plane * sizeof(float);
      if (l0 < p1 && p0 < l1)
        return noalloc_fail(VCA_E_ARG, "vca_reduce_frames_noalloc: last_H_Y overlaps prev_H_Y");
    }
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return noalloc_fail(VCA_E_CUDA, "vca_reduce_frames_noalloc: no usable current device");
  }
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      e = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_noalloc_ptr[dev] = nullptr;
        cudaGetLastError();
        snprintf(msg, sizeof msg, "vca_reduce_frames_noalloc: cudaGetSymbolAddress failed: %s (%d)",
                 cudaGetErrorString(e), (int)e);
        return noalloc_fail(VCA_E_CUDA, msg);
      }
    }
    scratch = g_noalloc_ptr[dev];
  }

  Geometry g{};
  g.C = blocks_per_plane;
  g.w = block_size;
  g.nc = block_size / 2;
  g.ncv = g.nc;
  int64_t launches = 0;
  e = launch_reduce(g, n_frames, block_values, prev_H_Y, prev_H_Y != nullptr, last_H_Y, features,
                    static_cast<unsigned long long*>(scratch),
                    reinterpret_cast<unsigned int*>(static_cast<unsigned char*>(scratch) + kNoAllocPartialBytes),
                    static_cast<cudaStream_t>(cuda_stream), &launches);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(msg, sizeof msg, "vca_reduce_frames_noalloc: launch failed: %s (%d)", cudaGetErrorString(e), (int)e);
    return noalloc_fail(VCA_E_CUDA, msg);
  }
  return VCA_OK;
}
