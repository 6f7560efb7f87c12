// Frame reduction of the analyzer (Section 2 of the paper: the seven per-frame features).
//
// Each frame is summed by kSlices CTAs.  CTA s takes the blocks [s*C/kSlices, (s+1)*C/kSlices):
// thread i sums blocks i, i + 256, ... of the slice exactly in fixed point, then a fixed FP64
// shared-memory tree gives the slice's seven partial sums.  The last CTA of the frame to finish
// (a per-frame arrival counter) adds the kSlices partials in slice order and writes the
// features, so the result does not depend on scheduling:
//   E_P = sum_k H_{P,k} / (C N_P^2), L_P = sum_k L_{P,k} / C,
//   h_t = sum_k |H_{Y,k,t} - H_{Y,k,t-1}| / (C w^2), and h = 0 without a previous frame.
// The CTAs of the last frame also copy its luma energies as the next call's previous-frame state
// (into a buffer distinct from the one read here).
#include <cstdio>
#include <mutex>

#include "vca.h"
#include "vca_internal.h"

namespace vca {
namespace {

constexpr int kThreads = 256;
constexpr int kSlices = 8;
constexpr int kSums = 7;  // H_Y, L_Y, H_U, L_U, H_V, L_V, |dH_Y|

// Slice `slice` of frame f (one CTA of kThreads threads).
__device__ __forceinline__ void reduce_slice(const ReduceArgs& a, int f, int slice) {
  __shared__ double part[kSums][kThreads];
  __shared__ bool last;
  const int tid = threadIdx.x;
  const int64_t C = a.C;
  const int64_t k0 = C * slice / kSlices, k1 = C * (slice + 1) / kSlices;
  const float* bv = a.blockvals + (int64_t)f * N_ROWS * C;
  const float* prev = f > 0 ? a.blockvals + (int64_t)(f - 1) * N_ROWS * C + ROW_H_Y * C : a.prevH_in;
  const bool has_prev = f > 0 || a.has_prev;

  // Per-thread sums in fixed point, v * 2^23 as an unsigned integer.  Every block value the
  // analyzer writes is 0 or at least 1 (H sums weights >= 1 times integers |Z| < 2^16; L is the
  // square root of an integer), so it is a multiple of 2^-23 below 2^30 and converts exactly;
  // the sums, and |H_t - H_{t-1}|, are then exact integer arithmetic (a thread adds at most
  // 2^20 / (8 * 256) = 512 values below 2^53).  The per-thread sums enter the FP64 tree below.
  unsigned long long q[kSums] = {0, 0, 0, 0, 0, 0, 0};
  for (int64_t k = k0 + tid; k < k1; k += kThreads) {
    unsigned long long v[N_ROWS];
#pragma unroll
    for (int r = 0; r < N_ROWS; ++r) {
      v[r] = __float2ull_rn(bv[r * C + k] * 8388608.0f);
      q[r] += v[r];
    }
    if (has_prev) {
      const unsigned long long p = __float2ull_rn(prev[k] * 8388608.0f);
      q[6] += v[ROW_H_Y] > p ? v[ROW_H_Y] - p : p - v[ROW_H_Y];
    }
  }
  double s[kSums];
#pragma unroll
  for (int r = 0; r < kSums; ++r) s[r] = (double)q[r] * 1.1920928955078125e-07;  // 2^-23
  if (f == a.nframes - 1) {
    for (int64_t k = k0 + tid; k < k1; k += kThreads) a.prevH_out[k] = bv[ROW_H_Y * C + k];
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
    double* mine = a.partials + ((int64_t)f * kSlices + slice) * kSums;
#pragma unroll
    for (int r = 0; r < kSums; ++r) mine[r] = part[r][0];
    __threadfence();
    last = atomicAdd(&a.counters[f], 1u) == kSlices - 1;
  }
  __syncthreads();
  if (last && tid == 0) {
    __threadfence();
    const volatile double* all = a.partials + (int64_t)f * kSlices * kSums;
    double t[kSums] = {0, 0, 0, 0, 0, 0, 0};
    for (int sl = 0; sl < kSlices; ++sl)
#pragma unroll
      for (int r = 0; r < kSums; ++r) t[r] += all[sl * kSums + r];
    double* out = a.feats + (int64_t)f * FEAT_STRIDE;
    const double Cd = (double)C;
    out[0] = t[ROW_H_Y] / a.normY;  // E_Y
    out[1] = t[6] / a.normY;        // h
    out[2] = t[ROW_L_Y] / Cd;       // L_Y
    out[3] = t[ROW_H_U] / a.normC;  // E_U
    out[4] = t[ROW_H_V] / a.normC;  // E_V
    out[5] = t[ROW_L_U] / Cd;       // L_U
    out[6] = t[ROW_L_V] / Cd;       // L_V
    out[7] = 0.0;
    a.counters[f] = 0;  // ready for the next launch (stream order separates launches)
  }
}

__global__ void __launch_bounds__(kThreads) reduce_kernel(const ReduceArgs a) {
  reduce_slice(a, blockIdx.x / kSlices, blockIdx.x % kSlices);
}

// One frame per analyzer of a batch: args[m] describes analyzer m (nframes 0: skipped this tick).
__global__ void __launch_bounds__(kThreads) reduce_batch_kernel(const ReduceArgs* __restrict__ args) {
  const ReduceArgs a = args[blockIdx.x / kSlices];
  if (a.nframes == 0) return;
  reduce_slice(a, 0, blockIdx.x % kSlices);
}

}  // namespace

size_t reduce_partials_bytes(int max_frames) { return (size_t)max_frames * kSlices * kSums * sizeof(double); }

cudaError_t launch_reduce(const Geometry& g, int nframes, const float* blockvals, const float* prevH_in,
                          int has_prev, float* prevH_out, double* feats, double* partials, unsigned int* counters,
                          cudaStream_t s, int64_t* launches) {
  if (nframes <= 0) return cudaSuccess;
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
  a.normC = (double)g.C * g.nc * g.nc;
  reduce_kernel<<<nframes * kSlices, kThreads, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) ++*launches;
  return e;
}

ReduceArgs reduce_args(const Geometry& g, int nframes, const float* blockvals, const float* prevH_in, int has_prev,
                       float* prevH_out, double* feats, double* partials, unsigned int* counters) {
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
  a.normC = (double)g.C * g.nc * g.nc;
  return a;
}

cudaError_t launch_reduce_batch(const ReduceArgs* d_args, int n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  reduce_batch_kernel<<<n * kSlices, kThreads, 0, s>>>(d_args);
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
constexpr size_t kNoAllocPartialBytes = (size_t)kNoAllocMaxFrames * kSlices * kSums * sizeof(double);
constexpr size_t kNoAllocBytes = kNoAllocPartialBytes + (size_t)kNoAllocMaxFrames * sizeof(unsigned int);
static_assert(kNoAllocPartialBytes % 256 == 0, "counters start on a 256-byte boundary");

// 114,688 B of partial sums (256 frames x 8 slices x 7 doubles), then 256 counters.
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
  if (prev_H_Y == last_H_Y)
    return noalloc_fail(VCA_E_ARG, "vca_reduce_frames_noalloc: prev_H_Y and last_H_Y must be different buffers");

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
  int64_t launches = 0;
  e = launch_reduce(g, n_frames, block_values, prev_H_Y, prev_H_Y != nullptr, last_H_Y, features,
                    static_cast<double*>(scratch),
                    reinterpret_cast<unsigned int*>(static_cast<unsigned char*>(scratch) + kNoAllocPartialBytes),
                    static_cast<cudaStream_t>(cuda_stream), &launches);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(msg, sizeof msg, "vca_reduce_frames_noalloc: launch failed: %s (%d)", cudaGetErrorString(e), (int)e);
    return noalloc_fail(VCA_E_CUDA, msg);
  }
  return VCA_OK;
}
