// SI / TI: the spatial and temporal information features that the paper compares VCA with
// (Section 2: SI = max over frames of std[Sobel(F)], TI = max over frames of std[F_t - F_{t-1}]).
//
// Per frame, on the luma plane F in raw sample values:
//   SI_t = std over the interior pixels of sqrt(Gx^2 + Gy^2), Gx / Gy the 3x3 Sobel responses;
//   TI_t = std over all pixels of F_t - F_{t-1}, and 0 without a previous frame;
// the sequence values are the maxima (TI over t >= 1).  std is the population deviation.
//
// One kernel pass per push reads every frame once (each warp keeps the three rows around its
// current row in registers and takes the horizontal neighbours from the adjacent lanes) and
// accumulates four sums per frame: sum Gx^2 + Gy^2 and sum D, sum D^2 exactly in 64-bit
// integers, and sum sqrt(Gx^2 + Gy^2) (FP32 square root) in fixed point (2^-16 steps) -- integer
// sums, so the warp-level atomics give the same result in any order.  A finalize kernel turns the
// sums into the two deviations in FP64.  The luma plane of the push's last frame stays on the
// device as the previous frame of the next push.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "vca.h"
#include "vca_internal.h"

namespace {

constexpr int kWarps = 4;       // warps per CTA
constexpr int kPx = 4;          // consecutive samples per lane
constexpr int kStrip = 32 * kPx;  // columns per warp
constexpr int kRun = 32;        // rows per warp
constexpr double kMagScale = 65536.0;

struct SitiArgs {
  const uint8_t* y;       // frame 0
  int64_t pitch, fstride; // bytes
  const uint8_t* prev;    // luma of the frame before frame 0, or nullptr
  int64_t prev_pitch;
  int W, H;
  unsigned long long* acc;  // [frame][4]: sum m2, sum mag * 2^16, sum D (two's complement), sum D^2
};

// Samples x0 .. x0+3 of one row (one 4- or 8-byte load when they all lie inside the row, else one
// load each, zero past the edge).
template <typename Pix>
__device__ __forceinline__ void load4(const uint8_t* rowp, int x0, int W, int (&v)[kPx]) {
  const Pix* row = reinterpret_cast<const Pix*>(rowp);
  if (x0 + kPx - 1 < W) {
    if (sizeof(Pix) == 1) {
      const uint32_t w = *reinterpret_cast<const uint32_t*>(row + x0);
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] = (int)((w >> (8 * i)) & 0xffu);
    } else {
      const uint2 w = *reinterpret_cast<const uint2*>(row + x0);
      v[0] = (int)(w.x & 0xffffu);
      v[1] = (int)(w.x >> 16);
      v[2] = (int)(w.y & 0xffffu);
      v[3] = (int)(w.y >> 16);
    }
  } else {
#pragma unroll
    for (int i = 0; i < kPx; ++i) v[i] = x0 + i < W ? (int)row[x0 + i] : 0;
  }
}

// One row of a lane's window: its 4 samples and the neighbours on either side (from the adjacent
// lanes, or loaded at the warp's edges): p[0] = x0 - 1, p[1 + i] = x0 + i, p[5] = x0 + 4.
template <typename Pix>
__device__ __forceinline__ void load_row(const uint8_t* rowp, int x0, int W, int lane, int (&p)[kPx + 2]) {
  int v[kPx];
  load4<Pix>(rowp, x0, W, v);
  const Pix* row = reinterpret_cast<const Pix*>(rowp);
  int left = __shfl_up_sync(0xffffffffu, v[kPx - 1], 1);
  int right = __shfl_down_sync(0xffffffffu, v[0], 1);
  if (lane == 0) left = x0 > 0 && x0 - 1 < W ? (int)row[x0 - 1] : 0;
  if (lane == 31) right = x0 + kPx < W ? (int)row[x0 + kPx] : 0;
  p[0] = left;
#pragma unroll
  for (int i = 0; i < kPx; ++i) p[i + 1] = v[i];
  p[kPx + 1] = right;
}

// Each warp walks down kRun rows of a 128-column strip of one frame with the three rows around
// the current one in registers: per row one load of its 4 samples per lane, the neighbours by
// shuffle, and the same for the previous frame.
template <typename Pix, bool kWide>
__global__ void __launch_bounds__(kWarps * 32) siti_kernel(const SitiArgs a) {
  // A lane covers at most kRun * 4 = 128 pixels.  Up to 10-bit samples gx^2 + gy^2 < 2^25, so the
  // lane's sum fits 32 bits, and a row's 4 magnitudes (each < 2^29 in 2^-16 steps) too; 12-bit
  // samples take 64 bits for both (gx^2 + gy^2 < 2^30, magnitudes < 2^31).  D^2 < 2^24 and
  // |D| < 2^12 at every depth, so the lane's sums of those fit 32 bits.
  using Acc = typename std::conditional<kWide, unsigned long long, unsigned int>::type;
  const int lane = threadIdx.x & 31;
  const int f = blockIdx.z;
  const int y0 = (blockIdx.y * kWarps + (threadIdx.x >> 5)) * kRun;
  if (y0 >= a.H) return;  // whole warps only
  const int y1 = min(y0 + kRun, a.H);
  const int x0 = blockIdx.x * kStrip + lane * kPx;
  const uint8_t* F = a.y + (int64_t)f * a.fstride;
  const uint8_t* P = f > 0 ? a.y + (int64_t)(f - 1) * a.fstride : a.prev;
  const int64_t pp = f > 0 ? a.pitch : a.prev_pitch;
  Acc m2 = 0;
  unsigned long long mag = 0;
  unsigned int d2 = 0;
  int d1 = 0;
  int up[kPx + 2], mid[kPx + 2], dn[kPx + 2];
#pragma unroll
  for (int i = 0; i < kPx + 2; ++i) up[i] = 0;
  if (y0 > 0) load_row<Pix>(F + (int64_t)(y0 - 1) * a.pitch, x0, a.W, lane, up);
  load_row<Pix>(F + (int64_t)y0 * a.pitch, x0, a.W, lane, mid);
  for (int r = y0; r < y1; ++r) {
    if (r + 1 < a.H) {
      load_row<Pix>(F + (int64_t)(r + 1) * a.pitch, x0, a.W, lane, dn);
    } else {
#pragma unroll
      for (int i = 0; i < kPx + 2; ++i) dn[i] = 0;
    }
    if (P) {
      int pv[kPx];
      load4<Pix>(P + (int64_t)r * pp, x0, a.W, pv);
#pragma unroll
      for (int i = 0; i < kPx; ++i) {
        if (x0 + i < a.W) {
          const int d = mid[i + 1] - pv[i];
          d1 += d;
          d2 += (unsigned int)(d * d);
        }
      }
    }
    if (r >= 1 && r <= a.H - 2) {
      // Separable Sobel: per column the vertical smoothing up + 2 mid + dn and difference dn - up.
      int sm[kPx + 2], df[kPx + 2];
#pragma unroll
      for (int i = 0; i < kPx + 2; ++i) {
        sm[i] = up[i] + 2 * mid[i] + dn[i];
        df[i] = dn[i] - up[i];
      }
      Acc row_mag = 0;
#pragma unroll
      for (int i = 0; i < kPx; ++i) {
        const int x = x0 + i;
        if (x >= 1 && x <= a.W - 2) {
          const int gx = sm[i + 2] - sm[i];
          const int gy = df[i] + 2 * df[i + 1] + df[i + 2];
          const unsigned int sq = (unsigned int)(gx * gx + gy * gy);
          m2 += sq;
          // the magnitude in 2^-16 steps, below 2^31: a 32-bit conversion rounds it as a 64-bit one would
          row_mag += (Acc)(unsigned int)__float2int_rn(__fsqrt_rn((float)sq) * (float)kMagScale);
        }
      }
      mag += row_mag;
    }
#pragma unroll
    for (int i = 0; i < kPx + 2; ++i) {
      up[i] = mid[i];
      mid[i] = dn[i];
    }
  }
  unsigned long long s0 = m2, s2 = (unsigned long long)(long long)d1, s3 = d2;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    mag += __shfl_xor_sync(0xffffffffu, mag, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s3 += __shfl_xor_sync(0xffffffffu, s3, o);
  }
  if (lane == 0) {
    unsigned long long* acc = a.acc + (int64_t)f * 4;
    atomicAdd(acc + 0, s0);
    atomicAdd(acc + 1, mag);
    atomicAdd(acc + 2, s2);
    atomicAdd(acc + 3, s3);
  }
}

__global__ void siti_finalize(const unsigned long long* acc, int n, int W, int H, int has_prev, double* out) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n) return;
  const unsigned long long* s = acc + (int64_t)f * 4;
  const double ni = (double)(W - 2) * (double)(H - 2);
  double si = 0.0;
  if (ni > 0) {
    const double mean = (double)s[1] / kMagScale / ni;
    const double var = (double)s[0] / ni - mean * mean;
    si = var > 0 ? sqrt(var) : 0.0;
  }
  double ti = 0.0;
  if (f > 0 || has_prev) {
    const double na = (double)W * (double)H;
    const double mean = (double)(long long)s[2] / na;
    const double var = (double)s[3] / na - mean * mean;
    ti = var > 0 ? sqrt(var) : 0.0;
  }
  out[2 * f] = si;
  out[2 * f + 1] = ti;
}

vca_status sfail(vca_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  vca::record_error(buf);
  return s;
}

}  // namespace

struct vca_siti {
  int W = 0, H = 0, B = 8, bps = 1, max_batch = 0;
  cudaStream_t stream = nullptr;
  uint8_t* d_prev = nullptr;  // luma of the last pushed frame, pitch prev_pitch
  int64_t prev_pitch = 0;
  bool has_prev = false;
  uint8_t* d_stage = nullptr;  // host frames are copied here (pitch prev_pitch)
  size_t stage_bytes = 0;
  unsigned long long* d_acc = nullptr;
  double* d_out = nullptr;
  double* h_out = nullptr;  // pinned, max_batch x 2
  std::vector<vca_siti_features> done;
  int64_t frames = 0;
  double si_max = 0.0, ti_max = 0.0;
  int64_t launches = 0;
};

extern "C" {

vca_status vca_siti_open(int32_t width, int32_t height, int32_t bit_depth, int32_t max_batch, void* cuda_stream,
                         vca_siti** out) {
  if (!out) return sfail(VCA_E_ARG, "out is NULL");
  *out = nullptr;
  if (width < 3 || height < 3 || width > 16384 || height > 16384)
    return sfail(VCA_E_ARG, "width and height must be in [3, 16384]");
  if (bit_depth != 8 && bit_depth != 10 && bit_depth != 12) return sfail(VCA_E_ARG, "bit_depth must be 8, 10 or 12");
  if (max_batch < 1 || max_batch > 4096) return sfail(VCA_E_ARG, "max_batch must be in [1, 4096]");
  vca_siti* s = new (std::nothrow) vca_siti();
  if (!s) return sfail(VCA_E_NOMEM, "host allocation failed");
  s->W = width;
  s->H = height;
  s->B = bit_depth;
  s->bps = bit_depth > 8 ? 2 : 1;
  s->max_batch = max_batch;
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  s->prev_pitch = (int64_t)((width * s->bps + 255) / 256 * 256);
  cudaError_t e = cudaMalloc(&s->d_prev, (size_t)s->prev_pitch * height);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_acc, (size_t)max_batch * 4 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_out, (size_t)max_batch * 2 * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_out, (size_t)max_batch * 2 * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    vca_siti_close(s);
    return sfail(e == cudaErrorMemoryAllocation ? VCA_E_NOMEM : VCA_E_CUDA, "allocating SI/TI buffers: %s",
                 cudaGetErrorString(e));
  }
  *out = s;
  return VCA_OK;
}

vca_status vca_siti_push(vca_siti* s, const void* y, int64_t pitch, int64_t frame_stride, int32_t n_frames,
                         int32_t on_device) {
  if (!s || !y) return sfail(VCA_E_ARG, "NULL argument");
  if (n_frames < 1 || n_frames > s->max_batch) return sfail(VCA_E_ARG, "n_frames must be in [1, %d]", s->max_batch);
  if (pitch < (int64_t)s->W * s->bps) return sfail(VCA_E_ARG, "pitch smaller than a row");
  if (n_frames > 1 && frame_stride < pitch * s->H) return sfail(VCA_E_ARG, "frame stride smaller than a frame");
  if (on_device && (((uintptr_t)y & 15) || (pitch & 15))) return sfail(VCA_E_ARG, "device planes must be 16-byte aligned");
  const uint8_t* src = static_cast<const uint8_t*>(y);
  int64_t p = pitch, fs = frame_stride;
  cudaError_t e = cudaSuccess;
  if (!on_device) {
    const size_t fb = (size_t)s->prev_pitch * s->H;
    if (fb * n_frames > s->stage_bytes) {  // grows on demand; host frames only
      e = cudaStreamSynchronize(s->stream);
      cudaFree(s->d_stage);
      s->d_stage = nullptr;
      s->stage_bytes = 0;
      if (e == cudaSuccess) e = cudaMalloc(&s->d_stage, fb * n_frames);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return sfail(VCA_E_NOMEM, "allocating the SI/TI staging buffer: %s", cudaGetErrorString(e));
      }
      s->stage_bytes = fb * n_frames;
    }
    for (int i = 0; i < n_frames && e == cudaSuccess; ++i)
      e = cudaMemcpy2DAsync(s->d_stage + fb * i, s->prev_pitch, src + frame_stride * i, pitch, (size_t)s->W * s->bps,
                            s->H, cudaMemcpyHostToDevice, s->stream);
    src = s->d_stage;
    p = s->prev_pitch;
    fs = (int64_t)fb;
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_acc, 0, (size_t)n_frames * 4 * sizeof(unsigned long long), s->stream);
  if (e == cudaSuccess) {
    SitiArgs a{src, p, fs, s->has_prev ? s->d_prev : nullptr, s->prev_pitch, s->W, s->H, s->d_acc};
    const int runs = (s->H + kRun - 1) / kRun;
    const dim3 grid((unsigned)((s->W + kStrip - 1) / kStrip), (unsigned)((runs + kWarps - 1) / kWarps),
                    (unsigned)n_frames);
    if (s->bps == 1)
      siti_kernel<uint8_t, false><<<grid, kWarps * 32, 0, s->stream>>>(a);
    else if (s->B <= 10)
      siti_kernel<uint16_t, false><<<grid, kWarps * 32, 0, s->stream>>>(a);
    else
      siti_kernel<uint16_t, true><<<grid, kWarps * 32, 0, s->stream>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    siti_finalize<<<(n_frames + 127) / 128, 128, 0, s->stream>>>(s->d_acc, n_frames, s->W, s->H, s->has_prev ? 1 : 0,
                                                                   s->d_out);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(s->d_prev, s->prev_pitch, src + fs * (n_frames - 1), p, (size_t)s->W * s->bps, s->H,
                          cudaMemcpyDeviceToDevice, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->h_out, s->d_out, (size_t)n_frames * 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return sfail(VCA_E_CUDA, "SI/TI push: %s", cudaGetErrorString(e));
  }
  s->launches += 2;
  for (int i = 0; i < n_frames; ++i) {
    vca_siti_features f{s->frames + i, s->h_out[2 * i], s->h_out[2 * i + 1]};
    s->done.push_back(f);
    if (f.SI > s->si_max) s->si_max = f.SI;
    if ((s->frames + i > 0) && f.TI > s->ti_max) s->ti_max = f.TI;
  }
  s->frames += n_frames;
  s->has_prev = true;
  return VCA_OK;
}

vca_status vca_siti_read(vca_siti* s, int64_t frame, vca_siti_features* out) {
  if (!s || !out) return sfail(VCA_E_ARG, "NULL argument");
  if (frame < 0 || frame >= (int64_t)s->done.size()) return sfail(VCA_E_ARG, "frame %lld not pushed", (long long)frame);
  *out = s->done[(size_t)frame];
  return VCA_OK;
}

vca_status vca_siti_sequence(vca_siti* s, double* si, double* ti, int64_t* frames) {
  if (!s || !si || !ti || !frames) return sfail(VCA_E_ARG, "NULL argument");
  *si = s->si_max;
  *ti = s->ti_max;
  *frames = s->frames;
  return VCA_OK;
}

vca_status vca_siti_launch_count(vca_siti* s, int64_t* launches) {
  if (!s || !launches) return sfail(VCA_E_ARG, "NULL argument");
  *launches = s->launches;
  return VCA_OK;
}

vca_status vca_siti_close(vca_siti* s) {
  if (!s) return VCA_OK;
  if (s->stream) cudaStreamSynchronize(s->stream);
  cudaFree(s->d_prev);
  cudaFree(s->d_stage);
  cudaFree(s->d_acc);
  cudaFree(s->d_out);
  if (s->h_out) cudaFreeHost(s->h_out);
  delete s;
  return VCA_OK;
}

}  // extern "C"
