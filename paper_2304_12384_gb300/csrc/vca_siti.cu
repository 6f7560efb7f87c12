// SI / TI: the spatial and temporal information features that the paper compares VCA with
// (Section 2: SI = max over frames of std[Sobel(F)], TI = max over frames of std[F_t - F_{t-1}]).
//
// Per frame, on the luma plane F in raw sample values:
//   SI_t = std over the interior pixels of sqrt(Gx^2 + Gy^2), Gx / Gy the 3x3 Sobel responses;
//   TI_t = std over all pixels of F_t - F_{t-1}, and 0 without a previous frame;
// the sequence values are the maxima (TI over t >= 1).  std is the population deviation.
//
// One kernel pass per push reads every frame once (the 3x3 neighbourhood comes from L1/L2) and
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
#include <vector>

#include "vca.h"
#include "vca_internal.h"

namespace {

constexpr int kThreads = 256;
constexpr int kRows = 4;  // rows per CTA
constexpr double kMagScale = 65536.0;

struct SitiArgs {
  const uint8_t* y;       // frame 0
  int64_t pitch, fstride; // bytes
  const uint8_t* prev;    // luma of the frame before frame 0, or nullptr
  int64_t prev_pitch;
  int W, H;
  unsigned long long* acc;  // [frame][4]: sum m2, sum mag * 2^16, sum D (two's complement), sum D^2
};

template <typename Pix>
__device__ __forceinline__ int px(const uint8_t* base, int64_t pitch, int y, int x) {
  return (int)reinterpret_cast<const Pix*>(base + (int64_t)y * pitch)[x];
}

template <typename Pix>
__global__ void __launch_bounds__(kThreads) siti_kernel(const SitiArgs a) {
  const int f = blockIdx.y;
  const uint8_t* F = a.y + (int64_t)f * a.fstride;
  const uint8_t* P = f > 0 ? a.y + (int64_t)(f - 1) * a.fstride : a.prev;
  const int64_t pp = f > 0 ? a.pitch : a.prev_pitch;
  unsigned long long m2 = 0, mag = 0, d1 = 0, d2 = 0;
  const int y0 = blockIdx.x * kRows;
  for (int yy = y0; yy < min(y0 + kRows, a.H); ++yy) {
    for (int x = threadIdx.x; x < a.W; x += kThreads) {
      const int c = px<Pix>(F, a.pitch, yy, x);
      if (P) {
        const long long d = (long long)c - px<Pix>(P, pp, yy, x);
        d1 += (unsigned long long)d;
        d2 += (unsigned long long)(d * d);
      }
      if (yy >= 1 && yy <= a.H - 2 && x >= 1 && x <= a.W - 2) {
        const int tl = px<Pix>(F, a.pitch, yy - 1, x - 1), tc = px<Pix>(F, a.pitch, yy - 1, x),
                  tr = px<Pix>(F, a.pitch, yy - 1, x + 1);
        const int ml = px<Pix>(F, a.pitch, yy, x - 1), mr = px<Pix>(F, a.pitch, yy, x + 1);
        const int bl = px<Pix>(F, a.pitch, yy + 1, x - 1), bc = px<Pix>(F, a.pitch, yy + 1, x),
                  br = px<Pix>(F, a.pitch, yy + 1, x + 1);
        const long long gx = (long long)(tr + 2 * mr + br) - (tl + 2 * ml + bl);
        const long long gy = (long long)(bl + 2 * bc + br) - (tl + 2 * tc + tr);
        const unsigned long long s = (unsigned long long)(gx * gx + gy * gy);
        m2 += s;
        mag += (unsigned long long)__float2ll_rn(__fsqrt_rn((float)s) * (float)kMagScale);
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    m2 += __shfl_xor_sync(0xffffffffu, m2, o);
    mag += __shfl_xor_sync(0xffffffffu, mag, o);
    d1 += __shfl_xor_sync(0xffffffffu, d1, o);
    d2 += __shfl_xor_sync(0xffffffffu, d2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    unsigned long long* acc = a.acc + (int64_t)f * 4;
    atomicAdd(acc + 0, m2);
    atomicAdd(acc + 1, mag);
    atomicAdd(acc + 2, d1);
    atomicAdd(acc + 3, d2);
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
    const dim3 grid((unsigned)((s->H + kRows - 1) / kRows), (unsigned)n_frames);
    if (s->bps == 1)
      siti_kernel<uint8_t><<<grid, kThreads, 0, s->stream>>>(a);
    else
      siti_kernel<uint16_t><<<grid, kThreads, 0, s->stream>>>(a);
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
