// Internal declarations shared by the analyzer's host runtime and its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vca {

// Per-frame block values are stored as [frame][6][C] FP32: the order of the six rows.
enum BlockValueRow { ROW_H_Y = 0, ROW_L_Y = 1, ROW_H_U = 2, ROW_L_U = 3, ROW_H_V = 4, ROW_L_V = 5, N_ROWS = 6 };

// Per-frame features are stored as 8 doubles: E_Y, h, L_Y, E_U, E_V, L_U, L_V, spare.
constexpr int FEAT_STRIDE = 8;

struct Geometry {
  int W, H;          // luma plane size (samples)
  int cw, ch;        // chroma plane size (samples)
  int B;             // bit depth (8 or 10)
  int bps;           // bytes per sample (1 or 2)
  int w;             // luma block size
  int nc;            // chroma block size (w / 2)
  int nbx, nby;      // block grid (shared by all planes)
  int64_t C;         // blocks per plane
  bool low_pass;
  int s1y, s2y;      // transform shifts, luma
  int s1c, s2c;      // transform shifts, chroma
};

// Planes of frame 0 of a batch and the byte strides to the next row / frame.
struct FramePlanes {
  const uint8_t* y;
  const uint8_t* u;
  const uint8_t* v;
  int64_t pitch_y, pitch_uv;
  int64_t fstride_y, fstride_uv;
};

// Device copies of the integer DCT matrices and FP32 energy weights (weight (0,0) = 0).
struct DeviceTables {
  const int8_t* M_y;   // w x w
  const int8_t* M_c;   // (w/2) x (w/2)
  const float* W_y;    // w x w
  const float* W_c;    // (w/2) x (w/2)
};

// Integer DCT matrix M_N[k][n] = round_half_away(64 sqrt(N) alpha_k cos(pi (2n+1) k / 2N)).
void make_dct_matrix(int N, int8_t* out);
// Energy weights w_N(u,v) = exp(|((u+1)(v+1)/N^2)^2 - 1|) rounded to FP32, with (0,0) set to 0.
void make_energy_weights(int N, float* out);
// Stage shifts s1 = log2 N + B - 9, s2 = log2 N + 6.
void transform_shifts(int N, int B, int* s1, int* s2);

// CUDA-core analysis of n frames: writes block values (and, when the dump pointers are
// non-null, the quantised coefficients of frame 0).  Returns the launch status and adds
// the number of kernels launched to *launches.
cudaError_t launch_plain(const Geometry& g, const FramePlanes& fp, int nframes, const DeviceTables& t,
                         float* blockvals, int16_t* const zdump[3], cudaStream_t s, int64_t* launches);

// Tensor-core analysis (same outputs).  Returns cudaErrorNotSupported if the geometry is
// outside what the tensor-core kernel handles.  *err (device) receives a nonzero code if a
// bounded wait inside the kernel gave up.
cudaError_t launch_tc(const Geometry& g, const FramePlanes& fp, int nframes, const DeviceTables& t,
                      float* blockvals, int16_t* const zdump[3], int* err, cudaStream_t s, int64_t* launches);
bool tc_supported(const Geometry& g);

// Deterministic FP64 frame reduction: features of n frames and the h state update.  `partials`
// holds reduce_partials_bytes(max frames) of scratch; `counters` (one per frame) must be zero on
// entry and is zero again on exit.
size_t reduce_partials_bytes(int max_frames);
cudaError_t launch_reduce(const Geometry& g, int nframes, const float* blockvals, const float* prevH_in,
                          int has_prev, float* prevH_out, double* feats, double* partials, unsigned int* counters,
                          cudaStream_t s, int64_t* launches);

// Sets the calling thread's vca_last_error message.
void record_error(const char* msg);

}  // namespace vca
