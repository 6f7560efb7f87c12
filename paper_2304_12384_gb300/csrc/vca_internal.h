// Internal declarations shared by the analyzer's host runtime and its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vca.h"

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
  int nc;            // chroma block columns (w / 2; w in 4:4:4)
  int ncv;           // chroma block rows (nc, except w in 4:2:2)
  int nbx, nby;      // block grid (shared by all planes)
  int64_t C;         // blocks per plane
  bool low_pass;
  int s1y, s2y;      // transform shifts, luma
  int s1c, s2c;      // transform shifts, chroma (s1 of the row length nc, s2 of the column length ncv)
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
  const int8_t* M_c;   // nc x nc: the chroma row transform
  const int8_t* M_cv;  // ncv x ncv: the chroma column transform (M_c, or M_y in 4:2:2)
  const float* W_y;    // w x w
  const float* W_c;    // ncv x nc (row stride nc)
};

// Arguments of one launch of the plain block routine (one plane kind of a batch of frames).
struct PlainArgs {
  const uint8_t* base[2];  // plane of frame 0, per plane in this launch
  int64_t pitch;           // bytes between rows
  int64_t fstride;         // bytes between frames
  int width, height;       // plane size in samples
  int nbx;
  int64_t C;
  int s1, s2;
  const int8_t* M;         // NH x NH: the row transform
  const int8_t* M2;        // NV x NV: the column transform (M when the blocks are square)
  const float* W;          // NV x NH, W[0] = 0
  float* outH[2];
  float* outL[2];
  int64_t out_fstride;     // floats between frames of block values
  int16_t* zdump[2];       // optional coefficient dump (frame 0 only)
};

// Arguments of the frame reduction of one analyzer's batch of frames.
struct ReduceArgs {
  const float* blockvals;
  const float* prevH_in;
  float* prevH_out;
  double* feats;
  unsigned long long* partials;  // [frame][slice][sum] 128-bit slice totals (reduce_partials_bytes)
  unsigned int* counters;  // [frame], zero on entry, left at zero on exit
  int64_t C;
  int nframes;
  int has_prev;
  double normY, normC;  // C w^2 and C (w/2)^2
};

// Integer DCT matrix M_N[k][n] = round_half_away(64 sqrt(N) alpha_k cos(pi (2n+1) k / 2N)).
void make_dct_matrix(int N, int8_t* out);
// Energy weights w_N(u,v) = exp(|((u+1)(v+1)/N^2)^2 - 1|) rounded to FP32, with (0,0) set to 0.
void make_energy_weights(int N, float* out);
// Rectangular form for blocks of Nv rows and Nh columns: w(u,v) = exp(|((u+1)(v+1)/(Nv Nh))^2 - 1|)
// at out[u * Nh + v], (0,0) set to 0.
void make_energy_weights_rect(int Nv, int Nh, float* out);
// Stage shifts s1 = log2 N + B - 9, s2 = log2 N + 6.
void transform_shifts(int N, int B, int* s1, int* s2);
// True if m (N x N, row-major) can replace the round-cosine matrix for B-bit samples: N in
// {4, 8, 16, 32}, m[0][0] = 64, the even/odd DCT symmetry at every level (what the butterfly
// form and the tensor-core bias cancellation rely on), and T within 16 bits for B <= 10.  Else
// false with a one-line reason in why.
bool check_dct_matrix(int N, int B, const int8_t* m, char* why, size_t why_len);

// CUDA-core analysis of n frames: writes block values (and, when the dump pointers are
// non-null, the quantised coefficients of frame 0).  Returns the launch status and adds
// the number of kernels launched to *launches.
// warps: CTA size of the block routine, 2, 4 or 8 warps (blocks per CTA = warps * 32 / N).
cudaError_t launch_plain(const Geometry& g, const FramePlanes& fp, int nframes, const DeviceTables& t,
                         float* blockvals, int16_t* const zdump[3], cudaStream_t s, int64_t* launches,
                         int warps = 4);

// Tensor-core analysis (same outputs).  Returns cudaErrorNotSupported if the geometry is
// outside what the tensor-core kernel handles.  *err (device) receives a nonzero code if a
// bounded wait inside the kernel gave up.
// ctas: CTAs of the launch (0: one per SM; never more than the SMs or the tiles).  wait_ns: limit
// of the kernel's bounded waits (0: about 2 s); withhold >= 0: a work item (128x128 tile, counted
// over the launch) whose copies are not issued, so that the wait for it runs out (failure-path
// tests).
cudaError_t launch_tc(const Geometry& g, const FramePlanes& fp, int nframes, const DeviceTables& t,
                      float* blockvals, int16_t* const zdump[3], int* err, cudaStream_t s, int64_t* launches,
                      int ctas = 0, long long wait_ns = 0, int withhold = -1);
bool tc_supported(const Geometry& g);

// Batched tensor-core analysis: one frame of each of up to tc_batch_max_members() analyzers of
// one sample size in one launch of the persistent kernel.  The launch's member table and tensor
// maps are its kernel parameters (tc_batch_params_bytes(), about 29 KB), which the host fills
// with tc_batch_fill; a captured launch's parameters are replaced per tick in the graph.
// A member's tensor maps for its most recent distinct frames: frames pushed from a ring of
// device buffers repeat their plane addresses, and a tick whose frame matches an entry (plane
// pointers and pitches) copies its three maps instead of encoding them again.  One cache per
// member of a batch (the member's geometry is fixed), owned by the batch.
struct TcMapCache;
TcMapCache* tc_map_cache_new();
void tc_map_cache_free(TcMapCache* c);
// Members of one batched tensor-core launch (a tick with more members of one sample size takes
// several launches).
constexpr int kMaxBatchMembers = 64;
struct TcBatchFrame {
  const Geometry* g;   // the member's analysis geometry (tc_supported)
  FramePlanes fp;      // its frame (frame strides unused)
  float* blockvals;    // its [6][C] block values
  TcMapCache* maps;    // the member's map cache, or null to encode every tick
  int red;             // its entry in the batch's TcRedMember table
  int red_flags;       // kRedHasPrev | kRedPrevBuf * (previous energies in prevH[1]) | kRedGraph * k
};
// Frame reduction fused into a batched tensor-core tick, per member (device memory, written when
// the batch is made).  At the end of the launch each CTA adds the exact fixed-point sums of its
// own tiles' block values (and of |dH_Y|, reading the previous energies and writing this tick's)
// to the member's accumulators and counts its tiles; the CTA that completes the count writes the
// features and leaves the accumulators and the count at zero.  Tick graph k uses acc[k], done[k],
// feats[k], so that a tick that failed leaves the other graph's state clean.
struct TcRedMember {
  unsigned long long* acc[2];  // kRedSums x (low 32-bit part, rest) totals
  unsigned int* done[2];       // tiles counted
  float* prevH[2];             // the analyzer's two previous-energy buffers
  double* feats[2];            // the member's feature row (FEAT_STRIDE doubles; mapped host memory)
  double normY, normC;         // C w^2 and C Nv Nh
};
constexpr int kRedSums = 7;  // H_Y, L_Y, H_U, L_U, H_V, L_V, |dH_Y|
constexpr int kRedHasPrev = 1, kRedPrevBuf = 2, kRedGraph = 4;
int tc_batch_max_members();
size_t tc_batch_params_bytes();
// Fills the parameter block at params (host memory, tc_batch_params_bytes()) for n frames, the
// DCT tables t, the device error flag err, the fused reduction's member table red (device) and
// err_host (the tick's flag in mapped host memory, set to the code of a wait that ran out);
// cudaErrorInvalidValue if n is out of range, the frames' sample sizes differ or a tensor map
// cannot be encoded.
cudaError_t tc_batch_fill(void* params, const TcBatchFrame* frames, int n, const DeviceTables& t, int* err,
                          const TcRedMember* red, double* err_host, long long wait_ns = 0, int withhold = -1);
// Sets up the kernel instance for this sample size and low_pass (outside any stream capture).
cudaError_t tc_batch_prepare(int w, bool c444, int bps, bool low_pass);
// Work items (128x128 luma tiles) of a filled parameter block.
int tc_batch_items(const void* params);
// The kernel a batched launch of this sample size and low_pass runs (to find its graph node).
const void* tc_batch_kernel(int w, bool c444, int bps, bool low_pass);
// Kernel-node parameters of one batched tensor-core launch (its function, grid, block and dynamic
// shared memory; args[0] points at its parameter block), for a graph built node by node.
cudaError_t tc_batch_node_params(int w, bool c444, int bps, bool low_pass, int grid, void** args,
                                 cudaKernelNodeParams* kp);

// Exact frame reduction: features of n frames (the block sums exact in 128-bit fixed point, each
// total rounded once to FP64) and the h state update.  `partials` holds reduce_partials_bytes(max
// frames) of scratch; `counters` (one per frame) must be zero on entry and is zero again on exit.
// feats may be mapped pinned host memory.  If err is not null, the launch also copies the analysis
// kernel's timeout flag *err into *err_out (which may be mapped host memory) and clears *err.
size_t reduce_partials_bytes(int max_frames);
cudaError_t launch_reduce(const Geometry& g, int nframes, const float* blockvals, const float* prevH_in,
                          int has_prev, float* prevH_out, double* feats, unsigned long long* partials,
                          unsigned int* counters, cudaStream_t s, int64_t* launches, int* err = nullptr,
                          int* err_out = nullptr);

// Reduction arguments of one analyzer (reduce_partials_bytes(nframes) of `partials`; `counters`
// zero on entry).
ReduceArgs reduce_args(const Geometry& g, int nframes, const float* blockvals, const float* prevH_in, int has_prev,
                       float* prevH_out, double* feats, unsigned long long* partials, unsigned int* counters);
// Frame reduction of one frame per analyzer of a batch, in one launch: d_args (device) holds n
// ReduceArgs with nframes 1 (or 0 for an analyzer skipped this tick).
cudaError_t launch_reduce_batch(const ReduceArgs* d_args, int n, int slices, cudaStream_t s);
// Slices per frame of a batched reduction whose largest member has max_C blocks per plane.
int reduce_batch_slices(int64_t max_C);

// One CTA of the batched plain kernel: analyzer `member`, plane kind (0 luma, 1 chroma), plane
// within the kind (chroma: 0 U, 1 V) and block chunk (BPC blocks).
struct BatchCta {
  uint16_t member;
  uint8_t kind;
  uint8_t plane;
  uint32_t chunk;
};
// Per-analyzer arguments of one batched tick: the plain routine's arguments for luma and chroma,
// the sample size, and whether the analyzer takes part in this tick.
struct BatchMemberArgs {
  PlainArgs pa[2];
  int32_t bps;
  int32_t active;
  int32_t pad[2];
};
// Blocks per CTA of the (4-warp) plain routine for blocks of NV rows.
constexpr int plain_blocks_per_cta(int NV) { return 4 * (32 / NV); }
// The batched plain analysis of one frame per analyzer: n_cta CTAs described by d_map (device),
// arguments d_args (device, one per analyzer).  All analyzers share block sizes w (luma) and
// ncv x nc (chroma rows x columns) and low_pass.
cudaError_t launch_batch_plain(const BatchCta* d_map, int n_cta, const BatchMemberArgs* d_args, int w, int nc,
                               int ncv, bool low_pass, cudaStream_t s);

// One plane of the 2x2 downsample: n frames of w x h samples at src (pitch, frame stride in
// bytes) -> wd x hd = ceil(w/2) x ceil(h/2) samples at dst.
struct DownPlane {
  const uint8_t* src;
  int64_t src_pitch, src_fstride;
  uint8_t* dst;
  int64_t dst_pitch, dst_fstride;
  int w, h, wd, hd;
};
struct DownArgs {
  DownPlane p[3];  // Y, U, V
};
// Halves the three planes of n frames (the downsample reading of the low-pass option).
cudaError_t launch_downsample(const DownArgs& a, int nframes, int bps, cudaStream_t s);

// Sets the calling thread's vca_last_error message.
void record_error(const char* msg);

// Launch shapes (vca_tune.cpp): the table entry of a configuration, if any; an analyzer's CTA
// size of the CUDA-core form (2, 4 or 8 warps) and CTA count of a tensor-core launch (0: one per SM).
bool tune_lookup(const vca_config& c, vca_tune_entry* out);
vca_status set_launch_shape(vca_analyzer* a, int plain_warps, int tc_ctas);

}  // namespace vca
