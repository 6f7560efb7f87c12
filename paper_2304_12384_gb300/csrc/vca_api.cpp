// Host runtime behind include/vca.h: configuration checks, device state, launch
// sequencing, the pinned result ring and the cross-frame (h) state.
//
// Per push: analysis kernel(s) write per-block H and L for every frame of the batch,
// the FP64 reduction kernel turns them into the seven features (Section 2 of the
// paper) and updates the previous-frame luma energies, and one device-to-host copy
// moves the features into a pinned ring slot whose event tells readers when it landed.
#include <cuda_runtime.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <vector>

#include "vca.h"
#include "vca_internal.h"

using vca::DeviceTables;
using vca::FramePlanes;
using vca::Geometry;

namespace {

thread_local std::string g_last_error;

vca_status fail(vca_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return s;
}

}  // namespace

// Lets entry points defined in other translation units report a message through vca_last_error.
void vca::record_error(const char* msg) { g_last_error = msg; }

namespace {

vca_status cuda_fail(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky-free error so later calls are not blamed for it
  return fail(e == cudaErrorMemoryAllocation ? VCA_E_NOMEM : VCA_E_CUDA, "%s: %s (%d)", what,
              cudaGetErrorString(e), (int)e);
}

#define VCA_CUDA(call, what)                    \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

constexpr int kRing = 8;        // pushes whose features may be in flight at once
constexpr int kDefaultBatch = 64;
constexpr int kMaxBatch = 4096;
constexpr char kStateMagic[8] = {'V', 'C', 'A', 'S', 'T', 'A', 'T', '1'};

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

struct StateHeader {
  char magic[8];
  int64_t C;
  int64_t frames;
  int32_t has_prev;
  int32_t block_size;
  double seq_sum[7];
  int64_t seq_n;
  int64_t seq_nh;
};

}  // namespace

struct vca_analyzer {
  vca_config cfg{};
  Geometry g{};
  int kernel = VCA_KERNEL_PLAIN;
  int device = 0;
  cudaStream_t stream = nullptr;
  int max_batch = kDefaultBatch;

  void* d_tables = nullptr;
  DeviceTables tables{};
  float* d_blockvals = nullptr;  // (max_batch + 1) frames of [6][C]; the last slot serves coefficient dumps
  float* d_prevH[2] = {nullptr, nullptr};
  int cur_prev = 0;
  double* d_feats = nullptr;     // max_batch * FEAT_STRIDE
  int* d_err = nullptr;          // kernel wait-timeout flag of the current push
  double* d_red_partials = nullptr;       // frame-reduction scratch
  unsigned int* d_red_counters = nullptr; // one arrival counter per frame, kept at zero between launches
  uint8_t* d_staging = nullptr;  // host frames are copied here
  size_t staging_bytes = 0;

  double* h_ring = nullptr;      // pinned, kRing slots of max_batch * FEAT_STRIDE
  int* h_err = nullptr;          // pinned, one timeout flag per ring slot
  cudaEvent_t ring_ev[kRing] = {};
  cudaEvent_t t0_ev[kRing] = {};   // analysis-kernel timing, per ring slot
  cudaEvent_t t1_ev[kRing] = {};
  cudaEvent_t copy_ev = nullptr;
  bool timing = false;
  double kernel_ms = 0.0;
  int64_t timed_pushes = 0;

  struct Pending {
    int64_t first;
    int n;
    int slot;
    bool first_has_prev;
    bool timed;
  };
  std::deque<Pending> pending;
  int next_slot = 0;
  std::vector<vca_frame_features> done;
  int64_t done_base = 0;
  int64_t frames_pushed = 0;
  int has_prev = 0;
  int last_n = 0;
  int64_t launches = 0;
  double seq_sum[7] = {0, 0, 0, 0, 0, 0, 0};
  int64_t seq_n = 0;
  int64_t seq_nh = 0;
};

namespace {

vca_status check_config(const vca_config* c, Geometry* g) {
  if (!c) return fail(VCA_E_ARG, "config is NULL");
  if (c->width < 2 || c->height < 2 || (c->width & 1) || (c->height & 1) || c->width > 16384 ||
      c->height > 16384)
    return fail(VCA_E_ARG, "width/height must be even and in [2, 16384] (got %d x %d)", c->width, c->height);
  if (c->bit_depth != 8 && c->bit_depth != 10) return fail(VCA_E_ARG, "bit_depth must be 8 or 10");
  if (c->block_size != 16 && c->block_size != 32) {
    if (c->block_size == 8) return fail(VCA_E_UNSUPPORTED, "block_size 8 (4x4 chroma) is not supported");
    return fail(VCA_E_ARG, "block_size must be 16 or 32");
  }
  if (c->low_pass != 0 && c->low_pass != 1) return fail(VCA_E_ARG, "low_pass must be 0 or 1");
  if (c->pad_mode != VCA_PAD_REPLICATE && c->pad_mode != VCA_PAD_SKIP) return fail(VCA_E_ARG, "bad pad_mode");
  if (c->kernel < VCA_KERNEL_AUTO || c->kernel > VCA_KERNEL_TC) return fail(VCA_E_ARG, "bad kernel selector");
  if (c->max_batch < 0 || c->max_batch > kMaxBatch) return fail(VCA_E_ARG, "max_batch must be in [0, %d]", kMaxBatch);
  Geometry q{};
  q.W = c->width;
  q.H = c->height;
  q.cw = c->width / 2;
  q.ch = c->height / 2;
  q.B = c->bit_depth;
  q.bps = c->bit_depth > 8 ? 2 : 1;
  q.w = c->block_size;
  q.nc = c->block_size / 2;
  if (c->pad_mode == VCA_PAD_REPLICATE) {
    q.nbx = (q.W + q.w - 1) / q.w;
    q.nby = (q.H + q.w - 1) / q.w;
  } else {
    q.nbx = q.W / q.w;
    q.nby = q.H / q.w;
  }
  q.C = (int64_t)q.nbx * q.nby;
  if (q.C <= 0) return fail(VCA_E_ARG, "frame smaller than one block with pad_mode skip");
  q.low_pass = c->low_pass != 0;
  vca::transform_shifts(q.w, q.B, &q.s1y, &q.s2y);
  vca::transform_shifts(q.nc, q.B, &q.s1c, &q.s2c);
  if (g) *g = q;
  return VCA_OK;
}

void destroy(vca_analyzer* a) {
  if (!a) return;
  int prev_dev = -1;
  cudaGetDevice(&prev_dev);
  cudaSetDevice(a->device);
  cudaStreamSynchronize(a->stream);
  cudaFree(a->d_tables);
  cudaFree(a->d_blockvals);
  cudaFree(a->d_prevH[0]);
  cudaFree(a->d_prevH[1]);
  cudaFree(a->d_feats);
  cudaFree(a->d_err);
  cudaFree(a->d_red_partials);
  cudaFree(a->d_red_counters);
  if (a->h_err) cudaFreeHost(a->h_err);
  cudaFree(a->d_staging);
  if (a->h_ring) cudaFreeHost(a->h_ring);
  for (auto& e : a->ring_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : a->t0_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : a->t1_ev)
    if (e) cudaEventDestroy(e);
  if (a->copy_ev) cudaEventDestroy(a->copy_ev);
  if (prev_dev >= 0) cudaSetDevice(prev_dev);
  delete a;
}

vca_status harvest_front(vca_analyzer* a, bool blocking) {
  const auto p = a->pending.front();
  if (blocking) {
    VCA_CUDA(cudaEventSynchronize(a->ring_ev[p.slot]), "waiting for frame features");
  } else {
    cudaError_t q = cudaEventQuery(a->ring_ev[p.slot]);
    if (q == cudaErrorNotReady) return fail(VCA_E_AGAIN, "frame features not ready yet");
    if (q != cudaSuccess) return cuda_fail(q, "querying frame features");
  }
  if (p.timed) {
    float ms = 0.0f;
    VCA_CUDA(cudaEventElapsedTime(&ms, a->t0_ev[p.slot], a->t1_ev[p.slot]), "reading kernel timing");
    a->kernel_ms += ms;
    a->timed_pushes += 1;
  }
  if (a->h_err[p.slot] != 0) {
    a->pending.pop_front();
    return fail(VCA_E_TIMEOUT, "analysis kernel gave up on a bounded wait (code %d); frames %lld..%lld are lost",
                a->h_err[p.slot], (long long)p.first, (long long)(p.first + p.n - 1));
  }
  const double* base = a->h_ring + (size_t)p.slot * a->max_batch * vca::FEAT_STRIDE;
  for (int i = 0; i < p.n; ++i) {
    const double* f = base + (size_t)i * vca::FEAT_STRIDE;
    vca_frame_features ff;
    ff.frame = p.first + i;
    ff.E_Y = f[0];
    ff.h = f[1];
    ff.L_Y = f[2];
    ff.E_U = f[3];
    ff.E_V = f[4];
    ff.L_U = f[5];
    ff.L_V = f[6];
    a->done.push_back(ff);
    const double v[7] = {ff.E_Y, ff.h, ff.L_Y, ff.E_U, ff.E_V, ff.L_U, ff.L_V};
    for (int j = 0; j < 7; ++j) a->seq_sum[j] += v[j];
    a->seq_n += 1;
    if (i > 0 || p.first_has_prev) a->seq_nh += 1;
  }
  a->pending.pop_front();
  return VCA_OK;
}

vca_status harvest_all(vca_analyzer* a) {
  while (!a->pending.empty()) {
    vca_status s = harvest_front(a, true);
    if (s != VCA_OK) return s;
  }
  return VCA_OK;
}

vca_status check_planes(const vca_analyzer* a, const void* y, const void* u, const void* v, int64_t pitch_y,
                        int64_t pitch_uv) {
  const Geometry& g = a->g;
  if (!y || !u || !v) return fail(VCA_E_ARG, "plane pointer is NULL");
  if (!aligned16(y) || !aligned16(u) || !aligned16(v)) return fail(VCA_E_ARG, "plane pointers must be 16-byte aligned");
  if (pitch_y < (int64_t)g.W * g.bps || pitch_uv < (int64_t)g.cw * g.bps)
    return fail(VCA_E_ARG, "pitch smaller than a row (pitch_y %lld, pitch_uv %lld)", (long long)pitch_y,
                (long long)pitch_uv);
  if ((pitch_y & 15) || (pitch_uv & 15)) return fail(VCA_E_ARG, "pitches must be multiples of 16 bytes");
  return VCA_OK;
}

// Copies n host frames into the staging buffer (allocating it on first use) and points fp at it.
vca_status stage_host_frames(vca_analyzer* a, FramePlanes* fp, int n) {
  const Geometry& g = a->g;
  const size_t py = round_up((size_t)g.W * g.bps, 64), pc = round_up((size_t)g.cw * g.bps, 64);
  const size_t ybytes = round_up(py * g.H, 256), cbytes = round_up(pc * g.ch, 256);
  const size_t fbytes = ybytes + 2 * cbytes;
  const size_t need = fbytes * (size_t)n;
  if (need > a->staging_bytes) {
    VCA_CUDA(cudaStreamSynchronize(a->stream), "sync before staging growth");
    cudaFree(a->d_staging);
    a->d_staging = nullptr;
    a->staging_bytes = 0;
    VCA_CUDA(cudaMalloc(&a->d_staging, need), "allocating staging buffer");
    a->staging_bytes = need;
  }
  for (int i = 0; i < n; ++i) {
    uint8_t* dst = a->d_staging + fbytes * i;
    VCA_CUDA(cudaMemcpy2DAsync(dst, py, fp->y + fp->fstride_y * i, fp->pitch_y, (size_t)g.W * g.bps, g.H,
                               cudaMemcpyHostToDevice, a->stream), "copying Y plane");
    VCA_CUDA(cudaMemcpy2DAsync(dst + ybytes, pc, fp->u + fp->fstride_uv * i, fp->pitch_uv, (size_t)g.cw * g.bps,
                               g.ch, cudaMemcpyHostToDevice, a->stream), "copying U plane");
    VCA_CUDA(cudaMemcpy2DAsync(dst + ybytes + cbytes, pc, fp->v + fp->fstride_uv * i, fp->pitch_uv,
                               (size_t)g.cw * g.bps, g.ch, cudaMemcpyHostToDevice, a->stream), "copying V plane");
  }
  fp->y = a->d_staging;
  fp->u = a->d_staging + ybytes;
  fp->v = a->d_staging + ybytes + cbytes;
  fp->pitch_y = (int64_t)py;
  fp->pitch_uv = (int64_t)pc;
  fp->fstride_y = fp->fstride_uv = (int64_t)fbytes;
  return VCA_OK;
}

cudaError_t run_analysis(vca_analyzer* a, const FramePlanes& fp, int n, float* blockvals, int16_t* const zdump[3]) {
  if (a->kernel == VCA_KERNEL_TC)
    return vca::launch_tc(a->g, fp, n, a->tables, blockvals, zdump, a->d_err, a->stream, &a->launches);
  return vca::launch_plain(a->g, fp, n, a->tables, blockvals, zdump, a->stream, &a->launches);
}

}  // namespace

extern "C" {

vca_status vca_block_count(const vca_config* cfg, int64_t* blocks_x, int64_t* blocks_y) {
  Geometry g{};
  vca_status s = check_config(cfg, &g);
  if (s != VCA_OK) return s;
  if (blocks_x) *blocks_x = g.nbx;
  if (blocks_y) *blocks_y = g.nby;
  return VCA_OK;
}

vca_status vca_open(const vca_config* cfg, void* cuda_stream, vca_analyzer** out) {
  if (!out) return fail(VCA_E_ARG, "out is NULL");
  *out = nullptr;
  Geometry g{};
  vca_status s = check_config(cfg, &g);
  if (s != VCA_OK) return s;
  int kernel = cfg->kernel;
  if (kernel == VCA_KERNEL_AUTO) kernel = vca::tc_supported(g) ? VCA_KERNEL_TC : VCA_KERNEL_PLAIN;
  if (kernel == VCA_KERNEL_TC && !vca::tc_supported(g))
    return fail(VCA_E_UNSUPPORTED, "the tensor-core kernel does not support this configuration");

  vca_analyzer* a = new (std::nothrow) vca_analyzer();
  if (!a) return fail(VCA_E_NOMEM, "host allocation failed");
  a->cfg = *cfg;
  a->g = g;
  a->kernel = kernel;
  a->stream = (cudaStream_t)cuda_stream;
  a->max_batch = cfg->max_batch > 0 ? cfg->max_batch : kDefaultBatch;
  cudaError_t e = cudaGetDevice(&a->device);
  if (e != cudaSuccess) {
    destroy(a);
    return cuda_fail(e, "cudaGetDevice");
  }

#define OPEN_CUDA(call, what)  \
  do {                         \
    cudaError_t e2 = (call);   \
    if (e2 != cudaSuccess) {   \
      vca_status st = cuda_fail(e2, what); \
      destroy(a);              \
      return st;               \
    }                          \
  } while (0)

  // Tables: M_y | M_c | W_y | W_c, each 256-byte aligned.
  const int w = g.w, nc = g.nc;
  const size_t oMc = round_up((size_t)w * w, 256);
  const size_t oWy = oMc + round_up((size_t)nc * nc, 256);
  const size_t oWc = oWy + round_up((size_t)w * w * 4, 256);
  const size_t tbytes = oWc + round_up((size_t)nc * nc * 4, 256);
  std::vector<uint8_t> host(tbytes, 0);
  vca::make_dct_matrix(w, reinterpret_cast<int8_t*>(host.data()));
  vca::make_dct_matrix(nc, reinterpret_cast<int8_t*>(host.data() + oMc));
  vca::make_energy_weights(w, reinterpret_cast<float*>(host.data() + oWy));
  vca::make_energy_weights(nc, reinterpret_cast<float*>(host.data() + oWc));
  OPEN_CUDA(cudaMalloc(&a->d_tables, tbytes), "allocating tables");
  OPEN_CUDA(cudaMemcpy(a->d_tables, host.data(), tbytes, cudaMemcpyHostToDevice), "uploading tables");
  uint8_t* tb = static_cast<uint8_t*>(a->d_tables);
  a->tables.M_y = reinterpret_cast<const int8_t*>(tb);
  a->tables.M_c = reinterpret_cast<const int8_t*>(tb + oMc);
  a->tables.W_y = reinterpret_cast<const float*>(tb + oWy);
  a->tables.W_c = reinterpret_cast<const float*>(tb + oWc);

  const size_t bv = (size_t)(a->max_batch + 1) * vca::N_ROWS * g.C * sizeof(float);
  OPEN_CUDA(cudaMalloc(&a->d_blockvals, bv), "allocating block values");
  OPEN_CUDA(cudaMemset(a->d_blockvals, 0, bv), "clearing block values");
  for (int i = 0; i < 2; ++i) {
    OPEN_CUDA(cudaMalloc(&a->d_prevH[i], (size_t)g.C * sizeof(float)), "allocating h state");
    OPEN_CUDA(cudaMemset(a->d_prevH[i], 0, (size_t)g.C * sizeof(float)), "clearing h state");
  }
  OPEN_CUDA(cudaMalloc(&a->d_feats, (size_t)a->max_batch * vca::FEAT_STRIDE * sizeof(double)), "allocating features");
  OPEN_CUDA(cudaMalloc(&a->d_red_partials, vca::reduce_partials_bytes(a->max_batch)), "allocating reduction scratch");
  OPEN_CUDA(cudaMalloc(&a->d_red_counters, (size_t)a->max_batch * sizeof(unsigned int)), "allocating counters");
  OPEN_CUDA(cudaMemset(a->d_red_counters, 0, (size_t)a->max_batch * sizeof(unsigned int)), "clearing counters");
  OPEN_CUDA(cudaMalloc(&a->d_err, sizeof(int)), "allocating the error flag");
  OPEN_CUDA(cudaMemset(a->d_err, 0, sizeof(int)), "clearing the error flag");
  OPEN_CUDA(cudaMallocHost(&a->h_err, kRing * sizeof(int)), "allocating pinned error flags");
  memset(a->h_err, 0, kRing * sizeof(int));
  OPEN_CUDA(cudaMallocHost(&a->h_ring, (size_t)kRing * a->max_batch * vca::FEAT_STRIDE * sizeof(double)),
            "allocating pinned feature ring");
  for (auto& ev : a->ring_ev) OPEN_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "creating events");
  for (auto& ev : a->t0_ev) OPEN_CUDA(cudaEventCreate(&ev), "creating timing events");
  for (auto& ev : a->t1_ev) OPEN_CUDA(cudaEventCreate(&ev), "creating timing events");
  OPEN_CUDA(cudaEventCreateWithFlags(&a->copy_ev, cudaEventDisableTiming), "creating events");
#undef OPEN_CUDA
  *out = a;
  return VCA_OK;
}

vca_status vca_push_frames(vca_analyzer* a, const void* y, const void* u, const void* v, int64_t pitch_y,
                           int64_t pitch_uv, int64_t frame_stride_y, int64_t frame_stride_uv, int32_t n_frames,
                           int32_t on_device) {
  if (!a) return fail(VCA_E_ARG, "analyzer is NULL");
  if (n_frames < 1 || n_frames > a->max_batch)
    return fail(VCA_E_ARG, "n_frames must be in [1, %d] (got %d)", a->max_batch, n_frames);
  vca_status s = check_planes(a, y, u, v, pitch_y, pitch_uv);
  if (s != VCA_OK) return s;
  if (n_frames > 1 && ((frame_stride_y & 15) || (frame_stride_uv & 15) || frame_stride_y <= 0 || frame_stride_uv <= 0))
    return fail(VCA_E_ARG, "frame strides must be positive multiples of 16 bytes");
  if (n_frames > 1 && (frame_stride_y < pitch_y * a->g.H || frame_stride_uv < pitch_uv * a->g.ch))
    return fail(VCA_E_ARG, "frame strides must not be smaller than one plane (frames may not overlap)");
  if (on_device != 0 && on_device != 1) return fail(VCA_E_ARG, "on_device must be 0 or 1");

  FramePlanes fp{static_cast<const uint8_t*>(y), static_cast<const uint8_t*>(u), static_cast<const uint8_t*>(v),
                 pitch_y, pitch_uv, frame_stride_y, frame_stride_uv};
  if (!on_device) {
    s = stage_host_frames(a, &fp, n_frames);
    if (s != VCA_OK) return s;
    VCA_CUDA(cudaEventRecord(a->copy_ev, a->stream), "recording copy event");
  }
  if ((int)a->pending.size() == kRing) {
    s = harvest_front(a, true);
    if (s != VCA_OK) return s;
  }
  const int slot = a->next_slot;
  const bool timed = a->timing;
  VCA_CUDA(cudaMemsetAsync(a->d_err, 0, sizeof(int), a->stream), "clearing the error flag");
  if (timed) VCA_CUDA(cudaEventRecord(a->t0_ev[slot], a->stream), "recording timing event");
  cudaError_t e = run_analysis(a, fp, n_frames, a->d_blockvals, nullptr);
  if (e != cudaSuccess) return cuda_fail(e, "launching the analysis kernel");
  if (timed) VCA_CUDA(cudaEventRecord(a->t1_ev[slot], a->stream), "recording timing event");
  e = vca::launch_reduce(a->g, n_frames, a->d_blockvals, a->d_prevH[a->cur_prev], a->has_prev,
                         a->d_prevH[a->cur_prev ^ 1], a->d_feats, a->d_red_partials, a->d_red_counters, a->stream,
                         &a->launches);
  if (e != cudaSuccess) return cuda_fail(e, "launching the frame reduction");
  VCA_CUDA(cudaMemcpyAsync(a->h_ring + (size_t)slot * a->max_batch * vca::FEAT_STRIDE, a->d_feats,
                           (size_t)n_frames * vca::FEAT_STRIDE * sizeof(double), cudaMemcpyDeviceToHost, a->stream),
           "copying features to the host");
  VCA_CUDA(cudaMemcpyAsync(a->h_err + slot, a->d_err, sizeof(int), cudaMemcpyDeviceToHost, a->stream),
           "copying the error flag");
  VCA_CUDA(cudaEventRecord(a->ring_ev[slot], a->stream), "recording feature event");
  a->pending.push_back({a->frames_pushed, n_frames, slot, a->has_prev != 0, timed});
  a->next_slot = (slot + 1) % kRing;
  a->cur_prev ^= 1;
  a->has_prev = 1;
  a->frames_pushed += n_frames;
  a->last_n = n_frames;
  if (!on_device) VCA_CUDA(cudaEventSynchronize(a->copy_ev), "waiting for host frame copies");
  return VCA_OK;
}

vca_status vca_push_frame(vca_analyzer* a, const void* y, const void* u, const void* v, int64_t pitch_y,
                          int64_t pitch_uv, int32_t on_device) {
  return vca_push_frames(a, y, u, v, pitch_y, pitch_uv, 0, 0, 1, on_device);
}

vca_status vca_read_frame_features(vca_analyzer* a, int64_t frame, int32_t blocking, vca_frame_features* out) {
  if (!a || !out) return fail(VCA_E_ARG, "NULL argument");
  if (frame < a->done_base || frame >= a->frames_pushed)
    return fail(VCA_E_ARG, "frame %lld is not available (pushed %lld)", (long long)frame, (long long)a->frames_pushed);
  while (frame >= a->done_base + (int64_t)a->done.size()) {
    vca_status s = harvest_front(a, blocking != 0);
    if (s != VCA_OK) return s;
  }
  *out = a->done[(size_t)(frame - a->done_base)];
  return VCA_OK;
}

vca_status vca_read_sequence_features(vca_analyzer* a, vca_sequence_features* out) {
  if (!a || !out) return fail(VCA_E_ARG, "NULL argument");
  vca_status s = harvest_all(a);
  if (s != VCA_OK) return s;
  out->frames = a->seq_n;
  const double n = a->seq_n > 0 ? (double)a->seq_n : 1.0;
  out->E_Y = a->seq_sum[0] / n;
  out->h = a->seq_nh > 0 ? a->seq_sum[1] / (double)a->seq_nh : 0.0;
  out->L_Y = a->seq_sum[2] / n;
  out->E_U = a->seq_sum[3] / n;
  out->E_V = a->seq_sum[4] / n;
  out->L_U = a->seq_sum[5] / n;
  out->L_V = a->seq_sum[6] / n;
  return VCA_OK;
}

vca_status vca_read_block_values(vca_analyzer* a, int32_t index, float* H_Y, float* L_Y, float* H_U, float* L_U,
                                 float* H_V, float* L_V) {
  if (!a) return fail(VCA_E_ARG, "analyzer is NULL");
  if (a->last_n == 0 || index < 0 || index >= a->last_n)
    return fail(VCA_E_ARG, "index %d outside the last push (%d frames)", index, a->last_n);
  VCA_CUDA(cudaStreamSynchronize(a->stream), "waiting for block values");
  float* const dst[6] = {H_Y, L_Y, H_U, L_U, H_V, L_V};
  const float* src = a->d_blockvals + (size_t)index * vca::N_ROWS * a->g.C;
  for (int r = 0; r < 6; ++r) {
    if (!dst[r]) continue;
    VCA_CUDA(cudaMemcpy(dst[r], src + (size_t)r * a->g.C, (size_t)a->g.C * sizeof(float), cudaMemcpyDeviceToHost),
             "copying block values");
  }
  return VCA_OK;
}

vca_status vca_dump_coefficients(vca_analyzer* a, const void* y, const void* u, const void* v, int64_t pitch_y,
                                 int64_t pitch_uv, int16_t* zy, int16_t* zu, int16_t* zv) {
  if (!a) return fail(VCA_E_ARG, "analyzer is NULL");
  vca_status s = check_planes(a, y, u, v, pitch_y, pitch_uv);
  if (s != VCA_OK) return s;
  if (!zy || !zu || !zv) return fail(VCA_E_ARG, "coefficient buffer is NULL");
  FramePlanes fp{static_cast<const uint8_t*>(y), static_cast<const uint8_t*>(u), static_cast<const uint8_t*>(v),
                 pitch_y, pitch_uv, 0, 0};
  int16_t* const z[3] = {zy, zu, zv};
  float* scratch = a->d_blockvals + (size_t)a->max_batch * vca::N_ROWS * a->g.C;
  cudaError_t e = run_analysis(a, fp, 1, scratch, z);
  if (e != cudaSuccess) return cuda_fail(e, "launching the coefficient dump");
  return VCA_OK;
}

vca_status vca_sync(vca_analyzer* a) {
  if (!a) return fail(VCA_E_ARG, "analyzer is NULL");
  VCA_CUDA(cudaStreamSynchronize(a->stream), "synchronising the analyzer stream");
  return VCA_OK;
}

vca_status vca_export_state(vca_analyzer* a, void* buf, size_t* len) {
  if (!a || !len) return fail(VCA_E_ARG, "NULL argument");
  const size_t need = sizeof(StateHeader) + (size_t)a->g.C * sizeof(float);
  if (!buf) {
    *len = need;
    return VCA_OK;
  }
  if (*len < need) return fail(VCA_E_ARG, "state buffer too small (%zu < %zu)", *len, need);
  vca_status s = harvest_all(a);
  if (s != VCA_OK) return s;
  VCA_CUDA(cudaStreamSynchronize(a->stream), "waiting before state export");
  StateHeader h{};
  memcpy(h.magic, kStateMagic, 8);
  h.C = a->g.C;
  h.frames = a->frames_pushed;
  h.has_prev = a->has_prev;
  h.block_size = a->g.w;
  for (int j = 0; j < 7; ++j) h.seq_sum[j] = a->seq_sum[j];
  h.seq_n = a->seq_n;
  h.seq_nh = a->seq_nh;
  memcpy(buf, &h, sizeof h);
  VCA_CUDA(cudaMemcpy(static_cast<uint8_t*>(buf) + sizeof h, a->d_prevH[a->cur_prev], (size_t)a->g.C * sizeof(float),
                      cudaMemcpyDeviceToHost), "copying h state");
  *len = need;
  return VCA_OK;
}

vca_status vca_import_state(vca_analyzer* a, const void* buf, size_t len) {
  if (!a || !buf) return fail(VCA_E_ARG, "NULL argument");
  if (len < sizeof(StateHeader)) return fail(VCA_E_ARG, "state buffer too small");
  StateHeader h;
  memcpy(&h, buf, sizeof h);
  if (memcmp(h.magic, kStateMagic, 8) != 0) return fail(VCA_E_ARG, "not an analyzer state buffer");
  if (h.C != a->g.C || h.block_size != a->g.w) return fail(VCA_E_ARG, "state belongs to another block grid");
  if (len < sizeof h + (size_t)h.C * sizeof(float) || h.frames < 0) return fail(VCA_E_ARG, "truncated state buffer");
  vca_status s = harvest_all(a);
  if (s != VCA_OK) return s;
  VCA_CUDA(cudaStreamSynchronize(a->stream), "waiting before state import");
  VCA_CUDA(cudaMemcpy(a->d_prevH[a->cur_prev], static_cast<const uint8_t*>(buf) + sizeof h,
                      (size_t)h.C * sizeof(float), cudaMemcpyHostToDevice), "restoring h state");
  a->has_prev = h.has_prev != 0;
  a->frames_pushed = h.frames;
  a->done.clear();
  a->done_base = h.frames;
  a->last_n = 0;
  for (int j = 0; j < 7; ++j) a->seq_sum[j] = h.seq_sum[j];
  a->seq_n = h.seq_n;
  a->seq_nh = h.seq_nh;
  return VCA_OK;
}

vca_status vca_frames_pushed(vca_analyzer* a, int64_t* frames) {
  if (!a || !frames) return fail(VCA_E_ARG, "NULL argument");
  *frames = a->frames_pushed;
  return VCA_OK;
}

vca_status vca_launch_count(vca_analyzer* a, int64_t* launches) {
  if (!a || !launches) return fail(VCA_E_ARG, "NULL argument");
  *launches = a->launches;
  return VCA_OK;
}

vca_status vca_set_kernel_timing(vca_analyzer* a, int32_t enable) {
  if (!a) return fail(VCA_E_ARG, "analyzer is NULL");
  a->timing = enable != 0;
  return VCA_OK;
}

vca_status vca_read_kernel_timing(vca_analyzer* a, double* total_ms, int64_t* timed_pushes) {
  if (!a || !total_ms || !timed_pushes) return fail(VCA_E_ARG, "NULL argument");
  vca_status s = harvest_all(a);
  if (s != VCA_OK) return s;
  *total_ms = a->kernel_ms;
  *timed_pushes = a->timed_pushes;
  return VCA_OK;
}

vca_status vca_kernel_in_use(vca_analyzer* a, int32_t* kernel) {
  if (!a || !kernel) return fail(VCA_E_ARG, "NULL argument");
  *kernel = a->kernel;
  return VCA_OK;
}

vca_status vca_close(vca_analyzer* a) {
  destroy(a);
  return VCA_OK;
}

const char* vca_status_str(vca_status s) {
  switch (s) {
    case VCA_OK: return "ok";
    case VCA_E_ARG: return "invalid argument";
    case VCA_E_UNSUPPORTED: return "unsupported configuration";
    case VCA_E_NOMEM: return "out of memory";
    case VCA_E_CUDA: return "CUDA error";
    case VCA_E_AGAIN: return "not ready";
    case VCA_E_TIMEOUT: return "device wait timed out";
    case VCA_E_STATE: return "invalid state";
  }
  return "unknown status";
}

const char* vca_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
