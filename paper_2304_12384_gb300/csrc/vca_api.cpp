// Host runtime behind include/vca.h: configuration checks, device state, launch
// sequencing, the pinned result ring and the cross-frame (h) state.
//
// Per push: analysis kernel(s) write per-block H and L for every frame of the batch,
// the FP64 reduction kernel turns them into the seven features (Section 2 of the
// paper) and updates the previous-frame luma energies, and one device-to-host copy
// moves the features into a pinned ring slot whose event tells readers when it landed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
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
  vca_batch* batch = nullptr;  // the batch this analyzer belongs to, if any
  vca_config cfg{};
  Geometry g{};    // geometry the analysis runs on (the halved planes under the downsample reading)
  Geometry gin{};  // geometry of the pushed frames
  uint8_t* d_down = nullptr;     // halved planes of up to max_batch frames (downsample reading)
  size_t down_fbytes = 0;        // bytes per frame in d_down: Y | U | V
  int64_t down_pitch_y = 0, down_pitch_uv = 0;
  size_t down_off_u = 0, down_off_v = 0;
  int kernel = VCA_KERNEL_PLAIN;
  int plain_warps = 4;   // CTA size of the CUDA-core form (launch-shape table or 4)
  int tc_ctas = 0;       // CTAs of a tensor-core launch (0: one per SM)
  long long dbg_wait_ns = 0;  // failure-path test hook (vca_debug_wait): wait limit of the kernel
  int dbg_withhold = -1;      // and the tile of the next push whose copies are withheld
  int device = 0;
  cudaStream_t stream = nullptr;
  int max_batch = kDefaultBatch;

  void* d_tables = nullptr;
  DeviceTables tables{};
  int8_t M_host[2][32 * 32] = {};  // host copies of the luma and chroma matrices (N = g.w, g.nc)
  float* d_blockvals = nullptr;  // 2 x max_batch + 1 frames of [6][C]: two push buffers, then a dump slot
  float* last_bv = nullptr;      // block values of the most recent push
  int bv_slot = 0;               // push buffer of the next push
  cudaStream_t side = nullptr;   // reduction and feature read-back, overlapping the next analysis
  cudaEvent_t an_done[2] = {nullptr, nullptr};   // analysis of the push in buffer b finished
  cudaEvent_t red_done[2] = {nullptr, nullptr};  // reduction that read buffer b finished
  bool red_recorded[2] = {false, false};
  float* d_prevH[2] = {nullptr, nullptr};
  int cur_prev = 0;
  int* d_err = nullptr;          // kernel wait-timeout flags: one per push buffer, one for dumps
  unsigned long long* d_red_partials = nullptr;  // frame-reduction scratch
  unsigned int* d_red_counters = nullptr; // one arrival counter per frame, kept at zero between launches
  uint8_t* d_staging = nullptr;  // host frames are copied here
  size_t staging_bytes = 0;

  double* h_ring = nullptr;      // pinned and mapped, kRing slots of max_batch * FEAT_STRIDE
  double* h_ring_dev = nullptr;  // the device's view of h_ring (the reduction writes there)
  int* h_err = nullptr;          // pinned and mapped, one timeout flag per ring slot
  int* h_err_dev = nullptr;      // the device's view of h_err
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

// A batch of analyzers ticked together: one frame each per tick, analysed by the batched
// tensor-core kernel (every member on the tensor-core kernel: one launch per sample size and
// chunk of up to tc_batch_max_members() members) or by one launch of the batched plain kernel,
// then the batched reduction, replayed from a CUDA graph.  A tensor-core batch passes every
// per-tick argument as kernel parameters, replaced in the graph's kernel nodes each tick (the
// analysis launches' member tables and tensor maps, the reduction's arguments), and its reduction
// writes the features (and the analysis timeout flag beside them) straight into mapped pinned
// host memory, so its graph is the analysis launches and the reductions, nothing else; it is
// built node by node.  A plain batch's per-tick arguments
// live in pinned host memory that a copy node of the graph uploads, and a copy node reads the
// features back.  Two graphs alternate so that a tick's arguments and results can be in use
// while the previous tick runs.
struct vca_batch {
  std::vector<vca_analyzer*> m;
  int n = 0;
  int device = 0;
  int w = 32;
  int nc = 16;
  int ncv = 16;
  bool low_pass = false;
  bool tc = false;                 // analysis on the tensor-core kernel
  // Tensor-core launches: one per sample size (8-bit samples in bytes, 10-bit in 16-bit words)
  // and chunk of up to tc_batch_max_members() members.  The sample sizes are two branches of the
  // graph that run side by side on a split of the SMs, each branch's chunks one after another.
  struct TcLaunch {
    int bps = 1;
    int branch = 0;
    std::vector<uint8_t> params;            // the launch's parameter block (member table, tensor maps)
    std::vector<vca::TcBatchFrame> frames;  // this tick's frames of its members
    cudaGraphNode_t node[2] = {};           // its node in each graph
  };
  std::vector<TcLaunch> tcl;
  std::vector<int> tcl_of;  // per member: its launch
  int branches = 1;
  int branch_bps[2] = {1, 2};
  float w16 = 1.15f;  // a tile of 16-bit words against a byte tile, when the SMs are split
  long long dbg_wait_ns = 0;  // failure-path test hook (vca_batch_debug_wait)
  int dbg_withhold = -1;
  int sms = 1;                     // SMs of the device: the CTAs of a tick's tensor-core launches
  cudaStream_t stream = nullptr;
  vca::BatchCta* d_map = nullptr;
  int n_cta = 0;
  size_t ma_bytes = 0, desc_bytes = 0;
  uint8_t* d_desc = nullptr;       // CUDA-core batches: BatchMemberArgs[n] | ReduceArgs[n]
  uint8_t* h_desc[2] = {nullptr, nullptr};
  int* d_err = nullptr;            // the tensor-core kernel's wait-timeout flag
  int* h_err = nullptr;            // pinned, one per graph
  // Tensor-core batches: the frame reduction runs inside the analysis launches; per member its
  // table entry (device), and per tick graph its accumulators and tile count (zero between ticks).
  vca::TcRedMember* d_red = nullptr;
  unsigned long long* d_red_acc = nullptr;  // [2][n][kRedSums][2]
  unsigned int* d_red_done = nullptr;       // [2][n]
  std::vector<vca::TcMapCache*> tc_maps;  // per member: tensor maps of its recent frames
  double* d_feats = nullptr;       // CUDA-core batches: n x FEAT_STRIDE
  double* h_feats[2] = {nullptr, nullptr};  // pinned, per graph (tensor-core batches: mapped, + flag row)
  double* h_feats_dev[2] = {nullptr, nullptr};  // the device's view of h_feats (tensor-core batches)
  unsigned long long* d_partials = nullptr;  // CUDA-core batches: the reduction's scratch
  int red_slices = 1;              // slices per frame of the batched reduction
  unsigned int* d_counters = nullptr;
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  struct Member {
    int index;
    int64_t frame;
    bool has_prev;
  };
  struct Tick {
    int k;
    std::vector<Member> members;
  };
  std::deque<Tick> pending;
  int next_k = 0;
  int64_t ticks = 0;
  int64_t launches = 0;
};

namespace {

vca_status check_config(const vca_config* c, Geometry* g, Geometry* gin = nullptr) {
  if (!c) return fail(VCA_E_ARG, "config is NULL");
  if (c->width < 2 || c->height < 2 || (c->width & 1) || (c->height & 1) || c->width > 16384 ||
      c->height > 16384)
    return fail(VCA_E_ARG, "width/height must be even and in [2, 16384] (got %d x %d)", c->width, c->height);
  if (c->bit_depth != 8 && c->bit_depth != 10 && c->bit_depth != 12)
    return fail(VCA_E_ARG, "bit_depth must be 8, 10 or 12");
  if (c->block_size != 8 && c->block_size != 16 && c->block_size != 32)
    return fail(VCA_E_ARG, "block_size must be 8, 16 or 32");
  if (c->chroma_format != VCA_CHROMA_420 && c->chroma_format != VCA_CHROMA_444 &&
      c->chroma_format != VCA_CHROMA_422)
    return fail(VCA_E_ARG, "chroma_format must be VCA_CHROMA_420, VCA_CHROMA_444 or VCA_CHROMA_422");
  if (c->low_pass < VCA_LOWPASS_OFF || c->low_pass > VCA_LOWPASS_DOWNSAMPLE)
    return fail(VCA_E_ARG, "low_pass must be 0, 1 or 2");
  if (c->low_pass == VCA_LOWPASS_DOWNSAMPLE && (c->block_size != 32 || c->chroma_format != VCA_CHROMA_420))
    return fail(VCA_E_UNSUPPORTED,
                "the downsample reading needs block_size 32 and 4:2:0 (16 x 16 / 8 x 8 blocks after halving)");
  if (c->pad_mode != VCA_PAD_REPLICATE && c->pad_mode != VCA_PAD_SKIP) return fail(VCA_E_ARG, "bad pad_mode");
  if (c->kernel < VCA_KERNEL_AUTO || c->kernel > VCA_KERNEL_TC) return fail(VCA_E_ARG, "bad kernel selector");
  if (c->max_batch < 0 || c->max_batch > kMaxBatch) return fail(VCA_E_ARG, "max_batch must be in [0, %d]", kMaxBatch);
  Geometry q{};
  q.W = c->width;
  q.H = c->height;
  const bool full_chroma = c->chroma_format == VCA_CHROMA_444;
  const bool chroma_422 = c->chroma_format == VCA_CHROMA_422;
  q.cw = full_chroma ? c->width : c->width / 2;
  q.ch = full_chroma || chroma_422 ? c->height : c->height / 2;
  q.B = c->bit_depth;
  q.bps = c->bit_depth > 8 ? 2 : 1;
  q.w = c->block_size;
  q.nc = full_chroma ? c->block_size : c->block_size / 2;
  q.ncv = chroma_422 ? c->block_size : q.nc;  // 4:2:2: w rows of w/2 samples
  if (c->pad_mode == VCA_PAD_REPLICATE) {
    q.nbx = (q.W + q.w - 1) / q.w;
    q.nby = (q.H + q.w - 1) / q.w;
  } else {
    q.nbx = q.W / q.w;
    q.nby = q.H / q.w;
  }
  q.C = (int64_t)q.nbx * q.nby;
  if (q.C <= 0) return fail(VCA_E_ARG, "frame smaller than one block with pad_mode skip");
  q.low_pass = c->low_pass == VCA_LOWPASS_QUARTER;
  vca::transform_shifts(q.w, q.B, &q.s1y, &q.s2y);
  int unused;
  vca::transform_shifts(q.nc, q.B, &q.s1c, &unused);
  vca::transform_shifts(q.ncv, q.B, &unused, &q.s2c);
  if (gin) *gin = q;
  if (c->low_pass == VCA_LOWPASS_DOWNSAMPLE) {
    // Halved planes, half-size blocks, same block grid (ceil(ceil(W/2) / (w/2)) = ceil(W/w)).
    q.W = (q.W + 1) / 2;
    q.H = (q.H + 1) / 2;
    q.cw = (q.cw + 1) / 2;
    q.ch = (q.ch + 1) / 2;
    q.w /= 2;
    q.nc /= 2;
    q.ncv /= 2;
    vca::transform_shifts(q.w, q.B, &q.s1y, &q.s2y);
    vca::transform_shifts(q.nc, q.B, &q.s1c, &q.s2c);
  }
  if (g) *g = q;
  return VCA_OK;
}

void destroy(vca_analyzer* a) {
  if (!a) return;
  int prev_dev = -1;
  cudaGetDevice(&prev_dev);
  cudaSetDevice(a->device);
  cudaStreamSynchronize(a->stream);
  if (a->side) cudaStreamSynchronize(a->side);
  cudaFree(a->d_tables);
  cudaFree(a->d_blockvals);
  cudaFree(a->d_prevH[0]);
  cudaFree(a->d_prevH[1]);
  cudaFree(a->d_err);
  cudaFree(a->d_red_partials);
  cudaFree(a->d_red_counters);
  if (a->h_err) cudaFreeHost(a->h_err);
  cudaFree(a->d_staging);
  cudaFree(a->d_down);
  if (a->h_ring) cudaFreeHost(a->h_ring);
  for (auto& e : a->ring_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : a->t0_ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : a->t1_ev)
    if (e) cudaEventDestroy(e);
  if (a->copy_ev) cudaEventDestroy(a->copy_ev);
  for (int b = 0; b < 2; ++b) {
    if (a->an_done[b]) cudaEventDestroy(a->an_done[b]);
    if (a->red_done[b]) cudaEventDestroy(a->red_done[b]);
  }
  if (a->side) cudaStreamDestroy(a->side);
  if (prev_dev >= 0) cudaSetDevice(prev_dev);
  delete a;
}

// The result list keeps one entry per pushed frame: a frame lost to a kernel wait timeout has frame
// number -1 (reading it gives VCA_E_TIMEOUT).
vca_frame_features lost_frame() {
  vca_frame_features ff{};
  ff.frame = -1;
  ff.E_Y = ff.h = ff.L_Y = ff.E_U = ff.E_V = ff.L_U = ff.L_V = std::nan("");
  return ff;
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
    a->has_prev = 0;  // the lost frames' energies are no previous-frame state: h restarts
    for (int i = 0; i < p.n; ++i) a->done.push_back(lost_frame());
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
  const Geometry& g = a->gin;
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
  const Geometry& g = a->gin;
  // Dense host planes (rows back to back, frames back to back): one copy per plane for all n
  // frames into a plane-major staging buffer with the host's pitch (190 GB/s from pinned memory
  // against 172 GB/s for a 2-D copy per plane and frame, measured at 2160p).
  const size_t ry = (size_t)g.W * g.bps, rc = (size_t)g.cw * g.bps;
  const bool dense = (size_t)fp->pitch_y == ry && (size_t)fp->pitch_uv == rc &&
                     (n == 1 || ((size_t)fp->fstride_y == ry * g.H && (size_t)fp->fstride_uv == rc * g.ch));
  if (dense) {
    const size_t yb = ry * g.H * n, cb = rc * g.ch * n;
    const size_t off_u = round_up(yb, 256), off_v = off_u + round_up(cb, 256);
    const size_t need = off_v + round_up(cb, 256);
    if (need > a->staging_bytes) {
      VCA_CUDA(cudaStreamSynchronize(a->stream), "sync before staging growth");
      cudaFree(a->d_staging);
      a->d_staging = nullptr;
      a->staging_bytes = 0;
      VCA_CUDA(cudaMalloc(&a->d_staging, need), "allocating staging buffer");
      a->staging_bytes = need;
    }
    VCA_CUDA(cudaMemcpyAsync(a->d_staging, fp->y, yb, cudaMemcpyHostToDevice, a->stream), "copying Y planes");
    VCA_CUDA(cudaMemcpyAsync(a->d_staging + off_u, fp->u, cb, cudaMemcpyHostToDevice, a->stream), "copying U planes");
    VCA_CUDA(cudaMemcpyAsync(a->d_staging + off_v, fp->v, cb, cudaMemcpyHostToDevice, a->stream), "copying V planes");
    fp->y = a->d_staging;
    fp->u = a->d_staging + off_u;
    fp->v = a->d_staging + off_v;
    fp->fstride_y = (int64_t)(ry * g.H);
    fp->fstride_uv = (int64_t)(rc * g.ch);
    return VCA_OK;
  }
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

cudaError_t run_analysis(vca_analyzer* a, const FramePlanes& fp_in, int n, float* blockvals, int16_t* const zdump[3],
                         int* err) {
  FramePlanes fp = fp_in;
  if (a->cfg.low_pass == VCA_LOWPASS_DOWNSAMPLE) {
    vca::DownArgs d{};
    const uint8_t* src[3] = {fp_in.y, fp_in.u, fp_in.v};
    const size_t off[3] = {0, a->down_off_u, a->down_off_v};
    for (int p = 0; p < 3; ++p) {
      vca::DownPlane& P = d.p[p];
      P.src = src[p];
      P.src_pitch = p == 0 ? fp_in.pitch_y : fp_in.pitch_uv;
      P.src_fstride = p == 0 ? fp_in.fstride_y : fp_in.fstride_uv;
      P.dst = a->d_down + off[p];
      P.dst_pitch = p == 0 ? a->down_pitch_y : a->down_pitch_uv;
      P.dst_fstride = (int64_t)a->down_fbytes;
      P.w = p == 0 ? a->gin.W : a->gin.cw;
      P.h = p == 0 ? a->gin.H : a->gin.ch;
      P.wd = p == 0 ? a->g.W : a->g.cw;
      P.hd = p == 0 ? a->g.H : a->g.ch;
    }
    cudaError_t e = vca::launch_downsample(d, n, a->g.bps, a->stream);
    if (e != cudaSuccess) return e;
    ++a->launches;
    fp = FramePlanes{a->d_down, a->d_down + a->down_off_u, a->d_down + a->down_off_v, a->down_pitch_y,
                     a->down_pitch_uv, (int64_t)a->down_fbytes, (int64_t)a->down_fbytes};
  }
  if (a->kernel == VCA_KERNEL_TC)
  {
    const int withhold = a->dbg_withhold;
    a->dbg_withhold = -1;  // one push only
    return vca::launch_tc(a->g, fp, n, a->tables, blockvals, zdump, err, a->stream, &a->launches, a->tc_ctas,
                          a->dbg_wait_ns, withhold);
  }
  return vca::launch_plain(a->g, fp, n, a->tables, blockvals, zdump, a->stream, &a->launches, a->plain_warps);
}


// ---- batches ----------------------------------------------------------------------------

// Delivers the features of the oldest tick in flight to its analyzers.
// Bytes of a tensor-core batch's reduction accumulators: per tick graph and member, kRedSums sums
// of two 64-bit parts.
size_t red_acc_bytes(int n) { return 2 * (size_t)n * vca::kRedSums * 2 * sizeof(unsigned long long); }

vca_status batch_harvest_front(vca_batch* b, bool blocking) {
  const vca_batch::Tick t = b->pending.front();
  if (blocking) {
    VCA_CUDA(cudaEventSynchronize(b->ev[t.k]), "waiting for a batch tick");
  } else {
    cudaError_t q = cudaEventQuery(b->ev[t.k]);
    if (q == cudaErrorNotReady) return fail(VCA_E_AGAIN, "frame features not ready yet");
    if (q != cudaSuccess) return cuda_fail(q, "querying a batch tick");
  }
  const int code = b->tc ? (int)b->h_feats[t.k][(size_t)b->n * vca::FEAT_STRIDE] : b->h_err[t.k];
  if (code != 0) {
    b->h_err[t.k] = 0;
    if (b->tc) {
      // A tick that gave up leaves some members' sums and counts behind: clear graph t.k's set
      // before that graph runs again (stream order; the other graph's set is its own).
      cudaError_t e = cudaMemsetAsync(b->d_red_acc + (size_t)t.k * b->n * vca::kRedSums * 2, 0,
                                      red_acc_bytes(b->n) / 2, b->stream);
      if (e == cudaSuccess)
        e = cudaMemsetAsync(b->d_red_done + (size_t)t.k * b->n, 0, (size_t)b->n * sizeof(unsigned int), b->stream);
      if (e != cudaSuccess) return cuda_fail(e, "clearing the reduction state of a failed tick");
    }
    b->pending.pop_front();
    for (const auto& mm : t.members) {  // as for a single analyzer
      b->m[mm.index]->has_prev = 0;
      b->m[mm.index]->done.push_back(lost_frame());
    }
    return fail(VCA_E_TIMEOUT, "batched analysis kernel gave up on a bounded wait (code %d); the tick's frames are lost",
                code);
  }
  for (const auto& mm : t.members) {
    vca_analyzer* a = b->m[mm.index];
    const double* f = b->h_feats[t.k] + (size_t)mm.index * vca::FEAT_STRIDE;
    vca_frame_features ff;
    ff.frame = mm.frame;
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
    if (mm.has_prev) a->seq_nh += 1;
  }
  b->pending.pop_front();
  return VCA_OK;
}

vca_status batch_harvest_all(vca_batch* b) {
  while (!b->pending.empty()) {
    vca_status s = batch_harvest_front(b, true);
    if (s != VCA_OK) return s;
  }
  return VCA_OK;
}

// Brings an analyzer's results up to date: its own pushes, then its batch's ticks.
vca_status catch_up_all(vca_analyzer* a) {
  vca_status s = harvest_all(a);
  if (s == VCA_OK && a->batch) s = batch_harvest_all(a->batch);
  return s;
}

void destroy_batch(vca_batch* b) {
  if (!b) return;
  int prev_dev = -1;
  cudaGetDevice(&prev_dev);
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (vca_analyzer* a : b->m)
    if (a && a->batch == b) a->batch = nullptr;
  for (int k = 0; k < 2; ++k) {
    if (b->exec[k]) cudaGraphExecDestroy(b->exec[k]);
    if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
    if (b->ev[k]) cudaEventDestroy(b->ev[k]);
    if (b->h_desc[k]) cudaFreeHost(b->h_desc[k]);
    if (b->h_feats[k]) cudaFreeHost(b->h_feats[k]);
  }
  for (vca::TcMapCache* c : b->tc_maps) vca::tc_map_cache_free(c);
  cudaFree(b->d_map);
  cudaFree(b->d_desc);
  cudaFree(b->d_err);
  if (b->h_err) cudaFreeHost(b->h_err);
  cudaFree(b->d_red);
  cudaFree(b->d_red_acc);
  cudaFree(b->d_red_done);
  cudaFree(b->d_feats);
  cudaFree(b->d_partials);
  cudaFree(b->d_counters);
  if (b->stream) cudaStreamDestroy(b->stream);
  if (prev_dev >= 0) cudaSetDevice(prev_dev);
  delete b;
}

// Bytes of a tick's features on the host: n rows, then (tensor-core batches) the row holding the
// analysis kernel's timeout flag.
size_t feats_bytes(const vca_batch* b) {
  return (size_t)(b->n + (b->tc ? 1 : 0)) * vca::FEAT_STRIDE * sizeof(double);
}

// Builds tick graph k.  Tensor-core batches: node by node -- each branch's launches one after
// another (each launch also reduces its members' frames to features).  CUDA-core batches:
// captured -- upload the arguments, analyse, reduce, read the features back.
cudaError_t build_tick_graph(vca_batch* b, int k) {
  if (b->tc) {
    cudaError_t e = cudaGraphCreate(&b->graph[k], 0);
    cudaGraphNode_t tail[2] = {nullptr, nullptr};
    for (auto& L : b->tcl) {
      if (e != cudaSuccess) return e;
      void* args[1] = {L.params.data()};
      cudaKernelNodeParams kp;
      e = vca::tc_batch_node_params(b->w, b->nc == b->w, L.bps, b->low_pass, b->sms, args, &kp);
      if (e != cudaSuccess) return e;
      const cudaGraphNode_t dep = tail[L.branch];
      e = cudaGraphAddKernelNode(&L.node[k], b->graph[k], dep ? &dep : nullptr, dep ? 1 : 0, &kp);
      tail[L.branch] = L.node[k];
    }
    if (e != cudaSuccess) return e;
    return cudaGraphInstantiate(&b->exec[k], b->graph[k], 0);
  }
  cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t e1 = cudaMemcpyAsync(b->d_desc, b->h_desc[k], b->desc_bytes, cudaMemcpyHostToDevice, b->stream);
  if (e1 == cudaSuccess)
    e1 = vca::launch_batch_plain(b->d_map, b->n_cta, reinterpret_cast<const vca::BatchMemberArgs*>(b->d_desc), b->w,
                                 b->nc, b->ncv, b->low_pass, b->stream);
  if (e1 == cudaSuccess)
    e1 = vca::launch_reduce_batch(reinterpret_cast<const vca::ReduceArgs*>(b->d_desc + b->ma_bytes), b->n,
                                  b->red_slices, b->stream);
  if (e1 == cudaSuccess)
    e1 = cudaMemcpyAsync(b->h_feats[k], b->d_feats, feats_bytes(b), cudaMemcpyDeviceToHost, b->stream);
  e = cudaStreamEndCapture(b->stream, &b->graph[k]);
  if (e1 != cudaSuccess) return e1;
  if (e != cudaSuccess) return e;
  return cudaGraphInstantiate(&b->exec[k], b->graph[k], 0);
}

// Plain-routine arguments of one frame of analyzer a: kind 0 luma, 1 both chroma planes.
vca::PlainArgs member_plain_args(const vca_analyzer* a, int kind, const vca_frame_ref& f) {
  const Geometry& g = a->g;
  vca::PlainArgs pa{};
  pa.nbx = g.nbx;
  pa.C = g.C;
  pa.out_fstride = 0;
  pa.fstride = 0;
  float* bv = a->d_blockvals;
  if (kind == 0) {
    pa.base[0] = static_cast<const uint8_t*>(f.y);
    pa.pitch = f.pitch_y;
    pa.width = g.W;
    pa.height = g.H;
    pa.s1 = g.s1y;
    pa.s2 = g.s2y;
    pa.M = a->tables.M_y;
    pa.M2 = a->tables.M_y;
    pa.W = a->tables.W_y;
    pa.outH[0] = bv + vca::ROW_H_Y * g.C;
    pa.outL[0] = bv + vca::ROW_L_Y * g.C;
  } else {
    pa.base[0] = static_cast<const uint8_t*>(f.u);
    pa.base[1] = static_cast<const uint8_t*>(f.v);
    pa.pitch = f.pitch_uv;
    pa.width = g.cw;
    pa.height = g.ch;
    pa.s1 = g.s1c;
    pa.s2 = g.s2c;
    pa.M = a->tables.M_c;
    pa.M2 = a->tables.M_cv;
    pa.W = a->tables.W_c;
    pa.outH[0] = bv + vca::ROW_H_U * g.C;
    pa.outL[0] = bv + vca::ROW_L_U * g.C;
    pa.outH[1] = bv + vca::ROW_H_V * g.C;
    pa.outL[1] = bv + vca::ROW_L_V * g.C;
  }
  return pa;
}

}  // namespace

namespace vca {
vca_status set_launch_shape(vca_analyzer* a, int plain_warps, int tc_ctas) {
  if (!a || (plain_warps != 2 && plain_warps != 4 && plain_warps != 8) || tc_ctas < 0)
    return fail(VCA_E_ARG, "launch shape: plain_warps 2, 4 or 8 and tc_ctas >= 0");
  a->plain_warps = plain_warps;
  a->tc_ctas = tc_ctas;
  return VCA_OK;
}
}  // namespace vca

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
  Geometry g{}, gin{};
  vca_status s = check_config(cfg, &g, &gin);
  if (s != VCA_OK) return s;
  int kernel = cfg->kernel;
  // The launch-shape table (vca_autotune / vca_tune_*) gives this configuration's CTA sizes and,
  // for VCA_KERNEL_AUTO, the kernel family.
  vca_tune_entry shape{};
  const bool tuned = vca::tune_lookup(*cfg, &shape);
  if (kernel == VCA_KERNEL_AUTO)
    kernel = tuned && (shape.kernel == VCA_KERNEL_PLAIN || vca::tc_supported(g))
                 ? shape.kernel
                 : (vca::tc_supported(g) ? VCA_KERNEL_TC : VCA_KERNEL_PLAIN);
  if (kernel == VCA_KERNEL_TC && !vca::tc_supported(g))
    return fail(VCA_E_UNSUPPORTED, "the tensor-core kernel does not support this configuration");

  vca_analyzer* a = new (std::nothrow) vca_analyzer();
  if (!a) return fail(VCA_E_NOMEM, "host allocation failed");
  a->cfg = *cfg;
  a->g = g;
  a->gin = gin;
  a->kernel = kernel;
  if (tuned) {
    a->plain_warps = shape.plain_warps;
    a->tc_ctas = shape.tc_ctas;
  }
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

  // Tables: M_y | M_c | W_y | W_c, each 256-byte aligned.  The chroma column matrix is M_c, or
  // M_y when the chroma blocks are w rows tall (4:2:2).
  const int w = g.w, nc = g.nc, ncv = g.ncv;
  const size_t oMc = round_up((size_t)w * w, 256);
  const size_t oWy = oMc + round_up((size_t)nc * nc, 256);
  const size_t oWc = oWy + round_up((size_t)w * w * 4, 256);
  const size_t tbytes = oWc + round_up((size_t)ncv * nc * 4, 256);
  std::vector<uint8_t> host(tbytes, 0);
  vca::make_dct_matrix(w, reinterpret_cast<int8_t*>(host.data()));
  vca::make_dct_matrix(nc, reinterpret_cast<int8_t*>(host.data() + oMc));
  vca::make_energy_weights(w, reinterpret_cast<float*>(host.data() + oWy));
  vca::make_energy_weights_rect(ncv, nc, reinterpret_cast<float*>(host.data() + oWc));
  OPEN_CUDA(cudaMalloc(&a->d_tables, tbytes), "allocating tables");
  OPEN_CUDA(cudaMemcpy(a->d_tables, host.data(), tbytes, cudaMemcpyHostToDevice), "uploading tables");
  uint8_t* tb = static_cast<uint8_t*>(a->d_tables);
  a->tables.M_y = reinterpret_cast<const int8_t*>(tb);
  a->tables.M_c = reinterpret_cast<const int8_t*>(tb + oMc);
  a->tables.M_cv = ncv == nc ? a->tables.M_c : a->tables.M_y;
  a->tables.W_y = reinterpret_cast<const float*>(tb + oWy);
  a->tables.W_c = reinterpret_cast<const float*>(tb + oWc);
  memcpy(a->M_host[0], host.data(), (size_t)w * w);
  memcpy(a->M_host[1], host.data() + oMc, (size_t)nc * nc);

  const size_t bv = (size_t)(2 * a->max_batch + 1) * vca::N_ROWS * g.C * sizeof(float);
  OPEN_CUDA(cudaMalloc(&a->d_blockvals, bv), "allocating block values");
  OPEN_CUDA(cudaMemset(a->d_blockvals, 0, bv), "clearing block values");
  for (int i = 0; i < 2; ++i) {
    OPEN_CUDA(cudaMalloc(&a->d_prevH[i], (size_t)g.C * sizeof(float)), "allocating h state");
    OPEN_CUDA(cudaMemset(a->d_prevH[i], 0, (size_t)g.C * sizeof(float)), "clearing h state");
  }
  OPEN_CUDA(cudaMalloc(&a->d_red_partials, vca::reduce_partials_bytes(a->max_batch)), "allocating reduction scratch");
  OPEN_CUDA(cudaMalloc(&a->d_red_counters, (size_t)a->max_batch * sizeof(unsigned int)), "allocating counters");
  OPEN_CUDA(cudaMemset(a->d_red_counters, 0, (size_t)a->max_batch * sizeof(unsigned int)), "clearing counters");
  a->last_bv = a->d_blockvals;
  if (cfg->low_pass == VCA_LOWPASS_DOWNSAMPLE) {
    a->down_pitch_y = (int64_t)round_up((size_t)g.W * g.bps, 256);
    a->down_pitch_uv = (int64_t)round_up((size_t)g.cw * g.bps, 256);
    a->down_off_u = round_up((size_t)a->down_pitch_y * g.H, 256);
    a->down_off_v = a->down_off_u + round_up((size_t)a->down_pitch_uv * g.ch, 256);
    a->down_fbytes = a->down_off_v + round_up((size_t)a->down_pitch_uv * g.ch, 256);
    OPEN_CUDA(cudaMalloc(&a->d_down, a->down_fbytes * a->max_batch), "allocating the downsampled frames");
  }
  OPEN_CUDA(cudaMalloc(&a->d_err, 3 * sizeof(int)), "allocating the error flags");
  OPEN_CUDA(cudaMemset(a->d_err, 0, 3 * sizeof(int)), "clearing the error flags");
  OPEN_CUDA(cudaStreamCreateWithFlags(&a->side, cudaStreamNonBlocking), "creating the reduction stream");
  for (int b = 0; b < 2; ++b) {
    OPEN_CUDA(cudaEventCreateWithFlags(&a->an_done[b], cudaEventDisableTiming), "creating events");
    OPEN_CUDA(cudaEventCreateWithFlags(&a->red_done[b], cudaEventDisableTiming), "creating events");
  }
  OPEN_CUDA(cudaHostAlloc(&a->h_err, kRing * sizeof(int), cudaHostAllocMapped), "allocating pinned error flags");
  memset(a->h_err, 0, kRing * sizeof(int));
  OPEN_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&a->h_err_dev), a->h_err, 0), "mapping error flags");
  OPEN_CUDA(cudaHostAlloc(&a->h_ring, (size_t)kRing * a->max_batch * vca::FEAT_STRIDE * sizeof(double),
                          cudaHostAllocMapped),
            "allocating pinned feature ring");
  OPEN_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&a->h_ring_dev), a->h_ring, 0), "mapping the feature ring");
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
  if (a->batch) return fail(VCA_E_STATE, "the analyzer belongs to a batch; push through vca_batch_tick");
  if (n_frames < 1 || n_frames > a->max_batch)
    return fail(VCA_E_ARG, "n_frames must be in [1, %d] (got %d)", a->max_batch, n_frames);
  vca_status s = check_planes(a, y, u, v, pitch_y, pitch_uv);
  if (s != VCA_OK) return s;
  if (n_frames > 1 && ((frame_stride_y & 15) || (frame_stride_uv & 15) || frame_stride_y <= 0 || frame_stride_uv <= 0))
    return fail(VCA_E_ARG, "frame strides must be positive multiples of 16 bytes");
  if (n_frames > 1 && (frame_stride_y < pitch_y * a->gin.H || frame_stride_uv < pitch_uv * a->gin.ch))
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
  // Analysis on the analyzer's stream into push buffer bs; the reduction on the side stream, so it
  // overlaps the next push's analysis (which uses the other buffer).  The reduction writes the
  // features and the analysis kernel's timeout flag (which it then clears) straight into the
  // mapped pinned ring slot: no copies.
  const int bs = a->bv_slot;
  float* bv = a->d_blockvals + (size_t)bs * a->max_batch * vca::N_ROWS * a->g.C;
  int* derr = a->d_err + bs;
  if (a->red_recorded[bs])
    VCA_CUDA(cudaStreamWaitEvent(a->stream, a->red_done[bs], 0), "ordering after the previous reduction");
  if (timed) VCA_CUDA(cudaEventRecord(a->t0_ev[slot], a->stream), "recording timing event");
  cudaError_t e = run_analysis(a, fp, n_frames, bv, nullptr, derr);
  if (e != cudaSuccess) return cuda_fail(e, "launching the analysis kernel");
  if (timed) VCA_CUDA(cudaEventRecord(a->t1_ev[slot], a->stream), "recording timing event");
  VCA_CUDA(cudaEventRecord(a->an_done[bs], a->stream), "recording analysis event");
  VCA_CUDA(cudaStreamWaitEvent(a->side, a->an_done[bs], 0), "ordering the reduction");
  e = vca::launch_reduce(a->g, n_frames, bv, a->d_prevH[a->cur_prev], a->has_prev, a->d_prevH[a->cur_prev ^ 1],
                         a->h_ring_dev + (size_t)slot * a->max_batch * vca::FEAT_STRIDE, a->d_red_partials,
                         a->d_red_counters, a->side, &a->launches, derr, a->h_err_dev + slot);
  if (e != cudaSuccess) return cuda_fail(e, "launching the frame reduction");
  VCA_CUDA(cudaEventRecord(a->ring_ev[slot], a->side), "recording feature event");
  VCA_CUDA(cudaEventRecord(a->red_done[bs], a->side), "recording reduction event");
  a->red_recorded[bs] = true;
  a->bv_slot = bs ^ 1;
  a->last_bv = bv;
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
    vca_status s = !a->pending.empty() ? harvest_front(a, blocking != 0)
                   : a->batch && !a->batch->pending.empty() ? batch_harvest_front(a->batch, blocking != 0)
                   : fail(VCA_E_STATE, "frame %lld has no pending work", (long long)frame);
    if (s != VCA_OK) return s;
  }
  *out = a->done[(size_t)(frame - a->done_base)];
  if (out->frame < 0) return fail(VCA_E_TIMEOUT, "frame %lld was lost to a kernel wait timeout", (long long)frame);
  return VCA_OK;
}

vca_status vca_read_sequence_features(vca_analyzer* a, vca_sequence_features* out) {
  if (!a || !out) return fail(VCA_E_ARG, "NULL argument");
  vca_status s = catch_up_all(a);
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
  VCA_CUDA(cudaStreamSynchronize(a->batch ? a->batch->stream : a->stream), "waiting for block values");
  VCA_CUDA(cudaStreamSynchronize(a->side), "waiting for block values");
  float* const dst[6] = {H_Y, L_Y, H_U, L_U, H_V, L_V};
  const float* src = a->last_bv + (size_t)index * vca::N_ROWS * a->g.C;
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
  if (a->batch) return fail(VCA_E_STATE, "the analyzer belongs to a batch");
  vca_status s = check_planes(a, y, u, v, pitch_y, pitch_uv);
  if (s != VCA_OK) return s;
  if (!zy || !zu || !zv) return fail(VCA_E_ARG, "coefficient buffer is NULL");
  FramePlanes fp{static_cast<const uint8_t*>(y), static_cast<const uint8_t*>(u), static_cast<const uint8_t*>(v),
                 pitch_y, pitch_uv, 0, 0};
  int16_t* const z[3] = {zy, zu, zv};
  float* scratch = a->d_blockvals + (size_t)2 * a->max_batch * vca::N_ROWS * a->g.C;
  cudaError_t e = run_analysis(a, fp, 1, scratch, z, a->d_err + 2);
  if (e != cudaSuccess) return cuda_fail(e, "launching the coefficient dump");
  return VCA_OK;
}

vca_status vca_stream_join(vca_analyzer* a) {
  if (!a) return fail(VCA_E_ARG, "analyzer is NULL");
  for (int b = 0; b < 2; ++b)
    if (a->red_recorded[b]) VCA_CUDA(cudaStreamWaitEvent(a->stream, a->red_done[b], 0), "joining the reduction stream");
  return VCA_OK;
}

vca_status vca_sync(vca_analyzer* a) {
  if (!a) return fail(VCA_E_ARG, "analyzer is NULL");
  VCA_CUDA(cudaStreamSynchronize(a->stream), "synchronising the analyzer stream");
  VCA_CUDA(cudaStreamSynchronize(a->side), "synchronising the reduction stream");
  if (a->batch) VCA_CUDA(cudaStreamSynchronize(a->batch->stream), "synchronising the batch stream");
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
  vca_status s = catch_up_all(a);
  if (s != VCA_OK) return s;
  VCA_CUDA(cudaStreamSynchronize(a->stream), "waiting before state export");
  VCA_CUDA(cudaStreamSynchronize(a->side), "waiting before state export");
  StateHeader h{};
  memcpy(h.magic, kStateMagic, 8);
  h.C = a->g.C;
  h.frames = a->frames_pushed;
  h.has_prev = a->has_prev;
  h.block_size = a->cfg.block_size;
  for (int j = 0; j < 7; ++j) h.seq_sum[j] = a->seq_sum[j];
  h.seq_n = a->seq_n;
  h.seq_nh = a->seq_nh;
  memcpy(buf, &h, sizeof h);
  VCA_CUDA(cudaMemcpy(static_cast<uint8_t*>(buf) + sizeof h, a->d_prevH[a->cur_prev], (size_t)a->g.C * sizeof(float),
                      cudaMemcpyDeviceToHost), "copying h state");
  *len = need;
  return VCA_OK;
}

vca_status vca_check_dct_matrix(int32_t n, int32_t bit_depth, const int8_t* matrix) {
  if (!matrix) return fail(VCA_E_ARG, "matrix is NULL");
  if (bit_depth != 8 && bit_depth != 10 && bit_depth != 12) return fail(VCA_E_ARG, "bit_depth must be 8, 10 or 12");
  char why[160];
  if (!vca::check_dct_matrix(n, bit_depth, matrix, why, sizeof why)) return fail(VCA_E_ARG, "DCT matrix rejected: %s", why);
  return VCA_OK;
}

vca_status vca_set_dct_matrix(vca_analyzer* a, int32_t n, const int8_t* matrix) {
  if (!a || !matrix) return fail(VCA_E_ARG, "NULL argument");
  if (a->batch) return fail(VCA_E_STATE, "the analyzer belongs to a batch");
  if (a->frames_pushed != 0 || !a->pending.empty())
    return fail(VCA_E_STATE, "the DCT matrix can only be set before the first push");
  if (n != a->g.w && n != a->g.nc)
    return fail(VCA_E_ARG, "matrix size %d is not a transform size of this analyzer (%d, %d)", n, a->g.w, a->g.nc);
  vca_status s = vca_check_dct_matrix(n, a->g.B, matrix);
  if (s != VCA_OK) return s;
  const size_t oMc = round_up((size_t)a->g.w * a->g.w, 256);  // the table layout of vca_open
  uint8_t* tb = static_cast<uint8_t*>(a->d_tables);
  for (int i = 0; i < 2; ++i) {
    if (n != (i == 0 ? a->g.w : a->g.nc)) continue;
    VCA_CUDA(cudaMemcpy(tb + (i == 0 ? 0 : oMc), matrix, (size_t)n * n, cudaMemcpyHostToDevice),
             "uploading the DCT matrix");
    memcpy(a->M_host[i], matrix, (size_t)n * n);
  }
  return VCA_OK;
}

vca_status vca_import_state(vca_analyzer* a, const void* buf, size_t len) {
  if (!a || !buf) return fail(VCA_E_ARG, "NULL argument");
  if (len < sizeof(StateHeader)) return fail(VCA_E_ARG, "state buffer too small");
  StateHeader h;
  memcpy(&h, buf, sizeof h);
  if (memcmp(h.magic, kStateMagic, 8) != 0) return fail(VCA_E_ARG, "not an analyzer state buffer");
  if (h.C != a->g.C || h.block_size != a->cfg.block_size) return fail(VCA_E_ARG, "state belongs to another block grid");
  if (len < sizeof h + (size_t)h.C * sizeof(float) || h.frames < 0) return fail(VCA_E_ARG, "truncated state buffer");
  if (a->batch) return fail(VCA_E_STATE, "the analyzer belongs to a batch");
  vca_status s = harvest_all(a);
  if (s != VCA_OK) return s;
  VCA_CUDA(cudaStreamSynchronize(a->stream), "waiting before state import");
  VCA_CUDA(cudaStreamSynchronize(a->side), "waiting before state import");
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
  if (a && a->batch) return fail(VCA_E_STATE, "the analyzer belongs to a batch; destroy the batch first");
  destroy(a);
  return VCA_OK;
}

vca_status vca_batch_create(vca_analyzer* const* members, int32_t n, vca_batch** out) {
  if (!out) return fail(VCA_E_ARG, "out is NULL");
  *out = nullptr;
  if (!members || n < 1 || n > 65535) return fail(VCA_E_ARG, "need 1 to 65535 analyzers (got %d)", n);
  for (int i = 0; i < n; ++i) {
    vca_analyzer* a = members[i];
    if (!a) return fail(VCA_E_ARG, "analyzer %d is NULL", i);
    if (a->batch) return fail(VCA_E_STATE, "analyzer %d already belongs to a batch", i);
    for (int j = 0; j < i; ++j)
      if (members[j] == a) return fail(VCA_E_ARG, "analyzer %d appears twice", i);
    if (a->device != members[0]->device) return fail(VCA_E_ARG, "analyzers of a batch must share one device");
    if (a->g.w != members[0]->g.w || a->g.nc != members[0]->g.nc || a->g.ncv != members[0]->g.ncv ||
        a->g.low_pass != members[0]->g.low_pass)
      return fail(VCA_E_ARG, "analyzers of a batch must share block size, chroma format and low_pass");
    if (a->cfg.low_pass == VCA_LOWPASS_DOWNSAMPLE)
      return fail(VCA_E_UNSUPPORTED, "the downsample reading is not available in batches");
  }
  vca_batch* b = new (std::nothrow) vca_batch();
  if (!b) return fail(VCA_E_NOMEM, "host allocation failed");
  b->m.assign(members, members + n);
  b->n = n;
  b->device = members[0]->device;
  b->w = members[0]->g.w;
  b->nc = members[0]->g.nc;
  b->ncv = members[0]->g.ncv;
  b->low_pass = members[0]->g.low_pass;
  b->tc = true;
  for (int i = 0; i < n; ++i) {
    const vca_analyzer* a = members[i];
    b->tc = b->tc && a->kernel == VCA_KERNEL_TC;
    // one launch reads one pair of matrices: the members must share them
    b->tc = b->tc && memcmp(a->M_host[0], members[0]->M_host[0], (size_t)a->g.w * a->g.w) == 0 &&
            memcmp(a->M_host[1], members[0]->M_host[1], (size_t)a->g.nc * a->g.nc) == 0;
  }
  bool has_bps[3] = {false, false, false};
  for (int i = 0; i < n; ++i) has_bps[members[i]->g.bps] = true;
  b->branches = has_bps[1] && has_bps[2] ? 2 : 1;
  if (b->branches == 1) b->branch_bps[0] = members[0]->g.bps;
  if (b->tc) {  // each branch's members in chunks of up to tc_batch_max_members(), in member order
    b->tcl_of.assign(n, -1);
    const int cap = vca::tc_batch_max_members();
    for (int br = 0; br < b->branches; ++br) {
      int cur = -1, count = 0;
      for (int i = 0; i < n; ++i) {
        if (members[i]->g.bps != b->branch_bps[br]) continue;
        if (cur < 0 || count == cap) {
          b->tcl.emplace_back();
          cur = (int)b->tcl.size() - 1;
          b->tcl[cur].bps = b->branch_bps[br];
          b->tcl[cur].branch = br;
          count = 0;
        }
        b->tcl_of[i] = cur;
        ++count;
      }
    }
  }
  int64_t max_C = 0;
  for (int i = 0; i < n; ++i) max_C = members[i]->g.C > max_C ? members[i]->g.C : max_C;
  b->red_slices = vca::reduce_batch_slices(max_C);
  int prev_dev = -1;
  cudaGetDevice(&prev_dev);

#define BATCH_CUDA(call, what)             \
  do {                                     \
    cudaError_t e2 = (call);               \
    if (e2 != cudaSuccess) {               \
      vca_status st = cuda_fail(e2, what); \
      destroy_batch(b);                    \
      if (prev_dev >= 0) cudaSetDevice(prev_dev); \
      return st;                           \
    }                                      \
  } while (0)

  BATCH_CUDA(cudaSetDevice(b->device), "selecting the batch device");
  for (int i = 0; i < n; ++i) {
    vca_status st = harvest_all(members[i]);
    if (st != VCA_OK) {
      destroy_batch(b);
      if (prev_dev >= 0) cudaSetDevice(prev_dev);
      return st;
    }
    BATCH_CUDA(cudaStreamSynchronize(members[i]->stream), "waiting for an analyzer's earlier work");
    BATCH_CUDA(cudaStreamSynchronize(members[i]->side), "waiting for an analyzer's earlier work");
  }
  std::vector<vca::BatchCta> map;
  for (int i = 0; i < n && !b->tc; ++i) {
    const Geometry& g = members[i]->g;
    const int64_t cl = (g.C + vca::plain_blocks_per_cta(g.w) - 1) / vca::plain_blocks_per_cta(g.w);
    const int64_t cc = (g.C + vca::plain_blocks_per_cta(g.ncv) - 1) / vca::plain_blocks_per_cta(g.ncv);
    for (int64_t c = 0; c < cl; ++c) map.push_back({(uint16_t)i, 0, 0, (uint32_t)c});
    for (int pl = 0; pl < 2; ++pl)
      for (int64_t c = 0; c < cc; ++c) map.push_back({(uint16_t)i, 1, (uint8_t)pl, (uint32_t)c});
  }
  if (map.size() > (size_t)INT32_MAX) {
    destroy_batch(b);
    return fail(VCA_E_ARG, "batch too large");
  }
  b->n_cta = (int)map.size();
  for (auto& L : b->tcl) {
    L.params.assign(vca::tc_batch_params_bytes(), 0);
    L.frames.reserve((size_t)vca::tc_batch_max_members());
  }
  b->ma_bytes = b->tc ? 0 : round_up((size_t)n * sizeof(vca::BatchMemberArgs), 256);
  b->desc_bytes = b->ma_bytes + (size_t)n * sizeof(vca::ReduceArgs);
  BATCH_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "creating the batch stream");
  if (!b->tc) {
    BATCH_CUDA(cudaMalloc(&b->d_map, map.size() * sizeof(vca::BatchCta)), "allocating the CTA map");
    BATCH_CUDA(cudaMemcpy(b->d_map, map.data(), map.size() * sizeof(vca::BatchCta), cudaMemcpyHostToDevice),
               "uploading the CTA map");
  }
  for (int br = 0; b->tc && br < b->branches; ++br)
    BATCH_CUDA(vca::tc_batch_prepare(b->w, b->nc == b->w, b->branch_bps[br], b->low_pass), "preparing the tensor-core kernel");
  BATCH_CUDA(cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->device), "querying the SM count");
  if (b->sms < 1) b->sms = 1;
  BATCH_CUDA(cudaMalloc(&b->d_err, sizeof(int)), "allocating the error flag");
  BATCH_CUDA(cudaMemset(b->d_err, 0, sizeof(int)), "clearing the error flag");
  BATCH_CUDA(cudaMallocHost(&b->h_err, 2 * sizeof(int)), "allocating pinned error flags");
  b->h_err[0] = b->h_err[1] = 0;
  for (int i = 0; b->tc && i < n; ++i) {
    b->tc_maps.push_back(vca::tc_map_cache_new());
    if (!b->tc_maps.back()) {
      destroy_batch(b);
      if (prev_dev >= 0) cudaSetDevice(prev_dev);
      return fail(VCA_E_NOMEM, "allocating tensor-map caches");
    }
  }
  if (b->tc) {
    BATCH_CUDA(cudaMalloc(&b->d_red, (size_t)n * sizeof(vca::TcRedMember)), "allocating the reduction table");
    BATCH_CUDA(cudaMalloc(&b->d_red_acc, red_acc_bytes(n)), "allocating reduction accumulators");
    BATCH_CUDA(cudaMemset(b->d_red_acc, 0, red_acc_bytes(n)), "clearing reduction accumulators");
    BATCH_CUDA(cudaMalloc(&b->d_red_done, 2 * (size_t)n * sizeof(unsigned int)), "allocating reduction counters");
    BATCH_CUDA(cudaMemset(b->d_red_done, 0, 2 * (size_t)n * sizeof(unsigned int)), "clearing reduction counters");
  } else {
    BATCH_CUDA(cudaMalloc(&b->d_desc, b->desc_bytes), "allocating tick arguments");
    BATCH_CUDA(cudaMalloc(&b->d_feats, feats_bytes(b)), "allocating features");
    BATCH_CUDA(cudaMalloc(&b->d_partials, vca::reduce_partials_bytes(n)), "allocating reduction scratch");
    BATCH_CUDA(cudaMalloc(&b->d_counters, (size_t)n * sizeof(unsigned int)), "allocating counters");
    BATCH_CUDA(cudaMemset(b->d_counters, 0, (size_t)n * sizeof(unsigned int)), "clearing counters");
  }
  for (int k = 0; k < 2; ++k) {
    if (!b->tc) {
      BATCH_CUDA(cudaMallocHost(&b->h_desc[k], b->desc_bytes), "allocating pinned tick arguments");
      memset(b->h_desc[k], 0, b->desc_bytes);
    }
    BATCH_CUDA(cudaHostAlloc(&b->h_feats[k], feats_bytes(b), b->tc ? cudaHostAllocMapped : cudaHostAllocDefault),
               "allocating pinned features");
    memset(b->h_feats[k], 0, feats_bytes(b));
    if (b->tc) {
      BATCH_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&b->h_feats_dev[k]), b->h_feats[k], 0),
                 "mapping the features");
    }
    BATCH_CUDA(cudaEventCreateWithFlags(&b->ev[k], cudaEventDisableTiming), "creating batch events");
    BATCH_CUDA(build_tick_graph(b, k), "capturing the tick graph");
  }
  if (b->tc) {
    std::vector<vca::TcRedMember> red((size_t)n);
    for (int i = 0; i < n; ++i) {
      const Geometry& g = members[i]->g;
      vca::TcRedMember& r = red[(size_t)i];
      for (int k = 0; k < 2; ++k) {
        r.acc[k] = b->d_red_acc + ((size_t)k * n + i) * vca::kRedSums * 2;
        r.done[k] = b->d_red_done + (size_t)k * n + i;
        r.prevH[k] = members[i]->d_prevH[k];
        r.feats[k] = b->h_feats_dev[k] + (size_t)i * vca::FEAT_STRIDE;
      }
      r.normY = (double)g.C * g.w * g.w;
      r.normC = (double)g.C * g.ncv * g.nc;
    }
    BATCH_CUDA(cudaMemcpy(b->d_red, red.data(), red.size() * sizeof(vca::TcRedMember), cudaMemcpyHostToDevice),
               "uploading the reduction table");
  }
#undef BATCH_CUDA
  for (int i = 0; i < n; ++i) members[i]->batch = b;
  if (prev_dev >= 0) cudaSetDevice(prev_dev);
  *out = b;
  return VCA_OK;
}

vca_status vca_batch_tick(vca_batch* b, const vca_frame_ref* frames) {
  if (!b || !frames) return fail(VCA_E_ARG, "NULL argument");
  const int k = b->next_k;
  // The pinned arguments of graph k are rewritten only after its previous tick has run.
  while (!b->pending.empty() && (b->pending.size() >= 2 || b->pending.front().k == k)) {
    vca_status s = batch_harvest_front(b, true);
    if (s != VCA_OK) return s;
  }
  for (int i = 0; i < b->n; ++i) {
    if (!frames[i].y) continue;
    vca_status s = check_planes(b->m[i], frames[i].y, frames[i].u, frames[i].v, frames[i].pitch_y, frames[i].pitch_uv);
    if (s != VCA_OK) return fail(s, "frame of analyzer %d: %s", i, vca_last_error());
  }
  auto* ma = b->tc ? nullptr : reinterpret_cast<vca::BatchMemberArgs*>(b->h_desc[k]);
  auto* ra = b->tc ? nullptr : reinterpret_cast<vca::ReduceArgs*>(b->h_desc[k] + b->ma_bytes);
  vca_batch::Tick tick;
  tick.k = k;
  for (auto& L : b->tcl) L.frames.clear();
  for (int i = 0; i < b->n; ++i) {
    vca_analyzer* a = b->m[i];
    if (!frames[i].y) {
      if (!b->tc) {
        ma[i].active = 0;
        ra[i].nframes = 0;
      }
      continue;
    }
    if (b->tc) {
      // The launch reduces the frame too: the member's table entry, whether it has a previous
      // frame and which of its buffers holds that frame's energies, and the graph's state set.
      const vca_frame_ref& f = frames[i];
      const int flags = (a->has_prev ? vca::kRedHasPrev : 0) | (a->cur_prev ? vca::kRedPrevBuf : 0) |
                        (k ? vca::kRedGraph : 0);
      b->tcl[b->tcl_of[i]].frames.push_back({&a->g,
                              {static_cast<const uint8_t*>(f.y), static_cast<const uint8_t*>(f.u),
                               static_cast<const uint8_t*>(f.v), f.pitch_y, f.pitch_uv, 0, 0},
                              a->d_blockvals, b->tc_maps[i], i, flags});
    } else {
      ma[i].pa[0] = member_plain_args(a, 0, frames[i]);
      ma[i].pa[1] = member_plain_args(a, 1, frames[i]);
      ma[i].bps = a->g.bps;
      ma[i].active = 1;
      ra[i] = vca::reduce_args(a->g, 1, a->d_blockvals, a->d_prevH[a->cur_prev], a->has_prev,
                               a->d_prevH[a->cur_prev ^ 1], b->d_feats + (size_t)i * vca::FEAT_STRIDE,
                               b->d_partials + (size_t)i * vca::reduce_partials_bytes(1) / sizeof(unsigned long long),
                               b->d_counters + i);
    }
    tick.members.push_back({i, a->frames_pushed, a->has_prev != 0});
  }
  int grid[2] = {b->sms, b->sms};
  // The tick's timeout flag, beside the features in mapped memory: the launches set it only when a
  // wait runs out (graph k's previous tick has been read).
  if (b->tc) b->h_feats[k][(size_t)b->n * vca::FEAT_STRIDE] = 0.0;
  for (size_t li = 0; li < b->tcl.size(); ++li) {
    auto& L = b->tcl[li];
    cudaError_t e = vca::tc_batch_fill(L.params.data(), L.frames.data(), (int)L.frames.size(), b->m[0]->tables,
                                       b->d_err, b->d_red, b->h_feats_dev[k] + (size_t)b->n * vca::FEAT_STRIDE,
                                       b->dbg_wait_ns, li == 0 ? b->dbg_withhold : -1);
    if (e != cudaSuccess) return cuda_fail(e, "encoding the tensor maps of a batch tick");
  }
  b->dbg_withhold = -1;  // one tick only
  if (b->tc && b->branches == 2 && b->sms >= 2) {
    // The two sample sizes' launches run side by side on disjoint SMs (a CTA holds a whole SM),
    // the SMs split in proportion to their work: a tile of 16-bit words costs about 1.15 x a tile
    // of bytes.  So the tick pays one pipeline fill and drain instead of two in sequence.  Each
    // share is even: with an odd split one SM pair held a CTA of each launch, and those two CTAs
    // ran 1.6x slower than all the others (measured), which set the tick's time.
    double w[2] = {0.0, 0.0};
    for (const auto& L : b->tcl)
      w[L.branch] += vca::tc_batch_items(L.params.data()) * (L.bps == 2 ? (double)b->w16 : 1.0);
    int g0 = w[0] + w[1] > 0.0 ? (int)std::lround(b->sms * w[0] / (w[0] + w[1])) : b->sms / 2;
    g0 = (g0 + 1) & ~1;
    const int lo = b->sms >= 4 ? 2 : 1;  // a launch with no tiles this tick still gets a (full) SM pair
    g0 = std::min(std::max(g0, lo), b->sms - lo);
    grid[0] = g0;
    grid[1] = b->sms - g0;
  }
  for (auto& L : b->tcl) {
    // The graph's launch takes this tick's parameter block (copied by the call) and its branch's grid.
    void* args[1] = {L.params.data()};
    cudaKernelNodeParams kp;
    cudaError_t e = vca::tc_batch_node_params(b->w, b->nc == b->w, L.bps, b->low_pass, grid[L.branch], args, &kp);
    if (e == cudaSuccess) e = cudaGraphExecKernelNodeSetParams(b->exec[k], L.node[k], &kp);
    if (e != cudaSuccess) return cuda_fail(e, "setting the parameters of a batch tick");
  }
  int prev_dev = -1;
  cudaGetDevice(&prev_dev);
  if (prev_dev != b->device) VCA_CUDA(cudaSetDevice(b->device), "selecting the batch device");
  cudaError_t e = cudaGraphLaunch(b->exec[k], b->stream);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev[k], b->stream);
  if (prev_dev >= 0 && prev_dev != b->device) cudaSetDevice(prev_dev);
  if (e != cudaSuccess) return cuda_fail(e, "launching a batch tick");
  for (const auto& mm : tick.members) {
    vca_analyzer* a = b->m[mm.index];
    a->cur_prev ^= 1;
    a->has_prev = 1;
    a->frames_pushed += 1;
    a->last_n = 1;
    a->last_bv = a->d_blockvals;
  }
  b->pending.push_back(std::move(tick));
  b->next_k ^= 1;
  b->ticks += 1;
  // tensor-core: one launch (analysis and reduction) per sample size and chunk; CUDA-core: analysis
  // and reduction
  b->launches += b->tc ? (int64_t)b->tcl.size() : 2;
  return VCA_OK;
}

vca_status vca_batch_sync(vca_batch* b) {
  if (!b) return fail(VCA_E_ARG, "batch is NULL");
  return batch_harvest_all(b);
}

vca_status vca_batch_kernel(vca_batch* b, int32_t* kernel) {
  if (!b || !kernel) return fail(VCA_E_ARG, "NULL argument");
  *kernel = b->tc ? VCA_KERNEL_TC : VCA_KERNEL_PLAIN;
  return VCA_OK;
}

vca_status vca_debug_wait(vca_analyzer* a, int64_t wait_limit_ns, int32_t withhold_tile) {
  if (!a || wait_limit_ns < 0 || withhold_tile < -1) return fail(VCA_E_ARG, "vca_debug_wait: bad argument");
  if (a->kernel != VCA_KERNEL_TC) return fail(VCA_E_UNSUPPORTED, "vca_debug_wait: the CUDA-core form has no waits");
  a->dbg_wait_ns = wait_limit_ns;
  a->dbg_withhold = withhold_tile;
  return VCA_OK;
}

vca_status vca_batch_debug_wait(vca_batch* b, int64_t wait_limit_ns, int32_t withhold_tile) {
  if (!b || wait_limit_ns < 0 || withhold_tile < -1) return fail(VCA_E_ARG, "vca_batch_debug_wait: bad argument");
  if (!b->tc) return fail(VCA_E_UNSUPPORTED, "vca_batch_debug_wait: the batch runs the CUDA-core form");
  b->dbg_wait_ns = wait_limit_ns;
  b->dbg_withhold = withhold_tile;
  return VCA_OK;
}

vca_status vca_batch_split_weight(vca_batch* b, float weight) {
  if (!b || !(weight >= 0.25f && weight <= 4.0f)) return fail(VCA_E_ARG, "split weight must be in [0.25, 4]");
  b->w16 = weight;
  return VCA_OK;
}

vca_status vca_batch_autotune(vca_batch* b, const vca_frame_ref* frames, int32_t reps, float* weight,
                              float* ms_per_tick) {
  if (!b || !frames || reps < 1) return fail(VCA_E_ARG, "vca_batch_autotune: needs a batch, frames and reps >= 1");
  const float cands[] = {1.0f, 1.15f, 1.3f, 1.5f, 1.75f};
  const bool split = b->tc && b->branches == 2;
  float best_w = b->w16, best_ms = -1.0f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  VCA_CUDA(cudaEventCreate(&e0), "creating tuning events");
  VCA_CUDA(cudaEventCreate(&e1), "creating tuning events");
  vca_status st = VCA_OK;
  for (float w : cands) {
    if (!split && w != cands[0]) break;  // one sample size: nothing to split, one timing
    if (split) b->w16 = w;
    for (int r = 0; st == VCA_OK && r < 2; ++r) st = vca_batch_tick(b, frames);  // warm-up
    if (st == VCA_OK) st = vca_batch_sync(b);
    if (st != VCA_OK) break;
    cudaEventRecord(e0, b->stream);
    for (int r = 0; st == VCA_OK && r < reps; ++r) st = vca_batch_tick(b, frames);
    cudaEventRecord(e1, b->stream);
    if (st == VCA_OK) st = vca_batch_sync(b);
    if (st != VCA_OK) break;
    float ms = 0.0f;
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= (float)reps;
    if (best_ms < 0.0f || ms < best_ms) {
      best_ms = ms;
      best_w = w;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != VCA_OK) return st;
  b->w16 = best_w;
  if (weight) *weight = best_w;
  if (ms_per_tick) *ms_per_tick = best_ms;
  return VCA_OK;
}

vca_status vca_batch_launch_count(vca_batch* b, int64_t* launches) {
  if (!b || !launches) return fail(VCA_E_ARG, "NULL argument");
  *launches = b->launches;
  return VCA_OK;
}

vca_status vca_batch_destroy(vca_batch* b) {
  if (!b) return VCA_OK;
  vca_status s = batch_harvest_all(b);
  destroy_batch(b);
  return s;
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
