// Serving runtime on top of the analyzer and batch API (include/vca.h): live channels submit
// segments of frames that already sit in the server's device memory, and a scheduler thread
// analyses them (Section 2 of the paper for every frame) under one of two policies:
//   segments (default): a segment whose frames have landed is one work item -- its frames go to
//     the channel's own analyzer in multi-frame pushes (one launch of the block kernel and one of
//     the reduction per push, the h chain inside the push), on the channel's own stream, so
//     channels run side by side and a segment waits for nobody's frames but its own;
//   ticks: frame-interleaved continuous batching -- every tick takes the next frame of every
//     channel that has a segment in progress and analyses them together (one batched tick), so
//     channels join and leave ticks as their segments arrive and finish.
// The h state of every channel stays on the device between segments.
//
// Admission is by device memory: a channel costs its analyzer's state plus a two-slot ring of
// segment buffers in HBM (a producer, e.g. a decoder, fills one slot while the other is being
// analysed); vca_server_add_channel refuses a channel whose cost would exceed the budget.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "vca.h"
#include "vca_internal.h"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Most frames of one push under the segments policy (longer segments take several pushes).
constexpr int kPushFrames = 128;

vca_status sfail(vca_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  vca::record_error(buf);
  return s;
}

struct Segment {
  int slot;
  int n;
  uint64_t tag;
  int64_t t_submit;
  int64_t first_frame;  // analyzer frame index of the segment's first frame
  int next = 0;         // frames queued into ticks so far
  cudaEvent_t ready = nullptr;
};

struct Channel {
  int id = -1;
  bool live = false;
  vca_config cfg{};
  vca_analyzer* an = nullptr;
  uint8_t* ring = nullptr;  // two slots, each plane-major: Y of every frame, then U, then V
  size_t slot_bytes = 0;
  size_t ystride = 0, cstride = 0;  // bytes between frames of one plane (pitch x rows)
  int64_t pitch_y = 0, pitch_uv = 0;
  size_t off_u = 0, off_v = 0;      // plane offsets within a slot
  int max_frames = 0;
  size_t cost = 0;
  std::deque<Segment> queue;       // submitted, oldest first (at most two: one per slot)
  std::deque<Segment> finishing;   // every frame queued; waiting for the last frame's features
  int64_t frames_queued = 0;       // frames handed to ticks
};

}  // namespace

struct vca_server {
  int device = 0;
  int policy = VCA_SERVE_SEGMENTS;
  size_t budget = 0;
  size_t used = 0;
  std::deque<Channel> ch;    // references stay valid as channels are added
  vca_batch* batch = nullptr;
  std::vector<int> members;  // channel ids of the batch, in member order
  bool rebuild = false;
  std::mutex mu;   // queues, channel list, counters
  std::mutex eng;  // every call into the analyzers and the batch
  std::condition_variable cv;
  std::deque<vca_segment_done> done;
  std::thread worker;
  std::atomic<bool> stop{false};
  vca_status worker_status = VCA_OK;
  char worker_error[256] = {0};
  int64_t ticks = 0;
  int64_t frames = 0;
  int64_t launches_retired = 0;  // launches of batches already destroyed
  cudaStream_t copy_stream = nullptr;  // copies of vca_server_submit_frames
};

namespace {

// Device bytes of an analyzer of this configuration (the allocations vca_open makes for
// c.max_batch frames per push), rounded up generously for allocator granularity.
size_t analyzer_cost(const vca_config& c, int64_t C) {
  const size_t w = c.block_size, nc = c.chroma_format == VCA_CHROMA_444 ? w : w / 2;
  const size_t ncv = c.chroma_format == VCA_CHROMA_422 ? w : nc;
  const size_t mb = (size_t)c.max_batch;
  size_t b = round_up(w * w + nc * nc + 4 * (w * w + ncv * nc), 4096);
  b += round_up((2 * mb + 1) * 6 * (size_t)C * 4, 4096);  // block values: two push buffers + a dump slot
  b += 2 * round_up((size_t)C * 4, 4096);                  // previous-frame luma energies
  b += round_up(vca::reduce_partials_bytes((int)mb), 4096) + round_up(mb * 4, 4096);  // reduction scratch
  b += 4 * 4096;                                            // features, flag
  return b;
}

// Chroma plane rows and columns of a configuration.
void chroma_size(const vca_config& c, int* cw, int* ch) {
  const bool full = c.chroma_format == VCA_CHROMA_444, c422 = c.chroma_format == VCA_CHROMA_422;
  *cw = full ? c.width : c.width / 2;
  *ch = full || c422 ? c.height : c.height / 2;
}

// Moves segments whose last frame's features have arrived to the completion queue.
void finish_segments(vca_server* s, bool blocking) {
  size_t n;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    n = s->ch.size();
  }
  for (size_t i = 0; i < n; ++i) {
    Channel* cp;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      cp = &s->ch[i];  // element addresses of a deque survive push_back; its index map may not
    }
    Channel& c = *cp;
    for (;;) {
      Segment g;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        if (!c.live || c.finishing.empty()) break;
        g = c.finishing.front();
      }
      vca_frame_features ff;
      vca_status st;
      {
        std::lock_guard<std::mutex> le(s->eng);
        st = vca_read_frame_features(c.an, g.first_frame + g.n - 1, blocking ? 1 : 0, &ff);
      }
      if (st == VCA_E_AGAIN) break;
      vca_segment_done d{};
      d.channel = c.id;
      d.tag = g.tag;
      d.first_frame = g.first_frame;
      d.n_frames = g.n;
      d.submit_ns = g.t_submit;
      d.ready_ns = now_ns();
      d.status = st;
      if (g.ready) cudaEventDestroy(g.ready);
      std::lock_guard<std::mutex> lk(s->mu);
      c.finishing.pop_front();
      s->done.push_back(d);
    }
  }
}

// Segments policy: every channel whose oldest segment has landed gets it pushed as one work item
// (pushes of up to kPushFrames frames).  Returns false when the scheduler must stop.
bool push_landed_segments(vca_server* s, bool* pushed) {
  size_t n;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    n = s->ch.size();
  }
  for (size_t i = 0; i < n; ++i) {
    Channel* cp;
    Segment g;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      cp = &s->ch[i];
      if (!cp->live || cp->queue.empty()) continue;
      g = cp->queue.front();
      if (g.ready) {
        cudaError_t q = cudaEventQuery(g.ready);
        if (q == cudaErrorNotReady) continue;
        cudaGetLastError();
      }
    }
    Channel& c = *cp;
    const uint8_t* base = c.ring + (size_t)g.slot * c.slot_bytes;
    vca_status st = VCA_OK;
    int pushes = 0;
    for (int f = 0; f < g.n && st == VCA_OK; f += kPushFrames, ++pushes) {
      const int k = g.n - f < kPushFrames ? g.n - f : kPushFrames;
      std::lock_guard<std::mutex> le(s->eng);
      st = vca_push_frames(c.an, base + (size_t)f * c.ystride, base + c.off_u + (size_t)f * c.cstride,
                           base + c.off_v + (size_t)f * c.cstride, c.pitch_y, c.pitch_uv, (int64_t)c.ystride,
                           (int64_t)c.cstride, k, 1);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (st != VCA_OK) {
      s->worker_status = st;
      snprintf(s->worker_error, sizeof s->worker_error, "%s", vca_last_error());
      return false;
    }
    g.first_frame = c.frames_queued;
    g.next = g.n;
    c.frames_queued += g.n;
    c.finishing.push_back(g);
    c.queue.pop_front();
    s->ticks += pushes;
    s->frames += g.n;
    *pushed = true;
  }
  return true;
}

void worker_main(vca_server* s) {
  cudaSetDevice(s->device);
  std::vector<vca_frame_ref> refs;
  std::vector<Channel*> active;
  for (;;) {
    if (s->policy == VCA_SERVE_SEGMENTS) {
      {
        std::unique_lock<std::mutex> lk(s->mu);
        auto has_work = [&] {
          if (s->stop) return true;
          for (auto& c : s->ch)
            if (c.live && (!c.queue.empty() || !c.finishing.empty())) return true;
          return false;
        };
        s->cv.wait_for(lk, std::chrono::milliseconds(50), has_work);
        if (s->stop) break;
      }
      bool pushed = false;
      if (!push_landed_segments(s, &pushed)) break;
      finish_segments(s, false);
      if (!pushed) std::this_thread::sleep_for(std::chrono::microseconds(20));
      continue;
    }
    bool rebuild = false;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      auto has_work = [&] {
        if (s->stop || s->rebuild) return true;
        for (auto& c : s->ch)
          if (c.live && (!c.queue.empty() || !c.finishing.empty())) return true;
        return false;
      };
      s->cv.wait_for(lk, std::chrono::milliseconds(50), has_work);
      if (s->stop) break;
      rebuild = s->rebuild;
      s->rebuild = false;
    }
    if (rebuild) {
      if (s->batch) {
        int64_t l = 0;
        {
          std::lock_guard<std::mutex> le(s->eng);
          vca_batch_sync(s->batch);
        }
        finish_segments(s, true);
        std::lock_guard<std::mutex> le(s->eng);
        vca_batch_launch_count(s->batch, &l);
        s->launches_retired += l;
        vca_batch_destroy(s->batch);
        s->batch = nullptr;
      }
      std::vector<vca_analyzer*> an;
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->members.clear();
        for (auto& c : s->ch)
          if (c.live) {
            an.push_back(c.an);
            s->members.push_back(c.id);
          }
      }
      if (!an.empty()) {
        std::lock_guard<std::mutex> le(s->eng);
        vca_status st = vca_batch_create(an.data(), (int32_t)an.size(), &s->batch);
        if (st != VCA_OK) {
          std::lock_guard<std::mutex> lk(s->mu);
          s->worker_status = st;
          snprintf(s->worker_error, sizeof s->worker_error, "%s", vca_last_error());
          s->batch = nullptr;
        }
      }
    }
    if (!s->batch) continue;
    // One tick: the next frame of every channel whose oldest segment has landed.
    refs.assign(s->members.size(), vca_frame_ref{nullptr, nullptr, nullptr, 0, 0});
    active.clear();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      for (size_t i = 0; i < s->members.size(); ++i) {
        Channel& c = s->ch[s->members[i]];
        if (c.queue.empty()) continue;
        Segment& g = c.queue.front();
        if (g.ready) {
          cudaError_t q = cudaEventQuery(g.ready);
          if (q == cudaErrorNotReady) continue;
          cudaGetLastError();
        }
        const uint8_t* base = c.ring + (size_t)g.slot * c.slot_bytes;
        refs[i] = vca_frame_ref{base + (size_t)g.next * c.ystride, base + c.off_u + (size_t)g.next * c.cstride,
                                base + c.off_v + (size_t)g.next * c.cstride, c.pitch_y, c.pitch_uv};
        active.push_back(&c);
      }
    }
    if (!active.empty()) {
      vca_status st;
      {
        std::lock_guard<std::mutex> le(s->eng);
        st = vca_batch_tick(s->batch, refs.data());
      }
      if (st != VCA_OK) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->worker_status = st;
        snprintf(s->worker_error, sizeof s->worker_error, "%s", vca_last_error());
        break;
      }
      std::lock_guard<std::mutex> lk(s->mu);
      s->ticks += 1;
      s->frames += (int64_t)active.size();
      for (Channel* c : active) {
        Segment& g = c->queue.front();
        if (g.next == 0) g.first_frame = c->frames_queued;
        g.next += 1;
        c->frames_queued += 1;
        if (g.next == g.n) {
          c->finishing.push_back(g);
          c->queue.pop_front();
        }
      }
    }
    finish_segments(s, active.empty());
  }
  if (s->batch) {
    {
      std::lock_guard<std::mutex> le(s->eng);
      vca_batch_sync(s->batch);
    }
    finish_segments(s, true);
  }
}

}  // namespace

extern "C" {

vca_status vca_server_create(size_t device_budget_bytes, vca_server** out) {
  if (!out) return sfail(VCA_E_ARG, "out is NULL");
  *out = nullptr;
  vca_server* s = new (std::nothrow) vca_server();
  if (!s) return sfail(VCA_E_NOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&s->device);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    delete s;
    cudaGetLastError();
    return sfail(VCA_E_CUDA, "querying device memory: %s", cudaGetErrorString(e));
  }
  s->budget = device_budget_bytes ? device_budget_bytes : free_b / 10 * 9;
  if (s->budget > free_b) {
    delete s;
    return sfail(VCA_E_NOMEM, "budget %zu exceeds free device memory %zu", device_budget_bytes, free_b);
  }
  if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete s;
    return sfail(VCA_E_CUDA, "creating the copy stream");
  }
  try {
    s->worker = std::thread(worker_main, s);
  } catch (...) {
    delete s;
    return sfail(VCA_E_NOMEM, "could not start the scheduler thread");
  }
  *out = s;
  return VCA_OK;
}

vca_status vca_server_add_channel(vca_server* s, const vca_config* cfg, int32_t max_segment_frames, int32_t* id) {
  if (!s || !cfg || !id) return sfail(VCA_E_ARG, "NULL argument");
  if (max_segment_frames < 1 || max_segment_frames > 4096)
    return sfail(VCA_E_ARG, "max_segment_frames must be in [1, 4096]");
  int64_t bx = 0, by = 0;
  vca_status st = vca_block_count(cfg, &bx, &by);
  if (st != VCA_OK) return st;
  vca_config c = *cfg;
  int policy;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    policy = s->policy;
  }
  // Ticks analyse one frame per channel; segments push up to kPushFrames frames at a time.
  c.max_batch = policy == VCA_SERVE_TICKS ? 1 : (max_segment_frames < kPushFrames ? max_segment_frames : kPushFrames);
  const int bps = c.bit_depth > 8 ? 2 : 1;
  int cw, chh;
  chroma_size(c, &cw, &chh);
  const int64_t py = (int64_t)round_up((size_t)c.width * bps, 256), pc = (int64_t)round_up((size_t)cw * bps, 256);
  const size_t ystride = (size_t)py * c.height, cstride = (size_t)pc * chh;
  const size_t off_u = round_up(ystride * max_segment_frames, 256);
  const size_t off_v = off_u + round_up(cstride * max_segment_frames, 256);
  const size_t slot_bytes = off_v + round_up(cstride * max_segment_frames, 256);
  const size_t cost = analyzer_cost(c, bx * by) + 2 * slot_bytes;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->used + cost > s->budget)
      return sfail(VCA_E_NOMEM, "admission refused: channel needs %zu bytes, %zu of %zu left", cost,
                   s->budget - s->used, s->budget);
    s->used += cost;  // reserved while the channel is set up
  }
  Channel ch;
  ch.cfg = c;
  ch.ystride = ystride;
  ch.cstride = cstride;
  ch.slot_bytes = slot_bytes;
  ch.pitch_y = py;
  ch.pitch_uv = pc;
  ch.off_u = off_u;
  ch.off_v = off_v;
  ch.max_frames = max_segment_frames;
  ch.cost = cost;
  st = vca_open(&c, nullptr, &ch.an);
  cudaError_t e = cudaSuccess;
  if (st == VCA_OK) e = cudaMalloc(&ch.ring, 2 * slot_bytes);
  if (st != VCA_OK || e != cudaSuccess) {
    if (ch.an) vca_close(ch.an);
    cudaGetLastError();
    std::lock_guard<std::mutex> lk(s->mu);
    s->used -= cost;
    return st != VCA_OK ? st : sfail(VCA_E_NOMEM, "allocating the segment ring: %s", cudaGetErrorString(e));
  }
  cudaMemset(ch.ring, 0, 2 * slot_bytes);
  cudaStreamSynchronize(nullptr);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    ch.id = (int)s->ch.size();
    ch.live = true;
    s->ch.push_back(std::move(ch));
    *id = s->ch.back().id;
    s->rebuild = s->policy == VCA_SERVE_TICKS;
  }
  s->cv.notify_all();
  return VCA_OK;
}

vca_status vca_server_segment_buffer(vca_server* s, int32_t id, int32_t slot, vca_frame_ref* frame0,
                                     int64_t* frame_stride_y, int64_t* frame_stride_uv) {
  if (!s || !frame0 || !frame_stride_y || !frame_stride_uv) return sfail(VCA_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (id < 0 || id >= (int)s->ch.size() || !s->ch[id].live) return sfail(VCA_E_ARG, "no channel %d", id);
  if (slot != 0 && slot != 1) return sfail(VCA_E_ARG, "slot must be 0 or 1");
  const Channel& c = s->ch[id];
  const uint8_t* base = c.ring + (size_t)slot * c.slot_bytes;
  *frame0 = vca_frame_ref{base, base + c.off_u, base + c.off_v, c.pitch_y, c.pitch_uv};
  *frame_stride_y = (int64_t)c.ystride;
  *frame_stride_uv = (int64_t)c.cstride;
  return VCA_OK;
}

vca_status vca_server_submit(vca_server* s, int32_t id, int32_t slot, int32_t n_frames, uint64_t tag,
                             void* ready_event) {
  if (!s) return sfail(VCA_E_ARG, "server is NULL");
  cudaEvent_t ev = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->worker_status != VCA_OK) return sfail(s->worker_status, "scheduler stopped: %s", s->worker_error);
    if (id < 0 || id >= (int)s->ch.size() || !s->ch[id].live) return sfail(VCA_E_ARG, "no channel %d", id);
    Channel& c = s->ch[id];
    if (slot != 0 && slot != 1) return sfail(VCA_E_ARG, "slot must be 0 or 1");
    if (n_frames < 1 || n_frames > c.max_frames) return sfail(VCA_E_ARG, "n_frames must be in [1, %d]", c.max_frames);
    for (const auto& g : c.queue)
      if (g.slot == slot) return sfail(VCA_E_AGAIN, "slot %d of channel %d is still queued", slot, id);
    for (const auto& g : c.finishing)
      if (g.slot == slot) return sfail(VCA_E_AGAIN, "slot %d of channel %d is still being analysed", slot, id);
  }
  if (ready_event) {
    // A private event that completes with the producer's, so the caller may reuse its own.
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return sfail(VCA_E_CUDA, "creating an event");
    }
    cudaStream_t tmp = nullptr;
    if (cudaStreamCreateWithFlags(&tmp, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamWaitEvent(tmp, (cudaEvent_t)ready_event, 0) != cudaSuccess || cudaEventRecord(ev, tmp) != cudaSuccess) {
      cudaGetLastError();
      if (tmp) cudaStreamDestroy(tmp);
      cudaEventDestroy(ev);
      return sfail(VCA_E_CUDA, "chaining the producer's event");
    }
    cudaStreamDestroy(tmp);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Segment g;
    g.slot = slot;
    g.n = n_frames;
    g.tag = tag;
    g.t_submit = now_ns();
    g.first_frame = 0;
    g.ready = ev;
    s->ch[id].queue.push_back(g);
  }
  s->cv.notify_all();
  return VCA_OK;
}

vca_status vca_server_submit_frames(vca_server* s, int32_t id, const vca_frame_ref* frame0, int64_t frame_stride_y,
                                   int64_t frame_stride_uv, int32_t n_frames, uint64_t tag, void* ready_event) {
  if (!s || !frame0 || !frame0->y || !frame0->u || !frame0->v) return sfail(VCA_E_ARG, "NULL argument");
  int slot = -1;
  const Channel* cp = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->worker_status != VCA_OK) return sfail(s->worker_status, "scheduler stopped: %s", s->worker_error);
    if (id < 0 || id >= (int)s->ch.size() || !s->ch[id].live) return sfail(VCA_E_ARG, "no channel %d", id);
    const Channel& c = s->ch[id];
    if (n_frames < 1 || n_frames > c.max_frames) return sfail(VCA_E_ARG, "n_frames must be in [1, %d]", c.max_frames);
    if (n_frames > 1 && (frame_stride_y <= 0 || frame_stride_uv <= 0))
      return sfail(VCA_E_ARG, "frame strides must be positive");
    bool busy[2] = {false, false};
    for (const auto& g : c.queue) busy[g.slot] = true;
    for (const auto& g : c.finishing) busy[g.slot] = true;
    slot = !busy[0] ? 0 : !busy[1] ? 1 : -1;
    if (slot < 0) return sfail(VCA_E_AGAIN, "both segment slots of channel %d are in use", id);
    cp = &c;
  }
  const Channel& c = *cp;
  const int bps = c.cfg.bit_depth > 8 ? 2 : 1;
  int cw, hc;
  chroma_size(c.cfg, &cw, &hc);
  const size_t wy = (size_t)c.cfg.width * bps, wc = (size_t)cw * bps;
  if (frame0->pitch_y < (int64_t)wy || frame0->pitch_uv < (int64_t)wc) return sfail(VCA_E_ARG, "pitch smaller than a row");
  uint8_t* dst = c.ring + (size_t)slot * c.slot_bytes;
  const int h = c.cfg.height;
  cudaError_t e = cudaSuccess;
  if (ready_event) e = cudaStreamWaitEvent(s->copy_stream, (cudaEvent_t)ready_event, 0);
  // Frames stacked without gaps (frame stride = pitch x rows) copy as one 2-D copy per plane.
  const bool stacked = n_frames == 1 || (frame_stride_y == frame0->pitch_y * h && frame_stride_uv == frame0->pitch_uv * hc);
  const int nf = stacked ? 1 : n_frames;
  const int rows = stacked ? n_frames : 1;
  for (int i = 0; i < nf && e == cudaSuccess; ++i) {
    const uint8_t* sy = static_cast<const uint8_t*>(frame0->y) + (int64_t)i * frame_stride_y;
    const uint8_t* su = static_cast<const uint8_t*>(frame0->u) + (int64_t)i * frame_stride_uv;
    const uint8_t* sv = static_cast<const uint8_t*>(frame0->v) + (int64_t)i * frame_stride_uv;
    e = cudaMemcpy2DAsync(dst + (size_t)i * c.ystride, c.pitch_y, sy, frame0->pitch_y, wy, (size_t)h * rows,
                          cudaMemcpyDefault, s->copy_stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(dst + c.off_u + (size_t)i * c.cstride, c.pitch_uv, su, frame0->pitch_uv, wc,
                            (size_t)hc * rows, cudaMemcpyDefault, s->copy_stream);
    if (e == cudaSuccess)
      e = cudaMemcpy2DAsync(dst + c.off_v + (size_t)i * c.cstride, c.pitch_uv, sv, frame0->pitch_uv, wc,
                            (size_t)hc * rows, cudaMemcpyDefault, s->copy_stream);
  }
  cudaEvent_t ev = nullptr;
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, s->copy_stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (ev) cudaEventDestroy(ev);
    return sfail(VCA_E_CUDA, "copying a segment: %s", cudaGetErrorString(e));
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    Segment g;
    g.slot = slot;
    g.n = n_frames;
    g.tag = tag;
    g.t_submit = now_ns();
    g.first_frame = 0;
    g.ready = ev;
    s->ch[id].queue.push_back(g);
  }
  s->cv.notify_all();
  return VCA_OK;
}

vca_status vca_server_poll(vca_server* s, vca_segment_done* out, int32_t max, int32_t* n) {
  if (!s || !n || (max > 0 && !out)) return sfail(VCA_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  int k = 0;
  while (k < max && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  *n = k;
  if (s->worker_status != VCA_OK && k == 0) return sfail(s->worker_status, "scheduler stopped: %s", s->worker_error);
  return VCA_OK;
}

vca_status vca_server_read_features(vca_server* s, int32_t id, int64_t frame, vca_frame_features* out) {
  if (!s || !out) return sfail(VCA_E_ARG, "NULL argument");
  vca_analyzer* an = nullptr;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (id < 0 || id >= (int)s->ch.size() || !s->ch[id].live) return sfail(VCA_E_ARG, "no channel %d", id);
    an = s->ch[id].an;
  }
  std::lock_guard<std::mutex> le(s->eng);
  return vca_read_frame_features(an, frame, 1, out);
}

vca_status vca_server_stats(vca_server* s, vca_server_stats_t* st) {
  if (!s || !st) return sfail(VCA_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  st->ticks = s->ticks;
  st->frames = s->frames;
  st->budget_bytes = s->budget;
  st->used_bytes = s->used;
  int live = 0;
  for (auto& c : s->ch) live += c.live;
  st->channels = live;
  int64_t l = 0;
  {
    std::lock_guard<std::mutex> le(s->eng);
    if (s->batch) vca_batch_launch_count(s->batch, &l);
    for (auto& c : s->ch) {  // the channels' own pushes (segments policy)
      int64_t x = 0;
      if (c.live && c.an && vca_launch_count(c.an, &x) == VCA_OK) l += x;
    }
  }
  st->launches = s->launches_retired + l;
  return VCA_OK;
}

vca_status vca_server_set_policy(vca_server* s, int32_t policy) {
  if (!s) return sfail(VCA_E_ARG, "server is NULL");
  if (policy != VCA_SERVE_SEGMENTS && policy != VCA_SERVE_TICKS) return sfail(VCA_E_ARG, "unknown policy %d", policy);
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->ch.empty()) return sfail(VCA_E_STATE, "the policy is set before the first channel is added");
  s->policy = policy;
  return VCA_OK;
}

vca_status vca_server_destroy(vca_server* s) {
  if (!s) return VCA_OK;
  // Let queued segments finish, then stop the scheduler.
  for (;;) {
    bool busy = false;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->worker_status != VCA_OK) break;
      for (auto& c : s->ch)
        if (c.live && (!c.queue.empty() || !c.finishing.empty())) busy = true;
    }
    if (!busy) break;
    std::this_thread::sleep_for(std::chrono::microseconds(200));
  }
  s->stop = true;
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  vca_status st = s->worker_status;
  if (s->batch) vca_batch_destroy(s->batch);
  for (auto& c : s->ch) {
    for (auto& g : c.queue)
      if (g.ready) cudaEventDestroy(g.ready);
    if (c.an) vca_close(c.an);
    cudaFree(c.ring);
  }
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  delete s;
  return st;
}

}  // extern "C"
