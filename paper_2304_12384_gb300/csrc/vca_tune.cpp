// Launch-shape tuning: a process-wide table of launch shapes per analyzer configuration, the
// measurement that fills it (vca_autotune), its file form, and the tuning of a batch's SM split.
//
// The knobs are the ones the kernels take at run time: the kernel family (CUDA-core or
// tensor-core form), the CTA size of the CUDA-core form (2, 4 or 8 warps, i.e. 2, 4 or 8 times
// 32 / w blocks per CTA), the number of CTAs of a tensor-core launch, and, for a batch whose
// members come in two sample sizes, the weight of a 16-bit-word tile against a byte tile when the
// SMs are split between the two launches of a tick.  Every shape computes the same features bit
// for bit: only the time differs.
#include <cuda_runtime.h>

#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "vca.h"
#include "vca_internal.h"

namespace vca {
namespace {

std::mutex g_tune_mu;
std::vector<vca_tune_entry> g_tune;  // at most one entry per configuration
std::once_flag g_env_once;

bool same_key(const vca_tune_entry& e, const vca_config& c) {
  return e.width == c.width && e.height == c.height && e.bit_depth == c.bit_depth && e.block_size == c.block_size &&
         e.low_pass == c.low_pass && e.chroma_format == c.chroma_format;
}

bool same_key(const vca_tune_entry& a, const vca_tune_entry& b) {
  return a.width == b.width && a.height == b.height && a.bit_depth == b.bit_depth && a.block_size == b.block_size &&
         a.low_pass == b.low_pass && a.chroma_format == b.chroma_format;
}

bool valid_shape(const vca_tune_entry& e) {
  return (e.kernel == VCA_KERNEL_PLAIN || e.kernel == VCA_KERNEL_TC) &&
         (e.plain_warps == 2 || e.plain_warps == 4 || e.plain_warps == 8) && e.tc_ctas >= 0 && e.tc_ctas <= 4096;
}

void put(const vca_tune_entry& e) {
  for (auto& x : g_tune)
    if (same_key(x, e)) {
      x = e;
      return;
    }
  g_tune.push_back(e);
}

// One entry per line: width height bit_depth block_size low_pass chroma_format kernel plain_warps
// tc_ctas ms_per_frame.  Lines starting with '#' are comments.
vca_status load_file(const char* path, bool replace) {
  FILE* f = std::fopen(path, "r");
  if (!f) {
    char msg[300];
    std::snprintf(msg, sizeof msg, "cannot open tuning table %s: %s", path, std::strerror(errno));
    record_error(msg);
    return VCA_E_ARG;
  }
  std::vector<vca_tune_entry> got;
  char line[256];
  int lineno = 0;
  while (std::fgets(line, sizeof line, f)) {
    ++lineno;
    if (line[0] == '#' || line[0] == '\n' || line[0] == '\0') continue;
    vca_tune_entry e{};
    if (std::sscanf(line, "%d %d %d %d %d %d %d %d %d %f", &e.width, &e.height, &e.bit_depth, &e.block_size,
                    &e.low_pass, &e.chroma_format, &e.kernel, &e.plain_warps, &e.tc_ctas, &e.ms_per_frame) != 10 ||
        !valid_shape(e)) {
      std::fclose(f);
      char msg[300];
      std::snprintf(msg, sizeof msg, "tuning table %s: line %d is not an entry", path, lineno);
      record_error(msg);
      return VCA_E_ARG;
    }
    got.push_back(e);
  }
  std::fclose(f);
  std::lock_guard<std::mutex> lock(g_tune_mu);
  if (replace) g_tune.clear();
  for (const auto& e : got) put(e);
  return VCA_OK;
}

void load_env_once() {
  std::call_once(g_env_once, [] {
    const char* p = std::getenv("VCA_TUNE_FILE");
    if (p && *p) load_file(p, false);  // a missing or bad file leaves the table as it is
  });
}

}  // namespace

bool tune_lookup(const vca_config& c, vca_tune_entry* out) {
  load_env_once();
  std::lock_guard<std::mutex> lock(g_tune_mu);
  for (const auto& e : g_tune)
    if (same_key(e, c)) {
      *out = e;
      return true;
    }
  return false;
}

}  // namespace vca

extern "C" {

vca_status vca_tune_set(const vca_tune_entry* e) {
  if (!e || !vca::valid_shape(*e)) {
    vca::record_error("vca_tune_set: kernel must be plain or tc, plain_warps 2, 4 or 8, tc_ctas >= 0");
    return VCA_E_ARG;
  }
  vca_config c{};
  c.width = e->width;
  c.height = e->height;
  c.bit_depth = e->bit_depth;
  c.block_size = e->block_size;
  c.low_pass = e->low_pass;
  c.chroma_format = e->chroma_format;
  int64_t bx = 0, by = 0;
  vca_status s = vca_block_count(&c, &bx, &by);
  if (s != VCA_OK) return s;
  vca::load_env_once();
  std::lock_guard<std::mutex> lock(vca::g_tune_mu);
  vca::put(*e);
  return VCA_OK;
}

vca_status vca_tune_lookup(const vca_config* cfg, vca_tune_entry* out) {
  if (!cfg || !out) {
    vca::record_error("vca_tune_lookup: NULL argument");
    return VCA_E_ARG;
  }
  return vca::tune_lookup(*cfg, out) ? VCA_OK : VCA_E_AGAIN;
}

vca_status vca_tune_clear(void) {
  vca::load_env_once();
  std::lock_guard<std::mutex> lock(vca::g_tune_mu);
  vca::g_tune.clear();
  return VCA_OK;
}

vca_status vca_tune_save(const char* path) {
  if (!path) {
    vca::record_error("vca_tune_save: NULL path");
    return VCA_E_ARG;
  }
  vca::load_env_once();
  std::lock_guard<std::mutex> lock(vca::g_tune_mu);
  FILE* f = std::fopen(path, "w");
  if (!f) {
    char msg[300];
    std::snprintf(msg, sizeof msg, "cannot write tuning table %s: %s", path, std::strerror(errno));
    vca::record_error(msg);
    return VCA_E_ARG;
  }
  std::fprintf(f, "# width height bit_depth block_size low_pass chroma_format kernel plain_warps tc_ctas ms_per_frame\n");
  for (const auto& e : vca::g_tune)
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d %.6g\n", e.width, e.height, e.bit_depth, e.block_size, e.low_pass,
                 e.chroma_format, e.kernel, e.plain_warps, e.tc_ctas, (double)e.ms_per_frame);
  const bool ok = std::fclose(f) == 0;
  if (!ok) {
    vca::record_error("vca_tune_save: write failed");
    return VCA_E_ARG;
  }
  return VCA_OK;
}

vca_status vca_tune_load(const char* path) {
  if (!path) {
    vca::record_error("vca_tune_load: NULL path");
    return VCA_E_ARG;
  }
  vca::load_env_once();
  return vca::load_file(path, true);
}

vca_status vca_autotune(const vca_config* cfg, const void* y, const void* u, const void* v, int64_t pitch_y,
                        int64_t pitch_uv, int64_t frame_stride_y, int64_t frame_stride_uv, int32_t n_frames,
                        int32_t reps, void* cuda_stream, vca_tune_entry* candidates, int32_t max_candidates,
                        int32_t* n_candidates, vca_tune_entry* chosen) {
  if (!cfg || !y || !u || !v || n_frames < 1 || reps < 1) {
    vca::record_error("vca_autotune: needs a configuration, device frames, n_frames >= 1 and reps >= 1");
    return VCA_E_ARG;
  }
  int dev = 0, sms = 1;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                 cudaSuccess) {
    cudaGetLastError();
    vca::record_error("vca_autotune: no usable device");
    return VCA_E_CUDA;
  }
  // Candidates: the CUDA-core form with 2, 4 and 8 warps per CTA; the tensor-core form (where it
  // covers the configuration) on all, three quarters and half of the SMs.
  std::vector<vca_tune_entry> cand;
  vca_tune_entry base{};
  base.width = cfg->width;
  base.height = cfg->height;
  base.bit_depth = cfg->bit_depth;
  base.block_size = cfg->block_size;
  base.low_pass = cfg->low_pass;
  base.chroma_format = cfg->chroma_format;
  base.plain_warps = 4;
  for (int w : {2, 4, 8}) {
    vca_tune_entry e = base;
    e.kernel = VCA_KERNEL_PLAIN;
    e.plain_warps = w;
    cand.push_back(e);
  }
  {
    vca_config c = *cfg;
    c.kernel = VCA_KERNEL_TC;
    c.max_batch = n_frames;
    vca_analyzer* probe = nullptr;
    if (vca_open(&c, cuda_stream, &probe) == VCA_OK) {
      vca_close(probe);
      for (int ctas : {0, (sms * 3 / 4) & ~1, (sms / 2) & ~1}) {
        vca_tune_entry e = base;
        e.kernel = VCA_KERNEL_TC;
        e.tc_ctas = ctas;
        cand.push_back(e);
      }
    }
  }
  int best = -1;
  for (size_t i = 0; i < cand.size(); ++i) {
    vca_config c = *cfg;
    c.kernel = cand[i].kernel;
    c.max_batch = n_frames;
    vca_analyzer* a = nullptr;
    vca_status s = vca_open(&c, cuda_stream, &a);
    if (s != VCA_OK) return s;
    s = vca::set_launch_shape(a, cand[i].plain_warps, cand[i].tc_ctas);
    for (int r = 0; s == VCA_OK && r < 2; ++r)  // warm-up
      s = vca_push_frames(a, y, u, v, pitch_y, pitch_uv, frame_stride_y, frame_stride_uv, n_frames, 1);
    if (s == VCA_OK) s = vca_sync(a);
    if (s == VCA_OK) s = vca_set_kernel_timing(a, 1);
    for (int r = 0; s == VCA_OK && r < reps; ++r)
      s = vca_push_frames(a, y, u, v, pitch_y, pitch_uv, frame_stride_y, frame_stride_uv, n_frames, 1);
    if (s == VCA_OK) s = vca_sync(a);
    double ms = 0.0;
    int64_t pushes = 0;
    if (s == VCA_OK) s = vca_read_kernel_timing(a, &ms, &pushes);
    vca_close(a);
    if (s != VCA_OK) return s;
    cand[i].ms_per_frame = pushes > 0 ? (float)(ms / ((double)pushes * n_frames)) : 0.0f;
    if (best < 0 || cand[i].ms_per_frame < cand[best].ms_per_frame) best = (int)i;
  }
  if (n_candidates) *n_candidates = (int32_t)cand.size();
  for (int i = 0; candidates && i < (int)cand.size() && i < max_candidates; ++i) candidates[i] = cand[i];
  if (chosen) *chosen = cand[best];
  return vca_tune_set(&cand[best]);
}

}  // extern "C"
