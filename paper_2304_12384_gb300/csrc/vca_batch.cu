// Batched multi-stream analysis: one frame of every analyzer of a batch in one launch of the plain
// block routine (Section 2 of the paper, per block: integer DCT, texture energy H, brightness L).
//
// The analyzers may differ in frame size and bit depth but share block sizes (chroma format) and
// the low-pass option.  Each CTA reads its (analyzer, plane kind, plane, block chunk) from a map
// built once when the batch is created, and the analyzer's arguments for this tick from a table
// the host refreshes every tick; an analyzer skipped this tick has active = 0 and its CTAs return
// at once.
#include "vca_plain.cuh"

namespace vca {
namespace {

template <int Nl, int Ncv, int Nc, bool LP>
__global__ void __launch_bounds__(kWarps * 32)
    batch_plain_kernel(const BatchCta* __restrict__ map, const BatchMemberArgs* __restrict__ args) {
  __shared__ union {
    PlainSmem<Nl, Nl, LP> luma;
    PlainSmem<Ncv, Nc, LP> chroma;
  } sh;
  const BatchCta w = map[blockIdx.x];
  const BatchMemberArgs& ma = args[w.member];
  if (!ma.active) return;
  const PlainArgs a = ma.pa[w.kind];
  if (w.kind == 0) {
    if (ma.bps == 1)
      plain_blocks<Nl, Nl, LP, uint8_t>(a, w.plane, 0, w.chunk, sh.luma);
    else
      plain_blocks<Nl, Nl, LP, uint16_t>(a, w.plane, 0, w.chunk, sh.luma);
  } else {
    if (ma.bps == 1)
      plain_blocks<Ncv, Nc, LP, uint8_t>(a, w.plane, 0, w.chunk, sh.chroma);
    else
      plain_blocks<Ncv, Nc, LP, uint16_t>(a, w.plane, 0, w.chunk, sh.chroma);
  }
}

template <int Nl, int Ncv, int Nc>
cudaError_t launch_sizes(const BatchCta* d_map, int n_cta, const BatchMemberArgs* d_args, bool low_pass,
                         cudaStream_t s) {
  const dim3 grid((unsigned)n_cta), block(kWarps * 32);
  if (low_pass)
    batch_plain_kernel<Nl, Ncv, Nc, true><<<grid, block, 0, s>>>(d_map, d_args);
  else
    batch_plain_kernel<Nl, Ncv, Nc, false><<<grid, block, 0, s>>>(d_map, d_args);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_batch_plain(const BatchCta* d_map, int n_cta, const BatchMemberArgs* d_args, int w, int nc,
                               int ncv, bool low_pass, cudaStream_t s) {
  if (n_cta <= 0) return cudaSuccess;
  static_assert(plain_blocks_per_cta(32) == kWarps * 1 && plain_blocks_per_cta(16) == kWarps * 2,
                "blocks per CTA of the plain routine");
  if (ncv == nc) {  // 4:2:0 (w/2 blocks) and 4:4:4 (w blocks)
    if (w == 32 && nc == 16) return launch_sizes<32, 16, 16>(d_map, n_cta, d_args, low_pass, s);
    if (w == 16 && nc == 8) return launch_sizes<16, 8, 8>(d_map, n_cta, d_args, low_pass, s);
    if (w == 8 && nc == 4) return launch_sizes<8, 4, 4>(d_map, n_cta, d_args, low_pass, s);
    if (w == 32 && nc == 32) return launch_sizes<32, 32, 32>(d_map, n_cta, d_args, low_pass, s);
    if (w == 16 && nc == 16) return launch_sizes<16, 16, 16>(d_map, n_cta, d_args, low_pass, s);
    if (w == 8 && nc == 8) return launch_sizes<8, 8, 8>(d_map, n_cta, d_args, low_pass, s);
  } else if (ncv == w && nc == w / 2) {  // 4:2:2: w rows of w/2 samples
    if (w == 32) return launch_sizes<32, 32, 16>(d_map, n_cta, d_args, low_pass, s);
    if (w == 16) return launch_sizes<16, 16, 8>(d_map, n_cta, d_args, low_pass, s);
    if (w == 8) return launch_sizes<8, 8, 4>(d_map, n_cta, d_args, low_pass, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace vca
