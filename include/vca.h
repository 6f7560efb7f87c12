/*
 * vca.h -- C ABI of the GB300 Video Complexity Analyzer (VCA) hot path.
 *
 * The analyzer computes, for every frame of a planar YUV 4:2:0 video, the seven
 * blockwise DCT-energy features named in Section 2 of "Green Video Complexity
 * Analysis for Efficient Encoding in Adaptive Video Streaming" (GMSys '23):
 * the luma texture energy E_Y, its temporal gradient h, the luminescence L_Y,
 * the chroma texture energies E_U, E_V and the chrominances L_U, L_V.  Section 2
 * item (3) adds the low-pass option, which the library offers in two readings:
 * only the low-frequency quarter of each block's coefficients is computed
 * (VCA_LOWPASS_QUARTER), or every plane is first halved in each direction (rounded
 * 2x2 mean, (a + b + c + d + 2) >> 2, odd edges repeated) and analysed with half-size
 * blocks on the same block grid (VCA_LOWPASS_DOWNSAMPLE; the normalisations use the
 * half-size blocks).
 *
 * Definitions used (the paper names the features; these are the readings the
 * library implements, identically to the test oracle):
 *   blocks      luma w x w, chroma (w/2) x (w/2) (4:2:0) or w x w (4:4:4) on the
 *               same grid, C blocks per plane, raster order; partial edge blocks
 *               repeat the last row/column (VCA_PAD_REPLICATE) or are dropped
 *               (VCA_PAD_SKIP);
 *   transform   integer DCT, M_N[k][n] = round_half_away(64 sqrt(N) alpha_k
 *               cos(pi(2n+1)k/2N)); rows first, T = (X M^T + 2^(s1-1)) >> s1,
 *               then columns, Z = (M T + 2^(s2-1)) >> s2, s1 = log2 N + B - 9,
 *               s2 = log2 N + 6 (B = bit depth); results are bit-exact integers;
 *   block       H = sum_{(u,v) != (0,0)} w_N(u,v) |Z(u,v)| with
 *               w_N(u,v) = exp(|((u+1)(v+1)/N^2)^2 - 1|), in FP32;
 *               L = sqrt(Z(0,0)), in FP32;
 *   frame       E_P = sum_k H_{P,k} / (C N_P^2), L_P = sum_k L_{P,k} / C,
 *               h_t = sum_k |H_{Y,k,t} - H_{Y,k,t-1}| / (C w^2), h_0 = 0,
 *               the block sums exact (128-bit fixed point in units of 2^-23),
 *               each total rounded once to FP64, then divided (deterministic,
 *               and independent of how frames are batched);
 *   sequence    arithmetic mean over frames (h over frames t >= 1).
 *
 * Conventions for every call:
 *   - every call returns a vca_status; no exception or abort crosses the ABI;
 *     vca_last_error() gives a one-line message for the calling thread;
 *   - the caller owns frame buffers; the library owns its device state, which
 *     vca_close() frees;
 *   - device frame buffers must stay valid and unchanged until the pushed
 *     frames' features have been read (or vca_sync() returned); host frame
 *     buffers are consumed before vca_push_frame(s) returns;
 *   - plane base pointers and pitches must be multiples of 16 bytes;
 *     samples are uint8 (bit_depth 8) or little-endian 16-bit words holding
 *     values in [0, 2^B - 1] (bit_depth 10, 12); other values are undefined
 *     behaviour;
 *   - an analyzer is bound to one CUDA stream and is not thread-safe; distinct
 *     analyzers may be used from distinct threads.
 */
#ifndef VCA_H
#define VCA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum vca_status {
  VCA_OK = 0,
  VCA_E_ARG = -1,          /* invalid argument (NULL, size, alignment, range) */
  VCA_E_UNSUPPORTED = -2,  /* valid but unsupported configuration */
  VCA_E_NOMEM = -3,        /* device or pinned host allocation failed */
  VCA_E_CUDA = -4,         /* a CUDA runtime / driver call failed */
  VCA_E_AGAIN = -5,        /* result not ready (non-blocking read) */
  VCA_E_TIMEOUT = -6,      /* a bounded device wait gave up */
  VCA_E_STATE = -7         /* call not valid in the analyzer's current state */
} vca_status;

enum { VCA_PAD_REPLICATE = 0, VCA_PAD_SKIP = 1 };
enum { VCA_LOWPASS_OFF = 0, VCA_LOWPASS_QUARTER = 1, VCA_LOWPASS_DOWNSAMPLE = 2 };
enum { VCA_CHROMA_420 = 0, VCA_CHROMA_444 = 1, VCA_CHROMA_422 = 2 };
enum { VCA_KERNEL_AUTO = 0, VCA_KERNEL_PLAIN = 1, VCA_KERNEL_TC = 2 };

/* Analyzer configuration (Section 2: one analyzer per video). */
typedef struct vca_config {
  int32_t width;       /* luma width in samples, even, >= 2 */
  int32_t height;      /* luma height in samples, even, >= 2 */
  int32_t bit_depth;   /* 8, 10 or 12 */
  int32_t block_size;  /* luma block size w: 8, 16 or 32; chroma blocks cover the same area */
  int32_t low_pass;    /* VCA_LOWPASS_OFF: all coefficients; VCA_LOWPASS_QUARTER: only u, v < N/2;
                          VCA_LOWPASS_DOWNSAMPLE: halved planes, w/2 and w/4 blocks (block_size 32
                          only; not in batches) -- Section 2 item (3) */
  int32_t pad_mode;    /* VCA_PAD_REPLICATE (default) or VCA_PAD_SKIP */
  int32_t kernel;      /* VCA_KERNEL_AUTO, VCA_KERNEL_PLAIN (CUDA cores) or VCA_KERNEL_TC (tensor cores:
                          8- and 10-bit 4:2:0 and 4:4:4 with 32x32 or 16x16 luma blocks, the
                          downsample reading included; other configurations give VCA_E_UNSUPPORTED).  AUTO
                          takes the tensor cores where they cover the configuration. */
  int32_t max_batch;   /* most frames one vca_push_frames call may carry; 0 selects 64 */
  int32_t chroma_format; /* VCA_CHROMA_420 (default: half-size chroma planes, w/2 blocks),
                            VCA_CHROMA_444 (full-size chroma planes, w blocks) or VCA_CHROMA_422
                            (half-width, full-height chroma planes; blocks of w rows by w/2
                            columns: rows take the (w/2)-point transform, columns the w-point
                            one, each stage the shift of its own length; E_U and E_V divide by
                            C w^2/2).  The paper names no 4:2:2 block shape: this is the
                            co-located reading.  4:2:2 runs on the CUDA cores. */
} vca_config;

/* The seven features of one frame (Section 2), frame = 0-based index since vca_open. */
typedef struct vca_frame_features {
  int64_t frame;
  double E_Y, h, L_Y, E_U, E_V, L_U, L_V;
} vca_frame_features;

/* Means over all frames read so far; h averages frames t >= 1. */
typedef struct vca_sequence_features {
  int64_t frames;
  double E_Y, h, L_Y, E_U, E_V, L_U, L_V;
} vca_sequence_features;

typedef struct vca_analyzer vca_analyzer;

/* Number of blocks C per plane for a configuration (Section 2: blockwise features).
 * Returns VCA_E_ARG for an invalid configuration. */
vca_status vca_block_count(const vca_config* cfg, int64_t* blocks_x, int64_t* blocks_y);

/* Open an analyzer for one video (Section 2).  cuda_stream is a cudaStream_t
 * (NULL = the legacy default stream) on which all of the analyzer's device work
 * is ordered.  The current CUDA device at this call is the analyzer's device.
 * On success *out owns device buffers sized for cfg->max_batch frames. */
vca_status vca_open(const vca_config* cfg, void* cuda_stream, vca_analyzer** out);

/* Analyse one frame (Section 2: seven features per frame).  y, u, v point at the
 * first sample of each plane; pitch_y / pitch_uv are row strides in bytes.
 * on_device = 1: the planes are device memory, read asynchronously on the
 * analyzer's stream.  on_device = 0: host memory, copied to the device before
 * the call returns (pinned memory makes that copy faster). */
vca_status vca_push_frame(vca_analyzer* a, const void* y, const void* u, const void* v,
                          int64_t pitch_y, int64_t pitch_uv, int32_t on_device);

/* Analyse n_frames consecutive frames in one launch.  Frame i's planes start at
 * y + i*frame_stride_y, u + i*frame_stride_uv, v + i*frame_stride_uv (bytes).
 * Strides must be multiples of 16 bytes; 1 <= n_frames <= max_batch. */
vca_status vca_push_frames(vca_analyzer* a, const void* y, const void* u, const void* v,
                           int64_t pitch_y, int64_t pitch_uv,
                           int64_t frame_stride_y, int64_t frame_stride_uv,
                           int32_t n_frames, int32_t on_device);

/* Features of frame `frame` (0-based).  blocking = 0 returns VCA_E_AGAIN while the
 * frame is still being computed; blocking = 1 waits.  VCA_E_ARG for a frame not
 * pushed yet. */
vca_status vca_read_frame_features(vca_analyzer* a, int64_t frame, int32_t blocking, vca_frame_features* out);

/* Per-sequence features over every frame pushed so far (waits for them). */
vca_status vca_read_sequence_features(vca_analyzer* a, vca_sequence_features* out);

/* Per-block values (FP32, raster order, C entries each; any pointer may be NULL)
 * of frame `index` within the most recent vca_push_frame(s) call.  Waits for it. */
vca_status vca_read_block_values(vca_analyzer* a, int32_t index, float* H_Y, float* L_Y,
                                 float* H_U, float* L_U, float* H_V, float* L_V);

/* Quantised coefficients Z of one frame, computed by the analyzer's kernel with
 * the coefficient dump enabled (bit-exact integers; parity checks).  zy, zu, zv
 * are device buffers of C*Nk*Nk int16 each (Nk = N, or N/2 with VCA_LOWPASS_QUARTER;
 * N = w for Y, w/2 for U, V, halved again with VCA_LOWPASS_DOWNSAMPLE; in 4:2:2, U and V
 * hold C*Nkv*Nkh with Nkv, Nkh those of the w-row, w/2-column blocks), block-major,
 * then row u, then column v.  Planes are on the device.  Does not change the
 * analyzer's frame count or h state. */
vca_status vca_dump_coefficients(vca_analyzer* a, const void* y, const void* u, const void* v,
                                 int64_t pitch_y, int64_t pitch_uv,
                                 int16_t* zy, int16_t* zu, int16_t* zv);

/* Wait for all of the analyzer's device work. */
vca_status vca_sync(vca_analyzer* a);

/* The frame reduction and the feature read-back of a push run on a second stream of the
 * analyzer, overlapping the next push's analysis.  This makes the analyzer's own stream wait
 * (on the device, without blocking the host) for all of that work, so later work on that stream
 * -- or an event recorded there -- comes after every queued push is complete. */
vca_status vca_stream_join(vca_analyzer* a);

/* Cross-frame state (the previous frame's luma block energies that h needs, and
 * the frame counter) as bytes, so a channel can resume with a correct h.
 * Call with buf = NULL to get the size in *len. */
vca_status vca_export_state(vca_analyzer* a, void* buf, size_t* len);
vca_status vca_import_state(vca_analyzer* a, const void* buf, size_t len);

/* Drop-in DCT matrix (an encoder's own integer table, for example a standard's hand-tuned one,
 * in place of the round-cosine matrix M_N of the transform reading above; Section 2 item (2):
 * the analyzer's DCT is an encoder's integer routine).  matrix: n x n int8, row-major, row k =
 * basis function k, n one of the analyzer's transform sizes (w, and the chroma block size; a
 * 4:4:4 analyzer's planes share one size).  Every later push, coefficient dump and batch tick
 * uses it, on either kernel.  Requirements (vca_check_dct_matrix): n in {4, 8, 16, 32},
 * matrix[0][0] = 64, and the even/odd symmetry of the DCT at every level (the level-L matrix is
 * rows 0, n/L, 2n/L, ... on their first L columns; its row k is even about the middle for even k
 * and odd for odd k), so that the butterfly and the matrix forms agree and every row but the
 * first sums to 0; for bit depths up to 10, T = (X M^T + 2^(s1-1)) >> s1 must stay within 16
 * bits.  The library copies the matrix.  VCA_E_STATE after the first push or inside a batch;
 * VCA_E_ARG (with the reason in vca_last_error) for a wrong size or a matrix that fails a
 * requirement.  Analyzers whose matrices differ can share a batch, which then runs the CUDA-core
 * kernel. */
vca_status vca_set_dct_matrix(vca_analyzer* a, int32_t n, const int8_t* matrix);

/* Checks a matrix against the requirements of vca_set_dct_matrix for the given bit depth (8, 10
 * or 12), on the host only. */
vca_status vca_check_dct_matrix(int32_t n, int32_t bit_depth, const int8_t* matrix);

/* Frames pushed since vca_open (or since the frame count an imported state carried). */
vca_status vca_frames_pushed(vca_analyzer* a, int64_t* frames);

/* Number of kernel launches this analyzer has issued (for launch accounting). */
vca_status vca_launch_count(vca_analyzer* a, int64_t* launches);

/* Kernel timing: with enable = 1, every later push brackets its analysis kernel(s) with
 * CUDA events on the analyzer's stream; vca_read_kernel_timing returns the summed
 * device time (ms) and the number of timed pushes among the pushes read so far
 * (it waits for all pushed frames). */
vca_status vca_set_kernel_timing(vca_analyzer* a, int32_t enable);
vca_status vca_read_kernel_timing(vca_analyzer* a, double* total_ms, int64_t* timed_pushes);

/* Kernel the analyzer runs: VCA_KERNEL_PLAIN or VCA_KERNEL_TC. */
vca_status vca_kernel_in_use(vca_analyzer* a, int32_t* kernel);

/* Free the analyzer (waits for its device work). NULL is accepted. */
vca_status vca_close(vca_analyzer* a);

/* ---- Batched multi-stream ticks --------------------------------------------------------
 *
 * A batch ticks many analyzers (channels) together: each tick analyses one frame per analyzer
 * (Section 2 of the paper: integer DCT, texture energy and brightness of every block of every
 * channel, then the frame's seven features), replayed from a CUDA graph: with the persistent
 * tensor-core kernel, which also reduces the frames to their features, or with one launch of the
 * batched CUDA-core block kernel and one of the batched frame reduction.  The analyzers may differ in frame size and bit
 * depth; they must share device, block size, chroma format and low_pass.  Features arrive in each analyzer as
 * if its frames had been pushed one at a time: read them with vca_read_frame_features /
 * vca_read_sequence_features, and the h state carries across ticks and across the batch's
 * destruction.  While in a batch an analyzer accepts no vca_push_frame(s),
 * vca_dump_coefficients or vca_import_state (VCA_E_STATE) and cannot be closed. */
typedef struct vca_batch vca_batch;

/* One channel's frame of a tick: device planes (16-byte aligned, pitches multiples of 16 bytes),
 * or y = NULL to skip the channel this tick. */
typedef struct {
  const void* y;
  const void* u;
  const void* v;
  int64_t pitch_y;
  int64_t pitch_uv;
} vca_frame_ref;

/* Groups n analyzers (1 .. 65535, distinct, none already in a batch).  Waits for the analyzers'
 * earlier work and builds two tick graphs on a stream of its own.  If every analyzer runs the
 * tensor-core kernel (with the same DCT matrices), a tick analyses them with the persistent
 * tensor-core kernel: the 8-bit members and the 10-bit members on two branches of the tick
 * graph, side by side with the device's SMs split between them in proportion to their tiles,
 * each branch one launch per 64 members (one after another); each launch ends by reducing its
 * members' frames to their features (exact sums, identical to a single analyzer's).  The tensor
 * maps of a tick's frames are encoded on the host; each analyzer keeps those of its last 8
 * distinct frames (by plane pointers and pitches), so frames ticked from a ring of up to 8
 * buffers per channel are encoded once.  Otherwise a tick is one launch of the batched CUDA-core
 * kernel, whose CTA map is built here, and one of the batched reduction.  VCA_E_ARG for
 * mismatched devices, block sizes or low_pass. */
vca_status vca_batch_create(vca_analyzer* const* members, int32_t n, vca_batch** out);

/* The kernel family a batch's ticks run: VCA_KERNEL_TC or VCA_KERNEL_PLAIN. */
vca_status vca_batch_kernel(vca_batch* b, int32_t* kernel);

/* One tick: frames[i] (n entries, in the order of vca_batch_create) for analyzer i.  Returns
 * after queuing the tick (at most two ticks are in flight; the third waits for the first).
 * The frame buffers must stay valid until the tick's features are read or vca_batch_sync
 * returns.  A bad frame reference gives VCA_E_ARG and queues nothing. */
vca_status vca_batch_tick(vca_batch* b, const vca_frame_ref* frames);

/* Waits for every queued tick and delivers its features to the analyzers.  VCA_E_TIMEOUT if the
 * tensor-core kernel gave up on a bounded wait during a tick: that tick's features are lost (the
 * analyzers' frame counters and h state have moved on). */
vca_status vca_batch_sync(vca_batch* b);

/* Kernel launches issued by the batch's ticks: per tick, for a tensor-core batch one launch per
 * sample size and 64 members (analysis and reduction), else the analysis and the reduction. */
vca_status vca_batch_launch_count(vca_batch* b, int64_t* launches);

/* Waits for the batch's ticks and dissolves it; the analyzers stay open.  NULL is accepted. */
vca_status vca_batch_destroy(vca_batch* b);

/* ---- Launch-shape tuning ------------------------------------------------------------------
 * Run-time tuning of how the kernels are launched (the paper, whose speed comes from a CPU
 * design, has no counterpart).  The library keeps one table of launch shapes per process, one
 * entry per analyzer configuration (width, height, bit depth, block size, low-pass, chroma
 * format).  vca_open follows the entry of its configuration: the kernel family when cfg->kernel
 * is VCA_KERNEL_AUTO (an entry naming the tensor-core form where it cannot run is ignored), and
 * the CTA sizes whatever the kernel.  Every shape computes the same features, bit for bit.  The
 * table starts empty, or with the file named by the environment variable VCA_TUNE_FILE (read at
 * the first vca_open or tuning call; a missing or bad file is ignored). */
typedef struct {
  int32_t width, height, bit_depth, block_size, low_pass, chroma_format;  /* the configuration */
  int32_t kernel;       /* VCA_KERNEL_PLAIN or VCA_KERNEL_TC */
  int32_t plain_warps;  /* CTA size of the CUDA-core form: 2, 4 or 8 warps (blocks per CTA =
                           warps * 32 / w for luma, warps * 32 / (w/2) for 4:2:0 chroma) */
  int32_t tc_ctas;      /* CTAs of a tensor-core launch: 0 = one per SM (never more than the SMs) */
  float ms_per_frame;   /* analysis time per frame measured for this shape, 0 if not measured */
} vca_tune_entry;

/* Measures every candidate shape of configuration cfg on the current device -- the CUDA-core form
 * with 2, 4 and 8 warps per CTA; the tensor-core form, where it covers cfg, on all, three
 * quarters and half of the SMs (even counts) -- by pushing the caller's n_frames device frames
 * (planes as for vca_push_frames, 16-byte aligned) reps times through a temporary analyzer per
 * candidate (after two untimed pushes), timing the analysis kernels with CUDA events on
 * cuda_stream.  The fastest becomes cfg's table entry and is returned in *chosen; the first
 * max_candidates measured candidates go to candidates[] and their count to *n_candidates (either
 * may be NULL).  Allocates device memory for the temporary analyzers: not for a hot path.
 * VCA_E_ARG for a bad configuration or arguments; errors of vca_open / vca_push_frames pass on. */
vca_status vca_autotune(const vca_config* cfg, const void* y, const void* u, const void* v, int64_t pitch_y,
                        int64_t pitch_uv, int64_t frame_stride_y, int64_t frame_stride_uv, int32_t n_frames,
                        int32_t reps, void* cuda_stream, vca_tune_entry* candidates, int32_t max_candidates,
                        int32_t* n_candidates, vca_tune_entry* chosen);
/* Adds or replaces the entry of e's configuration (VCA_E_ARG for a bad configuration or shape). */
vca_status vca_tune_set(const vca_tune_entry* e);
/* The entry of cfg's configuration (cfg->kernel and max_batch are not part of the key);
 * VCA_E_AGAIN if the table has none. */
vca_status vca_tune_lookup(const vca_config* cfg, vca_tune_entry* out);
vca_status vca_tune_clear(void);
/* The table as text, one entry per line: width height bit_depth block_size low_pass
 * chroma_format kernel plain_warps tc_ctas ms_per_frame ('#' starts a comment line).  Load
 * replaces the table; a file with a malformed line gives VCA_E_ARG and leaves it unchanged. */
vca_status vca_tune_save(const char* path);
vca_status vca_tune_load(const char* path);

/* A batch whose tensor-core members come in two sample sizes runs a tick as two launches side by
 * side, with the SMs split in proportion to their tiles, a tile of 16-bit words weighted against a
 * byte tile.  vca_batch_split_weight sets that weight (0.25 .. 4; 1.15 at creation);
 * vca_batch_autotune ticks the batch reps times with frames (after two untimed ticks) for each
 * weight in {1.0, 1.15, 1.3, 1.5, 1.75}, timed with CUDA events on the batch's stream, keeps the
 * fastest for the batch and returns it with its milliseconds per tick (a batch of one sample size
 * is timed once and keeps its weight).  The ticks are real: their features reach the members.
 * Call with the batch's device current. */
vca_status vca_batch_split_weight(vca_batch* b, float weight);
vca_status vca_batch_autotune(vca_batch* b, const vca_frame_ref* frames, int32_t reps, float* weight,
                              float* ms_per_tick);

/* ---- Failure-path test hook ----------------------------------------------------------------
 * Every wait of the tensor-core kernel (on a barrier that a copy, an MMA or another role
 * completes) gives up after a time limit: the CTA raises a flag, stops its roles, waits for its
 * own copies and MMAs, frees its tensor memory and returns, and the push's (or tick's) features
 * are reported lost with VCA_E_TIMEOUT (by the read or sync that meets them, and by every later
 * read of one of those frames).  After such a report the analyzer (or each member of the batch)
 * restarts its h chain: the lost frames' energies are no previous-frame state, so the next frame
 * pushed after the report has h = 0 (a push queued before the report still compares with them).  These calls exercise that path without any fault: wait_limit_ns sets
 * the limit for the analyzer's (batch's) launches from now on (0: the default, about 2 s), and
 * withhold_tile >= 0 makes the next push's (tick's first launch's) work item of that number -- its
 * index among the launch's 128x128 tiles -- get no copies, so the wait for it runs out; -1 none.
 * No counterpart in the paper.  VCA_E_UNSUPPORTED for the CUDA-core form (it has no waits). */
vca_status vca_debug_wait(vca_analyzer* a, int64_t wait_limit_ns, int32_t withhold_tile);
vca_status vca_batch_debug_wait(vca_batch* b, int64_t wait_limit_ns, int32_t withhold_tile);

/* ---- Serving runtime ----------------------------------------------------------------------
 *
 * A server holds live channels (one analyzer each, h state kept on the device between segments)
 * and runs a scheduler thread of its own.  A channel's producer (a decoder writing into device
 * memory, say) fills one of the channel's two segment slots -- device buffers owned by the
 * server -- and submits it.  The scheduler follows one of two policies (vca_server_set_policy):
 *   VCA_SERVE_SEGMENTS (default): a segment whose frames have landed is one work item, pushed to
 *     the channel's own analyzer in vca_push_frames calls of up to 128 frames on the channel's
 *     own stream, so channels run side by side and a segment waits only for its own frames;
 *   VCA_SERVE_TICKS: frame-interleaved continuous batching, each tick analysing the next frame
 *     of every channel that has a submitted segment (one batched tick, vca_batch_tick), so
 *     channels join and leave ticks as segments arrive and finish; all channels then share
 *     block size, chroma format and low_pass (the batch rule).
 * A finished segment appears in vca_server_poll with its submit and feature-ready times (steady
 * clock, ns).  Admission is by device memory: a channel costs its analyzer's state (which under
 * the segments policy holds the block values of up to 2 x 128 frames) plus its two segment slots
 * (2 x max_segment_frames frames); vca_server_add_channel gives VCA_E_NOMEM when the budget
 * cannot hold it.  No counterpart in the paper (its analyzer runs one video at a time). */
typedef struct vca_server vca_server;
enum { VCA_SERVE_SEGMENTS = 0, VCA_SERVE_TICKS = 1 };

typedef struct {
  int32_t channel;
  int32_t status;      /* VCA_OK, or the error that ended the segment */
  uint64_t tag;        /* the caller's tag from vca_server_submit */
  int64_t first_frame; /* the channel's frame index of the segment's first frame */
  int32_t n_frames;
  int32_t pad;
  int64_t submit_ns;   /* steady clock at vca_server_submit */
  int64_t ready_ns;    /* steady clock when the last frame's features reached the host */
} vca_segment_done;

typedef struct {
  int64_t ticks, frames, launches;  /* ticks: batched ticks (VCA_SERVE_TICKS) or pushes (segments) */
  int64_t budget_bytes, used_bytes;
  int32_t channels;
  int32_t pad;
} vca_server_stats_t;

/* device_budget_bytes = 0: 90 % of the device memory free now.  Starts the scheduler thread
 * on the current device. */
vca_status vca_server_create(size_t device_budget_bytes, vca_server** out);
/* VCA_SERVE_SEGMENTS or VCA_SERVE_TICKS; before the first vca_server_add_channel (VCA_E_STATE
 * after it), VCA_E_ARG for any other value. */
vca_status vca_server_set_policy(vca_server* s, int32_t policy);
/* Admits a channel (cfg as for vca_open; max_batch is ignored) whose segments hold up to
 * max_segment_frames frames; *id receives its number. */
vca_status vca_server_add_channel(vca_server* s, const vca_config* cfg, int32_t max_segment_frames, int32_t* id);
/* Device address of frame 0 of segment slot `slot` (0 or 1) of channel id (pitches in *frame0)
 * and the byte strides between its frames: the slot holds the Y planes of all its frames one
 * after another, then the U planes, then the V planes. */
vca_status vca_server_segment_buffer(vca_server* s, int32_t id, int32_t slot, vca_frame_ref* frame0,
                                     int64_t* frame_stride_y, int64_t* frame_stride_uv);
/* Queues the n_frames frames of slot `slot` of channel id.  ready_event (a cudaEvent_t, or
 * NULL): the frames are analysed only after it completes.  VCA_E_AGAIN while that slot is still
 * queued or being analysed. */
vca_status vca_server_submit(vca_server* s, int32_t id, int32_t slot, int32_t n_frames, uint64_t tag,
                             void* ready_event);
/* Copies n_frames frames (frame i: Y at frame0.y + i * frame_stride_y bytes, U and V at
 * frame0.u / frame0.v + i * frame_stride_uv; device or host memory) into a free segment slot of
 * channel id on the
 * server's copy stream, after ready_event (or NULL), and queues them.  The source may be reused
 * once the segment is finished.  VCA_E_AGAIN when both slots are in use.  One thread at a time
 * may submit to a channel. */
vca_status vca_server_submit_frames(vca_server* s, int32_t id, const vca_frame_ref* frame0, int64_t frame_stride_y,
                                    int64_t frame_stride_uv, int32_t n_frames, uint64_t tag, void* ready_event);
/* Up to max finished segments, oldest first; *n receives the count (0 if none). */
vca_status vca_server_poll(vca_server* s, vca_segment_done* out, int32_t max, int32_t* n);
/* Features of frame `frame` of channel id (waits for them). */
vca_status vca_server_read_features(vca_server* s, int32_t id, int64_t frame, vca_frame_features* out);
vca_status vca_server_stats(vca_server* s, vca_server_stats_t* st);
/* Finishes every submitted segment, stops the scheduler and frees the channels. */
vca_status vca_server_destroy(vca_server* s);

/* ---- SI / TI ---------------------------------------------------------------------------
 *
 * The spatial and temporal information features that the paper compares VCA with (Section 2:
 * SI = max over frames of std[Sobel(F)], TI = max over frames of std[F_t - F_{t-1}]), on the luma
 * plane in raw sample values.  Per frame: SI_t = population standard deviation over the
 * interior pixels (the one-pixel border excluded) of sqrt(Gx^2 + Gy^2), Gx and Gy the 3x3 Sobel
 * responses; TI_t = population standard deviation over all pixels of F_t - F_{t-1}, 0 for the
 * first frame.  The sequence values are the maxima (TI over t >= 1).  Sums of Gx^2 + Gy^2 and of
 * the differences are exact integers; the gradient magnitudes use an FP32 square root and are
 * summed in 2^-16 fixed point; the deviations are formed in FP64. */
typedef struct vca_siti vca_siti;
typedef struct {
  int64_t frame;
  double SI, TI;
} vca_siti_features;

/* width, height in [3, 16384]; bit_depth 8, 10 or 12; up to max_batch frames per push. */
vca_status vca_siti_open(int32_t width, int32_t height, int32_t bit_depth, int32_t max_batch, void* cuda_stream,
                         vca_siti** out);
/* n_frames luma planes (pitch and frame stride in bytes; device planes 16-byte aligned, or host
 * planes with on_device = 0).  Returns when their features are on the host. */
vca_status vca_siti_push(vca_siti* s, const void* y, int64_t pitch, int64_t frame_stride, int32_t n_frames,
                         int32_t on_device);
vca_status vca_siti_read(vca_siti* s, int64_t frame, vca_siti_features* out);
vca_status vca_siti_sequence(vca_siti* s, double* si, double* ti, int64_t* frames);
vca_status vca_siti_launch_count(vca_siti* s, int64_t* launches);
vca_status vca_siti_close(vca_siti* s);

/* Frame features from per-block values already on the device, without allocating any device
 * memory.  The paper has no counterpart: this is a runtime convenience for callers that must not
 * call the CUDA allocator on their hot path (a serving loop that has budgeted all device memory
 * up front to decide admission; a host thread with other streams in flight, for which an
 * allocation may block and a free waits for the whole device).
 *
 * It runs the analyzer's own frame reduction: per frame f, E_P = sum_k H_{P,k} / (C N_P^2),
 * L_P = sum_k L_{P,k} / C, h = sum_k |H_{Y,k,f} - H_{Y,k,f-1}| / (C w^2), each sum exact in
 * 2^-23 fixed point and rounded once to FP64.
 *   block_values  device, [n_frames][6][C] FP32, rows H_Y, L_Y, H_U, L_U, H_V, L_V (C =
 *                 blocks_per_plane, raster block order) of a 4:2:0 analyzer; read only.  Each
 *                 value in [0, 2^30) is summed exactly after truncation toward zero to a
 *                 multiple of 2^-23 (every value the analyzer writes is a multiple already: 0
 *                 or at least 1).  Values outside [0, 2^30) -- negative (also -0.0), NaN,
 *                 infinite or too large -- count as 0.
 *   block_size    luma block size w: 32 or 16.  Chroma blocks are taken as w/2 x w/2 (4:2:0):
 *                 block values of a 4:4:4 analyzer would give E_U and E_V 4 times too large.
 *   n_frames      1 .. 256: the frames the fixed scratch holds; more gives VCA_E_ARG.
 *   prev_H_Y      device, C FP32 luma energies of the frame before frame 0, or NULL for h = 0
 *                 on frame 0.
 *   last_H_Y      device, C FP32, receives H_Y of frame n_frames - 1 (the next call's
 *                 prev_H_Y); its bytes must overlap neither prev_H_Y nor block_values.
 *   features      device, n_frames x 8 doubles: E_Y, h, L_Y, E_U, E_V, L_U, L_V, 0.
 *   cuda_stream   the stream the work is queued on (NULL: legacy default stream); the call
 *                 returns without waiting.
 * The caller owns every buffer.  The scratch is one fixed array per device: calls that may
 * overlap on the device (unordered streams, several host threads) race on it; order them.
 * The first call on a device looks the array up and may load the module, so make it before
 * any stream capture.  VCA_E_ARG for NULL outputs, a bad block size, a size outside the
 * limits or overlapping buffers; VCA_E_CUDA if the lookup or the launch fails. */
vca_status vca_reduce_frames_noalloc(const float* block_values, int64_t blocks_per_plane, int32_t block_size,
                                     int32_t n_frames, const float* prev_H_Y, float* last_H_Y,
                                     double* features, void* cuda_stream);

/* Static description of a status code, and the calling thread's last error message. */
const char* vca_status_str(vca_status s);
const char* vca_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VCA_H */
