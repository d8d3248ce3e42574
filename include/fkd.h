/*
 * fkd.h -- C ABI of the GB300 masked keypoint detector for video.
 *
 * Method: Baroffio, Cesana, Redondi, Tagliasacchi, "Fast keypoint detection
 * in video sequences" (arXiv 1503.06959). For every frame I_n the library
 *   1. builds the scale-space pyramid of octaves c_i and intra-octaves d_i
 *      (Sec. 2; Sec. 3.1 reuses it for the mask),
 *   2. builds the detection mask M'_n on an N_r x N_c grid of bins, either by
 *      the intensity difference test (Eq. 2, Sec. 3.1) or by keypoint
 *      binning of D_{n-1} (Eqs. 3-4, Sec. 3.2), with the first frame of a
 *      stream fully active,
 *   3. runs the segment test (16-pixel radius-3 Bresenham ring, 9 contiguous
 *      pixels brighter than I_p + t or darker than I_p - t), the corner score
 *      and 3x3 non-maximum suppression on every layer, at pixels whose bin is
 *      active (Sec. 2),
 *   4. returns D_n = new detections in active bins united with the keypoints
 *      of D_{n-1} in inactive bins (Eq. 1), sorted by (layer, y, x).
 *
 * Conventions shared by every entry point:
 *   - Return value: FKD_OK (0) or a negative FKD_E_* code. Nothing throws
 *     across the ABI. fkd_last_error() returns a message for the calling
 *     thread's last failure.
 *   - Frames are 8-bit grayscale, row-major, W x H pixels, with a row pitch
 *     in bytes (pitch >= W).
 *   - "on_device" arguments say whether a pointer is CUDA device memory (1)
 *     or host memory (0). Host buffers are copied on the stream's CUDA
 *     stream; pinned host memory makes those copies asynchronous.
 *   - Each fkd_stream is bound to one CUDA stream (given at creation; NULL
 *     is the legacy default stream) and is not thread-safe: one host thread
 *     drives one fkd_stream at a time. Different fkd_streams are independent.
 *   - The library owns all device state of a stream (pyramid, masks, the
 *     kept keypoint set D_{n-1}, scratch) and frees it in
 *     fkd_destroy_stream. The caller owns every buffer it passes in.
 */
#ifndef FKD_H
#define FKD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define FKD_VERSION 3u

/* status codes */
#define FKD_OK 0
#define FKD_E_ARG (-1)      /* invalid argument or parameter                 */
#define FKD_E_CAPACITY (-2) /* output larger than the buffer given / K_max   */
#define FKD_E_BUDGET (-3)   /* admission refused: memory budget exhausted    */
#define FKD_E_CUDA (-4)     /* a CUDA call failed (message has the details)  */
#define FKD_E_TIMEOUT (-5)  /* a bounded device wait ran out                 */
#define FKD_E_STATE (-6)    /* call out of order (e.g. no frame pushed yet)  */

/* mask modes (Sec. 3: "two efficient algorithms" plus plain detection) */
#define FKD_MASK_FULL 0 /* every bin active: the plain per-frame detector      */
#define FKD_MASK_ID 1   /* intensity difference detection mask, Eq. 2         */
#define FKD_MASK_KB 2   /* keypoint binning detection mask, Eqs. 3-4          */
#define FKD_MASK_IDP 3  /* Eq. 2 per pixel of every layer, option (i) of      */
                        /* Sec. 3.1: |L_n - L_{n-1}| > T_I at a pixel of      */
                        /* layer l activates that pixel of layer l; single    */
                        /* streams only (not groups or servers); the bin mask */
                        /* of fkd_get_mask is then all ones                   */

/*
 * Parameters, named as the paper names them.
 *   N_r, N_c    bin grid rows and columns (Sec. 3.2); a bin covers
 *               S_x = W/N_c by S_y = H/N_r pixels. 1 <= N_c <= W,
 *               1 <= N_r <= H, N_r*N_c <= 4096.
 *   T_I         intensity-difference threshold (Eq. 2). A bin is active when
 *               the mean of |L_n - L_{n-1}| over its pixels of the mask layer
 *               exceeds T_I (evaluated exactly as sum > T_I * count). >= 0.
 *   T_H         keypoint-binning threshold (Eq. 4): a bin is active when it
 *               held at least T_H keypoints of D_{n-1}. >= 0.
 *   O           octaves (Sec. 2), 1..6.
 *   intra       1: add the intra-octave layers d_i (scale 1.5 * 2^i);
 *               0: octaves only.
 *   t           segment-test threshold (Sec. 2), 1..255.
 *   n           contiguous ring pixels the test asks for; must be 9.
 *   mask_mode   FKD_MASK_FULL / FKD_MASK_ID / FKD_MASK_KB.
 *   mask_layer  layer the intensity difference is taken on (layer index as
 *               in fkd_layer_info); -1 selects the coarsest octave c_{O-1},
 *               the paper's choice in its experiments (Sec. 4).
 *   K_max       capacity of the kept keypoint set of one frame (>= 1).
 *   T_max       most frames one fkd_push_frames call may carry (>= 1); it
 *               sizes the per-batch scratch.
 *   nms_scale   0: a detection is a strict 3x3 maximum of scores within its
 *               layer; 1: it must also be strictly above every score of the
 *               3x3 window, in the layers just below and above in scale,
 *               around the pixel containing its centre (Sec. 2, "3x3
 *               scale-space neighbourhood"). 0 or 1.
 */
typedef struct {
  uint32_t version; /* FKD_VERSION */
  int32_t N_r, N_c;
  int32_t T_I;
  int32_t T_H;
  int32_t O;
  int32_t intra;
  int32_t t;
  int32_t n;
  int32_t mask_mode;
  int32_t mask_layer;
  int32_t K_max;
  int32_t T_max;
  int32_t nms_scale;
} fkd_params;

/*
 * One keypoint, 8 bytes. x, y are layer-pixel coordinates; the image
 * position is (floor(x*S/2), floor(y*S/2)) and the scale sigma = S/2, with S
 * the layer's scale code from fkd_layer_info (feature tuple of Sec. 3).
 * score is the largest threshold for which the segment test still fires
 * (>= t). flags bit 0 (FKD_KP_PROPAGATED) marks a keypoint carried over from
 * D_{n-1} because its bin was inactive (Eq. 1).
 */
typedef struct {
  uint16_t x, y;
  uint8_t layer, score;
  uint16_t flags;
} fkd_keypoint;
#define FKD_KP_PROPAGATED 1u

typedef struct fkd_stream fkd_stream;

/* Message of the calling thread's last failed call ("" if none). */
const char* fkd_last_error(void);

/* Fill *p with defaults: 8 x 8 bins, T_I 4, T_H 1, O 1, intra 0, t 20, n 9,
 * FKD_MASK_ID on layer 0, K_max 65536, T_max 1. */
int fkd_params_default(fkd_params* p);

/*
 * Create a stream for W x H frames (1..16384 each). cuda_stream is a
 * cudaStream_t (NULL: legacy default stream). On success *out owns the
 * device state; release it with fkd_destroy_stream.
 * Errors: FKD_E_ARG (bad parameters or sizes), FKD_E_CUDA (allocation).
 */
int fkd_create_stream(const fkd_params* p, int W, int H, void* cuda_stream, fkd_stream** out);

/* Synchronise the stream and free everything it owns. NULL is a no-op. */
int fkd_destroy_stream(fkd_stream* s);

/* Number of pyramid layers (O, or 2*O with intra-octaves). */
int fkd_num_layers(const fkd_stream* s, int* L);

/*
 * Geometry of layer `layer` (0 .. L-1, ordered by scale: c_0, d_0, c_1, d_1,
 * ... with intra-octaves, c_0, c_1, ... without). w, h: layer size; S: scale
 * code 2*sigma (2, 3, 4, 6, 8, 12, ...). c_{i+1} is c_i halved (floor);
 * d_0 has 2*floor(W/3) x 2*floor(H/3) pixels; d_{i+1} is d_i halved.
 * Any output pointer may be NULL. Errors: FKD_E_ARG.
 */
int fkd_layer_info(const fkd_stream* s, int layer, int* w, int* h, int* S);

/*
 * Process the next frame of the stream (steps 1-4 above), asynchronously on
 * the stream's CUDA stream. The result D_n replaces D_{n-1} and is read with
 * fkd_get_keypoints.
 *   frame, pitch: the W x H frame.
 *   on_device = 0: host memory, copied to device memory the stream owns. From
 *     pageable memory the copy completes before the call returns and the
 *     buffer may be reused at once; from pinned (page-locked) memory the copy
 *     is asynchronous and the buffer must stay unmodified until the next
 *     fkd_get_keypoints, fkd_get_mask or fkd_synchronize on this stream.
 *   on_device = 1: device memory read in place. It must stay valid and
 *     unmodified until the NEXT fkd_push_frame / fkd_push_frames call on this
 *     stream has completed, because that call compares against it (Eq. 2).
 * Errors: FKD_E_ARG, FKD_E_CUDA.
 */
int fkd_push_frame(fkd_stream* s, const uint8_t* frame, size_t pitch, int on_device);

/*
 * Wait for the last pushed frame and copy D_n, sorted by (layer, y, x), to
 * host memory `out` (room for `cap` records). *n_out receives |D_n| even
 * when it does not fit. Errors: FKD_E_STATE (no frame pushed yet),
 * FKD_E_CAPACITY (|D_n| > cap, or |D_n| > K_max: the set was truncated to
 * K_max on the device; nothing is copied in either case), FKD_E_CUDA.
 */
int fkd_get_keypoints(fkd_stream* s, fkd_keypoint* out, size_t cap, size_t* n_out);

/* Wait for the last pushed frame and copy its mask M'_n (N_r*N_c bytes, row
 * major, 1 = active bin) to host memory `out`. Errors: FKD_E_STATE, FKD_E_CUDA. */
int fkd_get_mask(fkd_stream* s, uint8_t* out);

/* FKD_MASK_IDP: the last frame's per-pixel mask of `layer` into host memory
 * (w*h bytes of 0/1, row-major, w and h as fkd_layer_info gives). Waits.
 * Errors: FKD_E_ARG (not FKD_MASK_IDP, bad layer), FKD_E_STATE (no frame). */
int fkd_get_pixel_mask(fkd_stream* s, int layer, uint8_t* out);

/*
 * Process T consecutive frames of the stream in one batched launch sequence
 * (1 <= T <= T_max). Output is bit-identical to T fkd_push_frame calls.
 *   frames: frame k at frames + k*frame_stride, rows `pitch` bytes apart;
 *     on_device as for fkd_push_frame (device frames must additionally stay
 *     valid until this call has completed; the last one as for
 *     fkd_push_frame).
 *   out, cap, offsets: D_{n0+k} for every k, concatenated; offsets[k] is the
 *     index of its first record and offsets[T] the total (T+1 entries).
 *   masks: NULL, or T*N_r*N_c bytes receiving M'_{n0+k}.
 *   out_on_device: 1 if out, offsets and masks are device memory. The call
 *     is then asynchronous on the stream's CUDA stream; records past `cap`
 *     are dropped, offsets still give the full counts, and the overflow is
 *     reported as FKD_E_CAPACITY by the next fkd_synchronize. 0: host
 *     memory; the call waits and returns FKD_E_CAPACITY itself (outputs
 *     filled up to cap).
 * With FKD_MASK_KB each frame's mask depends on the previous frame's
 * keypoints. A bin below T_H stays inactive (its part of D_n is D_{n-1}'s,
 * Eq. 1, so its count cannot grow), so the call detects spans of 16 frames
 * on the bins active at each span's first frame and then resolves every
 * frame's exact mask from the detection counts: the results are those of
 * frame-after-frame processing. Its profile puts the spans in the detect
 * stage (mask and worklist stages empty).
 * Errors: FKD_E_ARG, FKD_E_CAPACITY, FKD_E_CUDA.
 */
int fkd_push_frames(fkd_stream* s, const uint8_t* frames, size_t pitch, size_t frame_stride, int T,
                    int on_device, fkd_keypoint* out, size_t cap, uint32_t* offsets, uint8_t* masks,
                    int out_on_device);

/* Wait for all work of the stream; report a deferred FKD_E_CAPACITY from an
 * asynchronous fkd_push_frames (and clear it). */
int fkd_synchronize(fkd_stream* s);

/* Frames processed so far (the index n of the next frame). */
int fkd_frame_count(const fkd_stream* s, int64_t* n);

/*
 * Device pointers of the last frame's result, for callers that keep working
 * on the GPU: *records (K_max entries, the first *count_dev valid), *count_dev
 * (one uint32 on the device). Valid until the next push on this stream.
 */
int fkd_device_keypoints(fkd_stream* s, const fkd_keypoint** records, const uint32_t** count_dev);

/*
 * Forget the stream's history: the next frame is treated as the first one
 * (all bins active, nothing carried over), as after a scene cut. Waits for
 * the stream's pending work. Errors: FKD_E_ARG.
 */
int fkd_reset_stream(fkd_stream* s);

/*
 * Masked description (Sec. 3: the mask decides where keypoints are detected
 * and described, and a carried keypoint keeps its descriptor; Sec. 2: each
 * bit of a binary descriptor compares the smoothed intensities of one pair of
 * pixels sampled around the keypoint). The paper gives no sampling pattern,
 * so the caller supplies one.
 *   pattern: D rows of four int8 (ax, ay, bx, by), offsets in pixels of the
 *     keypoint's layer, each within +-FKD_DESC_RADIUS; host memory, copied.
 *     NULL with D = 0 turns description off.
 *   D: descriptor bits, a multiple of 32 in 32 .. FKD_DESC_MAX_BITS.
 * Bit i of the descriptor of keypoint (x, y) of layer l is set iff the sum of
 * the 5x5 pixels of layer l around (x + ax_i, y + ay_i) is below the sum
 * around (x + bx_i, y + by_i), pixel coordinates clamped to the layer; it is
 * bit i % 8 of byte i / 8. The pattern is upright (no orientation). Only
 * keypoints detected in a frame are described, on that frame's layer; a
 * carried keypoint (FKD_KP_PROPAGATED) keeps the descriptor it had in the
 * previous frame. Resets the stream (waits for its pending work). Streams of
 * a group or a server describe through fkd_group_set_descriptor and
 * fkd_server_set_descriptor.
 * Errors: FKD_E_ARG (D or an offset out of range), FKD_E_CUDA.
 */
#define FKD_DESC_RADIUS 13
#define FKD_DESC_MAX_BITS 512
int fkd_set_descriptor(fkd_stream* s, const int8_t* pattern, int D);

/*
 * Descriptors of the records of the last fkd_push_frame (the set
 * fkd_get_keypoints returns) or fkd_push_frames call (one per record its
 * `out` received, in that order), D/8 bytes each, into `out`: host memory,
 * or device memory with out_on_device = 1. *n_out = the number of those
 * records; at most `cap` descriptors are copied (out = NULL with cap = 0
 * only reports the count). Waits for the stream.
 * Errors: FKD_E_STATE (description off, or no frame pushed since it was
 * set), FKD_E_CAPACITY (more than cap: the first cap are copied),
 * FKD_E_ARG, FKD_E_CUDA.
 */
int fkd_get_descriptors(fkd_stream* s, uint8_t* out, size_t cap, size_t* n_out, int out_on_device);

/*
 * Per-stage timing of the launch sequence, for profiling. While enabled,
 * every batch records CUDA events around each of its kernels on the stream's
 * CUDA stream. fkd_profile_read waits for the stream, adds the elapsed times
 * of all batches since the last read (reset != 0 clears them afterwards).
 * Stages: FKD_STAGE_PYRAMID (pyramid + per-bin change sums), _MASK (mask and
 * source frames), _WORKLIST (active-tile compaction), _DETECT (segment test,
 * score, suppression), _COUNT and _EMIT (assembly of D_n), _DESCRIBE (masked
 * description; its launches count only batches that described).
 * tile_pixels counts the layer pixels inside the detection tiles processed
 * (each is one input byte the detection kernel must read), tiles the tiles.
 */
#define FKD_STAGE_PYRAMID 0
#define FKD_STAGE_MASK 1
#define FKD_STAGE_WORKLIST 2
#define FKD_STAGE_DETECT 3
#define FKD_STAGE_COUNT 4
#define FKD_STAGE_EMIT 5
#define FKD_STAGE_DESCRIBE 6
#define FKD_NUM_STAGES 7
typedef struct {
  double ms[FKD_NUM_STAGES];       /* summed kernel time per stage            */
  uint64_t launches[FKD_NUM_STAGES];
  uint64_t batches;                /* launch sequences recorded              */
  uint64_t frames;                 /* frames those sequences processed       */
  uint64_t tiles;                  /* detection tiles processed              */
  uint64_t tile_pixels;            /* layer pixels in those tiles            */
} fkd_profile;
int fkd_profile_enable(fkd_stream* s, int on);
int fkd_profile_read(fkd_stream* s, fkd_profile* out, int reset);

/*
 * Launch shape of the detection kernel and its autotuner. The paper (Sec. 2,
 * Sec. 3.1) fixes what is computed, not how the work is cut: the segment test
 * runs on tiles of tile_w x tile_h output pixels of one layer (tile_w = 128,
 * one 4-pixel word per lane), one tile per warp at a time, warps_per_cta
 * tiles in flight per CTA, ctas_per_sm persistent CTAs per SM. Smaller tiles
 * follow the active bins more closely (less work outside them); taller ones
 * re-read less halo. Every shape gives bit-identical keypoints.
 */
#define FKD_TILE_W 128
typedef struct {
  int32_t tile_h;        /* 8, 16 or 24 output rows per tile            */
  int32_t warps_per_cta; /* 4 or 8 tiles in flight per CTA              */
  int32_t ctas_per_sm;   /* 1 .. resident limit of that shape           */
} fkd_launch_config;

/* The shape the stream uses now (tile_h 16, 8 warps, as many CTAs per SM as
 * fit, unless set or tuned). Errors: FKD_E_ARG. */
int fkd_get_launch_config(const fkd_stream* s, fkd_launch_config* out);

/* Use shape *c for the stream's next batches (waits for pending work).
 * Errors: FKD_E_ARG (tile_h, warps_per_cta outside the lists above, or
 * ctas_per_sm outside 1 .. the number that fits on an SM). */
int fkd_set_launch_config(fkd_stream* s, const fkd_launch_config* c);

/* Autotuner: times a batch of the T frames at `frames` (device memory, row
 * pitch `pitch`, frame k at frames + k * frame_stride; T <= T_max) under every
 * candidate shape (tile_h x warps_per_cta x ctas_per_sm), `reps` timed runs
 * each after one untimed run, keeps the fastest (smallest of its runs, CUDA
 * events around the whole launch sequence; the current shape is timed first
 * and another replaces it only when more than 2 % faster), and returns it in
 * *best and its time in *best_ms (either may be NULL). Each run starts from a reset stream,
 * so the stream's history is discarded: tune before the first push. Results
 * of the runs are dropped. Errors: FKD_E_ARG, FKD_E_CUDA. */
int fkd_autotune(fkd_stream* s, const uint8_t* frames, size_t pitch, size_t frame_stride, int T, int reps,
                 fkd_launch_config* best, float* best_ms);

/*
 * Groups: many streams, one frame of each per tick, one launch sequence.
 *
 * A group serves many independent video streams of any sizes (for example a
 * mix of 320x240 ... 1920x1080 cameras). Each call to fkd_group_tick takes
 * the next frame of any subset of the group's streams and runs steps 1-4 for
 * all of them with one launch per kernel (persistent grids looping over the
 * tick's work), optionally replayed from a captured CUDA graph. The result of
 * every stream is bit-identical to feeding its frames to its own fkd_stream
 * one by one. All streams of a group share O and intra (the pyramid kernel
 * is compiled per octave count); every other parameter is per stream.
 * Streams keep on the device what the next frame's mask needs (copies of
 * their last two frames for change sums on c_0, or of the last frame's
 * coarser mask layer), so a tick's frames may come from transient buffers.
 */
typedef struct fkd_group fkd_group;

/* Create an empty group for streams with O octaves (1..6) and intra
 * (0 or 1), bound to cuda_stream (NULL: legacy default stream).
 * Errors: FKD_E_ARG, FKD_E_CUDA. */
int fkd_group_create(int O, int intra, void* cuda_stream, fkd_group** out);

/* Wait for the group's work and free it and all its streams. NULL: no-op. */
int fkd_group_destroy(fkd_group* g);

/* Add a stream (p->O and p->intra must match the group's; p->T_max is
 * ignored). *stream_id receives its index (ids are not reused). *bytes, if
 * not NULL, receives the device memory the stream holds. Waits for the
 * group's pending work. Errors: FKD_E_ARG, FKD_E_CUDA. */
int fkd_group_add_stream(fkd_group* g, const fkd_params* p, int W, int H, int* stream_id,
                         size_t* bytes);

/* Remove a stream and free its device memory (waits for pending work).
 * Errors: FKD_E_ARG (unknown id). */
int fkd_group_remove_stream(fkd_group* g, int stream_id);

/* One tick: frame frames[i] (device memory, row pitch pitches[i]) is the next
 * frame of stream ids[i], for i < n; a stream appears at most once. The
 * frames must stay valid until the tick has run (fkd_group_synchronize, or
 * any later call that waits). Asynchronous. Errors: FKD_E_ARG, FKD_E_CUDA. */
int fkd_group_tick(fkd_group* g, int n, const int* ids, const uint8_t* const* frames,
                   const size_t* pitches);

/* Replay ticks from captured CUDA graphs (on, the default) or launch the
 * kernels one by one (off). */
int fkd_group_use_graph(fkd_group* g, int on);

/* Wait for the group's work. Errors: FKD_E_CUDA. */
int fkd_group_synchronize(fkd_group* g);

/* The last tick's D_n of stream `id` (sorted by (layer, y, x)) into host
 * memory, as fkd_get_keypoints. Waits. Errors: FKD_E_ARG, FKD_E_STATE (the
 * stream has no frame yet), FKD_E_CAPACITY. */
int fkd_group_get_keypoints(fkd_group* g, int id, fkd_keypoint* out, size_t cap, size_t* n_out);

/* The last tick's mask of stream `id` (N_r*N_c bytes) into host memory. */
int fkd_group_get_mask(fkd_group* g, int id, uint8_t* out);

/* Device pointers of stream `id`'s last result: K_max records and the device
 * uint32 count. Valid until its next tick. Errors: FKD_E_ARG, FKD_E_STATE. */
int fkd_group_device_keypoints(fkd_group* g, int id, const fkd_keypoint** records,
                               const uint32_t** count_dev);

/* Masked description for a stream of the group (as fkd_set_descriptor),
 * before its first tick; the description pass then runs in the stream's ticks.
 * Errors: FKD_E_ARG, FKD_E_STATE (the stream has ticked), FKD_E_CUDA. */
int fkd_group_set_descriptor(fkd_group* G, int stream_id, const int8_t* pattern, int D);

/* Descriptors of the stream's last frame (the records fkd_group_get_keypoints
 * returns, in their order), D/8 bytes each, at most `cap`, into host memory
 * (device memory with out_on_device = 1); out = NULL with cap = 0 only
 * reports the count. Waits. Errors: FKD_E_ARG, FKD_E_STATE (no
 * frame yet, or the stream does not describe), FKD_E_CAPACITY, FKD_E_CUDA. */
int fkd_group_get_descriptors(fkd_group* G, int stream_id, uint8_t* out, size_t cap, size_t* n_out,
                              int out_on_device);

/* Summed CUDA-event times of the group's kernels over the ticks since the
 * last read (same stages and semantics as fkd_profile_read; `frames` counts
 * the frames of those ticks). */
int fkd_group_profile_enable(fkd_group* g, int on);
int fkd_group_profile_read(fkd_group* g, fkd_profile* out, int reset);

/* The detection launch shape of the whole group (one persistent launch runs
 * the tiles of all its streams), as fkd_get/set_launch_config. Setting it
 * waits for pending work and re-captures the tick graphs on the next tick. */
int fkd_group_get_launch_config(const fkd_group* g, fkd_launch_config* out);
int fkd_group_set_launch_config(fkd_group* g, const fkd_launch_config* c);

/* Group autotuner: m ticks over streams ids[0..n-1], tick j taking frame
 * frames[j * n + i] (device memory, row pitch pitches[i]) for stream ids[i],
 * timed under every candidate shape as fkd_autotune does (reps timed
 * sequences after one untimed one, each starting from reset streams). Keeps
 * the fastest shape; every stream of the group is reset afterwards. Errors:
 * FKD_E_ARG, FKD_E_CUDA. */
int fkd_group_autotune(fkd_group* g, int n, const int* ids, int m, const uint8_t* const* frames,
                       const size_t* pitches, int reps, fkd_launch_config* best, float* best_ms);

/*
 * Serving loop: frames of many streams arriving at any time.
 *
 * A server owns a group (above) and a worker thread. fkd_server_submit
 * copies a host frame into the stream's queue (a ring of 4 pinned frames) and
 * returns; the worker continuously batches: each round it takes the oldest
 * waiting frame of every stream that has one -- frames that arrived while
 * the previous round was on the GPU join the next round -- uploads them,
 * runs one group tick for all of them, and, while that tick runs, brings the
 * previous round's keypoints back to the streams' result queues. Streams are
 * admitted against a device-memory budget and release their memory when
 * closed. Latency is measured per frame from its arrival time (submit) to
 * its keypoints being on the host. Every stream's results are bit-identical
 * to running it alone. All functions are thread-safe.
 */
typedef struct fkd_server fkd_server;

typedef struct {
  uint64_t frames_done;       /* frames whose keypoints reached the host      */
  uint64_t ticks;             /* rounds launched                               */
  uint64_t rejected_frames;   /* submits refused because a queue was full      */
  uint64_t rejected_streams;  /* opens refused by the memory budget            */
  double p50_ms, p99_ms;      /* per-frame latency, arrival to results on host */
  double max_ms, mean_ms;
  double fps;                 /* frames done per second, first arrival to last */
  double mean_batch;          /* frames per round                              */
  size_t bytes_in_use;        /* device bytes charged to the budget            */
  size_t budget_bytes;
} fkd_server_stats;

/* Create a server for streams with O octaves and intra (as fkd_group_create),
 * a device-memory budget in bytes (covering its own buffers and every
 * admitted stream), and room for max_tick_keypoints records per round.
 * Errors: FKD_E_ARG, FKD_E_BUDGET (the server's own buffers exceed the
 * budget), FKD_E_CUDA. */
int fkd_server_create(int O, int intra, size_t budget_bytes, size_t max_tick_keypoints,
                      fkd_server** out);

/* Stop the worker (frames on the GPU finish), free everything. NULL: no-op. */
int fkd_server_destroy(fkd_server* s);

/* Admit a stream (p->O and p->intra as the server's). Errors: FKD_E_BUDGET
 * (its device memory would exceed the budget, or 1024 streams are open),
 * FKD_E_ARG, FKD_E_CUDA. */
int fkd_server_open_stream(fkd_server* s, const fkd_params* p, int W, int H, int* id);

/* Close a stream: frames already on the GPU finish, waiting frames and
 * unread results are dropped, its memory returns to the budget. */
int fkd_server_close_stream(fkd_server* s, int id);

/* Queue the next frame of stream `id` (host memory, copied before the call
 * returns). arrival_ns: its arrival time on the steady clock
 * (CLOCK_MONOTONIC), or <= 0 for "now". Errors: FKD_E_CAPACITY (4 frames of
 * this stream already waiting; the frame is not queued), FKD_E_ARG,
 * FKD_E_CUDA (an earlier round failed). */
int fkd_server_submit(fkd_server* s, int id, const uint8_t* frame, size_t pitch, int64_t arrival_ns);

/* As fkd_server_submit, but the frame is queued by reference and uploaded
 * from where it is (no copy on the host; pinned memory makes the upload
 * asynchronous): it must stay valid and unmodified until its result has
 * been collected (fkd_server_poll returns it, or fkd_server_drain returns).
 * For callers whose frames already sit in pinned buffers (a capture or
 * decode pipeline), and for load tests at rates a host copy cannot feed. */
int fkd_server_submit_ref(fkd_server* s, int id, const uint8_t* frame, size_t pitch, int64_t arrival_ns);

/* keep = 0: finished frames are counted and timed (fkd_server_get_stats)
 * but their keypoints are not kept for fkd_server_poll (load tests that
 * never poll); keep = 1 (the default): kept until polled. */
int fkd_server_keep_results(fkd_server* s, int keep);

/* Load generator: submits frame i of the n given (host memory, row pitch
 * pitches[i]) to stream ids[i] by reference (fkd_server_submit_ref) at its
 * arrival time arrival_ns[i] on the steady clock (CLOCK_MONOTONIC;
 * non-decreasing), waiting in this thread (sleeping through long gaps,
 * spinning through short ones) so that no interpreter sits in the loop.
 * A frame whose stream already has 4 frames waiting is dropped and counted
 * in *refused (may be NULL): offered load beyond what the loop serves shows
 * as dropped frames and queueing latency. The frames must stay valid until
 * fkd_server_drain returns. Errors: FKD_E_ARG (NULL argument, decreasing
 * arrival times), and those of fkd_server_submit_ref. */
int fkd_server_replay(fkd_server* s, int n, const int* ids, const uint8_t* const* frames, const size_t* pitches,
                      const int64_t* arrival_ns, uint64_t* refused);

/* Take the oldest finished frame of stream `id`: its index n and D_n
 * (sorted by (layer, y, x)) into host memory. Errors: FKD_E_STATE (nothing
 * finished yet), FKD_E_CAPACITY (more than cap records: the result stays
 * queued; or the frame exceeded K_max or the round's capacity: the result
 * is dropped), FKD_E_ARG. */
int fkd_server_poll(fkd_server* s, int id, int64_t* frame_index, fkd_keypoint* out, size_t cap,
                    size_t* n_out);

/* Masked description for stream `id` (as fkd_set_descriptor), before its
 * first frame; the descriptor buffers count against the budget. Errors:
 * FKD_E_ARG, FKD_E_STATE (frames already submitted), FKD_E_BUDGET, FKD_E_CUDA. */
int fkd_server_set_descriptor(fkd_server* s, int id, const int8_t* pattern, int D);

/* Descriptors of the result the last fkd_server_poll of stream `id` returned
 * (one per keypoint, in its order), D/8 bytes each, into host memory, at most
 * `cap`; out = NULL with cap = 0 only reports the count. Errors: FKD_E_ARG,
 * FKD_E_STATE (the stream does not describe, or nothing polled yet),
 * FKD_E_CAPACITY. */
int fkd_server_get_descriptors(fkd_server* s, int id, uint8_t* out, size_t cap, size_t* n_out);

/* Wait until no frame is waiting or on the GPU. Errors: FKD_E_TIMEOUT. */
int fkd_server_drain(fkd_server* s, int timeout_ms);

/* Statistics since creation or the last reset (reset != 0 clears them). */
int fkd_server_get_stats(fkd_server* s, fkd_server_stats* out, int reset);

/*
 * Debug build. The library also builds as libfkd_check.so (compiled with
 * FKD_CHECK=1; the paper has no counterpart: it stands in for a memory
 * checker). Its kernels check the index of their shared- and global-memory
 * accesses (staging, unit and word lists, score maps and bitmaps of the
 * detection pass; the pyramid's level tiles and bin sums; the assembly's
 * chunk words, set-bit lists and source frames): an index out of range is
 * recorded in a device word and the access skipped -- no fault and no trap
 * -- and the call that launched the work waits for it and returns
 * FKD_E_CUDA naming the access, the index and its range. Every device
 * allocation of a stream lies between two 256-byte guard bands of a known
 * byte. Release builds skip all of this.
 *   fkd_check_build: 1 in the debug build, 0 in the release build.
 *   fkd_check_guards: FKD_OK if every guard band of the stream's allocations
 *     is intact (always in the release build), else FKD_E_CUDA naming the
 *     allocation's size and the byte that changed. Waits for the stream.
 *   fkd_group_check_guards: the same for every stream of a group.
 */
int fkd_check_build(void);
int fkd_check_guards(const fkd_stream* s);
int fkd_group_check_guards(fkd_group* g);

/*
 * Allocation-free variant (the paper has no counterpart; it exists for
 * callers of this library that cannot let it allocate device memory: an
 * application that gives all GPU memory to its own allocator or budget at
 * start-up, a plugin inside a host program that owns the device memory, a
 * real-time loop that must not pay for cudaMalloc / cudaFree and the
 * synchronisation they imply).
 *
 * fkd_id_mask_noalloc computes the intensity-difference detection mask of
 * one frame pair -- bin (r, c) is 1 when the sum of |cur - prev| over its
 * pixels of the full-resolution frame exceeds T_I times their number, the
 * test fkd_push_frames applies with FKD_MASK_ID and mask_layer 0 -- without
 * allocating anything. cur, prev: device W x H frames sharing `pitch`;
 * mask_out: device buffer of N_r*N_c bytes (row-major); cuda_stream: the
 * cudaStream_t to run on (NULL: legacy default stream). Asynchronous.
 *
 * Its per-bin sums live in a fixed array of FKD_NOALLOC_MAX_BINS 64-bit
 * counters (32 KiB) in this library's device memory, present on every GPU
 * that loads the library until the process exits. The first call made in a
 * given CUDA context (normally a device's primary context) looks the array's
 * address up in that context (cudaGetSymbolAddress) and remembers it for
 * the context; make that first call outside stream capture: a first call
 * whose stream is being captured fails with FKD_E_STATE and launches
 * nothing. Every call clears the counters it uses and then reuses the same
 * array, so calls that overlap on the GPU (on different streams, or
 * different host threads) race and give wrong masks: serialise them.
 * Errors: FKD_E_ARG (NULL buffer, sizes outside 1..16384, pitch < W, a bin
 * grid that does not fit the frame, N_r*N_c > FKD_NOALLOC_MAX_BINS, T_I < 0),
 * FKD_E_STATE (see above), FKD_E_CUDA (also when a CUDA error from earlier
 * work on the calling thread is still pending: it is reported, left pending
 * for the caller, and nothing is launched). Calls no cudaMalloc, cudaFree or
 * other allocating routine.
 */
#define FKD_NOALLOC_MAX_BINS 4096
int fkd_id_mask_noalloc(const uint8_t* cur, const uint8_t* prev, int W, int H, size_t pitch, int N_r,
                        int N_c, int T_I, uint8_t* mask_out, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* FKD_H */
