// fkd_internal.cuh -- geometry, device tables and kernel launchers shared by
// the CUDA translation units of libfkd (not part of the public ABI).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fkd.h"

namespace fkd {

constexpr int kMaxLayers = 12;  // O <= 6 with intra-octaves
constexpr int kMaxBins = 4096;  // N_r * N_c

// Pyramid kernel: one CTA builds every layer of a 96 x 96 tile of c_0. 96 is a
// multiple of 3 * 2^5, so for O <= 6 every layer's tile is whole: the 2x2 box
// and the 3x3 -> 2x2 resampling never cross a tile edge.
constexpr int kPyrTile = 96;
constexpr int kPyrThreads = 256;

// Detection tile (output pixels) handled by one warp: one 4-pixel word per
// lane per row, kDetTW wide and kDetTH[shape] high. The staged input adds a
// 4-pixel halo (3 for the ring, 1 for the suppression neighbours), widened to
// 16 bytes left and right so that rows load as aligned 16-byte vectors.
// The launch shape (tile height, warps per CTA, CTAs per SM) is chosen per
// stream or group, by default or by the autotuner.
constexpr int kDetTW = 128;
constexpr int kDetShapes = 3;
constexpr int kDetTH[kDetShapes] = {8, 16, 24};
constexpr int kDetDefaultShape = 1;
// kDetTH[shape] where device code needs it with a run-time index
__host__ __device__ constexpr int det_th(int shape) { return shape == 0 ? 8 : shape == 1 ? 16 : 24; }
static_assert(det_th(0) == kDetTH[0] && det_th(1) == kDetTH[1] && det_th(2) == kDetTH[2], "tile heights");
constexpr int kDetMaxThreads = 256;  // warps per CTA: 4 or 8

// Launch shape of the detection kernel.
struct DetLaunch {
  int shape;  // index into kDetTH
  int warps;  // warps (tiles in flight) per CTA
  int grid;   // persistent CTAs
};

// Assembly: a chunk is a band of whole rows of one layer of the per-frame
// keypoint bitmap, about kAsmChunkWords words, handled by one CTA.
constexpr int kAsmThreads = 256;
constexpr int kAsmWordsPerThread = 8;
constexpr int kAsmChunkWords = kAsmThreads * kAsmWordsPerThread;

// Mask kernel: one CTA per bin walks the batch's frames 256 at a time.
constexpr int kMaskThreads = 256;

// Programmatic dependent launch. A kernel launched with pdl_launch may be
// scheduled while the kernel before it on the stream is still running; it
// waits in pdl_wait() -- its first statement -- until that kernel has
// completed and its memory is visible, so only launch latency overlaps.
// pdl_trigger() lets the next kernel be scheduled once every CTA of this one
// has started. Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Asynchronous 16-byte global -> shared copy (cp.async, LDGSTS): `bytes` of
// the 16 are read (0..16) and the rest of the destination is zero-filled.
// The source must be 16-byte aligned whenever bytes > 0.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, int bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gsrc), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// ------------------------------------------------------------ debug checks
// Built with FKD_CHECK=1 (the debug library libfkd_check.so), the kernels
// check the index of every shared- and global-memory access listed below
// against its range; an index outside records (site, index, limit) in a
// device record of its translation unit and the access is skipped -- no
// fault, no trap. The host collects the records after each launch sequence
// and returns the first as FKD_E_CUDA. Release builds compile the checks away.
#ifndef FKD_CHECK
#define FKD_CHECK 0
#endif
enum CheckSite : unsigned {
  kChkDetStage = 1,  // detection: staged input (shared) / its source rows
  kChkDetUnits,      // detection: (row, word) unit list
  kChkDetWlist,      // detection: candidate word list
  kChkDetScore,      // detection: score map (shared)
  kChkDetPass,       // detection: pass / keypoint bitmap words (shared)
  kChkDetBits,       // detection: the frame's keypoint bitmap (global)
  kChkDetDscore,     // detection: the frame's score map (global)
  kChkDetCells,      // detection: per-cell detection counts (global)
  kChkPyrSmem,       // pyramid: a level's tile (shared)
  kChkPyrBins,       // pyramid: per-bin change sums (shared / global)
  kChkAsmWords,      // assembly: a chunk's words (shared / global)
  kChkAsmPos,        // assembly: the chunk's list of set bits (shared)
  kChkAsmSrc,        // assembly: source frames of the chunk's bins (shared)
  kChkAsmBins,       // assembly: the kept set's per-bin counts (global)
  kChkSites
};
struct CheckRecord {
  unsigned hit, site;
  long long index, limit;
};
// every translation unit of a debug build registers a function that takes
// (and clears) its record
using CheckTake = int (*)(CheckRecord*);
int register_check(CheckTake take);
#if FKD_CHECK
static __device__ CheckRecord g_check_rec;  // one per translation unit
__device__ __forceinline__ bool check_index(unsigned site, long long idx, long long limit) {
  if (idx >= 0 && idx < limit) return true;
  if (atomicCAS(&g_check_rec.hit, 0u, 1u) == 0u) {
    g_check_rec.site = site;
    g_check_rec.index = idx;
    g_check_rec.limit = limit;
  }
  return false;
}
static int take_check_record(CheckRecord* out) {
  CheckRecord r{};
  if (cudaMemcpyFromSymbol(&r, g_check_rec, sizeof r) != cudaSuccess || !r.hit) return 0;
  const CheckRecord zero{};
  cudaMemcpyToSymbol(g_check_rec, &zero, sizeof zero);
  *out = r;
  return 1;
}
static const int g_check_registered = register_check(take_check_record);
#define FKD_IDX(site, idx, limit) ::fkd::check_index((site), (long long)(idx), (long long)(limit))
#else
#define FKD_IDX(site, idx, limit) true
#endif
// Host: after the stream's work has finished, FKD_OK or FKD_E_CUDA with the
// first recorded failure (debug builds; release builds return FKD_OK).
int collect_checks();
const char* check_site_name(unsigned site);

struct LayerGeom {
  int w, h, S;         // size and scale code 2*sigma
  int pitch;           // row pitch in the pyramid and score buffers (multiple of 16)
  long long pyr_off;   // byte offset in a frame's pyramid buffer (layers >= 1), -1 for c_0
  long long score_off; // byte offset in a frame's score map (all layers)
  int wpr;             // 32-bit words per row of the keypoint bitmap
  long long bit_off;   // word offset of the layer in a frame's bitmap
  int col_off;         // offset of the layer in the colblk table (w entries)
  int wb_off;          // offset of the layer in the wbins table (wpr entries)
  int row_off;         // offset of the layer in the rowblk table (h entries)
  int xs_off;          // offset of the layer in the xstart table (N_c + 1 entries)
};

struct Geometry {
  int W, H, L, O, intra;
  int N_r, N_c, NB;
  int mask_layer;
  LayerGeom layer[kMaxLayers];
  long long pyr_bytes;    // per frame, layers >= 1
  long long score_bytes;  // per frame, all layers
  long long bit_words;    // per frame, all layers
  int n_tiles;            // detection tiles per frame (current tile shape)
  int det_shape;          // current tile shape (index into kDetTH)
  int n_chunks;           // assembly chunks per frame
  int n_cells;            // (chunk, bin) cells per frame
  int pyr_tiles_x, pyr_tiles_y;
};

// One assembly chunk: rows y0 .. y1-1 of one layer, spanning bin rows
// rb0 .. rb1. Its cells -- the parts of the chunk inside one bin each --
// are numbered cell0 + (r - rb0) * N_c + c for bin (r, c).
struct AsmChunk {
  int layer, y0, y1;
  int cell0, rb0, rb1;
};

// One detection tile: a kDetTW x kDetTH[shape] rectangle of one layer, its
// pixel count inside the layer, and the rectangle of bins its pixels map to
// (inclusive), for the activity test.
struct DetTile {
  uint16_t layer, tx, ty, area;
  uint16_t rb0, rb1, cb0, cb1;
};

// Read-only device tables of a stream (built once on the host).
struct Tables {
  const uint16_t* colblk;  // per layer, per x: bin column of the pixel
  const uint16_t* rowblk;  // per layer, per y: bin row of the pixel
  const int* xstart;       // per layer, per bin column c: first x with colblk >= c
  const uint32_t* npix;    // per bin: pixels of the mask layer in it
  const DetTile* tiles;    // per detection tile of a frame
  const AsmChunk* chunks;  // per assembly chunk of a frame
  const uint32_t* wbins;   // per layer, per bitmap word column: first | last bin column << 16
  const uint32_t* wmask;   // per layer, per bitmap word column: bits of the word in its first bin
  const int* rowchunk;     // per layer, per y: the assembly chunk holding the row
  const int* rowcell;      // per layer, per y: cell of (the row's chunk, bin row, bin column 0)
  const int* bincell_off;  // per bin: start of its cells in bincell (NB + 1 entries)
  const int* bincell;      // the cells of every bin (all layers), bin after bin
};

// Arguments of one batch of T consecutive frames of one stream.
struct Batch {
  int T;
  long long first_frame;           // stream index of frame 0 of the batch
  const uint8_t* frames;           // frame k at frames + k * frame_stride
  long long frame_stride;
  int pitch;
  const uint8_t* prev;             // the frame before the batch (nullptr at stream start)
  int prev_pitch;
  int c0_vec;                      // frames and pitch allow 16-byte loads
};

struct Params {
  int T_I, T_H, t, mask_mode;
  int nms_scale;  // 1: suppression also against the adjacent layers
};

// Device scratch of a stream, sized for T_max frames.
struct Scratch {
  uint8_t* pyr;                    // [T_max][pyr_bytes]
  unsigned long long* bsum;        // [NB][bsum_stride]: bin-major, frame k at bin*bsum_stride + k; kept zero
  int bsum_stride;                 // T_max (1 in groups)
  uint8_t* mask;                   // [T_max][NB], then 4 bytes of padding
  int* src;                        // [T_max][NB]: batch frame whose detections the bin shows, -1 = kept set
  uint32_t* work;                  // [T_max * n_tiles] active (frame, tile) items
  uint32_t* work_count;            // [1]
  uint32_t* det_bits;              // [T_max][bit_words]
  uint8_t* det_score;              // [T_max][score_bytes]
  uint32_t* chunk_counts;          // [T_max][n_chunks]
  uint32_t* dcnt;                  // keypoint binning: [T_max][n_cells] detections of each frame in
                                   //   each cell (null for the other mask modes)
  uint8_t* alive;                  // [NB]: keypoint binning in spans, bins active at the next frame
  uint32_t* merged;                // [T_max][bit_words]: D_n bitmap of every frame of the batch
  uint32_t* frame_totals;          // [T_max]
  unsigned long long* out_base;    // [2]: running output offset (ping-pong)
  int* overflow;                   // [1]: bit 0 records dropped past a capacity, bit 1 a tile copy that did not land
  unsigned long long* tile_stats;  // [2]: detection tiles and their layer pixels (running totals)
  uint8_t* ml_prev;                // the mask layer of the stream's last frame (mask layers above c_0)
  uint32_t* pmask;                 // [T_max][bit_words]: per-pixel masks, FKD_MASK_IDP only (else null)
  uint8_t* pyr_last;               // FKD_MASK_IDP: layers >= 1 of the stream's last frame
};

// The kept keypoint set D_{n-1} as a per-pixel bitmap + score map, ping-pong.
struct State {
  const uint32_t* bits_in;
  const uint8_t* score_in;
  const uint32_t* cnt_in;          // keypoints per bin (for keypoint binning)
  uint32_t* bits_out;
  uint8_t* score_out;
  uint32_t* cnt_out;
};

struct Output {
  fkd_keypoint* rec;
  long long cap;
  uint32_t* offsets;               // T + 1 entries
  int base_slot;                   // out_base slot read; the other one is written
  uint32_t* row_base;              // null, or [T][rows]: index of the first record of each layer row
  int rows;                        // layer rows per frame (all layers)
};

// Masked description: binary descriptors of D bits (D / 32 words per record,
// bit i in word i / 32 at bit i % 32) over a caller-given pattern of pairs
// with offsets within +-kDescR.
constexpr int kDescR = FKD_DESC_RADIUS;
constexpr int kDescMaxBits = FKD_DESC_MAX_BITS;
struct Describe {
  const int8_t* pattern;           // [D][4]: ax, ay, bx, by
  int D;
  uint32_t* desc;                  // descriptor of output record i at desc + i * D / 32
  const fkd_keypoint* keep_rec_in; // the kept set: the previous batch's last frame, canonical order
  const uint32_t* keep_desc_in;
  const uint32_t* keep_n_in;
  fkd_keypoint* keep_rec_out;      // this batch's last frame, for the next batch
  uint32_t* keep_desc_out;
  uint32_t* keep_n_out;
  long long keep_cap;              // records the kept set holds (K_max)
  const uint32_t* keep_row_in;     // [rows + 1]: first kept record of each layer row, then the count
  uint32_t* keep_row_out;
  uint32_t* count;                 // end index of the described records (device word)
  uint32_t* next_group;            // work counter of the new-record pass (zero between batches)
  int* missing;                    // set when a carried record's origin is absent (after an overflow)
};

// ---------------------------------------------------------------- groups
// A group runs one frame of each of many streams (any mix of sizes) per
// tick, with one launch per kernel for the whole tick. Each stream's static
// description lives in device memory (StreamDev); each tick uploads one
// TickItem per participating stream and a TickHeader with the totals. The
// group kernels are persistent (fixed grids looping over the tick's work),
// so one captured CUDA graph replays every tick whatever its composition.

// Resident description of one stream of a group (device memory).
struct StreamDev {
  Geometry g;
  Tables tb;
  Scratch s;                 // sized for one frame (T_max = 1)
  Params p;
  uint32_t* state_bits[2];
  uint8_t* state_score[2];
  uint32_t* state_cnt[2];
  uint8_t* last[2];          // copies of the stream's last two frames (c_0, pitch layer[0].pitch)
  fkd_keypoint* rec[2];      // D_n of frame n in rec[n & 1] (K_max records each)
  uint32_t* rec_offsets[2];  // [2] each: 0 and |D_n|
  long long K_max;
  // masked description (D == 0: off): descriptors of rec[n & 1] in
  // desc[n & 1], and the first record of every layer row in row_base[n & 1]
  int D;
  const int8_t* pattern;
  uint32_t* desc[2];
  uint32_t* row_base[2];
  int rows;
};

// One participating stream of a tick.
struct TickItem {
  int sid;                   // index of the stream's StreamDev
  int state_cur;             // kept-set buffer holding D_{n-1}
  long long frame_index;     // n
  const uint8_t* frame;      // I_n (device), row pitch `pitch`
  int pitch;
  int pyr_base, bin_base, tile_base, chunk_base;  // prefix sums of the tick's work
};

struct TickHeader {
  int n_items;
  int total_pyr, total_bins, total_tiles, total_chunks;
};

constexpr int kMaxTickItems = 1024;

// Group launchers (persistent grids; all asynchronous on `st`).
int group_pyramid_grid(int O, int intra);
void launch_group_pyramid(int O, int intra, const StreamDev* devs, const TickHeader* hdr,
                          const TickItem* items, int grid, cudaStream_t st);
void launch_group_mask(const StreamDev* devs, const TickHeader* hdr, const TickItem* items,
                       uint32_t* work_count, int grid, cudaStream_t st);
void launch_group_worklist(const StreamDev* devs, const TickHeader* hdr, const TickItem* items,
                           uint32_t* work, uint32_t* work_count, int grid, cudaStream_t st);
void launch_group_detect(const StreamDev* devs, const TickItem* items, const uint32_t* work,
                         const uint32_t* work_count, const DetLaunch& dl, cudaStream_t st);
void launch_group_count(const StreamDev* devs, const TickHeader* hdr, const TickItem* items,
                        int grid, cudaStream_t st);
void launch_group_emit(const StreamDev* devs, const TickHeader* hdr, const TickItem* items,
                       int grid, cudaStream_t st);

// Where one stream's result of one frame lives (device): K_max records and
// the offsets pair (0, |D_n|).
struct ResultRef {
  const fkd_keypoint* rec;
  const uint32_t* off;
  long long cap;  // records rec can hold (K_max)
};

// Serving: frames copied from device-accessible host memory (pinned) into
// device staging by one kernel for all the frames of a round.
struct UploadItem {
  const uint8_t* src;  // device-accessible address of the host frame
  long long src_pitch;
  uint8_t* dst;
  int dst_pitch, W, H;
};
void launch_upload(const UploadItem* items, int n, cudaStream_t st);

// counts[i] = |D_n| of refs[i] (may exceed its cap); offsets[i] = records
// gathered before item i, each item contributing min(count, cap), offsets[n]
// = their total; records copied to out (up to out_cap) in that order.
// `offsets` holds n + 1 words followed by the n counts.
void launch_gather(const ResultRef* refs, int n, uint32_t* offsets, fkd_keypoint* out, long long out_cap,
                   cudaStream_t st);

// Index of the item whose [base, next base) range holds j (bases ascending).
template <typename F>
__device__ __forceinline__ int find_item(int n, int j, F base_of) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base_of(mid) <= j) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Launchers (all asynchronous on `st`).
void launch_pyramid(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                    const Params& p, cudaStream_t st);
void launch_mask(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                 const Params& p, const State& state, cudaStream_t st, int reset_base_slot);
void launch_worklist(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                     cudaStream_t st, int k_lo = 0, int k_hi = -1);
// Keypoint binning in spans of frames: the masks of frames k_lo .. k_hi-1
// set to the bins still active (first: from the kept set's counts), then
// resolved exactly from the detection counts; and the source frames of a
// batch whose masks are given.
constexpr int kKbSpan = 16;
void launch_kb_span(const Geometry& g, const Batch& b, const Scratch& s, const Params& p, const State& state,
                    int k_lo, int k_hi, int first, cudaStream_t st);
void launch_kb_resolve(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s, const Params& p,
                       int k_lo, int k_hi, cudaStream_t st);
void launch_source_frames(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                          const Params& p, const State& state, cudaStream_t st, int reset_base_slot);
void launch_detect(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                   const Params& p, const DetLaunch& dl, cudaStream_t st);
void launch_count(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                  const State& state, cudaStream_t st);

void launch_emit(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                 const State& state, const Output& out, cudaStream_t st);
// FKD_MASK_IDP: per-pixel masks of every layer of the batch (Eq. 2 per
// pixel), and D_n of every frame by the per-pixel recurrence of Eq. 1.
void launch_pixel_mask(const Geometry& g, const Batch& b, const Scratch& s, const Params& p,
                       cudaStream_t st);
void launch_count_pixel(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                        const State& state, cudaStream_t st);
// CTAs of the detection kernel resident per SM for a tile shape and warp
// count (0 when it cannot launch), and the SM count.
int detect_ctas_per_sm(int shape, int warps);
int sm_count();
// Scale-space suppression of the detections of the active tiles (after the
// detection kernel): single-stream batch and group tick.
void launch_scale_nms(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                      const Params& p, cudaStream_t st);
void launch_group_scale_nms(const StreamDev* devs, const TickItem* items, const uint32_t* work,
                            const uint32_t* work_count, cudaStream_t st);

// Descriptors of a batch's records (after the emission kernel), and of a
// group tick's records for the streams that describe.
void launch_describe(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s, const Output& out,
                     const Describe& d, cudaStream_t st);
void launch_group_describe(const StreamDev* devs, const TickHeader* hdr, const TickItem* items, cudaStream_t st);

// Record a message for fkd_last_error (printf format) and return `code`.
int set_error(int code, const char* fmt, ...);

// Group internals used by the serving loop.
int group_result_ref(fkd_group* G, int id, long long frame_index, ResultRef* ref);
long long group_stream_frames(fkd_group* G, int id);
int group_stream_kmax(fkd_group* G, int id);
cudaStream_t group_cuda_stream(fkd_group* G);

}  // namespace fkd
