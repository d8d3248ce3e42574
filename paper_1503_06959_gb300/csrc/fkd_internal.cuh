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

// Detection kernel tile (output pixels); the input tile adds a 4-pixel halo
// (3 for the ring, 1 for the suppression neighbours), widened to 16 bytes on
// each side so that rows load as aligned 16-byte vectors.
constexpr int kDetTW = 64;
constexpr int kDetTH = 16;
constexpr int kDetThreads = 256;

// Assembly: words of the per-frame keypoint bitmap handled by one CTA.
constexpr int kAsmThreads = 256;
constexpr int kAsmWordsPerThread = 8;
constexpr int kAsmChunkWords = kAsmThreads * kAsmWordsPerThread;

struct LayerGeom {
  int w, h, S;         // size and scale code 2*sigma
  int pitch;           // row pitch in the pyramid and score buffers (multiple of 16)
  long long pyr_off;   // byte offset in a frame's pyramid buffer (layers >= 1), -1 for c_0
  long long score_off; // byte offset in a frame's score map (all layers)
  int wpr;             // 32-bit words per row of the keypoint bitmap
  long long bit_off;   // word offset of the layer in a frame's bitmap
  int col_off;         // offset of the layer in the colblk table (w entries)
  int row_off;         // offset of the layer in the rowblk table (h entries)
  int xs_off;          // offset of the layer in the xstart table (N_c + 1 entries)
  int tile_off;        // first detection tile of the layer
};

struct Geometry {
  int W, H, L, O, intra;
  int N_r, N_c, NB;
  int mask_layer;
  LayerGeom layer[kMaxLayers];
  long long pyr_bytes;    // per frame, layers >= 1
  long long score_bytes;  // per frame, all layers
  long long bit_words;    // per frame, all layers
  int n_tiles;            // detection tiles per frame
  int n_chunks;           // assembly chunks per frame
  int pyr_tiles_x, pyr_tiles_y;
};

// One detection tile: a kDetTW x kDetTH rectangle of one layer, and the
// rectangle of bins its pixels map to (inclusive), for the activity test.
struct DetTile {
  uint16_t layer, tx, ty, pad;
  uint16_t rb0, rb1, cb0, cb1;
};

// Read-only device tables of a stream (built once on the host).
struct Tables {
  const uint16_t* colblk;  // per layer, per x: bin column of the pixel
  const uint16_t* rowblk;  // per layer, per y: bin row of the pixel
  const int* xstart;       // per layer, per bin column c: first x with colblk >= c
  const uint32_t* npix;    // per bin: pixels of the mask layer in it
  const DetTile* tiles;    // per detection tile of a frame
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
};

// Device scratch of a stream, sized for T_max frames.
struct Scratch {
  uint8_t* pyr;                    // [T_max][pyr_bytes]
  unsigned long long* bsum;        // [T_max][NB]; kept zero between batches
  uint8_t* mask;                   // [T_max][NB]
  int* src;                        // [T_max][NB]: batch frame whose detections the bin shows, -1 = kept set
  uint32_t* work;                  // [T_max * n_tiles] active (frame, tile) items
  uint32_t* work_count;            // [1]
  uint32_t* det_bits;              // [T_max][bit_words]
  uint8_t* det_score;              // [T_max][score_bytes]
  uint32_t* chunk_counts;          // [T_max][n_chunks]
  uint32_t* frame_totals;          // [T_max]
  unsigned long long* out_base;    // [2]: running output offset (ping-pong)
  int* overflow;                   // [1]
  unsigned long long* tile_stats;  // [2]: detection tiles and their layer pixels (running totals)
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
};

// Launchers (all asynchronous on `st`).
void launch_pyramid(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                    const Params& p, cudaStream_t st);
void launch_mask(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                 const Params& p, const State& state, cudaStream_t st, int reset_base_slot);
void launch_worklist(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                     cudaStream_t st);
void launch_detect(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                   const Params& p, int grid, cudaStream_t st);
void launch_count(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                  const State& state, cudaStream_t st);
void launch_emit(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                 const State& state, const Output& out, cudaStream_t st);
int detect_grid_size();

}  // namespace fkd
