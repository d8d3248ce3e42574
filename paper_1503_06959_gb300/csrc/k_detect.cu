// k_detect.cu -- masked segment test, corner score and 3x3 non-maximum
// suppression (Sec. 2) over the active detection tiles of a batch, and the
// optional scale-space suppression against the adjacent layers.
//
// Every warp works alone on one 128 x tile_h tile of one layer at a time (no
// block-wide barriers; each warp owns a slice of shared memory), pulling
// (frame, tile) items from the compacted list of active tiles; tile_h (8, 16
// or 24), warps per CTA and CTAs per SM are the launch shape the caller sets
// or the autotuner picks. Per tile:
//   A. stage the tile plus a 4-pixel halo (3 for the ring, 1 for the
//      suppression neighbours), widened to 16 bytes left and right:
//      (tile_h + 8) rows x 160 bytes, copied with cp.async, zero-filled
//      outside the layer;
//   B. for each 4-pixel word and score row, decide from the bin mask (or the
//      per-pixel mask) whether any pixel there, or one of its neighbours, is
//      in an active region; prefilter the words that are, one word per lane
//      per row, with packed byte arithmetic: a pixel can pass the segment
//      test at threshold t only if two adjacent compass points of its ring
//      (12, 3, 6, 9 o'clock) differ from it by more than t, because every
//      9-pixel arc of the 16-pixel ring holds two adjacent compass points;
//      words with survivors are compacted with one ballot per row;
//   C. expand those words into candidate pixels (four bit-position ballots
//      per 32 words) and score them exactly, two per lane in 16-bit lanes:
//      with I_k the ring values, the bright score is max over arcs of (min
//      over the arc of I_k) - I_p and the dark one I_p - min over arcs of
//      (max over the arc); arc extrema are 3-input extrema of 3-input extrema;
//   D. a pixel of the tile is kept when its score is >= t and strictly above
//      its 8 neighbours' (scores below t count as 0, which never changes the
//      outcome); write the tile's bitmap words and the kept scores.
// Bins are not consulted beyond B: assembly takes each pixel from the frame
// its bin points to, so the kernel only has to be right on the tiles it runs.
#include <algorithm>
#include <type_traits>

#include "fkd_internal.cuh"

namespace fkd {
namespace {

constexpr int TW = kDetTW;   // output pixels per tile row: one 4-pixel word per lane
constexpr int IN_W = TW + 32;  // input row: x in [x0-16, x0+TW+16)
constexpr int SC_P = TW + 8;   // score row pitch; column = x - x0 + 4
constexpr int RING = 256;      // candidate pixels waiting to be scored, per warp (power of two)
constexpr int PASS = 256;      // passing-pixel list per warp (entries); beyond it the pass bitmap is scanned
constexpr int MIN_BLOCKS = 2;  // 256-thread CTAs resident per SM the register budget is sized for
static_assert(TW == 32 * 4, "one 4-pixel word per lane per row");
static_assert(RING >= 64 + 128 && (RING & (RING - 1)) == 0, "a round leaves < 64, an expansion adds <= 128");

// Per-warp sizes for a tile height TH (output rows y0 .. y0+TH-1).
template <int TH>
struct Shape {
  static constexpr int IN_H = TH + 8;            // input rows: y in [y0-4, y0+TH+4)
  static constexpr int SC_H = TH + 2;            // score rows: y in [y0-1, y0+TH]
  static constexpr int IN_BYTES = IN_W * IN_H;
  static constexpr int SC_BYTES = SC_P * SC_H;
  static constexpr int DET_WORDS = TH * (TW / 32);
  static constexpr int WLIST = (SC_H * 34 + 7) / 8 * 8;  // candidate words: 32 per score row + 2 edge words
  // input buffer(s), score map, keypoint and pass bitmaps, candidate words,
  // candidate ring and pass list
  static constexpr int WARP_SMEM = IN_BYTES + SC_BYTES + 2 * DET_WORDS * 4 + WLIST * 4 + RING * 2 + PASS * 2;
  static_assert(TH % 8 == 0 && TH + 4 <= 32, "one lane per dilated score row; whole 32-word rounds");
  static_assert(IN_BYTES % 16 == 0 && SC_BYTES % 16 == 0, "16-byte aligned slices");
};

// Per byte: bit 7 set where e >= T1 (T1 in 1..255, the same in every byte).
__device__ __forceinline__ uint32_t bytes_ge(uint32_t e, uint32_t t1_low7, bool t1_high) {
  const uint32_t u = (e | 0x80808080u) - t1_low7;  // no borrow crosses a byte
  return t1_high ? (e & u) : (e | u);
}

__device__ __forceinline__ uint32_t ld32(const uint8_t* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// Prefilter of the word at input offset o (4 pixels): bit 7 of each byte set
// where two adjacent compass points differ from the pixel by more than t.
__device__ __forceinline__ uint32_t prefilter(const uint8_t* in, int o, uint32_t t1_low7,
                                              bool t1_high) {
  const uint32_t C = ld32(in + o), Cp = ld32(in + o - 4), Cn = ld32(in + o + 4);
  const uint32_t N = ld32(in + o - 3 * IN_W), S = ld32(in + o + 3 * IN_W);
  const uint32_t E = __funnelshift_r(C, Cn, 24);  // bytes x+3 .. x+6
  const uint32_t Wd = __funnelshift_r(Cp, C, 8);  // bytes x-3 .. x
  const uint32_t gN = bytes_ge(__vabsdiffu4(N, C), t1_low7, t1_high);
  const uint32_t gS = bytes_ge(__vabsdiffu4(S, C), t1_low7, t1_high);
  const uint32_t gE = bytes_ge(__vabsdiffu4(E, C), t1_low7, t1_high);
  const uint32_t gW = bytes_ge(__vabsdiffu4(Wd, C), t1_low7, t1_high);
  return (gN | gS) & (gE | gW) & 0x80808080u;
}

// 16 ring samples, ring order from straight above clockwise (y down).
#define FKD_RING(X)                                                                     \
  X(0, 0, -3) X(1, 1, -3) X(2, 2, -2) X(3, 3, -1) X(4, 3, 0) X(5, 3, 1) X(6, 2, 2)    \
  X(7, 1, 3) X(8, 0, 3) X(9, -1, 3) X(10, -2, 2) X(11, -3, 1) X(12, -3, 0)            \
  X(13, -3, -1) X(14, -2, -2) X(15, -1, -3)

// Exact scores of the pixels at input offsets o1, o2, in the two 16-bit lanes.
__device__ __forceinline__ uint32_t score_pair(const uint8_t* in, int o1, int o2) {
  uint32_t v[16];
#define FKD_LOAD(k, dx, dy)                                        \
  v[k] = __byte_perm((uint32_t)in[o1 + (dy) * IN_W + (dx)],        \
                     (uint32_t)in[o2 + (dy) * IN_W + (dx)], 0x5410);
  FKD_RING(FKD_LOAD)
#undef FKD_LOAD
  const uint32_t ip = __byte_perm((uint32_t)in[o1], (uint32_t)in[o2], 0x5410);
  uint32_t mn3[16], mx3[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    mn3[j] = __vimin3_u16x2(v[j], v[(j + 1) & 15], v[(j + 2) & 15]);
    mx3[j] = __vimax3_u16x2(v[j], v[(j + 1) & 15], v[(j + 2) & 15]);
  }
  uint32_t a = 0u, bmin = 0xffffffffu;
#pragma unroll
  for (int j = 0; j < 16; j += 2) {
    const uint32_t a0 = __vimin3_u16x2(mn3[j], mn3[(j + 3) & 15], mn3[(j + 6) & 15]);
    const uint32_t a1 = __vimin3_u16x2(mn3[j + 1], mn3[(j + 4) & 15], mn3[(j + 7) & 15]);
    a = __vimax3_u16x2(a, a0, a1);
    const uint32_t b0 = __vimax3_u16x2(mx3[j], mx3[(j + 3) & 15], mx3[(j + 6) & 15]);
    const uint32_t b1 = __vimax3_u16x2(mx3[j + 1], mx3[(j + 4) & 15], mx3[(j + 7) & 15]);
    bmin = __vimin3_u16x2(bmin, b0, b1);
  }
  // bright - 1 = a - (I_p + 1); dark - 1 = (I_p - 1) - bmin; clamp at 0
  const uint32_t sb = __vsub2(a, __vadd2(ip, 0x00010001u));
  const uint32_t sd = __vsub2(__vsub2(ip, 0x00010001u), bmin);
  return __vimax_s16x2_relu(sb, sd);
}

// One (frame, tile) work item, with everything the kernel body needs.
struct Item {
  int x0, y0, w, h;          // tile origin, layer size
  const uint8_t* src;        // the layer (row 0)
  int pitch;
  uint32_t* bits;            // the frame's keypoint bitmap of this layer (row 0)
  int wpr;
  uint8_t* dscore;           // the frame's score map of this layer (row 0)
  int dpitch;
  int t;                     // segment-test threshold
  const uint8_t* mask;       // the frame's bin mask (null: every bin active)
  const uint16_t* colblk;    // bin column of each layer column
  const uint16_t* rowblk;    // bin row of each layer row
  int N_c;
  const uint32_t* pmask;     // per-pixel mask of the layer (row 0; FKD_MASK_IDP), else null
  uint32_t* dcnt;            // the frame's detections per cell (keypoint binning), else null
  int n_cells;               // cells per frame
  const int* rowcell;        // the layer's first cell of each row
  const uint32_t* wbins;     // the layer's bin columns of each bitmap word column
  const uint32_t* wmask;     // the layer's bits of each word column in its first bin
  const int* xstart;         // the layer's first column of each bin column
};

// Add (sign = 1) or remove (sign = -1) the detections of bitmap word `word`,
// word column wx of a row whose cells start at `cells`, to the counts of the
// cells its pixels lie in: words inside one or two bin columns split by the
// precomputed mask, wider ones (coarse layers, narrow bins) walk their bins.
__device__ __forceinline__ void count_word_v(uint32_t* cells, uint32_t word, int wx, int w, uint32_t wb,
                                             uint32_t m, const int* xstart, int sign) {
  const int c_lo = wb & 0xffffu, c_hi = wb >> 16;
  if (c_hi - c_lo <= 1) {
    const int n0 = __popc(word & m), n1 = __popc(word & ~m);
    if (n0) atomicAdd(cells + c_lo, (uint32_t)(sign * n0));
    if (n1) atomicAdd(cells + c_hi, (uint32_t)(sign * n1));
    return;
  }
  const int xlo = wx * 32, xhi = min(xlo + 32, w);
  for (int c = c_lo; c <= c_hi; ++c) {
    const int a = max(xstart[c], xlo) - xlo, e = min(xstart[c + 1], xhi) - xlo;
    if (e <= a) continue;
    const uint32_t m = (e - a == 32) ? 0xffffffffu : (((1u << (e - a)) - 1u) << a);
    const int n = __popc(word & m);
    if (n) atomicAdd(cells + c, (uint32_t)(sign * n));
  }
}
__device__ __forceinline__ void count_word(uint32_t* cells, uint32_t word, int wx, int w, const uint32_t* wbins,
                                           const uint32_t* wmask, const int* xstart, int sign) {
  count_word_v(cells, word, wx, w, wbins[wx], wmask[wx], xstart, sign);
}

// One layer of a frame, for the scale-space suppression. Its scale code S
// is 2^sh or 3 * 2^sh (sh >= 1 or the 3 alone), so n / (2 S) is a shift and
// at most one division by the constant 3.
struct LayerView {
  const uint8_t* p;  // null: no such layer
  int pitch, w, h, S;
  __device__ __forceinline__ int div2S(int n) const {
    const int q = n >> (__ffs(S) - 1 + 1);  // n / (2 * 2^v2(S))
    return (S & (S - 1)) ? q / 3 : q;       // S = 3 * 2^k: one more / 3
  }
};

// What the scale-space suppression needs of a (frame, tile) work item.
struct ScaleItem {
  bool on;              // the stream asked for it
  int layer, L, th, tx, ty, h, S;
  uint32_t* bits;       // the frame's keypoint bitmap of the layer (row 0)
  int wpr;
  const uint8_t* dscore;
  int dpitch;
  LayerView adj[2];     // the layers just below and above in scale
  int w;                // layer width
  uint32_t* dcnt;       // as Item: the cell counts of the detections (null: none kept)
  const int* rowcell;
  const uint32_t* wbins;
  const uint32_t* wmask;
  const int* xstart;
};

// Work items of one stream's batch of T frames.
struct SingleSrc {
  Geometry g;
  Batch b;
  Scratch s;
  Tables tb;
  Params p;
  __device__ __forceinline__ uint32_t count() const { return *s.work_count; }
  __device__ __forceinline__ uint32_t wi_at(uint32_t item) const { return s.work[item]; }
  template <int TH>
  __device__ __forceinline__ Item decode(uint32_t wi) const {
    const DetTile tile = tb.tiles[wi % (uint32_t)g.n_tiles];
    const int k = (int)(wi / (uint32_t)g.n_tiles);
    const LayerGeom& lg = g.layer[tile.layer];
    Item it;
    it.w = lg.w;
    it.h = lg.h;
    it.x0 = tile.tx * TW;
    it.y0 = tile.ty * TH;
    if (tile.layer == 0) {
      it.src = b.frames + (long long)k * b.frame_stride;
      it.pitch = b.pitch;
    } else {
      it.src = s.pyr + (long long)k * g.pyr_bytes + lg.pyr_off;
      it.pitch = lg.pitch;
    }
    it.bits = s.det_bits + (long long)k * g.bit_words + lg.bit_off;
    it.wpr = lg.wpr;
    it.dscore = s.det_score + (long long)k * g.score_bytes + lg.score_off;
    it.dpitch = lg.pitch;
    it.t = p.t;
    it.mask = p.mask_mode == FKD_MASK_FULL ? nullptr : s.mask + (long long)k * g.NB;
    it.colblk = tb.colblk + lg.col_off;
    it.rowblk = tb.rowblk + lg.row_off;
    it.N_c = g.N_c;
    it.pmask = s.pmask ? s.pmask + (long long)k * g.bit_words + lg.bit_off : nullptr;
    it.dcnt = s.dcnt ? s.dcnt + (long long)k * g.n_cells : nullptr;
    it.n_cells = g.n_cells;
    it.rowcell = tb.rowcell + lg.row_off;
    it.wbins = tb.wbins + lg.wb_off;
    it.wmask = tb.wmask + lg.wb_off;
    it.xstart = tb.xstart + lg.xs_off;
    return it;
  }
  __device__ __forceinline__ ScaleItem scale_item(uint32_t item) const {
    const uint32_t wi = s.work[item];
    const DetTile tile = tb.tiles[wi % (uint32_t)g.n_tiles];
    const int k = (int)(wi / (uint32_t)g.n_tiles);
    ScaleItem si;
    si.on = p.nms_scale != 0;
    si.layer = tile.layer;
    si.L = g.L;
    si.th = det_th(g.det_shape);
    si.tx = tile.tx;
    si.ty = tile.ty;
    const LayerGeom& lg = g.layer[tile.layer];
    si.h = lg.h;
    si.S = lg.S;
    si.bits = s.det_bits + (long long)k * g.bit_words + lg.bit_off;
    si.wpr = lg.wpr;
    si.dscore = s.det_score + (long long)k * g.score_bytes + lg.score_off;
    si.dpitch = lg.pitch;
    si.w = lg.w;
    si.dcnt = s.dcnt ? s.dcnt + (long long)k * g.n_cells : nullptr;
    si.rowcell = tb.rowcell + lg.row_off;
    si.wbins = tb.wbins + lg.wb_off;
    si.wmask = tb.wmask + lg.wb_off;
    si.xstart = tb.xstart + lg.xs_off;
    for (int j = 0; j < 2; ++j) {
      const int m = tile.layer + (j ? 1 : -1);
      LayerView& v = si.adj[j];
      if (m < 0 || m >= g.L) {
        v = LayerView{nullptr, 0, 0, 0, 2};
        continue;
      }
      const LayerGeom& lm = g.layer[m];
      v.w = lm.w;
      v.h = lm.h;
      v.S = lm.S;
      if (m == 0) {
        v.p = b.frames + (long long)k * b.frame_stride;
        v.pitch = b.pitch;
      } else {
        v.p = s.pyr + (long long)k * g.pyr_bytes + lm.pyr_off;
        v.pitch = lm.pitch;
      }
    }
    return si;
  }
};

// Work items of a group tick (one frame of each of many streams).
struct GroupSrc {
  const StreamDev* devs;
  const TickItem* items;
  const uint32_t* work;
  const uint32_t* work_count;
  __device__ __forceinline__ uint32_t count() const { return *work_count; }
  __device__ __forceinline__ uint32_t wi_at(uint32_t item) const { return work[item]; }
  template <int TH>
  __device__ __forceinline__ Item decode(uint32_t wi) const {
    const TickItem ti = items[wi >> 22];
    const StreamDev& d = devs[ti.sid];
    const DetTile tile = d.tb.tiles[wi & 0x3fffffu];
    const LayerGeom& lg = d.g.layer[tile.layer];
    Item it;
    it.w = lg.w;
    it.h = lg.h;
    it.x0 = tile.tx * TW;
    it.y0 = tile.ty * TH;
    if (tile.layer == 0) {
      it.src = ti.frame;
      it.pitch = ti.pitch;
    } else {
      it.src = d.s.pyr + lg.pyr_off;
      it.pitch = lg.pitch;
    }
    it.bits = d.s.det_bits + lg.bit_off;
    it.wpr = lg.wpr;
    it.dscore = d.s.det_score + lg.score_off;
    it.dpitch = lg.pitch;
    it.t = d.p.t;
    it.mask = d.p.mask_mode == FKD_MASK_FULL ? nullptr : d.s.mask;
    it.colblk = d.tb.colblk + lg.col_off;
    it.rowblk = d.tb.rowblk + lg.row_off;
    it.N_c = d.g.N_c;
    it.pmask = nullptr;  // groups use bin masks
    it.dcnt = d.s.dcnt;
    it.n_cells = d.g.n_cells;
    it.rowcell = d.tb.rowcell + lg.row_off;
    it.wbins = d.tb.wbins + lg.wb_off;
    it.wmask = d.tb.wmask + lg.wb_off;
    it.xstart = d.tb.xstart + lg.xs_off;
    return it;
  }
  __device__ __forceinline__ ScaleItem scale_item(uint32_t item) const {
    const uint32_t wi = work[item];
    const TickItem ti = items[wi >> 22];
    const StreamDev& d = devs[ti.sid];
    const DetTile tile = d.tb.tiles[wi & 0x3fffffu];
    ScaleItem si;
    si.on = d.p.nms_scale != 0;
    si.layer = tile.layer;
    si.L = d.g.L;
    si.th = det_th(d.g.det_shape);
    si.tx = tile.tx;
    si.ty = tile.ty;
    const LayerGeom& lg = d.g.layer[tile.layer];
    si.h = lg.h;
    si.S = lg.S;
    si.bits = d.s.det_bits + lg.bit_off;
    si.wpr = lg.wpr;
    si.dscore = d.s.det_score + lg.score_off;
    si.dpitch = lg.pitch;
    si.w = lg.w;
    si.dcnt = d.s.dcnt;
    si.rowcell = d.tb.rowcell + lg.row_off;
    si.wbins = d.tb.wbins + lg.wb_off;
    si.wmask = d.tb.wmask + lg.wb_off;
    si.xstart = d.tb.xstart + lg.xs_off;
    for (int j = 0; j < 2; ++j) {
      const int m = tile.layer + (j ? 1 : -1);
      LayerView& v = si.adj[j];
      if (m < 0 || m >= d.g.L) {
        v = LayerView{nullptr, 0, 0, 0, 2};
        continue;
      }
      const LayerGeom& lm = d.g.layer[m];
      v.w = lm.w;
      v.h = lm.h;
      v.S = lm.S;
      if (m == 0) {
        v.p = ti.frame;
        v.pitch = ti.pitch;
      } else {
        v.p = d.s.pyr + lm.pyr_off;
        v.pitch = lm.pitch;
      }
    }
    return si;
  }
};

// Which score rows of the tile each lane must score: a pixel needs a score
// only if its 3x3 neighbourhood holds a pixel of an active bin (detections
// there use it for suppression; elsewhere assembly ignores the result).
// Returns one bit per score row (bit rr: row y0-1+rr) for this lane's word
// x0+4*lane .. +3, dilated by one pixel each way; all ones when every bin is
// active or the tile spans more than 32 bin rows.
template <int TH>
__device__ __forceinline__ uint32_t active_rows(const Item& it, int lane) {
  constexpr int SC_H = Shape<TH>::SC_H;
  if (it.pmask) {
    // per-pixel masks, bit-parallel: lane r loads mask row y0-2+r (words
    // x0-32 .. x0+159), dilates it by one pixel left and right; rows r .. r+2
    // are OR-ed (the vertical dilation) for score row r; the 128 bits of a
    // score row shrink to one bit per 4-pixel word; a 32 x 32 bit transpose
    // gives each lane its word's rows
    const int yy = it.y0 - 2 + lane, wb = it.x0 >> 5;
    const bool row_ok = lane < TH + 4 && yy >= 0 && yy < it.h;
    uint32_t W[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
      const int wx = wb - 1 + i;
      W[i] = (row_ok && wx >= 0 && wx < it.wpr) ? it.pmask[(long long)yy * it.wpr + wx] : 0u;
    }
    uint32_t act32 = 0u;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint32_t c = W[i + 1];
      const uint32_t dh = c | (c << 1) | (c >> 1) | (W[i] >> 31) | (W[i + 2] << 31);
      const uint32_t dv = dh | __shfl_down_sync(0xffffffffu, dh, 1) | __shfl_down_sync(0xffffffffu, dh, 2);
      // any bit of each 4-bit group -> bits 0, 4, ..., 28 -> bits 0 .. 7
      uint32_t n = (dv | (dv >> 1) | (dv >> 2) | (dv >> 3)) & 0x11111111u;
      n = (n | (n >> 3)) & 0x03030303u;
      n = (n | (n >> 6)) & 0x000f000fu;
      n = (n | (n >> 12)) & 0xffu;
      act32 |= n << (8 * i);
    }
    if (lane >= SC_H) act32 = 0u;
    uint32_t rows = 0u;
#pragma unroll
    for (int rr = 0; rr < SC_H; ++rr) rows |= ((__shfl_sync(0xffffffffu, act32, rr) >> lane) & 1u) << rr;
    return rows;
  }
  if (!it.mask) return 0xffffffffu;
  const int x = it.x0 + 4 * lane;
  const int xa = max(0, min(it.w - 1, x - 1)), xb = max(0, min(it.w - 1, x + 4));
  const int ca = it.colblk[xa], cb = it.colblk[xb];
  // bin row of each dilated score row: rows y0-2 .. y0+TH+1, one per lane
  const int yr = max(0, min(it.h - 1, it.y0 - 2 + lane));
  const int rb = lane < TH + 4 ? (int)it.rowblk[yr] : 0;
  const int r_lo = __shfl_sync(0xffffffffu, rb, 0), r_hi = __shfl_sync(0xffffffffu, rb, TH + 3);
  if (r_hi - r_lo >= 32) return 0xffffffffu;
  uint32_t binrows = 0;  // bit (r - r_lo): bin row r active within [ca, cb]
  for (int r = r_lo; r <= r_hi; ++r)
    for (int c = ca; c <= cb; ++c)
      if (it.mask[r * it.N_c + c]) {
        binrows |= 1u << (r - r_lo);
        break;
      }
  uint32_t rows = 0;
#pragma unroll
  for (int rr = 0; rr < SC_H; ++rr) {
    // score row rr needs rows rr-1 .. rr+1, i.e. dilated rows rr .. rr+2
    const int a = __shfl_sync(0xffffffffu, rb, rr) - r_lo, b = __shfl_sync(0xffffffffu, rb, rr + 2) - r_lo;
    const uint32_t span = (b - a == 31) ? 0xffffffffu : ((2u << (b - a)) - 1u);
    if ((binrows >> a) & span) rows |= 1u << rr;
  }
  return rows;
}

// A. stage input rows r_lo .. r_hi (input row r is layer row y0-4+r) and the
// 16-byte chunks c_lo .. c_hi of each (chunk c covers columns
// x0-16+16c .. +15), zeros outside the layer: the part of the tile plus halo
// that the active words need. x0 is a multiple of 128, so each chunk is
// either wholly left of the layer or starts inside it.
template <int TH>
__device__ __forceinline__ void stage(uint8_t* in, const Item& it, int lane, int r_lo, int r_hi, int c_lo,
                                      int c_hi) {
  const bool vec = ((reinterpret_cast<uintptr_t>(it.src) | (uintptr_t)it.pitch) & 15) == 0;
  const int nch = c_hi - c_lo + 1, n = (r_hi - r_lo + 1) * nch;
  const float inv = 1.0f / (float)nch;
  const int gy0 = it.y0 - 4 + r_lo, gx0 = it.x0 - 16 + 16 * c_lo;
  if (vec && gx0 >= 0 && it.x0 - 16 + 16 * c_hi + 16 <= it.w && gy0 >= 0 && it.y0 - 4 + r_hi < it.h) {
    // the whole staged rectangle lies inside the layer: no checks, no zero fill
    const uint8_t* base = it.src + (long long)gy0 * it.pitch + gx0;
    uint8_t* dst = in + r_lo * IN_W + 16 * c_lo;
    for (int q = lane; q < n; q += 32) {
      const int r = __float2int_rz(((float)q + 0.5f) * inv), c = q - r * nch;
      if (FKD_IDX(kChkDetStage, (r_lo + r) * IN_W + 16 * (c_lo + c), Shape<TH>::IN_BYTES - 15) &&
          FKD_IDX(kChkDetStage, gy0 + r, it.h))
        cp_async16(dst + r * IN_W + 16 * c, base + (long long)r * it.pitch + 16 * c, 16);
    }
    return;
  }
  for (int q = lane; q < n; q += 32) {
    const int rq = __float2int_rz(((float)q + 0.5f) * inv);
    const int r = r_lo + rq, c = (c_lo + q - rq * nch) * 16;
    const int gy = it.y0 - 4 + r, gx = it.x0 - 16 + c;
    uint8_t* d = in + r * IN_W + c;
    const bool row_ok = gy >= 0 && gy < it.h;
    if (!FKD_IDX(kChkDetStage, r * IN_W + c, Shape<TH>::IN_BYTES - 15)) continue;
    if (vec) {
      const int bytes = (row_ok && gx >= 0) ? max(0, min(16, it.w - gx)) : 0;
      cp_async16(d, bytes ? it.src + (long long)gy * it.pitch + gx : it.src, bytes);
    } else {
      uint32_t wd[4] = {0u, 0u, 0u, 0u};
      if (row_ok) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (gx + j >= 0 && gx + j < it.w)
            wd[j >> 2] |= (uint32_t)it.src[(long long)gy * it.pitch + gx + j] << (8 * (j & 3));
      }
      *reinterpret_cast<uint4*>(d) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
  }
}

// Score-map offset of the pixel at input offset o.
__device__ __forceinline__ int sc_of(int o) { return (o / IN_W - 3) * SC_P + (o % IN_W) - 12; }

template <class Src, int TH>
__global__ void __launch_bounds__(kDetMaxThreads, MIN_BLOCKS) k_detect(Src src) {
  pdl_wait();
  pdl_trigger();
  using Sh = Shape<TH>;
  constexpr int SC_H = Sh::SC_H, IN_BYTES = Sh::IN_BYTES, SC_BYTES = Sh::SC_BYTES, DET_WORDS = Sh::DET_WORDS;
  extern __shared__ __align__(16) uint8_t smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, warps = blockDim.x >> 5;
  uint8_t* inbuf = smem + warp * Sh::WARP_SMEM;
  uint8_t* sc = inbuf + IN_BYTES;
  uint32_t* detw = reinterpret_cast<uint32_t*>(sc + SC_BYTES);
  uint32_t* passw = detw + DET_WORDS;
  uint32_t* wlist = passw + DET_WORDS;
  uint16_t* ring = reinterpret_cast<uint16_t*>(wlist + Sh::WLIST);
  uint16_t* plist = ring + RING;

  const uint32_t count_items = src.count();
  const uint32_t stride = gridDim.x * warps;
  const unsigned lt = (1u << lane) - 1u;

  uint32_t item = blockIdx.x * warps + warp;
  uint32_t wi_next = item < count_items ? src.wi_at(item) : 0u;
  for (; item < count_items; item += stride) {
    // the next item's work entry is loaded a tile ahead
    const uint32_t wi = wi_next;
    if (item + stride < count_items) wi_next = src.wi_at(item + stride);
    const Item it = src.template decode<TH>(wi);
    const uint8_t* in = inbuf;
    const int w = it.w, h = it.h, x0 = it.x0, y0 = it.y0;
    const uint32_t t = (uint32_t)it.t;
    const uint32_t t1 = t + 1u;  // score >= t  <=>  some arc beyond I_p +- t
    const uint32_t t1_low7 = (t1 & 0x7fu) * 0x01010101u;
    const bool t1_high = t1 >= 128u;
    const bool none = t1 > 255u;
    const bool interior = x0 - 1 >= 3 && x0 + TW < w - 3 && y0 - 1 >= 3 && y0 + TH < h - 3;

    // rows this lane's word must score: active bins, inside the scorable band
    // (active_rows may set bits beyond the tile's SC_H score rows: cleared)
    constexpr uint32_t kAllRows = (SC_H == 32) ? 0xffffffffu : ((1u << SC_H) - 1u);
    uint32_t rows = active_rows<TH>(it, lane) & kAllRows;
    if (!interior) {
#pragma unroll
      for (int rr = 0; rr < SC_H; ++rr) {
        const int y = y0 - 1 + rr;
        if (y < 3 || y >= h - 3) rows &= ~(1u << rr);
      }
    }
    if (none) rows = 0u;
    const uint32_t rows_any = __reduce_or_sync(0xffffffffu, rows);
    const unsigned lanes_any = __ballot_sync(0xffffffffu, rows != 0u);

    // the cell tables of this lane's bitmap words (phase E), loaded now so
    // that their latency hides behind the tile's work
    constexpr int EJ = DET_WORDS / 32;
    const int e_wx = x0 / 32 + (lane & 3);
    uint32_t e_wb = 0u, e_wm = 0u;
    int e_cell[EJ];
    if (it.dcnt && e_wx < it.wpr) {
      e_wb = it.wbins[e_wx];
      e_wm = it.wmask[e_wx];
    }
#pragma unroll
    for (int j = 0; j < EJ; ++j) {
      const int y = y0 + (lane >> 2) + 8 * j;
      e_cell[j] = (it.dcnt && y < h) ? it.rowcell[y] : 0;
    }

    // A. stage what the active words need: score rows rr read input rows
    //    rr .. rr+6; word l reads input columns 4l+12 .. 4l+23
    if (rows_any) {
      const int rr_lo = __ffs(rows_any) - 1, rr_hi = 31 - __clz(rows_any);
      const int wl_lo = __ffs(lanes_any) - 1, wl_hi = 31 - __clz(lanes_any);
      stage<TH>(inbuf, it, lane, rr_lo, rr_hi + 6, (4 * wl_lo + 12) >> 4, (4 * wl_hi + 23) >> 4);
    }
    cp_async_commit();
    for (int q = lane; q < SC_BYTES / 16; q += 32)
      reinterpret_cast<uint4*>(sc)[q] = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int q = lane; q < DET_WORDS; q += 32) detw[q] = passw[q] = 0u;
    cp_async_wait<0>();
    __syncwarp();

    // B. prefilter the score rows y0-1 .. y0+TH (input rows 3 .. TH+4), lane
    //    -> word x0+4*lane .. +3, and the two edge columns; words holding
    //    candidates are compacted (one ballot per 32 words) into the word
    //    list, each entry the prefilter bits (bit 7 of byte i: pixel i) with
    //    the score row in bits 0-4 and the word column + 1 (0: left edge, 33:
    //    right edge) in bits 8-13.
    int nw = 0;     // words in the list (warp-uniform)
    int npass = 0;  // passing tile pixels (warp-uniform)
    auto add_word = [&](uint32_t entry) {
      const unsigned bal = __ballot_sync(0xffffffffu, (entry & 0x80808080u) != 0u);
      if ((entry & 0x80808080u) && FKD_IDX(kChkDetWlist, nw + __popc(bal & lt), Sh::WLIST))
        wlist[nw + __popc(bal & lt)] = entry;
      nw += __popc(bal);
    };
    if (rows_any) {
      auto colmask_of = [&](int wl) {  // pixels of word wl inside the scorable band
        uint32_t m = 0x80808080u;
        if (!interior) {
          const int x = x0 + 4 * wl;
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (x + i < 3 || x + i >= w - 3) m &= ~(0x80u << (8 * i));
        }
        return m;
      };
      if (__all_sync(0xffffffffu, rows == kAllRows)) {
        // every row of every word: no per-row tests
        const int c = 16 + 4 * lane;
        const uint32_t colmask = colmask_of(lane), code = (uint32_t)(lane + 1) << 8;
#pragma unroll 2
        for (int rr = 0; rr < SC_H; ++rr)
          add_word((prefilter(in, (rr + 3) * IN_W + c, t1_low7, t1_high) & colmask) | code | (uint32_t)rr);
      } else {
        // only the (row, word) units some bin needs: list them (lane order,
        // then row order) at the head of the word list, then prefilter them
        // 32 at a time, one unit per lane
        const int cnt = __popc(rows);
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int o = __shfl_up_sync(0xffffffffu, incl, d);
          if (lane >= d) incl += o;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        int at = incl - cnt;
        for (uint32_t r = rows; r; r &= r - 1u, ++at)
          if (FKD_IDX(kChkDetUnits, at, Sh::WLIST)) wlist[at] = ((uint32_t)(lane + 1) << 8) | (uint32_t)(__ffs(r) - 1);
        __syncwarp();
        for (int u0 = 0; u0 < total; u0 += 32) {
          const uint32_t unit = u0 + lane < total ? wlist[u0 + lane] : 0u;
          __syncwarp();  // every unit of this round is read before entries overwrite them
          uint32_t keep = 0u;
          if (unit) {
            const int wl = (int)(unit >> 8) - 1, rr = (int)(unit & 31u);
            keep = prefilter(in, (rr + 3) * IN_W + 16 + 4 * wl, t1_low7, t1_high) & colmask_of(wl);
          }
          add_word(keep | unit);
        }
      }
      // the score region's edge columns x0-1 and x0+TW: lane rr < SC_H owns
      // row rr; they are needed when the tile's first / last word is
      const uint32_t rows_l = __shfl_sync(0xffffffffu, rows, 0), rows_r = __shfl_sync(0xffffffffu, rows, 31);
      uint32_t kl = 0, kr = 0;
      if (lane < SC_H) {
        const int r = (lane + 3) * IN_W;
        if (((rows_l >> lane) & 1u) && x0 - 1 >= 3 && x0 - 1 < w - 3)
          kl = prefilter(in, r + 12, t1_low7, t1_high) & 0x80000000u;
        if (((rows_r >> lane) & 1u) && x0 + TW >= 3 && x0 + TW < w - 3)
          kr = prefilter(in, r + 16 + TW, t1_low7, t1_high) & 0x80u;
      }
      add_word(kl | (uint32_t)lane);
      add_word(kr | (33u << 8) | (uint32_t)lane);
    }
    __syncwarp();

    // C. expand the words 32 at a time into candidate pixels (a ring), and
    //    score the ring 64 at a time -- two candidates per lane in 16-bit
    //    lanes. A pixel of the tile scoring >= t goes to the pass list (and
    //    the pass bitmap).
    int head = 0, tail = 0;  // ring positions (warp-uniform), taken mod RING
    auto score_round = [&](int n) {
      const int i1 = 2 * lane;
      bool pass[2] = {false, false};
      int po[2] = {0, 0};
      if (i1 < n) {
        const bool two = i1 + 1 < n;
        const int o1 = ring[(tail + i1) & (RING - 1)];
        const int o2 = two ? ring[(tail + i1 + 1) & (RING - 1)] : o1;
        const uint32_t sp = score_pair(in, o1, o2);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          if (j == 0 || two) {
            const int o = j ? o2 : o1;
            const uint32_t v = (sp >> (16 * j)) & 0xffffu;
            const bool ok = v >= t;
            if (FKD_IDX(kChkDetScore, sc_of(o), SC_BYTES)) sc[sc_of(o)] = ok ? (uint8_t)v : 0;
            const int r = o / IN_W, cc = o % IN_W;  // tile pixel: rows 4..TH+3, cols 16..TW+15
            if (ok && r >= 4 && r < TH + 4 && cc >= 16 && cc < TW + 16) {
              const int ly = r - 4, lx = cc - 16;
              if (FKD_IDX(kChkDetPass, ly * (TW / 32) + (lx >> 5), DET_WORDS))
                atomicOr(&passw[ly * (TW / 32) + (lx >> 5)], 1u << (lx & 31));
              pass[j] = true;
              po[j] = o;
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const unsigned bal = __ballot_sync(0xffffffffu, pass[j]);
        const int at = npass + __popc(bal & lt);
        if (pass[j] && at < PASS) plist[at] = (uint16_t)po[j];
        npass += __popc(bal);
      }
      tail += n;
    };
    for (int wb = 0; wb < nw; wb += 32) {
      const uint32_t e = wb + lane < nw ? wlist[wb + lane] : 0u;
      // input offset of the word's first pixel: row (score row + 3), column
      // 16 + 4 * word column = 12 + 4 * (word column + 1)
      const int o0 = (int)((e & 31u) + 3u) * IN_W + 12 + 4 * (int)((e >> 8) & 63u);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const bool has = (e >> (8 * b + 7)) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, has);
        if (has) ring[(head + __popc(bal & lt)) & (RING - 1)] = (uint16_t)(o0 + b);
        head += __popc(bal);
      }
      __syncwarp();
      while (head - tail >= 64) score_round(64);
    }
    if (head > tail) score_round(head - tail);
    __syncwarp();

    // D. strict 3x3 maxima among the tile's passing pixels: from the pass
    //    list, or from the pass bitmap when the list overflowed
    uint8_t* dscore = it.dscore;
    if (npass <= PASS) {
      for (int i = lane; i < npass; i += 32) {
        const int o = plist[i];
        const int ly = o / IN_W - 4, lx = o % IN_W - 16;
        const uint8_t* q = sc + (ly + 1) * SC_P + 4 + lx;
        const int v = q[0];
        if (v > q[-SC_P - 1] && v > q[-SC_P] && v > q[-SC_P + 1] && v > q[-1] && v > q[1] &&
            v > q[SC_P - 1] && v > q[SC_P] && v > q[SC_P + 1]) {
          if (FKD_IDX(kChkDetPass, ly * (TW / 32) + (lx >> 5), DET_WORDS))
            atomicOr(&detw[ly * (TW / 32) + (lx >> 5)], 1u << (lx & 31));
          if (FKD_IDX(kChkDetDscore, y0 + ly, h) && FKD_IDX(kChkDetDscore, x0 + lx, w))
            dscore[(long long)(y0 + ly) * it.dpitch + x0 + lx] = (uint8_t)v;
        }
      }
    } else
#pragma unroll
    for (int j = 0; j < DET_WORDS / 32; ++j) {
      const int idx = lane + 32 * j;
      const int ly = idx / (TW / 32), lx0 = (idx % (TW / 32)) * 32;
      uint32_t pw = passw[idx];
      while (pw) {
        const int bb = __ffs(pw) - 1;
        pw &= pw - 1;
        const int lx = lx0 + bb;
        const uint8_t* q = sc + (ly + 1) * SC_P + 4 + lx;
        const int v = q[0];
        if (v > q[-SC_P - 1] && v > q[-SC_P] && v > q[-SC_P + 1] && v > q[-1] && v > q[1] &&
            v > q[SC_P - 1] && v > q[SC_P] && v > q[SC_P + 1]) {
          atomicOr(&detw[idx], 1u << bb);
          if (FKD_IDX(kChkDetDscore, y0 + ly, h) && FKD_IDX(kChkDetDscore, x0 + lx, w))
            dscore[(long long)(y0 + ly) * it.dpitch + x0 + lx] = (uint8_t)v;
        }
      }
    }
    __syncwarp();

    // E. the tile's bitmap words (TH rows x TW/32 words), their detections
    //    counted into the cells (chunk x bin) of their pixels
    uint32_t* bits = it.bits;
#pragma unroll
    for (int j = 0; j < DET_WORDS / 32; ++j) {
      const int idx = lane + 32 * j;
      const int ly = idx / (TW / 32), wx = x0 / 32 + idx % (TW / 32);
      if (y0 + ly < h && wx < it.wpr) {
        const uint32_t word = detw[idx];
        if (FKD_IDX(kChkDetBits, (long long)(y0 + ly) * it.wpr + wx, (long long)h * it.wpr))
          bits[(long long)(y0 + ly) * it.wpr + wx] = word;
        if (word && it.dcnt && FKD_IDX(kChkDetCells, e_cell[j] + (int)(e_wb >> 16), it.n_cells))
          count_word_v(it.dcnt + e_cell[j], word, wx, w, e_wb, e_wm, it.xstart, 1);
      }
    }
    __syncwarp();
  }
}

// Does the segment test fire at threshold v (>= 1) at pixel (x, y) of the
// layer, i.e. is its score >= v (Sec. 2)? 0 within 3 px of the layer edge.
// The bright and dark ring pixels form 16-bit masks; a run of 9 around the
// ring is found on the mask doubled to 32 bits by shift-and doubling.
__device__ __forceinline__ bool fires(const LayerView& L, int x, int y, int v) {
  if (x < 3 || y < 3 || x >= L.w - 3 || y >= L.h - 3) return false;
  const uint8_t* c = L.p + (long long)y * L.pitch + x;
  const int ip = c[0];
  // two adjacent compass points must both be beyond ip +- v (see the prefilter)
  const int n = c[-3 * L.pitch], e = c[3], so = c[3 * L.pitch], wv = c[-3];
  const auto far = [&](int q) { return q > ip + v || q < ip - v; };
  if (!((far(n) || far(so)) && (far(e) || far(wv)))) return false;
  uint32_t br = 0, dk = 0;
#define FKD_MASKS(k, dx, dy)                              \
  {                                                       \
    const int q = c[(dy) * L.pitch + (dx)];               \
    br |= (uint32_t)(q > ip + v) << (k);                  \
    dk |= (uint32_t)(q < ip - v) << (k);                  \
  }
  FKD_RING(FKD_MASKS)
#undef FKD_MASKS
  auto run9 = [](uint32_t m) {
    const uint32_t d = m | (m << 16);
    const uint32_t r2 = d & (d >> 1), r4 = r2 & (r2 >> 2), r8 = r4 & (r4 >> 4);
    return ((r8 & (d >> 8)) & 0xffffu) != 0u;
  };
  return run9(br) || run9(dk);
}

// Scale-space suppression (Sec. 2, "3x3 scale-space neighbourhood"): a
// detection of layer l survives only if its score is strictly above every
// score of the 3x3 window, in the layers l-1 and l+1, around the pixel that
// contains its centre (x' = floor((2x + 1) * S_l / (2 S_l')), likewise y').
// One warp per active (frame, tile) item, 32 bitmap words at a time: every
// (detection, window pixel) pair of those words becomes one task, the tasks
// are spread over the lanes, and a window pixel whose segment test fires at
// the detection's score clears the detection's bit.
constexpr int kScaleWarps = 8;
template <class Src>
__global__ void __launch_bounds__(kScaleWarps * 32) k_scale_nms(Src src) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t wsm[kScaleWarps][32], pre[kScaleWarps][32], dom[kScaleWarps][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t n_items = src.count();
  for (uint32_t item = blockIdx.x * kScaleWarps + warp; item < n_items; item += gridDim.x * kScaleWarps) {
    const ScaleItem si = src.scale_item(item);
    const int n_adj = (si.adj[0].p ? 1 : 0) + (si.adj[1].p ? 1 : 0);
    if (!si.on || n_adj == 0) continue;
    const int nbs = 9 * n_adj;  // window pixels per detection
    const int words = si.th * (TW / 32);
    for (int c0 = 0; c0 < words; c0 += 32) {
      const int wi = c0 + lane;
      const int y = si.ty * si.th + wi / (TW / 32);
      const int wx = si.tx * (TW / 32) + wi % (TW / 32);
      const bool valid = wi < words && y < si.h && wx < si.wpr;
      uint32_t* wp = si.bits + (long long)y * si.wpr + wx;
      const uint32_t w = valid ? *wp : 0u;
      // exclusive prefix of the lanes' task counts
      const int cnt = __popc(w) * nbs;
      int incl = cnt;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int o = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += o;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      if (total == 0) continue;
      wsm[warp][lane] = w;
      pre[warp][lane] = (uint32_t)(incl - cnt);
      dom[warp][lane] = 0u;
      __syncwarp();
      for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        if (t < total) {
          // the lane whose tasks hold t: the last with pre <= t
          int lo = 0, hi = 31;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((int)pre[warp][mid] <= t) lo = mid;
            else hi = mid - 1;
          }
          const int owner = lo, local = t - (int)pre[warp][owner];
          const int bi = local / nbs, nb = local % nbs;
          uint32_t m = wsm[warp][owner];
          for (int q = 0; q < bi; ++q) m &= m - 1;
          const int bit = __ffs(m) - 1;
          const int owi = c0 + owner;
          const int oy = si.ty * si.th + owi / (TW / 32);
          const int ox = (si.tx * (TW / 32) + owi % (TW / 32)) * 32 + bit;
          const int v = si.dscore[(long long)oy * si.dpitch + ox];
          const LayerView L = (nb < 9 && si.adj[0].p) ? si.adj[0] : si.adj[1];
          const int cx = L.div2S((2 * ox + 1) * si.S), cy = L.div2S((2 * oy + 1) * si.S);
          const int k9 = nb % 9;
          if (fires(L, cx + k9 % 3 - 1, cy + k9 / 3 - 1, v)) atomicOr(&dom[warp][owner], 1u << bit);
        }
      }
      __syncwarp();
      const uint32_t d = dom[warp][lane];
      if (valid && d) {
        *wp = w & ~d;
        if (si.dcnt) count_word(si.dcnt + si.rowcell[y], d, wx, si.w, si.wbins, si.wmask, si.xstart, -1);
      }
      __syncwarp();
    }
  }
}

}  // namespace

void launch_scale_nms(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                      const Params& p, cudaStream_t st) {
  pdl_launch(k_scale_nms<SingleSrc>, dim3(sm_count() * 8), dim3(kScaleWarps * 32), 0, st, SingleSrc{g, b, s, tb, p});
}

void launch_group_scale_nms(const StreamDev* devs, const TickItem* items, const uint32_t* work,
                            const uint32_t* work_count, cudaStream_t st) {
  k_scale_nms<GroupSrc><<<sm_count() * 8, kScaleWarps * 32, 0, st>>>(GroupSrc{devs, items, work, work_count});
}

template <int TH>
int ctas_per_sm(int warps) {
  constexpr int smem = Shape<TH>::WARP_SMEM;
  const int max_smem = (kDetMaxThreads / 32) * smem;
  if (cudaFuncSetAttribute(k_detect<SingleSrc, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem) ||
      cudaFuncSetAttribute(k_detect<GroupSrc, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem))
    return 0;
  int n = 0, m = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_detect<SingleSrc, TH>, warps * 32, warps * smem) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, k_detect<GroupSrc, TH>, warps * 32, warps * smem))
    return 0;
  return std::min(n, m);
}

static_assert(kDetShapes == 3, "one launch case per tile shape");

int detect_ctas_per_sm(int shape, int warps) {
  if (warps < 1 || warps > kDetMaxThreads / 32) return 0;
  switch (shape) {
    case 0: return ctas_per_sm<kDetTH[0]>(warps);
    case 1: return ctas_per_sm<kDetTH[1]>(warps);
    case 2: return ctas_per_sm<kDetTH[2]>(warps);
    default: return 0;
  }
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

// Batches launch with programmatic dependence (the kernel before is on the
// same stream); group ticks, replayed from captured graphs, plainly.
template <class Src>
constexpr bool kPdl = std::is_same<Src, SingleSrc>::value;

template <class Src>
void launch_shape(const Src& src, const DetLaunch& dl, cudaStream_t st) {
  switch (dl.shape) {
#define FKD_DET_CASE(i)                                                                         \
  case i:                                                                                       \
    if constexpr (kPdl<Src>)                                                                    \
      pdl_launch(k_detect<Src, kDetTH[i]>, dim3(dl.grid), dim3(dl.warps * 32),                  \
                 (size_t)dl.warps * Shape<kDetTH[i]>::WARP_SMEM, st, src);                      \
    else                                                                                        \
      k_detect<Src, kDetTH[i]><<<dl.grid, dl.warps * 32, dl.warps * Shape<kDetTH[i]>::WARP_SMEM, st>>>(src); \
    break;
    FKD_DET_CASE(0)
    FKD_DET_CASE(1)
    FKD_DET_CASE(2)
#undef FKD_DET_CASE
  }
}

void launch_detect(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                   const Params& p, const DetLaunch& dl, cudaStream_t st) {
  launch_shape(SingleSrc{g, b, s, tb, p}, dl, st);
}

void launch_group_detect(const StreamDev* devs, const TickItem* items, const uint32_t* work,
                         const uint32_t* work_count, const DetLaunch& dl, cudaStream_t st) {
  launch_shape(GroupSrc{devs, items, work, work_count}, dl, st);
}

}  // namespace fkd
