// k_mask.cu -- detection mask M'_n per bin, the source frame of each bin's
// keypoints across a batch, and the compacted list of active detection tiles.
#include <algorithm>

#include "fkd_internal.cuh"

namespace fkd {
namespace {

// The pixels of `bin` in the mask layer: columns [x0, x1) from the bin-column
// starts; rows [y0, y1), since layer row y is in bin row
// floor(floor(y*S/2) * N_r / H) (Eq. 3), so bin row r starts at row
// ceil(2 * ceil(r*H/N_r) / S).
struct BinRect {
  int x0, x1, y0, y1;
};
__device__ __forceinline__ BinRect bin_rect(const Geometry& g, const Tables& tb, int bin) {
  const LayerGeom& lg = g.layer[g.mask_layer];
  const int r = bin / g.N_c, c = bin % g.N_c;
  auto row_start = [&](int rr) {
    const long long q = ((long long)rr * g.H + g.N_r - 1) / g.N_r;
    return (int)min((long long)lg.h, (2 * q + lg.S - 1) / lg.S);
  };
  return BinRect{tb.xstart[lg.xs_off + c], tb.xstart[lg.xs_off + c + 1], row_start(r), row_start(r + 1)};
}

// Sum of |L_n - L_{n-1}| over the pixels of a bin of the mask layer (a layer
// above c_0, row pitch `pitch` in both buffers), by one warp: lane i takes
// pixels i, i + 32, ... of the bin in row-major order. If `copy` is not null,
// the warp then stores the bin's pixels of L_n there (same layout).
__device__ __forceinline__ unsigned long long layer_change_warp(const BinRect& br, const uint8_t* cur,
                                                                const uint8_t* prv, int pitch, uint8_t* copy) {
  const int lane = threadIdx.x & 31;
  const int bw = br.x1 - br.x0;
  // lanes over the bin: 32 columns of a row at a time when the bin is at
  // least 32 wide, else 32 / bw rows of bw lanes (one division per lane)
  const bool wide = bw >= 32;
  const int rows_per = wide ? 1 : 32 / max(bw, 1), step_x = wide ? 32 : max(bw, 1);
  const int lr = wide ? 0 : lane / max(bw, 1), lc = wide ? lane : lane - lr * bw;
  unsigned long long sum = 0;
  if (lr < rows_per && bw > 0)
    for (int y = br.y0 + lr; y < br.y1; y += rows_per) {
      const long long ro = (long long)y * pitch;
      for (int x = br.x0 + lc; x < br.x1; x += step_x) {
        const int d = (int)cur[ro + x] - (int)prv[ro + x];
        sum += (unsigned long long)(d < 0 ? -d : d);
      }
    }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
  if (copy) {
    __syncwarp();
    if (lr < rows_per && bw > 0)
      for (int y = br.y0 + lr; y < br.y1; y += rows_per) {
        const long long ro = (long long)y * pitch;
        for (int x = br.x0 + lc; x < br.x1; x += step_x) copy[ro + x] = cur[ro + x];
      }
  }
  return sum;
}

// Per-bin sums of |L_k - L_{k-1}| on a mask layer above c_0, one CTA per frame
// of the batch, into the same per-bin sums the pyramid kernel fills for c_0
// (L_{-1}: the stream's copy of the previous batch's last frame, refreshed by
// k_mask). Thread t takes a run of consecutive pixels (row-major) and adds to
// a shared bin whenever the bin changes.
constexpr int kLayerSumBins = kMaxBins;
__global__ void __launch_bounds__(kMaskThreads) k_layer_sums(Geometry g, Tables tb, Batch b, Scratch s) {
  pdl_wait();
  pdl_trigger();
  __shared__ unsigned long long bins[kLayerSumBins];
  const int k = blockIdx.x;
  const LayerGeom& lg = g.layer[g.mask_layer];
  for (int q = threadIdx.x; q < g.NB; q += kMaskThreads) bins[q] = 0;
  __syncthreads();
  const uint8_t* cur = s.pyr + (long long)k * g.pyr_bytes + lg.pyr_off;
  const uint8_t* prv = k > 0 ? cur - g.pyr_bytes : s.ml_prev;
  const int npx = lg.w * lg.h;  // < 2^28 (layers are at most 16384 x 16384)
  const int per = (npx + kMaskThreads - 1) / kMaskThreads;
  const int i0 = min(npx, (int)threadIdx.x * per), n = min(npx, i0 + per) - i0;
  int y = lg.w > 0 ? i0 / lg.w : 0, x = i0 - y * lg.w;
  int cur_bin = -1;
  unsigned long long acc = 0;
  for (int i = 0; i < n; ++i) {
    const int bin = tb.rowblk[lg.row_off + y] * g.N_c + tb.colblk[lg.col_off + x];
    if (bin != cur_bin) {
      if (acc) atomicAdd(&bins[cur_bin], acc);
      cur_bin = bin;
      acc = 0;
    }
    const long long o = (long long)y * lg.pitch + x;
    const int d = (int)cur[o] - (int)prv[o];
    acc += (unsigned long long)(d < 0 ? -d : d);
    if (++x == lg.w) {
      x = 0;
      ++y;
    }
  }
  if (acc) atomicAdd(&bins[cur_bin], acc);
  __syncthreads();
  for (int q = threadIdx.x; q < g.NB; q += kMaskThreads) s.bsum[(long long)q * s.bsum_stride + k] = bins[q];
}

// One CTA per bin, walking the batch's frames 256 at a time.
//   mask:  first frame of the stream or FKD_MASK_FULL -> 1; FKD_MASK_ID ->
//          sum |L_n - L_{n-1}| > T_I * (pixels of the bin) (Eq. 2 read as
//          "detect where the content changed"), the sums of c_0 coming from
//          the pyramid kernel and those of a coarser mask layer computed
//          here from the batch's pyramids; FKD_MASK_KB -> keypoints of
//          D_{n-1} in the bin >= T_H (Eqs. 3-4, batches of one frame).
//   src:   Eq. 1 applied frame after frame means a bin of frame k shows the
//          detections of the last frame m <= k in which the bin was active;
//          src = m, or -1 when no such frame is in the batch (the kept set):
//          an inclusive max-scan of (active ? k : -1) over the frames.
//   With masks_given (keypoint binning in spans) the masks are already in
//   s.mask and only the source frames are computed.
__global__ void __launch_bounds__(kMaskThreads) k_mask(Geometry g, Tables tb, Batch b, Scratch s,
                                                       Params p, State st, int reset_base_slot, int masks_given) {
  pdl_wait();
  pdl_trigger();
  __shared__ int wmax[kMaskThreads / 32];
  const int bin = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool layer_sums = p.mask_mode == FKD_MASK_ID && g.mask_layer > 0;
  const BinRect br = bin_rect(g, tb, bin);
  const LayerGeom& mlg = g.layer[g.mask_layer];
  if (bin == 0) {
    for (int k = tid; k < b.T; k += kMaskThreads) s.frame_totals[k] = 0;
    if (tid == 0) {
      *s.work_count = 0;
      if (reset_base_slot >= 0) s.out_base[reset_base_slot] = 0;
    }
  }
  if (tid == 0) st.cnt_out[bin] = 0;
  int carry = -1;
  for (int k0 = 0; k0 < b.T; k0 += kMaskThreads) {
    const int k = k0 + tid;
    int m = 0;
    if (k < b.T) {
      const long long n = b.first_frame + k;
      if (masks_given) {
        m = s.mask[(long long)k * g.NB + bin];
      } else if (n == 0 || p.mask_mode == FKD_MASK_FULL || p.mask_mode == FKD_MASK_IDP) {
        m = 1;  // (per-pixel masks decide in the detection and assembly passes)
      } else if (p.mask_mode == FKD_MASK_ID) {
        unsigned long long* sum = s.bsum + (long long)bin * s.bsum_stride + k;
        m = *sum > (unsigned long long)p.T_I * tb.npix[bin];
        *sum = 0;  // ready for the next batch
      } else {
        m = st.cnt_in[bin] >= (uint32_t)p.T_H;
      }
      if (!masks_given) s.mask[(long long)k * g.NB + bin] = (uint8_t)m;
    }
    int v = m ? k : -1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int o = __shfl_up_sync(0xffffffffu, v, d);
      if (lane >= d) v = max(v, o);
    }
    if (lane == 31) wmax[warp] = v;
    __syncthreads();
    int before = carry, all = carry;
#pragma unroll
    for (int w = 0; w < kMaskThreads / 32; ++w) {
      if (w < warp) before = max(before, wmax[w]);
      all = max(all, wmax[w]);
    }
    if (k < b.T) s.src[(long long)k * g.NB + bin] = max(v, before);
    carry = all;
    __syncthreads();
  }
  if (layer_sums) {
    // the batch's last frame becomes L_{n-1} of the next batch (this bin's
    // pixels only; frame 0 read the old ones before the barriers above)
    const uint8_t* last = s.pyr + (long long)(b.T - 1) * g.pyr_bytes + mlg.pyr_off;
    const int bw = br.x1 - br.x0, npx = bw * max(0, br.y1 - br.y0);
    for (int i = tid; i < npx; i += kMaskThreads) {
      const long long o = (long long)(br.y0 + i / bw) * mlg.pitch + br.x0 + i % bw;
      s.ml_prev[o] = last[o];
    }
  }
}

// One thread per (frame, tile) of frames k_lo .. k_hi-1 of the batch: a tile
// is active when any bin its pixels map to is active. Active items are
// compacted with a warp ballot, a popcount and one atomic per warp.
__global__ void k_worklist(Geometry g, Tables tb, Batch b, Scratch s, int k_lo, int k_hi) {
  pdl_wait();
  pdl_trigger();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)(k_hi - k_lo) * g.n_tiles;
  for (long long q = i; q < (long long)(k_hi - k_lo) * g.n_chunks; q += (long long)gridDim.x * blockDim.x)
    s.chunk_counts[(long long)k_lo * g.n_chunks + q] = 0;  // summed by the assembly count pass
  if (s.dcnt)
    for (long long q = i; q < (long long)(k_hi - k_lo) * g.n_cells; q += (long long)gridDim.x * blockDim.x)
      s.dcnt[(long long)k_lo * g.n_cells + q] = 0;  // the detection pass counts into them
  bool act = false;
  uint32_t area = 0;
  const long long item = (long long)k_lo * g.n_tiles + i;
  if (i < total) {
    const int k = (int)(item / g.n_tiles), tile = (int)(item % g.n_tiles);
    const DetTile t = tb.tiles[tile];
    if (s.pmask) {
      // per-pixel masks: a tile is active when any of its own pixels is
      const LayerGeom& lg = g.layer[t.layer];
      const int th = det_th(g.det_shape), wpt = kDetTW / 32;
      const uint32_t* pm = s.pmask + (long long)k * g.bit_words + lg.bit_off;
      const int y1 = min(lg.h, (t.ty + 1) * th), w1 = min(lg.wpr, (t.tx + 1) * wpt);
      for (int y = t.ty * th; y < y1 && !act; ++y)
        for (int wx = t.tx * wpt; wx < w1; ++wx)
          if (pm[(long long)y * lg.wpr + wx]) { act = true; break; }
    } else {
      // the tile's bins of each bin row, four mask bytes per load (the mask
      // buffer is padded so that the last word stays inside it)
      const long long m0 = (long long)k * g.NB;
      for (int r = t.rb0; r <= t.rb1 && !act; ++r) {
        const long long lo = m0 + r * g.N_c + t.cb0, hi = m0 + r * g.N_c + t.cb1;  // bytes lo..hi
        for (long long w = lo >> 2; w <= (hi >> 2); ++w) {
          uint32_t v = reinterpret_cast<const uint32_t*>(s.mask)[w];
          if (w == (lo >> 2)) v &= 0xffffffffu << (8 * (lo & 3));
          if (w == (hi >> 2)) v &= 0xffffffffu >> (8 * (3 - (hi & 3)));
          if (v) {
            act = true;
            break;
          }
        }
      }
    }
    if (act) area = t.area;
  }
  const unsigned bal = __ballot_sync(0xffffffffu, act);
  if (bal == 0) return;
  area = __reduce_add_sync(0xffffffffu, area);
  const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
  uint32_t base = 0;
  if (lane == leader) {
    base = atomicAdd(s.work_count, (uint32_t)__popc(bal));
    atomicAdd(&s.tile_stats[0], (unsigned long long)__popc(bal));
    atomicAdd(&s.tile_stats[1], (unsigned long long)area);
  }
  base = __shfl_sync(0xffffffffu, base, leader);
  if (act) s.work[base + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)item;
}

// Keypoint binning (Eqs. 3-4) in spans of frames. A bin is active in frame n
// when D_{n-1} holds at least T_H keypoints in it; while a bin is inactive its
// part of D_n is D_{n-1}'s (Eq. 1), so its count cannot change and it stays
// inactive. The bins active at a span's first frame are therefore a superset
// of the active bins of every later frame of the span: the span's frames are
// detected on that set, and the exact masks are resolved afterwards from the
// detection counts, frame after frame (identical to running the frames one
// by one). alive[bin]: the bin is active at the next frame to resolve.
//
// Span start: the masks of frames k_lo .. k_hi-1 are the alive set (from the
// kept set's counts at the first span of a batch), and the work list is
// emptied for the span's active tiles.
__global__ void k_kb_span(Geometry g, Batch b, Scratch s, Params p, State st, int k_lo, int k_hi, int first) {
  pdl_wait();
  pdl_trigger();
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin == 0) *s.work_count = 0;
  if (bin >= g.NB) return;
  uint8_t a;
  if (first) {
    a = (b.first_frame + k_lo == 0) ? 1 : (st.cnt_in[bin] >= (uint32_t)p.T_H ? 1 : 0);
    s.alive[bin] = a;
  } else {
    a = s.alive[bin];
  }
  for (int k = k_lo; k < k_hi; ++k) s.mask[(long long)k * g.NB + bin] = a;
}

// Span end: the exact masks of frames k_lo .. k_hi-1. A bin active in frame k
// stays active in frame k+1 when its detections in frame k (the sum over its
// cells) reach T_H; the first frame of a stream is active everywhere.
__global__ void k_kb_resolve(Geometry g, Tables tb, Batch b, Scratch s, Params p, int k_lo, int k_hi) {
  pdl_wait();
  pdl_trigger();
  const int bin = blockIdx.x * blockDim.x + threadIdx.x;
  if (bin >= g.NB) return;
  uint8_t a = s.alive[bin];
  const int c0 = tb.bincell_off[bin], c1 = tb.bincell_off[bin + 1];
  for (int k = k_lo; k < k_hi; ++k) {
    const uint8_t m = (b.first_frame + k == 0) ? 1 : a;
    s.mask[(long long)k * g.NB + bin] = m;
    if (m) {
      const uint32_t* dc = s.dcnt + (long long)k * g.n_cells;
      uint32_t cnt = 0;
      for (int c = c0; c < c1; ++c) cnt += dc[tb.bincell[c]];
      a = cnt >= (uint32_t)p.T_H ? 1 : 0;
    }
  }
  s.alive[bin] = a;
}

// Group tick, one frame per stream: the mask and source frame of every bin
// of every participating stream (src = 0 for active bins, -1 = kept set).
// (6 resident CTAs per SM: the per-(stream, bin) load chains are latency-bound)
__global__ void __launch_bounds__(256, 6) k_group_mask(const StreamDev* devs, const TickHeader* hdr,
                                                       const TickItem* items, uint32_t* work_count) {
  // one warp per (stream, bin) of the tick
  const int n = hdr->n_items, total = hdr->total_bins;
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) *work_count = 0;
  for (int j = gwarp; j < total; j += nwarps) {
    const int i = find_item(n, j, [&](int q) { return items[q].bin_base; });
    const TickItem it = items[i];
    const StreamDev& d = devs[it.sid];
    const int bin = j - it.bin_base;
    unsigned long long change = 0;
    if (d.p.mask_mode == FKD_MASK_ID && d.g.mask_layer > 0) {
      // a coarser mask layer: this frame's layer against the stream's copy
      // of the previous one, which then takes this frame's pixels of the bin
      const LayerGeom& lg = d.g.layer[d.g.mask_layer];
      change = layer_change_warp(bin_rect(d.g, d.tb, bin), d.s.pyr + lg.pyr_off, d.s.ml_prev, lg.pitch,
                                 d.s.ml_prev);
    }
    if (lane == 0) {
      int m;
      if (it.frame_index == 0 || d.p.mask_mode == FKD_MASK_FULL) {
        m = 1;
      } else if (d.p.mask_mode == FKD_MASK_ID && d.g.mask_layer > 0) {
        m = change > (unsigned long long)d.p.T_I * d.tb.npix[bin];
      } else if (d.p.mask_mode == FKD_MASK_ID) {
        m = d.s.bsum[bin] > (unsigned long long)d.p.T_I * d.tb.npix[bin];
        d.s.bsum[bin] = 0;
      } else {
        m = d.state_cnt[it.state_cur][bin] >= (uint32_t)d.p.T_H;
      }
      d.s.mask[bin] = (uint8_t)m;
      d.s.src[bin] = m ? 0 : -1;
      d.state_cnt[it.state_cur ^ 1][bin] = 0;
      if (bin == 0) {
        d.s.frame_totals[0] = 0;
        d.s.out_base[0] = 0;
      }
    }
    for (int q = bin + lane * d.g.NB; q < d.g.n_chunks; q += 32 * d.g.NB) d.s.chunk_counts[q] = 0;
  }
}

// Group tick: active (stream, tile) items of every participating stream,
// compacted into one list (item index << 22 | tile).
__global__ void k_group_worklist(const StreamDev* devs, const TickHeader* hdr, const TickItem* items,
                                 uint32_t* work, uint32_t* work_count) {
  const int n = hdr->n_items, total = hdr->total_tiles;
  const int lane = threadIdx.x & 31;
  for (int j0 = blockIdx.x * blockDim.x; j0 < total; j0 += gridDim.x * blockDim.x) {
    const int j = j0 + threadIdx.x;
    bool act = false;
    uint32_t entry = 0, area = 0;
    int sid_act = -1;  // item of an active tile, else -1
    if (j < total) {
      const int i = find_item(n, j, [&](int q) { return items[q].tile_base; });
      const TickItem it = items[i];
      const StreamDev& d = devs[it.sid];
      const int tile = j - it.tile_base;
      const DetTile t = d.tb.tiles[tile];
      // four mask bytes per load (the mask buffer is padded)
      for (int r = t.rb0; r <= t.rb1 && !act; ++r) {
        const int lo = r * d.g.N_c + t.cb0, hi = r * d.g.N_c + t.cb1;
        for (int w = lo >> 2; w <= (hi >> 2); ++w) {
          uint32_t v = reinterpret_cast<const uint32_t*>(d.s.mask)[w];
          if (w == (lo >> 2)) v &= 0xffffffffu << (8 * (lo & 3));
          if (w == (hi >> 2)) v &= 0xffffffffu >> (8 * (3 - (hi & 3)));
          if (v) {
            act = true;
            break;
          }
        }
      }
      if (act) {
        entry = ((uint32_t)i << 22) | (uint32_t)tile;
        area = t.area;
      }
      sid_act = act ? i : -1;
    }
    // tile statistics: one atomic pair per stream and warp
    const unsigned peers = __match_any_sync(0xffffffffu, sid_act);
    if (sid_act >= 0) {
      const unsigned long long sum_area = __reduce_add_sync(peers, area);
      if ((int)lane == __ffs(peers) - 1) {
        const StreamDev& d = devs[items[sid_act].sid];
        atomicAdd(&d.s.tile_stats[0], (unsigned long long)__popc(peers));
        atomicAdd(&d.s.tile_stats[1], sum_area);
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, act);
    if (bal == 0) continue;
    const int leader = __ffs(bal) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(work_count, (uint32_t)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (act) work[base + __popc(bal & ((1u << lane) - 1u))] = entry;
  }
}

}  // namespace

void launch_group_mask(const StreamDev* devs, const TickHeader* hdr, const TickItem* items,
                       uint32_t* work_count, int grid, cudaStream_t st) {
  k_group_mask<<<grid, 256, 0, st>>>(devs, hdr, items, work_count);
}

void launch_group_worklist(const StreamDev* devs, const TickHeader* hdr, const TickItem* items,
                           uint32_t* work, uint32_t* work_count, int grid, cudaStream_t st) {
  k_group_worklist<<<grid, 256, 0, st>>>(devs, hdr, items, work, work_count);
}

void launch_mask(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                 const Params& p, const State& state, cudaStream_t st, int reset_base_slot) {
  if (p.mask_mode == FKD_MASK_ID && g.mask_layer > 0)
    pdl_launch(k_layer_sums, dim3(b.T), dim3(kMaskThreads), 0, st, g, tb, b, s);
  pdl_launch(k_mask, dim3(g.NB), dim3(kMaskThreads), 0, st, g, tb, b, s, p, state, reset_base_slot, 0);
}

void launch_source_frames(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                          const Params& p, const State& state, cudaStream_t st, int reset_base_slot) {
  pdl_launch(k_mask, dim3(g.NB), dim3(kMaskThreads), 0, st, g, tb, b, s, p, state, reset_base_slot, 1);
}

void launch_worklist(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                     cudaStream_t st, int k_lo, int k_hi) {
  if (k_hi < 0) k_hi = b.T;
  const int threads = 256;
  const long long total = (long long)(k_hi - k_lo) * g.n_tiles;
  const int blocks = (int)std::max<long long>(1, (total + threads - 1) / threads);
  pdl_launch(k_worklist, dim3(blocks), dim3(threads), 0, st, g, tb, b, s, k_lo, k_hi);
}

void launch_kb_span(const Geometry& g, const Batch& b, const Scratch& s, const Params& p, const State& state,
                    int k_lo, int k_hi, int first, cudaStream_t st) {
  pdl_launch(k_kb_span, dim3((g.NB + 255) / 256), dim3(256), 0, st, g, b, s, p, state, k_lo, k_hi, first);
}

void launch_kb_resolve(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s, const Params& p,
                       int k_lo, int k_hi, cudaStream_t st) {
  pdl_launch(k_kb_resolve, dim3((g.NB + 255) / 256), dim3(256), 0, st, g, tb, b, s, p, k_lo, k_hi);
}

}  // namespace fkd
