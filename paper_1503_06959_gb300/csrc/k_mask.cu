// k_mask.cu -- detection mask M'_n per bin, the source frame of each bin's
// keypoints across a batch, and the compacted list of active detection tiles.
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

// Sum of |L_n - L_{n-1}| over the pixels of `bin` in the mask layer (a layer
// above c_0, row pitch `pitch` in both buffers).
__device__ __forceinline__ unsigned long long layer_change(const BinRect& br, const uint8_t* cur,
                                                           const uint8_t* prv, int pitch) {
  unsigned long long sum = 0;
  for (int y = br.y0; y < br.y1; ++y) {
    uint32_t row = 0;
    for (int x = br.x0; x < br.x1; ++x) {
      const int d = (int)cur[(long long)y * pitch + x] - (int)prv[(long long)y * pitch + x];
      row += (uint32_t)(d < 0 ? -d : d);
    }
    sum += row;
  }
  return sum;
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
__global__ void __launch_bounds__(kMaskThreads) k_mask(Geometry g, Tables tb, Batch b, Scratch s,
                                                       Params p, State st, int reset_base_slot) {
  __shared__ int wmax[kMaskThreads / 32];
  const int bin = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
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
      if (n == 0 || p.mask_mode == FKD_MASK_FULL) {
        m = 1;
      } else if (p.mask_mode == FKD_MASK_ID && g.mask_layer > 0) {
        // L_{n-1} of the batch's first frame: the previous batch's last frame
        const LayerGeom& lg = g.layer[g.mask_layer];
        const uint8_t* cur = s.pyr + (long long)k * g.pyr_bytes + lg.pyr_off;
        const uint8_t* prv = k > 0 ? cur - g.pyr_bytes : s.ml_prev;
        m = layer_change(bin_rect(g, tb, bin), cur, prv, lg.pitch) > (unsigned long long)p.T_I * tb.npix[bin];
      } else if (p.mask_mode == FKD_MASK_ID) {
        unsigned long long* sum = s.bsum + (long long)bin * s.bsum_stride + k;
        m = *sum > (unsigned long long)p.T_I * tb.npix[bin];
        *sum = 0;  // ready for the next batch
      } else {
        m = st.cnt_in[bin] >= (uint32_t)p.T_H;
      }
      s.mask[(long long)k * g.NB + bin] = (uint8_t)m;
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
  if (p.mask_mode == FKD_MASK_ID && g.mask_layer > 0) {
    // the batch's last frame becomes L_{n-1} of the next batch (this bin's
    // pixels only; frame 0 read the old ones before the barrier above)
    const LayerGeom& lg = g.layer[g.mask_layer];
    const BinRect br = bin_rect(g, tb, bin);
    const uint8_t* last = s.pyr + (long long)(b.T - 1) * g.pyr_bytes + lg.pyr_off;
    for (int y = br.y0; y < br.y1; ++y)
      for (int x = br.x0 + tid; x < br.x1; x += kMaskThreads)
        s.ml_prev[(long long)y * lg.pitch + x] = last[(long long)y * lg.pitch + x];
  }
}

// One thread per (frame, tile): a tile is active when any bin its pixels map
// to is active. Active items are compacted with a warp ballot, a popcount and
// one atomic per warp.
__global__ void k_worklist(Geometry g, Tables tb, Batch b, Scratch s) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)b.T * g.n_tiles;
  for (long long q = i; q < (long long)b.T * g.n_chunks; q += (long long)gridDim.x * blockDim.x)
    s.chunk_counts[q] = 0;  // summed by the assembly count pass
  bool act = false;
  uint32_t area = 0;
  if (i < total) {
    const int k = (int)(i / g.n_tiles), tile = (int)(i % g.n_tiles);
    const DetTile t = tb.tiles[tile];
    const uint8_t* m = s.mask + (long long)k * g.NB;
    for (int r = t.rb0; r <= t.rb1 && !act; ++r)
      for (int c = t.cb0; c <= t.cb1; ++c)
        if (m[r * g.N_c + c]) { act = true; break; }
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
  if (act) s.work[base + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)i;
}

// Group tick, one frame per stream: the mask and source frame of every bin
// of every participating stream (src = 0 for active bins, -1 = kept set).
__global__ void k_group_mask(const StreamDev* devs, const TickHeader* hdr, const TickItem* items,
                             uint32_t* work_count) {
  const int n = hdr->n_items, total = hdr->total_bins;
  const int gtid = blockIdx.x * blockDim.x + threadIdx.x;
  if (gtid == 0) *work_count = 0;
  for (int j = gtid; j < total; j += gridDim.x * blockDim.x) {
    const int i = find_item(n, j, [&](int q) { return items[q].bin_base; });
    const TickItem it = items[i];
    const StreamDev& d = devs[it.sid];
    const int bin = j - it.bin_base;
    int m;
    if (it.frame_index == 0 || d.p.mask_mode == FKD_MASK_FULL) {
      m = 1;
    } else if (d.p.mask_mode == FKD_MASK_ID && d.g.mask_layer > 0) {
      // a coarser mask layer: this frame's layer against the stream's copy
      // of the previous one, which then takes this frame's pixels of the bin
      const LayerGeom& lg = d.g.layer[d.g.mask_layer];
      const uint8_t* cur = d.s.pyr + lg.pyr_off;
      const BinRect br = bin_rect(d.g, d.tb, bin);
      m = layer_change(br, cur, d.s.ml_prev, lg.pitch) > (unsigned long long)d.p.T_I * d.tb.npix[bin];
    } else if (d.p.mask_mode == FKD_MASK_ID) {
      m = d.s.bsum[bin] > (unsigned long long)d.p.T_I * d.tb.npix[bin];
      d.s.bsum[bin] = 0;
    } else {
      m = d.state_cnt[it.state_cur][bin] >= (uint32_t)d.p.T_H;
    }
    if (d.p.mask_mode == FKD_MASK_ID && d.g.mask_layer > 0) {
      const LayerGeom& lg = d.g.layer[d.g.mask_layer];
      const BinRect br = bin_rect(d.g, d.tb, bin);
      for (int y = br.y0; y < br.y1; ++y)
        for (int x = br.x0; x < br.x1; ++x)
          d.s.ml_prev[(long long)y * lg.pitch + x] = d.s.pyr[lg.pyr_off + (long long)y * lg.pitch + x];
    }
    d.s.mask[bin] = (uint8_t)m;
    d.s.src[bin] = m ? 0 : -1;
    d.state_cnt[it.state_cur ^ 1][bin] = 0;
    if (bin == 0) {
      d.s.frame_totals[0] = 0;
      d.s.out_base[0] = 0;
    }
    for (int q = bin; q < d.g.n_chunks; q += d.g.NB) d.s.chunk_counts[q] = 0;
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
    uint32_t entry = 0;
    if (j < total) {
      const int i = find_item(n, j, [&](int q) { return items[q].tile_base; });
      const TickItem it = items[i];
      const StreamDev& d = devs[it.sid];
      const int tile = j - it.tile_base;
      const DetTile t = d.tb.tiles[tile];
      for (int r = t.rb0; r <= t.rb1 && !act; ++r)
        for (int c = t.cb0; c <= t.cb1; ++c)
          if (d.s.mask[r * d.g.N_c + c]) { act = true; break; }
      if (act) {
        entry = ((uint32_t)i << 22) | (uint32_t)tile;
        atomicAdd(&d.s.tile_stats[0], 1ull);
        atomicAdd(&d.s.tile_stats[1], (unsigned long long)t.area);
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
  k_mask<<<g.NB, kMaskThreads, 0, st>>>(g, tb, b, s, p, state, reset_base_slot);
}

void launch_worklist(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                     cudaStream_t st) {
  const int threads = 256;
  const long long total = (long long)b.T * g.n_tiles;
  const int blocks = (int)((total + threads - 1) / threads);
  k_worklist<<<blocks, threads, 0, st>>>(g, tb, b, s);
}

}  // namespace fkd
