// k_describe.cu -- masked description (Sec. 3): binary descriptors for the
// keypoints a batch detected, carried descriptors for the ones it kept.
//
// Descriptor of keypoint (x, y) of layer l (Sec. 2: one bit per pair of
// sampled pixels, comparing smoothed intensities): bit i is set iff the sum
// of the 5x5 layer pixels around (x + ax_i, y + ay_i) is below the sum around
// (x + bx_i, y + by_i), coordinates clamped to the layer, for a caller-given
// pattern of D pairs with offsets within +-kDescR.
//
//   k_describe_new:     one warp per newly detected record (warps take
//                       groups of 32 records from a counter). Lane c loads
//                       column c of the 32 x 32 window around the keypoint
//                       (one coalesced read per row, clamped to the layer),
//                       sums 5 rows in registers (two rows per register as
//                       16-bit halves), adds 5 columns with shuffles, and
//                       stores the 27 x 27 box sums to shared memory, where
//                       32 pairs are compared per ballot.
//   k_describe_carried: one thread per carried record. Eq. 1 makes a carried
//                       record a copy of the record with the same position in
//                       the frame that last detected there: src(k, bin) for
//                       the block masks, the last frame whose per-pixel mask
//                       bit was set for FKD_MASK_IDP, or the kept set of the
//                       batch before. A binary search within its layer row of
//                       that frame's records (canonical order; the emission
//                       pass records where every row starts) finds it; its
//                       descriptor is copied. The carried pass runs after
//                       the new pass, so every source descriptor is final.
// Both passes also copy the batch's last frame (records, descriptors, row
// starts) into the kept set of the next batch. The group passes do the same
// for one frame of each describing stream of a tick, the previous frame's
// records being the kept set.
#include "fkd_internal.cuh"

namespace fkd {
namespace {

constexpr int kDescBox = 2 * kDescR + 1;  // 27: box centres per row and column
constexpr int kHalfRows = 14;             // box rows r and r + 14 share a word
constexpr int kBoxPitch = 27;             // words per row pair: banks (c - 5 r) % 32 spread the pattern's lookups
constexpr int kNewWarps = 8;
constexpr int kNewMinBlocks = 4;
constexpr int kCarriedThreads = 256;
static_assert(kDescBox == 27 && 2 * kHalfRows >= kDescBox, "window of 32 rows and columns");

// 16-bit index of the box sum of row r, column c in a warp's box array:
// word (r % 14) * 27 + c, low half for r < 14, high half for r >= 14.
__host__ __device__ constexpr int box_half(int r, int c) {
  return 2 * ((r % kHalfRows) * kBoxPitch + c) + r / kHalfRows;
}

__device__ __forceinline__ unsigned long long rec_key(uint2 r) {
  return ((unsigned long long)(r.y & 0xffu) << 32) | r.x;  // (layer, y, x)
}

// Index of the record with `key` in recs[lo, hi) (canonical order), or -1.
__device__ __forceinline__ long long find_record(const uint2* recs, long long lo, long long hi,
                                                 unsigned long long key) {
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    const unsigned long long k = rec_key(recs[mid]);
    if (k == key) return mid;
    if (k < key) lo = mid + 1;
    else hi = mid;
  }
  return -1;
}

// Pixels of layer l of batch frame k.
__device__ __forceinline__ const uint8_t* layer_base(const Geometry& g, const Batch& b, const Scratch& s,
                                                     int k, int l, int* pitch) {
  if (l == 0) {
    *pitch = b.pitch;
    return b.frames + (long long)k * b.frame_stride;
  }
  *pitch = g.layer[l].pitch;
  return s.pyr + (long long)k * g.pyr_bytes + g.layer[l].pyr_off;
}

// Descriptor of the keypoint at (x, y) of a w x h layer (pixels at img,
// row pitch `pitch`) by one warp: pat holds the D / 32 words' pairs as
// 16-bit box indices, bw the warp's box array. Returns word j in lane j.
__device__ __forceinline__ uint32_t describe_record(const uint8_t* img, int pitch, int w, int h, int x, int y,
                                                   const uint32_t* pat, uint32_t* bw, int DW, int lane) {
  const uint16_t* box16 = reinterpret_cast<const uint16_t*>(bw);
  // 1. lane c: column x - 15 + c of rows y - 15 .. y + 16, clamped
  const uint8_t* col = img + min(max(x - kDescR - 2 + lane, 0), w - 1);
  uint32_t px[32];
  if (y >= kDescR + 2 && y + kDescR + 4 <= h) {
    const uint8_t* p = col + (long long)(y - kDescR - 2) * pitch;
#pragma unroll
    for (int rr = 0; rr < 32; ++rr) px[rr] = p[(long long)rr * pitch];
  } else {
#pragma unroll
    for (int rr = 0; rr < 32; ++rr)
      px[rr] = col[(long long)min(max(y - kDescR - 2 + rr, 0), h - 1) * pitch];
  }
  // 2. 5-row sums of the column: P[m] = (sum of rows m..m+4, sum of rows
  //    m+14..m+18) as 16-bit halves, sliding down
  uint32_t P[kHalfRows];
  {
    uint32_t q[kHalfRows + 4];
#pragma unroll
    for (int m = 0; m < kHalfRows + 4; ++m) q[m] = px[m] | (px[m + kHalfRows] << 16);
    P[0] = q[0] + q[1] + q[2] + q[3] + q[4];
#pragma unroll
    for (int m = 1; m < kHalfRows; ++m) P[m] = P[m - 1] + q[m + 4] - q[m - 1];
  }
  // 3. 5-column sums across lanes (lane c: columns c..c+4, valid for
  //    c < 27), stored for the pair tests
  __syncwarp();  // the previous record's tests are done with the array
#pragma unroll
  for (int m = 0; m < kHalfRows; ++m) {
    const uint32_t a2 = P[m] + __shfl_down_sync(0xffffffffu, P[m], 1);
    const uint32_t a4 = a2 + __shfl_down_sync(0xffffffffu, a2, 2);
    const uint32_t box = a4 + __shfl_down_sync(0xffffffffu, P[m], 4);
    if (lane < kDescBox) bw[m * kBoxPitch + lane] = box;
  }
  __syncwarp();

  // 4. 32 pairs per ballot; lane j keeps word j
  uint32_t mine = 0u;
  for (int j = 0; j < DW; ++j) {
    const uint32_t q = pat[j * 32 + lane];
    const uint32_t word = __ballot_sync(0xffffffffu, box16[q & 0xffffu] < box16[q >> 16]);
    if (lane == j) mine = word;
  }
  return mine;
}

__global__ void __launch_bounds__(kNewWarps * 32, kNewMinBlocks)
    k_describe_new(Geometry g, Batch b, Scratch s, Output out, Describe d) {
  pdl_wait();
  pdl_trigger();
  __shared__ uint32_t pat[kDescMaxBits];                  // pair i: 16-bit indices of its two box sums
  __shared__ uint32_t boxes[kNewWarps][kHalfRows * kBoxPitch];  // 5 x 5 sums, two rows per word
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < d.D; i += blockDim.x) {
    const char4 q = reinterpret_cast<const char4*>(d.pattern)[i];
    pat[i] = (uint32_t)box_half(q.y + kDescR, q.x + kDescR) |
             (uint32_t)box_half(q.w + kDescR, q.z + kDescR) << 16;
  }
  __syncthreads();

  const int T = b.T;
  const uint32_t* off = out.offsets;
  const long long first = off[0];
  const long long end = min((long long)off[T], out.cap);
  const long long last_first = off[T - 1];
  const int DW = d.D >> 5;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *d.count = (uint32_t)max(end, 0LL);
    const long long n_last = (long long)off[T] - last_first;
    const long long kept = max(0LL, end - last_first);
    *d.keep_n_out = (uint32_t)min(kept, d.keep_cap);
    if (kept < n_last || kept > d.keep_cap) atomicOr(s.overflow, 1);
  }
  const long long groups = end > first ? (end - first + 31) / 32 : 0;
  const uint2* recs = reinterpret_cast<const uint2*>(out.rec);
  uint32_t* bw = boxes[warp];
  for (;;) {
    unsigned long long gi = 0;
    if (lane == 0) gi = atomicAdd(d.next_group, 1u);
    gi = __shfl_sync(0xffffffffu, gi, 0);
    if ((long long)gi >= groups) break;
    const long long base = first + (long long)gi * 32;
    const long long idx = base + lane;
    uint2 r = make_uint2(0u, 0u);
    bool is_new = false;
    int k = 0;
    if (idx < end) {
      r = recs[idx];
      is_new = ((r.y >> 16) & FKD_KP_PROPAGATED) == 0u;
      if (is_new) k = find_item(T, (int)(idx - first), [&](int q) { return (int)(off[q] - first); });
    }
    uint32_t todo = __ballot_sync(0xffffffffu, is_new);
    while (todo) {
      const int src_lane = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t rx = __shfl_sync(0xffffffffu, r.x, src_lane);
      const uint32_t ry = __shfl_sync(0xffffffffu, r.y, src_lane);
      const int kk = __shfl_sync(0xffffffffu, k, src_lane);
      const long long ridx = base + src_lane;
      const int x = (int)(rx & 0xffffu), y = (int)(rx >> 16), l = (int)(ry & 0xffu);
      const LayerGeom& lg = g.layer[l];
      int pitch;
      const uint8_t* img = layer_base(g, b, s, kk, l, &pitch);

      const uint32_t mine = describe_record(img, pitch, lg.w, lg.h, x, y, pat, bw, DW, lane);
      if (lane < DW) d.desc[ridx * DW + lane] = mine;
      if (ridx >= last_first && ridx - last_first < d.keep_cap) {
        const long long kidx = ridx - last_first;
        if (lane < DW) d.keep_desc_out[kidx * DW + lane] = mine;
        if (lane == 0) reinterpret_cast<uint2*>(d.keep_rec_out)[kidx] = make_uint2(rx, ry);
      }
    }
  }
}

__global__ void __launch_bounds__(kCarriedThreads) k_describe_carried(Geometry g, Tables tb, Batch b, Scratch s,
                                                                      Output out, Describe d) {
  pdl_wait();
  pdl_trigger();
  const int T = b.T;
  const uint32_t* off = out.offsets;
  const long long first = off[0];
  const long long end = min((long long)off[T], out.cap);
  const long long last_first = off[T - 1];
  const int DW = d.D >> 5;
  const uint2* recs = reinterpret_cast<const uint2*>(out.rec);
  const uint2* keep = reinterpret_cast<const uint2*>(d.keep_rec_in);
  const long long n_keep = *d.keep_n_in;
  if (blockIdx.x == 0 && threadIdx.x == 0) *d.next_group = 0u;  // the new pass is done with it
  {
    // row starts of the last frame, relative to its first record: the kept
    // set's row index for the next batch
    const long long kept_end = min(end, last_first + d.keep_cap);
    const uint32_t* rb = out.row_base + (long long)(T - 1) * out.rows;
    for (int gr = blockIdx.x * blockDim.x + threadIdx.x; gr <= out.rows; gr += gridDim.x * blockDim.x) {
      const long long v = gr < out.rows ? (long long)rb[gr] : (long long)off[T];
      d.keep_row_out[gr] = (uint32_t)(min(max(v, last_first), max(kept_end, last_first)) - last_first);
    }
  }
  for (long long idx = first + blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < end;
       idx += (long long)gridDim.x * blockDim.x) {
    const uint2 r = recs[idx];
    if (((r.y >> 16) & FKD_KP_PROPAGATED) == 0u) continue;
    const int k = find_item(T, (int)(idx - first), [&](int q) { return (int)(off[q] - first); });
    const int x = (int)(r.x & 0xffffu), y = (int)(r.x >> 16), l = (int)(r.y & 0xffu);
    const LayerGeom& lg = g.layer[l];
    int sf = -1;  // the batch frame holding the record's origin, -1 = the kept set
    if (s.pmask) {
      const long long word = lg.bit_off + (long long)y * lg.wpr + (x >> 5);
      for (int q = k - 1; q >= 0; --q)
        if ((s.pmask[(long long)q * g.bit_words + word] >> (x & 31)) & 1u) {
          sf = q;
          break;
        }
    } else {
      const int bin = tb.rowblk[lg.row_off + y] * g.N_c + tb.colblk[lg.col_off + x];
      sf = s.src[(long long)k * g.NB + bin];
    }
    // the origin is in the same layer row of its frame: search that row only
    const unsigned long long key = rec_key(r);
    const int gr = lg.row_off + y;
    const uint32_t* from = nullptr;
    if (sf >= 0) {
      const uint32_t* rb = out.row_base + (long long)sf * out.rows;
      const long long lo = rb[gr], hi = gr + 1 < out.rows ? rb[gr + 1] : off[sf + 1];
      const long long j = find_record(recs, lo, min(hi, out.cap), key);
      if (j >= 0) from = d.desc + j * DW;
    } else {
      const long long j = find_record(keep, d.keep_row_in[gr], min((long long)d.keep_row_in[gr + 1], n_keep), key);
      if (j >= 0) from = d.keep_desc_in + j * DW;
    }
    if (!from) {
      atomicOr(d.missing, 1);  // only after an overflow dropped the origin record
      continue;
    }
    uint32_t* to = d.desc + idx * DW;
    const bool keep_it = idx >= last_first && idx - last_first < d.keep_cap;
    uint32_t* kto = keep_it ? d.keep_desc_out + (idx - last_first) * DW : nullptr;
    if ((DW & 3) == 0) {  // rows of 16-byte multiples: vector copies
      for (int q = 0; q < DW; q += 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(from + q);
        *reinterpret_cast<uint4*>(to + q) = v;
        if (kto) *reinterpret_cast<uint4*>(kto + q) = v;
      }
    } else {
      for (int q = 0; q < DW; ++q) {
        const uint32_t v = from[q];
        to[q] = v;
        if (kto) kto[q] = v;
      }
    }
    if (keep_it) reinterpret_cast<uint2*>(d.keep_rec_out)[idx - last_first] = r;
  }
}

// Group tick: one frame of each participating stream; a stream describes if
// its StreamDev has D > 0. The previous frame's records (rec[(n-1) & 1]) are
// the kept set, and its row starts index them. The tick's records, taken
// stream by stream, are numbered in a running sum that each warp (thread)
// keeps as it walks the items, so work is spread over all warps (threads)
// whatever the mix of streams.
__device__ __forceinline__ const uint8_t* group_layer(const StreamDev& d, const TickItem& ti, int l, int* pitch) {
  if (l == 0) {
    *pitch = ti.pitch;
    return ti.frame;
  }
  *pitch = d.g.layer[l].pitch;
  return d.s.pyr + d.g.layer[l].pyr_off;
}

constexpr int kGroupNewBlocks = 3;  // CTAs per SM of the group pass (its grid)

// Units of work of every tick item in shared memory: pre[i] = units of the
// items before item i, pre[n] = the tick's total. A unit is a group of 32
// records (`groups`) or one record of a frame with a previous frame; items of
// streams that do not describe have none. Ends with a barrier.
__device__ __forceinline__ void tick_prefix(const StreamDev* devs, const TickItem* items, int n, bool groups,
                                            uint32_t* pre) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const TickItem& ti = items[i];
    const StreamDev& d = devs[ti.sid];
    uint32_t u = 0;
    if (d.D && (groups || ti.frame_index > 0)) {
      const int par = (int)(ti.frame_index & 1);
      const long long first = d.rec_offsets[par][0];
      const long long end = min((long long)d.rec_offsets[par][1], d.K_max);
      const long long m = max(0LL, end - first);
      u = (uint32_t)(groups ? (m + 31) / 32 : m);
    }
    pre[i] = u;
  }
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan, 32 items at a time
    const int lane = threadIdx.x;
    uint32_t carry = 0;
    for (int c0 = 0; c0 < n; c0 += 32) {
      const int i = c0 + lane;
      const uint32_t v = i < n ? pre[i] : 0u;
      uint32_t incl = v;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, incl, dd);
        if (lane >= dd) incl += o;
      }
      if (i < n) pre[i] = carry + incl - v;
      carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) pre[n] = carry;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kNewWarps * 32, kGroupNewBlocks)
    k_group_describe_new(const StreamDev* devs, const TickHeader* hdr, const TickItem* items) {
  __shared__ uint32_t pat[kNewWarps][kDescMaxBits];       // the current stream's pairs, per warp
  __shared__ uint32_t boxes[kNewWarps][kHalfRows * kBoxPitch];
  __shared__ uint32_t pre[kMaxTickItems + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int n_items = hdr->n_items;
  tick_prefix(devs, items, n_items, true, pre);
  const uint32_t total = pre[n_items];
  uint32_t* bw = boxes[warp];
  uint32_t* pw = pat[warp];
  int loaded = -1;  // stream whose pairs are in pw
  // the tick's 32-record groups, numbered item after item, spread over the warps
  for (uint32_t g = blockIdx.x * kNewWarps + warp; g < total; g += gridDim.x * kNewWarps) {
    const int i = find_item(n_items, (int)g, [&](int q) { return (int)pre[q]; });
    const TickItem ti = items[i];
    const StreamDev& d = devs[ti.sid];
    const int par = (int)(ti.frame_index & 1);
    const long long first = d.rec_offsets[par][0];
    const long long end = min((long long)d.rec_offsets[par][1], d.K_max);
    const int DW = d.D >> 5;
    if (loaded != ti.sid) {
      __syncwarp();  // the previous stream's tests are done with pw
      for (int q = lane; q < d.D; q += 32) {
        const char4 c = reinterpret_cast<const char4*>(d.pattern)[q];
        pw[q] = (uint32_t)box_half(c.y + kDescR, c.x + kDescR) | (uint32_t)box_half(c.w + kDescR, c.z + kDescR) << 16;
      }
      __syncwarp();
      loaded = ti.sid;
    }
    const uint2* recs = reinterpret_cast<const uint2*>(d.rec[par]);
    const long long base = first + (long long)(g - pre[i]) * 32, idx = base + lane;
    uint2 r = make_uint2(0u, 0u);
    bool is_new = false;
    if (idx < end) {
      r = recs[idx];
      is_new = ((r.y >> 16) & FKD_KP_PROPAGATED) == 0u;
    }
    uint32_t todo = __ballot_sync(0xffffffffu, is_new);
    while (todo) {
      const int src_lane = __ffs(todo) - 1;
      todo &= todo - 1;
      const uint32_t rx = __shfl_sync(0xffffffffu, r.x, src_lane);
      const uint32_t ry = __shfl_sync(0xffffffffu, r.y, src_lane);
      const int x = (int)(rx & 0xffffu), y = (int)(rx >> 16), l = (int)(ry & 0xffu);
      const LayerGeom& lg = d.g.layer[l];
      int pitch;
      const uint8_t* img = group_layer(d, ti, l, &pitch);
      const uint32_t mine = describe_record(img, pitch, lg.w, lg.h, x, y, pw, bw, DW, lane);
      if (lane < DW) d.desc[par][(base + src_lane) * DW + lane] = mine;
    }
  }
}

__global__ void __launch_bounds__(kCarriedThreads)
    k_group_describe_carried(const StreamDev* devs, const TickHeader* hdr, const TickItem* items) {
  __shared__ uint32_t pre[kMaxTickItems + 1];
  const int n_items = hdr->n_items;
  tick_prefix(devs, items, n_items, false, pre);
  const uint32_t total = pre[n_items];
  // the tick's records (of frames with a previous frame), one per thread
  for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < total; u += gridDim.x * blockDim.x) {
    const int i = find_item(n_items, (int)u, [&](int q) { return (int)pre[q]; });
    const TickItem ti = items[i];
    const StreamDev& d = devs[ti.sid];
    const int par = (int)(ti.frame_index & 1), pp = par ^ 1;
    const long long idx = d.rec_offsets[par][0] + (long long)(u - pre[i]);
    const uint2 r = reinterpret_cast<const uint2*>(d.rec[par])[idx];
    if (((r.y >> 16) & FKD_KP_PROPAGATED) == 0u) continue;
    const int DW = d.D >> 5;
    const uint2* prev = reinterpret_cast<const uint2*>(d.rec[pp]);
    const long long prev_end = min((long long)d.rec_offsets[pp][1], d.K_max);
    const int y = (int)(r.x >> 16), l = (int)(r.y & 0xffu);
    const int gr = d.g.layer[l].row_off + y;
    const long long lo = d.row_base[pp][gr];
    const long long hi = gr + 1 < d.rows ? (long long)d.row_base[pp][gr + 1] : prev_end;
    const long long o = find_record(prev, lo, min(hi, prev_end), rec_key(r));
    if (o < 0) {
      atomicOr(d.s.overflow, 1);  // only after an overflow dropped the origin record
      continue;
    }
    const uint32_t* from = d.desc[pp] + o * DW;
    uint32_t* to = d.desc[par] + idx * DW;
    for (int q = 0; q < DW; ++q) to[q] = from[q];
  }
}

}  // namespace

void launch_describe(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s, const Output& out,
                     const Describe& d, cudaStream_t st) {
  const int sms = sm_count();
  pdl_launch(k_describe_new, dim3(sms * kNewMinBlocks), dim3(kNewWarps * 32), 0, st, g, b, s, out, d);
  pdl_launch(k_describe_carried, dim3(sms * 8), dim3(kCarriedThreads), 0, st, g, tb, b, s, out, d);
}

void launch_group_describe(const StreamDev* devs, const TickHeader* hdr, const TickItem* items, cudaStream_t st) {
  const int sms = sm_count();
  k_group_describe_new<<<sms * kGroupNewBlocks, kNewWarps * 32, 0, st>>>(devs, hdr, items);
  k_group_describe_carried<<<sms * 4, kCarriedThreads, 0, st>>>(devs, hdr, items);
}

}  // namespace fkd
