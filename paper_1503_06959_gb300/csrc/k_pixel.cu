// k_pixel.cu -- Eq. 2 per pixel of every layer (mask mode FKD_MASK_IDP,
// option (i) of Sec. 3.1: the mask of layer l decides the pixels of layer l)
// and Eq. 1 with per-pixel masks.
//
//   k_pixel_mask:  bit of pixel p of layer l in frame k = |L_k,l(p) - L_{k-1},l(p)|
//                  > T_I (every pixel on the stream's first frame), stored in
//                  the layout of the keypoint bitmaps;
//   k_count_pixel: D_k = (detections of frame k & M_k) | (D_{k-1} & ~M_k),
//                  word by word, the frames of the batch in order (each word
//                  position is one thread). The score of a carried keypoint
//                  is copied into frame k's score map, so that the records
//                  of every frame read their scores from their own frame.
//                  Counts per chunk and frame feed the same emission pass as
//                  the bin masks.
#include <algorithm>

#include "fkd_internal.cuh"

namespace fkd {
namespace {

// Layer and word of word j of a frame's bitmap (layers in order).
__device__ __forceinline__ int layer_of_word(const Geometry& g, long long j) {
  int l = 0;
  while (l + 1 < g.L && g.layer[l + 1].bit_off <= j) ++l;
  return l;
}

// Per byte: bit 7 set where e > T (0 <= T <= 254), without carries across bytes.
__device__ __forceinline__ uint32_t bytes_gt(uint32_t e, uint32_t t1_low7, bool t1_high) {
  const uint32_t u = (e | 0x80808080u) - t1_low7;  // T + 1 in every byte, low 7 bits
  return (t1_high ? (e & u) : (e | u)) & 0x80808080u;
}

__device__ __forceinline__ uint32_t gather_bits(uint32_t g) {
  // bit 7 of byte i -> bit i (the four bits land on distinct product bits)
  return (((g >> 7) & 0x01010101u) * 0x00204081u >> 21) & 0xfu;
}

__global__ void __launch_bounds__(256) k_pixel_mask(Geometry g, Batch b, Scratch s, Params p) {
  const long long total = (long long)b.T * g.bit_words;
  const uint32_t T1 = (uint32_t)p.T_I + 1u;
  const bool none = T1 > 255u;  // |d| <= 255 never exceeds T_I >= 255
  const uint32_t t1_low7 = (T1 & 0x7fu) * 0x01010101u;
  const bool t1_high = T1 >= 128u;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / g.bit_words);
    const long long j = i - (long long)k * g.bit_words;
    const int l = layer_of_word(g, j);
    const LayerGeom& lg = g.layer[l];
    const int y = (int)((j - lg.bit_off) / lg.wpr), wx = (int)((j - lg.bit_off) % lg.wpr);
    const int x0 = wx * 32, nx = min(32, lg.w - x0);
    const uint32_t valid = nx >= 32 ? 0xffffffffu : ((1u << nx) - 1u);
    uint32_t m;
    if (b.first_frame + k == 0) {
      m = valid;
    } else if (none) {
      m = 0u;
    } else {
      const uint8_t *cur, *prv;
      if (l == 0) {
        cur = b.frames + (long long)k * b.frame_stride + (long long)y * b.pitch;
        prv = (k > 0 ? b.frames + (long long)(k - 1) * b.frame_stride : b.prev) +
              (long long)y * (k > 0 ? b.pitch : b.prev_pitch);
      } else {
        cur = s.pyr + (long long)k * g.pyr_bytes + lg.pyr_off + (long long)y * lg.pitch;
        prv = (k > 0 ? s.pyr + (long long)(k - 1) * g.pyr_bytes : s.pyr_last) + lg.pyr_off +
              (long long)y * lg.pitch;
      }
      m = 0u;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int x = x0 + 4 * q;
        if (x >= lg.w) break;
        uint32_t a = 0u, c = 0u;
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (x + e < lg.w) {
            a |= (uint32_t)cur[x + e] << (8 * e);
            c |= (uint32_t)prv[x + e] << (8 * e);
          }
        m |= gather_bits(bytes_gt(__vabsdiffu4(a, c), t1_low7, t1_high)) << (4 * q);
      }
      m &= valid;
    }
    s.pmask[i] = m;
  }
}

// Last-CTA scan of the frame totals into record offsets (as the bin-mask
// count pass does).
__device__ __forceinline__ void scan_bases(const Scratch& s, int T) {
  const int lane = threadIdx.x & 31;
  __threadfence();
  uint32_t carry = 0;
  for (int e0 = 0; e0 < T; e0 += 32) {
    const int e = e0 + lane;
    const uint32_t c = e < T ? __ldcg(&s.frame_totals[e]) : 0u;
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    if (e < T) s.bases[e] = carry + incl - c;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) {
    s.bases[T] = carry;
    *s.done = 0u;
  }
}

constexpr int kCountThreads = 256;

__global__ void __launch_bounds__(kCountThreads) k_count_pixel(Geometry g, Tables tb, Batch b, Scratch s,
                                                               State st) {
  __shared__ int last_cta;
  const int lane = threadIdx.x & 31;
  const long long j = blockIdx.x * (long long)kCountThreads + threadIdx.x;
  const bool valid = j < g.bit_words;
  int l = 0, y = 0, wx = 0, chunk = -1;
  if (valid) {
    l = layer_of_word(g, j);
    const LayerGeom& lg = g.layer[l];
    y = (int)((j - lg.bit_off) / lg.wpr);
    wx = (int)((j - lg.bit_off) % lg.wpr);
    chunk = tb.rowchunk[lg.row_off + y];
  }
  const LayerGeom& lg = g.layer[l];
  // all lanes in one chunk: one atomic per warp, else one per lane
  const int chunk0 = __shfl_sync(0xffffffffu, chunk, 0);
  const bool one_chunk = __all_sync(0xffffffffu, !valid || chunk == chunk0);
  uint32_t prev = valid ? st.bits_in[j] : 0u;
  for (int k = 0; k < b.T; ++k) {
    uint32_t merged = 0u;
    if (valid) {
      const uint32_t m = s.pmask[(long long)k * g.bit_words + j];
      const uint32_t d = s.det_bits[(long long)k * g.bit_words + j];
      const uint32_t carried = prev & ~m;
      merged = (d & m) | carried;
      s.merged[(long long)k * g.bit_words + j] = merged;
      if (carried) {
        // a carried keypoint keeps its score: copy it into frame k's map
        uint8_t* dst = s.det_score + (long long)k * g.score_bytes + lg.score_off + (long long)y * lg.pitch;
        const uint8_t* src = k > 0 ? s.det_score + (long long)(k - 1) * g.score_bytes + lg.score_off +
                                         (long long)y * lg.pitch
                                   : st.score_in + lg.score_off + (long long)y * lg.pitch;
        for (uint32_t c = carried; c; c &= c - 1) {
          const int x = wx * 32 + __ffs(c) - 1;
          dst[x] = src[x];
        }
      }
      prev = merged;
    }
    const uint32_t cnt = __popc(merged);
    if (one_chunk) {
      const uint32_t sum = __reduce_add_sync(0xffffffffu, cnt);
      if (lane == 0 && sum) {
        atomicAdd(&s.chunk_counts[(long long)k * g.n_chunks + chunk0], sum);
        atomicAdd(&s.frame_totals[k], sum);
      }
    } else if (cnt) {
      atomicAdd(&s.chunk_counts[(long long)k * g.n_chunks + chunk], cnt);
      atomicAdd(&s.frame_totals[k], cnt);
    }
  }
  // the CTA that finishes last turns the frame totals into offsets
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last_cta = atomicAdd(s.done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last_cta && threadIdx.x < 32) scan_bases(s, b.T);
}

}  // namespace

void launch_pixel_mask(const Geometry& g, const Batch& b, const Scratch& s, const Params& p,
                       cudaStream_t st) {
  const long long total = (long long)b.T * g.bit_words;
  const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)sm_count() * 16);
  k_pixel_mask<<<std::max(blocks, 1), 256, 0, st>>>(g, b, s, p);
}

void launch_count_pixel(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                        const State& state, cudaStream_t st) {
  const int blocks = (int)((g.bit_words + kCountThreads - 1) / kCountThreads);
  k_count_pixel<<<std::max(blocks, 1), kCountThreads, 0, st>>>(g, tb, b, s, state);
}

}  // namespace fkd
