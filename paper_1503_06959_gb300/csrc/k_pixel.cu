// k_pixel.cu -- Eq. 2 per pixel of every layer (mask mode FKD_MASK_IDP,
// option (i) of Sec. 3.1: the mask of layer l decides the pixels of layer l)
// and Eq. 1 with per-pixel masks.
//
//   k_pixel_mask:  bit of pixel p of layer l in frame k = |L_k,l(p) - L_{k-1},l(p)|
//                  > T_I (every pixel on the stream's first frame), stored in
//                  the layout of the keypoint bitmaps;
//   k_merge_pixel: D_k = (detections of frame k & M_k) | (D_{k-1} & ~M_k),
//                  pixel by pixel, the frames of the batch in order (each
//                  pixel is one lane). The score of a carried keypoint is
//                  copied into frame k's score map, so that the records of
//                  every frame read their scores from their own frame. The
//                  bin-mask count pass then counts the merged words, and
//                  the same emission pass writes the records.
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
  pdl_wait();
  pdl_trigger();
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
      uint32_t a[8], c[8];
      const bool vec = nx == 32 && (((reinterpret_cast<uintptr_t>(cur + x0)) | reinterpret_cast<uintptr_t>(prv + x0)) & 15) == 0;
      if (vec) {  // 32 aligned bytes of each: two 16-byte loads
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const uint4 va = reinterpret_cast<const uint4*>(cur + x0)[h], vc = reinterpret_cast<const uint4*>(prv + x0)[h];
          a[4 * h] = va.x; a[4 * h + 1] = va.y; a[4 * h + 2] = va.z; a[4 * h + 3] = va.w;
          c[4 * h] = vc.x; c[4 * h + 1] = vc.y; c[4 * h + 2] = vc.z; c[4 * h + 3] = vc.w;
        }
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          a[q] = c[q] = 0u;
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (4 * q + e < nx) {
              a[q] |= (uint32_t)cur[x0 + 4 * q + e] << (8 * e);
              c[q] |= (uint32_t)prv[x0 + 4 * q + e] << (8 * e);
            }
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) m |= gather_bits(bytes_gt(__vabsdiffu4(a[q], c[q]), t1_low7, t1_high)) << (4 * q);
      m &= valid;
    }
    s.pmask[i] = m;
  }
}

// One warp per bitmap word, one lane per pixel of it: each lane runs the
// recurrence of its own pixel over the frames of the batch (keeping the
// pixel's keypoint score in a register while it is carried), and a ballot
// forms each frame's word. The counting pass then reads the merged words.
constexpr int kMergeWarps = 8;

__global__ void __launch_bounds__(kMergeWarps * 32) k_merge_pixel(Geometry g, Batch b, Scratch s, State st) {
  pdl_wait();
  pdl_trigger();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long j = blockIdx.x * (long long)kMergeWarps + warp;
  if (j >= g.bit_words) return;  // whole warps leave together
  const int l = layer_of_word(g, j);
  const LayerGeom& lg = g.layer[l];
  const int y = (int)((j - lg.bit_off) / lg.wpr), wx = (int)((j - lg.bit_off) % lg.wpr);
  const long long so = lg.score_off + (long long)y * lg.pitch + wx * 32 + lane;  // this lane's pixel
  uint32_t bit = (st.bits_in[j] >> lane) & 1u;
  // the keypoint's score is read only when it is first carried: from the
  // frame that detected it (src >= 0) or from the kept set (src = -1)
  int src = -1;
  bool have = false;
  uint8_t score = 0;
  // the mask and detection words of the next frames are loaded ahead (lane
  // q < AHEAD holds frame k + q's; the warp reads them by shuffles)
  constexpr int AHEAD = 16;
  uint32_t pm = 0u, pd = 0u;
  for (int k = 0; k < b.T; ++k) {
    if ((k % AHEAD) == 0) {
      const int kk = k + lane;
      pm = lane < AHEAD && kk < b.T ? s.pmask[(long long)kk * g.bit_words + j] : 0u;
      pd = lane < AHEAD && kk < b.T ? s.det_bits[(long long)kk * g.bit_words + j] : 0u;
    }
    const uint32_t m = (__shfl_sync(0xffffffffu, pm, k % AHEAD) >> lane) & 1u;
    const uint32_t d = (__shfl_sync(0xffffffffu, pd, k % AHEAD) >> lane) & 1u;
    if (m) {
      bit = d;  // detected anew, or nothing
      src = k;
      have = false;
    } else if (bit) {
      // carried: its score goes into frame k's map
      if (!have) {
        score = src < 0 ? st.score_in[so] : s.det_score[(long long)src * g.score_bytes + so];
        have = true;
      }
      s.det_score[(long long)k * g.score_bytes + so] = score;
    }
    const uint32_t word = __ballot_sync(0xffffffffu, bit != 0u);
    if (lane == 0) s.merged[(long long)k * g.bit_words + j] = word;
  }
}

}  // namespace

void launch_pixel_mask(const Geometry& g, const Batch& b, const Scratch& s, const Params& p,
                       cudaStream_t st) {
  const long long total = (long long)b.T * g.bit_words;
  const int blocks = (int)std::min<long long>((total + 255) / 256, (long long)sm_count() * 16);
  pdl_launch(k_pixel_mask, dim3(std::max(blocks, 1)), dim3(256), 0, st, g, b, s, p);
}

void launch_count_pixel(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                        const State& state, cudaStream_t st) {
  const int blocks = (int)((g.bit_words + kMergeWarps - 1) / kMergeWarps);
  pdl_launch(k_merge_pixel, dim3(std::max(blocks, 1)), dim3(kMergeWarps * 32), 0, st, g, b, s, state);
  launch_count(g, tb, b, s, state, st);  // counts the merged words
}

}  // namespace fkd
