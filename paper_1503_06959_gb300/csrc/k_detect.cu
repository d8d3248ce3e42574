// k_detect.cu -- masked segment test, corner score and 3x3 non-maximum
// suppression (Sec. 2) over the active detection tiles of a batch.
//
// Persistent CTAs walk the compacted list of active (frame, tile) items. Per
// item the CTA
//   A. stages the tile plus a 4-pixel halo in shared memory with 16-byte loads;
//   B. prefilters every pixel whose score the tile needs (the tile and a
//      1-pixel ring) with packed byte arithmetic, 4 pixels per 32-bit word: a
//      pixel can only pass the segment test at threshold t if two adjacent
//      compass points of its ring (12, 3, 6, 9 o'clock) differ from it by more
//      than t, since every 9-pixel arc of the 16-pixel ring contains two
//      adjacent ones; candidates are compacted with warp ballots;
//   C. scores the candidates exactly, two pixels per 32-bit word in 16-bit
//      lanes: with I_k the ring values, the bright score is
//      max over arcs of (min over the arc of I_k) - I_p and the dark score
//      I_p - min over arcs of (max over the arc of I_k); arc minima come from
//      3-input minima of 3-input minima;
//   D. keeps a candidate when its score is >= t and strictly above its 8
//      neighbours' scores (scores below t count as 0, which never changes the
//      outcome), and writes the tile's keypoint bitmap and scores.
// Bins are not consulted here: assembly takes each pixel from the frame its
// bin points to, so the kernel only has to be right on every pixel of every
// tile it processes.
#include "fkd_internal.cuh"

namespace fkd {
namespace {

constexpr int TW = kDetTW, TH = kDetTH;
constexpr int IN_W = TW + 32;  // smem input row: layer x in [x0-16, x0+TW+16)
constexpr int IN_H = TH + 8;   // smem input rows: layer y in [y0-4, y0+TH+4)
constexpr int SC_W = TW + 2;   // scores of x in [x0-1, x0+TW]
constexpr int SC_H = TH + 2;   // and y in [y0-1, y0+TH]
constexpr int PW = TW / 4 + 2; // prefilter words per row: x in [x0-4, x0+TW+4)
constexpr int PWORDS = PW * SC_H;
constexpr int MAX_CAND = PWORDS * 4;
static_assert(IN_W <= 256, "candidate entries pack the column in 8 bits");
static_assert(TW % 32 == 0, "bitmap words are whole inside a tile");

// Per byte: bit 7 set where e >= T1 (T1 in 1..255, the same in every byte).
__device__ __forceinline__ uint32_t bytes_ge(uint32_t e, uint32_t t1_low7, bool t1_high) {
  const uint32_t u = (e | 0x80808080u) - t1_low7;  // no borrow crosses a byte
  return t1_high ? (e & u) : (e | u);
}

__device__ __forceinline__ uint32_t ld32(const uint8_t* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// 16 ring samples of two pixels, packed in 16-bit lanes: ring order starts
// straight above the pixel and turns clockwise (y grows downwards).
#define FKD_RING(X)                                                                     \
  X(0, 0, -3) X(1, 1, -3) X(2, 2, -2) X(3, 3, -1) X(4, 3, 0) X(5, 3, 1) X(6, 2, 2)    \
  X(7, 1, 3) X(8, 0, 3) X(9, -1, 3) X(10, -2, 2) X(11, -3, 1) X(12, -3, 0)            \
  X(13, -3, -1) X(14, -2, -2) X(15, -1, -3)

// Exact scores of two pixels at smem offsets o1, o2 (score in 16-bit lanes).
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

__global__ void __launch_bounds__(kDetThreads) k_detect(Geometry g, Batch b, Scratch s, Tables tb,
                                                        Params p) {
  __shared__ __align__(16) uint8_t in[IN_H * IN_W];
  __shared__ uint8_t sc[SC_H * SC_W];
  __shared__ uint16_t cand[MAX_CAND];
  __shared__ uint32_t detw[TH * (TW / 32)];
  __shared__ int ncand;

  const uint32_t count = *s.work_count;
  const int tid = threadIdx.x, lane = tid & 31;
  const uint32_t t1 = (uint32_t)p.t + 1u;  // score >= t  <=>  some arc beyond I_p +- t
  const uint32_t t1_low7 = (t1 & 0x7fu) * 0x01010101u;
  const bool t1_high = t1 >= 128u;
  const bool none = t1 > 255u;

  for (uint32_t item = blockIdx.x; item < count; item += gridDim.x) {
    const uint32_t wi = s.work[item];
    const int k = (int)(wi / (uint32_t)g.n_tiles);
    const DetTile tile = tb.tiles[wi % (uint32_t)g.n_tiles];
    const int l = tile.layer;
    const LayerGeom& lg = g.layer[l];
    const int w = lg.w, h = lg.h;
    const int x0 = tile.tx * TW, y0 = tile.ty * TH;
    const uint8_t* src;
    int pitch;
    if (l == 0) {
      src = b.frames + (long long)k * b.frame_stride;
      pitch = b.pitch;
    } else {
      src = s.pyr + (long long)k * g.pyr_bytes + lg.pyr_off;
      pitch = lg.pitch;
    }
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | (uintptr_t)pitch) & 15) == 0;

    // A. stage rows y0-4 .. y0+TH+3, columns x0-16 .. x0+TW+15 (zeros outside)
    for (int q = tid; q < IN_H * (IN_W / 16); q += blockDim.x) {
      const int r = q / (IN_W / 16), c = (q % (IN_W / 16)) * 16;
      const int gy = y0 - 4 + r, gx = x0 - 16 + c;
      uint8_t* d = in + r * IN_W + c;
      if (gy >= 0 && gy < h && vec && gx >= 0 && gx + 16 <= w) {
        *reinterpret_cast<uint4*>(d) =
            __ldg(reinterpret_cast<const uint4*>(src + (long long)gy * pitch + gx));
      } else {
        const bool row_ok = gy >= 0 && gy < h;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          d[j] = (row_ok && gx + j >= 0 && gx + j < w) ? src[(long long)gy * pitch + gx + j] : 0;
      }
    }
    for (int q = tid; q < SC_H * SC_W; q += blockDim.x) sc[q] = 0;
    if (tid < TH * (TW / 32)) detw[tid] = 0;
    if (tid == 0) ncand = 0;
    __syncthreads();

    // B. prefilter, 4 pixels per word; word j of score row rr covers
    //    x = x0-4+4j .. x0-1+4j, y = y0-1+rr; in smem: row rr+3, column 12+4j.
    for (int base = 0; base < PWORDS; base += blockDim.x) {
      const int q = base + tid;
      uint32_t keep = 0;
      int r = 0, c = 0;
      if (q < PWORDS && !none) {
        const int rr = q / PW, j = q % PW;
        r = rr + 3;
        c = 12 + 4 * j;
        const uint8_t* row = in + r * IN_W + c;
        const uint32_t C = ld32(row), Cp = ld32(row - 4), Cn = ld32(row + 4);
        const uint32_t N = ld32(row - 3 * IN_W), S = ld32(row + 3 * IN_W);
        const uint32_t E = __funnelshift_r(C, Cn, 24);  // x+3
        const uint32_t Wd = __funnelshift_r(Cp, C, 8);  // x-3
        const uint32_t gN = bytes_ge(__vabsdiffu4(N, C), t1_low7, t1_high);
        const uint32_t gS = bytes_ge(__vabsdiffu4(S, C), t1_low7, t1_high);
        const uint32_t gE = bytes_ge(__vabsdiffu4(E, C), t1_low7, t1_high);
        const uint32_t gW = bytes_ge(__vabsdiffu4(Wd, C), t1_low7, t1_high);
        keep = (gN | gS) & (gE | gW) & 0x80808080u;
        if (keep) {
          // only the score region, and no pixel within 3 of the layer edge
          const int gy = y0 - 1 + rr, gx = x0 - 4 + 4 * j;
          if (gy < 3 || gy >= h - 3) keep = 0;
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int x = gx + i;
            const bool ok = x >= 3 && x < w - 3 && x >= x0 - 1 && x <= x0 + TW;
            if (!ok) keep &= ~(0x80u << (8 * i));
          }
        }
      }
      unsigned bal[4];
      int tot = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        bal[i] = __ballot_sync(0xffffffffu, (keep >> (8 * i + 7)) & 1u);
        tot += __popc(bal[i]);
      }
      if (tot) {
        int wbase = 0;
        if (lane == 0) wbase = atomicAdd(&ncand, tot);
        wbase = __shfl_sync(0xffffffffu, wbase, 0);
        const unsigned lt = (1u << lane) - 1u;
        int off = wbase;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          if ((bal[i] >> lane) & 1u) cand[off + __popc(bal[i] & lt)] = (uint16_t)((r << 8) | (c + i));
          off += __popc(bal[i]);
        }
      }
    }
    __syncthreads();

    // C. exact scores of the candidates, two per thread
    const int nc = ncand;
    for (int pi = tid; 2 * pi < nc; pi += blockDim.x) {
      const int e1 = cand[2 * pi], e2 = cand[min(2 * pi + 1, nc - 1)];
      const int o1 = (e1 >> 8) * IN_W + (e1 & 255), o2 = (e2 >> 8) * IN_W + (e2 & 255);
      const uint32_t sp = score_pair(in, o1, o2);
      const uint32_t s1 = sp & 0xffffu, s2 = sp >> 16;
      sc[((e1 >> 8) - 3) * SC_W + (e1 & 255) - 15] = s1 >= (uint32_t)p.t ? (uint8_t)s1 : 0;
      if (2 * pi + 1 < nc)
        sc[((e2 >> 8) - 3) * SC_W + (e2 & 255) - 15] = s2 >= (uint32_t)p.t ? (uint8_t)s2 : 0;
    }
    __syncthreads();

    // D. strict 3x3 maxima among the tile's own pixels
    uint8_t* dscore = s.det_score + (long long)k * g.score_bytes + lg.score_off;
    for (int ci = tid; ci < nc; ci += blockDim.x) {
      const int e = cand[ci];
      const int r = e >> 8, c = e & 255;
      if (r < 4 || r >= TH + 4 || c < 16 || c >= TW + 16) continue;
      const uint8_t* sp = sc + (r - 3) * SC_W + (c - 15);
      const int v = sp[0];
      if (v == 0) continue;
      const bool is_max = v > sp[-SC_W - 1] && v > sp[-SC_W] && v > sp[-SC_W + 1] && v > sp[-1] &&
                          v > sp[1] && v > sp[SC_W - 1] && v > sp[SC_W] && v > sp[SC_W + 1];
      if (is_max) {
        const int lx = c - 16, ly = r - 4;
        atomicOr(&detw[ly * (TW / 32) + (lx >> 5)], 1u << (lx & 31));
        dscore[(long long)(y0 + ly) * lg.pitch + x0 + lx] = (uint8_t)v;
      }
    }
    __syncthreads();

    // E. the tile's bitmap words
    if (tid < TH * (TW / 32)) {
      const int ly = tid / (TW / 32), wx = tid % (TW / 32);
      const int gy = y0 + ly, gw = x0 / 32 + wx;
      if (gy < h && gw < lg.wpr)
        s.det_bits[(long long)k * g.bit_words + lg.bit_off + (long long)gy * lg.wpr + gw] = detw[tid];
    }
    __syncthreads();
  }
}

}  // namespace

int detect_grid_size() {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_detect, kDetThreads, 0);
  if (sms <= 0) sms = 1;
  if (per_sm <= 0) per_sm = 1;
  return sms * per_sm;
}

void launch_detect(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                   const Params& p, int grid, cudaStream_t st) {
  k_detect<<<grid, kDetThreads, 0, st>>>(g, b, s, tb, p);
}

}  // namespace fkd
