// k_assemble.cu -- the keypoint set D_n of every frame of a batch (Eq. 1),
// emitted in canonical (layer, y, x) order without sorting.
//
// A frame's keypoints live in a per-pixel bitmap whose word order is the
// canonical order (layers by scale, then rows, then columns). For bitmap word
// i of frame k, each bin the word's pixels fall in contributes its bits from
// the frame src(k, bin) -- the last frame up to k in which the bin was active
// -- or from the kept set D_{n0-1} when the bin was inactive since the batch
// began. The count pass sums the popcounts per chunk of words; the emit pass
// turns chunk counts and frame totals into output offsets, scans the words of
// its chunk, and writes one record per set bit, in order. The last frame of
// the batch also becomes the new kept set (bitmap, scores, keypoints per bin).
#include "fkd_internal.cuh"

namespace fkd {
namespace {

struct WordPos {
  int l, y, wx;
};

__device__ __forceinline__ WordPos word_pos(const Geometry& g, long long i) {
  int l = 0;
  while (l + 1 < g.L && g.layer[l + 1].bit_off <= i) ++l;
  const long long r = i - g.layer[l].bit_off;
  WordPos p;
  p.l = l;
  p.y = (int)(r / g.layer[l].wpr);
  p.wx = (int)(r % g.layer[l].wpr);
  return p;
}

// Bits of bitmap word i (position p) of frame k taken from their bins' source
// frames. prop receives the bits whose source is not frame k (carried over).
__device__ __forceinline__ uint32_t merged_word(const Geometry& g, const Tables& tb,
                                                const Scratch& s, const State& st, int k,
                                                long long i, const WordPos& p, uint32_t* prop) {
  const LayerGeom& lg = g.layer[p.l];
  const uint16_t* colblk = tb.colblk + lg.col_off;
  const int* xstart = tb.xstart + lg.xs_off;
  const int r = tb.rowblk[lg.row_off + p.y];
  const int xlo = p.wx * 32, xhi = min(xlo + 32, lg.w);
  const int c_lo = colblk[xlo], c_hi = colblk[xhi - 1];
  const int* srcrow = s.src + (long long)k * g.NB + r * g.N_c;
  uint32_t word = 0, pm = 0;
  for (int c = c_lo; c <= c_hi; ++c) {
    const int a = max(xstart[c], xlo) - xlo, e = min(xstart[c + 1], xhi) - xlo;
    if (e <= a) continue;
    const uint32_t m = (e - a == 32) ? 0xffffffffu : (((1u << (e - a)) - 1u) << a);
    const int sf = srcrow[c];
    const uint32_t bits = sf < 0 ? st.bits_in[i] : s.det_bits[(long long)sf * g.bit_words + i];
    word |= bits & m;
    if (sf != k) pm |= m;
  }
  *prop = pm & word;
  return word;
}

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = __reduce_add_sync(0xffffffffu, v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  uint32_t t = 0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
  return t;
}

__global__ void __launch_bounds__(kAsmThreads) k_count(Geometry g, Tables tb, Batch b, Scratch s,
                                                       State st) {
  __shared__ uint32_t red[kAsmThreads / 32];
  const int k = blockIdx.y, chunk = blockIdx.x;
  const long long w0 = (long long)chunk * kAsmChunkWords + (long long)threadIdx.x * kAsmWordsPerThread;
  uint32_t cnt = 0;
  for (int j = 0; j < kAsmWordsPerThread; ++j) {
    const long long i = w0 + j;
    if (i >= g.bit_words) break;
    uint32_t pm;
    cnt += __popc(merged_word(g, tb, s, st, k, i, word_pos(g, i), &pm));
  }
  const uint32_t tot = block_sum(cnt, red);
  if (threadIdx.x == 0) {
    s.chunk_counts[(long long)k * g.n_chunks + chunk] = tot;
    if (tot) atomicAdd(&s.frame_totals[k], tot);
  }
}

__global__ void __launch_bounds__(kAsmThreads) k_emit(Geometry g, Tables tb, Batch b, Scratch s,
                                                      State st, Output out) {
  __shared__ uint32_t red[kAsmThreads / 32];
  __shared__ uint32_t wsum[kAsmThreads / 32];
  const int k = blockIdx.y, chunk = blockIdx.x;
  const bool last = k == b.T - 1;

  // offsets: kept-set base of this call + earlier frames + earlier chunks
  uint32_t part = 0;
  for (int q = threadIdx.x; q < k; q += blockDim.x) part += s.frame_totals[q];
  const uint32_t frame_base = block_sum(part, red);
  part = 0;
  for (int q = threadIdx.x; q < chunk; q += blockDim.x)
    part += s.chunk_counts[(long long)k * g.n_chunks + q];
  const uint32_t chunk_base = block_sum(part, red);
  const unsigned long long call_base = s.out_base[out.base_slot];
  if (chunk == 0 && threadIdx.x == 0) {
    out.offsets[k] = (uint32_t)(call_base + frame_base);
    if (last) {
      const unsigned long long end = call_base + frame_base + s.frame_totals[k];
      out.offsets[k + 1] = (uint32_t)end;
      s.out_base[out.base_slot ^ 1] = end;
    }
  }

  // this thread's words (contiguous, so the scan order is the canonical order)
  const long long w0 = (long long)chunk * kAsmChunkWords + (long long)threadIdx.x * kAsmWordsPerThread;
  uint32_t words[kAsmWordsPerThread], props[kAsmWordsPerThread];
  uint32_t cnt = 0;
#pragma unroll
  for (int j = 0; j < kAsmWordsPerThread; ++j) {
    const long long i = w0 + j;
    words[j] = props[j] = 0;
    if (i < g.bit_words) {
      words[j] = merged_word(g, tb, s, st, k, i, word_pos(g, i), &props[j]);
      if (last) st.bits_out[i] = words[j];
      cnt += __popc(words[j]);
    }
  }
  // exclusive scan of cnt over the CTA
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t incl = cnt;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
    if (lane >= d) incl += v;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  uint32_t before = 0;
  for (int q = 0; q < wid; ++q) before += wsum[q];
  unsigned long long idx = call_base + frame_base + chunk_base + before + incl - cnt;

  if (cnt == 0) return;
  for (int j = 0; j < kAsmWordsPerThread; ++j) {
    uint32_t wv = words[j];
    if (!wv) continue;
    const long long i = w0 + j;
    const WordPos pos = word_pos(g, i);
    const LayerGeom& lg = g.layer[pos.l];
    const int r = tb.rowblk[lg.row_off + pos.y];
    const int* srcrow = s.src + (long long)k * g.NB + r * g.N_c;
    const long long row_off = lg.score_off + (long long)pos.y * lg.pitch;
    while (wv) {
      const int bit = __ffs(wv) - 1;
      wv &= wv - 1;
      const int x = pos.wx * 32 + bit;
      const int c = tb.colblk[lg.col_off + x];
      const int sf = srcrow[c];
      const uint8_t score = sf < 0 ? st.score_in[row_off + x]
                                   : s.det_score[(long long)sf * g.score_bytes + row_off + x];
      const uint32_t flags = (props[j] >> bit) & 1u;
      if (idx < (unsigned long long)out.cap) {
        uint2 rec;
        rec.x = (uint32_t)x | ((uint32_t)pos.y << 16);
        rec.y = (uint32_t)pos.l | ((uint32_t)score << 8) | (flags << 16);
        reinterpret_cast<uint2*>(out.rec)[idx] = rec;
      } else {
        *s.overflow = 1;
      }
      ++idx;
      if (last) {
        st.score_out[row_off + x] = score;
        atomicAdd(&st.cnt_out[r * g.N_c + c], 1u);
      }
    }
  }
}

}  // namespace

void launch_count(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                  const State& state, cudaStream_t st) {
  k_count<<<dim3(g.n_chunks, b.T), kAsmThreads, 0, st>>>(g, tb, b, s, state);
}

void launch_emit(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                 const State& state, const Output& out, cudaStream_t st) {
  k_emit<<<dim3(g.n_chunks, b.T), kAsmThreads, 0, st>>>(g, tb, b, s, state, out);
}

}  // namespace fkd
