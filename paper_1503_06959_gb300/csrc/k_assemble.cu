// k_assemble.cu -- the keypoint set D_n of every frame of a batch (Eq. 1),
// emitted in canonical (layer, y, x) order without sorting.
//
// A frame's keypoints live in a per-pixel bitmap whose word order is the
// canonical order (layers by scale, then rows, then columns). For bitmap word
// i of frame k, each bin the word's pixels fall in contributes its bits from
// the frame src(k, bin) -- the last frame up to k in which the bin was active
// -- or from the kept set D_{n0-1} when the bin was inactive since the batch
// began. Work is cut into chunks of whole rows of one layer, so a CTA knows
// its layer and each row's bin row up front.
//   k_count: merge each word from its sources, store it, and sum the
//            popcounts per chunk and per frame;
//   k_emit:  turn chunk counts and frame totals into output offsets, scan the
//            chunk's stored words, and write one record per set bit, in order.
// The last frame of the batch also becomes the new kept set (bitmap, scores,
// keypoints per bin).
#include "fkd_internal.cuh"

namespace fkd {
namespace {

constexpr int kXsSmem = 1024;  // bin-column starts kept in shared memory when N_c < this

__device__ __forceinline__ uint32_t block_sum(uint32_t v, uint32_t* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = __reduce_add_sync(0xffffffffu, v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  uint32_t t = 0;
#pragma unroll
  for (int q = 0; q < kAsmThreads / 32; ++q) t += red[q];
  return t;
}

// Merge and count one chunk of frame k; ends with the block reduction's
// barriers, so a CTA can run it again at once.
__device__ __forceinline__ void count_chunk(const Geometry& g, const Tables& tb, const Scratch& s,
                                            const State& st, int k, int chunk) {
  __shared__ int xs[kXsSmem];
  __shared__ uint32_t red[kAsmThreads / 32];
  const AsmChunk ch = tb.chunks[chunk];
  const LayerGeom& lg = g.layer[ch.layer];
  const int wpr = lg.wpr, w = lg.w;
  const int nwords = (ch.y1 - ch.y0) * wpr;
  const long long word0 = lg.bit_off + (long long)ch.y0 * wpr;
  const int* xsg = tb.xstart + lg.xs_off;
  const bool xs_local = g.N_c < kXsSmem;
  if (xs_local)
    for (int q = threadIdx.x; q <= g.N_c; q += kAsmThreads) xs[q] = xsg[q];
  __syncthreads();
  const int* xst = xs_local ? xs : xsg;

  const int* src_k = s.src + (long long)k * g.NB;
  const uint32_t* det0 = s.det_bits + word0;
  uint32_t* out = s.merged + (long long)k * g.bit_words + word0;
  int j = threadIdx.x * kAsmWordsPerThread;
  int y = ch.y0 + j / wpr, wx = j % wpr;
  const int* srcrow = src_k + (j < nwords ? tb.rowblk[lg.row_off + y] : 0) * g.N_c;
  uint32_t cnt = 0;
  for (int jj = 0; jj < kAsmWordsPerThread && j < nwords; ++jj, ++j) {
    const uint32_t wb = tb.wbins[lg.wb_off + wx];
    const int c_lo = wb & 0xffffu, c_hi = wb >> 16;
    uint32_t word;
    if (c_lo == c_hi) {
      const int sf = srcrow[c_lo];
      word = sf < 0 ? st.bits_in[word0 + j] : det0[(long long)sf * g.bit_words + j];
    } else {
      const int xlo = wx * 32, xhi = min(xlo + 32, w);
      word = 0;
      for (int c = c_lo; c <= c_hi; ++c) {
        const int a = max(xst[c], xlo) - xlo, e = min(xst[c + 1], xhi) - xlo;
        if (e <= a) continue;
        const uint32_t m = (e - a == 32) ? 0xffffffffu : (((1u << (e - a)) - 1u) << a);
        const int sf = srcrow[c];
        const uint32_t bits = sf < 0 ? st.bits_in[word0 + j] : det0[(long long)sf * g.bit_words + j];
        word |= bits & m;
      }
    }
    out[j] = word;
    cnt += __popc(word);
    if (++wx == wpr) {
      wx = 0;
      ++y;
      if (y < ch.y1) srcrow = src_k + tb.rowblk[lg.row_off + y] * g.N_c;
    }
  }
  const uint32_t tot = block_sum(cnt, red);
  if (threadIdx.x == 0) {
    s.chunk_counts[(long long)k * g.n_chunks + chunk] = tot;
    if (tot) atomicAdd(&s.frame_totals[k], tot);
  }
  __syncthreads();  // xs and red are reused by the next chunk of this CTA
}

__device__ __forceinline__ void emit_records(const Geometry& g, const Tables& tb, const Scratch& s,
                                             const State& st, const Output& out, int k, bool last,
                                             const AsmChunk& ch, const LayerGeom& lg, int j0,
                                             const uint32_t* words, unsigned long long idx);

// Emit the records of one chunk of frame k of a batch of T frames; the last
// frame also writes the new kept set. Ends with a barrier.
__device__ __forceinline__ void emit_chunk(const Geometry& g, const Tables& tb, const Scratch& s,
                                           const State& st, const Output& out, int k, int T,
                                           int chunk) {
  __shared__ uint32_t red[kAsmThreads / 32];
  __shared__ uint32_t wsum[kAsmThreads / 32];
  const bool last = k == T - 1;
  const AsmChunk ch = tb.chunks[chunk];
  const LayerGeom& lg = g.layer[ch.layer];
  const int wpr = lg.wpr;
  const int nwords = (ch.y1 - ch.y0) * wpr;
  const long long word0 = lg.bit_off + (long long)ch.y0 * wpr;

  // offsets: base of this call + earlier frames + earlier chunks of this frame
  uint32_t part = 0;
  for (int q = threadIdx.x; q < k; q += kAsmThreads) part += s.frame_totals[q];
  const uint32_t frame_base = block_sum(part, red);
  part = 0;
  for (int q = threadIdx.x; q < chunk; q += kAsmThreads) part += s.chunk_counts[(long long)k * g.n_chunks + q];
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
  const int j0 = threadIdx.x * kAsmWordsPerThread;
  const uint32_t* merged = s.merged + (long long)k * g.bit_words + word0;
  uint32_t words[kAsmWordsPerThread];
  uint32_t cnt = 0;
#pragma unroll
  for (int jj = 0; jj < kAsmWordsPerThread; ++jj) {
    const int j = j0 + jj;
    words[jj] = j < nwords ? merged[j] : 0u;
    cnt += __popc(words[jj]);
    if (last && j < nwords) st.bits_out[word0 + j] = words[jj];
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
  if (cnt) emit_records(g, tb, s, st, out, k, last, ch, lg, j0, words, idx);
  __syncthreads();  // red and wsum are reused by the next chunk of this CTA
}

__device__ __forceinline__ void emit_records(const Geometry& g, const Tables& tb, const Scratch& s,
                                             const State& st, const Output& out, int k, bool last,
                                             const AsmChunk& ch, const LayerGeom& lg, int j0,
                                             const uint32_t* words, unsigned long long idx) {
  const int wpr = lg.wpr;
  const int* src_k = s.src + (long long)k * g.NB;
  const uint16_t* colblk = tb.colblk + lg.col_off;
  int y = ch.y0 + j0 / wpr, wx = j0 % wpr;
  for (int jj = 0; jj < kAsmWordsPerThread; ++jj) {
    uint32_t wv = words[jj];
    if (wv) {
      const int r = tb.rowblk[lg.row_off + y];
      const int* srcrow = src_k + r * g.N_c;
      const long long row_off = lg.score_off + (long long)y * lg.pitch;
      while (wv) {
        const int bit = __ffs(wv) - 1;
        wv &= wv - 1;
        const int x = wx * 32 + bit;
        const int c = colblk[x];
        const int sf = srcrow[c];
        const uint8_t score = sf < 0 ? st.score_in[row_off + x]
                                     : s.det_score[(long long)sf * g.score_bytes + row_off + x];
        const uint32_t flags = sf != k ? FKD_KP_PROPAGATED : 0u;
        if (idx < (unsigned long long)out.cap) {
          uint2 rec;
          rec.x = (uint32_t)x | ((uint32_t)y << 16);
          rec.y = (uint32_t)ch.layer | ((uint32_t)score << 8) | (flags << 16);
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
    if (++wx == wpr) {
      wx = 0;
      ++y;
    }
  }
}

__global__ void __launch_bounds__(kAsmThreads) k_count(Geometry g, Tables tb, Scratch s, State st) {
  count_chunk(g, tb, s, st, blockIdx.y, blockIdx.x);
}

__global__ void __launch_bounds__(kAsmThreads) k_emit(Geometry g, Tables tb, Batch b, Scratch s,
                                                      State st, Output out) {
  emit_chunk(g, tb, s, st, out, blockIdx.y, b.T, blockIdx.x);
}

__device__ __forceinline__ State state_of(const StreamDev& d, int cur) {
  State st;
  st.bits_in = d.state_bits[cur];
  st.score_in = d.state_score[cur];
  st.cnt_in = d.state_cnt[cur];
  st.bits_out = d.state_bits[cur ^ 1];
  st.score_out = d.state_score[cur ^ 1];
  st.cnt_out = d.state_cnt[cur ^ 1];
  return st;
}

// Group tick: persistent CTAs over the chunks of every participating frame.
__global__ void __launch_bounds__(kAsmThreads) k_group_count(const StreamDev* devs, const TickHeader* hdr,
                                                             const TickItem* items) {
  const int n = hdr->n_items, total = hdr->total_chunks;
  for (int j = blockIdx.x; j < total; j += gridDim.x) {
    const int i = find_item(n, j, [&](int q) { return items[q].chunk_base; });
    const TickItem it = items[i];
    const StreamDev& d = devs[it.sid];
    count_chunk(d.g, d.tb, d.s, state_of(d, it.state_cur), 0, j - it.chunk_base);
  }
}

__global__ void __launch_bounds__(kAsmThreads) k_group_emit(const StreamDev* devs, const TickHeader* hdr,
                                                            const TickItem* items) {
  const int n = hdr->n_items, total = hdr->total_chunks;
  for (int j = blockIdx.x; j < total; j += gridDim.x) {
    const int i = find_item(n, j, [&](int q) { return items[q].chunk_base; });
    const TickItem it = items[i];
    const StreamDev& d = devs[it.sid];
    const int par = (int)(it.frame_index & 1);
    Output o{d.rec[par], d.K_max, d.rec_offsets[par], 0};
    emit_chunk(d.g, d.tb, d.s, state_of(d, it.state_cur), o, 0, 1, j - it.chunk_base);
  }
}

}  // namespace

void launch_group_count(const StreamDev* devs, const TickHeader* hdr, const TickItem* items, int grid,
                        cudaStream_t st) {
  k_group_count<<<grid, kAsmThreads, 0, st>>>(devs, hdr, items);
}

void launch_group_emit(const StreamDev* devs, const TickHeader* hdr, const TickItem* items, int grid,
                       cudaStream_t st) {
  k_group_emit<<<grid, kAsmThreads, 0, st>>>(devs, hdr, items);
}

void launch_count(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                  const State& state, cudaStream_t st) {
  k_count<<<dim3(g.n_chunks, b.T), kAsmThreads, 0, st>>>(g, tb, s, state);
}

void launch_emit(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                 const State& state, const Output& out, cudaStream_t st) {
  k_emit<<<dim3(g.n_chunks, b.T), kAsmThreads, 0, st>>>(g, tb, b, s, state, out);
}

}  // namespace fkd
