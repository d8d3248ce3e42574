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
//   k_emit:  sum the totals of the frames before and the counts of the
//            chunks before into the chunk's output offset, scan the chunk's
//            stored words, and write one record per set bit, in order.
// The last frame of the batch also becomes the new kept set (bitmap, scores,
// keypoints per bin).
#include "fkd_internal.cuh"

namespace fkd {
namespace {

constexpr int kEmitList = 4096;
constexpr int kSrcCache = 512;  // source frames of a chunk's bins kept in shared memory  // set bits of a chunk emitted from a shared list (denser chunks: per thread)
static_assert(kAsmChunkWords * 32 <= 65536, "word * 32 + bit fits 16 bits");


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

// Bits of word j of the chunk (bin row r's sources in srcrow) taken from the
// frames the bins point to: words of one or two bins take a precomputed split
// mask, wider words (coarse layers, narrow bins) walk their bins.
__device__ __forceinline__ uint32_t merge_word(const Geometry& g, const Tables& tb, const Scratch& s,
                                               const State& st, const LayerGeom& lg, const int* xst,
                                               const int* srcrow, long long word0, int j, int wx) {
  const uint32_t wb = tb.wbins[lg.wb_off + wx];
  const int c_lo = wb & 0xffffu, c_hi = wb >> 16;
  const uint32_t* det0 = s.det_bits + word0;
  if (c_hi - c_lo <= 1) {
    const uint32_t m = tb.wmask[lg.wb_off + wx];
    const int sf0 = srcrow[c_lo], sf1 = srcrow[c_hi];
    const uint32_t b0 = sf0 < 0 ? st.bits_in[word0 + j] : det0[(long long)sf0 * g.bit_words + j];
    const uint32_t b1 = sf1 == sf0 ? b0 : (sf1 < 0 ? st.bits_in[word0 + j] : det0[(long long)sf1 * g.bit_words + j]);
    return (b0 & m) | (b1 & ~m);
  }
  const int xlo = wx * 32, xhi = min(xlo + 32, lg.w);
  uint32_t word = 0;
  for (int c = c_lo; c <= c_hi; ++c) {
    const int a = max(xst[c], xlo) - xlo, e = min(xst[c + 1], xhi) - xlo;
    if (e <= a) continue;
    const uint32_t m = (e - a == 32) ? 0xffffffffu : (((1u << (e - a)) - 1u) << a);
    const int sf = srcrow[c];
    word |= (sf < 0 ? st.bits_in[word0 + j] : det0[(long long)sf * g.bit_words + j]) & m;
  }
  return word;
}

// Merge and count one chunk of frame k: the CTA adds its popcount to the
// chunk's and the frame's counters (zeroed by the active-tile kernel). Ends
// with a barrier.
__device__ __forceinline__ void count_chunk(const Geometry& g, const Tables& tb, const Scratch& s,
                                            const State& st, int k, int chunk) {
  __shared__ uint32_t red[kAsmThreads / 32];
  const AsmChunk ch = tb.chunks[chunk];
  const LayerGeom& lg = g.layer[ch.layer];
  const int wpr = lg.wpr;
  const int nwords = (ch.y1 - ch.y0) * wpr;
  const long long word0 = lg.bit_off + (long long)ch.y0 * wpr;
  const int* xst = tb.xstart + lg.xs_off;
  const int* src_k = s.src + (long long)k * g.NB;
  // the source frames of the chunk's bin rows, in shared memory when they fit
  __shared__ int srcs[kSrcCache];
  const int nsrc = (ch.rb1 - ch.rb0 + 1) * g.N_c;
  const bool src_local = !s.pmask && nsrc <= kSrcCache;
  if (src_local)
    for (int i = threadIdx.x; i < nsrc; i += kAsmThreads) srcs[i] = src_k[ch.rb0 * g.N_c + i];
  __syncthreads();
  uint32_t* out = s.merged + (long long)k * g.bit_words + word0;
  // words tid, tid + 256, ...: coalesced; the count does not care about order
  const float inv_wpr = 1.0f / (float)wpr;
  uint32_t cnt = 0;
#pragma unroll
  for (int jj = 0; jj < kAsmWordsPerThread; ++jj) {
    const int j = threadIdx.x + jj * kAsmThreads;
    if (j < nwords) {
      int yy = __float2int_rz((float)j * inv_wpr);  // j / wpr, fixed up below
      if (yy * wpr > j) --yy;
      if ((yy + 1) * wpr <= j) ++yy;
      const int wx = j - yy * wpr;
      const int r = tb.rowblk[lg.row_off + ch.y0 + yy];
      const int* srcrow = src_local ? srcs + (r - ch.rb0) * g.N_c : src_k + r * g.N_c;
      uint32_t word;
      if (s.pmask) {
        word = out[j];  // per-pixel masks: merged by the per-pixel recurrence
      } else {
        word = merge_word(g, tb, s, st, lg, xst, srcrow, word0, j, wx);
        out[j] = word;
      }
      cnt += __popc(word);
    }
  }
  cnt = block_sum(cnt, red);
  if (threadIdx.x == 0 && cnt) {
    atomicAdd(&s.chunk_counts[(long long)k * g.n_chunks + chunk], cnt);
    atomicAdd(&s.frame_totals[k], cnt);
  }
  __syncthreads();  // red is reused by the next chunk of this CTA
}

__device__ __forceinline__ void emit_records(const Geometry& g, const Tables& tb, const Scratch& s,
                                             const State& st, const Output& out, int k, bool last,
                                             const AsmChunk& ch, const LayerGeom& lg, int j0,
                                             const uint32_t* words, unsigned long long idx, const int* srcs,
                                             bool src_local);

// Emit the records of one chunk of frame k of a batch of T frames; the last
// frame also writes the new kept set. Ends with a barrier.
__device__ __forceinline__ void emit_chunk(const Geometry& g, const Tables& tb, const Scratch& s,
                                           const State& st, const Output& out, int k, int T,
                                           int chunk) {
  __shared__ uint32_t red[kAsmThreads / 32];
  __shared__ uint32_t wsum[kAsmThreads / 32];
  __shared__ __align__(16) uint32_t stage_words[kAsmChunkWords];
  __shared__ uint16_t pos[kEmitList];  // set bits of the chunk in order: word * 32 + bit
  const bool last = k == T - 1;
  const AsmChunk ch = tb.chunks[chunk];
  const LayerGeom& lg = g.layer[ch.layer];
  const int wpr = lg.wpr;
  const int nwords = (ch.y1 - ch.y0) * wpr;
  const long long word0 = lg.bit_off + (long long)ch.y0 * wpr;
  // the chunk's merged words, loaded first so that the loads overlap the
  // offset sums below
  const uint32_t* merged = s.merged + (long long)k * g.bit_words + word0;
  uint32_t v[kAsmWordsPerThread];
#pragma unroll
  for (int jj = 0; jj < kAsmWordsPerThread; ++jj) {
    const int j = threadIdx.x + jj * kAsmThreads;
    v[jj] = j < nwords ? merged[j] : 0u;
  }
  // offsets: base of this call + earlier frames + earlier chunks of this
  // frame (partial sums per warp here, summed after the barrier below)
  {
    uint32_t pf = 0, pc = 0;
    for (int q = threadIdx.x; q < k; q += kAsmThreads) pf += s.frame_totals[q];
    for (int q = threadIdx.x; q < chunk; q += kAsmThreads) pc += s.chunk_counts[(long long)k * g.n_chunks + q];
    pf = __reduce_add_sync(0xffffffffu, pf);
    pc = __reduce_add_sync(0xffffffffu, pc);
    if ((threadIdx.x & 31) == 0) {
      red[threadIdx.x >> 5] = pf;
      wsum[threadIdx.x >> 5] = pc;
    }
  }
  // the source frames of the chunk's bin rows, in shared memory when they fit
  __shared__ int srcs[kSrcCache];
  const int* src_k = s.src + (long long)k * g.NB;
  const int nsrc = (ch.rb1 - ch.rb0 + 1) * g.N_c;
  const bool src_local = !s.pmask && nsrc <= kSrcCache;
  if (src_local)
    for (int i = threadIdx.x; i < nsrc; i += kAsmThreads) srcs[i] = src_k[ch.rb0 * g.N_c + i];
  __syncthreads();
  uint32_t frame_base = 0, chunk_base = 0;
#pragma unroll
  for (int q = 0; q < kAsmThreads / 32; ++q) {
    frame_base += red[q];
    chunk_base += wsum[q];  // (wsum is next written after the barrier below)
  }
  const unsigned long long call_base = s.out_base[out.base_slot];
  if (chunk == 0 && threadIdx.x == 0) {
    out.offsets[k] = (uint32_t)(call_base + frame_base);
    if (last) {
      const unsigned long long end = call_base + frame_base + s.frame_totals[k];
      out.offsets[k + 1] = (uint32_t)end;
      s.out_base[out.base_slot ^ 1] = end;
    }
  }

  // the chunk's words, coalesced, into shared memory; each thread then takes
  // 8 contiguous ones, so the scan order is the canonical order
#pragma unroll
  for (int jj = 0; jj < kAsmWordsPerThread; ++jj) {
    const int j = threadIdx.x + jj * kAsmThreads;
    if (FKD_IDX(kChkAsmWords, j, kAsmChunkWords)) stage_words[j] = v[jj];
    if (last && j < nwords) st.bits_out[word0 + j] = v[jj];
  }
  __syncthreads();
  const int j0 = threadIdx.x * kAsmWordsPerThread;
  uint32_t words[kAsmWordsPerThread];
  uint32_t cnt = 0;
#pragma unroll
  for (int jj = 0; jj < kAsmWordsPerThread; jj += 4) {
    const uint4 v = *reinterpret_cast<const uint4*>(&stage_words[j0 + jj]);
    words[jj] = v.x;
    words[jj + 1] = v.y;
    words[jj + 2] = v.z;
    words[jj + 3] = v.w;
  }
#pragma unroll
  for (int jj = 0; jj < kAsmWordsPerThread; ++jj) cnt += __popc(words[jj]);
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
  uint32_t before = 0, total = 0;
#pragma unroll
  for (int q = 0; q < kAsmThreads / 32; ++q) {
    before += q < wid ? wsum[q] : 0u;
    total += wsum[q];
  }
  const unsigned long long base = call_base + frame_base + chunk_base;
  if (out.row_base) {
    // index of the first record of every row starting in this thread's words
    // (the descriptor pass looks keypoints up by row)
    uint32_t* rb = out.row_base + (long long)k * out.rows + lg.row_off + ch.y0;
    const int nrows = ch.y1 - ch.y0;
    int row = (j0 + wpr - 1) / wpr;
    int next = row * wpr;
    unsigned long long at = base + before + incl - cnt;
#pragma unroll
    for (int jj = 0; jj < kAsmWordsPerThread; ++jj) {
      if (j0 + jj == next && row < nrows) {
        rb[row] = (uint32_t)at;
        ++row;
        next += wpr;
      }
      at += __popc(words[jj]);
    }
  }
  if (total > (uint32_t)kEmitList) {
    // a dense chunk: every thread emits its own words' records
    if (cnt) emit_records(g, tb, s, st, out, k, last, ch, lg, j0, words, base + before + incl - cnt, srcs, src_local);
    __syncthreads();  // red and wsum are reused by the next chunk of this CTA
    return;
  }
  // list the set bits in order, then emit one record per thread (balanced,
  // and consecutive threads write consecutive records)
  uint32_t at = before + incl - cnt;
#pragma unroll
  for (int jj = 0; jj < kAsmWordsPerThread; ++jj) {
    uint32_t wv = words[jj];
    while (wv) {
      const int bit = __ffs(wv) - 1;
      wv &= wv - 1;
      if (FKD_IDX(kChkAsmPos, at, kEmitList)) pos[at] = (uint16_t)((j0 + jj) * 32 + bit);
      ++at;
    }
  }
  __syncthreads();
  const int wpr_ = wpr;
  const float inv_wpr = 1.0f / (float)wpr_;
  const uint16_t* colblk = tb.colblk + lg.col_off;
  // (the loop runs whole warps, so that the kept set's per-bin counts can be
  // added once per bin and warp)
  for (uint32_t i0 = 0; i0 < total; i0 += kAsmThreads) {
    const uint32_t i = i0 + threadIdx.x;
    int bin = -1;
    if (i < total) {
      const int p = pos[i];
      const int j = p >> 5;
      int yy = __float2int_rz((float)j * inv_wpr);  // j / wpr, fixed up below
      if (yy * wpr_ > j) --yy;
      if ((yy + 1) * wpr_ <= j) ++yy;
      const int y = ch.y0 + yy;
      const int x = (j - yy * wpr_) * 32 + (p & 31);
      const int r = tb.rowblk[lg.row_off + y];
      const int c = colblk[x];
      const long long so = lg.score_off + (long long)y * lg.pitch + x;
      uint8_t score;
      uint32_t flags;
      if (s.pmask) {
        // per-pixel masks: every frame's map holds its keypoints' scores; a
        // keypoint is carried where its pixel was inactive
        score = s.det_score[(long long)k * g.score_bytes + so];
        const uint32_t mw = s.pmask[(long long)k * g.bit_words + word0 + j];
        flags = ((mw >> (p & 31)) & 1u) ? 0u : FKD_KP_PROPAGATED;
      } else {
        const int sf = src_local && FKD_IDX(kChkAsmSrc, (r - ch.rb0) * g.N_c + c, kSrcCache)
                           ? srcs[(r - ch.rb0) * g.N_c + c] : src_k[r * g.N_c + c];
        score = sf < 0 ? st.score_in[so] : s.det_score[(long long)sf * g.score_bytes + so];
        flags = sf != k ? FKD_KP_PROPAGATED : 0u;
      }
      const unsigned long long idx = base + i;
      if (idx < (unsigned long long)out.cap) {
        uint2 rec;
        rec.x = (uint32_t)x | ((uint32_t)y << 16);
        rec.y = (uint32_t)ch.layer | ((uint32_t)score << 8) | (flags << 16);
        reinterpret_cast<uint2*>(out.rec)[idx] = rec;
      } else {
        atomicOr(s.overflow, 1);
      }
      if (last) st.score_out[so] = score;
      bin = r * g.N_c + c;
    }
    if (last) {
      // consecutive records mostly share a bin: one atomic per bin and warp
      const unsigned peers = __match_any_sync(0xffffffffu, bin);
      if (bin >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1 && FKD_IDX(kChkAsmBins, bin, g.NB))
        atomicAdd(&st.cnt_out[bin], (uint32_t)__popc(peers));
    }
  }
  __syncthreads();  // red, wsum and pos are reused by the next chunk of this CTA
}

__device__ __forceinline__ void emit_records(const Geometry& g, const Tables& tb, const Scratch& s,
                                             const State& st, const Output& out, int k, bool last,
                                             const AsmChunk& ch, const LayerGeom& lg, int j0,
                                             const uint32_t* words, unsigned long long idx, const int* srcs,
                                             bool src_local) {
  const int wpr = lg.wpr;
  const int* src_k = s.src + (long long)k * g.NB;
  const uint16_t* colblk = tb.colblk + lg.col_off;
  int y = ch.y0 + j0 / wpr, wx = j0 % wpr;
  int run_bin = -1;
  uint32_t run_n = 0;
#pragma unroll
  for (int jj = 0; jj < kAsmWordsPerThread; ++jj) {
    uint32_t wv = words[jj];
    if (wv) {
      const int r = tb.rowblk[lg.row_off + y];
      const int* srcrow = src_local ? srcs + (r - ch.rb0) * g.N_c : src_k + r * g.N_c;
      const long long row_off = lg.score_off + (long long)y * lg.pitch;
      while (wv) {
        const int bit = __ffs(wv) - 1;
        wv &= wv - 1;
        const int x = wx * 32 + bit;
        const int c = colblk[x];
        uint8_t score;
        uint32_t flags;
        if (s.pmask) {  // per-pixel masks: as in the list path of emit_chunk
          score = s.det_score[(long long)k * g.score_bytes + row_off + x];
          const uint32_t mw = s.pmask[(long long)k * g.bit_words + lg.bit_off + (long long)y * wpr + wx];
          flags = ((mw >> bit) & 1u) ? 0u : FKD_KP_PROPAGATED;
        } else {
          const int sf = srcrow[c];
          score = sf < 0 ? st.score_in[row_off + x] : s.det_score[(long long)sf * g.score_bytes + row_off + x];
          flags = sf != k ? FKD_KP_PROPAGATED : 0u;
        }
        if (idx < (unsigned long long)out.cap) {
          uint2 rec;
          rec.x = (uint32_t)x | ((uint32_t)y << 16);
          rec.y = (uint32_t)ch.layer | ((uint32_t)score << 8) | (flags << 16);
          reinterpret_cast<uint2*>(out.rec)[idx] = rec;
        } else {
          atomicOr(s.overflow, 1);
        }
        ++idx;
        if (last) {
          st.score_out[row_off + x] = score;
          // a thread's records run along its words: one atomic per run of a bin
          const int bin = r * g.N_c + c;
          if (bin != run_bin) {
            if (run_n && FKD_IDX(kChkAsmBins, run_bin, g.NB)) atomicAdd(&st.cnt_out[run_bin], run_n);
            run_bin = bin;
            run_n = 0;
          }
          ++run_n;
        }
      }
    }
    if (++wx == wpr) {
      wx = 0;
      ++y;
    }
  }
  if (run_n && FKD_IDX(kChkAsmBins, run_bin, g.NB)) atomicAdd(&st.cnt_out[run_bin], run_n);
}

__global__ void __launch_bounds__(kAsmThreads) k_count(Geometry g, Tables tb, Scratch s, State st) {
  pdl_wait();
  pdl_trigger();
  count_chunk(g, tb, s, st, blockIdx.y, blockIdx.x);
}

__global__ void __launch_bounds__(kAsmThreads) k_emit(Geometry g, Tables tb, Batch b, Scratch s,
                                                      State st, Output out) {
  pdl_wait();
  pdl_trigger();
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
// (6 and 5 resident CTAs per SM, on a grid of 8 CTAs per SM: the CTAs beyond
// the resident ones start as others finish, which evens out the unequal
// chunks better than a grid of exactly the resident CTAs)
__global__ void __launch_bounds__(kAsmThreads, 6) k_group_count(const StreamDev* devs, const TickHeader* hdr,
                                                                const TickItem* items) {
  const int n = hdr->n_items, total = hdr->total_chunks;
  for (int j = blockIdx.x; j < total; j += gridDim.x) {
    const int i = find_item(n, j, [&](int q) { return items[q].chunk_base; });
    const TickItem it = items[i];
    const StreamDev& d = devs[it.sid];
    count_chunk(d.g, d.tb, d.s, state_of(d, it.state_cur), 0, j - it.chunk_base);
  }
}

__global__ void __launch_bounds__(kAsmThreads, 5) k_group_emit(const StreamDev* devs, const TickHeader* hdr,
                                                               const TickItem* items) {
  const int n = hdr->n_items, total = hdr->total_chunks;
  for (int j = blockIdx.x; j < total; j += gridDim.x) {
    const int i = find_item(n, j, [&](int q) { return items[q].chunk_base; });
    const TickItem it = items[i];
    const StreamDev& d = devs[it.sid];
    const int par = (int)(it.frame_index & 1);
    Output o{d.rec[par], d.K_max, d.rec_offsets[par], 0};
    if (d.D) {  // row starts for the descriptor pass
      o.row_base = d.row_base[par];
      o.rows = d.rows;
    }
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
  pdl_launch(k_count, dim3(g.n_chunks, b.T), dim3(kAsmThreads), 0, st, g, tb, s, state);
}

void launch_emit(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                 const State& state, const Output& out, cudaStream_t st) {
  pdl_launch(k_emit, dim3(g.n_chunks, b.T), dim3(kAsmThreads), 0, st, g, tb, b, s, state, out);
}

}  // namespace fkd
