// k_pyramid.cu -- pyramid of octaves / intra-octaves and per-bin change sums.
//
// One CTA owns a 96 x 96 tile of c_0 of one frame. It copies the tile into
// shared memory with cp.async, builds every layer of the tile there (Sec. 2:
// octaves c_i by 2x2 half-sampling, intra-octaves d_i by 2/3 resampling of
// c_0 then half-sampling), storing each output word both to shared memory
// (input of the next layer) and straight to the frame's pyramid buffer, and
// -- for the intensity difference mask (Eq. 2, Sec. 3.1, which reuses the
// pyramid) -- adds |L_n - L_{n-1}| of the mask layer into the per-bin sums.
// The previous frame's mask layer is rebuilt from its c_0 tile in shared
// memory rather than read back, so the frames of a batch do not depend on
// one another here. The kernel is instantiated per (octaves, intra-octaves)
// so that every level's size is a compile-time constant.
//
// 96 is a multiple of 3 * 2^5: for O <= 6 every layer's tile is whole, so the
// 2x2 box and the 3x3 -> 2x2 resampling never cross a tile edge.
//
// In a batch whose frames allow it (16-byte aligned base, pitch and frame
// stride) the c_0 tile -- and, for change sums on c_0, the previous frame's
// tile -- arrives by one tensor-memory-access copy each (a 96 x 96 box of a
// 3-D tensor map over the batch's frames, zero-filled outside the frame),
// completed on an mbarrier; otherwise, and in group ticks, by cp.async.
#include <mutex>

#include <cuda.h>

#include "fkd_internal.cuh"

namespace fkd {
namespace {

constexpr int P = kPyrTile;  // 96
constexpr int NT = kPyrThreads;
__host__ __device__ constexpr int c_side(int i) { return P >> i; }
__host__ __device__ constexpr int d_side(int i) { return (2 * P / 3) >> i; }
__host__ __device__ constexpr int r16(int v) { return (v + 15) / 16 * 16; }
__host__ __device__ constexpr int c_off(int i) { return i == 0 ? 0 : r16(c_off(i - 1) + c_side(i - 1) * c_side(i - 1)); }
__host__ __device__ constexpr int d_off(int i) { return i == 0 ? r16(c_off(6)) : r16(d_off(i - 1) + d_side(i - 1) * d_side(i - 1)); }
constexpr int kPyrSmem = d_off(6);

constexpr int kLocalBins = 256;  // bins a tile may span and still sum in shared memory
constexpr int kPrvOff = (kPyrSmem + 127) / 128 * 128;  // the previous frame's c_0 tile

// Dynamic shared memory of a CTA: the tile's levels (c_0 first), then -- when
// the change sums of c_0 may be needed -- the previous frame's c_0 tile and
// the tile's bin sums. Both c_0 tiles start on 128-byte boundaries (tensor
// copies land there).
__host__ __device__ constexpr int pyr_smem(bool diff) { return diff ? kPrvOff + P * P + kLocalBins * 4 : kPyrSmem; }
static_assert(kPyrSmem % 16 == 0 && (P * P) % 128 == 0, "aligned regions");

// ---- tensor-memory-access copy of a c_0 tile, completed on an mbarrier
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
  // make the initialised barrier visible to the copy engine
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// Box (x, y) .. (x + 95, y + 95) of frame z into `dst` (128-byte aligned).
// x is a multiple of 96, hence of 16 bytes.
__device__ __forceinline__ void tma_tile(uint8_t* dst, const CUtensorMap* map, int x, int y, int z,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// Wait for phase 0 of the barrier, for at most ~2^30 SM cycles (about half a
// second): false when the copies have not landed by then.
__device__ __forceinline__ bool mbar_wait0(uint64_t* bar) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(smem_addr(bar))
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1LL << 30)) return false;
  }
}

__device__ __forceinline__ uint32_t ld32(const uint8_t* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

// Where a level's outputs go in global memory: the tile's first pixel of the
// layer, the layer pitch, and how much of the tile lies inside the layer.
struct Out {
  uint8_t* p;
  int pitch, nx, ny;
};

// Start copying the 96 x 96 tile at (gx0, gy0) of a frame (zeros outside the
// frame): cp.async with zero fill when the frame allows 16-byte copies, plain
// byte loads otherwise. The caller commits, waits and syncs.
__device__ __forceinline__ void load_c0(uint8_t* dst, const uint8_t* frame, int pitch, int gx0,
                                        int gy0, int W, int H) {
  const bool vec = ((reinterpret_cast<uintptr_t>(frame) | (uintptr_t)pitch) & 15) == 0;
  constexpr int kChunks = P / 16;
#pragma unroll
  for (int q0 = 0; q0 < P * kChunks; q0 += NT) {
    const int q = q0 + threadIdx.x;
    if (q < P * kChunks) {
      const int r = q / kChunks, c = (q % kChunks) * 16;
      const int gy = gy0 + r, gx = gx0 + c;
      uint8_t* d = dst + r * P + c;
      if (vec) {
        const int bytes = gy < H ? max(0, min(16, W - gx)) : 0;
        cp_async16(d, bytes ? frame + (size_t)gy * pitch + gx : frame, bytes);
      } else {
        uint32_t wd[4] = {0u, 0u, 0u, 0u};
        if (gy < H) {
#pragma unroll
          for (int j = 0; j < 16; ++j)
            if (gx + j < W) wd[j >> 2] |= (uint32_t)frame[(size_t)gy * pitch + gx + j] << (8 * (j & 3));
        }
        *reinterpret_cast<uint4*>(d) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
      }
    }
  }
}

// 2x2 box mean with round-half-up of an N x N level into (N/2) x (N/2).
// Four outputs per step when N/2 is a multiple of 4: the even and odd bytes
// of two input rows are spread into 16-bit lanes, summed with +2, shifted by
// 2 and repacked. WRITE: also store the outputs inside the layer to `o`.
template <int N, bool WRITE>
__device__ __forceinline__ void half_level(const uint8_t* src, uint8_t* dst, const Out& o) {
  constexpr int M = N / 2;
  if constexpr (M % 4 == 0) {
    constexpr int WPR = M / 4, TOTAL = M * WPR;
#pragma unroll
    for (int q0 = 0; q0 < TOTAL; q0 += NT) {
      const int q = q0 + threadIdx.x;
      if (TOTAL % NT == 0 || q < TOTAL) {
        const int y = q / WPR, xw = q % WPR;
        const uint8_t* a = src + (2 * y) * N + 8 * xw;
        const uint32_t a0 = ld32(a), a1 = ld32(a + 4), b0 = ld32(a + N), b1 = ld32(a + N + 4);
        const uint32_t lo = __byte_perm(a0, 0, 0x4240) + __byte_perm(a0, 0, 0x4341) +
                            __byte_perm(b0, 0, 0x4240) + __byte_perm(b0, 0, 0x4341) + 0x00020002u;
        const uint32_t hi = __byte_perm(a1, 0, 0x4240) + __byte_perm(a1, 0, 0x4341) +
                            __byte_perm(b1, 0, 0x4240) + __byte_perm(b1, 0, 0x4341) + 0x00020002u;
        // lanes hold sums <= 1022; >> 2 leaves each result in its lane's low byte
        const uint32_t v = __byte_perm((lo >> 2) & 0x00ff00ffu, (hi >> 2) & 0x00ff00ffu, 0x6420);
        if (FKD_IDX(kChkPyrSmem, y * M + 4 * xw, M * M - 3)) *reinterpret_cast<uint32_t*>(dst + y * M + 4 * xw) = v;
        if (WRITE && y < o.ny) {
          const int x = 4 * xw;
          uint8_t* gp = o.p + (long long)y * o.pitch + x;
          if (x + 4 <= o.nx) {
            *reinterpret_cast<uint32_t*>(gp) = v;
          } else {
#pragma unroll
            for (int j = 0; j < 3; ++j)
              if (x + j < o.nx) gp[j] = (uint8_t)(v >> (8 * j));
          }
        }
      }
    }
  } else {
#pragma unroll
    for (int q0 = 0; q0 < M * M; q0 += NT) {
      const int q = q0 + threadIdx.x;
      if (q < M * M) {
        const int y = q / M, x = q % M;
        const uint8_t* sp = src + (2 * y) * N + 2 * x;
        const uint8_t v = (uint8_t)((sp[0] + sp[1] + sp[N] + sp[N + 1] + 2u) >> 2);
        if (FKD_IDX(kChkPyrSmem, q, M * M)) dst[q] = v;
        if (WRITE && y < o.ny && x < o.nx) o.p[(long long)y * o.pitch + x] = v;
      }
    }
  }
}

// 2/3 resampling of the 96 x 96 c_0 tile into the 64 x 64 d_0 tile: each 3x3
// block gives a 2x2 block; an output is the mean of its 1.5 x 1.5 footprint
// (weights 4 for the corner it sits on, 2 and 2 for the half-covered edge
// pixels, 1 for the quarter-covered centre, over 9), rounded to nearest.
//
// A thread takes four neighbouring blocks of one block row (a 3 x 12 input
// patch: nine aligned words), blocks 0 and 1 in the two 16-bit lanes of one
// set of registers and blocks 2 and 3 in another, so that every weighted sum
// (at most 9 * 255 + 4) is one lane-wise add for two outputs; the divisions
// by 9 run per lane, and each output row of the four blocks is 8 bytes.
template <bool WRITE>
__device__ __forceinline__ void two_thirds(const uint8_t* src, uint8_t* dst, const Out& o) {
  constexpr int NB = P / 3, N = P, M = 2 * P / 3;
  static_assert(NB * (NB / 4) == NT, "one thread per four blocks of a block row");
  const int by = threadIdx.x / (NB / 4), bq = threadIdx.x % (NB / 4);
  const uint8_t* sp = src + (3 * by) * N + 12 * bq;
  // lanes: L = left, C = middle, R = right column of each block; A = blocks
  // (0, 1) of the four, B = blocks (2, 3); index = row of the block
  uint32_t LA[3], CA[3], RA[3], LB[3], CB[3], RB[3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const uint32_t w0 = ld32(sp + r * N), w1 = ld32(sp + r * N + 4), w2 = ld32(sp + r * N + 8);
    LA[r] = __byte_perm(w0, 0u, 0x4340);                // bytes 0, 3
    CA[r] = __byte_perm(w0, w1, 0x0401) & 0x00ff00ffu;  // bytes 1, 4
    RA[r] = __byte_perm(w0, w1, 0x0502) & 0x00ff00ffu;  // bytes 2, 5
    LB[r] = __byte_perm(w1, w2, 0x0502) & 0x00ff00ffu;  // bytes 6, 9
    CB[r] = __byte_perm(w1, w2, 0x0603) & 0x00ff00ffu;  // bytes 7, 10
    RB[r] = __byte_perm(w2, 0u, 0x4340);                // bytes 8, 11
  }
  // per lane: top-left 4 p00 + 2 p01 + 2 p10 + p11 (+ 4 to round), etc.
  auto sums = [](const uint32_t* L, const uint32_t* C, const uint32_t* R, uint32_t* q) {
    const uint32_t e01 = 2u * C[0] + C[1] + 0x00040004u, e21 = 2u * C[2] + C[1] + 0x00040004u;
    q[0] = 4u * L[0] + 2u * L[1] + e01;  // top-left
    q[1] = 4u * R[0] + 2u * R[1] + e01;  // top-right
    q[2] = 4u * L[2] + 2u * L[1] + e21;  // bottom-left
    q[3] = 4u * R[2] + 2u * R[1] + e21;  // bottom-right
  };
  auto div9 = [](uint32_t v) { return ((v & 0xffffu) / 9u) | (((v >> 16) / 9u) << 16); };
  uint32_t qa[4], qb[4];
  sums(LA, CA, RA, qa);
  sums(LB, CB, RB, qb);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    qa[i] = div9(qa[i]);
    qb[i] = div9(qb[i]);
  }
  // output rows 2by (top) and 2by+1 (bottom), columns 8bq .. 8bq+7:
  // left, right of block 0, of block 1, ... -> bytes of (left | right << 8)
  const uint2 top = make_uint2(qa[0] | (qa[1] << 8), qb[0] | (qb[1] << 8));
  const uint2 bot = make_uint2(qa[2] | (qa[3] << 8), qb[2] | (qb[3] << 8));
  const int y = 2 * by, x = 8 * bq;
  if (FKD_IDX(kChkPyrSmem, (y + 1) * M + x, M * M - 7)) {
    *reinterpret_cast<uint2*>(dst + y * M + x) = top;
    *reinterpret_cast<uint2*>(dst + (y + 1) * M + x) = bot;
  }
  if (WRITE) {
    uint8_t* gp = o.p + (long long)y * o.pitch + x;
    if (x + 8 <= o.nx) {
      if (y < o.ny) *reinterpret_cast<uint2*>(gp) = top;
      if (y + 1 < o.ny) *reinterpret_cast<uint2*>(gp + o.pitch) = bot;
    } else if (x < o.nx) {
      for (int j = 0; j < o.nx - x; ++j) {
        const uint32_t tw = j < 4 ? top.x : top.y, bw = j < 4 ? bot.x : bot.y;
        if (y < o.ny) gp[j] = (uint8_t)(tw >> (8 * (j & 3)));
        if (y + 1 < o.ny) gp[o.pitch + j] = (uint8_t)(bw >> (8 * (j & 3)));
      }
    }
  }
}

__device__ __forceinline__ Out out_of(const Geometry& g, uint8_t* pyr, int l, int side, int tx,
                                      int ty) {
  const LayerGeom& lg = g.layer[l];
  const int gx0 = tx * side, gy0 = ty * side;
  Out o;
  o.p = pyr + lg.pyr_off + (long long)gy0 * lg.pitch + gx0;
  o.pitch = lg.pitch;
  o.nx = min(side, lg.w - gx0);
  o.ny = min(side, lg.h - gy0);
  return o;
}

// Octave chain c_I .. c_{O-1}, one level per step, up to layer `up_to`.
template <int O, int INTRA, int I, bool WRITE>
__device__ __forceinline__ void octaves(const Geometry& g, uint8_t* pyr, uint8_t* t, int tx, int ty,
                                        int up_to) {
  if constexpr (I < O) {
    constexpr int l = INTRA ? 2 * I : I;
    if (l > up_to) return;
    half_level<c_side(I - 1), WRITE>(t + c_off(I - 1), t + c_off(I),
                                     WRITE ? out_of(g, pyr, l, c_side(I), tx, ty) : Out{});
    __syncthreads();
    octaves<O, INTRA, I + 1, WRITE>(g, pyr, t, tx, ty, up_to);
  }
}

// Intra-octave chain d_I .. d_{O-1}.
template <int O, int I, bool WRITE>
__device__ __forceinline__ void intra_octaves(const Geometry& g, uint8_t* pyr, uint8_t* t, int tx,
                                              int ty, int up_to) {
  if constexpr (I < O) {
    constexpr int l = 2 * I + 1;
    if (l > up_to) return;
    half_level<d_side(I - 1), WRITE>(t + d_off(I - 1), t + d_off(I),
                                     WRITE ? out_of(g, pyr, l, d_side(I), tx, ty) : Out{});
    __syncthreads();
    intra_octaves<O, I + 1, WRITE>(g, pyr, t, tx, ty, up_to);
  }
}

template <int O, int INTRA, bool WRITE>
__device__ __forceinline__ void build(const Geometry& g, uint8_t* pyr, uint8_t* t, int tx, int ty,
                                      int up_to) {
  octaves<O, INTRA, 1, WRITE>(g, pyr, t, tx, ty, up_to);
  if constexpr (INTRA == 1) {
    if (up_to >= 1) {
      two_thirds<WRITE>(t, t + d_off(0), WRITE ? out_of(g, pyr, 1, d_side(0), tx, ty) : Out{});
      __syncthreads();
      intra_octaves<O, 1, WRITE>(g, pyr, t, tx, ty, up_to);
    }
  }
}

// One 96 x 96 tile of c_0 of one frame: pyramid, layer writes, per-bin sums
// of |I_n - I_{n-1}| on c_0 (if `diff`; the mask layer is c_0), and a copy of
// the c_0 tile to `keep` (if not null, pitch `keep_pitch`). Ends with a
// barrier, so a CTA can run it again at once.
//
// c0map (nullptr: cp.async): the batch's tensor map, this frame at z, the
// previous one (when prev_in_map) at z - 1. A copy that has not landed after
// the wait limit sets bit 1 of *err and the CTA leaves the tile.
template <int O, int INTRA>
__device__ __forceinline__ void pyramid_tile(uint8_t* smem, const Geometry& g, const Tables& tb,
                                             const uint8_t* frame, int pitch, const uint8_t* prevf,
                                             int prev_pitch, bool diff, uint8_t* pyr,
                                             unsigned long long* gsum, int gstride, uint8_t* keep,
                                             int keep_pitch, int tx, int ty,
                                             const CUtensorMap* c0map = nullptr, int z = 0,
                                             bool prev_in_map = false, int* err = nullptr) {
  __shared__ uint16_t tcol[P], trow[P], trun[P];
  __shared__ __align__(8) uint64_t tma_bar;
  uint8_t* cur = smem;
  uint8_t* prv = smem + kPrvOff;
  uint32_t* bins = reinterpret_cast<uint32_t*>(prv + P * P);

  const bool via_tma = c0map && (smem_addr(smem) & 127u) == 0;
  const bool prev_tma = via_tma && diff && prev_in_map;
  if (via_tma) {
    if (threadIdx.x == 0) mbar_init(&tma_bar);
    __syncthreads();
    if (threadIdx.x == 0) {
      mbar_expect_tx(&tma_bar, (prev_tma ? 2u : 1u) * P * P);
      tma_tile(cur, c0map, tx * P, ty * P, z, &tma_bar);
      if (prev_tma) tma_tile(prv, c0map, tx * P, ty * P, z - 1, &tma_bar);
    }
  } else {
    load_c0(cur, frame, pitch, tx * P, ty * P, g.W, g.H);
  }
  const LayerGeom& mlg = g.layer[0];
  constexpr int mn = P;
  const int mgx0 = tx * mn, mgy0 = ty * mn;
  const int mnx = min(mn, mlg.w - mgx0), mny = min(mn, mlg.h - mgy0);
  if (diff) {
    if (!prev_tma) load_c0(prv, prevf, prev_pitch, tx * P, ty * P, g.W, g.H);
    for (int q = threadIdx.x; q < kLocalBins; q += NT) bins[q] = 0;
    for (int q = threadIdx.x; q < mn; q += NT) {
      tcol[q] = q < mnx ? tb.colblk[mlg.col_off + mgx0 + q] : 0;
      const unsigned r = q < mny ? tb.rowblk[mlg.row_off + mgy0 + q] : 0u;
      trow[q] = (uint16_t)r;
      // end of the tile's run of rows in bin row r: layer row y is in bin
      // row floor(floor(y*S/2) * N_r / H) (Eq. 3), so bin row r + 1 starts
      // at row ceil(2 * ceil((r+1)*H/N_r) / S)
      const unsigned qh = ((r + 1u) * (unsigned)g.H + (unsigned)g.N_r - 1u) / (unsigned)g.N_r;
      const int next = (int)((2u * qh + (unsigned)mlg.S - 1u) / (unsigned)mlg.S) - mgy0;
      trun[q] = (uint16_t)min(next, mny);
    }
  }
  cp_async_commit();
  cp_async_wait<0>();
  if (via_tma) {
    const bool landed = mbar_wait0(&tma_bar);
    if (__syncthreads_or(!landed)) {
      // not landed: flag it, wait once more for the copies still in flight
      // (again bounded), and leave the tile
      if (threadIdx.x == 0) {
        if (err) atomicOr(err, 2);
        mbar_wait0(&tma_bar);
      }
      __syncthreads();
      return;
    }
  }
  __syncthreads();

  if (keep) {  // the frame's own copy of c_0, kept for the next frame's change test
    const int gx0 = tx * P, gy0 = ty * P;
    const int nx = min(P, g.W - gx0), ny = min(P, g.H - gy0);
    for (int q = threadIdx.x; q < P * (P / 4); q += NT) {
      const int y = q / (P / 4), x = 4 * (q % (P / 4));
      if (y < ny && x < nx) {
        uint8_t* d = keep + (long long)(gy0 + y) * keep_pitch + gx0 + x;
        const uint32_t v = ld32(cur + y * P + x);
        if (x + 4 <= nx) {
          *reinterpret_cast<uint32_t*>(d) = v;
        } else {
          for (int j = 0; j < nx - x; ++j) d[j] = (uint8_t)(v >> (8 * j));
        }
      }
    }
  }
  build<O, INTRA, true>(g, pyr, cur, tx, ty, g.L - 1);
  if (diff && mnx > 0 && mny > 0) {
    // Per-bin sums of |I_n - I_{n-1}| on c_0. Thread -> a 4-pixel
    // column word and a band of rows; the running sum is flushed into a
    // shared bin whenever the bin row changes (and split by pixel when the
    // word's pixels straddle bin columns).
    const int cb_lo = tcol[0], rb_lo = trow[0];
    const int ncols = tcol[mnx - 1] - cb_lo + 1, nrows = trow[mny - 1] - rb_lo + 1;
    const bool local = ncols * nrows <= kLocalBins;
    const uint8_t* A = cur;
    const uint8_t* B = prv;
    auto flush = [&](int rb, int cb, uint32_t v) {
      if (!v) return;
      if (local) {
        if (FKD_IDX(kChkPyrBins, (rb - rb_lo) * ncols + (cb - cb_lo), kLocalBins))
          atomicAdd(&bins[(rb - rb_lo) * ncols + (cb - cb_lo)], v);
      } else if (FKD_IDX(kChkPyrBins, rb * g.N_c + cb, g.NB)) {
        atomicAdd(&gsum[(long long)(rb * g.N_c + cb) * gstride], (unsigned long long)v);
      }
    };
    // warp w takes a band of rows, lane l the 4-pixel word column l
    static_assert(P / 4 <= 32 && NT == 256, "one lane per word column, 8 row bands");
    const int lane = threadIdx.x & 31, band = threadIdx.x >> 5;
    const int wcols = (mnx + 3) >> 2;
    const int rows_per = (mny + 7) >> 3;
    const int ya = band * rows_per, yb = min(mny, ya + rows_per);
    if (lane < wcols && ya < yb) {
      const int x = 4 * lane;
      const int nv = min(4, mnx - x);
      const uint32_t vmask = nv == 4 ? 0xffffffffu : ((1u << (8 * nv)) - 1u);
      const int c0 = tcol[x], c3 = tcol[x + nv - 1];
      if (c3 == c0) {
        // the word lies in one bin column: one sum per run of rows of one bin row
        for (int y = ya; y < yb;) {
          const int rb = trow[y], e = min(yb, (int)trun[y]);
          const uint8_t* pa = A + y * mn + x;
          const uint8_t* pb = B + y * mn + x;
          uint32_t run = 0;
#pragma unroll 4
          for (int yy = y; yy < e; ++yy, pa += mn, pb += mn) run += __vsadu4(ld32(pa) & vmask, ld32(pb) & vmask);
          flush(rb, c0, run);
          y = e;
        }
      } else {
        // the word straddles bin columns: split it pixel by pixel (bins
        // narrower than 4 pixels put middle pixels in further bins)
        uint32_t acc = 0, acc_hi = 0;
        int rb_cur = -1;
        for (int y = ya; y < yb; ++y) {
          const int rb = trow[y];
          if (rb != rb_cur) {
            if (rb_cur >= 0) {
              flush(rb_cur, c0, acc);
              flush(rb_cur, c3, acc_hi);
            }
            rb_cur = rb;
            acc = acc_hi = 0;
          }
          const uint32_t a = ld32(A + y * mn + x) & vmask, c = ld32(B + y * mn + x) & vmask;
          for (int i = 0; i < nv; ++i) {
            const int ci = tcol[x + i];
            const uint32_t d = __vabsdiffu4((a >> (8 * i)) & 0xffu, (c >> (8 * i)) & 0xffu);
            if (ci == c0) acc += d;
            else if (ci == c3) acc_hi += d;
            else flush(rb, ci, d);
          }
        }
        if (rb_cur >= 0) {
          flush(rb_cur, c0, acc);
          flush(rb_cur, c3, acc_hi);
        }
      }
    }
    if (local) {
      __syncthreads();
      for (int q = threadIdx.x; q < ncols * nrows; q += NT) {
        const uint32_t v = bins[q];
        if (v)
          atomicAdd(&gsum[(long long)((rb_lo + q / ncols) * g.N_c + cb_lo + q % ncols) * gstride],
                    (unsigned long long)v);
      }
    }
  }
  __syncthreads();
}

template <int O, int INTRA>
__global__ void __launch_bounds__(kPyrThreads, 8) k_pyramid(Geometry g, Tables tb, Batch b, Scratch s,
                                                         Params p, const __grid_constant__ CUtensorMap c0map,
                                                         int use_map) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(128) uint8_t smem_raw[];
  // the launch adds 128 bytes, so the tiles can start on a 128-byte boundary
  uint8_t* smem = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
  const int k = blockIdx.z;
  const uint8_t* frame = b.frames + (long long)k * b.frame_stride;
  // change sums of c_0 here; those of a coarser mask layer in the mask kernel
  const bool diff = p.mask_mode == FKD_MASK_ID && g.mask_layer == 0 && (b.first_frame + k) > 0;
  const uint8_t* pf = k == 0 ? b.prev : frame - b.frame_stride;
  const int pp = k == 0 ? b.prev_pitch : b.pitch;
  pyramid_tile<O, INTRA>(smem, g, tb, frame, b.pitch, pf, pp, diff, s.pyr + (long long)k * g.pyr_bytes,
                         s.bsum + k, s.bsum_stride, nullptr, 0, blockIdx.x, blockIdx.y,
                         use_map ? &c0map : nullptr, k, k > 0, s.overflow);
}

// Group tick: persistent CTAs over the c_0 tiles of every participating frame.
template <int O, int INTRA>
__global__ void __launch_bounds__(kPyrThreads, 4) k_group_pyramid(const StreamDev* devs,
                                                               const TickHeader* hdr,
                                                               const TickItem* items) {
  extern __shared__ __align__(128) uint8_t smem[];
  const int n = hdr->n_items, total = hdr->total_pyr;
  for (int j = blockIdx.x; j < total; j += gridDim.x) {
    const int i = find_item(n, j, [&](int q) { return items[q].pyr_base; });
    const TickItem it = items[i];
    const StreamDev& d = devs[it.sid];
    const int local = j - it.pyr_base;
    const int tx = local % d.g.pyr_tiles_x, ty = local / d.g.pyr_tiles_x;
    // change sums of c_0 here, against the stream's copy of its last frame;
    // those of a coarser mask layer in the mask kernel
    const bool c0_sums = d.p.mask_mode == FKD_MASK_ID && d.g.mask_layer == 0;
    const bool diff = c0_sums && it.frame_index > 0;
    const int kp = d.g.layer[0].pitch;
    pyramid_tile<O, INTRA>(smem, d.g, d.tb, it.frame, it.pitch, d.last[(it.frame_index + 1) & 1], kp, diff,
                           d.s.pyr, d.s.bsum, 1, c0_sums ? d.last[it.frame_index & 1] : nullptr, kp, tx, ty);
  }
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

// The batch's frames as a 3-D byte tensor (x, y, frame) with 96 x 96 x 1
// boxes, zero fill outside; false when the layout does not allow one (base,
// pitch or frame stride not a multiple of 16, overlapping frames) or the
// driver has no encoder.
bool encode_c0_map(CUtensorMap* map, const Geometry& g, const Batch& b) {
  static EncodeTiledFn encode = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<EncodeTiledFn>(f);
  });
  if (!encode || b.T < 1) return false;
  const long long plane = (long long)b.pitch * g.H;
  const long long fstride = b.T > 1 ? b.frame_stride : (plane + 15) / 16 * 16;
  if ((reinterpret_cast<uintptr_t>(b.frames) & 15) || (b.pitch & 15) || (fstride & 15) || fstride < plane)
    return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.W, (cuuint64_t)g.H, (cuuint64_t)b.T};
  const cuuint64_t strides[2] = {(cuuint64_t)b.pitch, (cuuint64_t)fstride};
  const cuuint32_t box[3] = {P, P, 1}, step[3] = {1, 1, 1};
  return encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<uint8_t*>(b.frames), dims, strides, box,
                step, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int O, int INTRA>
void launch_t(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s, const Params& p,
              cudaStream_t st) {
  dim3 grid(g.pyr_tiles_x, g.pyr_tiles_y, b.T);
  const int smem = pyr_smem(p.mask_mode == FKD_MASK_ID && g.mask_layer == 0);
  CUtensorMap map{};
  const int use_map = encode_c0_map(&map, g, b) ? 1 : 0;
  pdl_launch(k_pyramid<O, INTRA>, grid, dim3(kPyrThreads), smem + 128, st, g, tb, b, s, p, map, use_map);
}

template <int O, int INTRA>
void launch_group_t(const StreamDev* devs, const TickHeader* hdr, const TickItem* items, int grid,
                    cudaStream_t st) {
  k_group_pyramid<O, INTRA><<<grid, kPyrThreads, pyr_smem(true), st>>>(devs, hdr, items);
}

}  // namespace

void launch_pyramid(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                    const Params& p, cudaStream_t st) {
  using L = void (*)(const Geometry&, const Tables&, const Batch&, const Scratch&, const Params&,
                     cudaStream_t);
  static const L table[2][6] = {
      {launch_t<1, 0>, launch_t<2, 0>, launch_t<3, 0>, launch_t<4, 0>, launch_t<5, 0>, launch_t<6, 0>},
      {launch_t<1, 1>, launch_t<2, 1>, launch_t<3, 1>, launch_t<4, 1>, launch_t<5, 1>, launch_t<6, 1>}};
  table[g.intra ? 1 : 0][g.O - 1](g, tb, b, s, p, st);
}

int group_pyramid_grid(int O, int intra) {
  using K = void (*)(const StreamDev*, const TickHeader*, const TickItem*);
  static const K table[2][6] = {
      {k_group_pyramid<1, 0>, k_group_pyramid<2, 0>, k_group_pyramid<3, 0>, k_group_pyramid<4, 0>,
       k_group_pyramid<5, 0>, k_group_pyramid<6, 0>},
      {k_group_pyramid<1, 1>, k_group_pyramid<2, 1>, k_group_pyramid<3, 1>, k_group_pyramid<4, 1>,
       k_group_pyramid<5, 1>, k_group_pyramid<6, 1>}};
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, table[intra ? 1 : 0][O - 1], kPyrThreads,
                                                pyr_smem(true));
  return max(1, sms) * max(1, per_sm);
}

void launch_group_pyramid(int O, int intra, const StreamDev* devs, const TickHeader* hdr,
                          const TickItem* items, int grid, cudaStream_t st) {
  using L = void (*)(const StreamDev*, const TickHeader*, const TickItem*, int, cudaStream_t);
  static const L table[2][6] = {
      {launch_group_t<1, 0>, launch_group_t<2, 0>, launch_group_t<3, 0>, launch_group_t<4, 0>,
       launch_group_t<5, 0>, launch_group_t<6, 0>},
      {launch_group_t<1, 1>, launch_group_t<2, 1>, launch_group_t<3, 1>, launch_group_t<4, 1>,
       launch_group_t<5, 1>, launch_group_t<6, 1>}};
  table[intra ? 1 : 0][O - 1](devs, hdr, items, grid, st);
}

}  // namespace fkd
