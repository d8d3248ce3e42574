// k_pyramid.cu -- pyramid of octaves / intra-octaves and per-bin change sums.
//
// One CTA owns a 96 x 96 tile of c_0 of one frame. It loads the tile into
// shared memory with 16-byte vector loads, builds every layer of the tile in
// shared memory (Sec. 2: octaves c_i by 2x2 half-sampling, intra-octaves d_i
// by 2/3 resampling of c_0 then half-sampling), writes layers >= 1 to the
// frame's pyramid buffer, and -- for the intensity difference mask (Eq. 2,
// Sec. 3.1, which reuses the pyramid) -- adds |L_n - L_{n-1}| of the mask
// layer into the per-bin sums. The previous frame's mask layer is rebuilt
// from its c_0 tile in shared memory rather than read back, so the frames
// of a batch have no dependency on one another here.
#include "fkd_internal.cuh"

namespace fkd {
namespace {

// Shared-memory layout of one tile's pyramid for O <= 6: c_i is (96>>i)^2
// bytes, d_i is (64>>i)^2 bytes.
__host__ __device__ constexpr int c_size(int i) { return (kPyrTile >> i) * (kPyrTile >> i); }
__host__ __device__ constexpr int d_size(int i) { return ((2 * kPyrTile / 3) >> i) * ((2 * kPyrTile / 3) >> i); }
__host__ __device__ constexpr int c_off(int i) { return i == 0 ? 0 : c_off(i - 1) + c_size(i - 1); }
__host__ __device__ constexpr int d_off(int i) { return i == 0 ? c_off(6) : d_off(i - 1) + d_size(i - 1); }
constexpr int kPyrSmem = (d_off(6) + 15) / 16 * 16;
constexpr int kLocalBins = 1024;

struct Level {
  int off, n;  // smem offset and tile side
};

__device__ __forceinline__ Level level_of(int layer, int intra) {
  int i = intra ? layer >> 1 : layer;
  bool is_d = intra && (layer & 1);
  Level lv;
  lv.off = is_d ? d_off(i) : c_off(i);
  lv.n = is_d ? ((2 * kPyrTile / 3) >> i) : (kPyrTile >> i);
  return lv;
}

// Load a 96 x 96 tile of a frame (zeros outside the frame).
__device__ void load_c0(uint8_t* dst, const uint8_t* frame, int pitch, int gx0, int gy0, int W,
                        int H) {
  const bool vec = ((reinterpret_cast<uintptr_t>(frame) | (uintptr_t)pitch) & 15) == 0;
  constexpr int kChunks = kPyrTile / 16;
  for (int q = threadIdx.x; q < kPyrTile * kChunks; q += blockDim.x) {
    int r = q / kChunks, c = (q % kChunks) * 16;
    int gy = gy0 + r, gx = gx0 + c;
    uint8_t* d = dst + r * kPyrTile + c;
    if (gy < H && vec && gx + 16 <= W) {
      *reinterpret_cast<uint4*>(d) =
          __ldg(reinterpret_cast<const uint4*>(frame + (size_t)gy * pitch + gx));
    } else {
      for (int j = 0; j < 16; ++j)
        d[j] = (gy < H && gx + j < W) ? frame[(size_t)gy * pitch + gx + j] : 0;
    }
  }
}

// 2x2 box mean, round half up: src is n x n, dst (n/2) x (n/2).
__device__ void half_sample(const uint8_t* src, int n, uint8_t* dst) {
  const int m = n / 2;
  for (int q = threadIdx.x; q < m * m; q += blockDim.x) {
    int y = q / m, x = q % m;
    const uint8_t* s = src + (2 * y) * n + 2 * x;
    unsigned sum = s[0] + s[1] + s[n] + s[n + 1] + 2u;
    dst[q] = (uint8_t)(sum >> 2);
  }
}

// 2/3 resampling of the 96 x 96 c_0 tile into the 64 x 64 d_0 tile: each 3x3
// block gives a 2x2 block; an output is the mean of its 1.5 x 1.5 footprint
// (weights 4, 2, 2, 1 over 9), rounded to nearest.
__device__ void two_thirds(const uint8_t* src, uint8_t* dst) {
  constexpr int nb = kPyrTile / 3, n = kPyrTile, m = 2 * kPyrTile / 3;
  for (int q = threadIdx.x; q < nb * nb; q += blockDim.x) {
    int by = q / nb, bx = q % nb;
    const uint8_t* s = src + (3 * by) * n + 3 * bx;
    unsigned p00 = s[0], p01 = s[1], p02 = s[2];
    unsigned p10 = s[n], p11 = s[n + 1], p12 = s[n + 2];
    unsigned p20 = s[2 * n], p21 = s[2 * n + 1], p22 = s[2 * n + 2];
    uint8_t* d = dst + (2 * by) * m + 2 * bx;
    d[0] = (uint8_t)((4u * p00 + 2u * p01 + 2u * p10 + p11 + 4u) / 9u);
    d[1] = (uint8_t)((4u * p02 + 2u * p01 + 2u * p12 + p11 + 4u) / 9u);
    d[m] = (uint8_t)((4u * p20 + 2u * p21 + 2u * p10 + p11 + 4u) / 9u);
    d[m + 1] = (uint8_t)((4u * p22 + 2u * p21 + 2u * p12 + p11 + 4u) / 9u);
  }
}

// Build layers 1 .. up_to (inclusive) of the tile from its c_0.
__device__ void build_levels(uint8_t* pyr, int O, int intra, int up_to) {
  const int step = intra ? 2 : 1;
  for (int i = 1; i < O; ++i) {
    if (i * step > up_to) break;
    half_sample(pyr + c_off(i - 1), kPyrTile >> (i - 1), pyr + c_off(i));
    __syncthreads();
  }
  if (intra && up_to >= 1) {
    two_thirds(pyr, pyr + d_off(0));
    __syncthreads();
    for (int i = 1; i < O; ++i) {
      if (2 * i + 1 > up_to) break;
      half_sample(pyr + d_off(i - 1), (2 * kPyrTile / 3) >> (i - 1), pyr + d_off(i));
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kPyrThreads) k_pyramid(Geometry g, Tables tb, Batch b, Scratch s,
                                                         Params p) {
  __shared__ __align__(16) uint8_t cur[kPyrSmem];
  __shared__ __align__(16) uint8_t prv[kPyrSmem];
  __shared__ uint32_t bins[kLocalBins];

  const int k = blockIdx.z;
  const int tx = blockIdx.x, ty = blockIdx.y;
  const uint8_t* frame = b.frames + (long long)k * b.frame_stride;
  load_c0(cur, frame, b.pitch, tx * kPyrTile, ty * kPyrTile, g.W, g.H);

  const bool diff = p.mask_mode == FKD_MASK_ID && (b.first_frame + k) > 0;
  if (diff) {
    const uint8_t* pf = k == 0 ? b.prev : frame - b.frame_stride;
    const int pp = k == 0 ? b.prev_pitch : b.pitch;
    load_c0(prv, pf, pp, tx * kPyrTile, ty * kPyrTile, g.W, g.H);
  }
  for (int q = threadIdx.x; q < kLocalBins; q += blockDim.x) bins[q] = 0;
  __syncthreads();

  build_levels(cur, g.O, g.intra, g.L - 1);
  if (diff && g.mask_layer > 0) build_levels(prv, g.O, g.intra, g.mask_layer);

  // write layers >= 1 of the tile
  uint8_t* pyr = s.pyr + (long long)k * g.pyr_bytes;
  for (int l = 1; l < g.L; ++l) {
    const LayerGeom& lg = g.layer[l];
    Level lv = level_of(l, g.intra);
    const int gx0 = tx * lv.n, gy0 = ty * lv.n;
    const int nx = min(lv.n, lg.w - gx0), ny = min(lv.n, lg.h - gy0);
    if (nx <= 0 || ny <= 0) continue;
    uint8_t* dst = pyr + lg.pyr_off;
    for (int q = threadIdx.x; q < nx * ny; q += blockDim.x) {
      int y = q / nx, x = q % nx;
      dst[(long long)(gy0 + y) * lg.pitch + gx0 + x] = cur[lv.off + y * lv.n + x];
    }
  }

  if (!diff) return;

  // Per-bin sums of |L_n - L_{n-1}| on the mask layer. Each thread walks a
  // column of the layer tile, keeps a running sum while the bin row is the
  // same, and flushes it into a shared-memory bin when the row changes.
  const int ml = g.mask_layer;
  const LayerGeom& lg = g.layer[ml];
  const Level lv = level_of(ml, g.intra);
  const int gx0 = tx * lv.n, gy0 = ty * lv.n;
  const int nx = min(lv.n, lg.w - gx0), ny = min(lv.n, lg.h - gy0);
  if (nx <= 0 || ny <= 0) return;
  const uint16_t* colblk = tb.colblk + lg.col_off;
  const uint16_t* rowblk = tb.rowblk + lg.row_off;
  const int cb_lo = colblk[gx0], rb_lo = rowblk[gy0];
  const int ncols = colblk[gx0 + nx - 1] - cb_lo + 1;
  const int nrows = rowblk[gy0 + ny - 1] - rb_lo + 1;
  const bool local = ncols * nrows <= kLocalBins;
  unsigned long long* gsum = s.bsum + (long long)k * g.NB;

  const int groups = max(1, (int)blockDim.x / nx);
  const int rows_per = (ny + groups - 1) / groups;
  const int x = threadIdx.x % nx, grp = threadIdx.x / nx;
  if (grp < groups) {
    const int cb = colblk[gx0 + x];
    const uint8_t* a = cur + lv.off + x;
    const uint8_t* c = prv + lv.off + x;
    uint32_t acc = 0;
    int rb_cur = -1;
    const int y_end = min(ny, (grp + 1) * rows_per);
    for (int y = grp * rows_per; y < y_end; ++y) {
      int rb = rowblk[gy0 + y];
      if (rb != rb_cur) {
        if (rb_cur >= 0 && acc) {
          if (local) atomicAdd(&bins[(rb_cur - rb_lo) * ncols + (cb - cb_lo)], acc);
          else atomicAdd(&gsum[rb_cur * g.N_c + cb], (unsigned long long)acc);
        }
        rb_cur = rb;
        acc = 0;
      }
      int dv = (int)a[y * lv.n] - (int)c[y * lv.n];
      acc += (uint32_t)(dv < 0 ? -dv : dv);
    }
    if (rb_cur >= 0 && acc) {
      if (local) atomicAdd(&bins[(rb_cur - rb_lo) * ncols + (cb - cb_lo)], acc);
      else atomicAdd(&gsum[rb_cur * g.N_c + cb], (unsigned long long)acc);
    }
  }
  if (local) {
    __syncthreads();
    for (int q = threadIdx.x; q < ncols * nrows; q += blockDim.x) {
      uint32_t v = bins[q];
      if (v) atomicAdd(&gsum[(rb_lo + q / ncols) * g.N_c + cb_lo + q % ncols], (unsigned long long)v);
    }
  }
}

}  // namespace

void launch_pyramid(const Geometry& g, const Tables& tb, const Batch& b, const Scratch& s,
                    const Params& p, cudaStream_t st) {
  dim3 grid(g.pyr_tiles_x, g.pyr_tiles_y, b.T);
  k_pyramid<<<grid, kPyrThreads, 0, st>>>(g, tb, b, s, p);
}

}  // namespace fkd
