/*
 * fkd_oracle.c -- plain, slow, single-threaded CPU oracle of the masked
 * keypoint detector of arXiv 1503.06959 (Baroffio et al., "Fast keypoint
 * detection in video sequences").
 *
 * TEST INFRASTRUCTURE ONLY: it exists to check the CUDA library. Only the
 * test suite, the smoke check and the benchmark's CPU-baseline leg may load
 * it. It shares no code with the CUDA path. Every step follows the paper's
 * definitions in the paper's order, written as plain loops; where the paper
 * is silent the reading taken is stated beside the code.
 *
 * Steps per frame (Sec. 3):
 *   1. pyramid of octaves and intra-octaves (Sec. 2, Sec. 3.1)
 *   2. detection mask M'_n on the N_r x N_c grid: intensity difference
 *      (Eq. 2, Sec. 3.1) or keypoint binning (Eqs. 3-4, Sec. 3.2); or, per
 *      pixel of every layer, Eq. 2 itself (mode IDP)
 *   3. segment test with the 16-pixel radius-3 Bresenham ring, corner score,
 *      threshold t and 3x3 non-maximum suppression on every layer (Sec. 2),
 *      optionally over the scale-space neighbourhood (the adjacent layers)
 *   4. D_n = detections in active blocks united with the keypoints of
 *      D_{n-1} that lie in inactive blocks (Eq. 1).
 *   5. optionally, masked description: a binary pair-test descriptor for
 *      every keypoint detected in the frame, carried keypoints keeping
 *      theirs (Sec. 2, Sec. 3).
 */
#include "fkd_oracle.h"

#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ geometry */

int orc_num_layers(int O, int intra) { return intra ? 2 * O : O; }

/* Octave c_i has scale 2^i and is c_{i-1} halved (floor); the intra-octave
 * d_0 is the original resampled by 2/3 (floor(W/3)*2 columns) and d_i is d_{i-1}
 * halved (Sec. 2: octaves and intra-octaves by progressive half-sampling). */
int orc_layer_geom(int W, int H, int O, int intra, int l, int* w, int* h, int* S) {
  int L = orc_num_layers(O, intra);
  if (l < 0 || l >= L) return -1;
  int i = intra ? l / 2 : l;
  int is_d = intra ? (l % 2) : 0;
  int ww, hh, s;
  if (!is_d) {
    ww = W; hh = H; s = 2;
    for (int k = 0; k < i; ++k) { ww /= 2; hh /= 2; s *= 2; }
  } else {
    ww = (W / 3) * 2; hh = (H / 3) * 2; s = 3;
    for (int k = 0; k < i; ++k) { ww /= 2; hh /= 2; s *= 2; }
  }
  if (w) *w = ww;
  if (h) *h = hh;
  if (S) *S = s;
  return 0;
}

size_t orc_pyramid_bytes(int W, int H, int O, int intra) {
  size_t total = 0;
  for (int l = 0; l < orc_num_layers(O, intra); ++l) {
    int w, h, S;
    orc_layer_geom(W, H, O, intra, l, &w, &h, &S);
    total += (size_t)w * (size_t)h;
  }
  return total;
}

/* 2x2 box mean with round-half-up: the half-sampling step of the pyramid. */
static void half_sample(const uint8_t* src, int sw, int sh, uint8_t* dst, int dw, int dh) {
  (void)sh;
  for (int y = 0; y < dh; ++y)
    for (int x = 0; x < dw; ++x) {
      int a = src[(2 * y) * sw + 2 * x];
      int b = src[(2 * y) * sw + 2 * x + 1];
      int c = src[(2 * y + 1) * sw + 2 * x];
      int d = src[(2 * y + 1) * sw + 2 * x + 1];
      dst[y * dw + x] = (uint8_t)((a + b + c + d + 2) / 4);
    }
}

/* 2/3 resampling: every 3x3 input block becomes a 2x2 output block. Each output
 * pixel is the mean of its 1.5 x 1.5 input footprint, i.e. weights 4 (the
 * corner pixel it sits on), 2 and 2 (the two half-covered edge pixels) and 1
 * (the quarter-covered centre), over 9, rounded to nearest. */
static void two_thirds_sample(const uint8_t* src, int sw, int sh, uint8_t* dst, int dw, int dh) {
  (void)sh;
  for (int by = 0; by < dh / 2; ++by)
    for (int bx = 0; bx < dw / 2; ++bx) {
      int p[3][3]; /* p[row][col] */
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) p[r][c] = src[(3 * by + r) * sw + 3 * bx + c];
      for (int oy = 0; oy < 2; ++oy)
        for (int ox = 0; ox < 2; ++ox) {
          int cr = oy ? 2 : 0, cc = ox ? 2 : 0; /* the corner this output owns */
          int sum = 4 * p[cr][cc] + 2 * p[cr][1] + 2 * p[1][cc] + 1 * p[1][1];
          dst[(2 * by + oy) * dw + 2 * bx + ox] = (uint8_t)((sum + 4) / 9);
        }
    }
}

void orc_build_pyramid(const uint8_t* frame, int W, int H, int O, int intra, uint8_t* out) {
  int L = orc_num_layers(O, intra);
  size_t* off = (size_t*)calloc((size_t)L, sizeof(size_t));
  size_t acc = 0;
  for (int l = 0; l < L; ++l) {
    int w, h, S;
    orc_layer_geom(W, H, O, intra, l, &w, &h, &S);
    off[l] = acc;
    acc += (size_t)w * (size_t)h;
  }
  memcpy(out, frame, (size_t)W * (size_t)H);
  int step = intra ? 2 : 1;
  /* octaves: c_{i} from c_{i-1} */
  for (int i = 1; i < O; ++i) {
    int pl = (i - 1) * step, cl = i * step;
    int pw, ph, cw, ch, S;
    orc_layer_geom(W, H, O, intra, pl, &pw, &ph, &S);
    orc_layer_geom(W, H, O, intra, cl, &cw, &ch, &S);
    half_sample(out + off[pl], pw, ph, out + off[cl], cw, ch);
  }
  if (intra) {
    int w, h, S;
    orc_layer_geom(W, H, O, intra, 1, &w, &h, &S);
    two_thirds_sample(out, W, H, out + off[1], w, h);
    for (int i = 1; i < O; ++i) {
      int pl = 2 * (i - 1) + 1, cl = 2 * i + 1;
      int pw, ph, cw, ch;
      orc_layer_geom(W, H, O, intra, pl, &pw, &ph, &S);
      orc_layer_geom(W, H, O, intra, cl, &cw, &ch, &S);
      half_sample(out + off[pl], pw, ph, out + off[cl], cw, ch);
    }
  }
  free(off);
}

/* --------------------------------------------------------------- segment test */

/* The Bresenham circle of radius 3 around p, 16 pixels in ring order
 * (Sec. 2), starting straight above p and going clockwise (y grows down). */
static const int RING_DX[16] = {0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3, -3, -3, -2, -1};
static const int RING_DY[16] = {-3, -3, -2, -1, 0, 1, 2, 3, 3, 3, 2, 1, 0, -1, -2, -3};
#define ARC 9 /* contiguous pixels the test asks for (n = 9 of 16) */

/* Score: the largest t for which the segment test of Sec. 2 still fires, i.e.
 * 9 contiguous ring pixels all > I_p + t or all < I_p - t.  With
 * d_k = I_k - I_p, an arc j passes the bright test at t iff min over the arc of
 * d_k > t, so the largest passing t is (max over arcs of the arc minimum) - 1;
 * the dark side is the same on -d_k.  0 when no t >= 0 passes, and 0 within
 * 3 px of the image edge where the ring leaves the image. */
int orc_score(const uint8_t* img, int w, int h, int x, int y) {
  if (x < 3 || y < 3 || x >= w - 3 || y >= h - 3) return 0;
  int Ip = img[y * w + x];
  int d[16];
  for (int k = 0; k < 16; ++k) d[k] = (int)img[(y + RING_DY[k]) * w + (x + RING_DX[k])] - Ip;
  int best = -1000;
  for (int j = 0; j < 16; ++j) {
    int mn_b = 1000, mn_d = 1000;
    for (int m = 0; m < ARC; ++m) {
      int v = d[(j + m) % 16];
      if (v < mn_b) mn_b = v;
      if (-v < mn_d) mn_d = -v;
    }
    if (mn_b > best) best = mn_b;
    if (mn_d > best) best = mn_d;
  }
  int s = best - 1;
  return s > 0 ? s : 0;
}

void orc_score_image(const uint8_t* img, int w, int h, uint8_t* out) {
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) out[y * w + x] = (uint8_t)orc_score(img, w, h, x, y);
}

/* --------------------------------------------------------------- block grid */

/* A layer pixel (x, y) of scale code S sits at image position
 * X = floor(x*S/2), Y = floor(y*S/2); its bin is (floor(Y/S_y), floor(X/S_x))
 * with S_x = W/N_c and S_y = H/N_r (Eq. 3), evaluated exactly in integers as
 * floor(X*N_c/W), floor(Y*N_r/H). */
int orc_block_of(int x, int y, int S, int W, int H, int N_r, int N_c) {
  long X = ((long)x * S) / 2, Y = ((long)y * S) / 2;
  long c = (X * N_c) / W, r = (Y * N_r) / H;
  return (int)(r * N_c + c);
}

/* ------------------------------------------------------------------ streams */

struct orc_stream {
  orc_params p;
  int W, H, L;
  int lw[32], lh[32], lS[32];
  size_t loff[32];
  size_t pyr_bytes;
  uint8_t* pyr_prev; /* pyramid of I_{n-1} */
  uint8_t* pyr_cur;
  orc_keypoint* kp;  /* D_n, sorted by (layer, y, x) */
  size_t nkp, cap;
  uint8_t* mask;     /* M'_n, N_r*N_c */
  uint64_t* bsum;    /* block sums of |L_n - L_{n-1}| (ID) or bin counts (KB) */
  uint8_t* pmask;    /* IDP: per-pixel masks of every layer (pyramid layout) */
  long frame;        /* index of the last processed frame, -1 before any */
  int8_t* pattern;   /* description: D pairs (ax, ay, bx, by), or NULL */
  int D;             /* descriptor bits (0: no description) */
  uint8_t* desc;     /* descriptors of D_n, D/8 bytes each, in D_n's order */
};

/* Binary descriptor of pixel (x, y) of a w*h layer (Sec. 2: every bit
 * compares the smoothed intensities of one pair of pixels sampled around the
 * keypoint). The smoothed intensity at q is the sum of the 5x5 pixels around
 * q, coordinates clamped to the layer; bit i is set iff the sum at
 * (x + ax_i, y + ay_i) is below the sum at (x + bx_i, y + by_i), and lands
 * in byte i / 8 at bit i % 8. No orientation: the pattern is upright. */
static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int box5(const uint8_t* img, int w, int h, int qx, int qy) {
  int sum = 0;
  for (int dy = -2; dy <= 2; ++dy)
    for (int dx = -2; dx <= 2; ++dx)
      sum += img[(size_t)clampi(qy + dy, 0, h - 1) * w + clampi(qx + dx, 0, w - 1)];
  return sum;
}

int orc_describe(const uint8_t* img, int w, int h, int x, int y, const int8_t* pattern, int D,
                 uint8_t* out) {
  if (!img || !pattern || !out || w < 1 || h < 1 || x < 0 || y < 0 || x >= w || y >= h) return -1;
  if (D < 8 || (D & 7)) return -1;
  memset(out, 0, (size_t)D / 8);
  for (int i = 0; i < D; ++i) {
    const int8_t* q = pattern + 4 * i;
    int a = box5(img, w, h, x + q[0], y + q[1]);
    int b = box5(img, w, h, x + q[2], y + q[3]);
    if (a < b) out[i >> 3] |= (uint8_t)(1u << (i & 7));
  }
  return 0;
}

int orc_stream_create(const orc_params* p, int W, int H, orc_stream** out) {
  if (!p || !out || W < 1 || H < 1 || W > 16384 || H > 16384) return -1;
  if (p->N_r < 1 || p->N_c < 1 || p->N_r > H || p->N_c > W) return -1;
  if (p->O < 1 || p->O > 12 || (p->intra != 0 && p->intra != 1)) return -1;
  if (p->t < 1 || p->t > 255 || p->T_I < 0 || p->T_H < 0) return -1;
  if (p->mask_mode < ORC_MASK_FULL || p->mask_mode > ORC_MASK_IDP) return -1;
  if (p->nms_scale != 0 && p->nms_scale != 1) return -1;
  orc_stream* s = (orc_stream*)calloc(1, sizeof(orc_stream));
  s->p = *p;
  s->W = W; s->H = H;
  s->L = orc_num_layers(p->O, p->intra);
  if (s->p.mask_layer == -1) s->p.mask_layer = (p->O - 1) * (p->intra ? 2 : 1);
  if (s->p.mask_layer < 0 || s->p.mask_layer >= s->L) { free(s); return -1; }
  size_t acc = 0;
  for (int l = 0; l < s->L; ++l) {
    orc_layer_geom(W, H, p->O, p->intra, l, &s->lw[l], &s->lh[l], &s->lS[l]);
    s->loff[l] = acc;
    acc += (size_t)s->lw[l] * (size_t)s->lh[l];
  }
  s->pyr_bytes = acc;
  s->pyr_prev = (uint8_t*)calloc(acc, 1);
  s->pyr_cur = (uint8_t*)calloc(acc, 1);
  s->mask = (uint8_t*)calloc((size_t)p->N_r * p->N_c, 1);
  s->bsum = (uint64_t*)calloc((size_t)p->N_r * p->N_c, sizeof(uint64_t));
  s->pmask = (uint8_t*)calloc(acc + 1, 1);
  s->cap = 1024;
  s->kp = (orc_keypoint*)malloc(s->cap * sizeof(orc_keypoint));
  s->nkp = 0;
  s->frame = -1;
  *out = s;
  return 0;
}

void orc_stream_destroy(orc_stream* s) {
  if (!s) return;
  free(s->pyr_prev); free(s->pyr_cur); free(s->mask); free(s->bsum); free(s->kp); free(s->pmask);
  free(s->pattern); free(s->desc);
  free(s);
}

int orc_stream_set_descriptor(orc_stream* s, const int8_t* pattern, int D) {
  if (!s || s->frame >= 0) return -1;  /* before the first frame only */
  if (D != 0 && (!pattern || D < 8 || (D & 7))) return -1;
  free(s->pattern);
  s->pattern = NULL;
  s->D = D;
  if (D) {
    s->pattern = (int8_t*)malloc((size_t)D * 4);
    memcpy(s->pattern, pattern, (size_t)D * 4);
  }
  return 0;
}

static void kp_push(orc_keypoint** arr, size_t* n, size_t* cap, orc_keypoint k) {
  if (*n == *cap) {
    *cap *= 2;
    *arr = (orc_keypoint*)realloc(*arr, *cap * sizeof(orc_keypoint));
  }
  (*arr)[(*n)++] = k;
}

/* canonical order of D_n: (layer, y, x); positions in D_n are unique */
static int kp_cmp(const void* pa, const void* pb) {
  const orc_keypoint* a = (const orc_keypoint*)pa;
  const orc_keypoint* b = (const orc_keypoint*)pb;
  if (a->layer != b->layer) return a->layer < b->layer ? -1 : 1;
  if (a->y != b->y) return a->y < b->y ? -1 : 1;
  if (a->x != b->x) return a->x < b->x ? -1 : 1;
  return 0;
}

int orc_stream_push(orc_stream* s, const uint8_t* frame, size_t pitch, const uint8_t* mask_override) {
  const orc_params* p = &s->p;
  const int W = s->W, H = s->H, NB = p->N_r * p->N_c;
  if (pitch < (size_t)W) return -1;

  /* 1. pyramid L_n of the new frame (Sec. 3.1) */
  uint8_t* c0 = (uint8_t*)malloc((size_t)W * H);
  for (int y = 0; y < H; ++y) memcpy(c0 + (size_t)y * W, frame + (size_t)y * pitch, (size_t)W);
  orc_build_pyramid(c0, W, H, p->O, p->intra, s->pyr_cur);
  free(c0);

  /* 2. detection mask M'_n */
  memset(s->bsum, 0, (size_t)NB * sizeof(uint64_t));
  if (mask_override) {
    for (int b = 0; b < NB; ++b) s->mask[b] = mask_override[b] ? 1 : 0;
  } else if (s->frame < 0 || p->mask_mode == ORC_MASK_FULL) {
    /* the first frame has no history: detect everywhere */
    for (int b = 0; b < NB; ++b) s->mask[b] = 1;
  } else if (p->mask_mode == ORC_MASK_IDP) {
    /* per pixel, below */
  } else if (p->mask_mode == ORC_MASK_ID) {
    /* Eq. 2 read as "detect where the layer changed": block b is active iff
     * the sum of |L_n - L_{n-1}| over its pixels of the mask layer exceeds
     * T_I times their number (block mean above T_I). */
    int l = p->mask_layer;
    uint64_t* cnt = (uint64_t*)calloc((size_t)NB, sizeof(uint64_t));
    const uint8_t* a = s->pyr_cur + s->loff[l];
    const uint8_t* b = s->pyr_prev + s->loff[l];
    for (int y = 0; y < s->lh[l]; ++y)
      for (int x = 0; x < s->lw[l]; ++x) {
        int blk = orc_block_of(x, y, s->lS[l], W, H, p->N_r, p->N_c);
        int dv = (int)a[y * s->lw[l] + x] - (int)b[y * s->lw[l] + x];
        s->bsum[blk] += (uint64_t)(dv < 0 ? -dv : dv);
        cnt[blk] += 1;
      }
    for (int k = 0; k < NB; ++k) s->mask[k] = s->bsum[k] > (uint64_t)p->T_I * cnt[k] ? 1 : 0;
    free(cnt);
  } else {
    /* Eqs. 3-4: histogram of D_{n-1} over the bins, active iff count >= T_H */
    for (size_t i = 0; i < s->nkp; ++i) {
      const orc_keypoint* k = &s->kp[i];
      s->bsum[orc_block_of(k->x, k->y, s->lS[k->layer], W, H, p->N_r, p->N_c)] += 1;
    }
    for (int k = 0; k < NB; ++k) s->mask[k] = s->bsum[k] >= (uint64_t)p->T_H ? 1 : 0;
  }

  /* IDP: Eq. 2 per pixel of every layer, read as "active where the layer
   * changed by more than T_I" (the mask of layer l decides the pixels of
   * layer l); every pixel is active on the first frame. The block mask is
   * then all ones and plays no part. */
  if (p->mask_mode == ORC_MASK_IDP) {
    for (int b = 0; b < NB; ++b) s->mask[b] = 1;
    for (size_t i = 0; i < s->pyr_bytes; ++i) {
      int dv = (int)s->pyr_cur[i] - (int)s->pyr_prev[i];
      s->pmask[i] = (s->frame < 0 || (dv < 0 ? -dv : dv) > p->T_I) ? 1 : 0;
    }
  }
#define ORC_ACTIVE(l, x, y)                                                          \
  (p->mask_mode == ORC_MASK_IDP ? s->pmask[s->loff[l] + (size_t)(y) * s->lw[l] + (x)] \
                                : s->mask[orc_block_of((x), (y), s->lS[l], W, H, p->N_r, p->N_c)])

  /* 3+4. D_n (Eq. 1): keypoints of D_{n-1} in inactive blocks are kept ... */
  orc_keypoint* next = (orc_keypoint*)malloc(1024 * sizeof(orc_keypoint));
  size_t nn = 0, ncap = 1024;
  for (size_t i = 0; i < s->nkp; ++i) {
    orc_keypoint k = s->kp[i];
    if (!ORC_ACTIVE(k.layer, k.x, k.y)) {
      k.flags = 1;
      kp_push(&next, &nn, &ncap, k);
    }
  }
  /* ... and the detector runs on every layer (Sec. 2) at pixels of active
   * blocks: score >= t and strictly greater than all 8 neighbours' scores.
   * Neighbours are scored whatever their block's mask bit. */
  uint8_t* scores[32];
  for (int l = 0; l < s->L; ++l) {
    int w = s->lw[l], h = s->lh[l];
    scores[l] = (uint8_t*)malloc((size_t)w * h + 1);
    if (w > 0 && h > 0) orc_score_image(s->pyr_cur + s->loff[l], w, h, scores[l]);
  }
  for (int l = 0; l < s->L; ++l) {
    int w = s->lw[l], h = s->lh[l];
    if (w == 0 || h == 0) continue;
    const uint8_t* sc = scores[l];
    for (int y = 0; y < h; ++y)
      for (int x = 0; x < w; ++x) {
        int v = sc[y * w + x];
        if (v < p->t) continue;
        if (!ORC_ACTIVE(l, x, y)) continue;
        int is_max = 1;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (dx == 0 && dy == 0) continue;
            int qx = x + dx, qy = y + dy;
            int q = (qx >= 0 && qy >= 0 && qx < w && qy < h) ? sc[qy * w + qx] : 0;
            if (!(v > q)) is_max = 0;
          }
        /* Scale-space neighbourhood (Sec. 2, "3x3 scale-space"): the layers
         * just below and above in scale, each through the 3x3 window around
         * its pixel that contains this pixel's centre. Pixel x of scale code
         * S covers image columns [x*S/2, (x+1)*S/2), so its centre
         * (x + 1/2)*S/2 lies in pixel floor((2x + 1) * S / (2 S')) of the
         * layer with scale code S'. Pixels outside that layer count as 0. */
        for (int dl = -1; dl <= 1 && is_max && p->nms_scale; dl += 2) {
          int m = l + dl;
          if (m < 0 || m >= s->L) continue;
          int mw = s->lw[m], mh = s->lh[m];
          int cx = (int)(((long)(2 * x + 1) * s->lS[l]) / (2L * s->lS[m]));
          int cy = (int)(((long)(2 * y + 1) * s->lS[l]) / (2L * s->lS[m]));
          for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              int qx = cx + dx, qy = cy + dy;
              int q = (qx >= 0 && qy >= 0 && qx < mw && qy < mh) ? scores[m][qy * mw + qx] : 0;
              if (!(v > q)) is_max = 0;
            }
        }
        if (is_max) {
          orc_keypoint k;
          k.x = (uint16_t)x; k.y = (uint16_t)y; k.layer = (uint8_t)l; k.score = (uint8_t)v; k.flags = 0;
          kp_push(&next, &nn, &ncap, k);
        }
      }
  }
  for (int l = 0; l < s->L; ++l) free(scores[l]);
#undef ORC_ACTIVE
  qsort(next, nn, sizeof(orc_keypoint), kp_cmp);

  /* Description (Sec. 3): only the keypoints detected in this frame are
   * described, on their own layer of L_n; a carried keypoint keeps the
   * descriptor it had in D_{n-1} (found by its position, unique in D_{n-1}). */
  if (s->D) {
    const size_t DB = (size_t)s->D / 8;
    uint8_t* nd = (uint8_t*)malloc(nn * DB + 1);
    for (size_t i = 0; i < nn; ++i) {
      const orc_keypoint* k = &next[i];
      if (!(k->flags & 1)) {
        const int l = k->layer;
        orc_describe(s->pyr_cur + s->loff[l], s->lw[l], s->lh[l], k->x, k->y, s->pattern, s->D, nd + i * DB);
      } else {
        const orc_keypoint* o = (const orc_keypoint*)bsearch(k, s->kp, s->nkp, sizeof(orc_keypoint), kp_cmp);
        if (!o) { free(nd); free(next); return -1; }
        memcpy(nd + i * DB, s->desc + (size_t)(o - s->kp) * DB, DB);
      }
    }
    free(s->desc);
    s->desc = nd;
  }
  free(s->kp);
  s->kp = next; s->nkp = nn; s->cap = ncap;

  uint8_t* tmp = s->pyr_prev; s->pyr_prev = s->pyr_cur; s->pyr_cur = tmp;
  s->frame += 1;
  return 0;
}

size_t orc_stream_num_keypoints(const orc_stream* s) { return s->nkp; }
void orc_stream_keypoints(const orc_stream* s, orc_keypoint* out) {
  memcpy(out, s->kp, s->nkp * sizeof(orc_keypoint));
}
int orc_stream_descriptors(const orc_stream* s, uint8_t* out) {
  if (!s->D) return -1;
  memcpy(out, s->desc, s->nkp * ((size_t)s->D / 8));
  return 0;
}
void orc_stream_mask(const orc_stream* s, uint8_t* out) {
  memcpy(out, s->mask, (size_t)s->p.N_r * s->p.N_c);
}
int orc_stream_pixel_mask(const orc_stream* s, int l, uint8_t* out) {
  if (l < 0 || l >= s->L) return -1;
  memcpy(out, s->pmask + s->loff[l], (size_t)s->lw[l] * s->lh[l]);
  return 0;
}
void orc_stream_block_sums(const orc_stream* s, uint64_t* out) {
  memcpy(out, s->bsum, (size_t)s->p.N_r * s->p.N_c * sizeof(uint64_t));
}
long orc_stream_frame_index(const orc_stream* s) { return s->frame; }
