/*
 * fkd_oracle.h -- plain single-threaded CPU oracle of the masked keypoint
 * detector of Baroffio, Cesana, Redondi, Tagliasacchi, "Fast keypoint
 * detection in video sequences" (arXiv 1503.06959).
 *
 * TEST INFRASTRUCTURE ONLY. This library exists to check the CUDA path. Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it. It shares no code, header, table or constant with the CUDA
 * library: every definition below is restated from the paper on its own.
 *
 * Layers (Sec. 2, Sec. 3.1): layer index l orders the pyramid by scale.
 * With intra-octaves: l = 2i is octave c_i (scale 2^i), l = 2i+1 is the
 * intra-octave d_i (scale 1.5 * 2^i).  Without: l = i is c_i.  S = 2*scale is
 * the integer scale code (2, 3, 4, 6, 8, 12, ...).
 *
 * Keypoint record: x, y in layer-pixel coordinates, layer, score (the largest
 * segment-test threshold that still fires, Sec. 2) and flags (bit 0: the
 * keypoint was carried over from the previous frame, Eq. 1).
 */
#ifndef FKD_ORACLE_H
#define FKD_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  uint16_t x, y;
  uint8_t layer, score;
  uint16_t flags;
} orc_keypoint;

/* FULL: every pixel active; ID: the block-mean intensity difference (Eq. 2
 * read per block); KB: keypoint binning (Eqs. 3-4); IDP: Eq. 2 per pixel of
 * every layer, each layer's mask deciding its own pixels (option (i) of
 * Sec. 3.1). */
enum { ORC_MASK_FULL = 0, ORC_MASK_ID = 1, ORC_MASK_KB = 2, ORC_MASK_IDP = 3 };

typedef struct {
  int N_r, N_c;     /* block grid rows, columns (Sec. 3.2)              */
  int T_I;          /* intensity-difference threshold (Eq. 2)           */
  int T_H;          /* keypoint-binning threshold (Eq. 4)               */
  int O;            /* octaves (Sec. 2)                                 */
  int intra;        /* 1: add the intra-octave layers d_i               */
  int t;            /* segment-test threshold (Sec. 2)                  */
  int mask_mode;    /* ORC_MASK_FULL / ID / KB                          */
  int mask_layer;   /* layer the ID test reads; -1 = coarsest octave    */
  int nms_scale;    /* 0: 3x3 maxima within the layer; 1: also against  */
                    /* the 3x3 windows of the adjacent layers (Sec. 2)  */
} orc_params;

/* Geometry of layer l; returns 0, or -1 if l is out of range. */
int orc_num_layers(int O, int intra);
int orc_layer_geom(int W, int H, int O, int intra, int l, int* w, int* h, int* S);

/* Pyramid: all layers concatenated in layer order, each w*h bytes, row-major
 * with pitch w (layer 0 is a copy of the frame). */
size_t orc_pyramid_bytes(int W, int H, int O, int intra);
void orc_build_pyramid(const uint8_t* frame, int W, int H, int O, int intra, uint8_t* out);

/* Corner score of pixel (x, y) of a w*h image (0 within 3 px of the edge). */
int orc_score(const uint8_t* img, int w, int h, int x, int y);
void orc_score_image(const uint8_t* img, int w, int h, uint8_t* out);

/* Binary descriptor of pixel (x, y) of a w*h layer: D bits (D % 8 == 0),
 * bit i set iff the 5x5 sum around (x+ax_i, y+ay_i) is below the 5x5 sum
 * around (x+bx_i, y+by_i) (coordinates clamped to the layer); pattern holds
 * D rows (ax, ay, bx, by); bit i lands in out[i/8] at bit i%8. */
int orc_describe(const uint8_t* img, int w, int h, int x, int y, const int8_t* pattern, int D,
                 uint8_t* out);

/* Block index r*N_c + c of pixel (x, y) of a layer with scale code S. */
int orc_block_of(int x, int y, int S, int W, int H, int N_r, int N_c);

/* Streams. */
typedef struct orc_stream orc_stream;
int orc_stream_create(const orc_params* p, int W, int H, orc_stream** out);
void orc_stream_destroy(orc_stream* s);
/* Process one frame.  mask_override: NULL, or N_r*N_c bytes used as M'_n in
 * place of the configured test (a hook for the mask properties of Eq. 1). */
int orc_stream_push(orc_stream* s, const uint8_t* frame, size_t pitch, const uint8_t* mask_override);
/* Masked description: before the first frame, a D-bit pattern (NULL, 0:
 * off). Each frame then describes its newly detected keypoints and carries
 * the descriptors of carried ones; orc_stream_descriptors writes D/8 bytes
 * per keypoint of D_n, in D_n's order (-1 if description is off). */
int orc_stream_set_descriptor(orc_stream* s, const int8_t* pattern, int D);
int orc_stream_descriptors(const orc_stream* s, uint8_t* out);
size_t orc_stream_num_keypoints(const orc_stream* s);
void orc_stream_keypoints(const orc_stream* s, orc_keypoint* out);
void orc_stream_mask(const orc_stream* s, uint8_t* out);
/* IDP mode: the last frame's per-pixel mask of layer l (w*h bytes, 0/1). */
int orc_stream_pixel_mask(const orc_stream* s, int l, uint8_t* out);
void orc_stream_block_sums(const orc_stream* s, uint64_t* out);
long orc_stream_frame_index(const orc_stream* s);

#ifdef __cplusplus
}
#endif
#endif
