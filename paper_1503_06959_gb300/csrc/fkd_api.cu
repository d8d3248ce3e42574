// fkd_api.cu -- the C ABI of include/fkd.h: stream state, geometry tables
// and the launch sequence of one batch (pyramid -> mask -> active tiles ->
// detection -> assembly).
#include <algorithm>
#include <utility>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "fkd_internal.cuh"

using namespace fkd;

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(FKD_E_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                  __LINE__);                                                              \
  } while (0)

long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

}  // namespace

int fkd::set_error(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

namespace fkd {

// Debug checks (FKD_CHECK): the take-functions of every translation unit.
static std::vector<CheckTake>& check_takes() {
  static std::vector<CheckTake> v;
  return v;
}

int register_check(CheckTake take) {
  check_takes().push_back(take);
  return 1;
}

const char* check_site_name(unsigned site) {
  static const char* names[kChkSites] = {
      "?", "detection staging", "detection unit list", "detection word list", "detection score map",
      "detection pass bitmap", "detection keypoint bitmap", "detection score map (global)", "detection cell counts",
      "pyramid level tile", "pyramid bin sums", "assembly chunk words", "assembly set-bit list",
      "assembly source frames", "assembly kept-set bin counts"};
  return site < (unsigned)kChkSites ? names[site] : "?";
}

int collect_checks() {
  int rc = FKD_OK;
  for (CheckTake take : check_takes()) {
    CheckRecord r{};
    if (take(&r) && rc == FKD_OK)
      rc = set_error(FKD_E_CUDA, "index check failed in %s: index %lld outside [0, %lld)", check_site_name(r.site),
                     r.index, r.limit);
  }
  return rc;
}

}  // namespace fkd

namespace {
// Debug builds: every stream allocation sits between two guard bands of a
// known byte, checked by fkd_check_guards.
constexpr size_t kGuard = FKD_CHECK ? 256 : 0;
constexpr unsigned char kGuardByte = 0xA5;

// Debug builds: wait for the stream and report a failed index check.
int check_after(cudaStream_t st) {
  if (!FKD_CHECK) return FKD_OK;
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(FKD_E_CUDA, "cudaStreamSynchronize failed: %s", cudaGetErrorString(e));
  return collect_checks();
}
}  // namespace

struct fkd_stream {
  fkd_params p{};
  Geometry g{};
  cudaStream_t st = nullptr;
  cudaStream_t copy_st = nullptr;  // host-frame uploads, overlapped with the previous part's kernels
  static constexpr int kParts = 3;
  cudaEvent_t part_done[kParts] = {};  // upload of part i finished
  cudaEvent_t staging_free = nullptr;  // earlier work on the stream no longer needs the staging buffer
  std::vector<std::pair<void*, size_t>> allocs;  // device allocations and their sizes
  size_t bytes_held = 0;  // device bytes this stream allocated

  uint16_t* colblk = nullptr;
  uint16_t* rowblk = nullptr;
  int* xstart = nullptr;
  uint32_t* npix = nullptr;
  DetTile* tiles = nullptr;                  // the current shape's tiles
  DetTile* tile_shape[kDetShapes] = {};      // per tile shape
  int n_tiles_shape[kDetShapes] = {};
  int n_tiles_max = 0;
  AsmChunk* chunks = nullptr;
  uint32_t* wbins = nullptr;
  uint32_t* wmask = nullptr;
  int* rowchunk = nullptr;
  int* rowcell = nullptr;
  int* bincell_off = nullptr;  // per bin: start of its cells (NB + 1)
  int* bincell = nullptr;      // cells of every bin

  Scratch s{};
  uint32_t* state_bits[2] = {nullptr, nullptr};
  uint8_t* state_score[2] = {nullptr, nullptr};
  uint32_t* state_cnt[2] = {nullptr, nullptr};
  int state_cur = 0;

  uint8_t* staging[2] = {nullptr, nullptr};
  int staging_next = 0;
  long long staging_pitch = 0;

  fkd_keypoint* rec = nullptr;     // result of the last fkd_push_frame (K_max records)
  uint32_t* rec_offsets = nullptr; // [2]
  fkd_keypoint* host_out = nullptr;  // device staging for host-output batches
  long long host_out_cap = 0;
  uint32_t* host_offsets = nullptr;  // [T_max + 1]
  uint8_t* last_mask = nullptr;      // device pointer to the last frame's mask

  // masked description (off while desc_D == 0)
  int desc_D = 0;
  int8_t* desc_pattern = nullptr;          // [D][4]
  uint32_t* desc = nullptr;                // per output record, D / 32 words
  long long desc_cap = 0;                  // records desc holds
  fkd_keypoint* keep_rec[2] = {nullptr, nullptr};  // the last frame's records and descriptors, ping-pong
  uint32_t* keep_desc[2] = {nullptr, nullptr};     //   with the kept keypoint set (state_cur)
  uint32_t* keep_n = nullptr;              // [2]
  uint32_t* desc_count = nullptr;          // [2]: end index of the last call's described records, work counter
  uint32_t* desc_rows = nullptr;           // [T_max][rows]: first record of each layer row of each frame
  uint32_t* keep_row[2] = {nullptr, nullptr};  // [rows + 1]: the kept set's row starts, ping-pong
  int rows = 0;                            // layer rows per frame
  bool desc_ready = false;                 // a frame was described since description was set

  const uint8_t* prev = nullptr;
  int prev_pitch = 0;
  long long frame = 0;
  long long last_frame_slot = 0;  // batch slot of the last frame pushed
  DetLaunch dl{};
  fkd_launch_config lc{};
  bool have_frame_result = false;

  // profiling: events around each stage of each batch, read back lazily
  bool profiling = false;
  struct Pending {
    cudaEvent_t ev[FKD_NUM_STAGES + 1];
    int frames;
    bool described;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  fkd_profile prof{};
  unsigned long long tile_stats_seen[2] = {0, 0};

  cudaEvent_t take_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }

  template <class T>
  int alloc(T** p, size_t count) {
    void* d = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    cudaError_t e = cudaMalloc(&d, bytes + 2 * kGuard);
    if (e != cudaSuccess) return fail(FKD_E_CUDA, "cudaMalloc(%zu) failed: %s", bytes, cudaGetErrorString(e));
    if (kGuard) {
      e = cudaMemset(d, kGuardByte, kGuard);
      if (e == cudaSuccess) e = cudaMemset(static_cast<char*>(d) + kGuard + bytes, kGuardByte, kGuard);
      if (e != cudaSuccess) {
        cudaFree(d);
        return fail(FKD_E_CUDA, "guard fill failed: %s", cudaGetErrorString(e));
      }
    }
    void* user = static_cast<char*>(d) + kGuard;
    allocs.emplace_back(user, bytes);
    bytes_held += bytes + 2 * kGuard;
    *p = static_cast<T*>(user);
    return FKD_OK;
  }
  // free one allocation made by alloc()
  template <class T>
  void free_one(T*& p) {
    if (!p) return;
    auto it = std::find_if(allocs.begin(), allocs.end(), [&](const auto& a) { return a.first == (void*)p; });
    if (it != allocs.end()) {
      bytes_held -= it->second + 2 * kGuard;
      allocs.erase(it);
    }
    cudaFree(reinterpret_cast<char*>(p) - kGuard);
    p = nullptr;
  }
  void release() {
    for (auto& a : allocs) cudaFree(static_cast<char*>(a.first) - kGuard);
    allocs.clear();
    bytes_held = 0;
    for (auto& pd : pending)
      for (cudaEvent_t e : pd.ev) cudaEventDestroy(e);
    pending.clear();
    for (cudaEvent_t e : event_pool) cudaEventDestroy(e);
    event_pool.clear();
    for (cudaEvent_t& e : part_done)
      if (e) cudaEventDestroy(e), e = nullptr;
    if (staging_free) cudaEventDestroy(staging_free), staging_free = nullptr;
    if (copy_st) cudaStreamDestroy(copy_st), copy_st = nullptr;
  }
};

namespace {

int validate(const fkd_params* p, int W, int H) {
  if (!p) return fail(FKD_E_ARG, "params is NULL");
  if (p->version != FKD_VERSION) return fail(FKD_E_ARG, "params.version %u != %u", p->version, FKD_VERSION);
  if (W < 1 || H < 1 || W > 16384 || H > 16384) return fail(FKD_E_ARG, "frame size %dx%d outside 1..16384", W, H);
  if (p->N_r < 1 || p->N_c < 1 || p->N_c > W || p->N_r > H || p->N_r * p->N_c > kMaxBins)
    return fail(FKD_E_ARG, "bin grid %dx%d invalid for %dx%d frames", p->N_r, p->N_c, W, H);
  if (p->O < 1 || p->O > 6) return fail(FKD_E_ARG, "O=%d outside 1..6", p->O);
  if (p->intra != 0 && p->intra != 1) return fail(FKD_E_ARG, "intra must be 0 or 1");
  if (p->t < 1 || p->t > 255) return fail(FKD_E_ARG, "t=%d outside 1..255", p->t);
  if (p->n != 9) return fail(FKD_E_ARG, "arc length n=%d: only 9 is supported", p->n);
  if (p->T_I < 0 || p->T_H < 0) return fail(FKD_E_ARG, "thresholds must be >= 0");
  if (p->mask_mode < FKD_MASK_FULL || p->mask_mode > FKD_MASK_IDP) return fail(FKD_E_ARG, "bad mask_mode");
  const int L = p->intra ? 2 * p->O : p->O;
  if (p->mask_layer < -1 || p->mask_layer >= L) return fail(FKD_E_ARG, "mask_layer %d outside -1..%d", p->mask_layer, L - 1);
  if (p->K_max < 1) return fail(FKD_E_ARG, "K_max must be >= 1");
  if (p->T_max < 1 || p->T_max > 65535) return fail(FKD_E_ARG, "T_max outside 1..65535");
  if (p->nms_scale != 0 && p->nms_scale != 1) return fail(FKD_E_ARG, "nms_scale must be 0 or 1");
  return FKD_OK;
}

// Layer sizes: c_0 = W x H; c_{i+1} = floor(c_i / 2); d_0 = 2 floor(W/3) x
// 2 floor(H/3); d_{i+1} = floor(d_i / 2). Scale code S = 2 * sigma.
void layer_dims(int W, int H, int intra, int l, int* w, int* h, int* S) {
  const int i = intra ? l / 2 : l;
  const bool d = intra && (l & 1);
  int ww = d ? (W / 3) * 2 : W, hh = d ? (H / 3) * 2 : H;
  ww >>= i;
  hh >>= i;
  *w = ww;
  *h = hh;
  *S = (d ? 3 : 2) << i;
}

int build_geometry(fkd_stream* s, int W, int H) {
  const fkd_params& p = s->p;
  Geometry& g = s->g;
  g.W = W;
  g.H = H;
  g.O = p.O;
  g.intra = p.intra;
  g.L = p.intra ? 2 * p.O : p.O;
  g.N_r = p.N_r;
  g.N_c = p.N_c;
  g.NB = p.N_r * p.N_c;
  g.mask_layer = p.mask_layer == -1 ? (p.O - 1) * (p.intra ? 2 : 1) : p.mask_layer;

  std::vector<uint16_t> colblk, rowblk;
  std::vector<int> xstart;
  std::vector<DetTile> tiles[kDetShapes];
  std::vector<AsmChunk> chunks;
  std::vector<uint32_t> wbins, wmask;
  std::vector<int> rowchunk, rowcell;
  long long pyr = 0, score = 0, bits = 0;
  int cells = 0;
  for (int l = 0; l < g.L; ++l) {
    LayerGeom& lg = g.layer[l];
    layer_dims(W, H, p.intra, l, &lg.w, &lg.h, &lg.S);
    lg.pitch = (int)round_up(std::max(lg.w, 1), 16);
    if (l == 0) {
      lg.pyr_off = -1;
    } else {
      lg.pyr_off = pyr;
      pyr += round_up((long long)lg.pitch * lg.h, 256);
    }
    lg.score_off = score;
    score += round_up((long long)lg.pitch * lg.h, 256);
    lg.wpr = (lg.w + 31) / 32;
    lg.bit_off = bits;
    bits += (long long)lg.wpr * lg.h;
    // bins of the layer's pixels: image position X = floor(x*S/2), bin column
    // floor(X / (W/N_c)) = floor(X*N_c/W) (Eq. 3), rows likewise
    lg.col_off = (int)colblk.size();
    for (int x = 0; x < lg.w; ++x) colblk.push_back((uint16_t)(((long long)x * lg.S / 2) * p.N_c / W));
    lg.row_off = (int)rowblk.size();
    for (int y = 0; y < lg.h; ++y) rowblk.push_back((uint16_t)(((long long)y * lg.S / 2) * p.N_r / H));
    lg.xs_off = (int)xstart.size();
    for (int c = 0; c <= p.N_c; ++c) {
      int x = 0;
      while (x < lg.w && colblk[lg.col_off + x] < c) ++x;
      xstart.push_back(x);
    }
    // per bitmap word column: its first and last bin column
    lg.wb_off = (int)wbins.size();
    for (int wx = 0; wx < lg.wpr; ++wx) {
      const int x1 = std::min(32 * wx + 32, lg.w) - 1;
      const uint16_t c0 = colblk[lg.col_off + 32 * wx];
      wbins.push_back((uint32_t)c0 | ((uint32_t)colblk[lg.col_off + x1] << 16));
      uint32_t m = 0;
      for (int x = 32 * wx; x <= x1; ++x)
        if (colblk[lg.col_off + x] == c0) m |= 1u << (x - 32 * wx);
      wmask.push_back(m);
    }
    // assembly chunks: bands of whole rows, about kAsmChunkWords words each;
    // a chunk's cells are its parts in the bins of the bin rows it spans
    if (lg.wpr > 0) {
      const int rows = std::max(1, kAsmChunkWords / lg.wpr);
      for (int y0 = 0; y0 < lg.h; y0 += rows) {
        const int y1 = std::min(lg.h, y0 + rows);
        const int rb0 = rowblk[lg.row_off + y0], rb1 = rowblk[lg.row_off + y1 - 1];
        for (int y = y0; y < y1; ++y) {
          rowchunk.push_back((int)chunks.size());
          rowcell.push_back(cells + (rowblk[lg.row_off + y] - rb0) * p.N_c);
        }
        chunks.push_back(AsmChunk{l, y0, y1, cells, rb0, rb1});
        cells += (rb1 - rb0 + 1) * p.N_c;
      }
    } else {
      for (int y = 0; y < lg.h; ++y) {
        rowchunk.push_back(0);
        rowcell.push_back(0);
      }
    }
    // detection tiles of every shape: kDetTW x TH rectangles, row-major
    for (int k = 0; k < kDetShapes && lg.w > 0 && lg.h > 0; ++k) {
      const int TH = kDetTH[k];
      for (int ty = 0; ty * TH < lg.h; ++ty)
        for (int tx = 0; tx * kDetTW < lg.w; ++tx) {
          DetTile t{};
          t.layer = (uint16_t)l;
          t.tx = (uint16_t)tx;
          t.ty = (uint16_t)ty;
          const int x1 = std::min((tx + 1) * kDetTW, lg.w) - 1, y1 = std::min((ty + 1) * TH, lg.h) - 1;
          t.area = (uint16_t)((x1 - tx * kDetTW + 1) * (y1 - ty * TH + 1));
          t.cb0 = colblk[lg.col_off + tx * kDetTW];
          t.cb1 = colblk[lg.col_off + x1];
          t.rb0 = rowblk[lg.row_off + ty * TH];
          t.rb1 = rowblk[lg.row_off + y1];
          tiles[k].push_back(t);
        }
    }
  }
  g.pyr_bytes = std::max(pyr, 256LL);
  g.score_bytes = score;
  g.bit_words = bits;
  size_t all_tiles = 0;
  for (int k = 0; k < kDetShapes; ++k) {
    s->n_tiles_shape[k] = (int)tiles[k].size();
    s->n_tiles_max = std::max(s->n_tiles_max, s->n_tiles_shape[k]);
    all_tiles += tiles[k].size();
  }
  g.det_shape = kDetDefaultShape;
  g.n_tiles = s->n_tiles_shape[g.det_shape];
  g.n_chunks = (int)chunks.size();
  g.n_cells = cells;
  // the cells of every bin, for keypoint binning in spans
  std::vector<std::vector<int>> per_bin(g.NB);
  for (const AsmChunk& ch : chunks)
    for (int r = ch.rb0; r <= ch.rb1; ++r)
      for (int c = 0; c < p.N_c; ++c) per_bin[r * p.N_c + c].push_back(ch.cell0 + (r - ch.rb0) * p.N_c + c);
  std::vector<int> bincell_off(1, 0), bincell;
  for (const auto& v : per_bin) {
    bincell.insert(bincell.end(), v.begin(), v.end());
    bincell_off.push_back((int)bincell.size());
  }
  g.pyr_tiles_x = (W + kPyrTile - 1) / kPyrTile;
  g.pyr_tiles_y = (H + kPyrTile - 1) / kPyrTile;

  // pixels of the mask layer in each bin
  std::vector<uint32_t> npix(g.NB, 0);
  const LayerGeom& ml = g.layer[g.mask_layer];
  for (int y = 0; y < ml.h; ++y)
    for (int x = 0; x < ml.w; ++x) npix[rowblk[ml.row_off + y] * p.N_c + colblk[ml.col_off + x]] += 1;

  int rc;
  if ((rc = s->alloc(&s->colblk, colblk.size())) || (rc = s->alloc(&s->rowblk, rowblk.size())) ||
      (rc = s->alloc(&s->xstart, xstart.size())) || (rc = s->alloc(&s->npix, npix.size())) ||
      (rc = s->alloc(&s->tile_shape[0], all_tiles)) || (rc = s->alloc(&s->chunks, chunks.size())) ||
      (rc = s->alloc(&s->wbins, wbins.size())) || (rc = s->alloc(&s->wmask, wmask.size())) ||
      (rc = s->alloc(&s->rowchunk, rowchunk.size())) || (rc = s->alloc(&s->rowcell, rowcell.size())) ||
      (rc = s->alloc(&s->bincell_off, bincell_off.size())) || (rc = s->alloc(&s->bincell, bincell.size())))
    return rc;
  CK(cudaMemcpy(s->bincell_off, bincell_off.data(), bincell_off.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!bincell.empty())
    CK(cudaMemcpy(s->bincell, bincell.data(), bincell.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!rowcell.empty())
    CK(cudaMemcpy(s->rowcell, rowcell.data(), rowcell.size() * sizeof(int), cudaMemcpyHostToDevice));
  if (!rowchunk.empty())
    CK(cudaMemcpy(s->rowchunk, rowchunk.data(), rowchunk.size() * sizeof(int), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->wmask, wmask.data(), wmask.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->chunks, chunks.data(), chunks.size() * sizeof(AsmChunk), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->wbins, wbins.data(), wbins.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->colblk, colblk.data(), colblk.size() * 2, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->rowblk, rowblk.data(), rowblk.size() * 2, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->xstart, xstart.data(), xstart.size() * 4, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->npix, npix.data(), npix.size() * 4, cudaMemcpyHostToDevice));
  for (int k = 0; k < kDetShapes; ++k) {
    if (k > 0) s->tile_shape[k] = s->tile_shape[k - 1] + tiles[k - 1].size();
    if (!tiles[k].empty())
      CK(cudaMemcpy(s->tile_shape[k], tiles[k].data(), tiles[k].size() * sizeof(DetTile), cudaMemcpyHostToDevice));
  }
  s->tiles = s->tile_shape[g.det_shape];
  return FKD_OK;
}

int allocate_state(fkd_stream* s) {
  const Geometry& g = s->g;
  const long long T = s->p.T_max;
  Scratch& sc = s->s;
  int rc;
  if ((rc = s->alloc(&sc.pyr, (size_t)(T * g.pyr_bytes))) ||
      (rc = s->alloc(&sc.bsum, (size_t)(T * g.NB))) || (rc = s->alloc(&sc.mask, (size_t)(T * g.NB + 4))) ||
      (rc = s->alloc(&sc.src, (size_t)(T * g.NB))) ||
      (rc = s->alloc(&sc.work, (size_t)(T * std::max(s->n_tiles_max, 1)))) ||
      (rc = s->alloc(&sc.work_count, 1)) ||
      (rc = s->alloc(&sc.det_bits, (size_t)(T * std::max(g.bit_words, 1LL)))) ||
      (rc = s->alloc(&sc.det_score, (size_t)(T * g.score_bytes))) ||
      (rc = s->alloc(&sc.chunk_counts, (size_t)(T * std::max(g.n_chunks, 1)))) ||
      (rc = s->alloc(&sc.alive, (size_t)g.NB)) ||
      (rc = s->alloc(&sc.merged, (size_t)(T * std::max(g.bit_words, 1LL)))) ||
      (rc = s->alloc(&sc.frame_totals, (size_t)T)) || (rc = s->alloc(&sc.out_base, 2)) ||
      (rc = s->alloc(&sc.overflow, 1)) || (rc = s->alloc(&sc.tile_stats, 2)) ||
      (rc = s->alloc(&sc.ml_prev, (size_t)g.layer[g.mask_layer].pitch * std::max(g.layer[g.mask_layer].h, 1))))
    return rc;
  CK(cudaMemset(sc.tile_stats, 0, 16));
  sc.pmask = nullptr;
  sc.pyr_last = nullptr;
  sc.dcnt = nullptr;
  if (s->p.mask_mode == FKD_MASK_KB && (rc = s->alloc(&sc.dcnt, (size_t)(T * std::max(g.n_cells, 1))))) return rc;
  if (s->p.mask_mode == FKD_MASK_IDP &&
      ((rc = s->alloc(&sc.pmask, (size_t)(T * std::max(g.bit_words, 1LL)))) ||
       (rc = s->alloc(&sc.pyr_last, (size_t)g.pyr_bytes))))
    return rc;
  for (int i = 0; i < 2; ++i) {
    if ((rc = s->alloc(&s->state_bits[i], (size_t)std::max(g.bit_words, 1LL))) ||
        (rc = s->alloc(&s->state_score[i], (size_t)g.score_bytes)) ||
        (rc = s->alloc(&s->state_cnt[i], (size_t)g.NB)))
      return rc;
    CK(cudaMemset(s->state_bits[i], 0, (size_t)std::max(g.bit_words, 1LL) * 4));
    CK(cudaMemset(s->state_cnt[i], 0, (size_t)g.NB * 4));
  }
  CK(cudaMemset(sc.bsum, 0, (size_t)(T * g.NB) * 8));
  sc.bsum_stride = (int)T;
  CK(cudaMemset(sc.overflow, 0, 4));
  CK(cudaMemset(sc.out_base, 0, 16));
  if ((rc = s->alloc(&s->rec, (size_t)s->p.K_max)) || (rc = s->alloc(&s->rec_offsets, 2)) ||
      (rc = s->alloc(&s->host_offsets, (size_t)(T + 1))))
    return rc;
  CK(cudaMemset(s->rec_offsets, 0, 8));
  return FKD_OK;
}

// One batch of T frames already in device memory.
int run_batch(fkd_stream* s, const uint8_t* frames, int pitch, long long stride, int T,
              fkd_keypoint* out, long long cap, uint32_t* offsets, int base_slot, bool reset_base) {
  Batch b{};
  b.T = T;
  b.first_frame = s->frame;
  b.frames = frames;
  b.frame_stride = stride;
  b.pitch = pitch;
  b.prev = s->prev;
  b.prev_pitch = s->prev_pitch;
  b.c0_vec = 0;
  Params pr{s->p.T_I, s->p.T_H, s->p.t, s->p.mask_mode, s->p.nms_scale};
  Tables tb{s->colblk, s->rowblk, s->xstart, s->npix, s->tiles, s->chunks, s->wbins, s->wmask, s->rowchunk,
            s->rowcell, s->bincell_off, s->bincell};
  State stt{};
  stt.bits_in = s->state_bits[s->state_cur];
  stt.score_in = s->state_score[s->state_cur];
  stt.cnt_in = s->state_cnt[s->state_cur];
  stt.bits_out = s->state_bits[s->state_cur ^ 1];
  stt.score_out = s->state_score[s->state_cur ^ 1];
  stt.cnt_out = s->state_cnt[s->state_cur ^ 1];
  Output o{out, cap, offsets, base_slot};
  if (s->desc_D) {
    o.row_base = s->desc_rows;
    o.rows = s->rows;
  }

  fkd_stream::Pending pd{};
  const bool prof = s->profiling;
  auto mark = [&](int i) {
    if (prof) {
      pd.ev[i] = s->take_event();
      cudaEventRecord(pd.ev[i], s->st);
    }
  };
  mark(0);
  launch_pyramid(s->g, tb, b, s->s, pr, s->st);
  mark(1);
  if (pr.mask_mode == FKD_MASK_KB) {
    // keypoint binning: spans of frames detected on the bins still active
    // at the span's start, then the exact masks resolved from the detection
    // counts (the "mask" and "worklist" stages are empty; "detect" holds the
    // spans and the source-frame scan)
    mark(2);
    mark(3);
    for (int k0 = 0; k0 < T; k0 += kKbSpan) {
      const int k1 = std::min(T, k0 + kKbSpan);
      launch_kb_span(s->g, b, s->s, pr, stt, k0, k1, k0 == 0, s->st);
      launch_worklist(s->g, tb, b, s->s, s->st, k0, k1);
      launch_detect(s->g, tb, b, s->s, pr, s->dl, s->st);
      if (pr.nms_scale) launch_scale_nms(s->g, tb, b, s->s, pr, s->st);
      launch_kb_resolve(s->g, tb, b, s->s, pr, k0, k1, s->st);
    }
    launch_source_frames(s->g, tb, b, s->s, pr, stt, s->st, reset_base ? base_slot : -1);
  } else {
    launch_mask(s->g, tb, b, s->s, pr, stt, s->st, reset_base ? base_slot : -1);
    if (s->s.pmask) launch_pixel_mask(s->g, b, s->s, pr, s->st);
    mark(2);
    launch_worklist(s->g, tb, b, s->s, s->st);
    mark(3);
    launch_detect(s->g, tb, b, s->s, pr, s->dl, s->st);
    if (pr.nms_scale) launch_scale_nms(s->g, tb, b, s->s, pr, s->st);
  }
  mark(4);
  if (s->s.pmask) launch_count_pixel(s->g, tb, b, s->s, stt, s->st);
  else launch_count(s->g, tb, b, s->s, stt, s->st);
  mark(5);
  launch_emit(s->g, tb, b, s->s, stt, o, s->st);
  mark(6);
  pd.described = s->desc_D != 0;
  if (s->desc_D) {
    // descriptors of the detected records, carried ones copied (Sec. 3)
    Describe d{};
    d.pattern = s->desc_pattern;
    d.D = s->desc_D;
    d.desc = s->desc;
    d.keep_rec_in = s->keep_rec[s->state_cur];
    d.keep_desc_in = s->keep_desc[s->state_cur];
    d.keep_n_in = s->keep_n + s->state_cur;
    d.keep_rec_out = s->keep_rec[s->state_cur ^ 1];
    d.keep_desc_out = s->keep_desc[s->state_cur ^ 1];
    d.keep_n_out = s->keep_n + (s->state_cur ^ 1);
    d.keep_cap = s->p.K_max;
    d.keep_row_in = s->keep_row[s->state_cur];
    d.keep_row_out = s->keep_row[s->state_cur ^ 1];
    d.count = s->desc_count;
    d.next_group = s->desc_count + 1;
    d.missing = s->s.overflow;
    launch_describe(s->g, tb, b, s->s, o, d, s->st);
    s->desc_ready = true;
  }
  mark(7);
  if (s->s.pmask && s->g.L > 1)  // layers >= 1 of the batch's last frame: L_{n-1} of the next batch
    CK(cudaMemcpyAsync(s->s.pyr_last, s->s.pyr + (long long)(T - 1) * s->g.pyr_bytes, (size_t)s->g.pyr_bytes,
                       cudaMemcpyDeviceToDevice, s->st));
  CK(cudaGetLastError());
  if (int rc = check_after(s->st)) return rc;
  if (prof) {
    pd.frames = T;
    s->pending.push_back(pd);
  }

  s->state_cur ^= 1;
  s->prev = frames + (long long)(T - 1) * stride;
  s->prev_pitch = pitch;
  s->frame += T;
  s->last_mask = s->s.mask + (long long)(T - 1) * s->g.NB;
  s->last_frame_slot = T - 1;
  return FKD_OK;
}

// T frames in device memory as one batch (keypoint binning, whose mask needs
// the previous frame's keypoints, runs in spans inside the batch); masks, if
// not NULL, receive each frame's mask.
// With `parts` > 1 the frames arrive in that many equal parts (the last one
// shorter), part i ready once s->part_done[i] has fired; each part is then
// its own batch (exactly the same results), so its kernels start while the
// later parts are still uploading.
int run_frames(fkd_stream* s, const uint8_t* dframes, int dpitch, long long dstride, int T, fkd_keypoint* drec,
               long long cap, uint32_t* doff, uint8_t* masks, cudaMemcpyKind mask_kind, int parts = 1) {
  const int per_part = (T + parts - 1) / parts;
  int slot = 0, next_part = 0;
  for (int k0 = 0; k0 < T;) {
    if (parts > 1 && k0 == next_part * per_part) {
      CK(cudaStreamWaitEvent(s->st, s->part_done[next_part], 0));
      ++next_part;
    }
    const int n = parts > 1 ? std::min(per_part, T - k0) : T;
    int rc = run_batch(s, dframes + (long long)k0 * dstride, dpitch, dstride, n, drec, cap, doff + k0, slot, k0 == 0);
    if (rc) return rc;
    if (masks)
      CK(cudaMemcpyAsync(masks + (size_t)k0 * s->g.NB, s->s.mask, (size_t)n * s->g.NB, mask_kind, s->st));
    slot ^= 1;
    k0 += n;
  }
  s->have_frame_result = false;
  return FKD_OK;
}

void reset_history(fkd_stream* s) {
  s->frame = 0;
  s->prev = nullptr;
  s->prev_pitch = 0;
  s->have_frame_result = false;
  s->last_mask = nullptr;
}

// Check a launch shape and turn it into the kernel's launch arguments.
int resolve_launch(const fkd_launch_config* c, DetLaunch* dl) {
  if (!c) return fail(FKD_E_ARG, "launch config is NULL");
  int shape = -1;
  for (int k = 0; k < kDetShapes; ++k)
    if (c->tile_h == kDetTH[k]) shape = k;
  if (shape < 0) return fail(FKD_E_ARG, "tile_h %d: use 8, 16 or 24", c->tile_h);
  if (c->warps_per_cta != 4 && c->warps_per_cta != 8)
    return fail(FKD_E_ARG, "warps_per_cta %d: use 4 or 8", c->warps_per_cta);
  const int fit = detect_ctas_per_sm(shape, c->warps_per_cta);
  if (c->ctas_per_sm < 1 || c->ctas_per_sm > fit)
    return fail(FKD_E_ARG, "ctas_per_sm %d outside 1..%d for tile_h %d, %d warps", c->ctas_per_sm, fit, c->tile_h,
                c->warps_per_cta);
  dl->shape = shape;
  dl->warps = c->warps_per_cta;
  dl->grid = c->ctas_per_sm * sm_count();
  return FKD_OK;
}

fkd_launch_config default_launch() {
  fkd_launch_config c{};
  c.tile_h = kDetTH[kDetDefaultShape];
  c.warps_per_cta = kDetMaxThreads / 32;
  c.ctas_per_sm = std::max(1, detect_ctas_per_sm(kDetDefaultShape, c.warps_per_cta));
  return c;
}

// Point the stream's tables at the tiles of `dl.shape` (no pending work may
// still use the stream's work list).
void apply_launch(fkd_stream* s, const fkd_launch_config& c, const DetLaunch& dl) {
  s->lc = c;
  s->dl = dl;
  s->g.det_shape = dl.shape;
  s->g.n_tiles = s->n_tiles_shape[dl.shape];
  s->tiles = s->tile_shape[dl.shape];
}

// Every candidate shape of the autotuner, the current one first: a later
// candidate wins only when it is faster by more than the margin, so that
// near-ties keep the current shape instead of following timing noise.
constexpr float kTuneMargin = 0.98f;
std::vector<fkd_launch_config> launch_candidates(const fkd_launch_config& current) {
  std::vector<fkd_launch_config> v{current};
  for (int k = 0; k < kDetShapes; ++k)
    for (int warps = 4; warps <= 8; warps += 4) {
      const int fit = detect_ctas_per_sm(k, warps);
      for (int c = 1; c <= fit; ++c)
        if (kDetTH[k] != current.tile_h || warps != current.warps_per_cta || c != current.ctas_per_sm)
          v.push_back(fkd_launch_config{kDetTH[k], warps, c});
    }
  return v;
}

bool is_pinned(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

}  // namespace

extern "C" {

const char* fkd_last_error(void) { return g_err.c_str(); }

int fkd_params_default(fkd_params* p) {
  if (!p) return fail(FKD_E_ARG, "params is NULL");
  std::memset(p, 0, sizeof *p);
  p->version = FKD_VERSION;
  p->N_r = 8;
  p->N_c = 8;
  p->T_I = 4;
  p->T_H = 1;
  p->O = 1;
  p->intra = 0;
  p->t = 20;
  p->n = 9;
  p->mask_mode = FKD_MASK_ID;
  p->mask_layer = 0;
  p->K_max = 65536;
  p->T_max = 1;
  p->nms_scale = 0;
  return FKD_OK;
}

int fkd_create_stream(const fkd_params* p, int W, int H, void* cuda_stream, fkd_stream** out) {
  if (!out) return fail(FKD_E_ARG, "out is NULL");
  *out = nullptr;
  int rc = validate(p, W, H);
  if (rc) return rc;
  fkd_stream* s = new (std::nothrow) fkd_stream();
  if (!s) return fail(FKD_E_ARG, "out of host memory");
  s->p = *p;
  s->st = static_cast<cudaStream_t>(cuda_stream);
  if ((rc = build_geometry(s, W, H)) || (rc = allocate_state(s))) {
    s->release();
    delete s;
    return rc;
  }
  s->staging_pitch = round_up(W, 16);
  {
    const fkd_launch_config c = default_launch();
    DetLaunch dl{};
    if ((rc = resolve_launch(&c, &dl))) {
      s->release();
      delete s;
      return rc;
    }
    apply_launch(s, c, dl);
  }
  *out = s;
  return FKD_OK;
}

int fkd_destroy_stream(fkd_stream* s) {
  if (!s) return FKD_OK;
  cudaStreamSynchronize(s->st);
  s->release();
  delete s;
  return FKD_OK;
}

int fkd_num_layers(const fkd_stream* s, int* L) {
  if (!s || !L) return fail(FKD_E_ARG, "NULL argument");
  *L = s->g.L;
  return FKD_OK;
}

int fkd_layer_info(const fkd_stream* s, int layer, int* w, int* h, int* S) {
  if (!s) return fail(FKD_E_ARG, "stream is NULL");
  if (layer < 0 || layer >= s->g.L) return fail(FKD_E_ARG, "layer %d outside 0..%d", layer, s->g.L - 1);
  if (w) *w = s->g.layer[layer].w;
  if (h) *h = s->g.layer[layer].h;
  if (S) *S = s->g.layer[layer].S;
  return FKD_OK;
}

int fkd_push_frames(fkd_stream* s, const uint8_t* frames, size_t pitch, size_t frame_stride, int T,
                    int on_device, fkd_keypoint* out, size_t cap, uint32_t* offsets, uint8_t* masks,
                    int out_on_device) {
  if (!s || !frames || !offsets || (!out && cap > 0)) return fail(FKD_E_ARG, "NULL argument");
  const Geometry& g = s->g;
  if (T < 1 || T > s->p.T_max) return fail(FKD_E_ARG, "T=%d outside 1..T_max=%d", T, s->p.T_max);
  if (pitch < (size_t)g.W || pitch > (1u << 30)) return fail(FKD_E_ARG, "pitch %zu < W=%d", pitch, g.W);
  if (T > 1 && frame_stride < pitch * (size_t)g.H) return fail(FKD_E_ARG, "frame_stride too small");
  if (cap > 0xffffffffull) return fail(FKD_E_ARG, "cap must fit in 32 bits");

  // 1. frames to device memory
  int parts = 1;
  const uint8_t* dframes = frames;
  int dpitch = (int)pitch;
  long long dstride = (long long)frame_stride;
  if (!on_device) {
    uint8_t*& buf = s->staging[s->staging_next];
    if (!buf) {
      int rc = s->alloc(&buf, (size_t)(s->staging_pitch * g.H * s->p.T_max));
      if (rc) return rc;
    }
    const bool back_to_back = T == 1 || frame_stride == pitch * (size_t)g.H;
    if (back_to_back && T >= 32 && !s->copy_st) {
      // first large host batch: a stream for the uploads, so that they
      // overlap the kernels of the frames before them
      cudaError_t e = cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking);
      for (int i = 0; i < fkd_stream::kParts && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&s->part_done[i], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->staging_free, cudaEventDisableTiming);
      if (e != cudaSuccess) return fail(FKD_E_CUDA, "upload stream setup failed: %s", cudaGetErrorString(e));
    }
    if (back_to_back && T >= 32) {
      // upload in parts on the copy stream, each part's kernels starting as
      // soon as it has arrived (after earlier work is done with the buffer)
      parts = fkd_stream::kParts;
      const int per_part = (T + parts - 1) / parts;
      CK(cudaEventRecord(s->staging_free, s->st));
      CK(cudaStreamWaitEvent(s->copy_st, s->staging_free, 0));
      for (int i = 0; i < parts; ++i) {
        const int k0 = i * per_part, k1 = std::min(T, k0 + per_part);
        if (k1 > k0)
          CK(cudaMemcpy2DAsync(buf + (long long)k0 * s->staging_pitch * g.H, s->staging_pitch,
                               frames + (size_t)k0 * frame_stride, pitch, g.W, (size_t)(k1 - k0) * g.H,
                               cudaMemcpyHostToDevice, s->copy_st));
        CK(cudaEventRecord(s->part_done[i], s->copy_st));
      }
    } else if (back_to_back) {
      // the frames' rows follow one another: one copy of T * H rows
      CK(cudaMemcpy2DAsync(buf, s->staging_pitch, frames, pitch, g.W, (size_t)T * g.H, cudaMemcpyHostToDevice,
                           s->st));
    } else {
      for (int k = 0; k < T; ++k)
        CK(cudaMemcpy2DAsync(buf + (long long)k * s->staging_pitch * g.H, s->staging_pitch,
                             frames + (size_t)k * frame_stride, pitch, g.W, g.H, cudaMemcpyHostToDevice,
                             s->st));
    }
    dframes = buf;
    dpitch = (int)s->staging_pitch;
    dstride = s->staging_pitch * g.H;
    s->staging_next ^= 1;
  }

  // 2. where the records go
  fkd_keypoint* drec = out;
  uint32_t* doff = offsets;
  if (!out_on_device) {
    if ((long long)cap > s->host_out_cap) {
      if (s->host_out) {
        CK(cudaStreamSynchronize(s->st));
        s->free_one(s->host_out);
        s->host_out_cap = 0;
      }
      fkd_keypoint* nb = nullptr;
      int rc = s->alloc(&nb, cap);
      if (rc) return rc;
      s->host_out = nb;
      s->host_out_cap = (long long)cap;
    }
    drec = s->host_out;
    doff = s->host_offsets;
  }

  // descriptors: one per record the call can write
  if (s->desc_D && (long long)cap > s->desc_cap) {
    CK(cudaStreamSynchronize(s->st));
    s->free_one(s->desc);
    s->desc_cap = 0;
    int rc = s->alloc(&s->desc, cap * (size_t)(s->desc_D / 32));
    if (rc) return rc;
    s->desc_cap = (long long)cap;
  }

  // 3. the batch
  int rc = run_frames(s, dframes, dpitch, dstride, T, drec, (long long)cap, doff, masks,
                      out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, parts);
  if (rc) return rc;

  if (out_on_device) return FKD_OK;
  CK(cudaMemcpyAsync(offsets, doff, (size_t)(T + 1) * 4, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  const long long total = offsets[T];
  const long long ncopy = std::min<long long>(total, (long long)cap);
  if (ncopy > 0)
    CK(cudaMemcpyAsync(out, drec, (size_t)ncopy * sizeof(fkd_keypoint), cudaMemcpyDeviceToHost, s->st));
  int ov = 0;
  CK(cudaMemcpyAsync(&ov, s->s.overflow, 4, cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemsetAsync(s->s.overflow, 0, 4, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (ov & 2) return fail(FKD_E_CUDA, "a pyramid tile copy did not complete");
  if (total > (long long)cap || ov)
    return fail(FKD_E_CAPACITY, "batch produced %lld keypoints, cap %zu", total, cap);
  return FKD_OK;
}

int fkd_push_frame(fkd_stream* s, const uint8_t* frame, size_t pitch, int on_device) {
  if (!s || !frame) return fail(FKD_E_ARG, "NULL argument");
  const Geometry& g = s->g;
  if (pitch < (size_t)g.W) return fail(FKD_E_ARG, "pitch %zu < W=%d", pitch, g.W);
  const uint8_t* dframe = frame;
  int dpitch = (int)pitch;
  if (!on_device) {
    uint8_t*& buf = s->staging[s->staging_next];
    if (!buf) {
      int rc = s->alloc(&buf, (size_t)(s->staging_pitch * g.H * s->p.T_max));
      if (rc) return rc;
    }
    CK(cudaMemcpy2DAsync(buf, s->staging_pitch, frame, pitch, g.W, g.H, cudaMemcpyHostToDevice, s->st));
    if (!is_pinned(frame)) CK(cudaStreamSynchronize(s->st));
    dframe = buf;
    dpitch = (int)s->staging_pitch;
    s->staging_next ^= 1;
  }
  int rc = run_batch(s, dframe, dpitch, (long long)dpitch * g.H, 1, s->rec, s->p.K_max, s->rec_offsets,
                     0, true);
  if (rc) return rc;
  s->have_frame_result = true;
  return FKD_OK;
}

int fkd_get_keypoints(fkd_stream* s, fkd_keypoint* out, size_t cap, size_t* n_out) {
  if (!s || !n_out || (!out && cap > 0)) return fail(FKD_E_ARG, "NULL argument");
  if (!s->have_frame_result) return fail(FKD_E_STATE, "no frame pushed with fkd_push_frame");
  uint32_t off[2];
  CK(cudaMemcpyAsync(off, s->rec_offsets, 8, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  const size_t n = off[1] - off[0];
  *n_out = n;
  if (n > (size_t)s->p.K_max) {
    CK(cudaMemset(s->s.overflow, 0, 4));
    return fail(FKD_E_CAPACITY, "frame has %zu keypoints > K_max %d", n, s->p.K_max);
  }
  if (n > cap) return fail(FKD_E_CAPACITY, "frame has %zu keypoints > cap %zu", n, cap);
  if (n) CK(cudaMemcpy(out, s->rec, n * sizeof(fkd_keypoint), cudaMemcpyDeviceToHost));
  return FKD_OK;
}

int fkd_get_mask(fkd_stream* s, uint8_t* out) {
  if (!s || !out) return fail(FKD_E_ARG, "NULL argument");
  if (!s->last_mask) return fail(FKD_E_STATE, "no frame pushed yet");
  CK(cudaMemcpyAsync(out, s->last_mask, (size_t)s->g.NB, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  return FKD_OK;
}

int fkd_get_pixel_mask(fkd_stream* s, int layer, uint8_t* out) {
  if (!s || !out) return fail(FKD_E_ARG, "NULL argument");
  if (!s->s.pmask) return fail(FKD_E_ARG, "the stream does not use FKD_MASK_IDP");
  if (layer < 0 || layer >= s->g.L) return fail(FKD_E_ARG, "layer %d outside 0..%d", layer, s->g.L - 1);
  if (!s->last_mask) return fail(FKD_E_STATE, "no frame pushed yet");
  const LayerGeom& lg = s->g.layer[layer];
  std::vector<uint32_t> words((size_t)lg.wpr * lg.h);
  const long long last = s->last_frame_slot;
  if (!words.empty())
    CK(cudaMemcpyAsync(words.data(), s->s.pmask + last * s->g.bit_words + lg.bit_off, words.size() * 4,
                       cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  for (int y = 0; y < lg.h; ++y)
    for (int x = 0; x < lg.w; ++x) out[(size_t)y * lg.w + x] = (words[(size_t)y * lg.wpr + x / 32] >> (x % 32)) & 1u;
  return FKD_OK;
}

int fkd_synchronize(fkd_stream* s) {
  if (!s) return fail(FKD_E_ARG, "stream is NULL");
  int ov = 0;
  CK(cudaMemcpyAsync(&ov, s->s.overflow, 4, cudaMemcpyDeviceToHost, s->st));
  CK(cudaMemsetAsync(s->s.overflow, 0, 4, s->st));
  CK(cudaStreamSynchronize(s->st));
  if (ov & 2) return fail(FKD_E_CUDA, "a pyramid tile copy did not complete");
  if (ov) return fail(FKD_E_CAPACITY, "an asynchronous batch dropped records past its capacity");
  return FKD_OK;
}

int fkd_frame_count(const fkd_stream* s, int64_t* n) {
  if (!s || !n) return fail(FKD_E_ARG, "NULL argument");
  *n = s->frame;
  return FKD_OK;
}

int fkd_reset_stream(fkd_stream* s) {
  if (!s) return fail(FKD_E_ARG, "stream is NULL");
  CK(cudaStreamSynchronize(s->st));
  reset_history(s);
  return FKD_OK;
}

int fkd_set_descriptor(fkd_stream* s, const int8_t* pattern, int D) {
  if (!s) return fail(FKD_E_ARG, "stream is NULL");
  if (D != 0) {
    if (!pattern) return fail(FKD_E_ARG, "pattern is NULL");
    if (D < 32 || D > FKD_DESC_MAX_BITS || D % 32)
      return fail(FKD_E_ARG, "D=%d: a multiple of 32 in 32..%d", D, FKD_DESC_MAX_BITS);
    for (int i = 0; i < 4 * D; ++i)
      if (pattern[i] < -FKD_DESC_RADIUS || pattern[i] > FKD_DESC_RADIUS)
        return fail(FKD_E_ARG, "pattern offset %d of pair %d outside +-%d", pattern[i], i / 4, FKD_DESC_RADIUS);
  }
  CK(cudaStreamSynchronize(s->st));
  reset_history(s);
  s->desc_ready = false;
  s->desc_D = 0;
  s->free_one(s->desc_pattern);
  s->free_one(s->desc);
  s->desc_cap = 0;
  for (int i = 0; i < 2; ++i) {
    s->free_one(s->keep_rec[i]);
    s->free_one(s->keep_desc[i]);
    s->free_one(s->keep_row[i]);
  }
  s->free_one(s->desc_rows);
  s->free_one(s->keep_n);
  s->free_one(s->desc_count);
  if (D == 0) return FKD_OK;
  const size_t words = (size_t)D / 32, K = (size_t)s->p.K_max;
  int rc;
  if ((rc = s->alloc(&s->desc_pattern, (size_t)D * 4)) || (rc = s->alloc(&s->desc, K * words)) ||
      (rc = s->alloc(&s->keep_n, 2)) || (rc = s->alloc(&s->desc_count, 2)))
    return rc;
  const LayerGeom& top = s->g.layer[s->g.L - 1];
  s->rows = top.row_off + top.h;
  for (int i = 0; i < 2; ++i) {
    if ((rc = s->alloc(&s->keep_rec[i], K)) || (rc = s->alloc(&s->keep_desc[i], K * words)) ||
        (rc = s->alloc(&s->keep_row[i], (size_t)s->rows + 1)))
      return rc;
    CK(cudaMemset(s->keep_row[i], 0, ((size_t)s->rows + 1) * 4));
  }
  if ((rc = s->alloc(&s->desc_rows, (size_t)s->p.T_max * s->rows))) return rc;
  s->desc_cap = (long long)K;
  CK(cudaMemcpy(s->desc_pattern, pattern, (size_t)D * 4, cudaMemcpyHostToDevice));
  CK(cudaMemset(s->keep_n, 0, 8));
  CK(cudaMemset(s->desc_count, 0, 8));
  s->desc_D = D;
  return FKD_OK;
}

int fkd_get_descriptors(fkd_stream* s, uint8_t* out, size_t cap, size_t* n_out, int out_on_device) {
  if (!s || !n_out || (!out && cap > 0)) return fail(FKD_E_ARG, "NULL argument");
  if (!s->desc_D) return fail(FKD_E_STATE, "description is off (fkd_set_descriptor)");
  if (!s->desc_ready) return fail(FKD_E_STATE, "no frame pushed since fkd_set_descriptor");
  uint32_t n = 0;
  CK(cudaMemcpyAsync(&n, s->desc_count, 4, cudaMemcpyDeviceToHost, s->st));
  CK(cudaStreamSynchronize(s->st));
  *n_out = n;
  const size_t bytes = (size_t)s->desc_D / 8;
  const size_t ncopy = std::min<size_t>(n, cap);
  if (ncopy)
    CK(cudaMemcpyAsync(out, s->desc, ncopy * bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       s->st));
  CK(cudaStreamSynchronize(s->st));
  if (n > cap && out) return fail(FKD_E_CAPACITY, "%u descriptors > cap %zu", n, cap);
  return FKD_OK;
}

int fkd_get_launch_config(const fkd_stream* s, fkd_launch_config* out) {
  if (!s || !out) return fail(FKD_E_ARG, "NULL argument");
  *out = s->lc;
  return FKD_OK;
}

int fkd_set_launch_config(fkd_stream* s, const fkd_launch_config* c) {
  if (!s) return fail(FKD_E_ARG, "stream is NULL");
  DetLaunch dl{};
  int rc = resolve_launch(c, &dl);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s->st));
  apply_launch(s, *c, dl);
  return FKD_OK;
}

int fkd_autotune(fkd_stream* s, const uint8_t* frames, size_t pitch, size_t frame_stride, int T, int reps,
                 fkd_launch_config* best, float* best_ms) {
  if (!s || !frames) return fail(FKD_E_ARG, "NULL argument");
  const Geometry& g = s->g;
  if (T < 1 || T > s->p.T_max) return fail(FKD_E_ARG, "T=%d outside 1..T_max=%d", T, s->p.T_max);
  if (pitch < (size_t)g.W || pitch > (1u << 30)) return fail(FKD_E_ARG, "pitch %zu < W=%d", pitch, g.W);
  if (T > 1 && frame_stride < pitch * (size_t)g.H) return fail(FKD_E_ARG, "frame_stride too small");
  if (reps < 1 || reps > 100) return fail(FKD_E_ARG, "reps %d outside 1..100", reps);
  CK(cudaStreamSynchronize(s->st));
  const bool prof = s->profiling;
  s->profiling = false;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  CK(cudaEventCreate(&ev[0]));
  CK(cudaEventCreate(&ev[1]));
  // records go to the per-frame result buffer (K_max of them; the rest are
  // dropped), offsets to the host-output offsets
  fkd_launch_config win = s->lc;
  float win_ms = -1.f;
  int rc = FKD_OK;
  for (const fkd_launch_config& c : launch_candidates(s->lc)) {
    DetLaunch dl{};
    if ((rc = resolve_launch(&c, &dl))) break;
    apply_launch(s, c, dl);
    float best_c = -1.f;
    for (int r = 0; r <= reps && rc == FKD_OK; ++r) {
      reset_history(s);
      cudaEventRecord(ev[0], s->st);
      rc = run_frames(s, frames, (int)pitch, (long long)frame_stride, T, s->rec, s->p.K_max, s->host_offsets,
                      nullptr, cudaMemcpyDeviceToDevice);
      cudaEventRecord(ev[1], s->st);
      cudaError_t e = cudaEventSynchronize(ev[1]);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (e != cudaSuccess && rc == FKD_OK) rc = fail(FKD_E_CUDA, "autotune timing failed: %s", cudaGetErrorString(e));
      if (r > 0 && (best_c < 0.f || ms < best_c)) best_c = ms;
    }
    if (rc) break;
    if (win_ms < 0.f || best_c < kTuneMargin * win_ms) {
      win_ms = best_c;
      win = c;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  s->profiling = prof;
  DetLaunch dl{};
  if (resolve_launch(&win, &dl) == FKD_OK) apply_launch(s, win, dl);
  reset_history(s);
  cudaMemsetAsync(s->s.overflow, 0, 4, s->st);
  cudaStreamSynchronize(s->st);
  cudaMemcpy(s->tile_stats_seen, s->s.tile_stats, 16, cudaMemcpyDeviceToHost);  // tuning runs are not profiled
  if (rc) return rc;
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return FKD_OK;
}

int fkd_profile_enable(fkd_stream* s, int on) {
  if (!s) return fail(FKD_E_ARG, "stream is NULL");
  s->profiling = on != 0;
  return FKD_OK;
}

int fkd_profile_read(fkd_stream* s, fkd_profile* out, int reset) {
  if (!s || !out) return fail(FKD_E_ARG, "NULL argument");
  CK(cudaStreamSynchronize(s->st));
  for (auto& pd : s->pending) {
    for (int i = 0; i < FKD_NUM_STAGES; ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, pd.ev[i], pd.ev[i + 1]));
      s->prof.ms[i] += ms;
      if (i != FKD_STAGE_DESCRIBE || pd.described) s->prof.launches[i] += 1;
    }
    s->prof.batches += 1;
    s->prof.frames += (uint64_t)pd.frames;
    for (cudaEvent_t e : pd.ev) s->event_pool.push_back(e);
  }
  s->pending.clear();
  unsigned long long ts[2];
  CK(cudaMemcpy(ts, s->s.tile_stats, 16, cudaMemcpyDeviceToHost));
  s->prof.tiles += ts[0] - s->tile_stats_seen[0];
  s->prof.tile_pixels += ts[1] - s->tile_stats_seen[1];
  s->tile_stats_seen[0] = ts[0];
  s->tile_stats_seen[1] = ts[1];
  *out = s->prof;
  if (reset) s->prof = fkd_profile{};
  return FKD_OK;
}

int fkd_device_keypoints(fkd_stream* s, const fkd_keypoint** records, const uint32_t** count_dev) {
  if (!s || !records || !count_dev) return fail(FKD_E_ARG, "NULL argument");
  if (!s->have_frame_result) return fail(FKD_E_STATE, "no frame pushed with fkd_push_frame");
  *records = s->rec;
  *count_dev = s->rec_offsets + 1;
  return FKD_OK;
}

int fkd_check_build(void) { return FKD_CHECK ? 1 : 0; }

int fkd_check_guards(const fkd_stream* s) {
  if (!s) return fail(FKD_E_ARG, "stream is NULL");
#if FKD_CHECK
  CK(cudaStreamSynchronize(s->st));
  std::vector<unsigned char> band(kGuard);
  for (const auto& a : s->allocs) {
    for (int side = 0; side < 2; ++side) {
      const char* at = static_cast<const char*>(a.first) + (side ? (long long)a.second : -(long long)kGuard);
      CK(cudaMemcpy(band.data(), at, kGuard, cudaMemcpyDeviceToHost));
      for (size_t i = 0; i < kGuard; ++i)
        if (band[i] != kGuardByte)
          return fail(FKD_E_CUDA, "guard band %s an allocation of %zu bytes changed at byte %zu",
                      side ? "after" : "before", a.second, i);
    }
  }
#endif
  return FKD_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ groups

namespace {

struct GroupStream {
  fkd_stream* s = nullptr;  // T_max = 1
  uint8_t* last[2] = {nullptr, nullptr};
  fkd_keypoint* rec1 = nullptr;  // results of odd frames (even frames use the stream's own)
  uint32_t* off1 = nullptr;
  uint32_t* desc1 = nullptr;      // descriptors of odd frames (even frames: the stream's own)
  uint32_t* rows1 = nullptr;      // row starts of odd frames
  size_t bytes = 0;
};

}  // namespace

struct fkd_group {
  int O = 1, intra = 0;
  cudaStream_t st = nullptr;
  std::vector<GroupStream> streams;  // indexed by stream id; s == nullptr once removed
  StreamDev* d_devs = nullptr;
  int devs_cap = 0;
  TickHeader* d_hdr = nullptr;       // followed by kMaxTickItems TickItems
  TickItem* d_items = nullptr;
  unsigned char* h_tick[2] = {nullptr, nullptr};  // pinned copies of header + items
  cudaEvent_t tick_done[2] = {nullptr, nullptr};
  uint32_t* d_work = nullptr;
  long long work_cap = 0;
  uint32_t* d_work_count = nullptr;
  int grid_pyr = 1, grid_small = 1, grid_asm = 1;
  fkd_launch_config lc{};            // detection launch shape of every stream
  DetLaunch dl{};
  bool any_nms_scale = false;        // some stream asked for scale-space suppression
  bool any_describe = false;         // some stream describes its keypoints
  bool use_graph = true;
  bool graph_valid = false;
  int graph_items = 0;               // items copied per tick by the captured graphs
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  long long ticks = 0;
  bool profiling = false;
  std::vector<fkd_stream::Pending> pending;
  std::vector<cudaEvent_t> event_pool;
  fkd_profile prof{};
  unsigned long long tile_seen[2] = {0, 0};

  cudaEvent_t take_event() {
    if (!event_pool.empty()) {
      cudaEvent_t e = event_pool.back();
      event_pool.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void drop_graphs() {
    for (auto& ge : graph)
      if (ge) {
        cudaGraphExecDestroy(ge);
        ge = nullptr;
      }
    graph_valid = false;
  }
};

namespace {

// Tick upload: the header, then the items at a 64-byte aligned offset (they
// hold 8-byte fields that the kernels load directly).
constexpr size_t kItemsOffset = 64;
static_assert(sizeof(TickHeader) <= kItemsOffset, "tick header fits before the items");
static_assert(alignof(TickItem) <= 64 && sizeof(TickItem) % alignof(TickItem) == 0, "aligned items");
constexpr size_t kTickBytes = kItemsOffset + kMaxTickItems * sizeof(TickItem);

StreamDev make_dev(const fkd_stream* s, const GroupStream& gs) {
  uint8_t* const* last = gs.last;
  StreamDev d{};
  d.g = s->g;
  d.tb = Tables{s->colblk, s->rowblk, s->xstart, s->npix, s->tiles, s->chunks, s->wbins, s->wmask, s->rowchunk,
                s->rowcell, s->bincell_off, s->bincell};
  d.s = s->s;
  d.s.dcnt = nullptr;   // detection counts serve keypoint binning in spans of a batch only
  d.p = Params{s->p.T_I, s->p.T_H, s->p.t, s->p.mask_mode, s->p.nms_scale};
  for (int i = 0; i < 2; ++i) {
    d.state_bits[i] = s->state_bits[i];
    d.state_score[i] = s->state_score[i];
    d.state_cnt[i] = s->state_cnt[i];
    d.last[i] = last[i];
  }
  d.rec[0] = s->rec;
  d.rec_offsets[0] = s->rec_offsets;
  d.rec[1] = gs.rec1;
  d.rec_offsets[1] = gs.off1;
  d.K_max = s->p.K_max;
  d.D = s->desc_D;
  d.pattern = s->desc_pattern;
  d.desc[0] = s->desc;
  d.desc[1] = gs.desc1;
  d.row_base[0] = s->desc_rows;
  d.row_base[1] = gs.rows1;
  d.rows = s->rows;
  return d;
}

// The tick's launch sequence: upload of header + items, then the kernels.
int group_launch(fkd_group* G, int b, int n_items, fkd_stream::Pending* pd) {
  auto mark = [&](int i) {
    if (pd) {
      pd->ev[i] = G->take_event();
      cudaEventRecord(pd->ev[i], G->st);
    }
  };
  CK(cudaMemcpyAsync(G->d_hdr, G->h_tick[b], kItemsOffset + (size_t)n_items * sizeof(TickItem),
                     cudaMemcpyHostToDevice, G->st));
  mark(0);
  launch_group_pyramid(G->O, G->intra, G->d_devs, G->d_hdr, G->d_items, G->grid_pyr, G->st);
  mark(1);
  launch_group_mask(G->d_devs, G->d_hdr, G->d_items, G->d_work_count, G->grid_small, G->st);
  mark(2);
  launch_group_worklist(G->d_devs, G->d_hdr, G->d_items, G->d_work, G->d_work_count, G->grid_small, G->st);
  mark(3);
  launch_group_detect(G->d_devs, G->d_items, G->d_work, G->d_work_count, G->dl, G->st);
  // streams without scale-space suppression skip their items inside
  if (G->any_nms_scale)
    launch_group_scale_nms(G->d_devs, G->d_items, G->d_work, G->d_work_count, G->st);
  mark(4);
  launch_group_count(G->d_devs, G->d_hdr, G->d_items, G->grid_asm, G->st);
  mark(5);
  launch_group_emit(G->d_devs, G->d_hdr, G->d_items, G->grid_asm, G->st);
  mark(6);
  // streams that do not describe skip their items inside
  if (G->any_describe) launch_group_describe(G->d_devs, G->d_hdr, G->d_items, G->st);
  mark(7);
  CK(cudaGetLastError());
  return FKD_OK;
}

int group_capture(fkd_group* G, int n_items) {
  G->drop_graphs();
  for (int b = 0; b < 2; ++b) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(G->st, cudaStreamCaptureModeThreadLocal));
    int rc = group_launch(G, b, n_items, nullptr);
    cudaError_t e = cudaStreamEndCapture(G->st, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      return rc;
    }
    if (e != cudaSuccess) return fail(FKD_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&G->graph[b], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(FKD_E_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  G->graph_valid = true;
  G->graph_items = n_items;
  return FKD_OK;
}

fkd_stream* group_member(fkd_group* G, int id) {
  if (!G || id < 0 || id >= (int)G->streams.size()) return nullptr;
  return G->streams[id].s;
}

}  // namespace

extern "C" {

int fkd_group_create(int O, int intra, void* cuda_stream, fkd_group** out) {
  if (!out) return fail(FKD_E_ARG, "out is NULL");
  *out = nullptr;
  if (O < 1 || O > 6 || (intra != 0 && intra != 1)) return fail(FKD_E_ARG, "O must be 1..6, intra 0 or 1");
  fkd_group* G = new (std::nothrow) fkd_group();
  if (!G) return fail(FKD_E_ARG, "out of host memory");
  G->O = O;
  G->intra = intra;
  G->st = static_cast<cudaStream_t>(cuda_stream);
  G->use_graph = G->st != nullptr;  // the legacy default stream cannot be captured
  auto bail = [&](int rc) {
    fkd_group_destroy(G);
    return rc;
  };
  cudaError_t e;
  if ((e = cudaMalloc(&G->d_hdr, kTickBytes)) != cudaSuccess ||
      (e = cudaMalloc(&G->d_work_count, 4)) != cudaSuccess ||
      (e = cudaHostAlloc(&G->h_tick[0], kTickBytes, cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaHostAlloc(&G->h_tick[1], kTickBytes, cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&G->tick_done[0], cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&G->tick_done[1], cudaEventDisableTiming)) != cudaSuccess)
    return bail(fail(FKD_E_CUDA, "group allocation failed: %s", cudaGetErrorString(e)));
  G->d_items = reinterpret_cast<TickItem*>(reinterpret_cast<unsigned char*>(G->d_hdr) + kItemsOffset);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  G->grid_pyr = group_pyramid_grid(O, intra);
  G->lc = default_launch();
  if (int rc = resolve_launch(&G->lc, &G->dl)) return bail(rc);
  G->grid_small = sms * 8;
  G->grid_asm = sms * 8;
  *out = G;
  return FKD_OK;
}

int fkd_group_destroy(fkd_group* G) {
  if (!G) return FKD_OK;
  cudaStreamSynchronize(G->st);
  G->drop_graphs();
  for (auto& gs : G->streams)
    if (gs.s) fkd_destroy_stream(gs.s);
  cudaFree(G->d_devs);
  cudaFree(G->d_hdr);
  cudaFree(G->d_work);
  cudaFree(G->d_work_count);
  for (int b = 0; b < 2; ++b) {
    if (G->h_tick[b]) cudaFreeHost(G->h_tick[b]);
    if (G->tick_done[b]) cudaEventDestroy(G->tick_done[b]);
  }
  for (auto& pd : G->pending)
    for (cudaEvent_t e : pd.ev) cudaEventDestroy(e);
  for (cudaEvent_t e : G->event_pool) cudaEventDestroy(e);
  delete G;
  return FKD_OK;
}

int fkd_group_add_stream(fkd_group* G, const fkd_params* p, int W, int H, int* stream_id, size_t* bytes) {
  if (!G || !p || !stream_id) return fail(FKD_E_ARG, "NULL argument");
  if (p->O != G->O || p->intra != G->intra)
    return fail(FKD_E_ARG, "stream O/intra (%d/%d) differ from the group's (%d/%d)", p->O, p->intra, G->O, G->intra);
  if (p->mask_mode == FKD_MASK_IDP) return fail(FKD_E_ARG, "FKD_MASK_IDP is for single streams, not groups");
  CK(cudaStreamSynchronize(G->st));
  fkd_params q = *p;
  q.T_max = 1;
  fkd_stream* s = nullptr;
  int rc = fkd_create_stream(&q, W, H, G->st, &s);
  if (rc) return rc;
  GroupStream gs;
  gs.s = s;
  // copies of the last two frames, for change sums on c_0 (coarser mask
  // layers keep their own copy of the layer)
  const size_t lbytes = (size_t)s->g.layer[0].pitch * (size_t)H;
  const bool c0_sums = s->p.mask_mode == FKD_MASK_ID && s->g.mask_layer == 0;
  for (int i = 0; i < 2 && c0_sums; ++i)
    if ((rc = s->alloc(&gs.last[i], lbytes))) {
      fkd_destroy_stream(s);
      return rc;
    }
  if ((rc = s->alloc(&gs.rec1, (size_t)s->p.K_max)) || (rc = s->alloc(&gs.off1, 2))) {
    fkd_destroy_stream(s);
    return rc;
  }
  gs.bytes = s->bytes_held;
  apply_launch(s, G->lc, G->dl);
  if (s->p.nms_scale && !G->any_nms_scale) {
    G->any_nms_scale = true;
    G->drop_graphs();  // the captured ticks lack the suppression pass
  }
  const int id = (int)G->streams.size();
  // device descriptors (grow: the captured graphs hold the old pointer)
  if (id >= G->devs_cap) {
    const int cap = std::max(16, 2 * G->devs_cap);
    StreamDev* nd = nullptr;
    cudaError_t e = cudaMalloc(&nd, (size_t)cap * sizeof(StreamDev));
    if (e != cudaSuccess) {
      fkd_destroy_stream(s);
      return fail(FKD_E_CUDA, "cudaMalloc failed: %s", cudaGetErrorString(e));
    }
    if (G->d_devs) {
      CK(cudaMemcpy(nd, G->d_devs, (size_t)G->devs_cap * sizeof(StreamDev), cudaMemcpyDeviceToDevice));
      cudaFree(G->d_devs);
    }
    G->d_devs = nd;
    G->devs_cap = cap;
    G->drop_graphs();
  }
  const StreamDev d = make_dev(s, gs);
  CK(cudaMemcpy(G->d_devs + id, &d, sizeof d, cudaMemcpyHostToDevice));
  // the tick's active-tile list holds at most the tiles of all live streams
  long long need = 0;
  for (auto& o : G->streams)
    if (o.s) need += o.s->n_tiles_max;
  need += s->n_tiles_max;
  if (need > G->work_cap) {
    const long long cap = std::max(need, 2 * G->work_cap);
    cudaFree(G->d_work);
    G->d_work = nullptr;
    cudaError_t e = cudaMalloc(&G->d_work, (size_t)cap * 4);
    if (e != cudaSuccess) {
      fkd_destroy_stream(s);
      G->work_cap = 0;
      return fail(FKD_E_CUDA, "cudaMalloc failed: %s", cudaGetErrorString(e));
    }
    G->work_cap = cap;
    G->drop_graphs();
  }
  G->streams.push_back(gs);
  *stream_id = id;
  if (bytes) *bytes = gs.bytes;
  return FKD_OK;
}

int fkd_group_remove_stream(fkd_group* G, int id) {
  fkd_stream* s = group_member(G, id);
  if (!s) return fail(FKD_E_ARG, "unknown stream id %d", id);
  CK(cudaStreamSynchronize(G->st));
  fkd_destroy_stream(s);
  G->streams[id].s = nullptr;
  return FKD_OK;
}

int fkd_group_use_graph(fkd_group* G, int on) {
  if (!G) return fail(FKD_E_ARG, "group is NULL");
  G->use_graph = on && G->st != nullptr;
  return FKD_OK;
}

int fkd_group_tick(fkd_group* G, int n, const int* ids, const uint8_t* const* frames, const size_t* pitches) {
  if (!G || n < 0 || (n > 0 && (!ids || !frames || !pitches))) return fail(FKD_E_ARG, "NULL argument");
  if (n > kMaxTickItems) return fail(FKD_E_ARG, "more than %d streams in one tick", kMaxTickItems);
  if (n == 0) return FKD_OK;
  const int b = (int)(G->ticks & 1);
  CK(cudaEventSynchronize(G->tick_done[b]));  // the pinned buffer's previous upload is done
  TickHeader* h = reinterpret_cast<TickHeader*>(G->h_tick[b]);
  TickItem* items = reinterpret_cast<TickItem*>(G->h_tick[b] + kItemsOffset);
  int pyr = 0, bins = 0, tiles = 0, chunks = 0;
  for (int i = 0; i < n; ++i) {
    fkd_stream* s = group_member(G, ids[i]);
    if (!s) return fail(FKD_E_ARG, "unknown stream id %d", ids[i]);
    if (!frames[i] || pitches[i] < (size_t)s->g.W || pitches[i] > (1u << 30))
      return fail(FKD_E_ARG, "bad frame or pitch for stream %d", ids[i]);
    for (int j = 0; j < i; ++j)
      if (ids[j] == ids[i]) return fail(FKD_E_ARG, "stream %d twice in one tick", ids[i]);
    TickItem& it = items[i];
    it.sid = ids[i];
    it.state_cur = s->state_cur;
    it.frame_index = s->frame;
    it.frame = frames[i];
    it.pitch = (int)pitches[i];
    it.pyr_base = pyr;
    it.bin_base = bins;
    it.tile_base = tiles;
    it.chunk_base = chunks;
    pyr += s->g.pyr_tiles_x * s->g.pyr_tiles_y;
    bins += s->g.NB;
    tiles += s->g.n_tiles;
    chunks += s->g.n_chunks;
  }
  if ((long long)tiles > G->work_cap) return fail(FKD_E_ARG, "tick larger than the group's work list");
  h->n_items = n;
  h->total_pyr = pyr;
  h->total_bins = bins;
  h->total_tiles = tiles;
  h->total_chunks = chunks;

  if (G->profiling) {
    fkd_stream::Pending pd{};
    int rc = group_launch(G, b, n, &pd);
    if (rc) return rc;
    pd.frames = n;
    G->pending.push_back(pd);
  } else if (G->use_graph) {
    int live = 0;
    for (auto& gs : G->streams) live += gs.s ? 1 : 0;
    if (!G->graph_valid || G->graph_items < n) {
      int rc = group_capture(G, std::max(n, live));
      if (rc) return rc;
    }
    CK(cudaGraphLaunch(G->graph[b], G->st));
  } else {
    int rc = group_launch(G, b, n, nullptr);
    if (rc) return rc;
  }
  CK(cudaEventRecord(G->tick_done[b], G->st));
  if (int rc = check_after(G->st)) return rc;
  G->ticks += 1;
  for (int i = 0; i < n; ++i) {
    fkd_stream* s = G->streams[ids[i]].s;
    s->state_cur ^= 1;
    s->frame += 1;
    s->have_frame_result = true;
    s->last_mask = s->s.mask;
  }
  return FKD_OK;
}

int fkd_group_synchronize(fkd_group* G) {
  if (!G) return fail(FKD_E_ARG, "group is NULL");
  CK(cudaStreamSynchronize(G->st));
  return FKD_OK;
}

namespace {
// Result buffers of the stream's last processed frame.
int group_last_result(fkd_group* G, int id, fkd_stream** s, const fkd_keypoint** rec, const uint32_t** off) {
  *s = group_member(G, id);
  if (!*s) return fail(FKD_E_ARG, "unknown stream id %d", id);
  if ((*s)->frame == 0) return fail(FKD_E_STATE, "stream %d has no frame yet", id);
  const bool odd = (((*s)->frame - 1) & 1) != 0;
  *rec = odd ? G->streams[id].rec1 : (*s)->rec;
  *off = odd ? G->streams[id].off1 : (*s)->rec_offsets;
  return FKD_OK;
}
}  // namespace

int fkd_group_get_keypoints(fkd_group* G, int id, fkd_keypoint* out, size_t cap, size_t* n_out) {
  if (!n_out || (!out && cap > 0)) return fail(FKD_E_ARG, "NULL argument");
  fkd_stream* s;
  const fkd_keypoint* rec;
  const uint32_t* off;
  int rc = group_last_result(G, id, &s, &rec, &off);
  if (rc) return rc;
  uint32_t o[2];
  CK(cudaMemcpyAsync(o, off, 8, cudaMemcpyDeviceToHost, G->st));
  CK(cudaStreamSynchronize(G->st));
  const size_t n = o[1] - o[0];
  *n_out = n;
  if (n > (size_t)s->p.K_max) return fail(FKD_E_CAPACITY, "frame has %zu keypoints > K_max %d", n, s->p.K_max);
  if (n > cap) return fail(FKD_E_CAPACITY, "frame has %zu keypoints > cap %zu", n, cap);
  if (n) CK(cudaMemcpy(out, rec, n * sizeof(fkd_keypoint), cudaMemcpyDeviceToHost));
  return FKD_OK;
}

int fkd_group_get_mask(fkd_group* G, int id, uint8_t* out) {
  fkd_stream* s = group_member(G, id);
  if (!s) return fail(FKD_E_ARG, "unknown stream id %d", id);
  return fkd_get_mask(s, out);
}

int fkd_group_device_keypoints(fkd_group* G, int id, const fkd_keypoint** records, const uint32_t** count_dev) {
  if (!records || !count_dev) return fail(FKD_E_ARG, "NULL argument");
  fkd_stream* s;
  const fkd_keypoint* rec;
  const uint32_t* off;
  int rc = group_last_result(G, id, &s, &rec, &off);
  if (rc) return rc;
  *records = rec;
  *count_dev = off + 1;
  return FKD_OK;
}

int fkd_group_set_descriptor(fkd_group* G, int id, const int8_t* pattern, int D) {
  fkd_stream* s = group_member(G, id);
  if (!s) return fail(FKD_E_ARG, "unknown stream id %d", id);
  if (s->frame != 0) return fail(FKD_E_STATE, "set the descriptor of stream %d before its first tick", id);
  CK(cudaStreamSynchronize(G->st));
  GroupStream& gs = G->streams[id];
  s->free_one(gs.desc1);
  s->free_one(gs.rows1);
  int rc = fkd_set_descriptor(s, pattern, D);  // validates, allocates the even frames' buffers
  if (rc) return rc;
  if (D) {
    if ((rc = s->alloc(&gs.desc1, (size_t)s->p.K_max * (size_t)(D / 32))) ||
        (rc = s->alloc(&gs.rows1, (size_t)s->rows + 1)))
      return rc;
    if (!G->any_describe) {
      G->any_describe = true;
      G->drop_graphs();  // the captured ticks lack the description pass
    }
  }
  gs.bytes = s->bytes_held;
  const StreamDev d = make_dev(s, gs);
  CK(cudaMemcpy(G->d_devs + id, &d, sizeof d, cudaMemcpyHostToDevice));
  return FKD_OK;
}

int fkd_group_get_descriptors(fkd_group* G, int id, uint8_t* out, size_t cap, size_t* n_out, int out_on_device) {
  if (!n_out || (!out && cap > 0)) return fail(FKD_E_ARG, "NULL argument");
  fkd_stream* s;
  const fkd_keypoint* rec;
  const uint32_t* off;
  int rc = group_last_result(G, id, &s, &rec, &off);
  if (rc) return rc;
  if (!s->desc_D) return fail(FKD_E_STATE, "stream %d does not describe (fkd_group_set_descriptor)", id);
  uint32_t o[2];
  CK(cudaMemcpyAsync(o, off, 8, cudaMemcpyDeviceToHost, G->st));
  CK(cudaStreamSynchronize(G->st));
  const size_t n = std::min<size_t>(o[1] - o[0], (size_t)s->p.K_max);
  *n_out = n;
  const size_t words = (size_t)s->desc_D / 32;
  const bool odd = ((s->frame - 1) & 1) != 0;
  const uint32_t* src = (odd ? G->streams[id].desc1 : s->desc) + (size_t)o[0] * words;
  const size_t ncopy = std::min(n, cap);
  if (ncopy)
    CK(cudaMemcpy(out, src, ncopy * words * 4, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost));
  if (n > cap && out) return fail(FKD_E_CAPACITY, "%zu descriptors > cap %zu", n, cap);
  return FKD_OK;
}

int fkd_group_profile_enable(fkd_group* G, int on) {
  if (!G) return fail(FKD_E_ARG, "group is NULL");
  G->profiling = on != 0;
  return FKD_OK;
}

int fkd_group_profile_read(fkd_group* G, fkd_profile* out, int reset) {
  if (!G || !out) return fail(FKD_E_ARG, "NULL argument");
  CK(cudaStreamSynchronize(G->st));
  for (auto& pd : G->pending) {
    for (int i = 0; i < FKD_NUM_STAGES; ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, pd.ev[i], pd.ev[i + 1]));
      G->prof.ms[i] += ms;
      if (i != FKD_STAGE_DESCRIBE || G->any_describe) G->prof.launches[i] += 1;
    }
    G->prof.batches += 1;
    G->prof.frames += (uint64_t)pd.frames;
    for (cudaEvent_t e : pd.ev) G->event_pool.push_back(e);
  }
  G->pending.clear();
  unsigned long long tiles = 0, px = 0;
  for (auto& gs : G->streams)
    if (gs.s) {
      unsigned long long ts[2];
      CK(cudaMemcpy(ts, gs.s->s.tile_stats, 16, cudaMemcpyDeviceToHost));
      tiles += ts[0] - gs.s->tile_stats_seen[0];
      px += ts[1] - gs.s->tile_stats_seen[1];
      gs.s->tile_stats_seen[0] = ts[0];
      gs.s->tile_stats_seen[1] = ts[1];
    }
  G->prof.tiles += tiles;
  G->prof.tile_pixels += px;
  *out = G->prof;
  if (reset) G->prof = fkd_profile{};
  return FKD_OK;
}

int fkd_group_get_launch_config(const fkd_group* G, fkd_launch_config* out) {
  if (!G || !out) return fail(FKD_E_ARG, "NULL argument");
  *out = G->lc;
  return FKD_OK;
}

int fkd_group_set_launch_config(fkd_group* G, const fkd_launch_config* c) {
  if (!G) return fail(FKD_E_ARG, "group is NULL");
  DetLaunch dl{};
  int rc = resolve_launch(c, &dl);
  if (rc) return rc;
  CK(cudaStreamSynchronize(G->st));
  G->lc = *c;
  G->dl = dl;
  for (int id = 0; id < (int)G->streams.size(); ++id) {
    GroupStream& gs = G->streams[id];
    if (!gs.s) continue;
    apply_launch(gs.s, *c, dl);
    const StreamDev d = make_dev(gs.s, gs);
    CK(cudaMemcpy(G->d_devs + id, &d, sizeof d, cudaMemcpyHostToDevice));
  }
  G->drop_graphs();
  return FKD_OK;
}

int fkd_group_autotune(fkd_group* G, int n, const int* ids, int m, const uint8_t* const* frames,
                       const size_t* pitches, int reps, fkd_launch_config* best, float* best_ms) {
  if (!G || n < 1 || m < 1 || !ids || !frames || !pitches) return fail(FKD_E_ARG, "NULL argument or empty tick");
  if (reps < 1 || reps > 100) return fail(FKD_E_ARG, "reps %d outside 1..100", reps);
  for (int i = 0; i < n; ++i)
    if (!group_member(G, ids[i])) return fail(FKD_E_ARG, "unknown stream id %d", ids[i]);
  CK(cudaStreamSynchronize(G->st));
  const bool prof = G->profiling;
  G->profiling = false;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  CK(cudaEventCreate(&ev[0]));
  CK(cudaEventCreate(&ev[1]));
  auto reset_all = [&]() {
    for (auto& gs : G->streams)
      if (gs.s) reset_history(gs.s);
  };
  const fkd_launch_config start = G->lc;
  fkd_launch_config win = start;
  float win_ms = -1.f;
  int rc = FKD_OK;
  for (const fkd_launch_config& c : launch_candidates(start)) {
    if ((rc = fkd_group_set_launch_config(G, &c))) break;
    float best_c = -1.f;
    for (int r = 0; r <= reps && rc == FKD_OK; ++r) {
      reset_all();
      cudaEventRecord(ev[0], G->st);
      for (int j = 0; j < m && rc == FKD_OK; ++j) rc = fkd_group_tick(G, n, ids, frames + (size_t)j * n, pitches);
      cudaEventRecord(ev[1], G->st);
      cudaError_t e = cudaEventSynchronize(ev[1]);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (e != cudaSuccess && rc == FKD_OK) rc = fail(FKD_E_CUDA, "autotune timing failed: %s", cudaGetErrorString(e));
      if (r > 0 && (best_c < 0.f || ms < best_c)) best_c = ms;
    }
    if (rc) break;
    if (win_ms < 0.f || best_c < kTuneMargin * win_ms) {
      win_ms = best_c;
      win = c;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  G->profiling = prof;
  const int rc2 = fkd_group_set_launch_config(G, rc ? &start : &win);
  reset_all();
  for (auto& gs : G->streams)
    if (gs.s) {
      cudaMemset(gs.s->s.overflow, 0, 4);
      cudaMemcpy(gs.s->tile_stats_seen, gs.s->s.tile_stats, 16, cudaMemcpyDeviceToHost);
    }
  if (rc) return rc;
  if (rc2) return rc2;
  if (best) *best = win;
  if (best_ms) *best_ms = win_ms;
  return FKD_OK;
}

int fkd_group_check_guards(fkd_group* G) {
  if (!G) return fail(FKD_E_ARG, "group is NULL");
  for (auto& gs : G->streams)
    if (gs.s)
      if (int rc = fkd_check_guards(gs.s)) return rc;
  return FKD_OK;
}

}  // extern "C"

// ------------------------------------------------------- internal (server)

namespace fkd {

int group_result_ref(fkd_group* G, int id, long long frame_index, ResultRef* ref) {
  fkd_stream* s = group_member(G, id);
  if (!s) return fail(FKD_E_ARG, "unknown stream id %d", id);
  const bool odd = (frame_index & 1) != 0;
  ref->rec = odd ? G->streams[id].rec1 : s->rec;
  ref->off = odd ? G->streams[id].off1 : s->rec_offsets;
  ref->cap = s->p.K_max;
  return FKD_OK;
}

int group_desc_ref(fkd_group* G, int id, long long frame_index, const uint32_t** desc, int* D) {
  fkd_stream* s = group_member(G, id);
  if (!s) return fail(FKD_E_ARG, "unknown stream id %d", id);
  *D = s->desc_D;
  *desc = (frame_index & 1) ? G->streams[id].desc1 : s->desc;
  return FKD_OK;
}

size_t group_stream_bytes(fkd_group* G, int id) {
  return group_member(G, id) ? G->streams[id].bytes : 0;
}

long long group_stream_frames(fkd_group* G, int id) {
  fkd_stream* s = group_member(G, id);
  return s ? s->frame : -1;
}

int group_stream_kmax(fkd_group* G, int id) {
  fkd_stream* s = group_member(G, id);
  return s ? s->p.K_max : 0;
}

cudaStream_t group_cuda_stream(fkd_group* G) { return G->st; }

}  // namespace fkd
