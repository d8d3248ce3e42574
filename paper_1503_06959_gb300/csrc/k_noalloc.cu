// k_noalloc.cu -- the intensity-difference detection mask of one frame pair
// for callers that cannot allocate device memory.
//
// fkd_create_stream allocates its own scratch with cudaMalloc. Some callers
// cannot let a library allocate: applications that hand every byte of GPU
// memory to their own allocator or memory budget at start-up, plugins that
// run inside a host program which owns all device memory, and real-time
// loops that must not pay for an allocation (or the implicit synchronisation
// of cudaMalloc / cudaFree) on their path. For them, fkd_id_mask_noalloc
// computes the mask of Eq. 2 (bin mean of |I_n - I_{n-1}| on c_0 above T_I,
// the same test fkd_push_frames applies with mask_layer 0) using only the
// caller's buffers and a fixed scratch array that lives in this library's
// device memory for as long as the library is loaded.
#include <mutex>

#include <cuda.h>

#include "fkd_internal.cuh"

namespace {

constexpr int kNoAllocMaxBins = 4096;  // == FKD_NOALLOC_MAX_BINS
constexpr int kRowsPerBlock = 64;
constexpr int kThreads = 256;

// Per-bin sums of |cur - prev|, shared by every call (see fkd.h).
static __device__ __align__(256) unsigned long long g_noalloc_bsum[kNoAllocMaxBins];

__global__ void k_noalloc_clear(unsigned long long* bsum, int nb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nb) bsum[i] = 0ull;
}

// One thread per pixel column of a band of kRowsPerBlock rows: a running sum
// of |cur - prev| that is added to the bin whenever the bin row changes.
__global__ void k_noalloc_sums(const uint8_t* cur, const uint8_t* prev, int W, int H, long long pitch,
                               int N_r, int N_c, unsigned long long* bsum) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y0 = blockIdx.y * kRowsPerBlock;
  if (x >= W) return;
  const int c = (int)(((long long)x * N_c) / W);
  const int y1 = min(H, y0 + kRowsPerBlock);
  int r_cur = -1;
  unsigned long long acc = 0;
  for (int y = y0; y < y1; ++y) {
    const int r = (int)(((long long)y * N_r) / H);
    if (r != r_cur) {
      if (acc) atomicAdd(&bsum[r_cur * N_c + c], acc);
      r_cur = r;
      acc = 0;
    }
    const int d = (int)cur[(long long)y * pitch + x] - (int)prev[(long long)y * pitch + x];
    acc += (unsigned long long)(d < 0 ? -d : d);
  }
  if (acc) atomicAdd(&bsum[r_cur * N_c + c], acc);
}

// Bin (r, c) of c_0 holds columns x with floor(x*N_c/W) == c, i.e.
// x in [ceil(c*W/N_c), ceil((c+1)*W/N_c)), and rows likewise.
__device__ __forceinline__ long long first_of(long long c, long long n, long long size) {
  return (c * size + n - 1) / n;
}

__global__ void k_noalloc_mask(const unsigned long long* bsum, int W, int H, int N_r, int N_c, int T_I,
                               uint8_t* mask) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= N_r * N_c) return;
  const int r = b / N_c, c = b % N_c;
  const long long w = first_of(c + 1, N_c, W) - first_of(c, N_c, W);
  const long long h = first_of(r + 1, N_r, H) - first_of(r, N_r, H);
  mask[b] = bsum[b] > (unsigned long long)T_I * (unsigned long long)(w * h) ? 1 : 0;
}

// Failures are reported through fkd_last_error like every other entry point.
int noalloc_fail(int code, const char* msg, cudaError_t e = cudaSuccess) {
  return fkd::set_error(code, "fkd_id_mask_noalloc: %s%s%s", msg, e != cudaSuccess ? ": " : "",
                        e != cudaSuccess ? cudaGetErrorString(e) : "");
}

// Device address of the scratch array in each CUDA context that has called
// this entry point, keyed by the driver's context ID (unique for the life of
// the process, so a context destroyed and created again at the same handle
// never finds a stale address). The address is looked up once per context,
// on its first call made outside stream capture.
constexpr int kMaxContexts = 64;
struct ScratchSlot {
  unsigned long long ctx_id;
  unsigned long long* ptr;
};
std::mutex g_scratch_mu;
ScratchSlot g_scratch[kMaxContexts] = {};
int g_scratch_n = 0;

// The driver's cuCtxGetCurrent and cuCtxGetId, fetched through the runtime
// (no link-time dependency on the driver library).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

int current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(f);
  });
  if (!get_current || !get_id) return noalloc_fail(FKD_E_CUDA, "driver context queries unavailable");
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return noalloc_fail(FKD_E_CUDA, "no current CUDA context");
  if (get_id(ctx, id) != CUDA_SUCCESS) return noalloc_fail(FKD_E_CUDA, "cuCtxGetId failed");
  return FKD_OK;
}

}  // namespace

extern "C" int fkd_id_mask_noalloc(const uint8_t* cur, const uint8_t* prev, int W, int H, size_t pitch,
                                   int N_r, int N_c, int T_I, uint8_t* mask_out, void* cuda_stream) {
  if (!cur || !prev || !mask_out) return noalloc_fail(FKD_E_ARG, "NULL buffer");
  if (W < 1 || H < 1 || W > 16384 || H > 16384) return noalloc_fail(FKD_E_ARG, "frame size outside 1..16384");
  if (pitch < (size_t)W) return noalloc_fail(FKD_E_ARG, "pitch smaller than W");
  if (N_r < 1 || N_c < 1 || N_r > H || N_c > W) return noalloc_fail(FKD_E_ARG, "bin grid does not fit the frame");
  if (N_r * N_c > kNoAllocMaxBins)
    return noalloc_fail(FKD_E_ARG, "N_r * N_c exceeds FKD_NOALLOC_MAX_BINS (4096)");
  if (T_I < 0) return noalloc_fail(FKD_E_ARG, "T_I must be >= 0");
  // an error left pending by earlier work on this thread belongs to the
  // caller: report it without clearing it, and launch nothing
  cudaError_t e = cudaPeekAtLastError();
  if (e != cudaSuccess) return noalloc_fail(FKD_E_CUDA, "a CUDA error was already pending", e);
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return noalloc_fail(FKD_E_CUDA, "cudaStreamIsCapturing failed", e);
  unsigned long long ctx_id = 0;
  if (int rc = current_context_id(&ctx_id)) return rc;
  unsigned long long* bsum = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    for (int i = 0; i < g_scratch_n; ++i)
      if (g_scratch[i].ctx_id == ctx_id) bsum = g_scratch[i].ptr;
    if (!bsum) {
      if (cap != cudaStreamCaptureStatusNone)
        return noalloc_fail(FKD_E_STATE,
                            "first call on this CUDA context made during stream capture; call once before capturing");
      if (g_scratch_n == kMaxContexts) return noalloc_fail(FKD_E_CUDA, "more than 64 CUDA contexts");
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_bsum);
      if (e != cudaSuccess) return noalloc_fail(FKD_E_CUDA, "cudaGetSymbolAddress failed", e);
      bsum = static_cast<unsigned long long*>(p);
      g_scratch[g_scratch_n++] = ScratchSlot{ctx_id, bsum};
    }
  }
  const int nb = N_r * N_c;
  k_noalloc_clear<<<(nb + kThreads - 1) / kThreads, kThreads, 0, st>>>(bsum, nb);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(FKD_E_CUDA, "clear kernel launch failed", e);
  dim3 grid((W + kThreads - 1) / kThreads, (H + kRowsPerBlock - 1) / kRowsPerBlock);
  k_noalloc_sums<<<grid, kThreads, 0, st>>>(cur, prev, W, H, (long long)pitch, N_r, N_c, bsum);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(FKD_E_CUDA, "sums kernel launch failed", e);
  k_noalloc_mask<<<(nb + kThreads - 1) / kThreads, kThreads, 0, st>>>(bsum, W, H, N_r, N_c, T_I, mask_out);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_fail(FKD_E_CUDA, "mask kernel launch failed", e);
  return FKD_OK;
}
