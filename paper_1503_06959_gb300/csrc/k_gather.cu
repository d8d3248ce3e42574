// k_gather.cu -- gather the keypoint sets of many streams into one buffer,
// and upload the frames of a serving round.
//
// After a group tick each stream's D_n sits in its own device buffer. The
// serving loop copies all of them back to the host at once: one kernel turns
// the counts into offsets (a block-wide scan), a second copies the records
// contiguously, so the host needs one copy for the offsets and one for the
// records whatever the number of streams.
#include "fkd_internal.cuh"

namespace fkd {
namespace {

constexpr int kGatherThreads = 1024;

__global__ void __launch_bounds__(kGatherThreads) k_gather_offsets(const ResultRef* refs, int n,
                                                                   uint32_t* offsets) {
  __shared__ uint32_t wsum[kGatherThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t carry = 0;
  for (int i0 = 0; i0 < n; i0 += kGatherThreads) {
    const int i = i0 + threadIdx.x;
    uint32_t c = 0;
    if (i < n) {
      const uint32_t raw = refs[i].off[1] - refs[i].off[0];
      offsets[n + 1 + i] = raw;
      c = (uint32_t)min((long long)raw, refs[i].cap);
    }
    uint32_t incl = c;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += v;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    uint32_t before = carry, all = carry;
    for (int w = 0; w < kGatherThreads / 32; ++w) {
      if (w < wid) before += wsum[w];
      all += wsum[w];
    }
    if (i < n) offsets[i] = before + incl - c;
    carry = all;
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[n] = carry;
}

__global__ void k_gather_copy(const ResultRef* refs, int n, const uint32_t* offsets, fkd_keypoint* out,
                              long long cap) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    const uint32_t o = offsets[i], c = offsets[i + 1] - o;
    const uint2* src = reinterpret_cast<const uint2*>(refs[i].rec);
    uint2* dst = reinterpret_cast<uint2*>(out);
    for (uint32_t j = threadIdx.x; j < c; j += blockDim.x)
      if ((long long)o + j < cap) dst[o + j] = src[j];
  }
}

}  // namespace

void launch_gather(const ResultRef* refs, int n, uint32_t* offsets, fkd_keypoint* out, long long out_cap,
                   cudaStream_t st) {
  k_gather_offsets<<<1, kGatherThreads, 0, st>>>(refs, n, offsets);
  k_gather_copy<<<max(1, min(n, 1024)), 256, 0, st>>>(refs, n, offsets, out, out_cap);
}

namespace {

// Frame upload of a round: CTA (part, item) copies rows part*H/8 ..
// (part+1)*H/8 - 1 of frame `item`, 16 bytes per thread per step when the
// addresses, pitches and width allow it.
constexpr int kUploadParts = 8;
__global__ void __launch_bounds__(256) k_upload(const UploadItem* items) {
  const UploadItem it = items[blockIdx.y];
  const int y0 = (int)((long long)blockIdx.x * it.H / kUploadParts);
  const int y1 = (int)((long long)(blockIdx.x + 1) * it.H / kUploadParts);
  const bool vec = ((reinterpret_cast<uintptr_t>(it.src) | (uintptr_t)it.src_pitch |
                     reinterpret_cast<uintptr_t>(it.dst) | (uintptr_t)it.dst_pitch | (uintptr_t)it.W) & 15) == 0;
  if (vec) {
    const int wv = it.W / 16;
    const long long total = (long long)(y1 - y0) * wv;
    for (long long q = threadIdx.x; q < total; q += blockDim.x) {
      const int y = y0 + (int)(q / wv), x = (int)(q % wv);
      reinterpret_cast<uint4*>(it.dst + (long long)y * it.dst_pitch)[x] =
          reinterpret_cast<const uint4*>(it.src + (long long)y * it.src_pitch)[x];
    }
  } else {
    const long long total = (long long)(y1 - y0) * it.W;
    for (long long q = threadIdx.x; q < total; q += blockDim.x) {
      const int y = y0 + (int)(q / it.W), x = (int)(q % it.W);
      it.dst[(long long)y * it.dst_pitch + x] = it.src[(long long)y * it.src_pitch + x];
    }
  }
}

}  // namespace

void launch_upload(const UploadItem* items, int n, cudaStream_t st) {
  if (n > 0) k_upload<<<dim3(kUploadParts, n), 256, 0, st>>>(items);
}

}  // namespace fkd
