// fkd_server.cu -- serving loop: many video streams, frames arriving at any
// time, continuous batching of ready frames into group ticks.
//
// A worker thread owns the GPU side. Each round it takes the oldest waiting
// frame of every stream that has one (frames that arrived while the previous
// tick was on the GPU join this one), copies them from the streams' pinned
// host rings to device staging on a copy stream, runs one group tick (one
// launch per kernel for all of them, replayed from a CUDA graph), gathers all
// results into one buffer and brings them back with two copies. Rounds are
// pipelined: while tick i runs on the GPU the worker collects tick i-1 and
// hands its keypoints to the streams' result queues. Streams are admitted
// against a device-memory budget and release their memory when closed, so
// waiting streams can be admitted as others leave.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "fkd_internal.cuh"

namespace fkd {
// Group internals for the description of served streams (fkd_api.cu).
int group_desc_ref(fkd_group* G, int id, long long frame_index, const uint32_t** desc, int* D);
size_t group_stream_bytes(fkd_group* G, int id);
}  // namespace fkd

using namespace fkd;

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr int kRingSlots = 4;

struct Result {
  int64_t index;
  bool truncated;
  std::vector<fkd_keypoint> kp;
  std::vector<uint8_t> desc;  // D/8 bytes per keypoint, if the stream describes
};

struct SStream {
  bool open = false;
  int W = 0, H = 0, pitch = 0, K_max = 0;
  size_t bytes = 0;            // device bytes charged to the budget
  uint8_t* ring = nullptr;     // pinned host frames, kRingSlots x W*H
  const uint8_t* ref[kRingSlots] = {};  // a caller's frame queued by reference (else null: the ring's copy)
  size_t ref_pitch[kRingSlots] = {};
  const uint8_t* src_dev[kRingSlots] = {};  // device-accessible address of the slot's frame (null: copy by DMA)
  uint8_t* ring_dev = nullptr;              // device-accessible address of the ring
  int64_t arrival[kRingSlots] = {};
  int head = 0, count = 0;     // queued frames (oldest at head), including in flight
  int in_flight = 0;           // of those, frames already in a launched tick
  int64_t taken = 0;           // frames handed to ticks so far
  uint8_t* dstage[2] = {nullptr, nullptr};  // device copies, by frame parity
  std::deque<Result> results;
  int D = 0;                       // descriptor bits (0: the stream does not describe)
  std::vector<uint8_t> last_desc;  // descriptors of the result the last poll returned
  bool have_last = false;
};

struct TickRec {
  std::vector<int> ids;
  std::vector<int64_t> index, arrival;
  int buf = 0;
};

}  // namespace

struct fkd_server {
  fkd_group* G = nullptr;
  size_t budget = 0, used = 0;
  cudaStream_t comp = nullptr, copy = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, done[2] = {nullptr, nullptr};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  int error = FKD_OK;
  std::vector<SStream> streams;  // by group stream id
  long long cap = 0;             // records one tick can bring back
  UploadItem* h_up[2] = {nullptr, nullptr};  // a round's frames read by the upload kernel
  UploadItem* d_up[2] = {nullptr, nullptr};
  ResultRef* h_refs[2] = {nullptr, nullptr};
  ResultRef* d_refs[2] = {nullptr, nullptr};
  uint32_t* h_off[2] = {nullptr, nullptr};  // n + 1 offsets, then n counts
  uint32_t* d_off[2] = {nullptr, nullptr};
  std::string err_msg;                        // message of a worker failure
  bool keep_results = true;                   // false: results are counted and timed, then dropped
  fkd_keypoint* h_out[2] = {nullptr, nullptr};
  fkd_keypoint* d_out[2] = {nullptr, nullptr};
  // statistics
  std::vector<double> lat_ms;
  uint64_t frames_done = 0, ticks = 0, rejected_frames = 0, rejected_streams = 0;
  double batch_sum = 0;
  int64_t t_first = 0, t_last = 0;

  void run();
  int launch_tick(TickRec& t, int b);
  void collect(const TickRec& t);
};

namespace {

// The sticky error of the worker, re-raised in the caller's thread.
int worker_error(fkd_server* S) { return set_error(S->error, "%s", S->err_msg.c_str()); }

bool any_ready(const fkd_server* S) {
  for (const auto& s : S->streams)
    if (s.open && s.count > s.in_flight) return true;
  return false;
}

}  // namespace

// Form and launch one tick from the streams' oldest waiting frames (lock held).
int fkd_server::launch_tick(TickRec& t, int b) {
  std::vector<const uint8_t*> frames;
  std::vector<size_t> pitches;
  int nup = 0;
  for (int id = 0; id < (int)streams.size(); ++id) {
    SStream& s = streams[id];
    if (!s.open || s.count <= s.in_flight) continue;
    const int slot = (s.head + s.in_flight) % kRingSlots;
    const int64_t idx = s.taken;
    uint8_t* dst = s.dstage[idx & 1];
    const uint8_t* from = s.ref[slot] ? s.ref[slot] : s.ring + (size_t)slot * s.W * s.H;
    const size_t from_pitch = s.ref[slot] ? s.ref_pitch[slot] : (size_t)s.W;
    if (s.src_dev[slot]) {
      // pinned host memory the GPU can read: copied by the round's upload kernel
      h_up[b][nup++] = UploadItem{s.src_dev[slot], (long long)from_pitch, dst, s.pitch, s.W, s.H};
    } else {
      cudaError_t e = cudaMemcpy2DAsync(dst, s.pitch, from, from_pitch, s.W, s.H, cudaMemcpyHostToDevice, copy);
      if (e != cudaSuccess) return set_error(FKD_E_CUDA, "frame upload failed: %s", cudaGetErrorString(e));
    }
    t.ids.push_back(id);
    t.index.push_back(idx);
    t.arrival.push_back(s.arrival[slot]);
    frames.push_back(dst);
    pitches.push_back((size_t)s.pitch);
    s.in_flight += 1;
    s.taken += 1;
  }
  const int n = (int)t.ids.size();
  t.buf = b;
  if (nup) {
    cudaError_t e = cudaMemcpyAsync(d_up[b], h_up[b], (size_t)nup * sizeof(UploadItem), cudaMemcpyHostToDevice, copy);
    if (e != cudaSuccess) return set_error(FKD_E_CUDA, "upload list copy failed: %s", cudaGetErrorString(e));
    launch_upload(d_up[b], nup, copy);
  }
  cudaEventRecord(copied[b], copy);
  cudaStreamWaitEvent(comp, copied[b], 0);
  int rc = fkd_group_tick(G, n, t.ids.data(), frames.data(), pitches.data());
  if (rc) return rc;
  for (int i = 0; i < n; ++i)
    if ((rc = group_result_ref(G, t.ids[i], t.index[i], &h_refs[b][i]))) return rc;
  cudaMemcpyAsync(d_refs[b], h_refs[b], (size_t)n * sizeof(ResultRef), cudaMemcpyHostToDevice, comp);
  launch_gather(d_refs[b], n, d_off[b], d_out[b], cap, comp);
  cudaMemcpyAsync(h_off[b], d_off[b], (size_t)(2 * n + 1) * 4, cudaMemcpyDeviceToHost, comp);
  cudaEventRecord(done[b], comp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(FKD_E_CUDA, "tick launch failed: %s", cudaGetErrorString(e));
  ticks += 1;
  batch_sum += n;
  return FKD_OK;
}

// Bring a finished tick's keypoints back and hand them out (lock not held
// while waiting for the GPU).
void fkd_server::collect(const TickRec& t) {
  const int b = t.buf, n = (int)t.ids.size();
  cudaError_t e = cudaEventSynchronize(done[b]);
  long long total = 0;
  if (e == cudaSuccess) {
    total = h_off[b][n];
    const long long ncopy = keep_results ? std::min(total, cap) : 0;
    if (ncopy > 0) e = cudaMemcpyAsync(h_out[b], d_out[b], (size_t)ncopy * sizeof(fkd_keypoint),
                                       cudaMemcpyDeviceToHost, copy);
    if (e == cudaSuccess) e = cudaStreamSynchronize(copy);
  }
  const int64_t t_done = now_ns();
  std::lock_guard<std::mutex> lk(mu);
  if (e != cudaSuccess) {
    error = FKD_E_CUDA;
    err_msg = std::string("tick failed: ") + cudaGetErrorString(e);
    cv_done.notify_all();
    return;
  }
  for (int i = 0; i < n; ++i) {
    SStream& s = streams[t.ids[i]];
    const long long o = h_off[b][i], c = (long long)h_off[b][i + 1] - o;
    const long long raw = h_off[b][n + 1 + i];
    s.head = (s.head + 1) % kRingSlots;
    s.count -= 1;
    s.in_flight -= 1;
    lat_ms.push_back((t_done - t.arrival[i]) * 1e-6);
    frames_done += 1;
    if (!keep_results) continue;
    Result r;
    r.index = t.index[i];
    const long long keep = std::max(0LL, std::min(c, cap - o));
    r.truncated = keep < raw;
    r.kp.assign(h_out[b] + o, h_out[b] + o + keep);
    if (s.D && !r.truncated && keep > 0) {
      // the frame's descriptors stay in the group's buffers of its parity
      // until the tick after next, which is launched after this collection
      const uint32_t* desc = nullptr;
      int D = 0;
      cudaError_t ed = cudaErrorInvalidValue;
      if (group_desc_ref(G, t.ids[i], t.index[i], &desc, &D) == FKD_OK && desc) {
        r.desc.resize((size_t)keep * (size_t)(D / 8));
        ed = cudaMemcpy(r.desc.data(), desc, r.desc.size(), cudaMemcpyDeviceToHost);
      }
      if (ed != cudaSuccess) {
        error = FKD_E_CUDA;
        err_msg = std::string("descriptor copy failed: ") + cudaGetErrorString(ed);
      }
    }
    s.results.push_back(std::move(r));
  }
  t_last = t_done;
  cv_done.notify_all();
}

void fkd_server::run() {
  std::unique_lock<std::mutex> lk(mu);
  TickRec pending;
  bool have_pending = false;
  int b = 0;
  for (;;) {
    cv_work.wait(lk, [&] { return stop || have_pending || (error == FKD_OK && any_ready(this)); });
    if (stop && !have_pending) break;
    TickRec cur;
    bool launched = false;
    if (!stop && error == FKD_OK && any_ready(this)) {
      const int rc = launch_tick(cur, b);
      if (rc) {
        error = rc;
        err_msg = fkd_last_error();
        cv_done.notify_all();
      } else {
        launched = true;
      }
    }
    if (have_pending) {
      lk.unlock();
      collect(pending);
      lk.lock();
    }
    have_pending = launched;
    if (launched) {
      pending = std::move(cur);
      b ^= 1;
    }
  }
}

extern "C" {

int fkd_server_create(int O, int intra, size_t budget_bytes, size_t max_tick_keypoints, fkd_server** out) {
  if (!out) return set_error(FKD_E_ARG, "out is NULL");
  *out = nullptr;
  if (max_tick_keypoints < 1 || max_tick_keypoints > ((size_t)1 << 31))
    return set_error(FKD_E_ARG, "max_tick_keypoints outside 1..2^31");
  const size_t fixed = 2 * (max_tick_keypoints * sizeof(fkd_keypoint) + (2 * kMaxTickItems + 1) * 4 +
                            kMaxTickItems * (sizeof(ResultRef) + sizeof(UploadItem)));
  if (fixed > budget_bytes)
    return set_error(FKD_E_BUDGET, "budget %zu below the server's own %zu bytes", budget_bytes, fixed);
  fkd_server* S = new (std::nothrow) fkd_server();
  if (!S) return set_error(FKD_E_ARG, "out of host memory");
  S->budget = budget_bytes;
  S->cap = (long long)max_tick_keypoints;
  auto bail = [&](int rc) {
    fkd_server_destroy(S);
    return rc;
  };
  cudaError_t e;
  if ((e = cudaStreamCreateWithFlags(&S->comp, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaStreamCreateWithFlags(&S->copy, cudaStreamNonBlocking)) != cudaSuccess)
    return bail(set_error(FKD_E_CUDA, "stream creation failed: %s", cudaGetErrorString(e)));
  for (int b = 0; b < 2; ++b) {
    if ((e = cudaEventCreateWithFlags(&S->copied[b], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&S->done[b], cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaHostAlloc(&S->h_up[b], kMaxTickItems * sizeof(UploadItem), cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaMalloc(&S->d_up[b], kMaxTickItems * sizeof(UploadItem))) != cudaSuccess ||
        (e = cudaHostAlloc(&S->h_refs[b], kMaxTickItems * sizeof(ResultRef), cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaMalloc(&S->d_refs[b], kMaxTickItems * sizeof(ResultRef))) != cudaSuccess ||
        (e = cudaHostAlloc(&S->h_off[b], (2 * kMaxTickItems + 1) * 4, cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaMalloc(&S->d_off[b], (2 * kMaxTickItems + 1) * 4)) != cudaSuccess ||
        (e = cudaHostAlloc(&S->h_out[b], max_tick_keypoints * sizeof(fkd_keypoint), cudaHostAllocDefault)) != cudaSuccess ||
        (e = cudaMalloc(&S->d_out[b], max_tick_keypoints * sizeof(fkd_keypoint))) != cudaSuccess)
      return bail(set_error(FKD_E_CUDA, "server allocation failed: %s", cudaGetErrorString(e)));
  }
  S->used = fixed;
  int rc = fkd_group_create(O, intra, S->comp, &S->G);
  if (rc) return bail(rc);
  S->worker = std::thread([S] { S->run(); });
  *out = S;
  return FKD_OK;
}

int fkd_server_destroy(fkd_server* S) {
  if (!S) return FKD_OK;
  if (S->worker.joinable()) {
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->stop = true;
    }
    S->cv_work.notify_all();
    S->worker.join();
  }
  if (S->comp) cudaStreamSynchronize(S->comp);
  if (S->G) fkd_group_destroy(S->G);
  for (auto& s : S->streams) {
    if (s.ring) cudaFreeHost(s.ring);
    for (auto* d : s.dstage) cudaFree(d);
  }
  for (int b = 0; b < 2; ++b) {
    if (S->copied[b]) cudaEventDestroy(S->copied[b]);
    if (S->done[b]) cudaEventDestroy(S->done[b]);
    if (S->h_refs[b]) cudaFreeHost(S->h_refs[b]);
    if (S->h_up[b]) cudaFreeHost(S->h_up[b]);
    cudaFree(S->d_up[b]);
    if (S->h_off[b]) cudaFreeHost(S->h_off[b]);
    if (S->h_out[b]) cudaFreeHost(S->h_out[b]);
    cudaFree(S->d_refs[b]);
    cudaFree(S->d_off[b]);
    cudaFree(S->d_out[b]);
  }
  if (S->copy) cudaStreamDestroy(S->copy);
  if (S->comp) cudaStreamDestroy(S->comp);
  delete S;
  return FKD_OK;
}

int fkd_server_open_stream(fkd_server* S, const fkd_params* p, int W, int H, int* id) {
  if (!S || !p || !id) return set_error(FKD_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->error) return worker_error(S);
  int open = 0;
  for (const auto& o : S->streams) open += o.open ? 1 : 0;
  if (open >= kMaxTickItems) return set_error(FKD_E_BUDGET, "at most %d open streams", kMaxTickItems);
  int gid = -1;
  size_t gbytes = 0;
  int rc = fkd_group_add_stream(S->G, p, W, H, &gid, &gbytes);
  if (rc) return rc;
  const int pitch = (W + 15) / 16 * 16;
  const size_t bytes = gbytes + 2 * (size_t)pitch * H;
  if (S->used + bytes > S->budget) {
    fkd_group_remove_stream(S->G, gid);
    S->rejected_streams += 1;
    return set_error(FKD_E_BUDGET, "stream needs %zu bytes, %zu of %zu in use", bytes, S->used, S->budget);
  }
  if ((int)S->streams.size() <= gid) S->streams.resize(gid + 1);
  SStream& s = S->streams[gid];
  s = SStream();
  s.W = W;
  s.H = H;
  s.pitch = pitch;
  s.K_max = p->K_max;
  s.bytes = bytes;
  cudaError_t e;
  if ((e = cudaHostAlloc(&s.ring, (size_t)kRingSlots * W * H, cudaHostAllocDefault)) != cudaSuccess ||
      (e = cudaMalloc(&s.dstage[0], (size_t)pitch * H)) != cudaSuccess ||
      (e = cudaMalloc(&s.dstage[1], (size_t)pitch * H)) != cudaSuccess) {
    if (s.ring) cudaFreeHost(s.ring);
    for (auto*& d : s.dstage) {
      cudaFree(d);
      d = nullptr;
    }
    s.ring = nullptr;
    fkd_group_remove_stream(S->G, gid);
    return set_error(FKD_E_CUDA, "stream buffers: %s", cudaGetErrorString(e));
  }
  {
    // the ring as the device addresses it (pinned memory is mapped under
    // unified addressing); without it frames are copied by DMA
    void* dp = nullptr;
    s.ring_dev = cudaHostGetDevicePointer(&dp, s.ring, 0) == cudaSuccess ? static_cast<uint8_t*>(dp) : nullptr;
    if (!s.ring_dev) cudaGetLastError();
  }
  s.open = true;
  S->used += bytes;
  *id = gid;
  return FKD_OK;
}

int fkd_server_close_stream(fkd_server* S, int id) {
  if (!S) return set_error(FKD_E_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  if (id < 0 || id >= (int)S->streams.size() || !S->streams[id].open)
    return set_error(FKD_E_ARG, "unknown stream id %d", id);
  SStream& s = S->streams[id];
  // frames already on the GPU finish; frames still waiting are dropped
  S->cv_done.wait(lk, [&] { return s.in_flight == 0 || S->error != FKD_OK; });
  s.open = false;
  s.count = 0;
  fkd_group_remove_stream(S->G, id);
  cudaFreeHost(s.ring);
  s.ring = nullptr;
  for (auto*& d : s.dstage) {
    cudaFree(d);
    d = nullptr;
  }
  s.results.clear();
  S->used -= s.bytes;
  return FKD_OK;
}

}  // extern "C"

namespace {

// Queue the next frame of stream `id`: a copy into the stream's pinned ring,
// or (by_ref) the caller's pointer, uploaded from where it is.
int submit_frame(fkd_server* S, int id, const uint8_t* frame, size_t pitch, int64_t arrival_ns, bool by_ref) {
  if (!S || !frame) return set_error(FKD_E_ARG, "NULL argument");
  const int64_t t = arrival_ns > 0 ? arrival_ns : now_ns();
  // a frame queued by reference is read by the upload kernel when it lies in
  // pinned host memory the device can address, else copied by DMA
  const uint8_t* src_dev = nullptr;
  if (by_ref) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, frame) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer)
      src_dev = static_cast<const uint8_t*>(a.devicePointer);
    else
      cudaGetLastError();  // an unregistered pointer is not an error of this call
  }
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (S->error) return worker_error(S);
    if (id < 0 || id >= (int)S->streams.size() || !S->streams[id].open)
      return set_error(FKD_E_ARG, "unknown stream id %d", id);
    SStream& s = S->streams[id];
    if (pitch < (size_t)s.W) return set_error(FKD_E_ARG, "pitch < W");
    if (s.count == kRingSlots) {
      S->rejected_frames += 1;
      return set_error(FKD_E_CAPACITY, "stream %d already has %d frames waiting", id, kRingSlots);
    }
    const int slot = (s.head + s.count) % kRingSlots;
    if (by_ref) {
      s.ref[slot] = frame;
      s.ref_pitch[slot] = pitch;
      s.src_dev[slot] = src_dev;
    } else {
      s.ref[slot] = nullptr;
      uint8_t* dst = s.ring + (size_t)slot * s.W * s.H;
      for (int y = 0; y < s.H; ++y) std::memcpy(dst + (size_t)y * s.W, frame + (size_t)y * pitch, (size_t)s.W);
      s.src_dev[slot] = s.ring_dev ? s.ring_dev + (size_t)slot * s.W * s.H : nullptr;
    }
    s.arrival[slot] = t;
    s.count += 1;
    if (!S->t_first) S->t_first = t;
  }
  S->cv_work.notify_one();
  return FKD_OK;
}

}  // namespace

extern "C" {

int fkd_server_submit(fkd_server* S, int id, const uint8_t* frame, size_t pitch, int64_t arrival_ns) {
  return submit_frame(S, id, frame, pitch, arrival_ns, false);
}

int fkd_server_submit_ref(fkd_server* S, int id, const uint8_t* frame, size_t pitch, int64_t arrival_ns) {
  return submit_frame(S, id, frame, pitch, arrival_ns, true);
}

int fkd_server_keep_results(fkd_server* S, int keep) {
  if (!S) return set_error(FKD_E_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  S->keep_results = keep != 0;
  return FKD_OK;
}

int fkd_server_replay(fkd_server* S, int n, const int* ids, const uint8_t* const* frames, const size_t* pitches,
                      const int64_t* arrival_ns, uint64_t* refused) {
  if (!S || n < 0 || (n > 0 && (!ids || !frames || !pitches || !arrival_ns))) return set_error(FKD_E_ARG, "NULL argument");
  uint64_t dropped = 0;
  for (int i = 0; i < n; ++i) {
    if (i > 0 && arrival_ns[i] < arrival_ns[i - 1]) return set_error(FKD_E_ARG, "arrival times must not decrease");
    // wait for the arrival: sleep through long gaps, spin through short ones
    for (;;) {
      const int64_t left = arrival_ns[i] - now_ns();
      if (left <= 0) break;
      if (left > 200000) std::this_thread::sleep_for(std::chrono::nanoseconds(left - 100000));
    }
    const int rc = submit_frame(S, ids[i], frames[i], pitches[i], arrival_ns[i], true);
    if (rc == FKD_E_CAPACITY) {
      dropped += 1;
    } else if (rc) {
      if (refused) *refused = dropped;
      return rc;
    }
  }
  if (refused) *refused = dropped;
  return FKD_OK;
}

int fkd_server_poll(fkd_server* S, int id, int64_t* frame_index, fkd_keypoint* out, size_t cap, size_t* n_out) {
  if (!S || !n_out || (!out && cap > 0)) return set_error(FKD_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (id < 0 || id >= (int)S->streams.size() || !S->streams[id].open)
    return set_error(FKD_E_ARG, "unknown stream id %d", id);
  SStream& s = S->streams[id];
  if (s.results.empty()) {
    if (S->error) return worker_error(S);
    return set_error(FKD_E_STATE, "no finished frame of stream %d", id);
  }
  Result& r = s.results.front();
  *n_out = r.kp.size();
  if (frame_index) *frame_index = r.index;
  if (r.truncated) {
    s.results.pop_front();
    return set_error(FKD_E_CAPACITY, "frame %lld of stream %d exceeded K_max or the tick's capacity",
                     (long long)r.index, id);
  }
  if (r.kp.size() > cap) return set_error(FKD_E_CAPACITY, "%zu keypoints > cap %zu", r.kp.size(), cap);
  if (!r.kp.empty()) std::memcpy(out, r.kp.data(), r.kp.size() * sizeof(fkd_keypoint));
  if (s.D) {
    s.last_desc = std::move(r.desc);
    s.have_last = true;
  }
  s.results.pop_front();
  return FKD_OK;
}

int fkd_server_set_descriptor(fkd_server* S, int id, const int8_t* pattern, int D) {
  if (!S) return set_error(FKD_E_ARG, "server is NULL");
  std::lock_guard<std::mutex> lk(S->mu);
  if (S->error) return worker_error(S);
  if (id < 0 || id >= (int)S->streams.size() || !S->streams[id].open)
    return set_error(FKD_E_ARG, "unknown stream id %d", id);
  SStream& s = S->streams[id];
  if (s.taken > 0 || s.count > 0) return set_error(FKD_E_STATE, "set the descriptor of stream %d before its first frame", id);
  int rc = fkd_group_set_descriptor(S->G, id, pattern, D);
  if (rc) return rc;
  const size_t bytes = group_stream_bytes(S->G, id) + 2 * (size_t)s.pitch * s.H;
  if (S->used - s.bytes + bytes > S->budget) {
    fkd_group_set_descriptor(S->G, id, nullptr, 0);
    return set_error(FKD_E_BUDGET, "description needs %zu more bytes, %zu of %zu in use", bytes - s.bytes, S->used,
                     S->budget);
  }
  S->used = S->used - s.bytes + bytes;
  s.bytes = bytes;
  s.D = D;
  s.last_desc.clear();
  s.have_last = false;
  return FKD_OK;
}

int fkd_server_get_descriptors(fkd_server* S, int id, uint8_t* out, size_t cap, size_t* n_out) {
  if (!S || !n_out || (!out && cap > 0)) return set_error(FKD_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  if (id < 0 || id >= (int)S->streams.size() || !S->streams[id].open)
    return set_error(FKD_E_ARG, "unknown stream id %d", id);
  SStream& s = S->streams[id];
  if (!s.D) return set_error(FKD_E_STATE, "stream %d does not describe (fkd_server_set_descriptor)", id);
  if (!s.have_last) return set_error(FKD_E_STATE, "no result of stream %d polled yet", id);
  const size_t bytes = (size_t)s.D / 8, n = s.last_desc.size() / bytes;
  *n_out = n;
  const size_t ncopy = std::min(n, cap);
  if (ncopy) std::memcpy(out, s.last_desc.data(), ncopy * bytes);
  if (n > cap && out) return set_error(FKD_E_CAPACITY, "%zu descriptors > cap %zu", n, cap);
  return FKD_OK;
}

int fkd_server_drain(fkd_server* S, int timeout_ms) {
  if (!S) return set_error(FKD_E_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(S->mu);
  auto idle = [&] {
    if (S->error) return true;
    for (const auto& s : S->streams)
      if (s.open && s.count > 0) return false;
    return true;
  };
  if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle))
    return set_error(FKD_E_TIMEOUT, "frames still waiting after %d ms", timeout_ms);
  return S->error ? worker_error(S) : FKD_OK;
}

int fkd_server_get_stats(fkd_server* S, fkd_server_stats* out, int reset) {
  if (!S || !out) return set_error(FKD_E_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(S->mu);
  std::memset(out, 0, sizeof *out);
  out->frames_done = S->frames_done;
  out->ticks = S->ticks;
  out->rejected_frames = S->rejected_frames;
  out->rejected_streams = S->rejected_streams;
  out->mean_batch = S->ticks ? S->batch_sum / (double)S->ticks : 0.0;
  out->bytes_in_use = S->used;
  out->budget_bytes = S->budget;
  if (!S->lat_ms.empty()) {
    std::vector<double> v = S->lat_ms;
    std::sort(v.begin(), v.end());
    auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5))]; };
    out->p50_ms = pct(0.50);
    out->p99_ms = pct(0.99);
    out->max_ms = v.back();
    double sum = 0;
    for (double x : v) sum += x;
    out->mean_ms = sum / (double)v.size();
  }
  if (S->t_last > S->t_first) out->fps = (double)S->frames_done / ((S->t_last - S->t_first) * 1e-9);
  if (reset) {
    S->lat_ms.clear();
    S->frames_done = S->ticks = S->rejected_frames = S->rejected_streams = 0;
    S->batch_sum = 0;
    S->t_first = S->t_last = 0;
  }
  return FKD_OK;
}

}  // extern "C"
