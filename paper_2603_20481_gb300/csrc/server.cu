// Serving: chunks of IQ from many radio streams, batched as they arrive
// (continuous batching) and run through the path with rise_detect_batch.
//
// Lanes: each lane is a host thread with its own context (its own scratch
// and CUDA stream).  A free lane takes every pending chunk it can get a
// device slot for (up to max_batch), copies them in, and runs the batch while
// other lanes pick up what arrives meanwhile, so batches overlap on the GPU.
//
// Streams are continuous across chunks: the samples a chunk leaves unused
// (from its last frame start on, fewer than N) stay on the device in the
// stream's carry buffer and are put in front of the next chunk.
//
// Window mode (window_frames = W > 0) detects fixed TF plots of W frames, as
// the real-time design of Sec. IV-D does with its T-row ping-pong buffer:
// the samples of a stream accumulate across chunks, every W consecutive
// frames form one plot, and each complete plot is detected (its STFT
// included) as soon as the chunk that completes it arrives; what is left
// (fewer than W frames) is carried.  Results are then one per plot.  The carry
// update of one chunk and the carry read of the next are ordered by an event
// when they run on different lanes; the dispatch of chunks (slot
// assignment, copies, carry update) happens under the server lock, so the
// per-stream order of these operations is the submission order.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "context.cuh"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Chunk {
  int stream;
  const void *host;
  int64_t n;
  uint64_t tag;
  int64_t seq;
  int64_t t_submit;
};

struct StreamState {
  float2 *carry = nullptr;      // device: N samples, or a plot's span in window mode
  int64_t carry_len = 0;
  int64_t next_seq = 0;
  int64_t next_frame = 0;
  int64_t next_window = 0;      // window mode: number of the next plot
  int64_t busy = 0;             // chunks queued or in flight
  cudaEvent_t ready = nullptr;  // the last carry update
  bool has_event = false;
};

struct Done {
  rise_result r;
  std::vector<rise_box> boxes;
};

struct Lane {
  rise_ctx *ctx = nullptr;
  std::thread th;
  int64_t captures = 0, generations = 0, relabels = 0;   // copied from the context after each batch
};

constexpr uint32_t kStateMagic = 0x52534531u;   // stream state blob, version 1
struct StateHeader {
  uint32_t magic;
  int32_t fft_size, hop, window;
  int64_t carry_len, next_seq, next_frame, next_window;
};

}  // namespace

struct rise_server {
  int device = 0;
  int N = 0, hop = 0;
  int64_t max_chunk = 0;
  int max_batch = 32, max_pending = 4096;
  int64_t window = 0;     // frames per plot in window mode, else 0
  int64_t span = 0;       // samples of one plot: (window - 1) * hop + N
  int64_t carry_cap = 0;  // samples a stream's carry buffer holds
  rise_thresholds thr;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Chunk> pending;
  std::vector<StreamState> streams;
  std::vector<float2 *> slot_dev;
  std::vector<int> free_slots;
  std::deque<Done> done;
  std::vector<Lane> lanes;
  bool keep_images = false;
  struct Image {
    int64_t T = 0;
    std::vector<uint8_t> px;
  };
  std::map<std::pair<int, int64_t>, Image> images;   // (stream, seq) -> kept 8-bit image
  bool stop = false;
  int64_t running = 0;
  int64_t st_submitted = 0, st_rejected = 0, st_completed = 0, st_batches = 0, st_max_batch = 0,
          st_max_inflight = 0, st_max_batch_us = 0;
};

namespace {

constexpr int64_t kLaneBoxes = 1 << 18;   // a lane's first box buffer (doubled on demand)

// The largest batch a lane can be given: max_batch chunks, each with the
// longest carry, split into captures as lane_main splits them.
std::vector<rise_capture> largest_batch(const rise_server *s) {
  std::vector<rise_capture> caps;
  if (s->slot_dev.empty()) return caps;
  const int nslot = (int)s->slot_dev.size();
  for (int b = 0; b < s->max_batch; ++b) {
    float2 *dst = s->slot_dev[b % nslot];
    if (s->window == 0) {
      const int64_t len = s->max_chunk + s->N - 1;   // a chunk after a carry of N - 1 samples
      caps.push_back(rise_capture{dst, len, s->N, s->hop});
    } else {
      const int64_t step = s->window * s->hop;
      const int64_t k = 1 + (s->max_chunk - 1) / step;   // plots of a chunk after the longest carry
      for (int64_t j = 0; j < k; ++j) caps.push_back(rise_capture{dst + j * step, s->span, s->N, s->hop});
    }
  }
  return caps;
}

void lane_main(rise_server *s, int li) {
  cudaSetDevice(s->device);
  rise_ctx *ctx = s->lanes[li].ctx;
  cudaStream_t cs = ctx->stream;
  struct Item {
    Chunk ch;
    int slot;
    int64_t first_frame, frames;
    int cap_index;      // index in caps, -1 when the chunk holds no frame (no plot)
    int64_t n_windows;  // window mode: plots the chunk completes
    int64_t first_window;
  };
  std::vector<Item> items;
  std::vector<rise_capture> caps;
  std::vector<int64_t> offs;
  std::vector<rise_box> boxes(kLaneBoxes);   // grown (and the context's box buffer with it) on demand
  for (;;) {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_work.wait(lk, [&] { return s->stop || (!s->pending.empty() && !s->free_slots.empty()); });
    if (s->stop) return;
    items.clear();
    caps.clear();
    while (!s->pending.empty() && !s->free_slots.empty() && (int)items.size() < s->max_batch) {
      Item it;
      it.ch = s->pending.front();
      s->pending.pop_front();
      it.slot = s->free_slots.back();
      s->free_slots.pop_back();
      StreamState &st = s->streams[it.ch.stream];
      float2 *dst = s->slot_dev[it.slot];
      // capture = carried samples, then the new ones
      if (st.has_event) cudaStreamWaitEvent(cs, st.ready, 0);
      if (st.carry_len)
        cudaMemcpyAsync(dst, st.carry, st.carry_len * sizeof(float2), cudaMemcpyDeviceToDevice, cs);
      cudaMemcpyAsync(dst + st.carry_len, it.ch.host, it.ch.n * sizeof(float2), cudaMemcpyHostToDevice, cs);
      const int64_t len = st.carry_len + it.ch.n;
      it.cap_index = -1;
      it.n_windows = 0;
      it.first_window = st.next_window;
      int64_t used;   // samples before the first one the next unit needs
      if (s->window == 0) {
        const int64_t T = len >= s->N ? (len - s->N) / s->hop + 1 : 0;
        used = T * s->hop;   // the rest, from the next frame start on, is < N samples
        it.first_frame = st.next_frame;
        it.frames = T;
        st.next_frame += T;
        if (T > 0) {
          it.cap_index = (int)caps.size();
          caps.push_back(rise_capture{dst, len, s->N, s->hop});
        }
      } else {
        // every complete plot of W frames: samples [j W hop, j W hop + span)
        const int64_t step = s->window * s->hop;
        const int64_t k = len >= s->span ? 1 + (len - s->span) / step : 0;
        used = k * step;     // the rest holds fewer than W frames: < span samples
        it.first_frame = st.next_frame;
        it.frames = k * s->window;
        st.next_frame += k * s->window;
        it.n_windows = k;
        st.next_window += k;
        if (k > 0) it.cap_index = (int)caps.size();
        for (int64_t j = 0; j < k; ++j) caps.push_back(rise_capture{dst + j * step, s->span, s->N, s->hop});
      }
      const int64_t keep = len - used;
      if (keep)
        cudaMemcpyAsync(st.carry, dst + used, keep * sizeof(float2), cudaMemcpyDeviceToDevice, cs);
      cudaEventRecord(st.ready, cs);
      st.has_event = true;
      st.carry_len = keep;
      items.push_back(it);
    }
    s->running += (int64_t)items.size();
    s->st_max_inflight = std::max(s->st_max_inflight, s->running);
    s->st_max_batch = std::max<int64_t>(s->st_max_batch, (int64_t)items.size());
    lk.unlock();

    const int64_t t_start = now_ns();
    int rc = RISE_OK;
    offs.assign(caps.size() + 1, 0);
    if (!caps.empty()) {
      rc = rise_detect_batch(ctx, caps.data(), (int)caps.size(), &s->thr, boxes.data(),
                             (int64_t)boxes.size(), offs.data());
      if (rc == RISE_ETRUNC) {
        // more boxes than the buffer: grow it and run the batch again (the
        // slots still hold the inputs)
        boxes.resize((size_t)2 * offs.back() + 1024);
        rc = rise_detect_batch(ctx, caps.data(), (int)caps.size(), &s->thr, boxes.data(),
                               (int64_t)boxes.size(), offs.data());
      }
    } else {
      rise::host::wait_stream(ctx);   // the carry copies of frame-less chunks
    }
    const int64_t t_done = now_ns();
    // introspection: every capture's 8-bit image, back to back in batch order
    std::vector<uint8_t> imgs;
    std::vector<int64_t> img_off;
    if (s->keep_images && rc == RISE_OK && !caps.empty()) {
      img_off.assign(caps.size() + 1, 0);
      for (size_t c = 0; c < caps.size(); ++c)
        img_off[c + 1] = img_off[c] + ((caps[c].n - s->N) / s->hop + 1) * (int64_t)s->N;
      imgs.resize((size_t)img_off.back());
      if (rise_debug_export(ctx, RISE_DBG_BATCH_IMAGES, imgs.data(), imgs.size()) != RISE_OK) imgs.clear();
    }

    lk.lock();
    for (const Item &it : items) {
      // chunk mode: one result per chunk; window mode: one per completed plot
      const int64_t nres = s->window == 0 ? 1 : it.n_windows;
      for (int64_t j = 0; j < nres; ++j) {
        Done d;
        std::memset(&d.r, 0, sizeof(d.r));
        d.r.stream = it.ch.stream;
        d.r.status = rc;
        d.r.tag = it.ch.tag;
        d.r.seq = s->window == 0 ? it.ch.seq : it.first_window + j;
        d.r.first_frame = s->window == 0 ? it.first_frame : it.first_frame + j * s->window;
        d.r.frames = s->window == 0 ? it.frames : s->window;
        d.r.t_submit_ns = it.ch.t_submit;
        d.r.t_start_ns = t_start;
        d.r.t_done_ns = t_done;
        if (rc == RISE_OK && it.cap_index >= 0) {
          const int64_t b0 = offs[it.cap_index + j], b1 = offs[it.cap_index + j + 1];
          d.boxes.assign(boxes.begin() + b0, boxes.begin() + b1);
          if (!imgs.empty()) {
            const int64_t ci = it.cap_index + j;
            rise_server::Image &im = s->images[{d.r.stream, d.r.seq}];
            im.T = (img_off[ci + 1] - img_off[ci]) / s->N;
            im.px.assign(imgs.begin() + img_off[ci], imgs.begin() + img_off[ci + 1]);
          }
        }
        d.r.n_boxes = (int64_t)d.boxes.size();
        s->done.push_back(std::move(d));
      }
      s->free_slots.push_back(it.slot);
      s->streams[it.ch.stream].busy -= 1;
    }
    s->running -= (int64_t)items.size();
    s->st_completed += (int64_t)items.size();
    s->st_batches += 1;
    s->st_max_batch_us = std::max<int64_t>(s->st_max_batch_us, (t_done - t_start) / 1000);
    s->lanes[li].captures = ctx->batch.captures;
    s->lanes[li].generations = (int64_t)ctx->gen;
    s->lanes[li].relabels = ctx->batch.relabels;
    lk.unlock();
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

void free_server(rise_server *s) {
  cudaSetDevice(s->device);
  for (auto &L : s->lanes)
    if (L.ctx) rise_destroy(L.ctx);
  for (float2 *p : s->slot_dev) cudaFree(p);
  for (auto &st : s->streams) {
    if (st.carry) cudaFree(st.carry);
    if (st.ready) cudaEventDestroy(st.ready);
  }
  delete s;
}

}  // namespace

extern "C" {

int rise_server_create(rise_server **out, const rise_server_config *cfg) {
  using namespace rise::host;
  if (!out || !cfg) return RISE_EINVAL;
  *out = nullptr;
  const int N = cfg->fft_size, hop = cfg->hop;
  if (!pow2(N) || N < RISE_MIN_FFT || N > RISE_MAX_FFT || hop < 1 || hop > N) return RISE_EINVAL;
  if (cfg->max_chunk < 1 || cfg->max_streams < 1) return RISE_EINVAL;
  const int lanes = cfg->lanes > 0 ? cfg->lanes : 2;
  const int max_batch = cfg->max_batch > 0 ? cfg->max_batch : 32;
  if (lanes > 64 || max_batch > 4096) return RISE_EINVAL;
  const int64_t window = cfg->window_frames;
  if (window < 0 || window > RISE_BATCH_MAX_ROWS) return RISE_EINVAL;
  const int64_t span = window ? (window - 1) * (int64_t)hop + N : 0;
  const int64_t carry_cap = window ? span : N;           // the carry is always shorter
  const int64_t max_len = cfg->max_chunk + carry_cap;    // carried + new samples
  if ((max_len - N) / hop + 1 > RISE_BATCH_MAX_ROWS && window == 0) return RISE_EINVAL;
  rise_thresholds thr;
  if (cfg->thr) thr = *cfg->thr;
  else rise_thresholds_default(&thr);
  if (check_thresholds(thr, N)) return RISE_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return RISE_ECUDA;
  }
  if (cfg->device < 0 || cfg->device >= ndev) return RISE_EINVAL;
  if (cudaSetDevice(cfg->device) != cudaSuccess) return RISE_ECUDA;
  // memory admission: slots of (max_chunk + N) samples plus each lane's
  // scratch for a full batch (float power, levels, mask, run arrays)
  const size_t slot_bytes = (size_t)max_len * sizeof(float2);
  const size_t px = (size_t)((max_len - N) / hop + 1) * N;
  const size_t scratch = (size_t)max_batch * px * 6 + ((size_t)80 << 20);
  int64_t slots = (int64_t)lanes * max_batch;
  if (cfg->mem_budget) {
    if (cfg->mem_budget < (size_t)lanes * (scratch + slot_bytes)) return RISE_ENOMEM;
    slots = std::min<int64_t>(slots, (int64_t)((cfg->mem_budget - lanes * scratch) / slot_bytes));
  }
  rise_server *s = new (std::nothrow) rise_server();
  if (!s) return RISE_ENOMEM;
  s->device = cfg->device;
  s->N = N;
  s->hop = hop;
  s->max_chunk = cfg->max_chunk;
  s->window = window;
  s->span = span;
  s->carry_cap = carry_cap;
  s->max_batch = max_batch;
  s->max_pending = cfg->max_pending > 0 ? cfg->max_pending : 4096;
  s->thr = thr;
  s->keep_images = cfg->keep_images != 0;
  int rc = RISE_OK;
  s->streams.resize(cfg->max_streams);
  for (auto &st : s->streams) {
    if (cudaMalloc(&st.carry, (size_t)carry_cap * sizeof(float2)) != cudaSuccess) { rc = RISE_ENOMEM; break; }
    if (cudaEventCreateWithFlags(&st.ready, cudaEventDisableTiming) != cudaSuccess) { rc = RISE_ECUDA; break; }
  }
  for (int64_t k = 0; k < slots && rc == RISE_OK; ++k) {
    float2 *p = nullptr;
    if (cudaMalloc(&p, slot_bytes) != cudaSuccess) { rc = RISE_ENOMEM; break; }
    s->slot_dev.push_back(p);
    s->free_slots.push_back((int)k);
  }
  s->lanes.resize(lanes);
  for (int li = 0; li < lanes && rc == RISE_OK; ++li) {
    rise_config cc{};
    cc.device = cfg->device;
    cc.mem_budget = cfg->mem_budget ? scratch + scratch / 2 : 0;
    if ((rc = rise_create(&s->lanes[li].ctx, &cc))) break;
    rise_set_option(s->lanes[li].ctx, RISE_OPT_AUTOTUNE, 0);   // batch sizes vary: fixed shapes
    rise_set_option(s->lanes[li].ctx, RISE_OPT_BLOCKING_WAIT, cfg->spin_wait ? 0 : 1);
    // window mode: plain launches (its batch compositions are many and a
    // capture inside a deadline costs more than the launches it saves)
    if (s->window) rise_set_option(s->lanes[li].ctx, RISE_OPT_GRAPH, 0);
  }
  if (rc == RISE_OK) {
    // every lane's buffers sized for its largest batch now: a lane that grew
    // while serving (a burst after a stall fills batches beyond any seen
    // before) would synchronise the device in the middle of the stream.
    // Best effort: a lane that cannot reserve grows on demand as before.
    const std::vector<rise_capture> worst = largest_batch(s);
    for (int li = 0; li < lanes && !worst.empty(); ++li)
      if (reserve_batch(s->lanes[li].ctx, worst.data(), (int)worst.size(), s->thr, kLaneBoxes) != RISE_OK)
        cudaGetLastError();
  }
  if (rc) {
    cudaGetLastError();
    free_server(s);
    return rc;
  }
  for (int li = 0; li < lanes; ++li) s->lanes[li].th = std::thread(lane_main, s, li);
  *out = s;
  return RISE_OK;
}

int rise_stream_submit(rise_server *s, int stream, const void *iq_host, int64_t n, uint64_t tag) {
  if (!s || !iq_host || stream < 0 || stream >= (int)s->streams.size() || n < 1 || n > s->max_chunk)
    return RISE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  if ((int64_t)s->pending.size() >= s->max_pending) {
    s->st_rejected += 1;
    return RISE_EAGAIN;
  }
  StreamState &st = s->streams[stream];
  s->pending.push_back(Chunk{stream, iq_host, n, tag, st.next_seq++, now_ns()});
  st.busy += 1;
  s->st_submitted += 1;
  s->cv_work.notify_one();
  return RISE_OK;
}

int rise_server_poll(rise_server *s, rise_result *res, int max_res, rise_box *arena, int64_t arena_cap,
                     int *n_res, int timeout_ms) {
  if (!s || !n_res || max_res < 0 || arena_cap < 0 || (max_res > 0 && !res) || (arena_cap > 0 && !arena))
    return RISE_EINVAL;
  *n_res = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  auto ready = [&] { return !s->done.empty(); };
  if (timeout_ms < 0) s->cv_done.wait(lk, ready);
  else if (timeout_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  int64_t used = 0;
  int k = 0;
  while (k < max_res && !s->done.empty()) {
    Done &d = s->done.front();
    const int64_t nb = (int64_t)d.boxes.size();
    rise_result r = d.r;
    if (used + nb > arena_cap) {
      if (k > 0) break;           // leave it for the next poll
      r.status = RISE_ETRUNC;     // alone and still too large: first arena_cap boxes
      r.n_boxes = arena_cap;
    }
    r.box_offset = used;
    const int64_t ncopy = std::min(nb, arena_cap - used);
    if (ncopy > 0) std::memcpy(arena + used, d.boxes.data(), (size_t)ncopy * sizeof(rise_box));
    used += ncopy;
    res[k++] = r;
    s->done.pop_front();
  }
  *n_res = k;
  return RISE_OK;
}

int rise_server_drain(rise_server *s, int timeout_ms) {
  if (!s) return RISE_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  auto idle = [&] { return s->pending.empty() && s->running == 0; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, idle);
    return RISE_OK;
  }
  return s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), idle) ? RISE_OK : RISE_ETIMEOUT;
}

int rise_stream_export(rise_server *s, int stream, void *buf, size_t bytes, size_t *need) {
  if (!s || stream < 0 || stream >= (int)s->streams.size()) return RISE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  StreamState &st = s->streams[stream];
  const size_t total = sizeof(StateHeader) + (size_t)st.carry_len * sizeof(float2);
  if (need) *need = total;
  if (!buf) return RISE_OK;
  if (st.busy != 0 || bytes < total) return RISE_EINVAL;
  StateHeader h{kStateMagic, s->N, s->hop, (int32_t)s->window, st.carry_len, st.next_seq,
                st.next_frame, st.next_window};
  std::memcpy(buf, &h, sizeof h);
  cudaSetDevice(s->device);
  if (st.has_event && cudaEventSynchronize(st.ready) != cudaSuccess) return RISE_ECUDA;
  if (st.carry_len &&
      cudaMemcpy(static_cast<char *>(buf) + sizeof h, st.carry, (size_t)st.carry_len * sizeof(float2),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return RISE_ECUDA;
  return RISE_OK;
}

int rise_stream_import(rise_server *s, int stream, const void *buf, size_t bytes) {
  if (!s || !buf || stream < 0 || stream >= (int)s->streams.size() || bytes < sizeof(StateHeader))
    return RISE_EINVAL;
  StateHeader h;
  std::memcpy(&h, buf, sizeof h);
  if (h.magic != kStateMagic || h.fft_size != s->N || h.hop != s->hop || h.window != s->window ||
      h.carry_len < 0 || h.carry_len >= s->carry_cap ||
      bytes < sizeof h + (size_t)h.carry_len * sizeof(float2))
    return RISE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  StreamState &st = s->streams[stream];
  if (st.busy != 0) return RISE_EINVAL;
  cudaSetDevice(s->device);
  if (st.has_event && cudaEventSynchronize(st.ready) != cudaSuccess) return RISE_ECUDA;
  if (h.carry_len &&
      cudaMemcpy(st.carry, static_cast<const char *>(buf) + sizeof h, (size_t)h.carry_len * sizeof(float2),
                 cudaMemcpyHostToDevice) != cudaSuccess)
    return RISE_ECUDA;
  st.carry_len = h.carry_len;
  st.next_seq = h.next_seq;
  st.next_frame = h.next_frame;
  st.next_window = h.next_window;
  st.has_event = false;
  return RISE_OK;
}

int rise_server_result_image(rise_server *s, int stream, int64_t seq, uint8_t *dst, size_t bytes,
                             int64_t *T) {
  if (!s || !T) return RISE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->images.find({stream, seq});
  if (it == s->images.end()) return RISE_EINVAL;
  *T = it->second.T;
  if (!dst) return RISE_OK;
  if (bytes < it->second.px.size()) return RISE_EINVAL;
  std::memcpy(dst, it->second.px.data(), it->second.px.size());
  s->images.erase(it);
  return RISE_OK;
}

int rise_server_stats(rise_server *s, int64_t *out, int n) {
  if (!s || !out || n < 0) return RISE_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  int64_t captures = 0, generations = 0, relabels = 0;
  for (const Lane &L : s->lanes) {
    captures += L.captures;
    generations += L.generations;
    relabels += L.relabels;
  }
  const int64_t w[12] = {s->st_submitted, s->st_rejected, s->st_completed, s->st_batches,
                         s->st_max_batch, s->st_max_inflight, (int64_t)s->slot_dev.size(),
                         (int64_t)s->lanes.size(), captures, generations, s->st_max_batch_us, relabels};
  for (int i = 0; i < n && i < 12; ++i) out[i] = w[i];
  return RISE_OK;
}

void rise_server_destroy(rise_server *s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto &L : s->lanes)
    if (L.th.joinable()) L.th.join();
  free_server(s);
}

}  // extern "C"
