// Private to the library: the context behind the opaque rise_ctx handle and
// the host helpers the entry points share (device scratch, tables, checks).
#pragma once

#include <cmath>
#include <map>
#include <vector>

#include "common.cuh"

namespace rise {
namespace host {

struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
};

// Per-FFT-size and radix-schedule tables (twiddles + Hann window), built once.
struct Tables {
  float2 *tw = nullptr;
  float *win = nullptr;
  int sched = 0;
};

struct Small {              // one device block of small per-call data
  DeviceStatus status;
  float edges[260];
  float qconst[4];
  int64_t floor_out[8];
  int64_t sgc[32];
  uint64_t energy[256];
  double ratio[256];   // 10^((j - 255.5) level_db / 10), j = 0..255
};

// Per-call tables of a batch: host staging (pinned) and device copy.
struct BatchState {
  Buf tab;                       // device blob of per-capture tables
  void *tab_h = nullptr;         // pinned host staging of the same blob
  size_t tab_h_bytes = 0;
  Buf small;                     // CapSmall[ncap]
  Buf counters;                  // int work counters of persistent launches
  int64_t *offs_h = nullptr;     // mapped pinned [ncap + 1] box offsets
  int64_t *offs_dev = nullptr;
  int64_t offs_cap = 0;
  // captured launch sequences, keyed by the batch's composition
  struct Graph {
    uint64_t key = 0;
    cudaGraphExec_t exec = nullptr;
    int launches = 0;            // kernels one replay runs
  };
  std::vector<Graph> graphs;
  std::vector<uint64_t> seen;    // compositions run once without a graph
  // tuned launch parameters, keyed by the batch's shape
  std::map<uint64_t, std::vector<int>> tuned;
  int64_t captures = 0;          // launch chains captured so far
  int64_t cache_hits = 0;        // compositions whose launch parameters came from the tune cache
  int64_t relabels = 0;          // batches run again with grown run arrays
  // the last batch: STFT groups, its launch parameters, replayed from a graph
  int last_groups = 0;
  std::vector<int> last_params;
  bool last_graph = false;
  // what the last batch left in the context's buffers, for rise_debug_export:
  // its captures' images (and float power) back to back, and their anchors
  bool last_valid = false;
  bool last_fixed = false;
  int last_ncap = 0;
  int64_t last_px = 0;
  double last_hi_db = 0.0;
};

// One call in flight: where its boxes, status and stage events land, and
// (for a host capture) the device copy of its samples.  Two slots let the
// next call be queued, and its samples copied in, while this one runs.
struct CallSlot {
  rise_box *hbox = nullptr;      // mapped pinned host buffer the compaction writes into
  rise_box *hbox_dev = nullptr;  // its device address
  int64_t hbox_cap = 0;
  DeviceStatus *st_h = nullptr;  // pinned, mapped status readback
  DeviceStatus *st_d = nullptr;  // its device address
  cudaEvent_t ev[8] = {};        // stage events
  cudaEvent_t done = nullptr;    // the call's work has finished
  cudaEvent_t copied = nullptr;  // its host samples are on the device
  Buf iq;                        // device copy of a host capture
  bool pending = false;
  // the queued call, kept to run it again if its run arrays overflow
  const void *src = nullptr;
  int64_t n = 0, T = 0, cap = 0;
  int N = 0, hop = 0, path = 0, fmt = 0, sched = 0;
  bool want_power = false;
  rise_thresholds thr{};
};

}  // namespace host
}  // namespace rise

struct rise_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t mem_budget = 0;
  size_t allocated = 0;
  int num_sms = 1;
  // options
  int keep_power = 0, keep_masks = 0, timing = 0, range_path = 0;
  int graphs = 1, autotune = 1;
  // bounds of the device waits (defaults of the kernels) and the test-only
  // withheld root-scan tile (-1: none)
  int spin_limit = rise::SCAN_SPIN_LIMIT, uf_limit = rise::UF_LIMIT;
  int64_t withhold_tile = -1;
  int copy_wait_limit = rise::STFT_WAIT_LIMIT;   // RISE_OPT_COPY_WAIT_LIMIT
  int64_t withhold_copy = -1;                    // RISE_OPT_TEST_WITHHOLD_COPY
  bool blocking_wait = false;                    // RISE_OPT_BLOCKING_WAIT
  cudaEvent_t wait_ev = nullptr;                 // blocking-sync event for it
  // radix schedule of single captures: 0 or 1 (default), or -1: the one the
  // batch tuner (or the tune cache) picked for the FFT size, else 1
  int fft_sched = 3;   // RISE_OPT_FFT_SCHEDULE: the library's schedule per size
  std::map<int, int> sched_pick;   // FFT size -> schedule picked by the batch tuner
  bool capturing = false;         // enqueueing into a graph capture
  // scratch
  rise::host::Buf power, img, hist, cols, effm1, mask, dbg[3], row_cnt, row_base, run_parent,
      run_sroot, rec, run_out, scan_tmp, boxes, merge, match_boxes, match_best, match_misc,
      contour;
  int64_t run_cap = 0;
  int64_t run_cap_req = 0;             // capacity asked for by RISE_OPT_RUN_CAPACITY
  rise::host::Small *small = nullptr;   // device
  // calls in flight: slots, queue order, the stream host captures are copied on
  rise::host::CallSlot slot[2];
  int cur = 0;                          // slot of the call being enqueued or finished
  int pend[2] = {0, 0};
  int npend = 0, next_slot = 0;
  cudaStream_t copy_stream = nullptr;
  rise::host::CallSlot &cs() { return slot[cur]; }
  const rise::DeviceStatus *last_status = nullptr;   // status of the last finished call
  std::map<int, rise::host::Tables> tables;   // key: FFT size * 4 + schedule
  double energy_level_db = NAN;
  int sg_m = -1;
  // last call
  int64_t last_T = 0;
  int last_F = 0;
  const uint8_t *last_img = nullptr;
  bool last_has_power = false, last_has_masks = false, last_valid = false;
  double last_anchor = 0.0;
  float stage_ms[8] = {};
  uint64_t gen = 0;              // bumped whenever a scratch buffer moves
  uint64_t last_key[2] = {0, 0}; // arguments of the last call in each slot
  bool last_replayed = false;    // the last single-capture call replayed a graph
  std::vector<rise::host::BatchState::Graph> single_graphs;
  rise::host::BatchState batch;
};

namespace rise {
namespace host {

inline int cuda_fail(cudaError_t e) {
  return e == cudaErrorMemoryAllocation ? RISE_ENOMEM : RISE_ECUDA;
}

#define CK(expr)                              \
  do {                                        \
    cudaError_t _e = (expr);                  \
    if (_e != cudaSuccess) return rise::host::cuda_fail(_e); \
  } while (0)

// A scratch buffer moved: bumps the buffer generation and drops every
// captured graph (each holds old addresses and can never be replayed),
// after the context's stream is idle.
void new_generation(rise_ctx *c);
// Grows b to at least `bytes` (with 1/8 headroom), within the memory budget.
int ensure(rise_ctx *c, Buf &b, size_t bytes);
// Mapped pinned host buffer for the current slot's boxes (at least `cap`).
int ensure_hbox(rise_ctx *c, int64_t cap);
// Twiddle and window tables of FFT size N and radix schedule S (built once
// per context).
int get_tables(rise_ctx *c, int N, int S, Tables **out);
// The radix schedule a single capture of FFT size N runs.
int single_sched(const rise_ctx *c, int N);
// Waits for the context's stream: spinning (the runtime's default for one
// context) or, with RISE_OPT_BLOCKING_WAIT, asleep on a blocking-sync event.
cudaError_t wait_stream(rise_ctx *c);
// True when an STFT test hook is set (RISE_OPT_COPY_WAIT_LIMIT not at its
// default, or RISE_OPT_TEST_WITHHOLD_COPY >= 0): the float-power STFT then
// runs its hooked instance (StftMode STFT_POWER_HOOKED).
inline bool stft_hooks_on(const rise_ctx *c) {
  return c->copy_wait_limit != rise::STFT_WAIT_LIMIT || c->withhold_copy >= 0;
}
bool pow2(int64_t v);
int check_thresholds(const rise_thresholds &t, int F);
void record(rise_ctx *c, int i);
// Energy and level-edge ratio tables of level_db (uploaded when it changes).
int upload_level_tables(rise_ctx *c, double level_db);
// The Savitzky-Golay weights of half window m (uploaded when m changes).
int upload_sg(rise_ctx *c, int m);
void destroy_batch(rise_ctx *c);
int detect_batch(rise_ctx *c, const rise_capture *caps, int ncap, const rise_thresholds *thr,
                 rise_box *out, int64_t cap, int64_t *offsets);
// Grows every buffer of the batch path to what a batch of these captures
// (and box capacity `cap`) needs, launching nothing: a caller that knows its
// largest batch reserves it once, so that no later batch of that size or
// less allocates (an allocation synchronises the device and drops graphs).
int reserve_batch(rise_ctx *c, const rise_capture *caps, int ncap, const rise_thresholds &thr,
                  int64_t cap);

}  // namespace host
}  // namespace rise
