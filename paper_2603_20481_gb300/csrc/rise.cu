// Host side of the RISE library: the context, its device scratch, the
// stage sequence of one detection and the exported C ABI (include/rise.h).
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <set>
#include <map>
#include <new>
#include <vector>

#include "context.cuh"

using namespace rise;

namespace rise {
static std::atomic<long long> g_launches{0};
void count_launches(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches_so_far() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace rise

namespace rise {
namespace host {
int ensure(rise_ctx *c, Buf &b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (b.bytes >= bytes) return RISE_OK;
  size_t grow = bytes + bytes / 8;
  if (c->mem_budget && c->allocated - b.bytes + grow > c->mem_budget) {
    grow = bytes;
    if (c->allocated - b.bytes + grow > c->mem_budget) return RISE_ENOMEM;
  }
  if (b.p) {
    CK(cudaStreamSynchronize(c->stream));
    cudaFree(b.p);
    c->allocated -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
  }
  void *p = nullptr;
  cudaError_t e = cudaMalloc(&p, grow);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return RISE_ENOMEM;
  }
  b.p = p;
  b.bytes = grow;
  c->allocated += grow;
  new_generation(c);
  return RISE_OK;
}

void new_generation(rise_ctx *c) {
  ++c->gen;
  c->batch.last_valid = false;   // a moved buffer lost the last batch's intermediates
  cudaStreamSynchronize(c->stream);
  for (auto &g : c->single_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->single_graphs.clear();
  c->last_key[0] = c->last_key[1] = 0;
  for (auto &g : c->batch.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->batch.graphs.clear();
  c->batch.seen.clear();
}

// Mapped pinned host buffer for the boxes (grown to at least `cap` entries).
int ensure_hbox(rise_ctx *c, int64_t cap) {
  if (c->cs().hbox_cap >= cap) return RISE_OK;
  if (c->cs().hbox) {
    CK(cudaStreamSynchronize(c->stream));
    cudaFreeHost(c->cs().hbox);
    c->cs().hbox = nullptr;
    c->cs().hbox_dev = nullptr;
    c->cs().hbox_cap = 0;
  }
  // doubled: every move of this buffer drops the context's graphs
  const int64_t want = std::max<int64_t>(2 * cap, 4096);
  void *h = nullptr;
  if (cudaHostAlloc(&h, (size_t)want * sizeof(rise_box), cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return RISE_ENOMEM;
  }
  void *d = nullptr;
  if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(h);
    return RISE_ECUDA;
  }
  c->cs().hbox = reinterpret_cast<rise_box *>(h);
  c->cs().hbox_dev = reinterpret_cast<rise_box *>(d);
  c->cs().hbox_cap = want;
  new_generation(c);
  return RISE_OK;
}

int get_tables(rise_ctx *c, int N, int S, Tables **out) {
  if (!stft_sched_distinct(N, S)) S = 0;
  const int key = N * 4 + S;
  auto it = c->tables.find(key);
  if (it != c->tables.end()) {
    *out = &it->second;
    return RISE_OK;
  }
  const size_t nf = stft_table_floats(N, S);
  std::vector<float> host(nf);
  const size_t ntw = (nf - N) / 2;
  stft_fill_tables(N, S, reinterpret_cast<float2 *>(host.data()), host.data() + 2 * ntw);
  void *d = nullptr;
  if (cudaMalloc(&d, nf * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return RISE_ENOMEM;
  }
  CK(cudaMemcpy(d, host.data(), nf * sizeof(float), cudaMemcpyHostToDevice));
  Tables t;
  t.tw = reinterpret_cast<float2 *>(d);
  t.win = reinterpret_cast<float *>(d) + 2 * ntw;
  t.sched = S;
  c->tables[key] = t;
  *out = &c->tables[key];
  return RISE_OK;
}

cudaError_t wait_stream(rise_ctx *c) {
  if (!c->blocking_wait) return cudaStreamSynchronize(c->stream);
  if (!c->wait_ev) {
    const cudaError_t e = cudaEventCreateWithFlags(&c->wait_ev, cudaEventBlockingSync | cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
  }
  const cudaError_t e = cudaEventRecord(c->wait_ev, c->stream);
  return e != cudaSuccess ? e : cudaEventSynchronize(c->wait_ev);
}

int single_sched(const rise_ctx *c, int N) {
  int S = c->fft_sched;
  if (S < 0) {
    auto it = c->sched_pick.find(N);
    S = it == c->sched_pick.end() ? 3 : it->second;
  }
  if (S == 3) S = stft_default_sched(N);
  return stft_sched_distinct(N, S) ? S : 0;
}

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }

int check_thresholds(const rise_thresholds &t, int F) {
  // level widths from 0.01 to 10 dB: the fast level estimate's error stays
  // below 1.5e-4 levels there, inside the exact-comparison guard band
  if (!(t.level_db >= 0.01 && t.level_db <= 10.0)) return RISE_EINVAL;
  if (t.range_mode != RISE_RANGE_AUTO_MAX && t.range_mode != RISE_RANGE_FIXED) return RISE_EINVAL;
  if (t.range_mode == RISE_RANGE_FIXED && !std::isfinite(t.hi_db)) return RISE_EINVAL;
  if (std::isnan(t.psd_offset_db) || std::isnan(t.power_offset_db)) return RISE_EINVAL;
  if (std::isinf(t.psd_offset_db) && t.psd_offset_db > 0) return RISE_EINVAL;
  if (std::isinf(t.power_offset_db) && t.power_offset_db > 0) return RISE_EINVAL;
  if (t.sg_half_window < 1 || t.sg_half_window > 16 || F < 2 * t.sg_half_window + 3) return RISE_EINVAL;
  if (t.morph_order != 0 && t.morph_order != 1) return RISE_EINVAL;
  return RISE_OK;
}

void record(rise_ctx *c, int i) {
  // inside a capture the event must become an event-record node
  if (c->timing)
    cudaEventRecordWithFlags(c->cs().ev[i], c->stream, c->capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
}

// Per-level tables that depend only on level_db: the energy of each level
// (round(2^32 * 10^((q-255) level_db/10))) and the power ratio of each level
// edge (10^((j-255.5) level_db/10)).
int upload_level_tables(rise_ctx *c, double level_db) {
  if (c->energy_level_db == level_db) return RISE_OK;
  uint64_t E[256];
  double R[256];
  for (int q = 0; q < 256; ++q) {
    E[q] = (uint64_t)std::llround(std::exp2(32.0) * std::pow(10.0, (double)(q - 255) * level_db / 10.0));
    R[q] = std::pow(10.0, ((double)q - 255.5) * level_db / 10.0);
  }
  CK(cudaMemcpyAsync(c->small->energy, E, sizeof(E), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->small->ratio, R, sizeof(R), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->energy_level_db = level_db;
  return RISE_OK;
}

// Integer Savitzky-Golay weights of the quadratic fit over 2m+1 points:
// c_i = 3(3m^2 + 3m - 1) - 15 i^2, norm D = (2m-1)(2m+1)(2m+3).
int upload_sg(rise_ctx *c, int m) {
  if (c->sg_m == m) return RISE_OK;
  int64_t coef[32];
  for (int i = 0; i <= m; ++i) coef[i] = 3LL * (3LL * m * m + 3LL * m - 1) - 15LL * i * i;
  CK(cudaMemcpyAsync(c->small->sgc, coef, sizeof(int64_t) * (m + 1), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->sg_m = m;
  return RISE_OK;
}

}  // namespace host
}  // namespace rise

using namespace rise::host;

namespace {

CclArgs ccl_args(rise_ctx *c, const uint8_t *img, int64_t T, int F, int64_t cap) {
  CclArgs la;
  la.mask = reinterpret_cast<const uint32_t *>(c->mask.p);
  la.img = img;
  la.T = T;
  la.F = F;
  la.energy = c->small->energy;
  la.row_base = reinterpret_cast<int64_t *>(c->row_base.p);
  la.row_cnt = reinterpret_cast<uint32_t *>(c->row_cnt.p);
  la.status = &c->small->status;
  la.status_out = c->cs().st_d;   // the status lands in mapped pinned host memory too
  la.boxes = c->cs().hbox_dev;   // boxes land directly in mapped pinned host memory
  la.box_cap = cap;
  la.run_cap = c->run_cap;
  la.run_parent = reinterpret_cast<int32_t *>(c->run_parent.p);
  la.run_sroot = reinterpret_cast<uint8_t *>(c->run_sroot.p);
  la.rec = reinterpret_cast<rise_box *>(c->rec.p);
  la.merge = reinterpret_cast<int2 *>(c->merge.p);
  la.run_out = reinterpret_cast<int64_t *>(c->run_out.p);
  la.scan_tmp = c->scan_tmp.p;
  la.scan_tmp_bytes = c->scan_tmp.bytes;
  la.uf_limit = c->uf_limit;
  la.spin_limit = c->spin_limit;
  la.withhold_tile = c->withhold_tile;
  return la;
}

// Host-side set-up of the image part (may allocate or synchronise, so it
// runs before any launch is enqueued).
int image_prepare(rise_ctx *c, const rise_thresholds &thr, int64_t cap) {
  int rc;
  if ((rc = upload_sg(c, thr.sg_half_window))) return rc;
  if ((rc = upload_level_tables(c, thr.level_db))) return rc;
  return ensure_hbox(c, std::max<int64_t>(cap, 1));
}

// Launches of everything from the 8-bit image on: histogram (unless already
// built), column statistics, morphology, labelling, status readback.
// Asynchronous only: it can be captured into a graph.
int image_enqueue(rise_ctx *c, const uint8_t *img, int64_t T, int F, const rise_thresholds &thr,
                  bool hist_ready, int64_t cap) {
  Small *sm = c->small;
  cudaStream_t s = c->stream;
  if (!hist_ready) {
    if (cluster_hist_accumulates(T))
      CK(cudaMemsetAsync(c->hist.p, 0, (size_t)F * 256 * sizeof(uint32_t), s));
    CK(launch_cluster_hist(img, false, T, F, nullptr, nullptr, nullptr,
                           reinterpret_cast<uint32_t *>(c->hist.p),
                           reinterpret_cast<rise_colstat *>(c->cols.p), nullptr, s));
  }
  record(c, 3);
  // column statistics
  const int m = thr.sg_half_window;
  const int64_t D = (int64_t)(2 * m - 1) * (2 * m + 1) * (2 * m + 3);
  ColArgs ca;
  ca.hist = reinterpret_cast<const uint32_t *>(c->hist.p);
  ca.T = T;
  ca.F = F;
  ca.m = m;
  ca.D = D;
  ca.sg_c = sm->sgc;
  ca.psd_on = !(std::isinf(thr.psd_offset_db) && thr.psd_offset_db < 0);
  ca.pow_on = !(std::isinf(thr.power_offset_db) && thr.power_offset_db < 0);
  const double DT = (double)(D * T);
  ca.delta_psd = ca.psd_on ? (int64_t)std::llround(thr.psd_offset_db / thr.level_db * DT) : 0;
  ca.delta_pow = ca.pow_on ? (int64_t)std::llround(thr.power_offset_db / thr.level_db * DT) : 0;
  ca.cols = reinterpret_cast<rise_colstat *>(c->cols.p);
  ca.effm1 = reinterpret_cast<uint8_t *>(c->effm1.p);
  ca.floor_out = sm->floor_out;
  ca.st = &sm->status;   // zeroed at the start of the call
  CK(launch_colstats(ca, cluster_hist_accumulates(T), s));
  record(c, 4);
  // mask + morphology
  MorphArgs ma;
  ma.img = img;
  ma.effm1 = ca.effm1;
  ma.T = T;
  ma.F = F;
  ma.order = thr.morph_order;
  ma.mask = reinterpret_cast<uint32_t *>(c->mask.p);
  ma.dbg0 = c->keep_masks ? reinterpret_cast<uint32_t *>(c->dbg[0].p) : nullptr;
  ma.dbg1 = c->keep_masks ? reinterpret_cast<uint32_t *>(c->dbg[1].p) : nullptr;
  ma.dbg2 = c->keep_masks ? reinterpret_cast<uint32_t *>(c->dbg[2].p) : nullptr;
  ma.row_cnt = reinterpret_cast<uint32_t *>(c->row_cnt.p);
  CK(cudaMemsetAsync(c->row_cnt.p, 0, (size_t)T * sizeof(uint32_t), s));
  CK(launch_morph(ma, s));
  record(c, 5);
  // labelling
  const CclArgs la = ccl_args(c, img, T, F, cap);
  CK(launch_ccl_count(la, c->num_sms, s));
  CK(launch_ccl_label(la, c->num_sms, s));   // its last kernel hands the status to the host
  record(c, 6);
  record(c, 7);
  return RISE_OK;
}

// Waits for the enqueued work, relabels with larger run arrays when they
// were too small, and copies the boxes out.
int image_finish(rise_ctx *c, const uint8_t *img, int64_t T, int F, rise_box *out, int64_t cap,
                 int64_t *n_boxes) {
  Small *sm = c->small;
  cudaStream_t s = c->stream;
  int rc;
  CK(cudaStreamSynchronize(s));
  DeviceStatus h = (*c->cs().st_h);
  if (h.err & ERR_RUN_CAPACITY) {
    // the run arrays were too small for this mask: grow to fit and relabel
    int64_t need = std::max<int64_t>(2 * h.n_runs, 2 * c->run_cap);   // doubled: few growths
    if ((rc = ensure(c, c->run_parent, need * sizeof(int32_t)))) return rc;
    if ((rc = ensure(c, c->run_sroot, need))) return rc;
    if ((rc = ensure(c, c->rec, need * sizeof(rise_box)))) return rc;
    if ((rc = ensure(c, c->merge, need * sizeof(int2)))) return rc;
    if ((rc = ensure(c, c->run_out, (need + 1) * sizeof(int64_t)))) return rc;
    if ((rc = ensure(c, c->scan_tmp, ccl_scan_tmp_bytes(std::max<int64_t>(need, T + 1))))) return rc;
    c->run_cap = need;
    const CclArgs la = ccl_args(c, img, T, F, cap);
    CK(cudaMemsetAsync(&sm->status.err, 0, sizeof(uint32_t), s));
    CK(launch_ccl_label(la, c->num_sms, s, false));   // the row scan is not run again
    record(c, 6);
    record(c, 7);
    CK(cudaStreamSynchronize(s));
    h = (*c->cs().st_h);
  }
  c->last_status = c->cs().st_h;
  if (h.err & (ERR_UNION_LIMIT | ERR_SCAN | ERR_COPY_WAIT)) return RISE_ETIMEOUT;
  if (h.err) return RISE_EINTERNAL;
  *n_boxes = h.n_boxes;
  const int64_t ncopy = std::min<int64_t>(h.n_boxes, cap);
  if (ncopy > 0 && out) std::memcpy(out, c->cs().hbox, (size_t)ncopy * sizeof(rise_box));
  if (c->timing) {
    for (int i = 0; i < 7; ++i) cudaEventElapsedTime(&c->stage_ms[i], c->cs().ev[i], c->cs().ev[i + 1]);
    cudaEventElapsedTime(&c->stage_ms[7], c->cs().ev[0], c->cs().ev[7]);
  }
  return h.n_boxes > cap ? RISE_ETRUNC : RISE_OK;
}

int prepare_image_buffers(rise_ctx *c, int64_t T, int F) {
  int rc;
  const size_t px = (size_t)T * F;
  if ((rc = ensure(c, c->hist, (size_t)F * 256 * sizeof(uint32_t)))) return rc;
  if ((rc = ensure(c, c->cols, (size_t)F * sizeof(rise_colstat)))) return rc;
  if ((rc = ensure(c, c->effm1, (size_t)F))) return rc;
  if ((rc = ensure(c, c->mask, px / 8))) return rc;
  if (c->keep_masks)
    for (auto &d : c->dbg)
      if ((rc = ensure(c, d, px / 8))) return rc;
  if ((rc = ensure(c, c->row_cnt, (size_t)T * sizeof(uint32_t)))) return rc;
  if ((rc = ensure(c, c->row_base, (size_t)(T + 1) * sizeof(int64_t)))) return rc;
  if (c->run_cap_req) {
    // a capacity asked for by the caller, once (the arrays still grow on overflow)
    const int64_t want = c->run_cap_req;
    c->run_cap_req = 0;
    if ((rc = ensure(c, c->run_parent, want * sizeof(int32_t)))) return rc;
    if ((rc = ensure(c, c->run_sroot, want))) return rc;
    if ((rc = ensure(c, c->rec, want * sizeof(rise_box)))) return rc;
    if ((rc = ensure(c, c->merge, want * sizeof(int2)))) return rc;
    if ((rc = ensure(c, c->run_out, (want + 1) * sizeof(int64_t)))) return rc;
    c->run_cap = want;
  }
  if (c->run_cap == 0) {
    int64_t cap0 = std::max<int64_t>(1 << 20, (int64_t)(px / 256));
    if ((rc = ensure(c, c->run_parent, cap0 * sizeof(int32_t)))) return rc;
    if ((rc = ensure(c, c->run_sroot, cap0))) return rc;
    if ((rc = ensure(c, c->rec, cap0 * sizeof(rise_box)))) return rc;
    if ((rc = ensure(c, c->merge, cap0 * sizeof(int2)))) return rc;
    if ((rc = ensure(c, c->run_out, (cap0 + 1) * sizeof(int64_t)))) return rc;
    c->run_cap = cap0;
  }
  if ((rc = ensure(c, c->scan_tmp, ccl_scan_tmp_bytes(std::max<int64_t>(c->run_cap, T + 1)))))
    return rc;
  return RISE_OK;
}

uint64_t fnv_mix(uint64_t h, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

// Launches of one capture's spectrum part, then the image part.
int enqueue_detect(rise_ctx *c, const void *iq, int fmt, int64_t n, int N, int hop, int64_t T,
                   const rise_thresholds &thr, int path, bool want_power, const Tables *tb,
                   int64_t cap) {
  cudaStream_t s = c->stream;
  Small *sm = c->small;
  const int F = N;
  CK(cudaMemsetAsync(&sm->status, 0, sizeof(DeviceStatus), s));
  record(c, 0);
  StftArgs a;
  a.iq = iq;
  a.fmt = fmt;
  a.n = n;
  a.N = N;
  a.hop = hop;
  a.T = T;
  a.img = reinterpret_cast<uint8_t *>(c->img.p);
  a.power = want_power ? reinterpret_cast<float *>(c->power.p) : nullptr;
  a.max_bits = &sm->status.max_bits;
  a.edges = sm->edges;
  a.qconst = sm->qconst;
  a.tw = tb->tw;
  a.win = tb->win;
  a.err = &sm->status.err;
  a.sched = tb->sched;
  a.wait_limit = c->copy_wait_limit;
  a.withhold_step = c->withhold_copy;
  bool hist_ready = false;
  if (thr.range_mode == RISE_RANGE_FIXED) {
    const double hp = std::pow(10.0, thr.hi_db / 10.0);
    record(c, 1);
    CK(launch_levels(a.max_bits, hp, 1, sm->ratio, thr.level_db, sm->edges, sm->qconst, s));
    CK(launch_stft(a, c->keep_power ? STFT_QUANT_POWER : STFT_QUANT, c->num_sms, s));
  } else if (path == 2) {
    CK(launch_stft(a, stft_hooks_on(c) ? STFT_POWER_HOOKED : STFT_POWER, c->num_sms, s));
    record(c, 1);
    if (cluster_hist_accumulates(T))
      CK(cudaMemsetAsync(c->hist.p, 0, (size_t)F * 256 * sizeof(uint32_t), s));
    // the level edges are built by the histogram kernel itself (no levels launch)
    CK(launch_cluster_hist(a.power, true, T, F, sm->edges, sm->qconst, a.img,
                           reinterpret_cast<uint32_t *>(c->hist.p),
                           reinterpret_cast<rise_colstat *>(c->cols.p), nullptr, s, a.max_bits, sm->ratio,
                           thr.level_db));
    hist_ready = true;
  } else {
    CK(launch_stft(a, STFT_MAX, c->num_sms, s));
    record(c, 1);
    CK(launch_levels(a.max_bits, 0.0, 0, sm->ratio, thr.level_db, sm->edges, sm->qconst, s));
    CK(launch_stft(a, c->keep_power ? STFT_QUANT_POWER : STFT_QUANT, c->num_sms, s));
  }
  record(c, 2);
  return image_enqueue(c, a.img, T, F, thr, hist_ready, cap);
}

// Queues one capture's detection in slot c->next_slot: validation and
// host-side set-up, then (for a host capture) its copy on the copy stream,
// then the launches on the context's stream, replayed from a graph when the
// same call comes again.  The result is taken by finish_call.
int submit_call(rise_ctx *c, const void *iq, int flags, int64_t n, int N, int hop,
                const rise_thresholds *thr_in, int64_t cap) {
  const bool on_host = (flags & RISE_IQ_HOST) != 0;
  const int fmt = (flags & RISE_IQ_SC16) ? IQ_SC16 : IQ_FC32;
  const size_t bps = fmt == IQ_SC16 ? 4 : 8;   // bytes per sample
  rise_thresholds thr;
  if (thr_in) thr = *thr_in;
  else rise_thresholds_default(&thr);
  if (!c || !iq || cap < 0) return RISE_EINVAL;
  if (!pow2(N) || N < RISE_MIN_FFT || N > RISE_MAX_FFT || hop < 1 || hop > N || n < N) return RISE_EINVAL;
  if (flags & ~(RISE_IQ_HOST | RISE_IQ_SC16)) return RISE_EINVAL;
  if (!on_host && (reinterpret_cast<uintptr_t>(iq) & (bps - 1)) != 0) return RISE_EINVAL;
  const int64_t T = (n - N) / hop + 1;
  if (T > RISE_MAX_ROWS) return RISE_EINVAL;
  int rc = check_thresholds(thr, N);
  if (rc) return rc;
  if (c->npend >= 2) return RISE_EAGAIN;
  CK(cudaSetDevice(c->device));
  c->batch.last_valid = false;   // this call overwrites the image buffer
  c->cur = c->next_slot;
  CallSlot &sl = c->cs();
  const int F = N;
  const size_t px = (size_t)T * F;
  // host-side set-up: buffers, tables (may allocate or synchronise)
  if ((rc = prepare_image_buffers(c, T, F))) return rc;
  if ((rc = ensure(c, c->img, px))) return rc;
  int path = c->range_path;
  if (path == 0) {
    // FFT once keeping float power when that image fits the budget, else twice
    const size_t need = px * sizeof(float);
    path = (!c->mem_budget || c->power.bytes >= need ||
            c->allocated - c->power.bytes + need <= c->mem_budget) ? 2 : 1;
  }
  const bool want_power = c->keep_power || (path == 2 && thr.range_mode == RISE_RANGE_AUTO_MAX);
  if (want_power && (rc = ensure(c, c->power, px * sizeof(float)))) return rc;
  Tables *tb;
  const int sched = single_sched(c, N);
  if ((rc = get_tables(c, N, sched, &tb))) return rc;
  if ((rc = image_prepare(c, thr, cap))) return rc;
  const void *src = iq;
  if (on_host) {
    // the samples go to this slot's device copy on the copy stream; the
    // launches wait for that copy only
    if ((rc = ensure(c, sl.iq, (size_t)n * bps))) return rc;
    CK(cudaMemcpyAsync(sl.iq.p, iq, (size_t)n * bps, cudaMemcpyHostToDevice, c->copy_stream));
    CK(cudaEventRecord(sl.copied, c->copy_stream));
    CK(cudaStreamWaitEvent(c->stream, sl.copied, 0));
    src = sl.iq.p;
  }
  // the launches: replayed from a graph when the same call comes again
  bool launched = false;
  if (c->graphs) {
    uint64_t key = 1469598103934665603ull;
    const int64_t kv[15] = {(int64_t)reinterpret_cast<uintptr_t>(src), n, N, hop, cap, path,
                            c->keep_power, c->keep_masks, c->timing, (int64_t)c->gen,
                            thr.range_mode, (int64_t)thr.sg_half_window * 2 + thr.morph_order,
                            c->cur, fmt, sched};
    const double dv[4] = {thr.hi_db, thr.level_db, thr.psd_offset_db, thr.power_offset_db};
    key = fnv_mix(key, kv, sizeof(kv));
    key = fnv_mix(key, dv, sizeof(dv));
    BatchState::Graph *gr = nullptr;
    for (auto &g : c->single_graphs)
      if (g.key == key) gr = &g;
    if (!gr && c->last_key[c->cur] == key) {
      // the second call with these arguments in this slot: capture it
      cudaGraph_t graph = nullptr;
      const long long l0 = launches_so_far();
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        c->capturing = true;
        const int erc = enqueue_detect(c, src, fmt, n, N, hop, T, thr, path, want_power, tb, cap);
        c->capturing = false;
        const cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
        cudaGraphExec_t exec = nullptr;
        if (erc == RISE_OK && ee == cudaSuccess && graph &&
            cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
          if (c->single_graphs.size() >= 8) {
            cudaGraphExecDestroy(c->single_graphs.front().exec);
            c->single_graphs.erase(c->single_graphs.begin());
          }
          BatchState::Graph g;
          g.key = key;
          g.exec = exec;
          g.launches = (int)(launches_so_far() - l0);
          c->single_graphs.push_back(g);
          gr = &c->single_graphs.back();
        }
        if (graph) cudaGraphDestroy(graph);
      }
      count_launches(-(int)(launches_so_far() - l0));   // counted when the graph runs
      cudaGetLastError();   // a failed capture falls back to direct launches
    }
    c->last_key[c->cur] = key;
    if (gr) {
      CK(cudaGraphLaunch(gr->exec, c->stream));
      count_launches(gr->launches);
      launched = true;
    }
  }
  c->last_replayed = launched;
  if (!launched && (rc = enqueue_detect(c, src, fmt, n, N, hop, T, thr, path, want_power, tb, cap))) return rc;
  CK(cudaEventRecord(sl.done, c->stream));
  sl.pending = true;
  sl.src = src;
  sl.fmt = fmt;
  sl.n = n;
  sl.T = T;
  sl.cap = cap;
  sl.N = N;
  sl.hop = hop;
  sl.path = path;
  sl.sched = sched;
  sl.want_power = want_power;
  sl.thr = thr;
  c->pend[c->npend++] = c->cur;
  c->next_slot ^= 1;
  c->last_T = T;
  c->last_F = F;
  c->last_img = reinterpret_cast<uint8_t *>(c->img.p);
  c->last_has_power = want_power;
  c->last_has_masks = c->keep_masks != 0;
  c->last_valid = true;
  return RISE_OK;
}

// Waits for the oldest queued call and returns its boxes.  If its run arrays
// overflowed, everything queued is waited for, the arrays grow, and the call
// runs again from its samples (still valid: a slot is reused only after it
// has been collected), followed by the call queued behind it, if any.
int finish_call(rise_ctx *c, rise_box *out, int64_t cap, int64_t *n_boxes) {
  if (!c || !n_boxes || cap < 0 || (cap > 0 && !out)) return RISE_EINVAL;
  if (c->npend == 0) return RISE_EINVAL;
  CK(cudaSetDevice(c->device));
  c->cur = c->pend[0];
  c->pend[0] = c->pend[1];
  c->npend -= 1;
  CallSlot &sl = c->cs();
  sl.pending = false;
  int rc;
  CK(cudaEventSynchronize(sl.done));
  DeviceStatus h = *sl.st_h;
  if (h.err & ERR_RUN_CAPACITY) {
    CK(cudaStreamSynchronize(c->stream));
    const int64_t need = std::max<int64_t>(2 * h.n_runs, 2 * c->run_cap);   // doubled: few growths
    if ((rc = ensure(c, c->run_parent, need * sizeof(int32_t)))) return rc;
    if ((rc = ensure(c, c->run_sroot, need))) return rc;
    if ((rc = ensure(c, c->rec, need * sizeof(rise_box)))) return rc;
    if ((rc = ensure(c, c->merge, need * sizeof(int2)))) return rc;
    if ((rc = ensure(c, c->run_out, (need + 1) * sizeof(int64_t)))) return rc;
    if ((rc = ensure(c, c->scan_tmp, ccl_scan_tmp_bytes(std::max<int64_t>(need, sl.T + 1))))) return rc;
    c->run_cap = need;
    Tables *tb;
    if ((rc = get_tables(c, sl.N, sl.sched, &tb))) return rc;
    if ((rc = enqueue_detect(c, sl.src, sl.fmt, sl.n, sl.N, sl.hop, sl.T, sl.thr, sl.path,
                             sl.want_power, tb, sl.cap)))
      return rc;
    CK(cudaStreamSynchronize(c->stream));
    h = *sl.st_h;
    if (c->npend) {
      // the call queued behind it ran before this re-run: run it again too,
      // so the image, masks and runs on the device are the latest call's
      const int me = c->cur;
      c->cur = c->pend[0];
      CallSlot &nx = c->cs();
      Tables *tb2;
      if ((rc = get_tables(c, nx.N, nx.sched, &tb2))) return rc;
      rc = enqueue_detect(c, nx.src, nx.fmt, nx.n, nx.N, nx.hop, nx.T, nx.thr, nx.path, nx.want_power,
                          tb2, nx.cap);
      c->cur = me;
      if (rc) return rc;
      CK(cudaEventRecord(nx.done, c->stream));
    } else {
      c->last_T = sl.T;
      c->last_F = sl.N;
      c->last_img = reinterpret_cast<uint8_t *>(c->img.p);
      c->last_has_power = sl.want_power;
    }
  }
  c->last_status = sl.st_h;
  if (sl.thr.range_mode == RISE_RANGE_FIXED) {
    c->last_anchor = std::pow(10.0, sl.thr.hi_db / 10.0);
  } else {
    float mf;
    std::memcpy(&mf, &h.max_bits, 4);
    c->last_anchor = mf;
  }
  if (h.err & (ERR_UNION_LIMIT | ERR_SCAN | ERR_COPY_WAIT)) return RISE_ETIMEOUT;
  if (h.err) return RISE_EINTERNAL;
  *n_boxes = h.n_boxes;
  const int64_t lim = std::min(cap, sl.cap);
  const int64_t ncopy = std::min<int64_t>(h.n_boxes, lim);
  if (ncopy > 0) std::memcpy(out, sl.hbox, (size_t)ncopy * sizeof(rise_box));
  if (c->timing) {
    for (int i = 0; i < 7; ++i) cudaEventElapsedTime(&c->stage_ms[i], sl.ev[i], sl.ev[i + 1]);
    cudaEventElapsedTime(&c->stage_ms[7], sl.ev[0], sl.ev[7]);
  }
  return h.n_boxes > lim ? RISE_ETRUNC : RISE_OK;
}

}  // namespace

extern "C" {

void rise_thresholds_default(rise_thresholds *t) {
  if (!t) return;
  t->range_mode = RISE_RANGE_AUTO_MAX;
  t->hi_db = 0.0;
  t->level_db = 0.25;
  t->psd_offset_db = 0.5;
  t->power_offset_db = 10.0;
  t->sg_half_window = 5;
  t->morph_order = 0;
}

void rise_boxes_widen(const rise_box *in, int64_t n, int64_t *out) {
  for (int64_t i = 0; i < n; ++i) {
    const rise_box &b = in[i];
    int64_t *o = out + 8 * i;
    o[0] = b.t0;
    o[1] = b.t1;
    o[2] = b.f0;
    o[3] = b.f1;
    o[4] = b.anchor;
    o[5] = b.area;
    o[6] = (int64_t)b.sum_q;
    o[7] = (int64_t)b.energy_fx;
  }
}

const char *rise_strerror(int code) {
  switch (code) {
    case RISE_OK: return "ok";
    case RISE_EINVAL: return "invalid argument";
    case RISE_ENOMEM: return "out of device memory or over the memory budget";
    case RISE_ETRUNC: return "more boxes than the output capacity";
    case RISE_ECUDA: return "CUDA runtime error";
    case RISE_ETIMEOUT: return "bounded device-side wait gave up";
    case RISE_EINTERNAL: return "internal consistency check failed";
    case RISE_ESCRATCH: return "size exceeds the fixed scratch of the allocation-free entry point";
  }
  return "unknown status";
}

int rise_create(rise_ctx **out, const rise_config *cfg) {
  if (!out || !cfg) return RISE_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return RISE_ECUDA;
  }
  if (cfg->device < 0 || cfg->device >= ndev) return RISE_EINVAL;
  {
    // every kernel loaded once per device, here rather than in a call
    static std::mutex mu;
    static std::set<int> loaded;
    std::lock_guard<std::mutex> lk(mu);
    if (!loaded.count(cfg->device) && cudaSetDevice(cfg->device) == cudaSuccess) {
      stft_preload();
      stft_s1_preload();
      stft_s2_preload();
      stft_sc16_preload();
      image_preload();
      ccl_preload();
      batch_preload();
      match_preload();
      loaded.insert(cfg->device);
    }
  }
  rise_ctx *c = new (std::nothrow) rise_ctx();
  if (!c) return RISE_ENOMEM;
  c->device = cfg->device;
  c->mem_budget = cfg->mem_budget;
  int rc = RISE_OK;
  do {
    if (cudaSetDevice(c->device) != cudaSuccess) { rc = RISE_ECUDA; break; }
    cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (cfg->cuda_stream) {
      c->stream = reinterpret_cast<cudaStream_t>(cfg->cuda_stream);
    } else {
      if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) { rc = RISE_ECUDA; break; }
      c->own_stream = true;
    }
    if (cudaMalloc(&c->small, sizeof(Small)) != cudaSuccess) { rc = RISE_ENOMEM; break; }
    cudaMemset(c->small, 0, sizeof(Small));
    if (cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking) != cudaSuccess) { rc = RISE_ECUDA; break; }
    for (auto &sl : c->slot) {
      void *p = nullptr;
      if (cudaHostAlloc(&p, sizeof(DeviceStatus), cudaHostAllocMapped) != cudaSuccess) { rc = RISE_ENOMEM; break; }
      sl.st_h = static_cast<DeviceStatus *>(p);
      void *pd = nullptr;
      if (cudaHostGetDevicePointer(&pd, p, 0) != cudaSuccess) { rc = RISE_ECUDA; break; }
      sl.st_d = static_cast<DeviceStatus *>(pd);
      std::memset(sl.st_h, 0, sizeof(DeviceStatus));
      for (auto &e : sl.ev)
        if (cudaEventCreate(&e) != cudaSuccess) rc = RISE_ECUDA;
      if (cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess) rc = RISE_ECUDA;
      if (cudaEventCreateWithFlags(&sl.copied, cudaEventDisableTiming) != cudaSuccess) rc = RISE_ECUDA;
      if (rc) break;
    }
    c->last_status = c->slot[0].st_h;
    if (rc) break;
    if (cfg->max_fft && (cfg->max_fft < RISE_MIN_FFT || cfg->max_fft > RISE_MAX_FFT || !pow2(cfg->max_fft))) {
      rc = RISE_EINVAL;
      break;
    }
    if (cfg->max_samples < 0 || cfg->max_boxes < 0) { rc = RISE_EINVAL; break; }
    if (cfg->max_samples > 0) {
      // the 8-bit image of a capture with hop >= F/2 has at most 2 pixels per sample
      if ((rc = ensure(c, c->img, (size_t)cfg->max_samples * 2))) break;
    }
    if (cfg->max_boxes > 0) {
      for (int k = 0; k < 2 && rc == RISE_OK; ++k) {
        c->cur = k;
        rc = ensure_hbox(c, cfg->max_boxes);
      }
      c->cur = 0;
      if (rc) break;
    }
  } while (0);
  if (rc) {
    cudaGetLastError();
    rise_destroy(c);
    return rc;
  }
  *out = c;
  return RISE_OK;
}

void rise_destroy(rise_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->wait_ev) cudaEventDestroy(c->wait_ev);
  Buf *bufs[] = {&c->power, &c->img, &c->hist, &c->cols, &c->effm1, &c->mask,
                 &c->dbg[0], &c->dbg[1], &c->dbg[2], &c->row_cnt, &c->row_base,
                 &c->run_parent, &c->run_sroot, &c->rec, &c->run_out, &c->scan_tmp, &c->boxes, &c->merge,
                 &c->match_boxes, &c->match_best, &c->match_misc, &c->contour};
  for (Buf *b : bufs)
    if (b->p) cudaFree(b->p);
  for (auto &kv : c->tables) cudaFree(kv.second.tw);
  destroy_batch(c);
  if (c->small) cudaFree(c->small);
  for (auto &sl : c->slot) {
    if (sl.hbox) cudaFreeHost(sl.hbox);
    if (sl.st_h) cudaFreeHost(sl.st_h);
    if (sl.iq.p) cudaFree(sl.iq.p);
    for (auto &e : sl.ev)
      if (e) cudaEventDestroy(e);
    if (sl.done) cudaEventDestroy(sl.done);
    if (sl.copied) cudaEventDestroy(sl.copied);
  }
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

int rise_detect(rise_ctx *c, const void *iq_dev, int64_t n, int fft_size, int hop,
                const rise_thresholds *thr, rise_box *out, int64_t cap, int64_t *n_boxes) {
  if (!c || !n_boxes || (cap > 0 && !out) || c->npend) return RISE_EINVAL;
  const int rc = submit_call(c, iq_dev, 0, n, fft_size, hop, thr, cap);
  return rc ? rc : finish_call(c, out, cap, n_boxes);
}

int rise_detect_host(rise_ctx *c, const void *iq_host, int64_t n, int fft_size, int hop,
                     const rise_thresholds *thr, rise_box *out, int64_t cap, int64_t *n_boxes) {
  if (!c || !n_boxes || (cap > 0 && !out) || c->npend) return RISE_EINVAL;
  const int rc = submit_call(c, iq_host, RISE_IQ_HOST, n, fft_size, hop, thr, cap);
  return rc ? rc : finish_call(c, out, cap, n_boxes);
}

int rise_submit(rise_ctx *c, const void *iq, int iq_flags, int64_t n, int fft_size, int hop,
                const rise_thresholds *thr, int64_t cap) {
  return submit_call(c, iq, iq_flags, n, fft_size, hop, thr, cap);
}

int rise_collect(rise_ctx *c, rise_box *out, int64_t cap, int64_t *n_boxes) {
  return finish_call(c, out, cap, n_boxes);
}

int rise_detect_image(rise_ctx *c, const uint8_t *img_dev, int64_t T, int F,
                      const rise_thresholds *thr_in, rise_box *out, int64_t cap, int64_t *n_boxes) {
  rise_thresholds thr;
  if (thr_in) thr = *thr_in;
  else rise_thresholds_default(&thr);
  if (!c || !img_dev || !n_boxes || (cap > 0 && !out) || cap < 0 || c->npend) return RISE_EINVAL;
  c->cur = 0;
  if (!pow2(F) || F < RISE_MIN_FFT || F > RISE_MAX_FFT || T < 1 || T > RISE_MAX_ROWS) return RISE_EINVAL;
  if ((reinterpret_cast<uintptr_t>(img_dev) & 31) != 0) return RISE_EINVAL;
  int rc = check_thresholds(thr, F);
  if (rc) return rc;
  CK(cudaSetDevice(c->device));
  c->batch.last_valid = false;
  if ((rc = prepare_image_buffers(c, T, F))) return rc;
  record(c, 0);
  CK(cudaMemsetAsync(&c->small->status, 0, sizeof(DeviceStatus), c->stream));
  record(c, 1);
  record(c, 2);
  c->last_T = T;
  c->last_F = F;
  c->last_img = img_dev;
  c->last_has_power = false;
  c->last_has_masks = c->keep_masks != 0;
  c->last_valid = true;
  if ((rc = image_prepare(c, thr, cap))) return rc;
  if ((rc = image_enqueue(c, img_dev, T, F, thr, false, cap))) return rc;
  return image_finish(c, img_dev, T, F, out, cap, n_boxes);
}

int rise_contours(rise_ctx *c, int32_t *runs, int64_t cap, int64_t *n_runs, uint32_t *boundary) {
  if (!c || !n_runs || cap < 0 || (cap > 0 && !runs) || c->npend || !c->last_valid || !c->last_status)
    return RISE_EINVAL;
  CK(cudaSetDevice(c->device));
  const int64_t T = c->last_T;
  const int F = c->last_F;
  const int64_t n = c->last_status->n_runs;
  if (n > c->run_cap) return RISE_EINTERNAL;
  *n_runs = n;
  const int64_t k = std::min(n, cap);
  const size_t bb = boundary ? (size_t)T * (F / 32) * sizeof(uint32_t) : 0;
  int rc;
  if ((rc = ensure(c, c->contour, std::max<size_t>((size_t)k * sizeof(int4), bb)))) return rc;
  cudaStream_t s = c->stream;
  if (k > 0) {
    const CclArgs la = ccl_args(c, c->last_img, T, F, 0);
    CK(launch_runs_export(la, static_cast<int4 *>(c->contour.p), k, c->num_sms, s));
    CK(cudaMemcpyAsync(runs, c->contour.p, (size_t)k * sizeof(int4), cudaMemcpyDeviceToHost, s));
  }
  if (boundary) {
    CK(cudaStreamSynchronize(s));   // the export above is done with the buffer
    CK(launch_boundary(static_cast<const uint32_t *>(c->mask.p), T, F, static_cast<uint32_t *>(c->contour.p),
                       c->num_sms, s));
    CK(cudaMemcpyAsync(boundary, c->contour.p, bb, cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  return n > cap ? RISE_ETRUNC : RISE_OK;
}

int rise_set_option(rise_ctx *c, int option, int64_t value) {
  if (!c) return RISE_EINVAL;
  switch (option) {
    case RISE_OPT_KEEP_POWER: c->keep_power = value != 0; return RISE_OK;
    case RISE_OPT_KEEP_MASKS: c->keep_masks = value != 0; return RISE_OK;
    case RISE_OPT_TIMING: c->timing = value != 0; return RISE_OK;
    case RISE_OPT_GRAPH: c->graphs = value != 0; return RISE_OK;
    case RISE_OPT_AUTOTUNE: c->autotune = value != 0; return RISE_OK;
    case RISE_OPT_RUN_CAPACITY:
      if (value < 1024 || value > (int64_t)1 << 31) return RISE_EINVAL;
      c->run_cap_req = value;
      return RISE_OK;
    case RISE_OPT_RANGE_PATH:
      if (value < 0 || value > 2) return RISE_EINVAL;
      c->range_path = (int)value;
      return RISE_OK;
    // the limits are kernel arguments inside captured graphs: a change drops them
    case RISE_OPT_SCAN_WAIT_LIMIT:
      if (value < 0 || value > INT32_MAX) return RISE_EINVAL;
      CK(cudaSetDevice(c->device));
      c->spin_limit = value ? (int)value : SCAN_SPIN_LIMIT;
      new_generation(c);
      return RISE_OK;
    case RISE_OPT_UNION_LIMIT:
      if (value < 0 || value > INT32_MAX) return RISE_EINVAL;
      CK(cudaSetDevice(c->device));
      c->uf_limit = value ? (int)value : UF_LIMIT;
      new_generation(c);
      return RISE_OK;
    case RISE_OPT_TEST_WITHHOLD:
      if (value < -1) return RISE_EINVAL;
      CK(cudaSetDevice(c->device));
      c->withhold_tile = value;
      new_generation(c);
      return RISE_OK;
    case RISE_OPT_FFT_SCHEDULE:
      if (value < -1 || value > 3) return RISE_EINVAL;
      c->fft_sched = (int)value;
      return RISE_OK;
    case RISE_OPT_COPY_WAIT_LIMIT:
      // at least 2^12 polls, far longer than an issued copy takes to land,
      // so that a block does not give up on a copy that is on its way
      if ((value != 0 && value < 4096) || value > INT32_MAX) return RISE_EINVAL;
      CK(cudaSetDevice(c->device));
      c->copy_wait_limit = value ? (int)value : STFT_WAIT_LIMIT;
      new_generation(c);
      return RISE_OK;
    case RISE_OPT_TEST_WITHHOLD_COPY:
      if (value < -1) return RISE_EINVAL;
      CK(cudaSetDevice(c->device));
      c->withhold_copy = value;
      new_generation(c);
      return RISE_OK;
    case RISE_OPT_BLOCKING_WAIT:
      if (value < 0 || value > 1) return RISE_EINVAL;
      c->blocking_wait = value != 0;
      return RISE_OK;
  }
  return RISE_EINVAL;
}

int rise_stage_times(rise_ctx *c, float *ms, int nstages) {
  if (!c || !ms || nstages < 0) return RISE_EINVAL;
  for (int i = 0; i < nstages && i < 8; ++i) ms[i] = c->stage_ms[i];
  return RISE_OK;
}

int rise_debug_export(rise_ctx *c, int what, void *dst, size_t bytes) {
  if (!c || !dst) return RISE_EINVAL;
  if (what == RISE_DBG_LAUNCHES) {
    if (bytes < sizeof(int64_t)) return RISE_EINVAL;
    int64_t v = (int64_t)launches_so_far();
    std::memcpy(dst, &v, sizeof v);
    return RISE_OK;
  }
  if (what == RISE_DBG_CCL) {
    if (bytes < 4 * sizeof(int64_t)) return RISE_EINVAL;
    const DeviceStatus &h = *c->last_status;
    const int64_t v[4] = {h.n_runs, h.n_merge, h.n_boxes, c->run_cap};
    std::memcpy(dst, v, sizeof v);
    return RISE_OK;
  }
  if (what == RISE_DBG_GRAPHS) {
    if (bytes < 4 * sizeof(int64_t)) return RISE_EINVAL;
    const int64_t v[4] = {c->last_replayed ? 1 : 0, (int64_t)c->single_graphs.size(),
                          (int64_t)c->batch.graphs.size(), 0};
    std::memcpy(dst, v, sizeof v);
    return RISE_OK;
  }
  if (what == RISE_DBG_BATCH_INFO) {
    if (bytes < 64 * sizeof(int64_t) || c->batch.last_groups == 0) return RISE_EINVAL;
    int64_t v[64] = {};
    v[0] = c->batch.last_groups;
    v[1] = c->batch.last_graph ? 1 : 0;
    for (size_t i = 0; i < c->batch.last_params.size() && i + 2 < 63; ++i) v[2 + i] = c->batch.last_params[i];
    v[63] = c->batch.cache_hits;
    std::memcpy(dst, v, sizeof v);
    return RISE_OK;
  }
  if (what == RISE_DBG_BATCH_IMAGES || what == RISE_DBG_BATCH_POWER || what == RISE_DBG_BATCH_ANCHORS) {
    const BatchState &b = c->batch;
    if (!b.last_valid) return RISE_EINVAL;
    CK(cudaSetDevice(c->device));
    if (what == RISE_DBG_BATCH_ANCHORS) {
      const size_t need = (size_t)b.last_ncap * sizeof(float);
      if (bytes < need) return RISE_EINVAL;
      float *o = static_cast<float *>(dst);
      if (b.last_fixed) {
        for (int k = 0; k < b.last_ncap; ++k) o[k] = (float)std::pow(10.0, b.last_hi_db / 10.0);
        return RISE_OK;
      }
      std::vector<CapSmall> cs((size_t)b.last_ncap);
      CK(cudaMemcpyAsync(cs.data(), b.small.p, cs.size() * sizeof(CapSmall), cudaMemcpyDeviceToHost,
                         c->stream));
      CK(cudaStreamSynchronize(c->stream));
      for (int k = 0; k < b.last_ncap; ++k) std::memcpy(&o[k], &cs[k].max_bits, sizeof(float));
      return RISE_OK;
    }
    if (what == RISE_DBG_BATCH_POWER && b.last_fixed) return RISE_EINVAL;
    const size_t need = (size_t)b.last_px * (what == RISE_DBG_BATCH_POWER ? sizeof(float) : 1);
    const void *src = what == RISE_DBG_BATCH_POWER ? c->power.p : c->img.p;
    if (bytes < need || !src) return RISE_EINVAL;
    CK(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return RISE_OK;
  }
  if (!c->last_valid) return RISE_EINVAL;
  CK(cudaSetDevice(c->device));
  const int64_t T = c->last_T;
  const int F = c->last_F;
  const size_t px = (size_t)T * F;
  const void *src = nullptr;
  size_t need = 0;
  switch (what) {
    case RISE_DBG_POWER_F32:
      if (!c->last_has_power) return RISE_EINVAL;
      src = c->power.p; need = px * sizeof(float); break;
    case RISE_DBG_IMAGE_U8: src = c->last_img; need = px; break;
    case RISE_DBG_HIST: src = c->hist.p; need = (size_t)F * 256 * sizeof(uint32_t); break;
    case RISE_DBG_COLSTATS: src = c->cols.p; need = (size_t)F * sizeof(rise_colstat); break;
    case RISE_DBG_FLOOR: src = c->small->floor_out; need = 8 * sizeof(int64_t); break;
    case RISE_DBG_MASK0: case RISE_DBG_MASK1: case RISE_DBG_MASK2:
      if (!c->last_has_masks) return RISE_EINVAL;
      src = c->dbg[what - RISE_DBG_MASK0].p; need = px / 8; break;
    case RISE_DBG_MASK3: src = c->mask.p; need = px / 8; break;
    case RISE_DBG_MAXPOW: {
      if (bytes < sizeof(float)) return RISE_EINVAL;
      float v = (float)c->last_anchor;
      std::memcpy(dst, &v, sizeof v);
      return RISE_OK;
    }
    case RISE_DBG_LEVEL_EDGES: src = c->small->edges; need = 257 * sizeof(float); break;
    default: return RISE_EINVAL;
  }
  if (bytes < need || !src) return RISE_EINVAL;
  CK(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return RISE_OK;
}

}  // extern "C"
