// Batched detection: many captures of uneven length and FFT size go through
// the path of Sec. IV-B together, one launch per stage for the whole batch
// (one STFT launch per FFT size), instead of one launch chain per capture.
//
// Every capture keeps its own results: its own 8-bit range anchor, column
// statistics, mask and components; only the launches are shared.  Each
// kernel finds its capture through a small device table built here.  The
// whole chain is captured once as a CUDA graph per batch composition and
// replayed when the same composition comes again, and the launch shapes that
// matter (frames per STFT work item, morphology warps per SM) are picked by
// timing candidates on the first batch of each composition.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>

#include "context.cuh"

namespace rise {
namespace host {
namespace {

// dst[i] = src[i] for i < n (src: pinned host memory, read over the bus)
__global__ void copy16_kernel(uint4 *dst, const uint4 *src, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

constexpr int kMaxGraphs = 64;
constexpr int kItemCands[] = {1, 2, 4, 8, 16};      // STFT work item = k x frames per step
constexpr int kMorphCands[] = {8, 16, 32};          // morphology warps per SM
constexpr int kNumCands = 5;

uint64_t fnv(uint64_t h, const void *p, size_t n) {
  const unsigned char *b = static_cast<const unsigned char *>(p);
  for (size_t i = 0; i < n; ++i) {
    h ^= b[i];
    h *= 1099511628211ull;
  }
  return h;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool tma_ok(const rise_capture &k) {
  return k.hop % 2 == 0 && (reinterpret_cast<uintptr_t>(k.iq_dev) & 15) == 0;
}

constexpr int64_t kHistSplitRows = 8192;

struct Plan {
  int ncap = 0;
  bool fixed = false;
  std::vector<int64_t> T, px_off, col_off, row0;   // row0: ncap + 1 entries
  int64_t total_px = 0, total_cols = 0, total_rows = 0;
  int max_F = 0;
  struct Group {
    int N;
    bool tma;
    int item0, n_items;
  };
  std::vector<Group> groups;
  std::vector<int> group_of;                      // capture -> group
  // tuned launch parameters: item multiplier and radix schedule per group,
  // morphology warps per SM
  std::vector<int> item_mult, sched;
  int morph_wps = 16;
  // blob layout
  size_t o_stft, o_items, o_hseg, o_hitem, o_col, o_mseg, o_mitem, o_wbase, o_rseg, o_row0, bytes;
  int n_items = 0, n_hitems = 0, total_warps = 0, hist_bands = 8;
  // histogram items of captures taller than kHistSplitRows come first and
  // run in clusters of hist_bands row bands; the rest run one block per
  // column group (hist_bands_small), which costs the least block time
  int n_hbig = 0, hist_bands_small = 1;
  uint64_t shape_key = 0;
};

void destroy_graphs(BatchState &b) {
  for (auto &g : b.graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  b.graphs.clear();
}

// Layout of one batch in the context's buffers and the blob of tables.
int make_plan(const rise_capture *caps, int ncap, bool fixed, Plan &p) {
  p.ncap = ncap;
  p.fixed = fixed;
  p.T.resize(ncap);
  p.px_off.resize(ncap);
  p.col_off.resize(ncap);
  p.row0.resize(ncap + 1);
  p.group_of.resize(ncap);
  uint64_t h = 1469598103934665603ull;
  h = fnv(h, &fixed, sizeof(fixed));
  for (int c = 0; c < ncap; ++c) {
    const rise_capture &k = caps[c];
    const int64_t T = (k.n - k.fft_size) / k.hop + 1;
    p.T[c] = T;
    p.px_off[c] = p.total_px;
    p.col_off[c] = p.total_cols;
    p.row0[c] = p.total_rows;
    p.total_px += T * k.fft_size;   // a multiple of 256: every offset stays 256-byte aligned
    p.total_cols += k.fft_size;
    p.total_rows += T;
    p.max_F = std::max(p.max_F, k.fft_size);
    const bool tma = tma_ok(k);
    int g = -1;
    for (size_t i = 0; i < p.groups.size(); ++i)
      if (p.groups[i].N == k.fft_size && p.groups[i].tma == tma) g = (int)i;
    if (g < 0) {
      p.groups.push_back({k.fft_size, tma, 0, 0});
      g = (int)p.groups.size() - 1;
    }
    p.group_of[c] = g;
    const int64_t key[4] = {k.n, k.fft_size, k.hop, tma};
    h = fnv(h, key, sizeof(key));
  }
  p.row0[ncap] = p.total_rows;
  p.shape_key = h;
  return RISE_OK;
}

// Work items, warps and table offsets for the plan's current launch parameters.
void size_tables(const rise_ctx *c, const rise_capture *caps, Plan &p) {
  p.n_items = 0;
  for (size_t g = 0; g < p.groups.size(); ++g) {
    p.groups[g].item0 = p.n_items;
    const int frames = p.item_mult[g] * stft_frames_per_step(p.groups[g].N);
    int cnt = 0;
    for (int c = 0; c < p.ncap; ++c)
      if (p.group_of[c] == (int)g) cnt += (int)((p.T[c] + frames - 1) / frames);
    p.groups[g].n_items = cnt;
    p.n_items += cnt;
  }
  p.n_hitems = 0;
  p.n_hbig = 0;
  p.total_warps = 0;
  int64_t max_T = 1, max_T_small = 1;
  for (int k = 0; k < p.ncap; ++k) {
    if (p.T[k] > kHistSplitRows) {
      max_T = std::max(max_T, p.T[k]);
      p.n_hbig += caps[k].fft_size / 64;
    } else {
      max_T_small = std::max(max_T_small, p.T[k]);
    }
  }
  for (int k = 0; k < p.ncap; ++k) {
    p.n_hitems += caps[k].fft_size / 64;
    int nx, rows, w;
    morph_plan(p.T[k], caps[k].fft_size, c->num_sms, p.morph_wps, 32, &nx, &rows, &w);
    p.total_warps += w;
  }
  p.hist_bands = p.n_hbig ? cluster_hist_bands(!p.fixed, p.n_hbig, max_T) : 1;
  p.hist_bands_small = (int)((max_T_small + 65534) / 65535);   // 1: a band holds up to 65535 rows
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align_up(o + bytes, 256);
    return at;
  };
  p.o_stft = take(sizeof(StftArgs) * p.ncap);
  p.o_items = take(sizeof(StftItem) * p.n_items);
  p.o_hseg = take(sizeof(HistArgs) * p.ncap);
  p.o_hitem = take(sizeof(HistItem) * p.n_hitems);
  p.o_col = take(sizeof(ColArgs) * p.ncap);
  p.o_mseg = take(sizeof(MorphArgs) * p.ncap);
  p.o_mitem = take(sizeof(MorphItem) * p.ncap);
  p.o_wbase = take(sizeof(int) * (p.ncap + 1));
  p.o_rseg = take(sizeof(RowSeg) * p.ncap);
  p.o_row0 = take(sizeof(int64_t) * (p.ncap + 1));
  p.bytes = o;
}

// The pinned staging blob of the tables (grown to at least `bytes`).  A
// captured graph reads the blob through its address, so a new blob is a new
// buffer generation: graphs captured with the old one are never replayed.
int ensure_pinned(rise_ctx *c, size_t bytes) {
  BatchState &b = c->batch;
  if (b.tab_h_bytes >= bytes) return RISE_OK;
  if (b.tab_h) {
    CK(cudaStreamSynchronize(c->stream));
    cudaFreeHost(b.tab_h);
  }
  b.tab_h = nullptr;
  b.tab_h_bytes = 0;
  const size_t want = std::max<size_t>(2 * bytes, 256 * 1024);   // few moves: each drops the graphs
  if (cudaMallocHost(&b.tab_h, want) != cudaSuccess) {
    cudaGetLastError();
    return RISE_ENOMEM;
  }
  b.tab_h_bytes = want;
  new_generation(c);
  return RISE_OK;
}

int ensure_offs(rise_ctx *c, int64_t n) {
  BatchState &b = c->batch;
  if (b.offs_cap >= n) return RISE_OK;
  if (b.offs_h) {
    CK(cudaStreamSynchronize(c->stream));
    cudaFreeHost(b.offs_h);
  }
  b.offs_h = nullptr;
  b.offs_dev = nullptr;
  b.offs_cap = 0;
  const int64_t want = std::max<int64_t>(n, 1024);
  void *h = nullptr;
  if (cudaHostAlloc(&h, (size_t)want * sizeof(int64_t), cudaHostAllocMapped) != cudaSuccess) {
    cudaGetLastError();
    return RISE_ENOMEM;
  }
  void *d = nullptr;
  if (cudaHostGetDevicePointer(&d, h, 0) != cudaSuccess) {
    cudaGetLastError();
    cudaFreeHost(h);
    return RISE_ECUDA;
  }
  b.offs_h = static_cast<int64_t *>(h);
  b.offs_dev = static_cast<int64_t *>(d);
  b.offs_cap = want;
  new_generation(c);
  return RISE_OK;
}

int ensure_buffers(rise_ctx *c, const Plan &p, int64_t cap) {
  int rc;
  const size_t px = (size_t)p.total_px;
  if (!p.fixed && (rc = ensure(c, c->power, px * sizeof(float)))) return rc;
  if ((rc = ensure(c, c->img, px))) return rc;
  if ((rc = ensure(c, c->hist, (size_t)p.total_cols * 256 * sizeof(uint32_t)))) return rc;
  if ((rc = ensure(c, c->cols, (size_t)p.total_cols * sizeof(rise_colstat)))) return rc;
  if ((rc = ensure(c, c->effm1, (size_t)p.total_cols))) return rc;
  if ((rc = ensure(c, c->mask, px / 8))) return rc;
  if ((rc = ensure(c, c->row_cnt, (size_t)p.total_rows * sizeof(uint32_t)))) return rc;
  if ((rc = ensure(c, c->row_base, (size_t)(p.total_rows + 1) * sizeof(int64_t)))) return rc;
  const int64_t want = std::max<int64_t>(1 << 20, (int64_t)(px / 64));
  if (c->run_cap < want) {
    if ((rc = ensure(c, c->run_parent, want * sizeof(int32_t)))) return rc;
    if ((rc = ensure(c, c->run_sroot, want))) return rc;
    if ((rc = ensure(c, c->rec, want * sizeof(rise_box)))) return rc;
    if ((rc = ensure(c, c->merge, want * sizeof(int2)))) return rc;
    if ((rc = ensure(c, c->run_out, (want + 1) * sizeof(int64_t)))) return rc;
    c->run_cap = want;
  }
  if ((rc = ensure(c, c->scan_tmp, ccl_scan_tmp_bytes(std::max<int64_t>(c->run_cap, p.total_rows + 1)))))
    return rc;
  BatchState &b = c->batch;
  if ((rc = ensure(c, b.small, sizeof(CapSmall) * p.ncap))) return rc;
  if ((rc = ensure(c, b.counters, sizeof(int) * 64))) return rc;
  if ((rc = ensure(c, b.tab, p.bytes))) return rc;
  if ((rc = ensure_pinned(c, p.bytes))) return rc;
  if ((rc = ensure_offs(c, p.ncap + 1))) return rc;
  if ((rc = ensure_hbox(c, std::max<int64_t>(cap, 1)))) return rc;
  return RISE_OK;
}

// Per-capture argument tables, written into the pinned staging blob.
int fill_tables(rise_ctx *c, const rise_capture *caps, const Plan &p, const rise_thresholds &thr) {
  char *h = static_cast<char *>(c->batch.tab_h);
  CapSmall *cs = static_cast<CapSmall *>(c->batch.small.p);
  auto *stft = reinterpret_cast<StftArgs *>(h + p.o_stft);
  auto *items = reinterpret_cast<StftItem *>(h + p.o_items);
  auto *hseg = reinterpret_cast<HistArgs *>(h + p.o_hseg);
  auto *hitem = reinterpret_cast<HistItem *>(h + p.o_hitem);
  auto *col = reinterpret_cast<ColArgs *>(h + p.o_col);
  auto *mseg = reinterpret_cast<MorphArgs *>(h + p.o_mseg);
  auto *mitem = reinterpret_cast<MorphItem *>(h + p.o_mitem);
  auto *wbase = reinterpret_cast<int *>(h + p.o_wbase);
  auto *rseg = reinterpret_cast<RowSeg *>(h + p.o_rseg);
  auto *row0 = reinterpret_cast<int64_t *>(h + p.o_row0);
  uint8_t *img = static_cast<uint8_t *>(c->img.p);
  float *power = p.fixed ? nullptr : static_cast<float *>(c->power.p);
  uint32_t *hist = static_cast<uint32_t *>(c->hist.p);
  rise_colstat *cols = static_cast<rise_colstat *>(c->cols.p);
  uint8_t *effm1 = static_cast<uint8_t *>(c->effm1.p);
  uint32_t *mask = static_cast<uint32_t *>(c->mask.p);
  uint32_t *row_cnt = static_cast<uint32_t *>(c->row_cnt.p);
  const int m = thr.sg_half_window;
  const int64_t D = (int64_t)(2 * m - 1) * (2 * m + 1) * (2 * m + 3);
  const bool psd_on = !(std::isinf(thr.psd_offset_db) && thr.psd_offset_db < 0);
  const bool pow_on = !(std::isinf(thr.power_offset_db) && thr.power_offset_db < 0);
  std::vector<int> next_item(p.groups.size());
  for (size_t g = 0; g < p.groups.size(); ++g) next_item[g] = p.groups[g].item0;
  int hi = 0, hs = p.n_hbig, warps = 0;   // histogram items: tall captures, then short ones
  for (int k = 0; k < p.ncap; ++k) {
    const rise_capture &cp = caps[k];
    const int F = cp.fft_size;
    const int64_t T = p.T[k];
    Tables *tb;
    int rc = get_tables(c, F, p.sched[p.group_of[k]], &tb);
    if (rc) return rc;
    StftArgs &a = stft[k];
    a.iq = cp.iq_dev;
    a.fmt = IQ_FC32;
    a.n = cp.n;
    a.N = F;
    a.hop = cp.hop;
    a.T = T;
    a.img = img + p.px_off[k];
    a.power = power ? power + p.px_off[k] : nullptr;
    a.max_bits = &cs[k].max_bits;
    a.edges = cs[k].edges;
    a.qconst = cs[k].qconst;
    a.tw = tb->tw;
    a.win = tb->win;
    a.err = &c->small->status.err;
    a.sched = tb->sched;
    a.wait_limit = c->copy_wait_limit;
    a.withhold_step = c->withhold_copy;
    const int g = p.group_of[k];
    const int frames = p.item_mult[g] * stft_frames_per_step(F);
    for (int64_t f0 = 0; f0 < T; f0 += frames) {
      StftItem &it = items[next_item[g]++];
      it.seg = k;
      it.pad = 0;
      it.f0 = f0;
      it.f1 = std::min<int64_t>(T, f0 + frames);
    }
    HistArgs &ha = hseg[k];
    ha = HistArgs{};   // edges come from the levels kernel of the batch
    ha.src = p.fixed ? static_cast<const void *>(a.img) : static_cast<const void *>(a.power);
    ha.T = T;
    ha.F = F;
    const bool big = T > kHistSplitRows;
    const int bands = big ? p.hist_bands : p.hist_bands_small;
    ha.rows_per_band = (T + bands - 1) / bands;
    ha.edges = cs[k].edges;
    ha.qconst = cs[k].qconst;
    ha.img = a.img;
    ha.hist = hist + p.col_off[k] * 256;
    ha.cols = cols + p.col_off[k];
    ha.accumulate = 0;
    for (int cg = 0; cg < F / 64; ++cg) hitem[big ? hi++ : hs++] = HistItem{k, cg};
    ColArgs &ca = col[k];
    ca = ColArgs{};
    ca.hist = ha.hist;
    ca.T = T;
    ca.F = F;
    ca.m = m;
    ca.D = D;
    ca.sg_c = c->small->sgc;
    const double DT = (double)(D * T);
    ca.psd_on = psd_on;
    ca.pow_on = pow_on;
    ca.delta_psd = psd_on ? (int64_t)std::llround(thr.psd_offset_db / thr.level_db * DT) : 0;
    ca.delta_pow = pow_on ? (int64_t)std::llround(thr.power_offset_db / thr.level_db * DT) : 0;
    ca.cols = ha.cols;
    ca.effm1 = effm1 + p.col_off[k];
    ca.floor_out = cs[k].floor_out;
    MorphArgs &ma = mseg[k];
    ma.img = a.img;
    ma.effm1 = ca.effm1;
    ma.T = T;
    ma.F = F;
    ma.order = thr.morph_order;
    ma.mask = mask + p.px_off[k] / 32;
    ma.dbg0 = ma.dbg1 = ma.dbg2 = nullptr;
    ma.row_cnt = row_cnt + p.row0[k];
    int nx, rows, nw;
    morph_plan(T, F, c->num_sms, p.morph_wps, 32, &nx, &rows, &nw);
    mitem[k] = MorphItem{nx, rows};
    wbase[k] = warps;
    warps += nw;
    rseg[k] = RowSeg{ma.mask, a.img, T, F, 0};
    row0[k] = p.row0[k];
  }
  wbase[p.ncap] = warps;
  row0[p.ncap] = p.row0[p.ncap];
  // largest items first inside each group: the persistent blocks end together
  for (const auto &g : p.groups)
    std::stable_sort(items + g.item0, items + g.item0 + g.n_items, [](const StftItem &x, const StftItem &y) {
      return (x.f1 - x.f0) > (y.f1 - y.f0);
    });
  return RISE_OK;
}

struct Events {
  cudaEvent_t e[16] = {};
  int n = 0;
};

// The launch chain of one batch (no host synchronisation inside, so that it
// can be captured).  `ev`, when given, gets an event after each STFT group
// and around the morphology (autotuning).
int enqueue(rise_ctx *c, const Plan &p, const rise_thresholds &thr, int64_t cap, Events *ev,
            int *launches, bool capturing) {
  cudaStream_t s = c->stream;
  // inside a capture, timing events must become event-record nodes
  auto record = [&](rise_ctx *cc, int i) {
    if (cc->timing)
      cudaEventRecordWithFlags(cc->cs().ev[i], s, capturing ? cudaEventRecordExternal : cudaEventRecordDefault);
  };
  BatchState &b = c->batch;
  const long long l0 = launches_so_far();
  char *d = static_cast<char *>(b.tab.p);
  auto *stft = reinterpret_cast<const StftArgs *>(d + p.o_stft);
  auto *items = reinterpret_cast<const StftItem *>(d + p.o_items);
  auto *hseg = reinterpret_cast<const HistArgs *>(d + p.o_hseg);
  auto *hitem = reinterpret_cast<const HistItem *>(d + p.o_hitem);
  auto *col = reinterpret_cast<const ColArgs *>(d + p.o_col);
  auto *mseg = reinterpret_cast<const MorphArgs *>(d + p.o_mseg);
  auto *mitem = reinterpret_cast<const MorphItem *>(d + p.o_mitem);
  auto *wbase = reinterpret_cast<const int *>(d + p.o_wbase);
  auto *rseg = reinterpret_cast<const RowSeg *>(d + p.o_rseg);
  auto *row0 = reinterpret_cast<const int64_t *>(d + p.o_row0);
  CapSmall *cs = static_cast<CapSmall *>(b.small.p);
  int *counters = static_cast<int *>(b.counters.p);
  Small *sm = c->small;
  auto mark = [&]() {
    if (ev) cudaEventRecord(ev->e[ev->n++], s);
  };
  record(c, 0);
  // the tables come over with SM loads from the pinned staging blob, not a
  // copy engine: H2D copies the caller queues (e.g. the next batch's
  // samples) would hold a copy-engine upload back
  {
    const int64_t n16 = (int64_t)(p.bytes / 16);
    const int g = (int)std::min<int64_t>(std::max<int64_t>((n16 + 255) / 256, 1), (int64_t)c->num_sms * 4);
    copy16_kernel<<<g, 256, 0, s>>>(static_cast<uint4 *>(b.tab.p), static_cast<const uint4 *>(b.tab_h), n16);
    count_launches(1);
  }
  CK(cudaMemsetAsync(&sm->status, 0, sizeof(DeviceStatus), s));
  CK(cudaMemsetAsync(cs, 0, sizeof(CapSmall) * p.ncap, s));
  CK(cudaMemsetAsync(counters, 0, sizeof(int) * p.groups.size(), s));
  const double hp = p.fixed ? std::pow(10.0, thr.hi_db / 10.0) : 0.0;
  if (p.fixed) CK(launch_levels_batch(cs, p.ncap, hp, 1, sm->ratio, thr.level_db, s));
  mark();
  for (size_t g = 0; g < p.groups.size(); ++g) {
    const auto &G = p.groups[g];
    CK(launch_stft_batch(G.N, p.sched[g], G.tma,
                         p.fixed ? STFT_QUANT : (stft_hooks_on(c) ? STFT_POWER_HOOKED : STFT_POWER), stft, items + G.item0,
                         G.n_items, counters + g, c->num_sms, s));
    mark();
  }
  record(c, 1);
  if (!p.fixed) CK(launch_levels_batch(cs, p.ncap, 0.0, 0, sm->ratio, thr.level_db, s));
  if (p.n_hbig) CK(launch_cluster_hist_batch(!p.fixed, hseg, hitem, p.n_hbig, p.hist_bands, s));
  if (p.n_hitems > p.n_hbig)
    CK(launch_cluster_hist_batch(!p.fixed, hseg, hitem + p.n_hbig, p.n_hitems - p.n_hbig, p.hist_bands_small, s));
  record(c, 2);
  record(c, 3);
  CK(launch_floor_batch(col, p.ncap, p.max_F, s));
  record(c, 4);
  CK(cudaMemsetAsync(c->row_cnt.p, 0, (size_t)p.total_rows * sizeof(uint32_t), s));
  mark();
  CK(launch_morph_batch(thr.morph_order, mseg, mitem, wbase, p.ncap, p.total_warps, s));
  mark();
  record(c, 5);
  CclArgs la{};
  la.mask = static_cast<const uint32_t *>(c->mask.p);
  la.img = static_cast<const uint8_t *>(c->img.p);
  la.T = p.total_rows;
  la.F = p.max_F;   // the widest capture: sizes the row pass's staging
  la.energy = sm->energy;
  la.row_base = static_cast<int64_t *>(c->row_base.p);
  la.row_cnt = static_cast<uint32_t *>(c->row_cnt.p);
  la.run_cap = c->run_cap;
  la.run_parent = static_cast<int32_t *>(c->run_parent.p);
  la.run_sroot = static_cast<uint8_t *>(c->run_sroot.p);
  la.rec = static_cast<rise_box *>(c->rec.p);
  la.merge = static_cast<int2 *>(c->merge.p);
  la.run_out = static_cast<int64_t *>(c->run_out.p);
  la.scan_tmp = c->scan_tmp.p;
  la.scan_tmp_bytes = c->scan_tmp.bytes;
  la.boxes = c->cs().hbox_dev;
  la.box_cap = cap;
  la.status = &sm->status;
  la.status_out = nullptr;   // the offsets kernel runs after the labelling: a copy node reads the status
  la.uf_limit = c->uf_limit;
  la.spin_limit = c->spin_limit;
  la.withhold_tile = c->withhold_tile;
  CK(launch_ccl_count(la, c->num_sms, s));
  CK(launch_ccl_label_batch(la, rseg, row0, p.ncap, b.offs_dev, c->num_sms, s));
  record(c, 6);
  CK(cudaMemcpyAsync(c->cs().st_h, &sm->status, sizeof(DeviceStatus), cudaMemcpyDeviceToHost, s));
  record(c, 7);
  if (launches) *launches = (int)(launches_so_far() - l0);
  return RISE_OK;
}

uint64_t graph_key(const Plan &p, const rise_thresholds &thr, int64_t cap, uint64_t gen, int timing) {
  uint64_t h = p.shape_key;
  const double dv[5] = {thr.hi_db, thr.level_db, thr.psd_offset_db, thr.power_offset_db, 0.0};
  const int iv[3] = {thr.range_mode, thr.sg_half_window, thr.morph_order};
  h = fnv(h, dv, sizeof(dv));
  h = fnv(h, iv, sizeof(iv));
  h = fnv(h, &cap, sizeof(cap));
  h = fnv(h, &gen, sizeof(gen));
  h = fnv(h, &timing, sizeof(timing));
  h = fnv(h, p.item_mult.data(), p.item_mult.size() * sizeof(int));
  h = fnv(h, p.sched.data(), p.sched.size() * sizeof(int));
  h = fnv(h, &p.morph_wps, sizeof(p.morph_wps));
  return h;
}

// Radix schedule of an untuned batch group: 1 (the small radix first, the
// faster one where it differs), the same as 0 for powers of 16.
int default_sched(int N) { return stft_default_sched(N); }

// Tuned parameters of a composition: item multiplier per STFT group, radix
// schedule per group, morphology warps per SM.
struct Tuned {
  std::vector<int> item_mult, sched;
  int morph_wps = 16;
};

std::vector<int> pack(const Tuned &t) {
  std::vector<int> v(t.item_mult);
  v.insert(v.end(), t.sched.begin(), t.sched.end());
  v.push_back(t.morph_wps);
  return v;
}

bool unpack(const std::vector<int> &v, size_t ng, Tuned *t) {
  if (v.size() != 2 * ng + 1) return false;
  t->item_mult.assign(v.begin(), v.begin() + ng);
  t->sched.assign(v.begin() + ng, v.begin() + 2 * ng);
  t->morph_wps = v.back();
  return true;
}

// ---------------------------------------------------------------------------
// Tune cache: a text file named by $RISE_TUNE_CACHE, one line per tuned
// composition, "rise-tune 1 <device> <composition key, 16 hex digits> <G>
// <G item multipliers> <G schedules> <morphology warps per SM>", where
// <device> is the device name (spaces as '_') and its SM count joined by
// ':'.  A line is appended whenever a composition is tuned; on reading, the
// last line for a device and key wins.  A process that finds its
// composition there runs it without tuning.
// ---------------------------------------------------------------------------
std::string device_tag(const rise_ctx *c) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, c->device) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string n(prop.name);
  for (char &ch : n)
    if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
  return n + ":" + std::to_string(prop.multiProcessorCount);
}

bool cache_lookup(const rise_ctx *c, uint64_t key, size_t ng, Tuned *out) {
  const char *path = std::getenv("RISE_TUNE_CACHE");
  if (!path || !*path) return false;
  FILE *f = std::fopen(path, "r");
  if (!f) return false;
  const std::string dev = device_tag(c);
  char line[4096];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    char tag[16], dname[512];
    int ver = 0, g = 0, off = 0;
    unsigned long long k = 0;
    if (std::sscanf(line, "%15s %d %511s %llx %d%n", tag, &ver, dname, &k, &g, &off) != 5) continue;
    if (std::strcmp(tag, "rise-tune") != 0 || ver != 1 || dev != dname || k != key || g != (int)ng) continue;
    std::vector<int> v;
    const char *q = line + off;
    for (size_t i = 0; i < 2 * ng + 1; ++i) {
      int x = 0, used = 0;
      if (std::sscanf(q, "%d%n", &x, &used) != 1) break;
      v.push_back(x);
      q += used;
    }
    Tuned t;
    if (!unpack(v, ng, &t)) continue;
    bool ok = t.morph_wps >= 1 && t.morph_wps <= 64;
    for (size_t i = 0; i < ng; ++i)
      ok = ok && t.item_mult[i] >= 1 && t.item_mult[i] <= 64 && t.sched[i] >= 0 && t.sched[i] <= 2;
    if (ok) {
      *out = t;
      found = true;
    }
  }
  std::fclose(f);
  return found;
}

void cache_store(const rise_ctx *c, uint64_t key, const Tuned &t) {
  const char *path = std::getenv("RISE_TUNE_CACHE");
  if (!path || !*path) return;
  std::string line = "rise-tune 1 " + device_tag(c);
  char hex[32];
  std::snprintf(hex, sizeof hex, " %016llx %d", (unsigned long long)key, (int)t.item_mult.size());
  line += hex;
  for (int v : pack(t)) line += " " + std::to_string(v);
  line += "\n";
  FILE *f = std::fopen(path, "a");   // one short append per tuned composition
  if (!f) return;
  std::fputs(line.c_str(), f);
  std::fclose(f);
}

// Runs the chain once per candidate launch shape and keeps, per STFT group,
// the fastest item size and, for the morphology, the fastest warps per SM;
// then, for groups whose FFT size has a second radix schedule, runs the chain
// with that schedule and keeps it where it is faster.
int autotune(rise_ctx *c, const rise_capture *caps, Plan &p, const rise_thresholds &thr,
             int64_t cap) {
  const size_t ng = p.groups.size();
  std::vector<float> best_g(ng, 1e30f);
  std::vector<int> pick_g(ng, 2);
  float best_m = 1e30f;
  int pick_m = 16;
  Events ev;
  for (auto &e : ev.e)
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return RISE_ECUDA;
    }
  int rc = RISE_OK;
  auto run_timed = [&](std::vector<float> *group_ms, float *morph_ms) -> int {
    size_tables(c, caps, p);
    int r2;
    if ((r2 = ensure_buffers(c, p, cap))) return r2;
    if ((r2 = fill_tables(c, caps, p, thr))) return r2;
    for (int rep = 0; rep < 2; ++rep) {   // the first run warms up
      ev.n = 0;
      if ((r2 = enqueue(c, p, thr, cap, &ev, nullptr, false))) return r2;
      if (cudaStreamSynchronize(c->stream) != cudaSuccess) return RISE_ECUDA;
    }
    for (size_t g = 0; g < ng; ++g) cudaEventElapsedTime(&(*group_ms)[g], ev.e[g], ev.e[g + 1]);
    cudaEventElapsedTime(morph_ms, ev.e[ng + 1], ev.e[ng + 2]);
    return RISE_OK;
  };
  std::vector<float> ms(ng);
  float mm = 0.f;
  p.sched.assign(ng, 0);
  for (int r = 0; r < kNumCands && rc == RISE_OK; ++r) {
    p.item_mult.assign(ng, kItemCands[r]);
    p.morph_wps = kMorphCands[r % 3];
    if ((rc = run_timed(&ms, &mm))) break;
    for (size_t g = 0; g < ng; ++g)
      if (ms[g] < best_g[g]) { best_g[g] = ms[g]; pick_g[g] = kItemCands[r]; }
    if (mm < best_m) { best_m = mm; pick_m = kMorphCands[r % 3]; }
  }
  // the radix schedule, one per FFT size (a size's groups differ only in
  // their input staging): each other schedule a size has is timed in one
  // more run, and the size keeps the one with the smallest total over its
  // groups
  std::vector<int> pick_s(ng, 0);
  std::map<int, float> best_n;   // FFT size -> total of its groups under its picked schedule
  for (size_t g = 0; g < ng; ++g) best_n[p.groups[g].N] += best_g[g];
  for (int alt = 1; alt <= 2 && rc == RISE_OK; ++alt) {
    bool any = false;
    for (size_t g = 0; g < ng; ++g) any = any || stft_sched_distinct(p.groups[g].N, alt);
    if (!any) continue;
    p.item_mult = pick_g;
    p.morph_wps = pick_m;
    for (size_t g = 0; g < ng; ++g) p.sched[g] = stft_sched_distinct(p.groups[g].N, alt) ? alt : pick_s[g];
    if ((rc = run_timed(&ms, &mm)) != RISE_OK) break;
    std::map<int, float> tot;
    for (size_t g = 0; g < ng; ++g) tot[p.groups[g].N] += ms[g];
    for (auto &kv : tot) {
      bool has = false;
      for (size_t g = 0; g < ng; ++g) has = has || (p.groups[g].N == kv.first && p.sched[g] == alt);
      if (has && kv.second < best_n[kv.first]) {
        best_n[kv.first] = kv.second;
        for (size_t g = 0; g < ng; ++g)
          if (p.groups[g].N == kv.first) pick_s[g] = alt;
      }
    }
  }
  for (auto &e : ev.e)
    if (e) cudaEventDestroy(e);
  if (rc) return rc;
  Tuned t;
  t.item_mult = pick_g;
  t.sched = pick_s;
  t.morph_wps = pick_m;
  c->batch.tuned[p.shape_key] = pack(t);
  cache_store(c, p.shape_key, t);
  return RISE_OK;
}

// per capture: the cluster histogram stores whole columns from one cluster
// of 8 row bands of at most 65535 rows
constexpr int64_t kBatchMaxRows = 8 * 65535;

int check_capture(const rise_capture &k) {
  if (!k.iq_dev || (reinterpret_cast<uintptr_t>(k.iq_dev) & 7) != 0) return RISE_EINVAL;
  if (!pow2(k.fft_size) || k.fft_size < RISE_MIN_FFT || k.fft_size > RISE_MAX_FFT) return RISE_EINVAL;
  if (k.hop < 1 || k.hop > k.fft_size || k.n < k.fft_size) return RISE_EINVAL;
  const int64_t T = (k.n - k.fft_size) / k.hop + 1;
  if (T > RISE_MAX_ROWS || T > kBatchMaxRows) return RISE_EINVAL;
  return RISE_OK;
}

}  // namespace

}  // namespace host
void batch_preload() { preload_kernel(host::copy16_kernel); }
namespace host {

void destroy_batch(rise_ctx *c) {
  BatchState &b = c->batch;
  destroy_graphs(b);
  for (auto &g : c->single_graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  c->single_graphs.clear();
  if (b.tab.p) cudaFree(b.tab.p);
  if (b.small.p) cudaFree(b.small.p);
  if (b.counters.p) cudaFree(b.counters.p);
  if (b.tab_h) cudaFreeHost(b.tab_h);
  if (b.offs_h) cudaFreeHost(b.offs_h);
  b = BatchState();
}

int reserve_batch(rise_ctx *c, const rise_capture *caps, int ncap, const rise_thresholds &thr,
                  int64_t cap) {
  if (!c || ncap < 1 || !caps || cap < 0 || c->npend) return RISE_EINVAL;
  c->cur = 0;   // the slot whose box buffer a batch uses
  for (int k = 0; k < ncap; ++k) {
    int rc = check_capture(caps[k]);
    if (rc) return rc;
    if ((rc = check_thresholds(thr, caps[k].fft_size))) return rc;
  }
  CK(cudaSetDevice(c->device));
  Plan p;
  int rc = make_plan(caps, ncap, thr.range_mode == RISE_RANGE_FIXED, p);
  if (rc) return rc;
  if ((rc = upload_level_tables(c, thr.level_db))) return rc;
  if ((rc = upload_sg(c, thr.sg_half_window))) return rc;
  for (const auto &g : p.groups) {
    Tables *tb;
    if ((rc = get_tables(c, g.N, default_sched(g.N), &tb))) return rc;
  }
  // the default launch parameters (what an untuned batch uses)
  p.item_mult.assign(p.groups.size(), 2);
  p.sched.assign(p.groups.size(), 0);
  for (size_t g = 0; g < p.groups.size(); ++g) p.sched[g] = default_sched(p.groups[g].N);
  p.morph_wps = 16;
  size_tables(c, caps, p);
  return ensure_buffers(c, p, cap);
}

int detect_batch(rise_ctx *c, const rise_capture *caps, int ncap, const rise_thresholds *thr_in,
                 rise_box *out, int64_t cap, int64_t *offsets) {
  rise_thresholds thr;
  if (thr_in) thr = *thr_in;
  else rise_thresholds_default(&thr);
  if (!c || !offsets || ncap < 0 || cap < 0 || (cap > 0 && !out) || (ncap > 0 && !caps) || c->npend)
    return RISE_EINVAL;
  c->cur = 0;
  if (ncap == 0) {
    offsets[0] = 0;
    return RISE_OK;
  }
  for (int k = 0; k < ncap; ++k) {
    int rc = check_capture(caps[k]);
    if (rc) return rc;
    if ((rc = check_thresholds(thr, caps[k].fft_size))) return rc;
  }
  CK(cudaSetDevice(c->device));
  c->last_valid = false;
  c->batch.last_valid = false;
  Plan p;
  int rc = make_plan(caps, ncap, thr.range_mode == RISE_RANGE_FIXED, p);
  if (rc) return rc;
  if ((rc = upload_level_tables(c, thr.level_db))) return rc;
  if ((rc = upload_sg(c, thr.sg_half_window))) return rc;
  // launch parameters: tuned once per composition (or read from the tune
  // cache), else the defaults
  const size_t ng = p.groups.size();
  auto it = c->batch.tuned.find(p.shape_key);
  if (it == c->batch.tuned.end() && c->autotune) {
    Tuned t;
    if (cache_lookup(c, p.shape_key, ng, &t)) {
      c->batch.tuned[p.shape_key] = pack(t);
      c->batch.cache_hits += 1;
    } else if ((rc = autotune(c, caps, p, thr, cap))) {
      return rc;
    }
    it = c->batch.tuned.find(p.shape_key);
  }
  Tuned use;
  if (it == c->batch.tuned.end() || !unpack(it->second, ng, &use)) {
    use.item_mult.assign(ng, 2);
    use.sched.assign(ng, 0);
    for (size_t g = 0; g < ng; ++g) use.sched[g] = default_sched(p.groups[g].N);
    use.morph_wps = 16;
  }
  p.item_mult = use.item_mult;
  p.sched = use.sched;
  p.morph_wps = use.morph_wps;
  for (size_t g = 0; g < ng; ++g) c->sched_pick[p.groups[g].N] = p.sched[g];
  size_tables(c, caps, p);
  if ((rc = ensure_buffers(c, p, cap))) return rc;
  if ((rc = fill_tables(c, caps, p, thr))) return rc;
  BatchState &b = c->batch;
  bool launched = false;
  if (c->graphs) {
    const uint64_t key = graph_key(p, thr, cap, c->gen, c->timing);
    BatchState::Graph *gr = nullptr;
    for (auto &g : b.graphs)
      if (g.key == key) gr = &g;
    // a composition is captured the second time it comes: one that comes
    // once (a served batch of an odd size) does not pay for a capture
    bool capture = false;
    if (!gr) {
      auto it = std::find(b.seen.begin(), b.seen.end(), key);
      if (it != b.seen.end()) {
        b.seen.erase(it);
        capture = true;
      } else {
        if (b.seen.size() >= 64) b.seen.erase(b.seen.begin());
        b.seen.push_back(key);
      }
    }
    if (capture) {
      cudaGraph_t graph = nullptr;
      int nl = 0;
      if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        const int erc = enqueue(c, p, thr, cap, nullptr, &nl, true);
        count_launches(-nl);   // counted when the graph runs
        const cudaError_t ee = cudaStreamEndCapture(c->stream, &graph);
        cudaGraphExec_t exec = nullptr;
        if (erc == RISE_OK && ee == cudaSuccess && graph &&
            cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
          if ((int)b.graphs.size() >= kMaxGraphs) {
            cudaGraphExecDestroy(b.graphs.front().exec);
            b.graphs.erase(b.graphs.begin());
          }
          b.graphs.push_back({key, exec});
          b.captures += 1;
          b.graphs.back().launches = nl;
          gr = &b.graphs.back();
        }
        if (graph) cudaGraphDestroy(graph);
      }
      cudaGetLastError();   // a failed capture falls back to direct launches
    }
    if (gr) {
      CK(cudaGraphLaunch(gr->exec, c->stream));
      count_launches(gr->launches);
      launched = true;
    }
  }
  if (!launched && (rc = enqueue(c, p, thr, cap, nullptr, nullptr, false))) return rc;
  CK(wait_stream(c));
  DeviceStatus h = (*c->cs().st_h);
  if (h.err & ERR_RUN_CAPACITY) {
    // more runs than the run arrays hold: grow them and run the chain again
    // doubled: each growth synchronises the device and drops the graphs
    const int64_t need = std::max<int64_t>(2 * h.n_runs, 2 * c->run_cap);
    c->batch.relabels += 1;
    if ((rc = ensure(c, c->run_parent, need * sizeof(int32_t)))) return rc;
    if ((rc = ensure(c, c->run_sroot, need))) return rc;
    if ((rc = ensure(c, c->rec, need * sizeof(rise_box)))) return rc;
    if ((rc = ensure(c, c->merge, need * sizeof(int2)))) return rc;
    if ((rc = ensure(c, c->run_out, (need + 1) * sizeof(int64_t)))) return rc;
    if ((rc = ensure(c, c->scan_tmp, ccl_scan_tmp_bytes(std::max<int64_t>(need, p.total_rows + 1)))))
      return rc;
    c->run_cap = need;
    if ((rc = fill_tables(c, caps, p, thr))) return rc;
    if ((rc = enqueue(c, p, thr, cap, nullptr, nullptr, false))) return rc;
    CK(wait_stream(c));
    h = (*c->cs().st_h);
  }
  c->last_status = c->cs().st_h;
  b.last_valid = true;   // images, power and anchors stay until the next call moves or overwrites them
  b.last_fixed = p.fixed;
  b.last_ncap = ncap;
  b.last_px = p.total_px;
  b.last_hi_db = thr.hi_db;
  if (h.err & (ERR_UNION_LIMIT | ERR_SCAN | ERR_COPY_WAIT)) return RISE_ETIMEOUT;
  if (h.err) return RISE_EINTERNAL;
  std::memcpy(offsets, b.offs_h, sizeof(int64_t) * (ncap + 1));
  const int64_t total = h.n_boxes;
  const int64_t ncopy = std::min<int64_t>(total, cap);
  if (ncopy > 0) std::memcpy(out, c->cs().hbox, (size_t)ncopy * sizeof(rise_box));
  if (c->timing) {
    for (int i = 0; i < 7; ++i) cudaEventElapsedTime(&c->stage_ms[i], c->cs().ev[i], c->cs().ev[i + 1]);
    cudaEventElapsedTime(&c->stage_ms[7], c->cs().ev[0], c->cs().ev[7]);
  }
  b.last_groups = (int)p.groups.size();
  b.last_params.assign(p.item_mult.begin(), p.item_mult.end());
  b.last_params.push_back(p.morph_wps);
  b.last_params.insert(b.last_params.end(), p.sched.begin(), p.sched.end());
  for (const auto &g : p.groups) b.last_params.push_back(g.N);
  b.last_graph = launched;
  return total > cap ? RISE_ETRUNC : RISE_OK;
}

}  // namespace host
}  // namespace rise

extern "C" int rise_detect_batch(rise_ctx *ctx, const rise_capture *caps, int ncap,
                                 const rise_thresholds *thr, rise_box *out, int64_t cap,
                                 int64_t *offsets) {
  return rise::host::detect_batch(ctx, caps, ncap, thr, out, cap, offsets);
}
