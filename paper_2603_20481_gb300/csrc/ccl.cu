// Connected-component labelling of the final mask and the per-component box
// reduction (RISE Sec. IV-B, "Bounding box generation": 4-neighbour
// connectivity; each block's box is the min/max of its time and frequency
// indices, Eq. 1).
//
// The unit of labelling is the run: a maximal horizontal segment of
// foreground pixels in one row.  Runs are numbered in raster order of their
// first pixel (row-major scan over the bit-packed mask), so the smallest run
// number of a component is its raster-first pixel -- the anchor.  Union-find
// links by smaller number, hence every root is the anchor run and the final
// roots, taken in run order, are the boxes in anchor order.
//
//   1. the morphology kernel counts the runs of each row; a single-pass
//      exclusive scan gives row_base[t], the number of the first run of row t.
//   2. init: every run is its own tree (done by the row-offset scan; a
//      separate kernel when the labelling runs again with grown arrays).
//   3. rows: one warp per row records each run's extent, area, level sum and
//      energy, and unites it with the runs of the next row that share a
//      column (4-connectivity), on a global lock-free union-find.
//   4. reduce: every run adds its record into its root's (warp-aggregated).
//   5. compact: a single-pass scan of the root flags gives each root its box
//      slot (boxes in run order) and writes its record there.
// Every stage touches only rows that hold runs: the foreground of a spectrum
// mask is sparse, so the work follows the runs, not the pixels.
#include "common.cuh"

namespace rise {
namespace {

constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 8, SCAN_BLOCK = SCAN_THREADS * SCAN_ITEMS;

// ---------------------------------------------------------------------------
// Single-pass exclusive scans (decoupled look-back).  A block takes the next
// tile of SCAN_BLOCK items by ticket, so every tile it waits for belongs to a
// block that started earlier and is running or done.  It publishes its tile
// sum at once, then walks back over its predecessors' published sums until
// one carries a full prefix, and publishes its own.  Published words hold a
// state in the top two bits and the value below.  The state words and the
// ticket live in the scan scratch and are zeroed before each scan; every
// wait is bounded (ERR_SCAN).
// ---------------------------------------------------------------------------
constexpr uint64_t LB_AGG = 1ull << 62, LB_INC = 2ull << 62, LB_VAL = (1ull << 62) - 1;

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint64_t *p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Warp 0 of tile `tile` (sum `agg`): the sum of all earlier tiles, returned
// to every lane.  The warp reads 32 predecessors at once (lane l: tile
// hi - l), waits until each has published (at most `spin_limit` polls),
// and adds the values up to and including the nearest full prefix; without
// one in the window it moves 32 tiles back.  Tiles before 0 read as a full
// prefix of 0.  The tile numbered `withhold` publishes nothing (a test of
// the bounded wait: its successors give up and report ERR_SCAN).
__device__ int64_t lookback(uint64_t *stat, int64_t tile, int64_t agg, DeviceStatus *st, int spin_limit,
                            int64_t withhold) {
  const int lane = threadIdx.x & 31;
  const bool publish = tile != withhold;
  if (tile == 0) {
    if (lane == 0 && publish) st_release(&stat[0], LB_INC | (uint64_t)agg);
    return 0;
  }
  if (lane == 0 && publish) st_release(&stat[tile], LB_AGG | (uint64_t)agg);
  int64_t excl = 0;
  for (int64_t hi = tile - 1;; hi -= 32) {
    const int64_t k = hi - lane;
    uint64_t w = LB_INC;
    bool late = false;
    if (k >= 0) {
      w = ld_acquire(&stat[k]);
      for (int spins = 0; (w >> 62) == 0; ++spins) {
        if (spins >= spin_limit) {
          late = true;
          break;
        }
        __nanosleep(32);
        w = ld_acquire(&stat[k]);
      }
    }
    if (__any_sync(0xffffffffu, late)) {
      if (lane == 0) set_err(st, ERR_SCAN);
      return excl;
    }
    const unsigned inc = __ballot_sync(0xffffffffu, (w >> 62) == 2);
    const int first = inc ? __ffs(inc) - 1 : 31;   // the nearest full prefix
    int64_t v = lane <= first ? (int64_t)(w & LB_VAL) : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (inc) break;
  }
  if (lane == 0 && publish) st_release(&stat[tile], LB_INC | (uint64_t)(excl + agg));
  return excl;
}

// Scan scratch: [0] ticket of the row scan, [1] ticket of the root scan,
// [2] blocks of the root scan done, [3, 3 + tiles) row-scan tile words, then
// root-scan tile words.
struct ScanState {
  uint64_t *ticket_rows, *ticket_roots, *done_roots, *rows, *roots;
};
__host__ __device__ inline int64_t scan_tiles(int64_t n) { return n / SCAN_BLOCK + 1; }
inline ScanState scan_state(void *tmp, int64_t row_tiles) {
  uint64_t *w = static_cast<uint64_t *>(tmp);
  return ScanState{w, w + 1, w + 2, w + 3, w + 3 + row_tiles};
}

// A tile's items, their exclusive offsets within the whole scan and (for the
// last tile) the total.  `ex` receives each item's offset; returns the tile's
// first offset.
template <typename In>
__device__ __forceinline__ void tile_scan(const In *in, int64_t n, int64_t tile, uint64_t *stat,
                                          DeviceStatus *st, int64_t (&v)[SCAN_ITEMS],
                                          int64_t (&ex)[SCAN_ITEMS], int spin_limit, int64_t withhold) {
  __shared__ int64_t scratch[32];
  __shared__ int64_t s_prefix;
  const int64_t base = tile * SCAN_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t sum = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t k = base + i;
    v[i] = k < n ? (int64_t)in[k] : 0;
    sum += v[i];
  }
  int64_t tot;
  const int64_t mine = block_exclusive_scan<int64_t>(sum, scratch, &tot);
  if (threadIdx.x < 32) {
    const int64_t e = lookback(stat, tile, tot, st, spin_limit, withhold);
    if (threadIdx.x == 0) s_prefix = e;
  }
  __syncthreads();
  int64_t run = s_prefix + mine;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    ex[i] = run;
    run += v[i];
  }
}

// Row offsets of the runs: row_base[t] = runs in rows before t, row_base[T]
// and n_runs = all runs.
__global__ void __launch_bounds__(SCAN_THREADS)
row_scan_kernel(const uint32_t *cnt, int64_t T, int64_t *row_base, DeviceStatus *st, ScanState ss,
                int32_t *run_parent, int64_t run_cap, int spin_limit) {
  __shared__ int64_t s_tile, s_lo, s_hi;
  if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(ss.ticket_rows), 1ull);
  __syncthreads();
  const int64_t tile = s_tile;
  if (tile >= scan_tiles(T)) return;
  int64_t v[SCAN_ITEMS], ex[SCAN_ITEMS];
  tile_scan<uint32_t>(cnt, T, tile, ss.rows, st, v, ex, spin_limit, -1);
  const int64_t base = tile * SCAN_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t k = base + i;
    if (k < T) row_base[k] = ex[i];
    if (k == T) {   // one past the last row: the total
      row_base[T] = ex[i];
      st->n_runs = ex[i];
      if (ex[i] > run_cap) set_err(st, ERR_RUN_CAPACITY);
    }
  }
  // the runs of this tile's rows start as trees of their own
  if (threadIdx.x == 0) s_lo = ex[0];
  if (threadIdx.x == SCAN_THREADS - 1) s_hi = ex[SCAN_ITEMS - 1] + v[SCAN_ITEMS - 1];
  __syncthreads();
  const int64_t hi = min(s_hi, run_cap);
  for (int64_t g = s_lo + threadIdx.x; g < hi; g += SCAN_THREADS) run_parent[g] = (int32_t)g;
}

// ---------------------------------------------------------------------------
// 2. per-run initialisation: every run is its own tree
// ---------------------------------------------------------------------------
__global__ void runs_init_kernel(CclArgs a, ScanState ss, int64_t root_tiles) {
  DeviceStatus *st = a.status;
  const int64_t n = st->n_runs;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *ss.ticket_roots = 0;   // the root scan's state (this chain may run again on a relabel)
    *ss.done_roots = 0;
  }
  if (n > a.run_cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_err(st, ERR_RUN_CAPACITY);
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->n_merge = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < root_tiles;
       k += (int64_t)gridDim.x * blockDim.x)
    ss.roots[k] = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    a.run_parent[g] = (int)g;
  }
}

// ---------------------------------------------------------------------------
// 3. one warp per row t: the row's runs (numbered from row_base[t] in column
//    order) get their extent, area, level sum and energy, and every run of
//    row t is united with the runs of row t+1 it touches (4-connectivity:
//    the two runs share a column).  Lane l handles row word 32c + l of chunk
//    c; run ranks come from a warp scan of run-start counts.
// ---------------------------------------------------------------------------
constexpr int ROW_WARPS = 8;

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int *total) {
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  *total = __shfl_sync(0xffffffffu, x, 31);
  return x - v;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Row t (of T) of an image of width F whose mask and levels start at
// mask0 / img0; tg is the row's index in the run-count arrays (the same as t
// for a single image).  Rows without runs are skipped by the callers.
// The row is latency-bound, so every load it needs is issued first: the
// next row's run count, both rows' run offsets and mask words (MAXC chunks
// of 32 words, in registers), then this lane's levels of its foreground
// words (asynchronous copies into `lq`, MAXC x 32 bytes of shared memory).
// Extents and unions are done while the levels are in flight; the level and
// energy sums come last.
template <int MAXC>
__device__ __forceinline__ void runs_row_body(const CclArgs &a, const unsigned long long *Es, uint8_t *lq,
                                              int64_t tg, int64_t t, int64_t T, int F,
                                              const uint32_t *mask0, const uint8_t *img0) {
  DeviceStatus *st = a.status;
  const int lane = threadIdx.x & 31;
  const int Wd = F / 32;
  const int nch = (Wd + 31) / 32;   // <= MAXC
  const bool next_in = t + 1 < T;
  const uint32_t *m = mask0 + t * Wd;
  const uint32_t *m2 = mask0 + (next_in ? t + 1 : t) * Wd;
  const uint32_t cnt2 = next_in ? a.row_cnt[tg + 1] : 0u;
  const int64_t base = a.row_base[tg];
  const int64_t base2 = next_in ? a.row_base[tg + 1] : 0;
  uint32_t X[MAXC], Y[MAXC];
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    const int w = 32 * c + lane;
    const bool in = c < nch && w < Wd;
    X[c] = in ? m[w] : 0u;
    Y[c] = in && next_in ? m2[w] : 0u;
  }
  const uint32_t lq_s = static_cast<uint32_t>(__cvta_generic_to_shared(lq));
  const uint8_t *qrow = img0 + t * F;
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    if (X[c]) {   // a foreground word: c < nch and w < Wd
      const uint8_t *src = qrow + 32 * (32 * c + lane);
      cp_async16(lq_s + 32 * c, src);
      cp_async16(lq_s + 32 * c + 16, src + 16);
    }
  }
  const bool has_next = cnt2 != 0;
  uint32_t SX[MAXC];
  int BS[MAXC];
  uint32_t cx = 0, cy = 0;       // previous chunk's last words
  int nst = 0, nen = 0, nsy = 0; // runs started / ended before this chunk
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    SX[c] = 0;
    BS[c] = 0;
    if (c >= nch) continue;   // warp-uniform
    const int w = 32 * c + lane;
    const uint32_t x = X[c];
    const uint32_t y = has_next ? Y[c] : 0u;
    uint32_t px = __shfl_up_sync(0xffffffffu, x, 1), py = __shfl_up_sync(0xffffffffu, y, 1);
    if (lane == 0) { px = cx; py = cy; }
    uint32_t nx = __shfl_down_sync(0xffffffffu, x, 1);
    const uint32_t nx0 = __shfl_sync(0xffffffffu, c + 1 < MAXC ? X[c + 1 < MAXC ? c + 1 : c] : 0u, 0);
    if (lane == 31) nx = (c + 1 < nch) ? nx0 : 0u;
    const uint32_t sx = run_starts(x, px), ex = run_ends(x, nx), sy = run_starts(y, py);
    int tot_s, tot_e, tot_y;
    const int bs = nst + warp_excl_scan(__popc(sx), lane, &tot_s);
    const int be = nen + warp_excl_scan(__popc(ex), lane, &tot_e);
    const int by = nsy + warp_excl_scan(__popc(sy), lane, &tot_y);
    SX[c] = sx;
    BS[c] = bs;
    if (x) {
      // extent: the start lane owns t0, t1, f0, anchor; the end lane owns f1
      uint32_t ss = sx;
      int id = bs;
      while (ss) {
        const int b = __ffs(ss) - 1;
        ss &= ss - 1;
        if (!ck_index(base + id, a.run_cap, st)) break;
        rise_box *rc = &a.rec[base + id++];
        rc->t0 = (int32_t)t;
        rc->t1 = (int32_t)t;
        rc->f0 = 32 * w + b;
        rc->anchor = t * F + 32 * w + b;
      }
      uint32_t ee = ex;
      id = be;
      while (ee) {
        const int b = __ffs(ee) - 1;
        ee &= ee - 1;
        if (!ck_index(base + id, a.run_cap, st)) break;
        a.rec[base + id++].f1 = 32 * w + b;
      }
    }
    // union with the runs of the next row that share a column
    const uint32_t ov = x & y;
    if (ov) {
      uint32_t os = ov & ~((ov << 1) | ((px & py) >> 31));
      while (os) {
        const int cc = __ffs(os) - 1;
        os &= os - 1;
        const int ia = (int)(base + bs + __popc(sx & mask_upto(cc)) - 1);
        const int ib = (int)(base2 + by + __popc(sy & mask_upto(cc)) - 1);
        if (kChecked && !(ck_index(ia, a.run_cap, st) && ck_index(ib, a.run_cap, st) && ia < ib)) {
          set_err(st, ERR_INDEX);
          continue;
        }
        // a lower run touched by one upper run (the common case) hangs under
        // it with one CAS: ib is still a root and ia < ib, so this is a union.
        // A failed CAS means ib already hangs elsewhere (it touches a second
        // upper run): that union is deferred until the chains built here are
        // flattened, so this pass walks no chains.
        if (atomicCAS(&a.run_parent[ib], ib, ia) != ib) {
          const unsigned long long k = atomicAdd(reinterpret_cast<unsigned long long *>(&st->n_merge), 1ull);
          if ((int64_t)k < a.run_cap) a.merge[k] = make_int2(ia, ib);
          else uf_union(a.run_parent, ia, ib, st, a.uf_limit);   // list full: unite now (slower)
        }
      }
    }
    nst += tot_s;
    nen += tot_e;
    nsy += tot_y;
    cx = __shfl_sync(0xffffffffu, x, 31);
    cy = __shfl_sync(0xffffffffu, y, 31);
  }
  // area, level and energy sums of each segment of set bits in a word: a
  // run's first segment is stored (no zeroed record needed), the segment
  // continuing a run from an earlier word (at most one per word) is added
  // once every first segment of the chunk is stored
  cp_async_wait_all();
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    uint32_t mm = X[c];
    const uint8_t *myq = lq + 32 * c;
    rise_box *cont = nullptr;
    unsigned long long c_area = 0, c_sq = 0, c_se = 0;
    while (mm) {
      const int b0 = __ffs(mm) - 1;
      const uint32_t inv = ~(mm >> b0);
      const int len = inv ? __ffs(inv) - 1 : 32 - b0;
      uint32_t sq = 0;
      unsigned long long se = 0;
      for (int b = b0; b < b0 + len; ++b) {
        const uint32_t q = myq[b];
        sq += q;
        se += Es[q];
      }
      const int64_t ri = base + BS[c] + __popc(SX[c] & mask_upto(b0)) - 1;
      if (!ck_index(ri, a.run_cap, st)) break;
      rise_box *rc = &a.rec[ri];
      if ((SX[c] >> b0) & 1u) {
        rc->area = len;
        rc->sum_q = sq;
        rc->energy_fx = se;
      } else {
        cont = rc;
        c_area = (unsigned long long)len;
        c_sq = sq;
        c_se = se;
      }
      mm &= (len + b0 >= 32) ? 0u : ~0u << (b0 + len);
    }
    __syncwarp();   // orders the chunk's first-segment stores before the adds
    if (cont) {
      atomicAdd(reinterpret_cast<unsigned long long *>(&cont->area), c_area);
      atomicAdd(reinterpret_cast<unsigned long long *>(&cont->sum_q), c_sq);
      atomicAdd(reinterpret_cast<unsigned long long *>(&cont->energy_fx), c_se);
    }
  }
}

// levels staged per lane: MAXC chunks x 32 bytes, lanes 16 bytes apart more
// than that (fewer bank conflicts on the byte reads; copies stay 16-aligned)
constexpr int row_lane_bytes(int maxc) { return maxc * 32 + 16; }
constexpr size_t row_smem(int maxc) { return (size_t)ROW_WARPS * 32 * row_lane_bytes(maxc); }

template <int MAXC>
__global__ void __launch_bounds__(32 * ROW_WARPS, MAXC >= 8 ? 3 : 4)
runs_row_kernel(CclArgs a) {
  __shared__ unsigned long long Es[256];
  extern __shared__ __align__(16) uint8_t lqs[];   // [ROW_WARPS][32 lanes][row_lane_bytes]
  for (int i = threadIdx.x; i < 256; i += blockDim.x) Es[i] = a.energy[i];
  __syncthreads();
  if (a.status->n_runs > a.run_cap) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * ROW_WARPS + wib;
  if (t >= a.T) return;
  if (a.row_cnt[t] == 0) return;   // no runs in this row: nothing to label or unite
  runs_row_body<MAXC>(a, Es, lqs + (wib * 32 + lane) * row_lane_bytes(MAXC), t, t, a.T, a.F, a.mask, a.img);
}

// Batch: rows of all captures, concatenated (a.T = total rows); row0[c] is
// the first row of capture c (ncap + 1 entries).  Rows of different
// captures are never united: has_next stops at the capture's last row.
template <int MAXC>
__global__ void __launch_bounds__(32 * ROW_WARPS, MAXC >= 8 ? 3 : 4)
runs_row_batch_kernel(CclArgs a, const RowSeg *segs, const int64_t *row0, int ncap) {
  __shared__ unsigned long long Es[256];
  extern __shared__ __align__(16) uint8_t lqs[];
  for (int i = threadIdx.x; i < 256; i += blockDim.x) Es[i] = a.energy[i];
  __syncthreads();
  if (a.status->n_runs > a.run_cap) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t tg = (int64_t)blockIdx.x * ROW_WARPS + wib;
  if (tg >= a.T) return;
  if (a.row_cnt[tg] == 0) return;
  int lo = 0, hi = ncap - 1;   // the last capture whose first row is <= tg
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&row0[mid]) <= tg) lo = mid;
    else hi = mid - 1;
  }
  const RowSeg rs = segs[lo];
  if (!ck_index(tg - __ldg(&row0[lo]), rs.T, a.status)) return;
  runs_row_body<MAXC>(a, Es, lqs + (wib * 32 + lane) * row_lane_bytes(MAXC), tg, tg - __ldg(&row0[lo]), rs.T, rs.F,
                      rs.mask, rs.img);
}

template <int MAXC>
cudaError_t launch_rows(const CclArgs &a, const RowSeg *segs, const int64_t *row0, int ncap, cudaStream_t s) {
  const unsigned row_blocks = (unsigned)((a.T + ROW_WARPS - 1) / ROW_WARPS);
  const size_t sm = row_smem(MAXC);
  cudaError_t e;
  if (segs) {
    e = cudaFuncSetAttribute(runs_row_batch_kernel<MAXC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    runs_row_batch_kernel<MAXC><<<row_blocks, 32 * ROW_WARPS, sm, s>>>(a, segs, row0, ncap);
  } else {
    e = cudaFuncSetAttribute(runs_row_kernel<MAXC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    runs_row_kernel<MAXC><<<row_blocks, 32 * ROW_WARPS, sm, s>>>(a);
  }
  count_launches(1);
  return cudaGetLastError();
}

// Batch: offs[c] = index of capture c's first box in the output (boxes of a
// batch are ordered by capture, then anchor); offs[ncap] = all boxes.
__global__ void ccl_offsets_kernel(CclArgs a, const int64_t *row0, int ncap, int64_t *offs) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > ncap) return;
  const DeviceStatus *st = a.status;
  const int64_t n = st->n_runs;
  if (n > a.run_cap) {
    offs[c] = 0;
    return;
  }
  if (c == ncap) {
    offs[c] = st->n_boxes;
    return;
  }
  if (!ck_index(row0[c], a.T + 1, a.status)) return;
  const int64_t r = a.row_base[row0[c]];   // the capture's first run
  offs[c] = r < n ? a.run_out[r] : st->n_boxes;
}

// ---------------------------------------------------------------------------
// 3b. point every run straight at its root (the row pass leaves chains as
//     tall as the component), then apply the deferred unions.
// ---------------------------------------------------------------------------
// FLATTEN: every thread points its runs at their roots; MERGE: it applies
// its share of the deferred unions.  With both in one launch (one image:
// few runs, the launch costs more than the overlap) the phases of different
// threads overlap, which the lock-free union-find allows: a path-halving
// store always writes an ancestor, and a union links one root under a
// smaller root with a CAS that fails if the root has moved.  Batches (many
// runs, tall chains) run the phases as two launches.
template <bool FLATTEN, bool MERGE>
__global__ void ccl_flatten_merge_kernel(CclArgs a) {
  DeviceStatus *st = a.status;
  const int64_t n = st->n_runs;
  if (n > a.run_cap) return;
  if (FLATTEN) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
         g += (int64_t)gridDim.x * blockDim.x) {
      const int r = uf_find(a.run_parent, (int)g, st, a.uf_limit);
      if (r != (int)g) *(volatile int *)&a.run_parent[g] = r;   // an ancestor: still valid
    }
  }
  if (!MERGE) return;
  const int64_t m = min(st->n_merge, a.run_cap);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 e = a.merge[k];
    uf_union(a.run_parent, e.x, e.y, st, a.uf_limit);
  }
}

// ---------------------------------------------------------------------------
// 4. every run that is not its component's root adds its record into the
//    root's; run_sroot is set to 1 exactly for the roots.  Lanes of a warp with
//    the same root combine first, so a tall component costs one atomic per
//    field per warp rather than per run.
// ---------------------------------------------------------------------------
__global__ void ccl_reduce_kernel(CclArgs a) {
  DeviceStatus *st = a.status;
  const int64_t n = st->n_runs;
  if (n > a.run_cap) return;
  const int lane = threadIdx.x & 31;
  for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x; g0 < n; g0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t g = g0 + threadIdx.x;
    const bool live = g < n;
    int r = live ? uf_find(a.run_parent, (int)g, st, a.uf_limit) : -1;
    const bool contrib = live && r != (int)g;
    if (live) a.run_sroot[g] = contrib ? 0 : 1;
    rise_box src;
    if (contrib) src = a.rec[g];
    const unsigned grp = __match_any_sync(0xffffffffu, contrib ? r : -1);
    if (contrib) {
      // every lane of the group walks the group's members in the same order;
      // the lowest lane accumulates and issues the atomics
      const int leader = __ffs(grp) - 1;
      int t1 = INT32_MIN, f0 = INT32_MAX, f1 = INT32_MIN;
      unsigned long long ar = 0, sq = 0, en = 0;
      for (unsigned mm = grp; mm; mm &= mm - 1) {
        const int sl = __ffs(mm) - 1;
        t1 = max(t1, __shfl_sync(grp, src.t1, sl));
        f0 = min(f0, __shfl_sync(grp, src.f0, sl));
        f1 = max(f1, __shfl_sync(grp, src.f1, sl));
        ar += __shfl_sync(grp, (unsigned long long)src.area, sl);
        sq += __shfl_sync(grp, (unsigned long long)src.sum_q, sl);
        en += __shfl_sync(grp, (unsigned long long)src.energy_fx, sl);
      }
      if (lane == leader) {
        rise_box *dst = &a.rec[r];
        atomicMax(&dst->t1, t1);
        atomicMin(&dst->f0, f0);
        atomicMax(&dst->f1, f1);
        atomicAdd(reinterpret_cast<unsigned long long *>(&dst->area), ar);
        atomicAdd(reinterpret_cast<unsigned long long *>(&dst->sum_q), sq);
        atomicAdd(reinterpret_cast<unsigned long long *>(&dst->energy_fx), en);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// 5. box slots of the global roots (run_sroot flags exactly them): one
//    single-pass scan that also writes each root's record to its slot; with
//    too many runs for the arrays, no boxes
// ---------------------------------------------------------------------------
__device__ __forceinline__ void root_scan_body(const CclArgs &a, const ScanState &ss) {
  DeviceStatus *st = a.status;
  const int64_t n = st->n_runs;
  if (n > a.run_cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) st->n_boxes = 0;
    return;
  }
  // persistent: the grid is sized on the capacity, the tiles on the runs
  const int64_t tiles = scan_tiles(n);
  __shared__ int64_t s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = (int64_t)atomicAdd(reinterpret_cast<unsigned long long *>(ss.ticket_roots), 1ull);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= tiles) return;
    int64_t v[SCAN_ITEMS], ex[SCAN_ITEMS];
    tile_scan<uint8_t>(a.run_sroot, n, tile, ss.roots, st, v, ex, a.spin_limit, a.withhold_tile);
    const int64_t base = tile * SCAN_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
      const int64_t k = base + i;
      if (k < n) {
        a.run_out[k] = ex[i];
        if (v[i] && ex[i] < a.box_cap) a.boxes[ex[i]] = a.rec[k];
      }
      if (k == n) {
        a.run_out[n] = ex[i];
        st->n_boxes = ex[i];
      }
    }
    __syncthreads();   // s_tile and the scan's shared words are reused
  }
}

// The last kernel of a single image's chain: after the scan, the last block
// to finish copies the status to the caller's mapped host copy (no copy
// node after the kernel).
__global__ void __launch_bounds__(SCAN_THREADS) root_scan_kernel(CclArgs a, ScanState ss) {
  root_scan_body(a, ss);
  if (!a.status_out) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned long long d = atomicAdd(reinterpret_cast<unsigned long long *>(ss.done_roots), 1ull);
    if (d == gridDim.x - 1) {   // every other block has finished its status writes
      __threadfence();
      const volatile uint32_t *src = reinterpret_cast<const volatile uint32_t *>(a.status);
      volatile uint32_t *dst = reinterpret_cast<volatile uint32_t *>(a.status_out);
      for (int i = 0; i < (int)(sizeof(DeviceStatus) / 4); ++i) dst[i] = src[i];
      __threadfence_system();
    }
  }
}

// ---------------------------------------------------------------------------
// Block shapes after labelling: every run's component (its box index) and
// span, and the boundary pixels of the final mask.
// ---------------------------------------------------------------------------
// A non-root run keeps its own record; a root's record became its
// component's box, so its own span is taken from its anchor and the mask.
__global__ void runs_export_kernel(CclArgs a, int4 *out, int64_t cap) {
  DeviceStatus *st = a.status;
  const int64_t n = st->n_runs;
  if (n > a.run_cap) return;
  const int Wd = a.F / 32;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < min(n, cap);
       g += (int64_t)gridDim.x * blockDim.x) {
    const int r = uf_find(a.run_parent, (int)g, st, a.uf_limit);
    const rise_box &b = a.rec[g];
    int t, f0, f1;
    if (r != (int)g) {
      t = b.t0;
      f0 = b.f0;
      f1 = b.f1;
    } else {
      if (!ck_index(b.anchor, a.T * (int64_t)a.F, st)) continue;
      t = (int)(b.anchor / a.F);
      f0 = (int)(b.anchor % a.F);
      const uint32_t *row = a.mask + (int64_t)t * Wd;
      f1 = a.F - 1;
      for (int w = f0 >> 5; w < Wd; ++w) {   // first background bit after f0
        const uint32_t z = ~row[w] & (w == (f0 >> 5) ? (~0u << (f0 & 31)) : ~0u);
        if (z) {
          f1 = 32 * w + __ffs(z) - 2;
          break;
        }
      }
    }
    out[g] = make_int4((int)a.run_out[r], t, f0, f1);
  }
}

// boundary = foreground with a background 4-neighbour (outside is background)
__global__ void boundary_kernel(const uint32_t *mask, int64_t T, int F, uint32_t *out) {
  const int Wd = F / 32;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < T * Wd;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = i / Wd;
    const int w = (int)(i % Wd);
    const uint32_t m = mask[i];
    const uint32_t up = t > 0 ? mask[i - Wd] : 0u, dn = t + 1 < T ? mask[i + Wd] : 0u;
    const uint32_t prev = w > 0 ? mask[i - 1] : 0u, next = w + 1 < Wd ? mask[i + 1] : 0u;
    const uint32_t left = (m << 1) | (prev >> 31);    // bit f: pixel f - 1
    const uint32_t right = (m >> 1) | (next << 31);   // bit f: pixel f + 1
    out[i] = m & ~(up & dn & left & right);
  }
}

// Grid of the run-indexed kernels (grid-stride loops), sized on the run
// capacity and capped at `per_sm` blocks per SM: one image's runs are
// usually a small fraction of the capacity (idle blocks still cost), a
// batch's are many (more threads shorten the union-find walks).
int grid_for(int64_t n, int threads, int num_sms, int per_sm) {
  int64_t g = (n + threads - 1) / threads;
  g = std::min<int64_t>(g, (int64_t)num_sms * per_sm);
  return (int)std::max<int64_t>(1, g);
}

}  // namespace

size_t ccl_scan_tmp_bytes(int64_t max_items) {
  return (size_t)(3 + 2 * scan_tiles(max_items)) * sizeof(uint64_t);
}

cudaError_t launch_ccl_count(const CclArgs &a, int num_sms, cudaStream_t s) {
  (void)num_sms;
  const int64_t tiles = scan_tiles(a.T);
  if ((size_t)(3 + tiles + scan_tiles(a.run_cap)) * sizeof(uint64_t) > a.scan_tmp_bytes)
    return cudaErrorInvalidValue;
  const ScanState ss = scan_state(a.scan_tmp, tiles);
  // both scans' tickets and tile words (the root scan's too: no init kernel
  // runs between the two on this path)
  cudaError_t e =
      cudaMemsetAsync(a.scan_tmp, 0, (size_t)(3 + tiles + scan_tiles(a.run_cap)) * sizeof(uint64_t), s);
  if (e != cudaSuccess) return e;
  row_scan_kernel<<<(unsigned)tiles, SCAN_THREADS, 0, s>>>(a.row_cnt, a.T, a.row_base, a.status, ss,
                                                          a.run_parent, a.run_cap, a.spin_limit);
  count_launches(1);
  return cudaGetLastError();
}

namespace {
cudaError_t label_common(const CclArgs &a, const RowSeg *segs, const int64_t *row0, int ncap,
                         int64_t *offs, int num_sms, cudaStream_t s, bool after_count) {
  // 16 blocks a SM: the run-indexed kernels chase parent pointers, and the
  // more walks in flight the better (a grid of 4 per SM took the stress
  // capture's labelling from 0.47 to 0.60 ms)
  const int g = grid_for(a.run_cap, 256, num_sms, 16);
  const int64_t root_tiles = scan_tiles(a.run_cap);
  if ((size_t)(3 + scan_tiles(a.T) + root_tiles) * sizeof(uint64_t) > a.scan_tmp_bytes)
    return cudaErrorInvalidValue;
  const ScanState ss = scan_state(a.scan_tmp, scan_tiles(a.T));
  if (!after_count) {   // a relabel with larger run arrays: the row scan is not run again
    runs_init_kernel<<<g, 256, 0, s>>>(a, ss, root_tiles);
    count_launches(1);
  }
  // widest image of the launch (a.F; for a batch, the largest F)
  const int nch = (a.F / 32 + 31) / 32;
  cudaError_t er = nch <= 1 ? launch_rows<1>(a, segs, row0, ncap, s)
                   : nch <= 2 ? launch_rows<2>(a, segs, row0, ncap, s)
                   : nch <= 4 ? launch_rows<4>(a, segs, row0, ncap, s)
                              : launch_rows<8>(a, segs, row0, ncap, s);
  if (er != cudaSuccess) return er;
  if (segs) {
    ccl_flatten_merge_kernel<true, false><<<g, 256, 0, s>>>(a);
    ccl_flatten_merge_kernel<false, true><<<g, 256, 0, s>>>(a);
    count_launches(2);
  } else {
    ccl_flatten_merge_kernel<true, true><<<g, 256, 0, s>>>(a);
    count_launches(1);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ccl_reduce_kernel<<<g, 256, 0, s>>>(a);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  root_scan_kernel<<<(unsigned)std::min<int64_t>(root_tiles, (int64_t)num_sms * (segs ? 4 : 1)), SCAN_THREADS,
                     0, s>>>(a, ss);
  count_launches(1);
  if (segs) {
    ccl_offsets_kernel<<<(ncap + 1 + 255) / 256, 256, 0, s>>>(a, row0, ncap, offs);
    count_launches(1);
  }
  return cudaGetLastError();
}
}  // namespace

void ccl_preload() {
  preload_kernel(row_scan_kernel);
  preload_kernel(runs_init_kernel);
  preload_kernel(runs_row_kernel<1>);
  preload_kernel(runs_row_kernel<2>);
  preload_kernel(runs_row_kernel<4>);
  preload_kernel(runs_row_kernel<8>);
  preload_kernel(runs_row_batch_kernel<1>);
  preload_kernel(runs_row_batch_kernel<2>);
  preload_kernel(runs_row_batch_kernel<4>);
  preload_kernel(runs_row_batch_kernel<8>);
  preload_kernel(ccl_offsets_kernel);
  preload_kernel(ccl_flatten_merge_kernel<true, true>);
  preload_kernel(ccl_flatten_merge_kernel<true, false>);
  preload_kernel(ccl_flatten_merge_kernel<false, true>);
  preload_kernel(ccl_reduce_kernel);
  preload_kernel(root_scan_kernel);
  preload_kernel(runs_export_kernel);
  preload_kernel(boundary_kernel);
}

cudaError_t launch_runs_export(const CclArgs &a, int4 *out, int64_t cap, int num_sms, cudaStream_t s) {
  const int g = grid_for(std::max<int64_t>(cap, 1), 256, num_sms, 8);
  runs_export_kernel<<<g, 256, 0, s>>>(a, out, cap);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_boundary(const uint32_t *mask, int64_t T, int F, uint32_t *out, int num_sms,
                            cudaStream_t s) {
  const int g = grid_for(T * (F / 32), 256, num_sms, 8);
  boundary_kernel<<<g, 256, 0, s>>>(mask, T, F, out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_ccl_label(const CclArgs &a, int num_sms, cudaStream_t s, bool after_count) {
  return label_common(a, nullptr, nullptr, 0, nullptr, num_sms, s, after_count);
}

cudaError_t launch_ccl_label_batch(const CclArgs &a, const RowSeg *segs, const int64_t *row0,
                                   int ncap, int64_t *offs, int num_sms, cudaStream_t s) {
  return label_common(a, segs, row0, ncap, offs, num_sms, s, true);
}

}  // namespace rise
