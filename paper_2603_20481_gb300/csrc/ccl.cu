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
//   1. the morphology kernel counts the runs of each row; an exclusive scan
//      gives row_base[t], the number of the first run of row t.
//   2. init: every run is its own tree, with zeroed sums.
//   3. rows: one warp per row records each run's extent, area, level sum and
//      energy, and unites it with the runs of the next row that share a
//      column (4-connectivity), on a global lock-free union-find.
//   4. reduce: every run adds its record into its root's (warp-aggregated).
//   5. compact: roots -> exclusive scan -> boxes in run order.
// Every stage touches only rows that hold runs: the foreground of a spectrum
// mask is sparse, so the work follows the runs, not the pixels.
#include "common.cuh"

namespace rise {
namespace {

constexpr int CCL_THREADS = 256;
constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 8, SCAN_BLOCK = SCAN_THREADS * SCAN_ITEMS;

// ---------------------------------------------------------------------------
// Generic exclusive scan of counts (uint32 or uint8) into int64 offsets.
// The item count may live on the device (n_dev); the grid covers n_host.
// ---------------------------------------------------------------------------
template <typename In>
__global__ void __launch_bounds__(SCAN_THREADS)
scan_reduce_kernel(const In *in, const int64_t *n_dev, int64_t n_host, int64_t *partial) {
  const int64_t n = n_dev ? min(*n_dev, n_host) : n_host;
  const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK;
  int64_t s = 0;
  for (int i = threadIdx.x; i < SCAN_BLOCK; i += SCAN_THREADS) {
    const int64_t k = base + i;
    if (k < n) s += (int64_t)in[k];
  }
  __shared__ int64_t scratch[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) scratch[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < SCAN_THREADS / 32; ++w) t += scratch[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) scan_partials_kernel(int64_t *partial, int64_t nblocks) {
  __shared__ int64_t scratch[32];
  int64_t carry = 0;
  for (int64_t c0 = 0; c0 < nblocks; c0 += 1024) {
    const int64_t k = c0 + threadIdx.x;
    const int64_t v = k < nblocks ? partial[k] : 0;
    int64_t tot;
    const int64_t ex = block_exclusive_scan<int64_t>(v, scratch, &tot);
    if (k < nblocks) partial[k] = carry + ex;
    carry += tot;
  }
}

template <typename In>
__global__ void __launch_bounds__(SCAN_THREADS)
scan_apply_kernel(const In *in, const int64_t *n_dev, int64_t n_host, const int64_t *partial,
                  int64_t *out, int64_t *total_out) {
  const int64_t n = n_dev ? min(*n_dev, n_host) : n_host;
  const int64_t base = (int64_t)blockIdx.x * SCAN_BLOCK + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS];
  int64_t s = 0;
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t k = base + i;
    v[i] = k < n ? (int64_t)in[k] : 0;
    s += v[i];
  }
  __shared__ int64_t scratch[32];
  int64_t tot;
  int64_t run = block_exclusive_scan<int64_t>(s, scratch, &tot) + partial[blockIdx.x];
#pragma unroll
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    const int64_t k = base + i;
    if (k < n) out[k] = run;
    if (k == n - 1) {
      out[n] = run + v[i];
      if (total_out) *total_out = run + v[i];
    }
    run += v[i];
  }
  if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) {
    out[0] = 0;
    if (total_out) *total_out = 0;
  }
}

template <typename In>
cudaError_t device_scan(const In *in, const int64_t *n_dev, int64_t n_host, int64_t *out,
                        int64_t *total_out, int64_t *partial, cudaStream_t s) {
  const int64_t nb = std::max<int64_t>(1, (n_host + SCAN_BLOCK - 1) / SCAN_BLOCK);
  scan_reduce_kernel<In><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n_dev, n_host, partial);
  count_launches(1);
  scan_partials_kernel<<<1, 1024, 0, s>>>(partial, nb);
  count_launches(1);
  scan_apply_kernel<In><<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, n_dev, n_host, partial, out,
                                                               total_out);
  count_launches(1);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// 2. per-run initialisation: every run is its own tree and record
// ---------------------------------------------------------------------------
__global__ void runs_init_kernel(CclArgs a) {
  DeviceStatus *st = a.status;
  const int64_t n = st->n_runs;
  if (n > a.run_cap) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_err(st, ERR_RUN_CAPACITY);
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) st->n_merge = 0;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    a.run_parent[g] = (int)g;
    a.run_sroot[g] = 1;
    a.rec[g].area = 0;
    a.rec[g].sum_q = 0;
    a.rec[g].energy_fx = 0;
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

// Row t (of T) of an image of width F whose mask and levels start at
// mask0 / img0; tg is the row's index in the run-count arrays (the same as t
// for a single image).  Rows without runs are skipped by the callers.
__device__ __forceinline__ void runs_row_body(const CclArgs &a, const unsigned long long *Es,
                                              uint8_t *myq, int64_t tg, int64_t t, int64_t T, int F,
                                              const uint32_t *mask0, const uint8_t *img0) {
  DeviceStatus *st = a.status;
  const int lane = threadIdx.x & 31;
  const int Wd = F / 32;
  const uint32_t *m = mask0 + t * Wd;
  const bool has_next = t + 1 < T && a.row_cnt[tg + 1] != 0;
  const uint32_t *m2 = has_next ? mask0 + (t + 1) * Wd : nullptr;
  const int64_t base = a.row_base[tg], base2 = has_next ? a.row_base[tg + 1] : 0;
  uint32_t cx = 0, cy = 0;       // previous chunk's last words
  int nst = 0, nen = 0, nsy = 0; // runs started / ended before this chunk
  for (int w0 = 0; w0 < Wd; w0 += 32) {
    const int w = w0 + lane;
    const uint32_t x = w < Wd ? m[w] : 0u;
    const uint32_t y = (has_next && w < Wd) ? m2[w] : 0u;
    uint32_t px = __shfl_up_sync(0xffffffffu, x, 1), py = __shfl_up_sync(0xffffffffu, y, 1);
    if (lane == 0) { px = cx; py = cy; }
    uint32_t nx = __shfl_down_sync(0xffffffffu, x, 1);
    if (lane == 31) nx = (w + 1 < Wd) ? m[w + 1] : 0u;
    const uint32_t sx = run_starts(x, px), ex = run_ends(x, nx), sy = run_starts(y, py);
    int tot_s, tot_e, tot_y;
    const int bs = nst + warp_excl_scan(__popc(sx), lane, &tot_s);
    const int be = nen + warp_excl_scan(__popc(ex), lane, &tot_e);
    const int by = nsy + warp_excl_scan(__popc(sy), lane, &tot_y);
    if (x) {
      // extent: the start lane owns t0, t1, f0, anchor; the end lane owns f1
      uint32_t ss = sx;
      int id = bs;
      while (ss) {
        const int b = __ffs(ss) - 1;
        ss &= ss - 1;
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
        a.rec[base + id++].f1 = 32 * w + b;
      }
      // area, level and energy sums of each segment of set bits in the word
      const uint4 *qv = reinterpret_cast<const uint4 *>(img0 + t * F + 32 * w);
      reinterpret_cast<uint4 *>(myq)[0] = __ldg(qv);
      reinterpret_cast<uint4 *>(myq)[1] = __ldg(qv + 1);   // read back by this lane only
      uint32_t mm = x;
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
        rise_box *rc = &a.rec[base + bs + __popc(sx & mask_upto(b0)) - 1];
        atomicAdd(reinterpret_cast<unsigned long long *>(&rc->area), (unsigned long long)len);
        atomicAdd(reinterpret_cast<unsigned long long *>(&rc->sum_q), (unsigned long long)sq);
        atomicAdd(reinterpret_cast<unsigned long long *>(&rc->energy_fx), se);
        mm &= (len + b0 >= 32) ? 0u : ~0u << (b0 + len);
      }
    }
    // union with the runs of the next row that share a column
    const uint32_t ov = x & y;
    if (ov) {
      uint32_t os = ov & ~((ov << 1) | ((px & py) >> 31));
      while (os) {
        const int c = __ffs(os) - 1;
        os &= os - 1;
        const int ia = (int)(base + bs + __popc(sx & mask_upto(c)) - 1);
        const int ib = (int)(base2 + by + __popc(sy & mask_upto(c)) - 1);
        // a lower run touched by one upper run (the common case) hangs under
        // it with one CAS: ib is still a root and ia < ib, so this is a union.
        // A failed CAS means ib already hangs elsewhere (it touches a second
        // upper run): that union is deferred until the chains built here are
        // flattened, so this pass walks no chains.
        if (atomicCAS(&a.run_parent[ib], ib, ia) != ib) {
          const unsigned long long k = atomicAdd(reinterpret_cast<unsigned long long *>(&st->n_merge), 1ull);
          if ((int64_t)k < a.run_cap) a.merge[k] = make_int2(ia, ib);
          else uf_union(a.run_parent, ia, ib, st);   // list full: unite now (slower)
        }
      }
    }
    nst += tot_s;
    nen += tot_e;
    nsy += tot_y;
    cx = __shfl_sync(0xffffffffu, x, 31);
    cy = __shfl_sync(0xffffffffu, y, 31);
  }
}

__global__ void __launch_bounds__(32 * ROW_WARPS, 4)
runs_row_kernel(CclArgs a) {
  __shared__ unsigned long long Es[256];
  __shared__ __align__(16) uint8_t qs[ROW_WARPS][32][32];   // each lane's 32 levels
  for (int i = threadIdx.x; i < 256; i += blockDim.x) Es[i] = a.energy[i];
  __syncthreads();
  if (a.status->n_runs > a.run_cap) return;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int64_t t = (int64_t)blockIdx.x * ROW_WARPS + wib;
  if (t >= a.T) return;
  if (a.row_cnt[t] == 0) return;   // no runs in this row: nothing to label or unite
  runs_row_body(a, Es, qs[wib][lane], t, t, a.T, a.F, a.mask, a.img);
}

// Batch: rows of all captures, concatenated (a.T = total rows); row0[c] is
// the first row of capture c (ncap + 1 entries).  Rows of different
// captures are never united: has_next stops at the capture's last row.
__global__ void __launch_bounds__(32 * ROW_WARPS, 4)
runs_row_batch_kernel(CclArgs a, const RowSeg *segs, const int64_t *row0, int ncap) {
  __shared__ unsigned long long Es[256];
  __shared__ __align__(16) uint8_t qs[ROW_WARPS][32][32];
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
  runs_row_body(a, Es, qs[wib][lane], tg, tg - __ldg(&row0[lo]), rs.T, rs.F, rs.mask, rs.img);
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
  const int64_t r = a.row_base[row0[c]];   // the capture's first run
  offs[c] = r < n ? a.run_out[r] : st->n_boxes;
}

// ---------------------------------------------------------------------------
// 3b. point every run straight at its root (the row pass leaves chains as
//     tall as the component), then apply the deferred unions on flat trees.
// ---------------------------------------------------------------------------
__global__ void ccl_flatten_kernel(CclArgs a) {
  DeviceStatus *st = a.status;
  const int64_t n = st->n_runs;
  if (n > a.run_cap) return;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    const int r = uf_find(a.run_parent, (int)g, st);
    if (r != (int)g) *(volatile int *)&a.run_parent[g] = r;   // an ancestor: still valid
  }
}

__global__ void ccl_merge_kernel(CclArgs a) {
  DeviceStatus *st = a.status;
  if (st->n_runs > a.run_cap) return;
  const int64_t m = min(st->n_merge, a.run_cap);
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < m;
       k += (int64_t)gridDim.x * blockDim.x) {
    const int2 e = a.merge[k];
    uf_union(a.run_parent, e.x, e.y, st);
  }
}

// ---------------------------------------------------------------------------
// 4. every run that is not its component's root adds its record into the
//    root's; run_sroot keeps 1 exactly for the roots.  Lanes of a warp with
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
    int r = live ? uf_find(a.run_parent, (int)g, st) : -1;
    const bool contrib = live && r != (int)g;
    if (live && contrib) a.run_sroot[g] = 0;
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
// 5. compaction of global roots (run_sroot now flags exactly them)
// ---------------------------------------------------------------------------
__global__ void ccl_compact_kernel(CclArgs a) {
  DeviceStatus *st = a.status;
  const int64_t n = st->n_runs;
  if (n > a.run_cap) return;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (!a.run_sroot[g]) continue;
    const int64_t idx = a.run_out[g];
    if (idx < a.box_cap) a.boxes[idx] = a.rec[g];
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
    const int r = uf_find(a.run_parent, (int)g, st);
    const rise_box &b = a.rec[g];
    int t, f0, f1;
    if (r != (int)g) {
      t = b.t0;
      f0 = b.f0;
      f1 = b.f1;
    } else {
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

__global__ void zero_if_over_kernel(DeviceStatus *st, int64_t run_cap) {
  if (st->n_runs > run_cap) st->n_boxes = 0;
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
  return (size_t)(max_items / SCAN_BLOCK + 2) * sizeof(int64_t);
}

cudaError_t launch_ccl_count(const CclArgs &a, int num_sms, cudaStream_t s) {
  return device_scan<uint32_t>(a.row_cnt, nullptr, a.T, a.row_base, &a.status->n_runs,
                               reinterpret_cast<int64_t *>(a.scan_tmp), s);
}

namespace {
cudaError_t label_common(const CclArgs &a, const RowSeg *segs, const int64_t *row0, int ncap,
                         int64_t *offs, int num_sms, cudaStream_t s) {
  const int g = grid_for(a.run_cap, 256, num_sms, segs ? 16 : 4);
  runs_init_kernel<<<g, 256, 0, s>>>(a);
  count_launches(1);
  const unsigned row_blocks = (unsigned)((a.T + ROW_WARPS - 1) / ROW_WARPS);
  if (segs)
    runs_row_batch_kernel<<<row_blocks, 32 * ROW_WARPS, 0, s>>>(a, segs, row0, ncap);
  else
    runs_row_kernel<<<row_blocks, 32 * ROW_WARPS, 0, s>>>(a);
  count_launches(1);
  ccl_flatten_kernel<<<g, 256, 0, s>>>(a);
  count_launches(1);
  ccl_merge_kernel<<<g, 256, 0, s>>>(a);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  ccl_reduce_kernel<<<g, 256, 0, s>>>(a);
  count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = device_scan<uint8_t>(a.run_sroot, &a.status->n_runs, a.run_cap, a.run_out,
                           &a.status->n_boxes, reinterpret_cast<int64_t *>(a.scan_tmp), s);
  if (e != cudaSuccess) return e;
  ccl_compact_kernel<<<g, 256, 0, s>>>(a);
  count_launches(1);
  zero_if_over_kernel<<<1, 1, 0, s>>>(a.status, a.run_cap);
  count_launches(1);
  if (segs) {
    ccl_offsets_kernel<<<(ncap + 1 + 255) / 256, 256, 0, s>>>(a, row0, ncap, offs);
    count_launches(1);
  }
  return cudaGetLastError();
}
}  // namespace

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

cudaError_t launch_ccl_label(const CclArgs &a, int num_sms, cudaStream_t s) {
  return label_common(a, nullptr, nullptr, 0, nullptr, num_sms, s);
}

cudaError_t launch_ccl_label_batch(const CclArgs &a, const RowSeg *segs, const int64_t *row0,
                                   int ncap, int64_t *offs, int num_sms, cudaStream_t s) {
  return label_common(a, segs, row0, ncap, offs, num_sms, s);
}

}  // namespace rise
