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
//   1. row_count: runs per row (popcount of run starts); exclusive scan ->
//      row_base[t], the number of the first run of row t.
//   2. strip: a block takes RS full-width rows, numbers their runs, unions
//      vertically overlapping runs inside the strip (in shared memory when
//      the strip has at most 4096 runs, else on the global parent array),
//      and accumulates box, area, level sum and energy into the records of
//      the strip-local roots.
//   3. merge: one warp per strip boundary unions overlapping runs of the two
//      rows that meet there, on the global parent array.
//   4. reduce: every strip-local root that is no longer a global root adds
//      its record into its global root's.
//   5. compact: global roots -> exclusive scan -> boxes in run order.
#include "common.cuh"

namespace rise {
namespace {

constexpr int CCL_THREADS = 256;
constexpr int SMEM_RUNS = 4096;
constexpr int STRIP_PX = 32768;              // pixels per strip
constexpr int STRIP_WORDS = STRIP_PX / 32;   // 1024
constexpr int SCAN_THREADS = 256, SCAN_ITEMS = 8, SCAN_BLOCK = SCAN_THREADS * SCAN_ITEMS;

int strip_rows(int F) {
  int rs = STRIP_PX / F;
  return rs < 1 ? 1 : rs;
}

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
// 1. runs per row
// ---------------------------------------------------------------------------
__global__ void row_count_kernel(const uint32_t *mask, int64_t T, int Wd, uint32_t *row_cnt,
                                 DeviceStatus *st, int max_row_runs) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= T) return;
  const uint32_t *m = mask + row * Wd;
  uint32_t carry = 0, cnt = 0;
  for (int w0 = 0; w0 < Wd; w0 += 32) {
    const int w = w0 + lane;
    const uint32_t x = w < Wd ? m[w] : 0u;
    uint32_t prev = __shfl_up_sync(0xffffffffu, x, 1);
    if (lane == 0) prev = carry;
    cnt += __popc(run_starts(x, prev));
    carry = __shfl_sync(0xffffffffu, x, 31);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) {
    row_cnt[row] = cnt;
    if ((int)cnt > max_row_runs) set_err(st, ERR_ROW_RUNS);
  }
}

// ---------------------------------------------------------------------------
// 2. strips
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CCL_THREADS)
ccl_strip_kernel(CclArgs a, int RS) {
  __shared__ uint32_t bits[STRIP_WORDS];
  __shared__ uint64_t pref[STRIP_WORDS];   // exclusive prefix: low 32 run starts, high 32 run ends
  __shared__ int parent_s[SMEM_RUNS];
  __shared__ uint64_t E[256];
  __shared__ uint64_t scratch[32];
  DeviceStatus *st = a.status;
  if (st->n_runs > a.run_cap) {
    if (threadIdx.x == 0) set_err(st, ERR_RUN_CAPACITY);
    return;
  }
  const int F = a.F, Wd = F / 32, tid = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * RS;
  const int rows = (int)(a.T - r0 < RS ? a.T - r0 : RS);
  const int nwords = rows * Wd;
  const uint32_t *src = a.mask + r0 * Wd;
  for (int i = tid; i < nwords; i += CCL_THREADS) bits[i] = src[i];
  for (int i = tid; i < 256; i += CCL_THREADS) E[i] = a.energy[i];
  __syncthreads();

  // run starts / ends per word, packed counts, block-wide exclusive scan
  const int per = (nwords + CCL_THREADS - 1) / CCL_THREADS;   // <= 4
  const int i0 = tid * per;
  uint64_t loc[4];
  uint64_t sum = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = i0 + k;
    uint64_t c = 0;
    if (k < per && i < nwords) {
      const int w = i % Wd;
      const uint32_t x = bits[i];
      const uint32_t prev = w > 0 ? bits[i - 1] : 0u, next = w < Wd - 1 ? bits[i + 1] : 0u;
      c = (uint64_t)__popc(run_starts(x, prev)) | ((uint64_t)__popc(run_ends(x, next)) << 32);
    }
    loc[k] = c;
    sum += c;
  }
  uint64_t total;
  uint64_t ex = block_exclusive_scan<uint64_t>(sum, scratch, &total);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = i0 + k;
    if (k < per && i < nwords) pref[i] = ex;
    ex += loc[k];
  }
  const int nr = (int)(total & 0xffffffffu);
  const int64_t rb0 = a.row_base[r0];
  if (rb0 + nr > a.run_cap) {   // cannot happen when n_runs <= run_cap
    if (tid == 0) set_err(st, ERR_INDEX);
    return;
  }
  const bool use_s = nr <= SMEM_RUNS;
  int *par = use_s ? parent_s : a.run_parent;
  const int off = use_s ? 0 : (int)rb0;
  for (int i = tid; i < nr; i += CCL_THREADS) par[i + off] = i + off;
  __syncthreads();

  // run geometry into the per-run records
  for (int i = tid; i < nwords; i += CCL_THREADS) {
    const int r = i / Wd, w = i % Wd;
    const uint32_t x = bits[i];
    if (!x) continue;
    const uint32_t prev = w > 0 ? bits[i - 1] : 0u, next = w < Wd - 1 ? bits[i + 1] : 0u;
    uint32_t s = run_starts(x, prev), e = run_ends(x, next);
    int id = (int)(pref[i] & 0xffffffffu);
    const int64_t t = r0 + r;
    while (s) {
      const int b = __ffs(s) - 1;
      s &= s - 1;
      rise_box *rc = &a.rec[rb0 + id];
      rc->t0 = (int32_t)t;
      rc->t1 = (int32_t)t;
      rc->f0 = 32 * w + b;
      rc->anchor = t * F + 32 * w + b;
      rc->area = 0;
      rc->sum_q = 0;
      rc->energy_fx = 0;
      ++id;
    }
    id = (int)(pref[i] >> 32);
    while (e) {
      const int b = __ffs(e) - 1;
      e &= e - 1;
      a.rec[rb0 + id].f1 = 32 * w + b;
      ++id;
    }
  }

  // unions of vertically overlapping runs inside the strip
  for (int i = tid; i < (rows - 1) * Wd; i += CCL_THREADS) {
    const int w = i % Wd;
    const uint32_t x = bits[i], y = bits[i + Wd];
    const uint32_t ov = x & y;
    if (!ov) continue;
    const uint32_t px = w > 0 ? bits[i - 1] : 0u, py = w > 0 ? bits[i - 1 + Wd] : 0u;
    uint32_t os = ov & ~((ov << 1) | ((px & py) >> 31));
    const uint32_t sx = run_starts(x, px), sy = run_starts(y, py);
    const int bx = (int)(pref[i] & 0xffffffffu), by = (int)(pref[i + Wd] & 0xffffffffu);
    while (os) {
      const int c = __ffs(os) - 1;
      os &= os - 1;
      const int la = bx + __popc(sx & mask_upto(c)) - 1;
      const int lb = by + __popc(sy & mask_upto(c)) - 1;
      uf_union(par, la + off, lb + off, st);
    }
  }
  __syncthreads();

  // flatten: every run points at its strip-local root.  A concurrent path-
  // halving store may later replace an entry by another ancestor, so roots
  // are always re-read through uf_find, never from a parent entry directly.
  for (int i = tid; i < nr; i += CCL_THREADS) {
    const int root = uf_find(par, i + off, st) - off;
    a.run_parent[rb0 + i] = (int)(rb0 + root);
    a.run_sroot[rb0 + i] = (uint8_t)(root == i);
  }
  __syncthreads();   // records initialised and unions finished before accumulating

  // box extent, area, level sum and energy into the strip-local roots
  for (int i = tid; i < nwords; i += CCL_THREADS) {
    const int r = i / Wd, w = i % Wd;
    const uint32_t x = bits[i];
    if (!x) continue;
    const uint32_t prev = w > 0 ? bits[i - 1] : 0u, next = w < Wd - 1 ? bits[i + 1] : 0u;
    const uint32_t s = run_starts(x, prev);
    const int base_s = (int)(pref[i] & 0xffffffffu);
    const int64_t t = r0 + r;
    auto root_of = [&](int id) -> int { return uf_find(par, id + off, st) - off; };
    {   // extent contributions of runs that start / end in this word
      uint32_t ss = s;
      int id = base_s;
      while (ss) {
        const int b = __ffs(ss) - 1;
        ss &= ss - 1;
        const int root = root_of(id);
        if (root != id) {
          rise_box *rc = &a.rec[rb0 + root];
          atomicMax(&rc->t1, (int32_t)t);
          atomicMin(&rc->f0, 32 * w + b);
        }
        ++id;
      }
      uint32_t ee = run_ends(x, next);
      id = (int)(pref[i] >> 32);
      while (ee) {
        const int b = __ffs(ee) - 1;
        ee &= ee - 1;
        const int root = root_of(id);
        if (root != id) atomicMax(&a.rec[rb0 + root].f1, 32 * w + b);
        ++id;
      }
    }
    // level sums over each maximal segment of set bits in this word
    const uint4 *qs = reinterpret_cast<const uint4 *>(a.img + t * F + 32 * w);
    const uint4 qa = __ldg(qs), qb = __ldg(qs + 1);
    const uint32_t qw[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
    uint32_t m = x;
    while (m) {
      const int b0 = __ffs(m) - 1;
      const uint32_t inv = ~(m >> b0);
      const int len = inv ? __ffs(inv) - 1 : 32 - b0;
      uint64_t sq = 0, se = 0;
      for (int b = b0; b < b0 + len; ++b) {
        const uint32_t q = (qw[b >> 2] >> (8 * (b & 3))) & 0xffu;
        sq += q;
        se += E[q];
      }
      const int id = base_s + __popc(s & mask_upto(b0)) - 1;
      const int root = root_of(id);
      rise_box *rc = &a.rec[rb0 + root];
      atomicAdd(reinterpret_cast<unsigned long long *>(&rc->area), (unsigned long long)len);
      atomicAdd(reinterpret_cast<unsigned long long *>(&rc->sum_q), (unsigned long long)sq);
      atomicAdd(reinterpret_cast<unsigned long long *>(&rc->energy_fx), (unsigned long long)se);
      m &= (len + b0 >= 32) ? 0u : ~0u << (b0 + len);
    }
  }
}

// ---------------------------------------------------------------------------
// 3. strip boundaries
// ---------------------------------------------------------------------------
__global__ void ccl_merge_kernel(CclArgs a, int RS, int64_t n_bound) {
  const int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  DeviceStatus *st = a.status;
  if (b >= n_bound || st->n_runs > a.run_cap) return;
  const int Wd = a.F / 32;
  const int64_t t = (b + 1) * RS - 1;
  if (t + 1 >= a.T) return;
  const uint32_t *ra = a.mask + t * Wd, *rb = a.mask + (t + 1) * Wd;
  const int64_t base_a = a.row_base[t], base_b = a.row_base[t + 1];
  uint32_t cx = 0, cy = 0;       // previous words (carried across chunks)
  int64_t na = 0, nb = 0;        // runs started in earlier words
  for (int w0 = 0; w0 < Wd; w0 += 32) {
    const int w = w0 + lane;
    const uint32_t x = w < Wd ? ra[w] : 0u, y = w < Wd ? rb[w] : 0u;
    uint32_t px = __shfl_up_sync(0xffffffffu, x, 1), py = __shfl_up_sync(0xffffffffu, y, 1);
    if (lane == 0) { px = cx; py = cy; }
    const uint32_t sx = run_starts(x, px), sy = run_starts(y, py);
    int ex = __popc(sx), ey = __popc(sy);
    int ix = ex, iy = ey;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int u = __shfl_up_sync(0xffffffffu, ix, o), v = __shfl_up_sync(0xffffffffu, iy, o);
      if (lane >= o) { ix += u; iy += v; }
    }
    const int64_t bx = base_a + na + (ix - ex), by = base_b + nb + (iy - ey);
    const uint32_t ov = x & y;
    uint32_t os = ov & ~((ov << 1) | ((px & py) >> 31));
    while (os) {
      const int c = __ffs(os) - 1;
      os &= os - 1;
      const int64_t ia = bx + __popc(sx & mask_upto(c)) - 1;
      const int64_t ib = by + __popc(sy & mask_upto(c)) - 1;
      uf_union(a.run_parent, (int)ia, (int)ib, st);
    }
    na += __shfl_sync(0xffffffffu, ix, 31);
    nb += __shfl_sync(0xffffffffu, iy, 31);
    cx = __shfl_sync(0xffffffffu, x, 31);
    cy = __shfl_sync(0xffffffffu, y, 31);
  }
}

// ---------------------------------------------------------------------------
// 4. strip-local roots into global roots; marks global roots in run_sroot
// ---------------------------------------------------------------------------
__global__ void ccl_reduce_kernel(CclArgs a) {
  DeviceStatus *st = a.status;
  const int64_t n = st->n_runs;
  if (n > a.run_cap) return;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < n;
       g += (int64_t)gridDim.x * blockDim.x) {
    if (!a.run_sroot[g]) continue;
    const int r = uf_find(a.run_parent, (int)g, st);
    if (r == (int)g) continue;
    a.run_sroot[g] = 0;   // no longer a root; only this thread touches entry g
    const rise_box src = a.rec[g];
    rise_box *dst = &a.rec[r];
    atomicMax(&dst->t1, src.t1);
    atomicMin(&dst->f0, src.f0);
    atomicMax(&dst->f1, src.f1);
    atomicAdd(reinterpret_cast<unsigned long long *>(&dst->area), (unsigned long long)src.area);
    atomicAdd(reinterpret_cast<unsigned long long *>(&dst->sum_q), (unsigned long long)src.sum_q);
    atomicAdd(reinterpret_cast<unsigned long long *>(&dst->energy_fx),
              (unsigned long long)src.energy_fx);
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

__global__ void zero_if_over_kernel(DeviceStatus *st, int64_t run_cap) {
  if (st->n_runs > run_cap) st->n_boxes = 0;
}

int grid_for(int64_t n, int threads, int num_sms) {
  int64_t g = (n + threads - 1) / threads;
  g = std::min<int64_t>(g, (int64_t)num_sms * 16);
  return (int)std::max<int64_t>(1, g);
}

}  // namespace

size_t ccl_scan_tmp_bytes(int64_t max_items) {
  return (size_t)(max_items / SCAN_BLOCK + 2) * sizeof(int64_t);
}

cudaError_t launch_ccl_count(const CclArgs &a, int num_sms, cudaStream_t s) {
  const int Wd = a.F / 32;
  const int64_t warps = a.T;
  row_count_kernel<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, s>>>(a.mask, a.T, Wd, a.row_cnt,
                                                                        a.status, a.F / 4 + 1);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = device_scan<uint32_t>(a.row_cnt, nullptr, a.T, a.row_base, &a.status->n_runs,
                            reinterpret_cast<int64_t *>(a.scan_tmp), s);
  return e;
}

cudaError_t launch_ccl_label(const CclArgs &a, int num_sms, cudaStream_t s) {
  const int RS = strip_rows(a.F);
  const int64_t n_strips = (a.T + RS - 1) / RS;
  ccl_strip_kernel<<<(unsigned)n_strips, CCL_THREADS, 0, s>>>(a, RS);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t n_bound = n_strips - 1;
  if (n_bound > 0) {
    ccl_merge_kernel<<<(unsigned)((n_bound * 32 + 255) / 256), 256, 0, s>>>(a, RS, n_bound);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const int g = grid_for(a.run_cap, 256, num_sms);
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
  return cudaGetLastError();
}

}  // namespace rise
