// Image stages of RISE (Sec. IV-B): column histograms of the 8-bit TF plot,
// the PSD (column sums) with Savitzky-Golay smoothing and the lowest local
// minimum N0, theta_PSD column pruning, exact per-column Otsu (Eq. 4) with
// the power floor, and the binary mask with one 2D closing, one 2D opening
// and one horizontal 1D opening (Eq. 5) on bit-packed tiles.
#include <cooperative_groups.h>

#include <algorithm>
#include <map>
#include <mutex>

#include <type_traits>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace rise {
namespace {

constexpr int HIST_MAX_ROWS = 65535;   // rows per band: 32-bit offsets inside a band suffice

// Level of a stored float |X|^2 (same rule as the STFT epilogue).
constexpr float kGuardQ = 3.0e-4f;   // the fast level coordinate is off by < 1e-4
__device__ __forceinline__ uint32_t level_of_q(float P, float inv_anchor, float c1,
                                               const float *edges) {
  const float v = fmaf(__log2f(P * inv_anchor), c1, 255.5f);
  uint32_t q = __float2uint_rd(fminf(v, 255.0f));   // floor, clamped to 0..255 (NaN, -inf: 0)
  if (fabsf(v - rintf(v)) < kGuardQ) {              // near a level edge: exact comparison
    int qi = (int)q;
    for (int it = 0; it < 256 && qi < 255 && P >= edges[qi + 1]; ++it) ++qi;
    for (int it = 0; it < 256 && qi > 0 && P < edges[qi]; ++it) --qi;
    q = (uint32_t)qi;
  }
  return q;
}

// ---------------------------------------------------------------------------
// Per-column Otsu (Eq. 4): one warp per column.  Lane l owns levels
// 8l..8l+7.  For a split theta (class 0 = levels <= theta) with n0, s0 the
// count and level sum of class 0 and n, s the column totals, sigma_b^2 is
// proportional to d^2 / (n0 n1) with d = s0 n - s n0; candidates are compared
// exactly by cross-multiplication in 128-bit integers and the smallest
// maximiser wins.  Also returns the column PSD S = s.
// ---------------------------------------------------------------------------
struct Cand {
  unsigned __int128 num;
  uint64_t den;
  int th;
};

__device__ __forceinline__ bool better(const Cand &a, const Cand &b) {
  // is a strictly better than b, or equally good with a smaller theta?
  if (a.th < 0) return false;
  if (b.th < 0) return true;
  const unsigned __int128 l = a.num * b.den, r = b.num * a.den;
  if (l != r) return l > r;
  return a.th < b.th;
}

__device__ __forceinline__ unsigned __int128 shfl_u128(unsigned __int128 x, int src) {
  uint64_t lo = (uint64_t)x, hi = (uint64_t)(x >> 64);
  lo = __shfl_sync(0xffffffffu, lo, src);
  hi = __shfl_sync(0xffffffffu, hi, src);
  return ((unsigned __int128)hi << 64) | lo;
}

// h: the column's 256 counts (lane reads h[8 lane .. 8 lane + 7]); all lanes
// return the same (S, theta).
__device__ __forceinline__ void otsu_warp(const uint32_t *h8, int lane, uint64_t *S, int *theta) {
  uint32_t h[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] = h8[i];
  uint64_t n_l = 0, s_l = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    n_l += h[i];
    s_l += (uint64_t)(8 * lane + i) * h[i];
  }
  uint64_t n_inc = n_l, s_inc = s_l;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint64_t a1 = __shfl_up_sync(0xffffffffu, n_inc, o), b1 = __shfl_up_sync(0xffffffffu, s_inc, o);
    if (lane >= o) { n_inc += a1; s_inc += b1; }
  }
  const uint64_t n = __shfl_sync(0xffffffffu, n_inc, 31), s = __shfl_sync(0xffffffffu, s_inc, 31);
  uint64_t n0 = n_inc - n_l, s0 = s_inc - s_l;
  Cand best{0, 1, -1};
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int th = 8 * lane + i;
    n0 += h[i];
    s0 += (uint64_t)th * h[i];
    if (th < 255 && n0 > 0 && n0 < n) {
      const __int128 d = (__int128)s0 * (__int128)n - (__int128)s * (__int128)n0;
      const unsigned __int128 ad = (unsigned __int128)(d < 0 ? -d : d);
      Cand c{ad * ad, n0 * (n - n0), th};
      if (better(c, best)) best = c;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Cand o_c;
    o_c.num = shfl_u128(best.num, lane ^ o);
    o_c.den = __shfl_sync(0xffffffffu, best.den, lane ^ o);
    o_c.th = __shfl_sync(0xffffffffu, best.th, lane ^ o);
    if (better(o_c, best)) best = o_c;
  }
  *S = s;
  *theta = best.th;
}

// Otsu of every column from the global histogram (used when the histogram
// needed more than one cluster of row bands).
__global__ void otsu_kernel(ColArgs a) {
  const int warp_g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp_g >= a.F) return;
  uint64_t S;
  int th;
  otsu_warp(a.hist + (size_t)warp_g * 256 + 8 * lane, lane, &S, &th);
  if (lane == 0) {
    a.cols[warp_g].S = S;
    a.cols[warp_g].otsu = th;
  }
}

// ---------------------------------------------------------------------------
// Column histogram, cluster version.  A block owns 64 columns of one row
// band; its 8 warps take interleaved rows.  Lane l reads 2 consecutive
// columns (2l, 2l+1) per row and counts column 2l+j in shared slot l+32j:
// 16-bit counters (a band holds at most 65535 rows), the two of lane l in
// one 32-bit word, level-major, so a warp's 32 lanes hit 32 banks, bumped
// with shared-memory reductions whose results are unused (32 KB of counters
// per block: three blocks fit an SM by registers).  The main loop takes
// whole groups of CH_UNROLL rows per warp with no bounds checks and issues
// the next group's loads before counting the current one; a tail loop takes
// the remaining rows.  Offsets inside a band are 32-bit (a band holds
// at most 65535 rows of at most 8192 columns).  The 8 blocks of a
// thread-block cluster cover the same 64 columns over 8 row bands; after
// counting, each block sums whole columns (8 of them) over the cluster
// through distributed shared memory, stores their histograms (plain stores:
// no zeroing, no global atomics) and runs Otsu on them, one warp per column.
// FROM_POWER: the input is float |X|^2, quantised here (same level rule as
// the STFT epilogue) and the 8-bit image is written alongside.
// ---------------------------------------------------------------------------
constexpr int CH_WARPS = 8, CH_COLS = 64, CH_BANDS = 8, CH_UNROLL = 8;
constexpr int CH_PX = CH_COLS / 32;                   // columns per lane
constexpr int CH_WORDS = 256 * CH_COLS / 2;          // 32-bit words of 16-bit counters per block
constexpr size_t ch_smem() { return (size_t)CH_WORDS * sizeof(uint32_t); }
constexpr int CH_NS = CH_COLS / CH_BANDS;            // columns each block reduces

__device__ __forceinline__ uint32_t shared_addr(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// one count into the shared counter word at byte address `addr`: inc is 1
// for the low 16-bit counter, 1 << 16 for the high one
__device__ __forceinline__ void ch_red(uint32_t addr, uint32_t inc) {
  asm volatile("red.shared::cta.add.u32 [%0], %1;" ::"r"(addr), "r"(inc));
}

// Column group cgx, row band `band` of one image (the bands of a column group
// form one cluster; the launch picks how many).
template <bool FROM_POWER>
__device__ __forceinline__ void cluster_hist_body(const HistArgs &a, int cgx, int band) {
  extern __shared__ uint4 sh4[];     // [256 levels][32 lanes] u32 = two u16 column counters
  uint32_t *sh = reinterpret_cast<uint32_t *>(sh4);
  __shared__ float edges[257];
  __shared__ __align__(16) uint32_t hs[CH_NS][256];   // reduced columns
  cg::cluster_group cluster = cg::this_cluster();
  const int64_t T = a.T;
  const int F = a.F;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < CH_WORDS / 4; i += blockDim.x) sh4[i] = make_uint4(0u, 0u, 0u, 0u);
  float inv_anchor = 0.f, c1 = 0.f;
  if constexpr (FROM_POWER) {
    if (a.max_bits) {
      // level j >= 1 is reached at M 10^((j - 255.5) level_db / 10): the
      // smallest float not below M ratio[j] (ratio in FP64)
      const double M = (double)__uint_as_float(*a.max_bits);
      const bool first = blockIdx.x == 0 && blockIdx.y == 0;
      for (int i = tid; i < 257; i += blockDim.x) {
        float e;
        if (i == 0) e = 0.0f;
        else if (i == 256 || !(M > 0.0)) e = __int_as_float(0x7f800000);
        else e = __double2float_ru(M * a.ratio[i]);
        edges[i] = e;
        if (first && a.edges_out) a.edges_out[i] = e;
      }
      inv_anchor = M > 0.0 ? (float)(1.0 / M) : 0.0f;
      c1 = (float)(3.0102999566398119521 / a.level_db);   // 10 log10(2) / level_db
      if (first && tid == 0 && a.qconst_out) {
        a.qconst_out[0] = inv_anchor;
        a.qconst_out[1] = c1;
      }
    } else {
      for (int i = tid; i < 257; i += blockDim.x) edges[i] = a.edges[i];
      inv_anchor = a.qconst[0];
      c1 = a.qconst[1];
    }
  }
  __syncthreads();
  const int c0 = cgx * CH_COLS + CH_PX * lane;
  const int64_t r0 = (int64_t)band * a.rows_per_band;
  const int64_t r1 = min(T, r0 + a.rows_per_band);
  const int K = (r1 - r0 > warp) ? (int)((r1 - r0 - warp + CH_WARPS - 1) / CH_WARPS) : 0;
  const uint32_t rstep = (uint32_t)CH_WARPS * (uint32_t)F;   // elements between a warp's rows
  const uint32_t cbase = shared_addr(sh) + 4u * lane;        // slots lane (low half), lane+32 (high)
  uint32_t off = (uint32_t)warp * (uint32_t)F;               // this warp's row, from the band start
  if constexpr (FROM_POWER) {
    const float *pb = reinterpret_cast<const float *>(a.src) + r0 * F + c0;
    uint8_t *ob = a.img + r0 * F + c0;
    // levels of one row pair of values, the image bytes and the counts
    auto one_row = [&](float2 x, uint32_t o) {
      float pv[2] = {x.x, x.y};
      uint32_t q[2];
      bool near = false;
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const float v = fmaf(__log2f(pv[j] * inv_anchor), c1, 255.5f);
        q[j] = min(__float2uint_rd(v), 255u);   // -inf, NaN: 0
        near |= fabsf(v - rintf(v)) < kGuardQ;
      }
      if (near) {
#pragma unroll
        for (int j = 0; j < 2; ++j) q[j] = level_of_q(pv[j], inv_anchor, c1, edges);
      }
      *reinterpret_cast<uint16_t *>(ob + o) = (uint16_t)(q[0] | (q[1] << 8));
      ch_red(cbase + (q[0] << 7), 1u);
      ch_red(cbase + (q[1] << 7), 1u << 16);
    };
    const int KF = K / CH_UNROLL * CH_UNROLL;
    float2 A[CH_UNROLL], B[CH_UNROLL];
    auto load = [&](float2 (&X)[CH_UNROLL], uint32_t o) {
#pragma unroll
      for (int u = 0; u < CH_UNROLL; ++u) X[u] = __ldg(reinterpret_cast<const float2 *>(pb + o + u * rstep));
    };
    auto count = [&](const float2 (&X)[CH_UNROLL], uint32_t o) {
#pragma unroll
      for (int u = 0; u < CH_UNROLL; ++u) one_row(X[u], o + u * rstep);
    };
    const uint32_t gstep = CH_UNROLL * rstep;
    int k = 0;
    if (KF > 0) load(A, off);
    while (k < KF) {
      if (k + CH_UNROLL < KF) load(B, off + gstep);
      count(A, off);
      k += CH_UNROLL;
      off += gstep;
      if (k >= KF) break;
      if (k + CH_UNROLL < KF) load(A, off + gstep);
      count(B, off);
      k += CH_UNROLL;
      off += gstep;
    }
    for (; k < K; ++k, off += rstep) one_row(__ldg(reinterpret_cast<const float2 *>(pb + off)), off);
  } else {
    const uint8_t *pb = reinterpret_cast<const uint8_t *>(a.src) + r0 * F + c0;
    auto one_row = [&](uint32_t w) {
      ch_red(cbase + ((w & 0xffu) << 7), 1u);
      ch_red(cbase + ((w >> 8) << 7), 1u << 16);
    };
    constexpr int U2 = 2 * CH_UNROLL;
    const int KF2 = K / U2 * U2;
    int k = 0;
    for (; k < KF2; k += U2, off += U2 * rstep) {
      uint32_t w[U2];
#pragma unroll
      for (int u = 0; u < U2; ++u) w[u] = __ldg(reinterpret_cast<const uint16_t *>(pb + off + u * rstep));
#pragma unroll
      for (int u = 0; u < U2; ++u) one_row(w[u]);
    }
    for (; k < K; ++k, off += rstep) one_row(__ldg(reinterpret_cast<const uint16_t *>(pb + off)));
  }
  cluster.sync();
  // this block's share of the 64 column slots, summed over the cluster's
  // bands in chunks of 8 columns, then one warp per column: store its
  // histogram, then PSD and Otsu threshold
  const int rank = (int)cluster.block_rank(), nb = (int)cluster.num_blocks();
  const int s_lo = rank * CH_COLS / nb, s_hi = (rank + 1) * CH_COLS / nb;
  for (int cs = s_lo; cs < s_hi; cs += CH_NS) {
    const int nc = min(CH_NS, s_hi - cs);
    for (int k = tid; k < nc * 256; k += blockDim.x) {
      const int sl = k % nc, v = k / nc;
      const int slot = cs + sl, i = v * 32 + (slot & 31), sh16 = 16 * (slot >> 5);
      uint32_t n = 0;
      for (int b = 0; b < nb; ++b) n += (cluster.map_shared_rank(sh, b)[i] >> sh16) & 0xffffu;
      hs[sl][v] = n;
    }
    __syncthreads();
    if (warp < nc) {
      const int sl = warp;
      const int slot = cs + sl;
      const int col = cgx * CH_COLS + CH_PX * (slot & 31) + (slot >> 5);
      uint32_t *dst = a.hist + (size_t)col * 256;
      if (a.accumulate) {
        for (int v = lane; v < 256; v += 32)
          if (hs[sl][v]) atomicAdd(&dst[v], hs[sl][v]);
      } else {
        for (int v = lane; v < 256; v += 32) dst[v] = hs[sl][v];
        uint64_t S;
        int th;
        otsu_warp(&hs[sl][8 * lane], lane, &S, &th);
        if (lane == 0) {
          a.cols[col].S = S;
          a.cols[col].otsu = th;
        }
      }
    }
    __syncthreads();   // hs is refilled by the next chunk
  }
  cluster.sync();   // remote reads finished before any block leaves
}

template <bool FROM_POWER>
__global__ void __launch_bounds__(32 * CH_WARPS, 3) cluster_hist_kernel(HistArgs a) {
  cluster_hist_body<FROM_POWER>(a, blockIdx.x, blockIdx.y);
}

// Batch: blockIdx.x indexes (capture, column group) items; the arguments of
// the item's capture are copied to shared memory first.
template <bool FROM_POWER>
__global__ void __launch_bounds__(32 * CH_WARPS, 3)
cluster_hist_batch_kernel(const HistArgs *segs, const HistItem *items) {
  __shared__ HistArgs sa;
  const HistItem it = items[blockIdx.x];
  if (threadIdx.x == 0) sa = segs[it.seg];
  __syncthreads();
  if (kChecked && (it.cg < 0 || it.cg >= sa.F / 64)) return;   // checked build: a column group of the capture
  cluster_hist_body<FROM_POWER>(sa, it.cg, blockIdx.y);
}

// ---------------------------------------------------------------------------
// Noise floor and per-column thresholds: one block of 1024 threads.
// ---------------------------------------------------------------------------
constexpr int FLOOR_THREADS = 1024;

__device__ __forceinline__ int64_t floor_div_d(int64_t a, int64_t b) {
  int64_t q = a / b;
  if ((a % b != 0) && (a < 0)) q -= 1;
  return q;
}

__device__ __forceinline__ void floor_body(const ColArgs &a) {
  // [F] D-scaled smoothing (int64), then [F] column PSD and [F] Otsu
  // thresholds (int32 each): S_f <= 255 T < 2^31 and |c_i| < 2^12, so each
  // tap is one 32 x 32 -> 64-bit product
  extern __shared__ int64_t Sh[];
  int32_t *S = reinterpret_cast<int32_t *>(Sh + a.F);
  int32_t *TH = S + a.F;
  __shared__ int64_t red_min[32], red_g[32];
  __shared__ int red_found[32];
  __shared__ int32_t c[64];
  __shared__ int64_t s_N0, s_Pq;
  const int F = a.F, m = a.m, tid = threadIdx.x;
  for (int i = tid; i <= m; i += blockDim.x) c[i] = (int32_t)a.sg_c[i];
  // one pass over the column records (the loads of a thread are independent)
#pragma unroll 4
  for (int f = tid; f < F; f += blockDim.x) {
    const rise_colstat cs = a.cols[f];
    S[f] = (int32_t)cs.S;
    TH[f] = cs.otsu;
  }
  __syncthreads();
  // Savitzky-Golay (D-scaled) on the interior, 0 elsewhere
#pragma unroll 4
  for (int f = tid; f < F; f += blockDim.x) {
    int64_t acc = 0;
    if (f >= m && f <= F - 1 - m) {
      acc = (int64_t)c[0] * S[f];
      for (int i = 1; i <= m; ++i) acc += (int64_t)c[i] * (int64_t)(S[f - i] + S[f + i]);
    }
    Sh[f] = acc;
    a.cols[f].Shat = acc;
  }
  __syncthreads();
  // lowest local minimum: strictly below the left neighbour, not above the right
  int64_t best = INT64_MAX, gmin = INT64_MAX;
  int found = 0;
  for (int f = m + tid; f <= F - 1 - m; f += blockDim.x) {
    const int64_t v = Sh[f];
    gmin = min(gmin, v);
    if (f >= m + 1 && f <= F - 2 - m && v < Sh[f - 1] && v <= Sh[f + 1]) {
      found = 1;
      best = min(best, v);
    }
  }
  const int lane = tid & 31, w = tid >> 5, nw = (int)(blockDim.x >> 5);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
    gmin = min(gmin, __shfl_xor_sync(0xffffffffu, gmin, o));
    found |= __shfl_xor_sync(0xffffffffu, found, o);
  }
  if (lane == 0) { red_min[w] = best; red_g[w] = gmin; red_found[w] = found; }
  __syncthreads();
  if (w == 0) {   // the warps' results, reduced by one warp
    int64_t bb = lane < nw ? red_min[lane] : INT64_MAX;
    int64_t gg = lane < nw ? red_g[lane] : INT64_MAX;
    int ff = lane < nw ? red_found[lane] : 0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      bb = min(bb, __shfl_xor_sync(0xffffffffu, bb, o));
      gg = min(gg, __shfl_xor_sync(0xffffffffu, gg, o));
      ff |= __shfl_xor_sync(0xffffffffu, ff, o);
    }
    if (lane == 0) {
      const int64_t N0 = ff ? bb : gg;
      const int64_t DT = a.D * a.T;
      int64_t Pq = 0;
      if (a.pow_on) {
        Pq = -floor_div_d(-(N0 + a.delta_pow), DT);   // ceil((N0 + delta_pow) / DT)
        Pq = Pq < 0 ? 0 : (Pq > 256 ? 256 : Pq);
      }
      s_N0 = N0;
      s_Pq = Pq;
      int64_t *fo = a.floor_out;
      fo[0] = N0; fo[1] = a.delta_psd; fo[2] = a.delta_pow; fo[3] = Pq;
      fo[4] = a.D; fo[5] = a.T; fo[6] = F; fo[7] = 0;
    }
  }
  __syncthreads();
  const int64_t N0 = s_N0, Pq = s_Pq;
#pragma unroll 4
  for (int f = tid; f < F; f += blockDim.x) {
    const int keep = a.psd_on ? (a.D * (int64_t)S[f] >= N0 + a.delta_psd) : 1;
    const int th = TH[f];
    int eff = 256;
    if (keep && th >= 0) eff = max(th + 1, (int)Pq);
    a.cols[f].keep = keep;
    a.cols[f].eff = eff;
    a.cols[f].pad = 0;
    a.effm1[f] = (uint8_t)min(255, max(0, eff - 1));
  }
}

// One image, column-parallel: the same floor in two launches of F/256
// blocks.  Keys map int64 order to reversed uint64 order, so that an
// atomicMax over keys is a minimum over values and the zeroed word is empty.
__device__ __forceinline__ unsigned long long min_key(int64_t v) {
  return ~((unsigned long long)v ^ 0x8000000000000000ull);
}
__device__ __forceinline__ int64_t key_value(unsigned long long k) {
  return (int64_t)(~k ^ 0x8000000000000000ull);
}
constexpr int FP_COLS = 256;

// Part 1: each block smooths its columns (with the neighbours it needs) and
// offers its lowest local minimum and lowest smoothed value.
__global__ void __launch_bounds__(FP_COLS) floor_part_kernel(ColArgs a) {
  __shared__ int32_t S[FP_COLS + 2 * 64];
  __shared__ int64_t Sh[FP_COLS + 2];
  __shared__ int32_t c[64];
  __shared__ unsigned long long r_best[FP_COLS / 32], r_gmin[FP_COLS / 32];
  __shared__ int r_found[FP_COLS / 32];
  const int F = a.F, m = a.m, tid = threadIdx.x;
  const int f0 = blockIdx.x * FP_COLS;
  const int lo = f0 - 1 - m;                // S[j] holds column lo + j
  for (int i = tid; i <= m; i += blockDim.x) c[i] = (int32_t)a.sg_c[i];
  for (int j = tid; j < FP_COLS + 2 + 2 * m; j += blockDim.x) {
    const int f = lo + j;
    S[j] = (f >= 0 && f < F) ? (int32_t)a.cols[f].S : 0;
  }
  __syncthreads();
  // Sh[1 + i] = smoothed column f0 + i, for i = -1 .. FP_COLS (0 off the interior)
  for (int i = tid - 1; i <= FP_COLS; i += blockDim.x) {
    const int f = f0 + i;
    int64_t acc = 0;
    if (f >= m && f <= F - 1 - m) {
      const int j = f - lo;
      acc = (int64_t)c[0] * S[j];
      for (int t = 1; t <= m; ++t) acc += (int64_t)c[t] * (int64_t)(S[j - t] + S[j + t]);
    }
    Sh[1 + i] = acc;
    if (i >= 0 && i < FP_COLS && f < F) a.cols[f].Shat = acc;
  }
  __syncthreads();
  const int f = f0 + tid;
  unsigned long long best = 0, gmin = 0;
  int found = 0;
  if (f >= m && f <= F - 1 - m) {
    const int64_t v = Sh[1 + tid];
    gmin = min_key(v);
    if (f >= m + 1 && f <= F - 2 - m && v < Sh[tid] && v <= Sh[2 + tid]) {
      found = 1;
      best = min_key(v);
    }
  }
  const int lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
    gmin = max(gmin, __shfl_xor_sync(0xffffffffu, gmin, o));
    found |= __shfl_xor_sync(0xffffffffu, found, o);
  }
  if (lane == 0) { r_best[w] = best; r_gmin[w] = gmin; r_found[w] = found; }
  __syncthreads();
  if (tid == 0) {
    for (int k = 1; k < FP_COLS / 32; ++k) {
      best = max(best, r_best[k]);
      gmin = max(gmin, r_gmin[k]);
      found |= r_found[k];
    }
    if (best) atomicMax(&a.st->floor_best, best);
    if (gmin) atomicMax(&a.st->floor_gmin, gmin);
    if (found) atomicOr(&a.st->floor_found, 1u);
  }
}

// Part 2: N0, P_q and every column's keep / eff (one thread per column).
__global__ void __launch_bounds__(FP_COLS) floor_eff_kernel(ColArgs a) {
  const DeviceStatus *st = a.st;
  const int64_t N0 = key_value(st->floor_found ? st->floor_best : st->floor_gmin);
  const int64_t DT = a.D * a.T;
  int64_t Pq = 0;
  if (a.pow_on) {
    Pq = -floor_div_d(-(N0 + a.delta_pow), DT);   // ceil((N0 + delta_pow) / DT)
    Pq = Pq < 0 ? 0 : (Pq > 256 ? 256 : Pq);
  }
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f == 0) {
    int64_t *fo = a.floor_out;
    fo[0] = N0; fo[1] = a.delta_psd; fo[2] = a.delta_pow; fo[3] = Pq;
    fo[4] = a.D; fo[5] = a.T; fo[6] = a.F; fo[7] = 0;
  }
  if (f >= a.F) return;
  const rise_colstat cs = a.cols[f];
  const int keep = a.psd_on ? (a.D * (int64_t)(int32_t)cs.S >= N0 + a.delta_psd) : 1;
  int eff = 256;
  if (keep && cs.otsu >= 0) eff = max(cs.otsu + 1, (int)Pq);
  a.cols[f].keep = keep;
  a.cols[f].eff = eff;
  a.cols[f].pad = 0;
  a.effm1[f] = (uint8_t)min(255, max(0, eff - 1));
}

// Batch: one block per capture.
__global__ void __launch_bounds__(FLOOR_THREADS) floor_batch_kernel(const ColArgs *segs) {
  __shared__ ColArgs sa;
  if (threadIdx.x == 0) sa = segs[blockIdx.x];
  __syncthreads();
  floor_body(sa);
}

// ---------------------------------------------------------------------------
// Threshold + morphology, streaming.  A warp owns a window of 32 row words
// (1024 columns) of a band of rows; lane l holds word w0-1+l, and only lanes
// 1..30 produce output (lanes 0 and 31 are halo: each of the six operations
// moves information by at most one column, so corruption entering at a
// window edge never reaches the 31st bit inward).  The warp walks down the
// band one input row per step; the six operations form a register pipeline:
// an operation keeps the horizontally processed last two rows of its input
// and emits one row per step (a 3x3 operation lags its input by one row), so
// the final row of step s is input row s-4.  Neighbour words come from the
// adjacent lanes by shuffle.  The band is read with a 4-row halo above and
// below; rows are prefetched 4 steps ahead.  A pixel outside the image takes
// no part in an operation: the operation sees 0 there for a dilation and 1
// for an erosion (the clipped window).  The kernel also counts the runs
// (maximal horizontal segments) starting in each row of the final mask.
// ---------------------------------------------------------------------------
constexpr int MS_LANES_OUT = 30, MS_PF = 4, MS_WARPS = 8;

template <bool ERODE, bool VERT>
struct MorphOp {
  uint32_t a = 0, b = 0;   // horizontal results of the two previous input rows
  // x: this step's input row (already this lane's word); in: row and lane inside the image
  __device__ __forceinline__ uint32_t step(uint32_t x, bool in) {
    if (!in) x = ERODE ? 0xffffffffu : 0u;
    const uint32_t l = __shfl_up_sync(0xffffffffu, x, 1);
    const uint32_t r = __shfl_down_sync(0xffffffffu, x, 1);
    const uint32_t xl = __funnelshift_l(l, x, 1);   // (x << 1) | (l >> 31): pixel f-1 moved to f
    const uint32_t xr = __funnelshift_r(x, r, 1);   // (x >> 1) | (r << 31): pixel f+1 moved to f
    const uint32_t h = ERODE ? (x & xl & xr) : (x | xl | xr);
    if constexpr (!VERT) return h;
    const uint32_t o = ERODE ? (a & b & h) : (a | b | h);   // output row = input row - 1
    a = b;
    b = h;
    return o;
  }
};

// Threshold of 4 pixels: the levels q (4 bytes) against the columns' eff-1
// (4 bytes); bit j of the result = [q_j > e_j] (unsigned bytes).  SWAR:
// t = (e | 0x80..) - (q & 0x7f..) never borrows across bytes and its bit 7 is
// [e mod 128 >= q mod 128]; q > e iff (q_7 and not e_7) or (q_7 == e_7 and
// not t_7).  The four bit-7 flags are gathered by one multiply: the factor
// 2^21 + 2^14 + 2^7 + 1 moves bits 7, 15, 23, 31 to 28..31, every other
// partial product landing below bit 28 on a distinct bit (no carries).
__device__ __forceinline__ uint32_t gt4(uint32_t q, uint32_t e) {
  const uint32_t t = (e | 0x80808080u) - (q & 0x7f7f7f7fu);
  const uint32_t g = ((q & ~e) | (~(q ^ e) & ~t)) & 0x80808080u;
  return (g * 0x00204081u) >> 28;
}

__device__ __forceinline__ uint32_t threshold32(const uint4 &q0, const uint4 &q1, const uint4 &e0,
                                                const uint4 &e1) {
  const uint32_t qs[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
  const uint32_t es[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
  uint32_t bits = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) bits = __funnelshift_r(bits, gt4(qs[k], es[k]), 4);   // nibble k -> bits 4k..
  return bits;   // foreground where q > eff-1
}

// ORDER 0: close3 (dilate, erode), open3 (erode, dilate), open1x3 (erode, dilate)
// ORDER 1: open1x3, close3, open3.  D_k = rows by which the input of op k lags.
template <int ORDER>
__device__ __forceinline__ void morph_body(const MorphArgs &a, int nx, int rows_per_band, int gwarp) {
  const int lane = threadIdx.x & 31;
  const int Wd = a.F / 32;
  const int T = (int)a.T;                                  // T <= 2^19
  const int xs = gwarp % nx;
  const int band = gwarp / nx;
  const int gw = xs * MS_LANES_OUT - 1 + lane;             // this lane's image word
  const bool lane_in = gw >= 0 && gw < Wd;
  const bool out_lane = lane >= 1 && lane <= MS_LANES_OUT && lane_in;
  const int tb0 = band * rows_per_band;
  const int tb1 = min(T, tb0 + rows_per_band);
  uint4 e0 = make_uint4(~0u, ~0u, ~0u, ~0u), e1 = e0;
  if (lane_in) {
    const uint4 *e = reinterpret_cast<const uint4 *>(a.effm1 + 32 * gw);
    e0 = __ldg(e);
    e1 = __ldg(e + 1);
  }
  MorphOp<ORDER == 0 ? false : true, ORDER == 0> op1;    // dilate3 | erode1x3
  MorphOp<ORDER == 0 ? true : false, ORDER == 0> op2;    // erode3  | dilate1x3
  MorphOp<ORDER == 0 ? true : false, true> op3;          // erode3  | dilate3
  MorphOp<ORDER == 0 ? false : true, true> op4;          // dilate3 | erode3
  MorphOp<true, ORDER == 1> op5;                         // erode1x3 | erode3
  MorphOp<false, ORDER == 1> op6;                        // dilate1x3 | dilate3
  // Software pipeline: at each step every operation consumes its
  // predecessor's output of the previous step, so the six operations of a
  // step are independent of one another.  Row of stage k's output at step s
  // (input row i = first + s): out_k = out_{k-1} - 1 - (op k is 3x3), out_0 = i;
  // the final stage lags 10 rows.  IN_k = input row lag of op k.
  constexpr int IN1 = 1, IN2 = ORDER == 0 ? 3 : 2, IN3 = ORDER == 0 ? 5 : 3;
  constexpr int IN4 = ORDER == 0 ? 7 : 5, IN5 = ORDER == 0 ? 9 : 7, IN6 = ORDER == 0 ? 10 : 9;
  constexpr int DBG1 = ORDER == 0 ? 4 : 2, DBG2 = ORDER == 0 ? 8 : 6, LAG = 10;
  const int first = tb0 - 4;
  const int nsteps = (tb1 - tb0) + 4 + LAG;
  // byte column of this lane; rows are reached by 64-bit pointer steps
  const uint8_t *base = a.img + 32 * (lane_in ? gw : 0);
  uint4 ring[MS_PF][2];
#pragma unroll
  for (int k = 0; k < MS_PF; ++k) {
    const int i = first + k;
    ring[k][0] = ring[k][1] = make_uint4(0, 0, 0, 0);
    if (lane_in && i >= 0 && i < T) {
      const uint4 *p = reinterpret_cast<const uint4 *>(base + (int64_t)i * a.F);
      ring[k][0] = __ldg(p);
      ring[k][1] = __ldg(p + 1);
    }
  }
  uint32_t p0 = 0, p1 = 0, p2 = 0, p3 = 0, p4 = 0, p5 = 0;   // previous-step stage outputs
  // Every row an operation takes in lies inside the image unless the band is
  // within LAG + 4 rows of the top or 9 rows of the bottom: then only the
  // lane's column decides whether an operation sees a pixel.
  const bool edge_band = tb0 < LAG + 4 || tb1 + 9 > T;
  const bool dbg = a.dbg0 || a.dbg1 || a.dbg2;
  auto run = [&](auto checked, auto with_dbg) {
    constexpr bool CHECK = decltype(checked)::value, DBG = decltype(with_dbg)::value;
    auto in_img = [&](int row) { return CHECK ? lane_in && (unsigned)row < (unsigned)T : lane_in; };
    for (int s0 = 0; s0 < nsteps; s0 += MS_PF) {
#pragma unroll
      for (int k = 0; k < MS_PF; ++k) {
        const int s = s0 + k;
        if (s < nsteps) {   // warp-uniform
          const int i = first + s;
          uint32_t x0 = 0;
          if (in_img(i) && i <= tb1 + 3) x0 = threshold32(ring[k][0], ring[k][1], e0, e1);
          const int ip = i + MS_PF;   // prefetch
          if (in_img(ip) && ip <= tb1 + 3) {
            const uint4 *p = reinterpret_cast<const uint4 *>(base + (int64_t)ip * a.F);
            ring[k][0] = __ldg(p);
            ring[k][1] = __ldg(p + 1);
          }
          const uint32_t x1 = op1.step(p0, in_img(i - IN1));
          const uint32_t x2 = op2.step(p1, in_img(i - IN2));
          const uint32_t x3 = op3.step(p2, in_img(i - IN3));
          const uint32_t x4 = op4.step(p3, in_img(i - IN4));
          const uint32_t x5 = op5.step(p4, in_img(i - IN5));
          const uint32_t x6 = op6.step(p5, in_img(i - IN6));
          p0 = x0; p1 = x1; p2 = x2; p3 = x3; p4 = x4; p5 = x5;
          if constexpr (DBG) {
            if (a.dbg0 && out_lane && i >= tb0 && i < tb1) a.dbg0[(int64_t)i * Wd + gw] = x0;
            if (a.dbg1) {
              const int r = i - DBG1;
              if (out_lane && r >= tb0 && r < tb1) a.dbg1[(int64_t)r * Wd + gw] = x2;
            }
            if (a.dbg2) {
              const int r = i - DBG2;
              if (out_lane && r >= tb0 && r < tb1) a.dbg2[(int64_t)r * Wd + gw] = x4;
            }
          }
          const int r = i - LAG;   // the final row of this step
          if (r >= tb0 && r < tb1) {   // warp-uniform
            // runs starting in this word: its bit 31 neighbour is the left lane's
            // word (exact on the halo lane too), or nothing at the image's left edge
            const uint32_t left = __shfl_up_sync(0xffffffffu, x6, 1);
            if (out_lane) {
              a.mask[(int64_t)r * Wd + gw] = x6;
              const uint32_t lft = gw > 0 ? left : 0u;
              const uint32_t n = __popc(x6 & ~((x6 << 1) | (lft >> 31)));
              if (n) atomicAdd(&a.row_cnt[r], n);
            }
          }
        }
      }
    }
  };
  using T_ = std::true_type;
  using F_ = std::false_type;
  if (dbg) {
    if (edge_band) run(T_{}, T_{});
    else run(F_{}, T_{});
  } else {
    if (edge_band) run(T_{}, F_{});
    else run(F_{}, F_{});
  }
}

template <int ORDER>
__global__ void __launch_bounds__(32 * MS_WARPS, 2)
morph_stream_kernel(MorphArgs a, int nx, int rows_per_band, int n_warps) {
  const int gwarp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (gwarp >= n_warps) return;
  morph_body<ORDER>(a, nx, rows_per_band, gwarp);
}

// Batch: warps are numbered over all captures; warp_base[c] is the first
// warp of capture c (ncap + 1 entries).  Each warp copies its capture's
// arguments to its own shared slot.
template <int ORDER>
__global__ void __launch_bounds__(32 * MS_WARPS, 2)
morph_batch_kernel(const MorphArgs *segs, const MorphItem *mi, const int *warp_base, int ncap,
                   int total_warps) {
  __shared__ MorphArgs sa[MS_WARPS];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * MS_WARPS + wib;
  if (gwarp >= total_warps) return;
  int lo = 0, hi = ncap - 1;   // the last capture whose first warp is <= gwarp
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(&warp_base[mid]) <= gwarp) lo = mid;
    else hi = mid - 1;
  }
  if (lane == 0) sa[wib] = segs[lo];
  __syncwarp();
  const MorphItem it = mi[lo];
  if (kChecked && gwarp - __ldg(&warp_base[lo]) >= __ldg(&warp_base[lo + 1]) - __ldg(&warp_base[lo])) return;
  morph_body<ORDER>(sa[wib], it.nx, it.rows, gwarp - __ldg(&warp_base[lo]));
}
// Bands per cluster.  Grid: (column groups) x (bands); the clusters that fit
// at once come from the occupancy API, and the band count minimises
// waves / bands (time ~ waves x rows per band), so that the last wave is not
// mostly idle.  At least ceil(T / HIST_MAX_ROWS) bands for a single cluster.
template <bool FP>
int bands_for(int groups, int64_t max_T) {
  // clusters of B blocks that fit on the device at once, from the occupancy
  // API once per process (it does not depend on the grid); -1: B does not fit
  static std::mutex mu;
  static int fit[CH_BANDS + 1];
  static bool known = false;
  const int need = (int)std::min<int64_t>(CH_BANDS, (max_T + HIST_MAX_ROWS - 1) / HIST_MAX_ROWS);
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!known) {
      const size_t sm = ch_smem();
      cudaFuncSetAttribute(cluster_hist_kernel<FP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      for (int B = 1; B <= CH_BANDS; ++B) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(1u, (unsigned)B);
        cfg.blockDim = dim3(32 * CH_WARPS);
        cfg.dynamicSmemBytes = sm;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeClusterDimension;
        at[0].val.clusterDim.x = 1;
        at[0].val.clusterDim.y = (unsigned)B;
        at[0].val.clusterDim.z = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, cluster_hist_kernel<FP>, &cfg) != cudaSuccess || n < 1) {
          cudaGetLastError();
          n = -1;
        }
        fit[B] = n;
      }
      known = true;
    }
  }
  int best = CH_BANDS;
  double best_cost = 1e30;
  for (int B = 1; B <= CH_BANDS; ++B) {
    if (fit[B] < 1) continue;
    const double cost = (double)((groups + fit[B] - 1) / fit[B]) / B;
    if (cost <= best_cost) {
      best_cost = cost;
      best = B;
    }
  }
  return std::max(best, need);
}

template <typename K, typename... Args>
cudaError_t launch_clustered(K kernel, size_t sm, dim3 grid, int B, cudaStream_t s, Args... args) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(32 * CH_WARPS);
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 1;
  at[0].val.clusterDim.y = (unsigned)B;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kernel, args...);
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

}  // namespace

void image_preload() {
  preload_kernel(otsu_kernel);
  preload_kernel(cluster_hist_kernel<true>);
  preload_kernel(cluster_hist_kernel<false>);
  preload_kernel(cluster_hist_batch_kernel<true>);
  preload_kernel(cluster_hist_batch_kernel<false>);
  preload_kernel(floor_part_kernel);
  preload_kernel(floor_eff_kernel);
  preload_kernel(floor_batch_kernel);
  preload_kernel(morph_stream_kernel<0>);
  preload_kernel(morph_stream_kernel<1>);
  preload_kernel(morph_batch_kernel<0>);
  preload_kernel(morph_batch_kernel<1>);
}

// Cluster histogram (optionally quantising float power on the way).  The
// histogram is written whole (no zeroing needed) unless T needs more than one
// cluster of bands, in which case the caller's zeroed histogram is accumulated.
bool cluster_hist_accumulates(int64_t T) { return T > (int64_t)CH_BANDS * HIST_MAX_ROWS; }

int cluster_hist_bands(bool from_power, int groups, int64_t max_T) {
  return from_power ? bands_for<true>(groups, max_T) : bands_for<false>(groups, max_T);
}

cudaError_t launch_cluster_hist(const void *src, bool from_power, int64_t T, int F,
                                const float *edges, const float *qconst, uint8_t *img,
                                uint32_t *hist, rise_colstat *cols, bool *needs_zero,
                                cudaStream_t s, const uint32_t *max_bits, const double *ratio,
                                double level_db) {
  static_assert(CH_WARPS >= CH_NS, "one warp per reduced column");
  const int groups_x = F / CH_COLS;
  int B = CH_BANDS;
  int64_t G = 1;
  if (cluster_hist_accumulates(T)) {
    while ((T + G * CH_BANDS - 1) / (G * CH_BANDS) > HIST_MAX_ROWS) ++G;
  } else {
    B = cluster_hist_bands(from_power, groups_x, T);
  }
  const int64_t rows = (T + G * B - 1) / (G * B);
  const int accumulate = G > 1;
  if (needs_zero) *needs_zero = accumulate;
  HistArgs ha{src, T, F, rows, edges, qconst, img, hist, cols, accumulate};
  if (max_bits) {   // the levels are built in the kernel; edges / qconst receive them
    ha.max_bits = max_bits;
    ha.ratio = ratio;
    ha.level_db = level_db;
    ha.edges_out = const_cast<float *>(edges);
    ha.qconst_out = const_cast<float *>(qconst);
  }
  const dim3 grid((unsigned)groups_x, (unsigned)(G * B));
  return from_power ? launch_clustered(cluster_hist_kernel<true>, ch_smem(), grid, B, s, ha)
                    : launch_clustered(cluster_hist_kernel<false>, ch_smem(), grid, B, s, ha);
}

cudaError_t launch_cluster_hist_batch(bool from_power, const HistArgs *segs, const HistItem *items,
                                      int n_items, int bands, cudaStream_t s) {
  if (n_items < 1) return cudaSuccess;
  const dim3 grid((unsigned)n_items, (unsigned)bands);
  return from_power
             ? launch_clustered(cluster_hist_batch_kernel<true>, ch_smem(), grid, bands, s, segs, items)
             : launch_clustered(cluster_hist_batch_kernel<false>, ch_smem(), grid, bands, s, segs, items);
}

cudaError_t launch_floor_batch(const ColArgs *segs, int ncap, int max_F, cudaStream_t s) {
  const size_t sm = 2 * (size_t)max_F * sizeof(int64_t);
  cudaError_t e = cudaFuncSetAttribute(floor_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  floor_batch_kernel<<<ncap, FLOOR_THREADS, sm, s>>>(segs);
  count_launches(1);
  return cudaGetLastError();
}

// Warps and rows per band of the streaming morphology on a T x F image
// (target: about `warps_per_sm` warps per SM for the whole launch).
void morph_plan(int64_t T, int F, int sms, int warps_per_sm, int min_rows, int *nx, int *rows,
                int *n_warps) {
  const int Wd = F / 32;
  *nx = (Wd + MS_LANES_OUT - 1) / MS_LANES_OUT;
  const int64_t want_warps = (int64_t)sms * warps_per_sm;
  int64_t bands = std::max<int64_t>(1, (want_warps + *nx - 1) / *nx);
  int64_t r = std::max<int64_t>(min_rows, (T + bands - 1) / bands);
  bands = (T + r - 1) / r;
  *rows = (int)r;
  *n_warps = (int)(bands * *nx);
}

cudaError_t launch_morph_batch(int order, const MorphArgs *segs, const MorphItem *items,
                               const int *warp_base, int ncap, int total_warps, cudaStream_t s) {
  if (total_warps < 1) return cudaSuccess;
  const unsigned blocks = (unsigned)((total_warps + MS_WARPS - 1) / MS_WARPS);
  if (order == 0)
    morph_batch_kernel<0><<<blocks, 32 * MS_WARPS, 0, s>>>(segs, items, warp_base, ncap, total_warps);
  else
    morph_batch_kernel<1><<<blocks, 32 * MS_WARPS, 0, s>>>(segs, items, warp_base, ncap, total_warps);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_colstats(const ColArgs &a, bool need_otsu, cudaStream_t s) {
  if (!a.st || a.m >= 64) return cudaErrorInvalidValue;
  cudaError_t e;
  if (need_otsu) {
    const int warps_per_block = 8;
    otsu_kernel<<<(a.F + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(a);
    count_launches(1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // column-parallel: two launches of F/256 blocks
  const unsigned g = (unsigned)((a.F + FP_COLS - 1) / FP_COLS);
  floor_part_kernel<<<g, FP_COLS, 0, s>>>(a);
  floor_eff_kernel<<<g, FP_COLS, 0, s>>>(a);
  count_launches(2);
  return cudaGetLastError();
}

cudaError_t launch_column_otsu(const uint32_t *hist, int64_t T, int F, rise_colstat *cols,
                               cudaStream_t s) {
  ColArgs a{};
  a.hist = hist;
  a.T = T;
  a.F = F;
  a.cols = cols;
  const int warps_per_block = 8;
  otsu_kernel<<<(F + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_morph(const MorphArgs &a, cudaStream_t s) {
  const int Wd = a.F / 32;
  const int nx = (Wd + MS_LANES_OUT - 1) / MS_LANES_OUT;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want_warps = (int64_t)sms * 16;
  int64_t bands = std::max<int64_t>(1, (want_warps + nx - 1) / nx);
  int64_t rows = std::max<int64_t>(32, (a.T + bands - 1) / bands);
  bands = (a.T + rows - 1) / rows;
  const int64_t n_warps = bands * nx;
  const unsigned blocks = (unsigned)((n_warps + MS_WARPS - 1) / MS_WARPS);
  if (a.order == 0)
    morph_stream_kernel<0><<<blocks, 32 * MS_WARPS, 0, s>>>(a, nx, (int)rows, (int)n_warps);
  else
    morph_stream_kernel<1><<<blocks, 32 * MS_WARPS, 0, s>>>(a, nx, (int)rows, (int)n_warps);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace rise
