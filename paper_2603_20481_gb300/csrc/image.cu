// Image stages of RISE (Sec. IV-B): column histograms of the 8-bit TF plot,
// the PSD (column sums) with Savitzky-Golay smoothing and the lowest local
// minimum N0, theta_PSD column pruning, exact per-column Otsu (Eq. 4) with
// the power floor, and the binary mask with one 2D closing, one 2D opening
// and one horizontal 1D opening (Eq. 5) on bit-packed tiles.
#include "common.cuh"

namespace rise {
namespace {

// ---------------------------------------------------------------------------
// Column histogram.  A block owns a strip of 128 columns and a band of rows.
// Lane l reads 4 consecutive columns (4l..4l+3) of a row as one 32-bit load;
// column 4l+j is counted in smem slot l+32j so that the 32 lanes of a warp
// always hit 32 different banks.  Each 32-bit smem word holds two 16-bit
// counters, levels v and v+128, so the strip's 128 x 256 counters fit in
// 64 KB; a band has at most 65535 rows so a counter cannot overflow.
// ---------------------------------------------------------------------------
constexpr int HIST_COLS = 128;
constexpr int HIST_THREADS = 256;
constexpr int HIST_MAX_ROWS = 65535;

__device__ __forceinline__ void hist_count(uint32_t *sh, int lane, uint32_t word4) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t v = (word4 >> (8 * j)) & 0xffu;
    atomicAdd(&sh[(v & 127u) * HIST_COLS + lane + 32 * j], (v & 128u) ? 65536u : 1u);
  }
}

__device__ __forceinline__ void hist_flush(const uint32_t *sh, uint32_t *hist, int c0) {
  for (int i = threadIdx.x; i < 128 * HIST_COLS; i += blockDim.x) {
    const uint32_t w = sh[i];
    if (!w) continue;
    const int vm = i / HIST_COLS, pc = i % HIST_COLS;
    const int col = c0 + 4 * (pc & 31) + (pc >> 5);
    const uint32_t lo = w & 0xffffu, hi = w >> 16;
    if (lo) atomicAdd(&hist[(size_t)col * 256 + vm], lo);
    if (hi) atomicAdd(&hist[(size_t)col * 256 + vm + 128], hi);
  }
}

__global__ void __launch_bounds__(HIST_THREADS)
hist_kernel(const uint8_t *__restrict__ img, int64_t T, int F, int64_t rows_per_block,
            uint32_t *hist) {
  extern __shared__ uint32_t sh[];
  for (int i = threadIdx.x; i < 128 * HIST_COLS; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const int c0 = blockIdx.x * HIST_COLS;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = min(T, r0 + rows_per_block);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  const uint8_t *base = img + c0 + 4 * lane;
  int64_t r = r0 + warp;
  for (; r + 3 * nw < r1; r += 4 * nw) {
    uint32_t w0 = __ldg(reinterpret_cast<const uint32_t *>(base + r * F));
    uint32_t w1 = __ldg(reinterpret_cast<const uint32_t *>(base + (r + nw) * F));
    uint32_t w2 = __ldg(reinterpret_cast<const uint32_t *>(base + (r + 2 * nw) * F));
    uint32_t w3 = __ldg(reinterpret_cast<const uint32_t *>(base + (r + 3 * nw) * F));
    hist_count(sh, lane, w0);
    hist_count(sh, lane, w1);
    hist_count(sh, lane, w2);
    hist_count(sh, lane, w3);
  }
  for (; r < r1; r += nw) hist_count(sh, lane, __ldg(reinterpret_cast<const uint32_t *>(base + r * F)));
  __syncthreads();
  hist_flush(sh, hist, c0);
}

// Quantise a stored float |X|^2 image (same level rule as the STFT epilogue)
// while counting the column histogram.
constexpr float kGuardQ = 1.0e-3f;
__device__ __forceinline__ int level_of_q(float P, float inv_anchor, float c1, const float *edges) {
  float v = fmaf(__log2f(P * inv_anchor), c1, 255.5f);
  float fl = floorf(v);
  float fr = v - fl;
  int q = (int)fminf(fmaxf(fl, 0.0f), 255.0f);
  if ((fr < kGuardQ || fr > 1.0f - kGuardQ) && v > 1.0f - 2.0f * kGuardQ && v < 255.0f + 2.0f * kGuardQ) {
    for (int it = 0; it < 256 && q < 255 && P >= edges[q + 1]; ++it) ++q;
    for (int it = 0; it < 256 && q > 0 && P < edges[q]; ++it) --q;
  }
  return q;
}

__global__ void __launch_bounds__(HIST_THREADS)
quant_hist_kernel(const float *__restrict__ power, int64_t T, int F, int64_t rows_per_block,
                  const float *edges_g, const float *qconst, uint8_t *img, uint32_t *hist) {
  extern __shared__ uint32_t sh[];
  __shared__ float edges[257];
  for (int i = threadIdx.x; i < 128 * HIST_COLS; i += blockDim.x) sh[i] = 0;
  for (int i = threadIdx.x; i < 257; i += blockDim.x) edges[i] = edges_g[i];
  const float inv_anchor = qconst[0], c1 = qconst[1];
  __syncthreads();
  const int c0 = blockIdx.x * HIST_COLS;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_block;
  const int64_t r1 = min(T, r0 + rows_per_block);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  for (int64_t r = r0 + warp; r < r1; r += nw) {
    const float4 p = __ldg(reinterpret_cast<const float4 *>(power + r * F + c0) + lane);
    const uint32_t q0 = level_of_q(p.x, inv_anchor, c1, edges);
    const uint32_t q1 = level_of_q(p.y, inv_anchor, c1, edges);
    const uint32_t q2 = level_of_q(p.z, inv_anchor, c1, edges);
    const uint32_t q3 = level_of_q(p.w, inv_anchor, c1, edges);
    const uint32_t w4 = q0 | (q1 << 8) | (q2 << 16) | (q3 << 24);
    reinterpret_cast<uint32_t *>(img + r * F + c0)[lane] = w4;
    hist_count(sh, lane, w4);
  }
  __syncthreads();
  hist_flush(sh, hist, c0);
}

void hist_grid(int64_t T, int F, int num_sms, dim3 &grid, int64_t &rows) {
  const int strips = F / HIST_COLS;
  int64_t want = std::max<int64_t>(1, (2 * (int64_t)num_sms + strips - 1) / strips);
  rows = (T + want - 1) / want;
  rows = std::max<int64_t>(rows, 256);
  rows = (rows + 7) / 8 * 8;
  rows = std::min<int64_t>(rows, HIST_MAX_ROWS / 8 * 8);   // 16-bit counters never wrap
  grid = dim3(strips, (unsigned)((T + rows - 1) / rows));
}

// ---------------------------------------------------------------------------
// Per-column Otsu: one warp per column.  Lane l owns levels 8l..8l+7.  For a
// split theta (class 0 = levels <= theta) with n0, s0 the count and level sum
// of class 0 and n, s the column totals, sigma_b^2 is proportional to
// d^2 / (n0 n1) with d = s0 n - s n0; candidates are compared exactly by
// cross-multiplication in 128-bit integers and the smallest maximiser wins.
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

__global__ void otsu_kernel(ColArgs a) {
  const int warp_g = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp_g >= a.F) return;
  const int f = warp_g;
  const uint4 *h4 = reinterpret_cast<const uint4 *>(a.hist + (size_t)f * 256 + 8 * lane);
  const uint4 x = h4[0], y = h4[1];
  uint32_t h[8] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
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
  if (lane == 0) {
    a.cols[f].S = s;
    a.cols[f].otsu = best.th;
  }
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

__global__ void __launch_bounds__(FLOOR_THREADS) floor_kernel(ColArgs a) {
  extern __shared__ int64_t S[];   // [F]
  __shared__ int64_t red_min[32];
  __shared__ int red_found[32];
  __shared__ int64_t c[64];
  const int F = a.F, m = a.m, tid = threadIdx.x;
  for (int i = tid; i <= m; i += blockDim.x) c[i] = a.sg_c[i];
  for (int f = tid; f < F; f += blockDim.x) S[f] = (int64_t)a.cols[f].S;
  __syncthreads();
  // Savitzky-Golay on the interior, lowest local minimum (strictly below the
  // left neighbour, not above the right one)
  int64_t best = INT64_MAX, gmin = INT64_MAX;
  int found = 0;
  auto shat = [&](int f) {
    int64_t acc = c[0] * S[f];
    for (int i = 1; i <= m; ++i) acc += c[i] * (S[f - i] + S[f + i]);
    return acc;
  };
  for (int f = m + tid; f <= F - 1 - m; f += blockDim.x) {
    const int64_t v = shat(f);
    a.cols[f].Shat = v;
    gmin = min(gmin, v);
    if (f >= m + 1 && f <= F - 2 - m) {
      const int64_t l = shat(f - 1), r = shat(f + 1);
      if (v < l && v <= r) { found = 1; best = min(best, v); }
    }
  }
  for (int f = tid; f < F; f += blockDim.x)
    if (f < m || f > F - 1 - m) a.cols[f].Shat = 0;
  // block reductions
  const int lane = tid & 31, w = tid >> 5;
  int64_t b2 = best, g2 = gmin;
  int fd = found;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    b2 = min(b2, __shfl_xor_sync(0xffffffffu, b2, o));
    g2 = min(g2, __shfl_xor_sync(0xffffffffu, g2, o));
    fd |= __shfl_xor_sync(0xffffffffu, fd, o);
  }
  __shared__ int64_t red_g[32];
  if (lane == 0) { red_min[w] = b2; red_g[w] = g2; red_found[w] = fd; }
  __syncthreads();
  __shared__ int64_t s_N0, s_Pq;
  if (tid == 0) {
    int64_t bb = INT64_MAX, gg = INT64_MAX;
    int ff = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      bb = min(bb, red_min[i]);
      gg = min(gg, red_g[i]);
      ff |= red_found[i];
    }
    const int64_t N0 = ff ? bb : gg;
    const int64_t DT = a.D * a.T;
    int64_t Pq = 0;
    if (a.pow_on) {
      Pq = -floor_div_d(-(N0 + a.delta_pow), DT);
      Pq = Pq < 0 ? 0 : (Pq > 256 ? 256 : Pq);
    }
    s_N0 = N0;
    s_Pq = Pq;
    int64_t *fo = a.floor_out;
    fo[0] = N0; fo[1] = a.delta_psd; fo[2] = a.delta_pow; fo[3] = Pq;
    fo[4] = a.D; fo[5] = a.T; fo[6] = F; fo[7] = 0;
  }
  __syncthreads();
  const int64_t N0 = s_N0, Pq = s_Pq;
  for (int f = tid; f < F; f += blockDim.x) {
    const int keep = a.psd_on ? (a.D * S[f] >= N0 + a.delta_psd) : 1;
    const int th = a.cols[f].otsu;
    int eff = 256;
    if (keep && th >= 0) eff = max(th + 1, (int)Pq);
    a.cols[f].keep = keep;
    a.cols[f].eff = eff;
    a.cols[f].pad = 0;
    a.effm1[f] = (uint8_t)min(255, max(0, eff - 1));
  }
}

// ---------------------------------------------------------------------------
// Threshold + morphology on bit-packed tiles.  A tile is 120 interior rows x
// 32 interior words (1024 columns) plus a halo of 4 rows and 1 word (32
// columns) on every side: the four 3x3 operations shift information by one
// row each and all six by one column each, so the interior is exact.  A
// pixel outside the image takes no part in an operation: it reads as 0 for a
// dilation and as 1 for an erosion (the clipped window).  544 threads: in
// each operation every thread computes one word-column of 8 rows.
// ---------------------------------------------------------------------------
constexpr int MT_ROWS = 128, MT_IN_ROWS = 120, MT_WORDS = 34, MT_IN_WORDS = 32;
constexpr int MT_RB = 8, MT_THREADS = MT_WORDS * (MT_ROWS / MT_RB);   // 544

struct TileCtx {
  int64_t t_base;   // image row of tile row 0
  int64_t w_base;   // image word of tile word 0
  int64_t T;
  int Wd;
};

template <bool ERODE>
__device__ __forceinline__ uint32_t tget(const uint32_t *in, int r, int w, const TileCtx &c) {
  const int64_t t = c.t_base + r, gw = c.w_base + w;
  if (t < 0 || t >= c.T || gw < 0 || gw >= c.Wd) return ERODE ? 0xffffffffu : 0u;
  if (r < 0 || r >= MT_ROWS || w < 0 || w >= MT_WORDS) return 0u;   // outside the tile: never used
  return in[r * MT_WORDS + w];
}

template <bool ERODE>
__device__ __forceinline__ uint32_t hop_row(const uint32_t *in, int r, int w, const TileCtx &c) {
  const uint32_t x = tget<ERODE>(in, r, w, c);
  const uint32_t l = tget<ERODE>(in, r, w - 1, c);
  const uint32_t rt = tget<ERODE>(in, r, w + 1, c);
  const uint32_t xl = (x << 1) | (l >> 31);    // pixel f-1 moved to f
  const uint32_t xr = (x >> 1) | (rt << 31);   // pixel f+1 moved to f
  return ERODE ? (x & xl & xr) : (x | xl | xr);
}

// one operation over the whole tile: 3x3 (VERT) or 1x3, dilation or erosion
template <bool ERODE, bool VERT>
__device__ __forceinline__ void morph_op(const uint32_t *in, uint32_t *out, const TileCtx &c) {
  const int w = threadIdx.x % MT_WORDS;
  const int r0 = (threadIdx.x / MT_WORDS) * MT_RB;
  if constexpr (VERT) {
    uint32_t above = hop_row<ERODE>(in, r0 - 1, w, c);
    uint32_t cur = hop_row<ERODE>(in, r0, w, c);
#pragma unroll
    for (int i = 0; i < MT_RB; ++i) {
      const uint32_t below = hop_row<ERODE>(in, r0 + i + 1, w, c);
      out[(r0 + i) * MT_WORDS + w] = ERODE ? (above & cur & below) : (above | cur | below);
      above = cur;
      cur = below;
    }
  } else {
#pragma unroll
    for (int i = 0; i < MT_RB; ++i) out[(r0 + i) * MT_WORDS + w] = hop_row<ERODE>(in, r0 + i, w, c);
  }
}

__device__ __forceinline__ uint32_t gather4(uint32_t m) {
  // bit j of the result = bit 0 of byte j (each byte of m is 0x00 or 0xff)
  return (((m & 0x01010101u) * 0x01020408u) >> 24) & 0xfu;
}

__device__ __forceinline__ void store_tile(const uint32_t *in, uint32_t *dst, const TileCtx &c) {
  for (int i = threadIdx.x; i < MT_IN_ROWS * MT_IN_WORDS; i += blockDim.x) {
    const int r = 4 + i / MT_IN_WORDS, w = 1 + i % MT_IN_WORDS;
    const int64_t t = c.t_base + r, gw = c.w_base + w;
    if (t < c.T && gw < c.Wd) dst[t * c.Wd + gw] = in[r * MT_WORDS + w];
  }
}

__global__ void __launch_bounds__(MT_THREADS)
morph_kernel(MorphArgs a) {
  __shared__ uint32_t A[MT_ROWS * MT_WORDS], B[MT_ROWS * MT_WORDS];
  __shared__ __align__(16) uint8_t eff[MT_WORDS * 32];
  const int Wd = a.F / 32;
  TileCtx c;
  c.t_base = (int64_t)blockIdx.y * MT_IN_ROWS - 4;
  c.w_base = (int64_t)blockIdx.x * MT_IN_WORDS - 1;
  c.T = a.T;
  c.Wd = Wd;
  for (int i = threadIdx.x; i < MT_WORDS * 32; i += blockDim.x) {
    const int64_t col = c.w_base * 32 + i;
    eff[i] = (col >= 0 && col < a.F) ? a.effm1[col] : 255;
  }
  __syncthreads();
  // threshold: foreground where q > eff-1
  for (int i = threadIdx.x; i < MT_ROWS * MT_WORDS; i += blockDim.x) {
    const int r = i / MT_WORDS, w = i % MT_WORDS;
    const int64_t t = c.t_base + r, gw = c.w_base + w;
    uint32_t bits = 0;
    if (t >= 0 && t < a.T && gw >= 0 && gw < Wd) {
      const uint4 *src = reinterpret_cast<const uint4 *>(a.img + t * a.F + gw * 32);
      const uint4 q0 = __ldg(src), q1 = __ldg(src + 1);
      const uint4 *e4 = reinterpret_cast<const uint4 *>(eff + w * 32);
      const uint4 e0 = e4[0], e1 = e4[1];
      const uint32_t qs[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
      const uint32_t es[8] = {e0.x, e0.y, e0.z, e0.w, e1.x, e1.y, e1.z, e1.w};
#pragma unroll
      for (int k = 0; k < 8; ++k) bits |= gather4(__vcmpgtu4(qs[k], es[k])) << (4 * k);
    }
    A[i] = bits;
  }
  __syncthreads();
  if (a.dbg0) store_tile(A, a.dbg0, c);
  if (a.order == 0) {
    morph_op<false, true>(A, B, c); __syncthreads();   // close 3x3: dilate
    morph_op<true, true>(B, A, c);  __syncthreads();   //            erode
    if (a.dbg1) store_tile(A, a.dbg1, c);
    morph_op<true, true>(A, B, c);  __syncthreads();   // open 3x3: erode
    morph_op<false, true>(B, A, c); __syncthreads();   //           dilate
    if (a.dbg2) store_tile(A, a.dbg2, c);
    morph_op<true, false>(A, B, c); __syncthreads();   // open 1x3: erode
    morph_op<false, false>(B, A, c); __syncthreads();  //           dilate
  } else {
    morph_op<true, false>(A, B, c); __syncthreads();   // open 1x3
    morph_op<false, false>(B, A, c); __syncthreads();
    if (a.dbg1) store_tile(A, a.dbg1, c);
    morph_op<false, true>(A, B, c); __syncthreads();   // close 3x3
    morph_op<true, true>(B, A, c);  __syncthreads();
    if (a.dbg2) store_tile(A, a.dbg2, c);
    morph_op<true, true>(A, B, c);  __syncthreads();   // open 3x3
    morph_op<false, true>(B, A, c); __syncthreads();
  }
  store_tile(A, a.mask, c);
}

}  // namespace

cudaError_t launch_hist(const uint8_t *img, int64_t T, int F, uint32_t *hist, int num_sms,
                        cudaStream_t s) {
  dim3 grid;
  int64_t rows;
  hist_grid(T, F, num_sms, grid, rows);
  const size_t sm = 128 * HIST_COLS * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  hist_kernel<<<grid, HIST_THREADS, sm, s>>>(img, T, F, rows, hist);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_quant_hist(const float *power, int64_t T, int F, const float *edges,
                              const float *qconst, uint8_t *img, uint32_t *hist, int num_sms,
                              cudaStream_t s) {
  dim3 grid;
  int64_t rows;
  hist_grid(T, F, num_sms, grid, rows);
  const size_t sm = 128 * HIST_COLS * sizeof(uint32_t);
  cudaError_t e = cudaFuncSetAttribute(quant_hist_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  quant_hist_kernel<<<grid, HIST_THREADS, sm, s>>>(power, T, F, rows, edges, qconst, img, hist);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_colstats(const ColArgs &a, cudaStream_t s) {
  const int warps_per_block = 8;
  otsu_kernel<<<(a.F + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, s>>>(a);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sm = (size_t)a.F * sizeof(int64_t);
  e = cudaFuncSetAttribute(floor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  floor_kernel<<<1, FLOOR_THREADS, sm, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_morph(const MorphArgs &a, cudaStream_t s) {
  const int Wd = a.F / 32;
  dim3 grid((Wd + MT_IN_WORDS - 1) / MT_IN_WORDS, (unsigned)((a.T + MT_IN_ROWS - 1) / MT_IN_ROWS));
  morph_kernel<<<grid, MT_THREADS, 0, s>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace rise
