// Shared device helpers and host-side declarations of the RISE CUDA library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rise.h"

namespace rise {

// ---------------------------------------------------------------------------
// Device error word: kernels record consistency failures here instead of
// trapping; the host maps a nonzero word to RISE_EINTERNAL / RISE_ETIMEOUT.
// ---------------------------------------------------------------------------
enum : uint32_t {
  ERR_NONE = 0,
  ERR_RUN_CAPACITY = 1u << 0,   // more runs than the run arrays hold (host regrows)
  ERR_UNION_LIMIT = 1u << 1,    // a union/find loop hit its iteration limit
  ERR_ROW_RUNS = 1u << 2,       // a row holds more runs than the morphology allows
  ERR_INDEX = 1u << 3,          // an index check failed
  ERR_SCAN = 1u << 4,           // a single-pass scan waited too long for a predecessor tile
  ERR_COPY_WAIT = 1u << 5,      // the STFT waited too long for a staged input copy
};

struct DeviceStatus {
  uint32_t err;        // OR of ERR_* bits
  uint32_t pad;
  int64_t n_runs;      // total runs of the final mask
  int64_t n_boxes;     // number of components
  uint32_t max_bits;   // float bits of the anchor power
  uint32_t pad2;
  int64_t n_merge;     // deferred unions recorded by the labelling row pass
  // noise floor of one image, gathered by the column blocks: order-reversed
  // keys of the lowest local minimum and of the lowest smoothed PSD (0: none
  // yet, so a zeroed status is the empty state), and whether a local
  // minimum exists
  unsigned long long floor_best, floor_gmin;
  uint32_t floor_found;
  uint32_t pad3;
};

__device__ __forceinline__ void set_err(DeviceStatus *st, uint32_t bit) {
  atomicOr(&st->err, bit);
}

// ---------------------------------------------------------------------------
// Checked build (compiled with -DRISE_CHECKED): indices that come from data
// (run offsets, union-find parents, table entries, frame ranges) are checked
// before use; a failed check records ERR_INDEX (the call returns
// RISE_EINTERNAL) and the access is skipped, so no kernel traps or touches
// memory out of range.  In the normal build every check is a constant true.
// ---------------------------------------------------------------------------
#ifdef RISE_CHECKED
constexpr bool kChecked = true;
__device__ __forceinline__ bool ck_index(int64_t i, int64_t n, uint32_t *err) {
  if (i >= 0 && i < n) return true;
  atomicOr(err, ERR_INDEX);
  return false;
}
#else
constexpr bool kChecked = false;
__device__ __forceinline__ bool ck_index(int64_t, int64_t, uint32_t *) { return true; }
#endif
__device__ __forceinline__ bool ck_index(int64_t i, int64_t n, DeviceStatus *st) {
  return ck_index(i, n, &st->err);
}

// bits 0..b inclusive
__device__ __forceinline__ uint32_t mask_upto(int b) {
  return b >= 31 ? 0xffffffffu : ((2u << b) - 1u);
}

// Start bits of runs in a row word: set where the pixel is on and the pixel
// to its left (bit b-1, or the previous word's bit 31) is off.
__device__ __forceinline__ uint32_t run_starts(uint32_t w, uint32_t prev_word) {
  return w & ~((w << 1) | (prev_word >> 31));
}
// End bits: set where the pixel is on and the pixel to its right is off.
__device__ __forceinline__ uint32_t run_ends(uint32_t w, uint32_t next_word) {
  return w & ~((w >> 1) | (next_word << 31));
}

// ---------------------------------------------------------------------------
// Lock-free union-find with union by smaller index (parent[x] <= x always),
// usable on shared or global memory through generic pointers.  Each loop is
// bounded (`limit` steps, UF_LIMIT by default); hitting the bound records
// ERR_UNION_LIMIT and returns an ancestor, so every index stays in range.
// ---------------------------------------------------------------------------
constexpr int UF_LIMIT = 1 << 26;
// Default bound of a single-pass scan's wait for a predecessor tile: polls
// 32 ns apart, about a second in all.
constexpr int SCAN_SPIN_LIMIT = 1 << 20;

__device__ __forceinline__ int uf_find(int *parent, int x, DeviceStatus *st, int limit = UF_LIMIT) {
  for (int it = 0; it < limit; ++it) {
    int p = *(volatile int *)&parent[x];
    if (p == x) return x;
    if (!ck_index(p, (int64_t)x, st)) return x;   // checked build: a parent is a smaller run
    int gp = *(volatile int *)&parent[p];
    // path halving: x is not a root and never becomes one, so any ancestor
    // (all smaller than x) is a valid parent; a plain store is enough
    if (gp != p) *(volatile int *)&parent[x] = gp;
    x = p;
  }
  set_err(st, ERR_UNION_LIMIT);
  return x;
}

__device__ __forceinline__ void uf_union(int *parent, int a, int b, DeviceStatus *st, int limit = UF_LIMIT) {
  for (int it = 0; it < limit; ++it) {
    a = uf_find(parent, a, st, limit);
    b = uf_find(parent, b, st, limit);
    if (a == b) return;
    if (a > b) { int t = a; a = b; b = t; }
    // link the larger root under the smaller one if it is still a root
    int old = atomicCAS(&parent[b], b, a);
    if (old == b) return;
  }
  set_err(st, ERR_UNION_LIMIT);
}

// Block-wide exclusive scan of one value per thread (blockDim.x <= 1024,
// multiple of 32).  `scratch` needs 32 entries.  Returns the exclusive
// prefix; *total receives the block sum.
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *scratch, T *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) scratch[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T s = lane < nwarps ? scratch[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    scratch[lane] = s;  // inclusive warp-total prefix
  }
  __syncthreads();
  T warp_base = warp > 0 ? scratch[warp - 1] : T(0);
  T tot = scratch[nwarps - 1];
  __syncthreads();
  if (total) *total = tot;
  return warp_base + x - v;
}

}  // namespace rise

// ---------------------------------------------------------------------------
// Host-side launchers implemented in the .cu files (internal, not exported).
// ---------------------------------------------------------------------------
namespace rise {

// Kernels launched by the library (process-wide), for launch accounting.
void count_launches(int k);
// Kernels load lazily on their first launch (milliseconds each for the
// large FFT instances): each translation unit's preload queries the
// attributes of all its kernels, which loads them, so that no detection
// call pays for a load.  Called once per process by rise_create.
template <typename K>
inline void preload_kernel(K k) {
  cudaFuncAttributes a;
  if (cudaFuncGetAttributes(&a, k) != cudaSuccess) cudaGetLastError();
}
void stft_preload();
void stft_s1_preload();
void stft_s2_preload();
void stft_sc16_preload();
void image_preload();
void ccl_preload();
void batch_preload();
void match_preload();
long long launches_so_far();

enum IqFormat { IQ_FC32 = 0, IQ_SC16 = 1 };

struct StftArgs {
  const void *iq;         // device, n complex samples (float2, or short2 for sc16)
  int64_t n;
  int N;                  // FFT size
  int hop;
  int64_t T;              // frames
  uint8_t *img;           // [T][N] levels (quantise mode)
  float *power;           // [T][N] |X|^2 (power mode / kept)
  uint32_t *max_bits;     // float bits of the running max (max/power mode)
  const float *edges;     // [257] level edges (quantise mode)
  const float *qconst;    // [2]: 1/anchor, dB-per-level scale (quantise mode)
  const float2 *tw;       // per-N twiddle tables (device)
  const float *win;       // per-N Hann window (device)
  uint32_t *err;          // device error word (ERR_* bits)
  int fmt;                // IqFormat
  int sched;              // radix schedule of the tables tw (0: radix-16 passes first, 1: the small radix
                          // first, 2: the frame split into two half-size transforms)
  int wait_limit;         // try_wait calls before a staged copy is given up (STFT_WAIT_LIMIT)
  int64_t withhold_step;  // test only: block 0 issues no copy for this step (-1: none)
};
// Default bound of the STFT's wait for a staged input copy, in try_wait calls
// (each suspends the thread for a hardware-defined interval).
constexpr int STFT_WAIT_LIMIT = 1 << 22;

// STFT_POWER_HOOKED is STFT_POWER in a separate kernel instance that also
// honours the copy-wait bound and the withheld copy of StftArgs (the test
// hooks); the other instances wait with the fixed bound STFT_WAIT_LIMIT and
// never withhold, so the hooks cost the default path nothing.
enum StftMode { STFT_MAX = 0, STFT_QUANT = 1, STFT_POWER = 2, STFT_QUANT_POWER = 3, STFT_POWER_HOOKED = 4 };
cudaError_t launch_stft_sc16(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s);
// Schedules 1 and 2 of complex64 input (their own translation units).
cudaError_t launch_stft_s1(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s);
cudaError_t launch_stft_s2(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s);
// True when schedule S of size N exists apart from schedule 0: S = 1 for N
// not a power of 16, S = 2 for N twice a power of 16.
bool stft_sched_distinct(int N, int S);
// The library's schedule for size N: 2 at N = 8192 (its two halves run
// decoupled), else 1 where it exists, else 0.
int stft_default_sched(int N);

// ---------------------------------------------------------------------------
// Batches: one launch per stage covers many captures; each block or warp
// reads its capture's arguments from a device table.
// ---------------------------------------------------------------------------
struct CapSmall {             // per-capture small state of a batch
  uint32_t max_bits;          // float bits of the capture's largest |X|^2
  uint32_t pad;
  float qconst[4];
  float edges[260];
  int64_t floor_out[8];
};
struct StftItem {             // frames [f0, f1) of capture `seg`
  int32_t seg, pad;
  int64_t f0, f1;
};
cudaError_t launch_stft_batch(int N, int sched, bool tma, StftMode mode, const StftArgs *segs,
                              const StftItem *items, int n_items, int *counter, int num_sms,
                              cudaStream_t s);
cudaError_t launch_stft_batch_s1(int N, bool tma, StftMode mode, const StftArgs *segs, const StftItem *items,
                                 int n_items, int *counter, int num_sms, cudaStream_t s);
cudaError_t launch_stft_batch_s2(int N, bool tma, StftMode mode, const StftArgs *segs, const StftItem *items,
                                 int n_items, int *counter, int num_sms, cudaStream_t s);
int stft_frames_per_step(int N);
cudaError_t launch_levels_batch(CapSmall *cs, int ncap, double hi_power, int use_fixed,
                                const double *ratio, double level_db, cudaStream_t s);

// Twiddle and window tables for FFT size N, radix schedule S (host-computed,
// FP64 -> float).
size_t stft_table_floats(int N, int S);
void stft_fill_tables(int N, int S, float2 *tw_host, float *win_host);
cudaError_t launch_stft(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s);
// Level edges from the anchor (AUTO: read from max_bits; FIXED: hi_power).
cudaError_t launch_levels(const uint32_t *max_bits, double hi_power, int use_fixed,
                          const double *ratio, double level_db, float *edges, float *qconst,
                          cudaStream_t s);

// Cluster histogram: 8-bit image (from_power = false) or float power quantised
// on the way (img written).  *needs_zero tells whether hist had to be zeroed
// (only for T > 8 * 65535); call with needs_zero to query before launching.
// Also writes each column's PSD S and Otsu threshold into cols (unless the
// histogram is accumulated over several clusters: then launch_colstats runs Otsu).
// launch_colstats is the one-image floor (it needs a.st, the call's zeroed
// status); batches use launch_floor_batch.
cudaError_t launch_cluster_hist(const void *src, bool from_power, int64_t T, int F,
                                const float *edges, const float *qconst, uint8_t *img,
                                uint32_t *hist, rise_colstat *cols, bool *needs_zero,
                                cudaStream_t s, const uint32_t *max_bits = nullptr,
                                const double *ratio = nullptr, double level_db = 0.0);
// True when T needs more than one cluster of row bands: then hist must be
// zeroed before launch_cluster_hist, which accumulates into it.
bool cluster_hist_accumulates(int64_t T);

struct ColArgs {
  const uint32_t *hist;   // [F][256]
  int64_t T;
  int F;
  int m;                  // SG half window
  int64_t D;              // SG norm
  const int64_t *sg_c;    // device [m+1] integer SG weights
  int64_t delta_psd;
  int64_t delta_pow;
  int psd_on, pow_on;
  rise_colstat *cols;     // [F]
  uint8_t *effm1;         // [F] eff-1 clamped to 0..255 (q > effm1 is foreground)
  int64_t *floor_out;     // [8]
  DeviceStatus *st;       // one image: the floor's gathering words (zeroed)
};
cudaError_t launch_colstats(const ColArgs &a, bool need_otsu, cudaStream_t s);

struct HistArgs {             // one image for the cluster histogram
  const void *src;            // float [T][F] power or uint8 [T][F] levels
  int64_t T;
  int F;
  int64_t rows_per_band;
  const float *edges;         // [257] level edges (float source)
  const float *qconst;        // fast-level constants (float source)
  uint8_t *img;               // [T][F] levels written (float source)
  uint32_t *hist;             // [F][256]
  rise_colstat *cols;         // [F] S and Otsu threshold
  int accumulate;             // add into a zeroed hist (no Otsu) instead of storing
  // float source, levels built in the kernel from the capture's maximum
  // (max_bits != NULL; the same rule as the levels kernel): the FP64 ratio
  // table and level step, and where block (0, 0) leaves the edges and
  // constants for later readers; else edges / qconst are read as given
  const uint32_t *max_bits;
  const double *ratio;
  double level_db;
  float *edges_out, *qconst_out;
};
struct HistItem {             // column group cg of capture seg
  int32_t seg, cg;
};
// Bands per cluster for `groups` column groups (chosen for whole waves, and
// at least enough that no band exceeds the per-band row limit for max_T).
int cluster_hist_bands(bool from_power, int groups, int64_t max_T);
cudaError_t launch_cluster_hist_batch(bool from_power, const HistArgs *segs, const HistItem *items,
                                      int n_items, int bands, cudaStream_t s);
cudaError_t launch_floor_batch(const ColArgs *segs, int ncap, int max_F, cudaStream_t s);
// S and Otsu threshold of every column of a given [F][256] histogram.
cudaError_t launch_column_otsu(const uint32_t *hist, int64_t T, int F, rise_colstat *cols,
                               cudaStream_t s);

struct MorphArgs {
  const uint8_t *img;     // [T][F]
  const uint8_t *effm1;   // [F]
  int64_t T;
  int F;
  int order;
  uint32_t *mask;         // [T][F/32] final
  uint32_t *dbg0, *dbg1, *dbg2;  // optional stage masks
  uint32_t *row_cnt;      // [T] runs per row of the final mask (zeroed by the caller)
};
cudaError_t launch_morph(const MorphArgs &a, cudaStream_t s);
struct MorphItem {            // launch shape of one capture in a batch
  int nx, rows;
};
void morph_plan(int64_t T, int F, int sms, int warps_per_sm, int min_rows, int *nx, int *rows,
                int *n_warps);
cudaError_t launch_morph_batch(int order, const MorphArgs *segs, const MorphItem *items,
                               const int *warp_base, int ncap, int total_warps, cudaStream_t s);

struct CclArgs {
  const uint32_t *mask;   // [T][W] final mask words, W = F/32
  const uint8_t *img;     // [T][F]
  int64_t T;
  int F;
  const uint64_t *energy; // [256] energy table
  int64_t *row_base;      // [T+1] run offsets per row (scan output)
  uint32_t *row_cnt;      // [T] runs per row (from the morphology kernel)
  int64_t run_cap;        // capacity of the run arrays
  int32_t *run_parent;    // [run_cap] union-find parent (a smaller run number, or itself)
  uint8_t *run_sroot;     // [run_cap] 1 = the run is its component's root
  rise_box *rec;          // [run_cap] per-run records, summed into the roots
  int2 *merge;            // [run_cap] deferred unions (upper run, lower run)
  int64_t *run_out;       // [run_cap + 1] compaction scan scratch
  void *scan_tmp;         // scan scratch
  size_t scan_tmp_bytes;
  rise_box *boxes;        // [box_cap] output
  int64_t box_cap;
  DeviceStatus *status;
  DeviceStatus *status_out;   // mapped host copy written by the last kernel, or NULL
  int uf_limit;               // steps before a union-find walk gives up (ERR_UNION_LIMIT)
  int spin_limit;             // polls before a look-back wait gives up (ERR_SCAN)
  int64_t withhold_tile;      // test only: this root-scan tile publishes no sum (-1: none)
};
size_t ccl_scan_tmp_bytes(int64_t max_items);
// Scan of the per-row run counts: fills row_base and status->n_runs.
cudaError_t launch_ccl_count(const CclArgs &a, int num_sms, cudaStream_t s);
// Run records, unions, reduction into roots and compaction (needs run_cap >=
// n_runs, checked on the device: on shortfall it sets ERR_RUN_CAPACITY and
// does nothing).
// after_count: launch_ccl_count ran just before (it initialised the run
// parents and the scan state); false for a relabel with grown run arrays.
cudaError_t launch_ccl_label(const CclArgs &a, int num_sms, cudaStream_t s, bool after_count = true);
struct RowSeg {               // one capture's image in a batch
  const uint32_t *mask;       // [T][F/32]
  const uint8_t *img;         // [T][F]
  int64_t T;
  int F, pad;
};
// After labelling one image: run g -> (box index, row, first, last column)
// for g < min(runs, cap); and the boundary bits of a [T][F/32] mask.
cudaError_t launch_runs_export(const CclArgs &a, int4 *out, int64_t cap, int num_sms, cudaStream_t s);
cudaError_t launch_boundary(const uint32_t *mask, int64_t T, int F, uint32_t *out, int num_sms,
                            cudaStream_t s);
// Batch labelling: a.T = rows of all captures; boxes come out ordered by
// capture then anchor, offs[c] (device, ncap + 1) = first box of capture c.
cudaError_t launch_ccl_label_batch(const CclArgs &a, const RowSeg *segs, const int64_t *row0,
                                   int ncap, int64_t *offs, int num_sms, cudaStream_t s);

}  // namespace rise
