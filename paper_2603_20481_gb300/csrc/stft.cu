// Windowed STFT, |X|^2 and the 8-bit level image (RISE Sec. III-A-1, the TF
// plot; the 8-bit image is the library's reading, anchored on a top power).
//
// One frame of N complex samples is transformed by N/16 threads, each
// holding 16 values in registers.  N = 16^a * r (r in {1,2,4,8}): a radix-16
// passes in registers (each thread one 16-point DFT) plus one pass of radix
// r (each thread 16/r DFTs), the radix-r pass last (schedule 0) or first
// (schedule 1, compiled in stft_s1.cu); for r = 2, schedule 2 (stft_s2.cu)
// splits the frame into two N/2-point transforms instead (see
// stft_frames_split).  The batch tuner times them.  Between
// passes the data cross shared memory once, in a layout padded by one slot
// per 16 so that every 16-lane group
// hits 16 distinct 8-byte bank pairs.  The decomposition is the
// decimation-in-frequency four-step recursion: pass i splits the current
// sub-transform of length M into R interleaved pieces, DFTs over the slow
// index, applies the twiddle W_M^(j p) and hands output digit p to the
// next sub-problem, so the last pass leaves X[k] in natural order.
//
// Epilogues: MAX (running max of |X|^2 for the anchor), QUANT (8-bit level
// per bin, stored with DC in column N/2), POWER (float |X|^2 stored plus the
// running max) and QUANT_POWER (both).
#include <vector>

#include "stft_impl.cuh"

namespace rise {
namespace {

// Edges of the 8-bit levels: level j >= 1 is reached at power
// anchor * 10^((j - 255.5) * level_db / 10); ratio[j] holds the power of ten
// (FP64, computed on the host), edges[j] is the smallest float not below
// anchor * ratio[j], so "P >= edges[j]" is the exact comparison for a float
// P.  edges[0] = 0, edges[256] = +inf.
__device__ __forceinline__ void levels_body(const uint32_t *max_bits, double hi_power, int use_fixed,
                                            const double *ratio, double level_db, float *edges,
                                            float *qconst) {
  const double M = use_fixed ? hi_power : (double)__uint_as_float(*max_bits);
  const int j = threadIdx.x;
  if (j == 0) {
    edges[0] = 0.0f;
  } else if (j == 256) {
    edges[256] = __int_as_float(0x7f800000);
  } else if (j < 256) {
    edges[j] = M > 0.0 ? __double2float_ru(M * ratio[j]) : __int_as_float(0x7f800000);
  }
  if (j == 0) {
    qconst[0] = M > 0.0 ? (float)(1.0 / M) : 0.0f;
    qconst[1] = (float)(3.0102999566398119521 / level_db);   // 10 log10(2) / level_db
  }
}

__global__ void levels_kernel(const uint32_t *max_bits, double hi_power, int use_fixed,
                              const double *ratio, double level_db, float *edges, float *qconst) {
  levels_body(max_bits, hi_power, use_fixed, ratio, level_db, edges, qconst);
}

// one block per capture of a batch
__global__ void levels_batch_kernel(CapSmall *cs, double hi_power, int use_fixed, const double *ratio,
                                    double level_db) {
  CapSmall &c = cs[blockIdx.x];
  levels_body(&c.max_bits, hi_power, use_fixed, ratio, level_db, c.edges, c.qconst);
}

}  // namespace

// Host mirror of Plan<N, S> (runtime) for table construction: the radix of
// every pass.
static std::vector<int> host_radices(int N, int S) {
  int l = 0;
  while ((1 << l) < N) ++l;
  const int np16 = l / 4, rs = 1 << (l % 4);
  std::vector<int> r;
  if (rs > 1 && S == 1) r.push_back(rs);
  for (int i = 0; i < np16; ++i) r.push_back(16);
  if (rs > 1 && S != 1) r.push_back(rs);
  return r;
}

// Schedule 2 (N = 2M, M a power of 16): the tables of schedule 0 of size M,
// then W_N^j for j < M/16, then the window of size N.
static bool host_split(int N, int S) {
  int l = 0;
  while ((1 << l) < N) ++l;
  return S == 2 && l % 4 == 1;
}

static size_t twiddle_complex(int N, int S) {
  const std::vector<int> rad = host_radices(N, S);
  size_t tw = 0;
  int L = 1;
  for (size_t i = 0; i + 1 < rad.size(); ++i) {
    const int R = rad[i];
    int Mi = N / L, Mp = Mi / R;
    tw += 15 * (size_t)Mp;
    L *= R;
  }
  return tw;
}

size_t stft_table_floats(int N, int S) {
  if (host_split(N, S)) return 2 * (twiddle_complex(N / 2, 0) + (size_t)N / 32) + N;
  const std::vector<int> rad = host_radices(N, S);
  size_t tw = 0;
  int L = 1;
  for (size_t i = 0; i + 1 < rad.size(); ++i) {
    const int R = rad[i];
    int Mi = N / L, Mp = Mi / R;
    tw += 15 * (size_t)Mp;
    L *= R;
  }
  return 2 * tw + N;  // complex twiddles + window
}

void stft_fill_tables(int N, int S, float2 *tw, float *win) {
  const double two_pi = 6.283185307179586476925286766559;
  if (host_split(N, S)) {
    const int M = N / 2;
    std::vector<float> half(stft_table_floats(M, 0));
    const size_t ntw = twiddle_complex(M, 0);
    stft_fill_tables(M, 0, tw, half.data() + 2 * ntw);   // M's twiddles; its window is not used
    for (int j = 0; j < M / 16; ++j) {
      const double ang = two_pi * (double)j / (double)N;   // W_N^j
      tw[ntw + j] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    for (int m = 0; m < N; ++m) win[m] = (float)(0.5 - 0.5 * std::cos(two_pi * (double)m / (double)N));
    return;
  }
  const std::vector<int> rad = host_radices(N, S);
  size_t off = 0;
  int L = 1;
  for (size_t i = 0; i + 1 < rad.size(); ++i) {
    const int R = rad[i];
    int Mi = N / L, Mp = Mi / R;
    for (int p = 1; p < 16; ++p)
      for (int j = 0; j < Mp; ++j) {
        long long e = ((long long)j * p) % Mi;   // W_Mi^(j p)
        double ang = two_pi * (double)e / (double)Mi;
        tw[off + (size_t)(p - 1) * Mp + j] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
      }
    off += 15 * (size_t)Mp;
    L *= R;
  }
  for (int m = 0; m < N; ++m) win[m] = (float)(0.5 - 0.5 * std::cos(two_pi * (double)m / (double)N));
}

void stft_preload() {
  preload_stft_in<float2, 0>();
  preload_kernel(levels_kernel);
  preload_kernel(levels_batch_kernel);
}

int stft_default_sched(int N) {
  if (N == 8192) return 2;
  return stft_sched_distinct(N, 1) ? 1 : 0;
}

bool stft_sched_distinct(int N, int S) {
  int l = 0;
  while ((1 << l) < N) ++l;
  return (S == 1 && l % 4 != 0) || (S == 2 && l % 4 == 1);
}

// The kernels of schedules 1 and 2 (where they differ from schedule 0) live
// in stft_s1.cu and stft_s2.cu, the 16-bit input's in stft_sc16.cu.
cudaError_t launch_stft(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s) {
  if (a.fmt == IQ_SC16) return launch_stft_sc16(a, mode, num_sms, s);
  if (stft_sched_distinct(a.N, a.sched)) {
    if (a.sched == 1) return launch_stft_s1(a, mode, num_sms, s);
    return launch_stft_s2(a, mode, num_sms, s);
  }
  return launch_stft_in<float2, 0>(a, mode, num_sms, s);
}

cudaError_t launch_stft_batch(int N, int sched, bool tma, StftMode mode, const StftArgs *segs,
                              const StftItem *items, int n_items, int *counter, int num_sms,
                              cudaStream_t s) {
  if (stft_sched_distinct(N, sched)) {
    if (sched == 1) return launch_stft_batch_s1(N, tma, mode, segs, items, n_items, counter, num_sms, s);
    return launch_stft_batch_s2(N, tma, mode, segs, items, n_items, counter, num_sms, s);
  }
  return launch_stft_batch_s<0>(N, tma, mode, segs, items, n_items, counter, num_sms, s);
}

int stft_frames_per_step(int N) {
  switch (N) {
    case 256: return Plan<256>::FPB;
    case 512: return Plan<512>::FPB;
    case 1024: return Plan<1024>::FPB;
    case 2048: return Plan<2048>::FPB;
    case 4096: return Plan<4096>::FPB;
    case 8192: return Plan<8192>::FPB;
  }
  return 1;
}

cudaError_t launch_levels_batch(CapSmall *cs, int ncap, double hi_power, int use_fixed,
                                const double *ratio, double level_db, cudaStream_t s) {
  levels_batch_kernel<<<ncap, 288, 0, s>>>(cs, hi_power, use_fixed, ratio, level_db);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_levels(const uint32_t *max_bits, double hi_power, int use_fixed,
                          const double *ratio, double level_db, float *edges, float *qconst,
                          cudaStream_t s) {
  levels_kernel<<<1, 288, 0, s>>>(max_bits, hi_power, use_fixed, ratio, level_db, edges, qconst);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace rise
