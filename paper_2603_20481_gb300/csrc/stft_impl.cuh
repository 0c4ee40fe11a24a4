// Device code of the STFT stage, shared by the fc32 (stft.cu) and sc16
// (stft_sc16.cu) translation units; see stft.cu for the design.
#pragma once

#include <cmath>
#include <type_traits>
#include <vector>

#include "common.cuh"

namespace rise {
namespace {

constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }

// Radix schedule S of an N-point transform, N = 16^a * r (r in {1,2,4,8}):
// S = 0 runs the a radix-16 passes first and the radix-r pass last; S = 1
// runs the radix-r pass first (the same schedule as S = 0 when r = 1);
// S = 2 (r = 2 only) splits the frame into two N/2-point transforms that
// the two halves of the threads run side by side (see stft_frames_split).
constexpr bool sched_split(int N, int S) { return S == 2 && (ilog2c(N) % 4) == 1; }
constexpr bool sched_distinct(int N, int S) {
  return (S == 1 && (ilog2c(N) % 4) != 0) || sched_split(N, S);
}

template <int N, int S = 0>
struct Plan {
  static constexpr int LOG2N = ilog2c(N);
  static constexpr int NP16 = LOG2N / 4;
  static constexpr int RSMALL = 1 << (LOG2N % 4);
  static constexpr bool SMALL_FIRST = S == 1 && sched_distinct(N, S);
  static constexpr int NPASS = NP16 + (RSMALL > 1 ? 1 : 0);
  static constexpr int TPF = N / 16;                       // threads per frame
  static constexpr int FPB = TPF >= 256 ? 1 : 256 / TPF;   // frames per block step
  static constexpr int THREADS = TPF * FPB;
  static constexpr int SLOT = N + N / 16;                  // padded complex per frame
  static constexpr int radix(int i) {
    return SMALL_FIRST ? (i == 0 ? RSMALL : 16) : (i < NP16 ? 16 : RSMALL);
  }
  static constexpr int lprev(int i) { return i == 0 ? 1 : lprev(i - 1) * radix(i - 1); }
  static constexpr int mi(int i) { return N / lprev(i); }
  static constexpr int mp(int i) { return mi(i) / radix(i); }
  // twiddle tables [15][mp(i)] of passes 0..NPASS-2; pass 0's share of a
  // thread ((16 / r0) (r0 - 1) values) is kept in registers, the rest in smem
  static constexpr int tw_off(int i) { return i == 0 ? 0 : tw_off(i - 1) + 15 * mp(i - 1); }
  static constexpr int TW_TOTAL = tw_off(NPASS - 1);
  static constexpr int TW_REST = TW_TOTAL - tw_off(1);
  static constexpr int TW0 = 16 - 16 / radix(0);
};

__device__ __forceinline__ int padi(int i) { return i + (i >> 4); }
// padi(b + c) = padi(b) + padc(c) for a constant offset c that is a multiple
// of 16, or when b % 16 + c stays below 16 plus the multiple of 16 in c (the
// callers' cases): the offsets then fold into the load and store instructions
constexpr int padc(int c) { return c + (c >> 4); }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 w) {
  return make_float2(a.x * w.x - a.y * w.y, a.x * w.y + a.y * w.x);
}
__device__ __forceinline__ float2 mul_negi(float2 a) { return make_float2(a.y, -a.x); }  // a * (-i)

constexpr float kR = 0.70710678118654752440f;   // cos(pi/4)
constexpr float kC = 0.92387953251128675613f;   // cos(pi/8)
constexpr float kS = 0.38268343236508977173f;   // sin(pi/8)

// a * (r - i r)  (W_8^1 = W_16^2)
__device__ __forceinline__ float2 mul_w8_1(float2 a) { return make_float2(kR * (a.x + a.y), kR * (a.y - a.x)); }
// a * (-r - i r)  (W_8^3 = W_16^6)
__device__ __forceinline__ float2 mul_w8_3(float2 a) { return make_float2(kR * (a.y - a.x), -kR * (a.x + a.y)); }

// forward DFTs in place, natural order, X[k] = sum_n x[n] e^{-2 pi i n k / R}
__device__ __forceinline__ void dft2(float2 &a, float2 &b) {
  float2 t = a;
  a = cadd(t, b);
  b = csub(t, b);
}
// Packed (f32x2) complex add / subtract: one instruction each, the same
// rounding as two scalar adds (a - b is computed as b * -1 + a, exact product).
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ void dft4(float2 &a0, float2 &a1, float2 &a2, float2 &a3) {
  const float2 t0 = padd(a0, a2), t1 = psub(a0, a2), t2 = padd(a1, a3);
  // (a1 - a3) with its components swapped, so that multiplying by -i becomes a
  // lane-wise sign: -i (x + i y) = y - i x
  const float2 ts = make_float2(a1.y - a3.y, a1.x - a3.x);
  a0 = padd(t0, t2);
  a2 = psub(t0, t2);
  a1 = __ffma2_rn(ts, make_float2(1.0f, -1.0f), t1);
  a3 = __ffma2_rn(ts, make_float2(-1.0f, 1.0f), t1);
}
__device__ __forceinline__ void dft8(float2 *v) {
  // n = 2 n1 + n2, k = k1 + 4 k2
  dft4(v[0], v[2], v[4], v[6]);
  dft4(v[1], v[3], v[5], v[7]);
  float2 b1 = mul_w8_1(v[3]), b2 = mul_negi(v[5]), b3 = mul_w8_3(v[7]);
  float2 x0 = cadd(v[0], v[1]), x4 = csub(v[0], v[1]);
  float2 x1 = cadd(v[2], b1), x5 = csub(v[2], b1);
  float2 x2 = cadd(v[4], b2), x6 = csub(v[4], b2);
  float2 x3 = cadd(v[6], b3), x7 = csub(v[6], b3);
  v[0] = x0; v[1] = x1; v[2] = x2; v[3] = x3; v[4] = x4; v[5] = x5; v[6] = x6; v[7] = x7;
}
__device__ __forceinline__ void dft16(float2 *v) {
  // n = 4 n1 + n2, k = k1 + 4 k2: DFT4 over n1, twiddle W16^(n2 k1), DFT4 over n2
  dft4(v[0], v[4], v[8], v[12]);
  dft4(v[1], v[5], v[9], v[13]);
  dft4(v[2], v[6], v[10], v[14]);
  dft4(v[3], v[7], v[11], v[15]);
  // y[n2][k1] sits at v[4 k1 + n2]
  v[5] = cmul(v[5], make_float2(kC, -kS));    // n2=1,k1=1: W^1
  v[9] = mul_w8_1(v[9]);                      // n2=1,k1=2: W^2
  v[13] = cmul(v[13], make_float2(kS, -kC));  // n2=1,k1=3: W^3
  v[6] = mul_w8_1(v[6]);                      // n2=2,k1=1: W^2
  v[10] = mul_negi(v[10]);                    // n2=2,k1=2: W^4
  v[14] = mul_w8_3(v[14]);                    // n2=2,k1=3: W^6
  v[7] = cmul(v[7], make_float2(kS, -kC));    // n2=3,k1=1: W^3
  v[11] = mul_w8_3(v[11]);                    // n2=3,k1=2: W^6
  v[15] = cmul(v[15], make_float2(-kC, kS));  // n2=3,k1=3: W^9
  dft4(v[0], v[1], v[2], v[3]);
  dft4(v[4], v[5], v[6], v[7]);
  dft4(v[8], v[9], v[10], v[11]);
  dft4(v[12], v[13], v[14], v[15]);
  // X[k1 + 4 k2] is at v[4 k1 + k2]: transpose 4x4 to natural order
  float2 t;
  t = v[1]; v[1] = v[4]; v[4] = t;
  t = v[2]; v[2] = v[8]; v[8] = t;
  t = v[3]; v[3] = v[12]; v[12] = t;
  t = v[6]; v[6] = v[9]; v[9] = t;
  t = v[7]; v[7] = v[13]; v[13] = t;
  t = v[11]; v[11] = v[14]; v[14] = t;
}

template <int R>
__device__ __forceinline__ void dft_r(float2 *v) {
  if constexpr (R == 16) dft16(v);
  else if constexpr (R == 8) dft8(v);
  else if constexpr (R == 4) dft4(v[0], v[1], v[2], v[3]);
  else dft2(v[0], v[1]);
}

constexpr float kGuard = 3.0e-4f;   // |fast level coordinate error| is below 1e-4

// 8-bit level of power P: the count of edges[1..255] that P reaches.  A fast
// estimate from log2(P / anchor) is trusted away from level edges (the float
// to unsigned conversion floors and clamps to 0..255, NaN and -inf give 0);
// within kGuard of an edge the power is compared against the exact edge table.
__device__ __forceinline__ uint32_t level_of(float P, float inv_anchor, float c1, const float *edges) {
  const float v = fmaf(__log2f(P * inv_anchor), c1, 255.5f);
  uint32_t q = __float2uint_rd(fminf(v, 255.0f));
  if (fabsf(v - rintf(v)) < kGuard) {
    int qi = (int)q;
    for (int it = 0; it < 256 && qi < 255 && P >= edges[qi + 1]; ++it) ++qi;
    for (int it = 0; it < 256 && qi > 0 && P < edges[qi]; ++it) --qi;
    q = (uint32_t)qi;
  }
  return q;
}

// ---- TMA bulk copies and mbarriers (inline PTX) ---------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint64_t *b) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(b))
      : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t *b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: try_wait suspends for a hardware-defined interval per call,
// and gives up after `limit` calls (STFT_WAIT_LIMIT unless an option lowers it)
__device__ __forceinline__ bool mbar_wait(uint64_t *b, uint32_t parity, int limit) {
  for (int i = 0; i < limit; ++i)
    if (mbar_test(b, parity)) return true;
  return false;
}

// Pass I of the transform.  Butterfly d = tau + (N/16) s (s < 16/R) of
// sub-problem P = d / MP takes the R values P MI + a MP + j (j = d % MP).
// The first pass takes its values from registers loaded in sample order
// (v[i] = x[tau + (N/16) i]), so a radix-r first pass first regroups them
// per butterfly (v[s r + a] = x[d + a N/r]).
template <int N, int S, int I, bool FIRST>
__device__ __forceinline__ void fft_pass(float2 (&v)[16], const float2 *src, float2 *dst, int tau,
                                         const float2 (&tw0)[15], const float2 *twr) {
  using PL = Plan<N, S>;
  constexpr int R = PL::radix(I);
  constexpr int MI = PL::mi(I), MP = PL::mp(I);
  constexpr bool LAST = (I == PL::NPASS - 1);
  static_assert(R == 16 || I == 0 || LAST, "a radix below 16 runs first or last");
  if constexpr (!FIRST) {
    // the R values of a butterfly sit MP apart from b = P MI + j: when MP or
    // MI is a multiple of 16 (then j < MP divides 16), padi(b + a MP) =
    // padi(b) + padc(a MP)
    constexpr bool LIN = (MP % 16 == 0) || (MI % 16 == 0 && 16 % MP == 0);
#pragma unroll
    for (int s = 0; s < 16 / R; ++s) {
      const int d = tau + (N / 16) * s;
      const int P = d / MP, j = d % MP;
      if constexpr (LIN) {
        const float2 *sb = src + padi(P * MI + j);
#pragma unroll
        for (int a = 0; a < R; ++a) v[s * R + a] = sb[padc(a * MP)];
      } else {
#pragma unroll
        for (int a = 0; a < R; ++a) v[s * R + a] = src[padi(P * MI + a * MP + j)];
      }
    }
  } else if constexpr (R < 16) {
    float2 t[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) t[i] = v[i];
#pragma unroll
    for (int s = 0; s < 16 / R; ++s)
#pragma unroll
      for (int a = 0; a < R; ++a) v[s * R + a] = t[s + (16 / R) * a];
  }
#pragma unroll
  for (int s = 0; s < 16 / R; ++s) dft_r<R>(&v[s * R]);
  if constexpr (!LAST) {
    if constexpr (I == 0) {
      // W_N^(d p) of butterfly s, output p >= 1
#pragma unroll
      for (int s = 0; s < 16 / R; ++s)
#pragma unroll
        for (int p = 1; p < R; ++p) v[s * R + p] = cmul(v[s * R + p], tw0[s * (R - 1) + p - 1]);
    } else {
      const int j = tau % MP;
      const float2 *t = twr + (PL::tw_off(I) - PL::tw_off(1));
#pragma unroll
      for (int p = 1; p < 16; ++p) v[p] = cmul(v[p], t[(p - 1) * MP + j]);
    }
  }
}

// Stores pass I's outputs: output p of sub-problem P becomes element P MP + j
// of sub-problem P + lprev(I) p.  With radix 16 that is slot tau + (N/16) p
// for v[p]; a radix-r first pass stores v[s r + p] at p N/r + tau + (N/16) s.
template <int N, int S, int I>
__device__ __forceinline__ void store_pass(const float2 (&v)[16], float2 *dst, int tau) {
  using PL = Plan<N, S>;
  constexpr int NR = N / 16, R = PL::radix(I);
  static_assert(NR % 16 == 0, "slot offsets are multiples of 16");
  float2 *db = dst + padi(tau);   // every other offset is a multiple of 16
  if constexpr (R == 16) {
#pragma unroll
    for (int p = 0; p < 16; ++p) db[padc(p * NR)] = v[p];
  } else {
    static_assert(I == 0, "a radix below 16 stores only as the first pass");
#pragma unroll
    for (int s = 0; s < 16 / R; ++s)
#pragma unroll
      for (int p = 0; p < R; ++p) db[padc(p * (N / R) + NR * s)] = v[s * R + p];
  }
}

// Exchange buffers: two (ping-pong, one barrier per pass) unless they would
// not fit next to the input stages, then one (two barriers per pass).
// Twiddles of the passes after the first, kept in shared memory: those of
// Plan<N, S>, or for the split schedule those of Plan<N/2, 0>.
template <int N, int S>
constexpr int tw_rest() {
  if constexpr (sched_split(N, S)) return Plan<N / 2, 0>::TW_REST;
  else return Plan<N, S>::TW_REST;
}

// Exchange buffers: two (ping-pong, one barrier per pass) unless they would
// not fit next to the input stages, then one (two barriers per pass).  The
// split schedule's blocks of more than 256 threads run alone on an SM and
// may use up to the 227 KB a block can have.
template <int N, int S, bool TMA>
struct Smem {
  using PL = Plan<N, S>;
  static constexpr size_t STAGE = TMA ? (size_t)PL::FPB * N : 0;   // complex in the input stage
  static constexpr size_t XB = (size_t)PL::FPB * PL::SLOT;         // complex per exchange buffer
  static constexpr int TWR = tw_rest<N, S>();
  static constexpr size_t FIXED = (size_t)TWR * 8 + 260 * 4;
  static constexpr size_t LIMIT = (sched_split(N, S) && PL::THREADS > 256) ? 226 * 1024 : 113 * 1024;
  static constexpr int NXB = (STAGE * 8 + 2 * XB * 8 + FIXED <= LIMIT) ? 2 : 1;
  static constexpr size_t BYTES = STAGE * 8 + NXB * XB * 8 + FIXED;
  static constexpr int BLOCKS = (BYTES <= 113 * 1024 && PL::THREADS <= 256) ? 2 : 1;  // per SM
};

// Frames [f_begin, f_end) of one capture: window, FFT, epilogue.  Returns
// false (after recording ERR_INDEX) when a staged copy never arrived.
// Input samples: interleaved float (fc32) or 16-bit integer (sc16) I/Q; a
// 16-bit sample is (I, Q) * 2^-15 (exact in float), so full scale is 1.
__device__ __forceinline__ float2 to_f2(float2 s) { return s; }
__device__ __forceinline__ float2 to_f2(short2 s) {
  return make_float2((float)s.x * 3.0517578125e-05f, (float)s.y * 3.0517578125e-05f);
}

template <int N, int S, int MODE, bool TMA, typename IN>
__device__ __forceinline__ bool stft_frames_plain(const StftArgs &a, int64_t f_begin, int64_t f_end,
                                                  float2 *smem, float *red, uint64_t *bar) {
  const IN *iq = static_cast<const IN *>(a.iq);
  using PL = Plan<N, S>;
  using SM = Smem<N, S, TMA>;
  constexpr int TPF = PL::TPF, FPB = PL::FPB, SLOT = PL::SLOT, NPASS = PL::NPASS, NXB = SM::NXB;
  constexpr bool HOOK = MODE == STFT_POWER_HOOKED;                // test hooks (see StftMode)
  constexpr int EM = HOOK ? STFT_POWER : MODE;                     // the mode's work
  constexpr bool DO_MAX = (EM == STFT_MAX || EM == STFT_POWER);
  constexpr bool DO_Q = (EM == STFT_QUANT || EM == STFT_QUANT_POWER);
  constexpr bool DO_P = (EM == STFT_POWER || EM == STFT_QUANT_POWER);
  const int wait_limit = HOOK ? a.wait_limit : STFT_WAIT_LIMIT;
  float2 *stage = smem;                                   // [STAGE] (TMA only)
  float2 *xb0 = smem + SM::STAGE;
  float2 *xb1 = xb0 + (NXB == 2 ? SM::XB : 0);
  float2 *twr = xb0 + NXB * SM::XB;
  float *edges = reinterpret_cast<float *>(twr + SM::TWR);

  const int tid = threadIdx.x;
  const int slot = tid / TPF, tau = tid % TPF;
  const int64_t nsteps = (f_end - f_begin + FPB - 1) / FPB;

  auto step_bytes = [&](int64_t st) -> uint32_t {
    const int64_t t0 = f_begin + st * FPB;
    const int64_t nfr = (f_end - t0 < FPB) ? (f_end - t0) : (int64_t)FPB;
    return (uint32_t)(((nfr - 1) * a.hop + N) * sizeof(IN));
  };
  // one input stage: the copy for step st+1 is issued as soon as every thread
  // has its step-st samples in registers, and lands while step st computes
  auto issue = [&](int64_t st) {
    const int64_t t0 = f_begin + st * FPB;
    const uint32_t bytes = step_bytes(st);
    if (kChecked && (t0 < 0 || t0 * (int64_t)a.hop * (int64_t)sizeof(IN) + bytes > a.n * (int64_t)sizeof(IN))) {
      atomicOr(a.err, ERR_INDEX);   // checked build: a frame beyond the capture
      return;
    }
    if (HOOK && blockIdx.x == 0 && st == a.withhold_step) return;   // test only: this copy never comes
    mbar_expect_tx(bar, bytes);
    bulk_g2s(stage, iq + t0 * (int64_t)a.hop, bytes, bar);
  };
  if constexpr (TMA) {
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_fence_init();
      fence_proxy_async();   // earlier generic reads of the stage come first
      if (nsteps > 0) issue(0);
    }
  }

  float win[16];
  float2 tw0[15];
#pragma unroll
  for (int i = 0; i < 16; ++i) win[i] = __ldg(&a.win[i * (N / 16) + tau]);
  {
    // pass 0: W_N^(d p) of butterfly d = tau + (N/16) s, table [15][N / r0]
    constexpr int R0 = PL::radix(0), MP0 = PL::mp(0);
#pragma unroll
    for (int s = 0; s < 16 / R0; ++s)
#pragma unroll
      for (int p = 1; p < R0; ++p)
        tw0[s * (R0 - 1) + p - 1] = __ldg(&a.tw[(p - 1) * MP0 + tau + (N / 16) * s]);
#pragma unroll
    for (int i = PL::TW0; i < 15; ++i) tw0[i] = make_float2(0.f, 0.f);
  }
  for (int i = tid; i < PL::TW_REST; i += PL::THREADS) twr[i] = a.tw[PL::tw_off(1) + i];
  float inv_anchor = 0.f, c1 = 0.f;
  if constexpr (DO_Q) {
    for (int i = tid; i < 257; i += PL::THREADS) edges[i] = a.edges[i];
    inv_anchor = a.qconst[0];
    c1 = a.qconst[1];
  }
  __syncthreads();

  float run_max = 0.0f;
  int parity = 0;
  bool failed = false;
  for (int64_t st = 0; st < nsteps; ++st, parity ^= (NXB == 2 && (NPASS & 1) == 0)) {
    const int64_t t0 = f_begin + st * FPB;
    const int64_t t = t0 + slot;
    const bool valid = t < f_end;
    float2 v[16];
    if constexpr (TMA) {
      if (!mbar_wait(bar, (uint32_t)(st & 1), wait_limit)) failed = true;
      const IN *x = reinterpret_cast<const IN *>(stage) + (valid ? slot * a.hop : 0) + tau;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float2 s = valid ? to_f2(x[i * (N / 16)]) : make_float2(0.f, 0.f);
        v[i] = make_float2(s.x * win[i], s.y * win[i]);
      }
    } else {
      const bool ok = !kChecked || !valid || ck_index(t * (int64_t)a.hop + N - 1, a.n, a.err);
      const IN *x = iq + (valid && ok ? t * (int64_t)a.hop : 0) + tau;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float2 s = valid && ok ? to_f2(__ldg(x + i * (N / 16))) : make_float2(0.f, 0.f);
        v[i] = make_float2(s.x * win[i], s.y * win[i]);
      }
    }
    float2 *b0 = (parity ? xb1 : xb0) + slot * SLOT;
    float2 *b1 = (parity ? xb0 : xb1) + slot * SLOT;
    if constexpr (NXB == 1) __syncthreads();   // previous frame's last reads done
    fft_pass<N, S, 0, true>(v, nullptr, b0, tau, tw0, twr);
    store_pass<N, S, 0>(v, b0, tau);
    if (__syncthreads_or(failed)) {
      // a staged copy never arrived: record it, let copies in flight land, leave
      if (tid == 0) {
        atomicOr(a.err, ERR_COPY_WAIT);
        if constexpr (TMA) mbar_wait(bar, (uint32_t)(st & 1), wait_limit);
      }
      return false;
    }
    if constexpr (TMA) {
      if (tid == 0 && st + 1 < nsteps) {
        fence_proxy_async();   // generic reads of the stage are ordered before the async write
        issue(st + 1);
      }
    }
    if constexpr (NPASS >= 2) {
      fft_pass<N, S, 1, false>(v, b0, b1, tau, tw0, twr);
      if constexpr (NPASS >= 3) {
        if constexpr (NXB == 1) __syncthreads();
        store_pass<N, S, 1>(v, b1, tau);
        __syncthreads();
        fft_pass<N, S, 2, false>(v, b1, b0, tau, tw0, twr);
        if constexpr (NPASS >= 4) {
          if constexpr (NXB == 1) __syncthreads();
          store_pass<N, S, 2>(v, b0, tau);
          __syncthreads();
          fft_pass<N, S, 3, false>(v, b0, b1, tau, tw0, twr);
        }
      }
    }
    if (valid && ck_index(t, a.T, a.err)) {
      constexpr int R = PL::radix(NPASS - 1);
      uint8_t *qrow = DO_Q ? a.img + t * (int64_t)N : nullptr;
      float *prow = DO_P ? a.power + t * (int64_t)N : nullptr;
      // bin k = tau + C, C = (N/16) s + (N/R) p a multiple of N/16 > tau, so
      // its column (k + N/2) mod N is tau + (C + N/2) mod N
      if constexpr (DO_Q) qrow += tau;
      if constexpr (DO_P) prow += tau;
#pragma unroll
      for (int s = 0; s < 16 / R; ++s) {
#pragma unroll
        for (int p = 0; p < R; ++p) {
          const int fc = ((N / 16) * s + (N / R) * p + N / 2) & (N - 1);
          const float2 z = v[s * R + p];
          const float P = fmaf(z.x, z.x, z.y * z.y);
          if constexpr (DO_MAX) run_max = fmaxf(run_max, P);
          if constexpr (DO_P) prow[fc] = P;
          if constexpr (DO_Q) qrow[fc] = (uint8_t)level_of(P, inv_anchor, c1, edges);
        }
      }
    }
  }
  if constexpr (DO_MAX) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) run_max = fmaxf(run_max, __shfl_xor_sync(0xffffffffu, run_max, o));
    if ((tid & 31) == 0) red[tid >> 5] = run_max;
    __syncthreads();
    if (tid == 0) {
      float m = 0.f;
      for (int w = 0; w < PL::THREADS / 32; ++w) m = fmaxf(m, red[w]);
      atomicMax(a.max_bits, __float_as_uint(m));   // P >= 0: bit order = value order
    }
  }
  return true;
}

// W_32^a = exp(-2 pi i a / 32), a = 0..15
__device__ __forceinline__ float2 mul_w32(float2 v, int a) {
  constexpr float c1 = 0.98078528040323044913f, s1 = 0.19509032201612826785f;   // pi/16
  constexpr float c3 = 0.83146961230254523708f, s3 = 0.55557023301960222474f;   // 3 pi/16
  switch (a) {
    case 0: return v;
    case 1: return cmul(v, make_float2(c1, -s1));
    case 2: return cmul(v, make_float2(kC, -kS));
    case 3: return cmul(v, make_float2(c3, -s3));
    case 4: return mul_w8_1(v);
    case 5: return cmul(v, make_float2(s3, -c3));
    case 6: return cmul(v, make_float2(kS, -kC));
    case 7: return cmul(v, make_float2(s1, -c1));
    case 8: return mul_negi(v);
    case 9: return cmul(v, make_float2(-s1, -c1));
    case 10: return cmul(v, make_float2(-kS, -kC));
    case 11: return cmul(v, make_float2(-s3, -c3));
    case 12: return mul_w8_3(v);
    case 13: return cmul(v, make_float2(-c3, -s3));
    case 14: return cmul(v, make_float2(-kC, -kS));
    default: return cmul(v, make_float2(-c1, -s1));
  }
}

// Schedule 2 of N = 2M (M a power of 16).  The first decimation-in-frequency
// radix-2 step turns the windowed frame into two M-point transforms,
//   y0[m] = x[m] w[m] + x[m+M] w[m+M]            (bins X[2k]),
//   y1[m] = (x[m] w[m] - x[m+M] w[m+M]) W_N^m    (bins X[2k+1]),
// and the periodic Hann window has w[m+M] = 1 - w[m], so y0 = x2 + w (x1 - x2)
// and y1 = (w (x1 + x2) - x2) W_N^m with x1 = x[m], x2 = x[m+M], w = w[m].
// Threads [0, M/16) of a frame run the passes of Plan<M, 0> on y0, threads
// [M/16, N/16) on y1, each group in its own half of the exchange buffer.
// The radix-2 step is folded into the first pass, which reads the 32
// samples it combines from the stage (every sample is read by the two
// groups), so the frame crosses shared memory one time fewer than a
// radix-2 pass of its own would make it.  With M/16 a multiple of 32 the
// groups are whole warps and synchronise after the second pass on named
// barriers of their own.  W_N^m = W_N^j W_32^a for m = j + (M/16) a.
template <int N, int MODE, bool TMA, typename IN>
__device__ __forceinline__ bool stft_frames_split(const StftArgs &a, int64_t f_begin, int64_t f_end,
                                                  float2 *smem, float *red, uint64_t *bar) {
  constexpr int M = N / 2;
  using PM = Plan<M, 0>;
  using PL = Plan<N, 2>;
  using SM = Smem<N, 2, TMA>;
  constexpr int TPF = PL::TPF, FPB = PL::FPB, SLOT = PL::SLOT, NXB = SM::NXB;
  constexpr int HALF = M / 16, SLOTM = M + M / 16, NPM = PM::NPASS;
  constexpr bool WARP_GROUPS = HALF % 32 == 0;
  static_assert(PM::RSMALL == 1 && NPM >= 2 && NPM <= 3, "M is 256 or 4096");
  static_assert(SLOT == 2 * SLOTM, "two padded halves per frame");
  constexpr bool HOOK = MODE == STFT_POWER_HOOKED;                // test hooks (see StftMode)
  constexpr int EM = HOOK ? STFT_POWER : MODE;                     // the mode's work
  constexpr bool DO_MAX = (EM == STFT_MAX || EM == STFT_POWER);
  constexpr bool DO_Q = (EM == STFT_QUANT || EM == STFT_QUANT_POWER);
  constexpr bool DO_P = (EM == STFT_POWER || EM == STFT_QUANT_POWER);
  const int wait_limit = HOOK ? a.wait_limit : STFT_WAIT_LIMIT;
  const IN *iq = static_cast<const IN *>(a.iq);
  float2 *stage = smem;
  float2 *xb0 = smem + SM::STAGE;
  float2 *xb1 = xb0 + (NXB == 2 ? SM::XB : 0);
  float2 *twr = xb0 + NXB * SM::XB;
  float *edges = reinterpret_cast<float *>(twr + SM::TWR);

  const int tid = threadIdx.x;
  const int slot = tid / TPF, tau = tid % TPF;
  const int P = tau / HALF, j = tau % HALF;            // parity group and its thread
  const int64_t nsteps = (f_end - f_begin + FPB - 1) / FPB;

  auto step_bytes = [&](int64_t st) -> uint32_t {
    const int64_t t0 = f_begin + st * FPB;
    const int64_t nfr = (f_end - t0 < FPB) ? (f_end - t0) : (int64_t)FPB;
    return (uint32_t)(((nfr - 1) * a.hop + N) * sizeof(IN));
  };
  auto issue = [&](int64_t st) {
    const int64_t t0 = f_begin + st * FPB;
    const uint32_t bytes = step_bytes(st);
    if (kChecked && (t0 < 0 || t0 * (int64_t)a.hop * (int64_t)sizeof(IN) + bytes > a.n * (int64_t)sizeof(IN))) {
      atomicOr(a.err, ERR_INDEX);   // checked build: a frame beyond the capture
      return;
    }
    if (HOOK && blockIdx.x == 0 && st == a.withhold_step) return;   // test only: this copy never comes
    mbar_expect_tx(bar, bytes);
    bulk_g2s(stage, iq + t0 * (int64_t)a.hop, bytes, bar);
  };
  if constexpr (TMA) {
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_fence_init();
      fence_proxy_async();
      if (nsteps > 0) issue(0);
    }
  }
  // tables: Plan<M, 0>'s twiddles (first pass [15][HALF] in registers, the
  // rest in shared memory), then W_N^j for j < HALF; the window of size N
  float win[16];
  float2 tw0[15];
#pragma unroll
  for (int i = 0; i < 16; ++i) win[i] = __ldg(&a.win[j + HALF * i]);
#pragma unroll
  for (int p = 1; p < 16; ++p) tw0[p - 1] = __ldg(&a.tw[(p - 1) * HALF + j]);
  const float2 wN = P ? __ldg(&a.tw[PM::TW_TOTAL + j]) : make_float2(1.f, 0.f);
  for (int i = tid; i < PM::TW_REST; i += PL::THREADS) twr[i] = a.tw[PM::tw_off(1) + i];
  float inv_anchor = 0.f, c1 = 0.f;
  if constexpr (DO_Q) {
    for (int i = tid; i < 257; i += PL::THREADS) edges[i] = a.edges[i];
    inv_anchor = a.qconst[0];
    c1 = a.qconst[1];
  }
  __syncthreads();
  auto group_sync = [&]() {
    if constexpr (WARP_GROUPS)
      asm volatile("bar.sync %0, %1;" ::"r"(1 + 2 * slot + P), "r"(HALF) : "memory");
    else
      __syncthreads();
  };

  float run_max = 0.0f;
  int parity = 0;
  bool failed = false;
  // with two passes per half and two buffers, frames alternate buffers
  for (int64_t st = 0; st < nsteps; ++st, parity ^= (NXB == 2 && (NPM & 1) == 0)) {
    const int64_t t0 = f_begin + st * FPB;
    const int64_t t = t0 + slot;
    const bool valid = t < f_end;
    float2 v[16];
    {
      const IN *x;
      bool ok = valid;
      if constexpr (TMA) {
        if (!mbar_wait(bar, (uint32_t)(st & 1), wait_limit)) failed = true;
        x = reinterpret_cast<const IN *>(stage) + (valid ? slot * a.hop : 0) + j;
      } else {
        ok = valid && (!kChecked || ck_index(t * (int64_t)a.hop + N - 1, a.n, a.err));
        x = iq + (ok ? t * (int64_t)a.hop : 0) + j;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float2 x1 = make_float2(0.f, 0.f), x2 = x1;
        if (ok) {
          if constexpr (TMA) {
            x1 = to_f2(x[HALF * i]);
            x2 = to_f2(x[HALF * i + M]);
          } else {
            x1 = to_f2(__ldg(x + HALF * i));
            x2 = to_f2(__ldg(x + HALF * i + M));
          }
        }
        const float w = win[i];
        if (P == 0) {
          v[i] = make_float2(fmaf(w, x1.x - x2.x, x2.x), fmaf(w, x1.y - x2.y, x2.y));
        } else {
          const float2 y = make_float2(fmaf(w, x1.x + x2.x, -x2.x), fmaf(w, x1.y + x2.y, -x2.y));
          v[i] = mul_w32(cmul(y, wN), i);
        }
      }
    }
    float2 *b0 = (parity ? xb1 : xb0) + slot * SLOT + P * SLOTM;
    float2 *b1 = (parity ? xb0 : xb1) + slot * SLOT + P * SLOTM;
    if constexpr (NXB == 1) __syncthreads();   // the previous frame's last reads are done
    fft_pass<M, 0, 0, true>(v, nullptr, b0, j, tw0, twr);    // the values are already loaded
    store_pass<M, 0, 0>(v, b0, j);
    if (__syncthreads_or(failed)) {
      if (tid == 0) {
        atomicOr(a.err, ERR_COPY_WAIT);
        if constexpr (TMA) mbar_wait(bar, (uint32_t)(st & 1), wait_limit);
      }
      return false;
    }
    if constexpr (TMA) {
      if (tid == 0 && st + 1 < nsteps) {
        fence_proxy_async();
        issue(st + 1);
      }
    }
    fft_pass<M, 0, 1, false>(v, b0, b1, j, tw0, twr);
    if constexpr (NPM >= 3) {
      if constexpr (NXB == 1) group_sync();
      store_pass<M, 0, 1>(v, b1, j);
      group_sync();
      fft_pass<M, 0, 2, false>(v, b1, b0, j, tw0, twr);
    }
    if (valid && ck_index(t, a.T, a.err)) {
      uint8_t *qrow = DO_Q ? a.img + t * (int64_t)N : nullptr;
      float *prow = DO_P ? a.power + t * (int64_t)N : nullptr;
      // bin 2 (j + (M/16) p) + P of the frame (bin j + (M/16) p of the half):
      // column 2j + P + (2 (M/16) p + N/2) mod N, since 2j + P < 2 (M/16)
      if constexpr (DO_Q) qrow += 2 * j + P;
      if constexpr (DO_P) prow += 2 * j + P;
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        const int f = (2 * HALF * p + N / 2) & (N - 1);
        const float2 z = v[p];
        const float Pw = fmaf(z.x, z.x, z.y * z.y);
        if constexpr (DO_MAX) run_max = fmaxf(run_max, Pw);
        if constexpr (DO_P) prow[f] = Pw;
        if constexpr (DO_Q) qrow[f] = (uint8_t)level_of(Pw, inv_anchor, c1, edges);
      }
    }
  }
  if constexpr (DO_MAX) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) run_max = fmaxf(run_max, __shfl_xor_sync(0xffffffffu, run_max, o));
    if ((tid & 31) == 0) red[tid >> 5] = run_max;
    __syncthreads();
    if (tid == 0) {
      float m = 0.f;
      for (int w = 0; w < PL::THREADS / 32; ++w) m = fmaxf(m, red[w]);
      atomicMax(a.max_bits, __float_as_uint(m));
    }
  }
  return true;
}

// Named barrier over `count` threads that also ORs a predicate across them.
__device__ __forceinline__ bool bar_or(int id, int count, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, %2, %3, q;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)pred), "r"(id), "r"(count)
      : "memory");
  return r != 0;
}

// Schedule 2 with the two halves of the block decoupled (one frame per block
// step, each half whole warps: N = 8192).  The halves run the same steps as
// in stft_frames_split but share nothing except the input stage, and never
// meet at a block barrier inside the frame loop: after its first pass each
// half counts itself out of the stage (thread 0 of the half, on a shared
// counter), and the half that counts out second issues the copy of the next
// frame.  A half can then run up to most of a frame ahead of the other, so
// the butterflies of one half overlap the exchanges of the other.  The two
// roles (even bins; odd bins with the extra twist by W_N^m) swap halves
// every frame, so both halves carry the same work over two frames.
template <int N, int MODE, bool TMA, typename IN>
__device__ __forceinline__ bool stft_frames_split_async(const StftArgs &a, int64_t f_begin, int64_t f_end,
                                                        float2 *smem, float *red, uint64_t *bar) {
  constexpr int M = N / 2;
  using PM = Plan<M, 0>;
  using PL = Plan<N, 2>;
  using SM = Smem<N, 2, TMA>;
  constexpr int HALF = M / 16, SLOTM = M + M / 16, NPM = PM::NPASS;
  static_assert(PL::FPB == 1 && HALF % 32 == 0 && NPM == 3 && SM::NXB == 2 && PL::SLOT == 2 * SLOTM,
                "one frame per step, whole-warp halves, three passes per half, two exchange buffers");
  constexpr bool HOOK = MODE == STFT_POWER_HOOKED;                // test hooks (see StftMode)
  constexpr int EM = HOOK ? STFT_POWER : MODE;                     // the mode's work
  constexpr bool DO_MAX = (EM == STFT_MAX || EM == STFT_POWER);
  constexpr bool DO_Q = (EM == STFT_QUANT || EM == STFT_QUANT_POWER);
  constexpr bool DO_P = (EM == STFT_POWER || EM == STFT_QUANT_POWER);
  const int wait_limit = HOOK ? a.wait_limit : STFT_WAIT_LIMIT;
  __shared__ int s_out, s_issued, s_fail;
  const IN *iq = static_cast<const IN *>(a.iq);
  float2 *stage = smem;
  float2 *xb0 = smem + SM::STAGE;
  float2 *xb1 = xb0 + SM::XB;
  float2 *twr = xb0 + 2 * SM::XB;
  float *edges = reinterpret_cast<float *>(twr + SM::TWR);

  const int tid = threadIdx.x;
  const int h = tid / HALF, j = tid % HALF;             // half of the block and its thread
  const int64_t nsteps = f_end - f_begin;
  auto issue = [&](int64_t st) -> bool {   // true when the copy is in flight
    const int64_t t = f_begin + st;
    constexpr uint32_t bytes = (uint32_t)(N * sizeof(IN));
    if (kChecked && (t < 0 || t * (int64_t)a.hop * (int64_t)sizeof(IN) + bytes > a.n * (int64_t)sizeof(IN))) {
      atomicOr(a.err, ERR_INDEX);   // checked build: a frame beyond the capture
      return false;
    }
    if (HOOK && blockIdx.x == 0 && st == a.withhold_step) return false;   // test only: this copy never comes
    mbar_expect_tx(bar, bytes);
    bulk_g2s(stage, iq + t * (int64_t)a.hop, bytes, bar);
    return true;
  };
  if (tid == 0) {
    s_out = 0;
    s_issued = 0;
    s_fail = 0;
    if constexpr (TMA) {
      mbar_init(bar, 1);
      mbar_fence_init();
      fence_proxy_async();
      if (nsteps > 0 && issue(0)) s_issued = 1;
    }
  }
  float win[16];
  float2 tw0[15];
#pragma unroll
  for (int i = 0; i < 16; ++i) win[i] = __ldg(&a.win[j + HALF * i]);
#pragma unroll
  for (int p = 1; p < 16; ++p) tw0[p - 1] = __ldg(&a.tw[(p - 1) * HALF + j]);
  const float2 wN = __ldg(&a.tw[PM::TW_TOTAL + j]);
  for (int i = tid; i < PM::TW_REST; i += PL::THREADS) twr[i] = a.tw[PM::tw_off(1) + i];
  float inv_anchor = 0.f, c1 = 0.f;
  if constexpr (DO_Q) {
    for (int i = tid; i < 257; i += PL::THREADS) edges[i] = a.edges[i];
    inv_anchor = a.qconst[0];
    c1 = a.qconst[1];
  }
  __syncthreads();
  const int bar_id = 1 + h;
  float2 *b0 = xb0 + h * SLOTM;
  float2 *b1 = xb1 + h * SLOTM;

  float run_max = 0.0f;
  for (int64_t st = 0; st < nsteps; ++st) {
    const int64_t t = f_begin + st;
    const int P = h ^ (int)(st & 1);                     // this frame's role: even or odd bins
    bool failed = false;
    float2 v[16];
    {
      const IN *x;
      bool ok = true;
      if constexpr (TMA) {
        if (!mbar_wait(bar, (uint32_t)(st & 1), wait_limit)) failed = true;
        x = reinterpret_cast<const IN *>(stage) + j;
      } else {
        ok = !kChecked || ck_index(t * (int64_t)a.hop + N - 1, a.n, a.err);
        x = iq + (ok ? t * (int64_t)a.hop : 0) + j;
      }
      if (P == 0) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float2 x1 = make_float2(0.f, 0.f), x2 = x1;
          if (ok) {
            if constexpr (TMA) {
              x1 = to_f2(x[HALF * i]);
              x2 = to_f2(x[HALF * i + M]);
            } else {
              x1 = to_f2(__ldg(x + HALF * i));
              x2 = to_f2(__ldg(x + HALF * i + M));
            }
          }
          const float w = win[i];
          v[i] = make_float2(fmaf(w, x1.x - x2.x, x2.x), fmaf(w, x1.y - x2.y, x2.y));
        }
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          float2 x1 = make_float2(0.f, 0.f), x2 = x1;
          if (ok) {
            if constexpr (TMA) {
              x1 = to_f2(x[HALF * i]);
              x2 = to_f2(x[HALF * i + M]);
            } else {
              x1 = to_f2(__ldg(x + HALF * i));
              x2 = to_f2(__ldg(x + HALF * i + M));
            }
          }
          const float w = win[i];
          const float2 y = make_float2(fmaf(w, x1.x + x2.x, -x2.x), fmaf(w, x1.y + x2.y, -x2.y));
          v[i] = mul_w32(cmul(y, wN), i);
        }
      }
    }
    fft_pass<M, 0, 0, true>(v, nullptr, b0, j, tw0, twr);   // the values are already loaded
    store_pass<M, 0, 0>(v, b0, j);
    // the half's stage reads and first-pass stores are done; a wait that ran
    // out in any thread of the half ends the half's loop
    if (bar_or(bar_id, HALF, failed)) {
      if (j == 0) {
        s_fail = 1;
        atomicOr(a.err, ERR_COPY_WAIT);
      }
      break;
    }
    if constexpr (TMA) {
      if (j == 0) {
        __threadfence_block();
        const int before = atomicAdd(&s_out, 1);
        __threadfence_block();
        if (before == 2 * (int)st + 1 && st + 1 < nsteps) {   // both halves are out of the stage
          fence_proxy_async();
          if (issue(st + 1)) s_issued = (int)st + 2;
        }
      }
    }
    fft_pass<M, 0, 1, false>(v, b0, b1, j, tw0, twr);
    store_pass<M, 0, 1>(v, b1, j);
    asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(HALF) : "memory");
    fft_pass<M, 0, 2, false>(v, b1, b0, j, tw0, twr);
    if (ck_index(t, a.T, a.err)) {
      uint8_t *qrow = DO_Q ? a.img + t * (int64_t)N : nullptr;
      float *prow = DO_P ? a.power + t * (int64_t)N : nullptr;
      // bin 2 (j + (M/16) p) + P of the frame: column 2j + P + (2 (M/16) p + N/2) mod N
      if constexpr (DO_Q) qrow += 2 * j + P;
      if constexpr (DO_P) prow += 2 * j + P;
#pragma unroll
      for (int p = 0; p < 16; ++p) {
        const int f = (2 * HALF * p + N / 2) & (N - 1);
        const float2 z = v[p];
        const float Pw = fmaf(z.x, z.x, z.y * z.y);
        if constexpr (DO_MAX) run_max = fmaxf(run_max, Pw);
        if constexpr (DO_P) prow[f] = Pw;
        if constexpr (DO_Q) qrow[f] = (uint8_t)level_of(Pw, inv_anchor, c1, edges);
      }
    }
  }
  __syncthreads();
  const bool failed = s_fail != 0;
  // after a wait ran out, the last copy issued may still be in flight: wait
  // (bounded) for it before the block lets go of its shared memory
  if (TMA && failed && tid == 0 && s_issued > 0) mbar_wait(bar, (uint32_t)((s_issued - 1) & 1), wait_limit);
  if constexpr (DO_MAX) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) run_max = fmaxf(run_max, __shfl_xor_sync(0xffffffffu, run_max, o));
    if ((tid & 31) == 0) red[tid >> 5] = run_max;
    __syncthreads();
    if (tid == 0) {
      float m = 0.f;
      for (int w = 0; w < PL::THREADS / 32; ++w) m = fmaxf(m, red[w]);
      atomicMax(a.max_bits, __float_as_uint(m));
    }
  }
  return !failed;
}

template <int N, int S, int MODE, bool TMA, typename IN>
__device__ __forceinline__ bool stft_frames(const StftArgs &a, int64_t f_begin, int64_t f_end,
                                            float2 *smem, float *red, uint64_t *bar) {
  if constexpr (sched_split(N, S) && N / 32 >= 256)
    return stft_frames_split_async<N, MODE, TMA, IN>(a, f_begin, f_end, smem, red, bar);
  else if constexpr (sched_split(N, S)) return stft_frames_split<N, MODE, TMA, IN>(a, f_begin, f_end, smem, red, bar);
  else return stft_frames_plain<N, S, MODE, TMA, IN>(a, f_begin, f_end, smem, red, bar);
}

template <int N, int S, int MODE, bool TMA, typename IN>
__global__ void __launch_bounds__(Plan<N, S>::THREADS, (Smem<N, S, TMA>::BLOCKS))
stft_kernel(StftArgs a, int64_t frames_per_block) {
  extern __shared__ __align__(128) float2 smem[];
  __shared__ float red[32];
  __shared__ __align__(8) uint64_t bar;
  const int64_t f_begin = (int64_t)blockIdx.x * frames_per_block;
  const int64_t f_end = min(a.T, f_begin + frames_per_block);
  stft_frames<N, S, MODE, TMA, IN>(a, f_begin, f_end, smem, red, &bar);
}

// Many captures of one FFT size in one launch: a persistent grid whose
// blocks take (capture, frame range) items from a shared counter until none
// are left, so uneven captures balance across the SMs.  Items come sorted by
// size, largest first.
template <int N, int S, int MODE, bool TMA>
__global__ void __launch_bounds__(Plan<N, S>::THREADS, (Smem<N, S, TMA>::BLOCKS))
stft_batch_kernel(const StftArgs *segs, const StftItem *items, int n_items, int *counter) {
  extern __shared__ __align__(128) float2 smem[];
  __shared__ float red[32];
  __shared__ __align__(8) uint64_t bar;
  __shared__ StftArgs sa;
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = atomicAdd(counter, 1);
      s_item = it;
      if (it < n_items) sa = segs[items[it].seg];
    }
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) return;
    const StftItem item = items[it];
    if (kChecked && (item.f0 < 0 || item.f1 > sa.T || item.f0 > item.f1)) {
      if (threadIdx.x == 0) atomicOr(sa.err, ERR_INDEX);   // checked build: frames of the capture
      __syncthreads();
      continue;
    }
    const bool ok = stft_frames<N, S, MODE, TMA, float2>(sa, item.f0, item.f1, smem, red, &bar);
    if (!ok) return;   // uniform over the block
    __syncthreads();   // every wait on the barrier and every read of sa is done
    if (TMA && threadIdx.x == 0) mbar_inval(&bar);
  }
}

template <int N, int S, int MODE, bool TMA, typename IN>
cudaError_t launch_n(const StftArgs &a, int num_sms, cudaStream_t s) {
  using PL = Plan<N, S>;
  auto kern = stft_kernel<N, S, MODE, TMA, IN>;
  const size_t sm = Smem<N, S, TMA>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, PL::THREADS, sm);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  const int64_t steps = (a.T + PL::FPB - 1) / PL::FPB;
  int64_t grid = std::min<int64_t>(steps, (int64_t)num_sms * occ);
  if (grid < 1) grid = 1;
  int64_t per = (steps + grid - 1) / grid * PL::FPB;
  grid = (a.T + per - 1) / per;
  kern<<<(unsigned)grid, PL::THREADS, sm, s>>>(a, per);
  count_launches(1);
  return cudaGetLastError();
}

template <int N, int S, bool TMA, typename IN>
cudaError_t launch_mode(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s) {
  switch (mode) {
    case STFT_MAX: return launch_n<N, S, STFT_MAX, TMA, IN>(a, num_sms, s);
    case STFT_QUANT: return launch_n<N, S, STFT_QUANT, TMA, IN>(a, num_sms, s);
    case STFT_POWER: return launch_n<N, S, STFT_POWER, TMA, IN>(a, num_sms, s);
    case STFT_QUANT_POWER: return launch_n<N, S, STFT_QUANT_POWER, TMA, IN>(a, num_sms, s);
    case STFT_POWER_HOOKED: return launch_n<N, S, STFT_POWER_HOOKED, TMA, IN>(a, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

template <int N, int S, int MODE, bool TMA>
cudaError_t launch_batch_n(const StftArgs *segs, const StftItem *items, int n_items, int *counter,
                           int num_sms, cudaStream_t s) {
  using PL = Plan<N, S>;
  auto kern = stft_batch_kernel<N, S, MODE, TMA>;
  const size_t sm = Smem<N, S, TMA>::BYTES;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  int occ = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, PL::THREADS, sm);
  if (e != cudaSuccess) return e;
  if (occ < 1) occ = 1;
  const int grid = (int)std::min<int64_t>(n_items, (int64_t)num_sms * occ);
  if (grid < 1) return cudaSuccess;
  kern<<<grid, PL::THREADS, sm, s>>>(segs, items, n_items, counter);
  count_launches(1);
  return cudaGetLastError();
}

template <int N, int S, bool TMA>
cudaError_t batch_mode(StftMode mode, const StftArgs *segs, const StftItem *items, int n_items,
                       int *counter, int num_sms, cudaStream_t s) {
  switch (mode) {
    case STFT_MAX: return launch_batch_n<N, S, STFT_MAX, TMA>(segs, items, n_items, counter, num_sms, s);
    case STFT_QUANT: return launch_batch_n<N, S, STFT_QUANT, TMA>(segs, items, n_items, counter, num_sms, s);
    case STFT_POWER: return launch_batch_n<N, S, STFT_POWER, TMA>(segs, items, n_items, counter, num_sms, s);
    case STFT_QUANT_POWER:
      return launch_batch_n<N, S, STFT_QUANT_POWER, TMA>(segs, items, n_items, counter, num_sms, s);
    case STFT_POWER_HOOKED:
      return launch_batch_n<N, S, STFT_POWER_HOOKED, TMA>(segs, items, n_items, counter, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

template <int N, int S>
cudaError_t batch_size(bool tma, StftMode mode, const StftArgs *segs, const StftItem *items,
                       int n_items, int *counter, int num_sms, cudaStream_t s) {
  return tma ? batch_mode<N, S, true>(mode, segs, items, n_items, counter, num_sms, s)
             : batch_mode<N, S, false>(mode, segs, items, n_items, counter, num_sms, s);
}

template <int N, int S, typename IN>
cudaError_t launch_size(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s) {
  // staged input needs every copy 16-byte aligned: hop * sample size a
  // multiple of 16 bytes and a 16-byte aligned base
  const bool tma = ((int64_t)a.hop * (int64_t)sizeof(IN)) % 16 == 0 &&
                   ((reinterpret_cast<uintptr_t>(a.iq) & 15) == 0);
  return tma ? launch_mode<N, S, true, IN>(a, mode, num_sms, s) : launch_mode<N, S, false, IN>(a, mode, num_sms, s);
}

template <int N, int S, typename IN, bool TMA>
void preload_stft_nt() {
  preload_kernel(stft_kernel<N, S, STFT_MAX, TMA, IN>);
  preload_kernel(stft_kernel<N, S, STFT_QUANT, TMA, IN>);
  preload_kernel(stft_kernel<N, S, STFT_POWER, TMA, IN>);
  preload_kernel(stft_kernel<N, S, STFT_QUANT_POWER, TMA, IN>);
  preload_kernel(stft_kernel<N, S, STFT_POWER_HOOKED, TMA, IN>);
  if constexpr (std::is_same<IN, float2>::value) {
    preload_kernel(stft_batch_kernel<N, S, STFT_MAX, TMA>);
    preload_kernel(stft_batch_kernel<N, S, STFT_QUANT, TMA>);
    preload_kernel(stft_batch_kernel<N, S, STFT_POWER, TMA>);
    preload_kernel(stft_batch_kernel<N, S, STFT_QUANT_POWER, TMA>);
    preload_kernel(stft_batch_kernel<N, S, STFT_POWER_HOOKED, TMA>);
  }
}
template <int N, int S, typename IN>
void preload_stft_n() {
  if constexpr (S == 0 || sched_distinct(N, S)) {
    preload_stft_nt<N, S, IN, false>();
    preload_stft_nt<N, S, IN, true>();
  }
}
template <typename IN, int S>
void preload_stft_in() {
  preload_stft_n<256, S, IN>();
  preload_stft_n<512, S, IN>();
  preload_stft_n<1024, S, IN>();
  preload_stft_n<2048, S, IN>();
  preload_stft_n<4096, S, IN>();
  preload_stft_n<8192, S, IN>();
}

// The launch for the input type IN and schedule S, by FFT size; a size
// whose schedule S equals schedule 0 runs schedule 0's kernels.
template <int N, int S, typename IN>
cudaError_t launch_sized(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s) {
  if constexpr (S == 0 || sched_distinct(N, S)) return launch_size<N, S, IN>(a, mode, num_sms, s);
  else return cudaErrorInvalidValue;
}
template <typename IN, int S>
cudaError_t launch_stft_in(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s) {
  switch (a.N) {
    case 256: return launch_sized<256, S, IN>(a, mode, num_sms, s);
    case 512: return launch_sized<512, S, IN>(a, mode, num_sms, s);
    case 1024: return launch_sized<1024, S, IN>(a, mode, num_sms, s);
    case 2048: return launch_sized<2048, S, IN>(a, mode, num_sms, s);
    case 4096: return launch_sized<4096, S, IN>(a, mode, num_sms, s);
    case 8192: return launch_sized<8192, S, IN>(a, mode, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

// The batch launch of schedule S, by FFT size.
template <int N, int S>
cudaError_t batch_sized(bool tma, StftMode mode, const StftArgs *segs, const StftItem *items, int n_items,
                        int *counter, int num_sms, cudaStream_t s) {
  if constexpr (S == 0 || sched_distinct(N, S)) return batch_size<N, S>(tma, mode, segs, items, n_items, counter, num_sms, s);
  else return cudaErrorInvalidValue;
}
template <int S>
cudaError_t launch_stft_batch_s(int N, bool tma, StftMode mode, const StftArgs *segs, const StftItem *items,
                                int n_items, int *counter, int num_sms, cudaStream_t s) {
  switch (N) {
    case 256: return batch_sized<256, S>(tma, mode, segs, items, n_items, counter, num_sms, s);
    case 512: return batch_sized<512, S>(tma, mode, segs, items, n_items, counter, num_sms, s);
    case 1024: return batch_sized<1024, S>(tma, mode, segs, items, n_items, counter, num_sms, s);
    case 2048: return batch_sized<2048, S>(tma, mode, segs, items, n_items, counter, num_sms, s);
    case 4096: return batch_sized<4096, S>(tma, mode, segs, items, n_items, counter, num_sms, s);
    case 8192: return batch_sized<8192, S>(tma, mode, segs, items, n_items, counter, num_sms, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace rise
