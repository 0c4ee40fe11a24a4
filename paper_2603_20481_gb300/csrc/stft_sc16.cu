// STFT launches for 16-bit integer I/Q (sc16) input, in a translation unit of
// their own so that the two input types compile in parallel; every radix
// schedule, so that 16-bit input gives the bits complex64 input gives.
#include "stft_impl.cuh"

namespace rise {

cudaError_t launch_stft_sc16(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s) {
  if (stft_sched_distinct(a.N, a.sched))
    return a.sched == 1 ? launch_stft_in<short2, 1>(a, mode, num_sms, s) : launch_stft_in<short2, 2>(a, mode, num_sms, s);
  return launch_stft_in<short2, 0>(a, mode, num_sms, s);
}

void stft_sc16_preload() {
  preload_stft_in<short2, 0>();
  preload_stft_in<short2, 1>();
  preload_stft_in<short2, 2>();
}

}  // namespace rise
