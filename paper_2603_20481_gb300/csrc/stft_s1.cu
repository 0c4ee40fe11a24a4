// STFT kernels of radix schedule 1 (the radix-r pass first) for complex64
// input, in a translation unit of their own so that they compile in parallel
// with the schedule-0 kernels of stft.cu.
#include "stft_impl.cuh"

namespace rise {

cudaError_t launch_stft_s1(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s) {
  return launch_stft_in<float2, 1>(a, mode, num_sms, s);
}

cudaError_t launch_stft_batch_s1(int N, bool tma, StftMode mode, const StftArgs *segs, const StftItem *items,
                                 int n_items, int *counter, int num_sms, cudaStream_t s) {
  return launch_stft_batch_s<1>(N, tma, mode, segs, items, n_items, counter, num_sms, s);
}

void stft_s1_preload() { preload_stft_in<float2, 1>(); }

}  // namespace rise
