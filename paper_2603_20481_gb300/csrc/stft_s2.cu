// STFT kernels of radix schedule 2 (the frame split into two half-size
// transforms, FFT sizes 512 and 8192) for complex64 input, in a translation
// unit of their own so that they compile in parallel with the others.
#include "stft_impl.cuh"

namespace rise {

cudaError_t launch_stft_s2(const StftArgs &a, StftMode mode, int num_sms, cudaStream_t s) {
  return launch_stft_in<float2, 2>(a, mode, num_sms, s);
}

cudaError_t launch_stft_batch_s2(int N, bool tma, StftMode mode, const StftArgs *segs, const StftItem *items,
                                 int n_items, int *counter, int num_sms, cudaStream_t s) {
  return launch_stft_batch_s<2>(N, tma, mode, segs, items, n_items, counter, num_sms, s);
}

void stft_s2_preload() { preload_stft_in<float2, 2>(); }

}  // namespace rise
