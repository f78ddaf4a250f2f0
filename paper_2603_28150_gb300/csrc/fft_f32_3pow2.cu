// FFT stage launchers, float precision, transform lengths 3 * 2^k in [24, 768].
#include "fft_kernels.cuh"

namespace pat {
PAT_FFT_INSTANTIATE(float, 24)
PAT_FFT_INSTANTIATE(float, 48)
PAT_FFT_INSTANTIATE(float, 96)
PAT_FFT_INSTANTIATE(float, 192)
PAT_FFT_INSTANTIATE(float, 384)
PAT_FFT_INSTANTIATE(float, 768)
}  // namespace pat
